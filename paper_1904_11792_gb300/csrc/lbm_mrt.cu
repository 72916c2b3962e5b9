// Force + collision + streaming kernels with the multiple-relaxation-time
// collision (collide_math_mrt in lbm_node.cuh): the same one- and two-node
// bodies as the paper's single-relaxation-time kernels of lbm_step.cu, all
// three streaming modes, one register budget (2 blocks of 256 threads per SM;
// the moment transforms hold 19 more values per node).  The psi pass is
// shared with the SRT step.
#include "lbm_node.cuh"

namespace lbm {

namespace {

template <int P, int MODE>
__global__ void __launch_bounds__(256, 2) collide_mrt_kernel(Geom g, Phys ph, const typename Prec<P>::T* src,
                                                             typename Prec<P>::T* dst,
                                                             const typename Prec<P>::C* __restrict__ psi) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x >= g.nx || y >= g.ny || z >= g.nz) return;
  advance_salt(ph);
  collide_node<P, MODE, COLL_MRT>(g, ph, src, dst, psi, x, y, z);
}

template <int P, int MODE>
__global__ void __launch_bounds__(256, 2) collide_pair_mrt_kernel(Geom g, Phys ph,
                                                                  const typename Prec<P>::T* src,
                                                                  typename Prec<P>::T* dst,
                                                                  const typename Prec<P>::C* __restrict__ psi) {
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x0 >= g.nx || y >= g.ny || z >= g.nz) return;
  advance_salt(ph);
  collide_pair<P, MODE, COLL_MRT>(g, ph, src, dst, psi, x0, y, z);
}

template <int P>
cudaError_t mrt_dispatch(int mode, bool vec, const Geom& g, const Phys& ph, const void* src, void* dst,
                         const void* psi, dim3 block, cudaStream_t s) {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  const T* in = (const T*)src;
  T* out = (T*)dst;
  const C* ps = (const C*)psi;
  const int ux = vec ? g.nx / 2 : g.nx;
  const dim3 grid((ux + block.x - 1) / block.x, (g.ny + block.y - 1) / block.y, (g.nz + block.z - 1) / block.z);
  if (vec) {
    switch (mode) {
      case MODE_AB: collide_pair_mrt_kernel<P, MODE_AB><<<grid, block, 0, s>>>(g, ph, in, out, ps); break;
      case MODE_AA_EVEN: collide_pair_mrt_kernel<P, MODE_AA_EVEN><<<grid, block, 0, s>>>(g, ph, in, out, ps); break;
      default: collide_pair_mrt_kernel<P, MODE_AA_ODD><<<grid, block, 0, s>>>(g, ph, in, out, ps); break;
    }
  } else {
    switch (mode) {
      case MODE_AB: collide_mrt_kernel<P, MODE_AB><<<grid, block, 0, s>>>(g, ph, in, out, ps); break;
      case MODE_AA_EVEN: collide_mrt_kernel<P, MODE_AA_EVEN><<<grid, block, 0, s>>>(g, ph, in, out, ps); break;
      default: collide_mrt_kernel<P, MODE_AA_ODD><<<grid, block, 0, s>>>(g, ph, in, out, ps); break;
    }
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_collide_mrt(int precision, int mode, bool vec, const Geom& g, const Phys& ph, const void* src,
                               void* dst, const void* psi, dim3 block, cudaStream_t s) {
  if ((long long)block.x * block.y * block.z > 256) return cudaErrorInvalidConfiguration;
  vec = vec && (g.nx % 2 == 0);
  switch (precision) {
    // FP64: one node per thread (two nodes' moments in doubles spill)
    case LBM_F64: return mrt_dispatch<LBM_F64>(mode, false, g, ph, src, dst, psi, block, s);
    case LBM_F32: return mrt_dispatch<LBM_F32>(mode, vec, g, ph, src, dst, psi, block, s);
    case LBM_F16DEV: return mrt_dispatch<LBM_F16DEV>(mode, vec, g, ph, src, dst, psi, block, s);
    case LBM_BF16DEV: return mrt_dispatch<LBM_BF16DEV>(mode, vec, g, ph, src, dst, psi, block, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
