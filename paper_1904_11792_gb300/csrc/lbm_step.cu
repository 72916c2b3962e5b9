// The two kernels of one time step (hot path), single lattice: the psi pass
// and the fused force + collision + streaming kernel (bodies in lbm_node.cuh).
//
// Memory layout: structure of arrays, plane a holds f_a of all nodes, x
// fastest, so a warp's 32 threads touch 32 consecutive x of one plane per
// load or store.  Both kernels are bound by HBM bandwidth (about 1 flop per
// byte); no tensor-core work exists on this path.
#include "lbm_node.cuh"

namespace lbm {

namespace {

// psi pass over all nodes of one lattice.
template <int P, int LAYOUT>
__global__ void __launch_bounds__(256) psi_kernel(Geom g, Phys ph, const typename Prec<P>::T* f,
                                                  typename Prec<P>::C* __restrict__ psi,
                                                  int* __restrict__ flag) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  psi_node<P, LAYOUT>(g, ph, f, psi, flag, i);
}

// Fused force + collision + streaming.  One thread per node.  MINB is the
// number of 256-thread blocks per SM the register allocation must allow
// (4: <= 64 registers, 3: <= 80, 2: <= 128); the autotuner picks it.
template <int P, int MODE, int MINB>
__global__ void __launch_bounds__(256, MINB) collide_kernel(Geom g, Phys ph,
                                                            const typename Prec<P>::T* src,
                                                            typename Prec<P>::T* dst,
                                                            const typename Prec<P>::C* __restrict__ psi) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x >= g.nx || y >= g.ny || z >= g.nz) return;
  advance_salt(ph);
  collide_node<P, MODE>(g, ph, src, dst, psi, x, y, z);
}

// Two-node forms (x even, nx even): one thread per node pair.
template <int P, int LAYOUT>
__global__ void __launch_bounds__(256) psi_pair_kernel(Geom g, Phys ph, const typename Prec<P>::T* f,
                                                       typename Prec<P>::C* __restrict__ psi,
                                                       int* __restrict__ flag) {
  const long long i = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= g.N) return;
  psi_pair<P, LAYOUT>(g, ph, f, psi, flag, i);
}

template <int P>
__global__ void __launch_bounds__(256) psi_quad_kernel(Geom g, Phys ph, const typename Prec<P>::T* f,
                                                       typename Prec<P>::C* __restrict__ psi,
                                                       int* __restrict__ flag) {
  const long long i = 4 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= g.N) return;
  psi_quad<P>(g, ph, f, psi, flag, i);
}

// Gather layout, four nodes per thread; every thread of the last block takes
// part in the warp shuffles (those past the lattice on its last quad).
template <int P>
__global__ void __launch_bounds__(256) psi_quad_gather_kernel(Geom g, Phys ph, const typename Prec<P>::T* f,
                                                              typename Prec<P>::C* __restrict__ psi,
                                                              int* __restrict__ flag) {
  long long i = 4 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  const bool live = i < g.N;
  if (!live) i = g.N - 4;
  psi_quad_gather<P>(g, ph, f, psi, flag, i, live);
}

template <int P, int MODE, int MINB>
__global__ void __launch_bounds__(256, MINB) collide_pair_kernel(Geom g, Phys ph,
                                                                 const typename Prec<P>::T* src,
                                                                 typename Prec<P>::T* dst,
                                                                 const typename Prec<P>::C* __restrict__ psi) {
  const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x0 >= g.nx || y >= g.ny || z >= g.nz) return;
  advance_salt(ph);
  collide_pair<P, MODE>(g, ph, src, dst, psi, x0, y, z);
}

template <int P>
cudaError_t psi_dispatch(int layout, bool vec, const Geom& g, const Phys& ph, const void* f,
                         void* psi, int* flag, cudaStream_t s) {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  const int threads = 256;
  if constexpr (P != LBM_F64) {
    const long long blocks = (g.N / 4 + threads - 1) / threads;
    if (vec && g.nx % 4 == 0 && layout == LAYOUT_LOCAL) {
      psi_quad_kernel<P><<<(unsigned)blocks, threads, 0, s>>>(g, ph, (const T*)f, (C*)psi, flag);
      return cudaGetLastError();
    }
    // the gather layout in four-node form for 2-byte storage only (FP32:
    // 10.28 ms against 9.84 ms per AA step on 1024x512x512 with node pairs)
    if constexpr (Prec<P>::dev) {
      if (vec && g.nx % 4 == 0) {
        psi_quad_gather_kernel<P><<<(unsigned)blocks, threads, 0, s>>>(g, ph, (const T*)f, (C*)psi, flag);
        return cudaGetLastError();
      }
    }
  }
  if (vec) {
    const long long blocks = (g.N / 2 + threads - 1) / threads;
    if (layout == LAYOUT_LOCAL)
      psi_pair_kernel<P, LAYOUT_LOCAL><<<(unsigned)blocks, threads, 0, s>>>(g, ph, (const T*)f, (C*)psi, flag);
    else
      psi_pair_kernel<P, LAYOUT_GATHER><<<(unsigned)blocks, threads, 0, s>>>(g, ph, (const T*)f, (C*)psi, flag);
    return cudaGetLastError();
  }
  const long long blocks = (g.N + threads - 1) / threads;
  if (layout == LAYOUT_LOCAL)
    psi_kernel<P, LAYOUT_LOCAL><<<(unsigned)blocks, threads, 0, s>>>(g, ph, (const T*)f, (C*)psi, flag);
  else
    psi_kernel<P, LAYOUT_GATHER><<<(unsigned)blocks, threads, 0, s>>>(g, ph, (const T*)f, (C*)psi, flag);
  return cudaGetLastError();
}

template <int P, int MINB, bool VEC>
cudaError_t collide_mode(int mode, const Geom& g, const Phys& ph, const void* src, void* dst,
                         const void* psi, dim3 grid, dim3 block, cudaStream_t s) {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  const T* in = (const T*)src;
  T* out = (T*)dst;
  const C* ps = (const C*)psi;
  if constexpr (VEC) {
    switch (mode) {
      case MODE_AB: collide_pair_kernel<P, MODE_AB, MINB><<<grid, block, 0, s>>>(g, ph, in, out, ps); break;
      case MODE_AA_EVEN: collide_pair_kernel<P, MODE_AA_EVEN, MINB><<<grid, block, 0, s>>>(g, ph, in, out, ps); break;
      default: collide_pair_kernel<P, MODE_AA_ODD, MINB><<<grid, block, 0, s>>>(g, ph, in, out, ps); break;
    }
  } else {
    switch (mode) {
      case MODE_AB: collide_kernel<P, MODE_AB, MINB><<<grid, block, 0, s>>>(g, ph, in, out, ps); break;
      case MODE_AA_EVEN: collide_kernel<P, MODE_AA_EVEN, MINB><<<grid, block, 0, s>>>(g, ph, in, out, ps); break;
      default: collide_kernel<P, MODE_AA_ODD, MINB><<<grid, block, 0, s>>>(g, ph, in, out, ps); break;
    }
  }
  return cudaGetLastError();
}

template <int P>
cudaError_t collide_dispatch(int mode, int minb, bool vec, const Geom& g, const Phys& ph,
                             const void* src, void* dst, const void* psi, dim3 block,
                             cudaStream_t s) {
  const int ux = vec ? g.nx / 2 : g.nx;  // threads needed along x
  dim3 grid((ux + block.x - 1) / block.x, (g.ny + block.y - 1) / block.y,
            (g.nz + block.z - 1) / block.z);
  if (vec) {
    switch (minb) {
      case 2: return collide_mode<P, 2, true>(mode, g, ph, src, dst, psi, grid, block, s);
      case 3: return collide_mode<P, 3, true>(mode, g, ph, src, dst, psi, grid, block, s);
      default: return collide_mode<P, 4, true>(mode, g, ph, src, dst, psi, grid, block, s);
    }
  }
  switch (minb) {
    case 2: return collide_mode<P, 2, false>(mode, g, ph, src, dst, psi, grid, block, s);
    case 3: return collide_mode<P, 3, false>(mode, g, ph, src, dst, psi, grid, block, s);
    default: return collide_mode<P, 4, false>(mode, g, ph, src, dst, psi, grid, block, s);
  }
}

}  // namespace

cudaError_t launch_psi(int precision, int layout, bool vec, const Geom& g, const Phys& ph,
                       const void* f, void* psi, int* flag, cudaStream_t s) {
  vec = vec && (g.nx % 2 == 0);
  switch (precision) {
    case LBM_F64: return psi_dispatch<LBM_F64>(layout, vec, g, ph, f, psi, flag, s);
    case LBM_F32: return psi_dispatch<LBM_F32>(layout, vec, g, ph, f, psi, flag, s);
    case LBM_F16DEV: return psi_dispatch<LBM_F16DEV>(layout, vec, g, ph, f, psi, flag, s);
    case LBM_BF16DEV: return psi_dispatch<LBM_BF16DEV>(layout, vec, g, ph, f, psi, flag, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_collide(int precision, int mode, int minb, bool vec, const Geom& g,
                           const Phys& ph, const void* src, void* dst, const void* psi, dim3 block,
                           cudaStream_t s) {
  if ((long long)block.x * block.y * block.z > 256) return cudaErrorInvalidConfiguration;
  vec = vec && (g.nx % 2 == 0);
  switch (precision) {
    case LBM_F64: return collide_dispatch<LBM_F64>(mode, minb, vec, g, ph, src, dst, psi, block, s);
    case LBM_F32: return collide_dispatch<LBM_F32>(mode, minb, vec, g, ph, src, dst, psi, block, s);
    case LBM_F16DEV: return collide_dispatch<LBM_F16DEV>(mode, minb, vec, g, ph, src, dst, psi, block, s);
    case LBM_BF16DEV: return collide_dispatch<LBM_BF16DEV>(mode, minb, vec, g, ph, src, dst, psi, block, s);
  }
  return cudaErrorInvalidValue;
}

size_t elem_size(int precision) {
  switch (precision) {
    case LBM_F64: return 8;
    case LBM_F32: return 4;
    default: return 2;
  }
}

}  // namespace lbm
