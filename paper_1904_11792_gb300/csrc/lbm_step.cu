// The two kernels of one time step (hot path):
//   psi_kernel      rho = sum_a f_a (Eq. 4) and psi(rho) for every node; the
//                   force of Eq. 5 needs psi of all 18 neighbours at the same
//                   time level, so psi exists for the whole lattice before any
//                   collision starts.
//   collide_kernel  per node: moments (Eq. 4), Shan-Chen force from the
//                   neighbour psi (Eq. 5), velocity shift u' = (j + tau F)/rho
//                   (Eq. 6), second-order equilibrium (Eq. 2, with the leading
//                   1), BGK relaxation (Eq. 3) and streaming to x + c_a.
//
// Memory layout: structure of arrays, plane a holds f_a of all nodes, x
// fastest, so a warp's 32 threads touch 32 consecutive x of one plane per
// load or store.  Both kernels are bound by HBM bandwidth (about 1 flop per
// byte); no tensor-core work exists on this path.
#include "lbm_internal.h"

namespace lbm {

namespace {

template <int P>
__device__ __forceinline__ typename Prec<P>::C shift_of(int a, double rho_ref) {
  using C = typename Prec<P>::C;
  if constexpr (Prec<P>::dev) {
    return (C)(wgt(a) * rho_ref);
  } else {
    return (C)0;
  }
}

// psi pass.  LAYOUT_LOCAL reads slot a at x; LAYOUT_GATHER (AA before an
// odd step) reads slot opp(a) at x - c_a.
template <int P, int LAYOUT>
__global__ void __launch_bounds__(256) psi_kernel(Geom g, Phys ph, const typename Prec<P>::T* f,
                                                  typename Prec<P>::C* __restrict__ psi,
                                                  int* __restrict__ flag) {
  using C = typename Prec<P>::C;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  const C s0 = shift_of<P>(0, ph.rho_ref), s1 = shift_of<P>(1, ph.rho_ref),
          s2 = shift_of<P>(7, ph.rho_ref);
  C rho = 0;
  if constexpr (LAYOUT == LAYOUT_LOCAL) {
#pragma unroll
    for (int a = 0; a < Q; ++a)
      rho += Prec<P>::load(f + (long long)a * g.N + i, a == 0 ? s0 : (a <= 6 ? s1 : s2));
  } else {
    const int x = (int)(i % g.nx);
    const long long r = i / g.nx;
    const int y = (int)(r % g.ny), z = (int)(r / g.ny);
    Nbr nb;
    nb.make(g, x, y, z);
#pragma unroll
    for (int a = 0; a < Q; ++a)
      rho += Prec<P>::load(f + (long long)opp(a) * g.N + nb.idx(-cx(a), -cy(a), -cz(a)),
                           a == 0 ? s0 : (a <= 6 ? s1 : s2));
  }
  psi[i] = psi_of<C>(rho, ph.psi_form, (C)ph.rho0);
  // non-positive, NaN or infinite density
  if (!(rho > (C)0) || !(rho <= (C)3.0e38)) atomicOr(flag, 1);
}

// Fused force + collision + streaming.  One thread per node.
template <int P, int MODE>
__global__ void __launch_bounds__(512) collide_kernel(Geom g, Phys ph,
                                                      const typename Prec<P>::T* src,
                                                      typename Prec<P>::T* dst,
                                                      const typename Prec<P>::C* __restrict__ psi) {
  using C = typename Prec<P>::C;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z * blockDim.z + threadIdx.z;
  if (x >= g.nx || y >= g.ny || z >= g.nz) return;
  Nbr nb;
  nb.make(g, x, y, z);
  const long long i = nb.idx(0, 0, 0);
  const long long N = g.N;
  const C s0 = shift_of<P>(0, ph.rho_ref), s1 = shift_of<P>(1, ph.rho_ref),
          s2 = shift_of<P>(7, ph.rho_ref);

  // pre-collision populations of this node
  C f[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const C sh = a == 0 ? s0 : (a <= 6 ? s1 : s2);
    if constexpr (MODE == MODE_AB)
      f[a] = Prec<P>::load(src + (long long)a * N + i, sh);
    else if constexpr (MODE == MODE_AA_EVEN)
      f[a] = Prec<P>::load_rw(src + (long long)a * N + i, sh);
    else
      f[a] = Prec<P>::load_rw(src + (long long)opp(a) * N + nb.idx(-cx(a), -cy(a), -cz(a)), sh);
  }

  // Eq. 4
  C rho = 0, jx = 0, jy = 0, jz = 0;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    rho += f[a];
    if (cx(a) > 0) jx += f[a];
    if (cx(a) < 0) jx -= f[a];
    if (cy(a) > 0) jy += f[a];
    if (cy(a) < 0) jy -= f[a];
    if (cz(a) > 0) jz += f[a];
    if (cz(a) < 0) jz -= f[a];
  }

  // Eq. 5: sum_a w_a psi(x + c_a) c_a, split by weight class
  C ax = 0, ay = 0, az = 0, dx = 0, dy = 0, dz = 0;
#pragma unroll
  for (int a = 1; a < Q; ++a) {
    const C p = __ldg(psi + nb.idx(cx(a), cy(a), cz(a)));
    if (a <= 6) {
      ax += cx(a) * p;
      ay += cy(a) * p;
      az += cz(a) * p;
    } else {
      dx += cx(a) * p;
      dy += cy(a) * p;
      dz += cz(a) * p;
    }
  }
  const C w1 = (C)(1.0 / 18.0), w2 = (C)(1.0 / 36.0);
  const C gp = -(C)ph.G * __ldg(psi + i);
  const C Fx = gp * (w1 * ax + w2 * dx);
  const C Fy = gp * (w1 * ay + w2 * dy);
  const C Fz = gp * (w1 * az + w2 * dz);

  // Eq. 6
  const C tau = (C)ph.tau;
  const C inv_rho = (C)1 / rho;
  const C ux = (jx + tau * Fx) * inv_rho;
  const C uy = (jy + tau * Fy) * inv_rho;
  const C uz = (jz + tau * Fz) * inv_rho;
  const C usq = (C)1.5 * (ux * ux + uy * uy + uz * uz);
  const C omega = (C)1 / tau;

  // Eq. 2 and Eq. 3, then streaming
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const C cu = cx(a) * ux + cy(a) * uy + cz(a) * uz;
    const C wr = (C)wgt(a) * rho;
    const C feq = wr * ((C)1 + (C)3 * cu + (C)4.5 * cu * cu - usq);
    const C fs = f[a] - omega * (f[a] - feq);
    const C sh = a == 0 ? s0 : (a <= 6 ? s1 : s2);
    long long d;
    if constexpr (MODE == MODE_AB)
      d = (long long)a * N + nb.idx(cx(a), cy(a), cz(a));
    else if constexpr (MODE == MODE_AA_EVEN)
      d = (long long)opp(a) * N + i;
    else
      d = (long long)a * N + nb.idx(cx(a), cy(a), cz(a));
    Prec<P>::store(dst + d, fs, sh);
  }
}

template <int P>
cudaError_t psi_dispatch(int layout, const Geom& g, const Phys& ph, const void* f, void* psi,
                         int* flag, cudaStream_t s) {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  const int threads = 256;
  const long long blocks = (g.N + threads - 1) / threads;
  if (layout == LAYOUT_LOCAL)
    psi_kernel<P, LAYOUT_LOCAL><<<(unsigned)blocks, threads, 0, s>>>(g, ph, (const T*)f, (C*)psi, flag);
  else
    psi_kernel<P, LAYOUT_GATHER><<<(unsigned)blocks, threads, 0, s>>>(g, ph, (const T*)f, (C*)psi, flag);
  return cudaGetLastError();
}

template <int P>
cudaError_t collide_dispatch(int mode, const Geom& g, const Phys& ph, const void* src, void* dst,
                             const void* psi, dim3 block, cudaStream_t s) {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  dim3 grid((g.nx + block.x - 1) / block.x, (g.ny + block.y - 1) / block.y,
            (g.nz + block.z - 1) / block.z);
  switch (mode) {
    case MODE_AB:
      collide_kernel<P, MODE_AB><<<grid, block, 0, s>>>(g, ph, (const T*)src, (T*)dst, (const C*)psi);
      break;
    case MODE_AA_EVEN:
      collide_kernel<P, MODE_AA_EVEN><<<grid, block, 0, s>>>(g, ph, (const T*)src, (T*)dst, (const C*)psi);
      break;
    default:
      collide_kernel<P, MODE_AA_ODD><<<grid, block, 0, s>>>(g, ph, (const T*)src, (T*)dst, (const C*)psi);
      break;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_psi(int precision, int layout, const Geom& g, const Phys& ph, const void* f,
                       void* psi, int* flag, cudaStream_t s) {
  switch (precision) {
    case LBM_F64: return psi_dispatch<LBM_F64>(layout, g, ph, f, psi, flag, s);
    case LBM_F32: return psi_dispatch<LBM_F32>(layout, g, ph, f, psi, flag, s);
    case LBM_F16DEV: return psi_dispatch<LBM_F16DEV>(layout, g, ph, f, psi, flag, s);
    case LBM_BF16DEV: return psi_dispatch<LBM_BF16DEV>(layout, g, ph, f, psi, flag, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_collide(int precision, int mode, const Geom& g, const Phys& ph, const void* src,
                           void* dst, const void* psi, dim3 block, cudaStream_t s) {
  switch (precision) {
    case LBM_F64: return collide_dispatch<LBM_F64>(mode, g, ph, src, dst, psi, block, s);
    case LBM_F32: return collide_dispatch<LBM_F32>(mode, g, ph, src, dst, psi, block, s);
    case LBM_F16DEV: return collide_dispatch<LBM_F16DEV>(mode, g, ph, src, dst, psi, block, s);
    case LBM_BF16DEV: return collide_dispatch<LBM_BF16DEV>(mode, g, ph, src, dst, psi, block, s);
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
