// Kernels around the time step: ligament initial condition, canonical
// population export/import, macroscopic fields, FP64 diagnostics and the
// connected-component labelling of the liquid (droplet count).
#include "lbm_internal.h"

namespace lbm {

namespace {

template <int P>
__device__ __forceinline__ double shift_d(int a, double rho_ref) {
  return Prec<P>::dev ? wgt(a) * rho_ref : 0.0;
}

__device__ __forceinline__ void coords(const Geom& g, long long i, int& x, int& y, int& z) {
  x = (int)(i % g.nx);
  const long long r = i / g.nx;
  y = (int)(r % g.ny);
  z = (int)(r / g.ny);
}

// Flat index in the storage of the pre-collision population a of node
// (x, y, z) for the given layout.
__device__ __forceinline__ long long slot_index(const Geom& g, int layout, int a, const Nbr& nb) {
  if (layout == LAYOUT_LOCAL) return (long long)a * g.N + nb.idx(0, 0, 0);
  return (long long)opp(a) * g.N + nb.idx(-cx(a), -cy(a), -cz(a));
}

// rho and j of a node in compute precision C (the same summation order as
// the collide kernel).
template <int P>
__device__ __forceinline__ void node_rho_j(const Geom& g, const Phys& ph, int layout,
                                           const typename Prec<P>::T* f, const Nbr& nb,
                                           typename Prec<P>::C& rho, typename Prec<P>::C j[3]) {
  using C = typename Prec<P>::C;
  rho = 0;
  j[0] = j[1] = j[2] = 0;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const C v = Prec<P>::load(f + slot_index(g, layout, a, nb), (C)shift_d<P>(a, ph.rho_ref));
    rho += v;
    if (cx(a)) j[0] += cx(a) > 0 ? v : -v;
    if (cy(a)) j[1] += cy(a) > 0 ? v : -v;
    if (cz(a)) j[2] += cz(a) > 0 ? v : -v;
  }
}

// ---------------------------------------------------------------------------
// Initial condition (section "Ligament set-up"): perturbed cylinder along x.
// ---------------------------------------------------------------------------
template <int P>
__global__ void init_kernel(Geom g, Phys ph, InitSpec sp, typename Prec<P>::T* f) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  int x, y, z;
  coords(g, i, x, y, z);
  const double R = sp.R0 * (1.0 + sp.eps * cos(6.283185307179586476925 * x / sp.lambda + sp.phase));
  const double dy = y - 0.5 * (g.ny - 1), dz = z - 0.5 * (g.nz - 1);
  const double d = sqrt(dy * dy + dz * dz) - R;
  double rho;
  if (sp.prof == nullptr) {
    rho = sp.rho_v + 0.5 * (sp.rho_l - sp.rho_v) * (1.0 - tanh(2.0 * d / sp.width));
  } else {
    const double s = (d - sp.d0) / sp.dd;
    if (s <= 0.0) {
      rho = sp.prof[0];
    } else if (s >= sp.n - 1) {
      rho = sp.prof[sp.n - 1];
    } else {
      const int k = (int)floor(s);
      const double t = s - k;
      rho = sp.prof[k] + t * (sp.prof[k + 1] - sp.prof[k]);
    }
  }
  using C = typename Prec<P>::C;
#pragma unroll
  for (int a = 0; a < Q; ++a)
    Prec<P>::store(f + (long long)a * g.N + i, (C)(wgt(a) * rho), (C)shift_d<P>(a, ph.rho_ref));
}

// ---------------------------------------------------------------------------
// Canonical FP64 plane a <-> storage.
// ---------------------------------------------------------------------------
template <int P>
__global__ void get_plane_kernel(Geom g, Phys ph, int layout, const typename Prec<P>::T* f, int a,
                                 double* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  int x, y, z;
  coords(g, i, x, y, z);
  Nbr nb;
  nb.make(g, x, y, z);
  using C = typename Prec<P>::C;
  out[i] = (double)Prec<P>::load(f + slot_index(g, layout, a, nb), (C)shift_d<P>(a, ph.rho_ref));
}

template <int P>
__global__ void set_plane_kernel(Geom g, Phys ph, int layout, typename Prec<P>::T* f, int a,
                                 const double* in) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  int x, y, z;
  coords(g, i, x, y, z);
  Nbr nb;
  nb.make(g, x, y, z);
  using C = typename Prec<P>::C;
  Prec<P>::store(f + slot_index(g, layout, a, nb), (C)in[i], (C)shift_d<P>(a, ph.rho_ref));
}

// ---------------------------------------------------------------------------
// Macroscopic fields: rho (Eq. 4) and u = (j + F/2)/rho, F from Eq. 5.
// which: 0 rho, 1..3 the velocity components.
// ---------------------------------------------------------------------------
template <int P>
__global__ void moments_kernel(Geom g, Phys ph, int layout, const typename Prec<P>::T* f,
                               const typename Prec<P>::C* psi, double* rho_o, double* ux,
                               double* uy, double* uz) {
  using C = typename Prec<P>::C;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  int x, y, z;
  coords(g, i, x, y, z);
  Nbr nb;
  nb.make(g, x, y, z);
  C rho, j[3];
  node_rho_j<P>(g, ph, layout, f, nb, rho, j);
  C s[3] = {0, 0, 0};
#pragma unroll
  for (int a = 1; a < Q; ++a) {
    const C p = psi[nb.idx(cx(a), cy(a), cz(a))];
    const C w = (C)wgt(a);
    s[0] += w * cx(a) * p;
    s[1] += w * cy(a) * p;
    s[2] += w * cz(a) * p;
  }
  const C gp = -(C)ph.G * psi[i];
  if (rho_o) rho_o[i] = (double)rho;
  const double r = (double)rho;
  if (ux) ux[i] = ((double)j[0] + 0.5 * (double)(gp * s[0])) / r;
  if (uy) uy[i] = ((double)j[1] + 0.5 * (double)(gp * s[1])) / r;
  if (uz) uz[i] = ((double)j[2] + 0.5 * (double)(gp * s[2])) / r;
}

// ---------------------------------------------------------------------------
// Diagnostics: deterministic two-kernel FP64 reduction.
// Block (32, 8): threadIdx.x walks x, threadIdx.y and blockIdx.y walk rows
// (y, z).  Per-thread accumulation in a fixed order, then fixed-order
// block reductions; the final kernel combines block partials in index order.
// ---------------------------------------------------------------------------
constexpr int DX = 32, DY = 8;
constexpr int NG = 12;  // global partial slots per block
// slots: 0 mass, 1-3 momentum, 4 volume_w, 5 count, 6 max_u, 7 rho_min,
// 8 rho_max, 9 bad, 10-11 unused

int diag_row_blocks(const Geom& g) {
  const long long rows = (long long)g.ny * g.nz;
  long long rb = (rows + DY - 1) / DY;
  if (rb > 64) rb = 64;
  return (int)rb;
}

template <int P>
__global__ void __launch_bounds__(DX* DY) diag_partial_kernel(Geom g, Phys ph, int layout,
                                                              const typename Prec<P>::T* f,
                                                              double rho_l, double rho_v,
                                                              double* slices, double* blocks) {
  using C = typename Prec<P>::C;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = blockIdx.x * DX + tx;
  const long long rows = (long long)g.ny * g.nz;
  const double thr = 0.5 * (rho_l + rho_v), inv = 1.0 / (rho_l - rho_v);
  double acc[NG];
#pragma unroll
  for (int k = 0; k < NG; ++k) acc[k] = 0.0;
  acc[7] = 1e300;
  acc[8] = -1e300;
  double sw = 0.0, sn = 0.0;
  if (x < g.nx) {
    for (long long r = (long long)blockIdx.y * DY + ty; r < rows; r += (long long)DY * gridDim.y) {
      const int y = (int)(r % g.ny), z = (int)(r / g.ny);
      Nbr nb;
      nb.make(g, x, y, z);
      C rho_c, j[3];
      node_rho_j<P>(g, ph, layout, f, nb, rho_c, j);
      const double rho = (double)rho_c;
      acc[0] += rho;
      acc[1] += (double)j[0];
      acc[2] += (double)j[1];
      acc[3] += (double)j[2];
      double phi = (rho - rho_v) * inv;
      phi = phi < 0.0 ? 0.0 : (phi > 1.0 ? 1.0 : phi);
      acc[4] += phi;
      sw += phi;
      if (rho > thr) {
        acc[5] += 1.0;
        sn += 1.0;
      }
      const double u = sqrt((double)j[0] * j[0] + (double)j[1] * j[1] + (double)j[2] * j[2]) / rho;
      if (u > acc[6]) acc[6] = u;
      if (rho < acc[7]) acc[7] = rho;
      if (rho > acc[8]) acc[8] = rho;
      if (!(rho > 0.0) || !(rho <= 1e300)) acc[9] = 1.0;
    }
  }
  __shared__ double sh_s[2][DY][DX];
  __shared__ double sh_g[NG][DY * DX];
  sh_s[0][ty][tx] = sw;
  sh_s[1][ty][tx] = sn;
  const int t = ty * DX + tx;
#pragma unroll
  for (int k = 0; k < NG; ++k) sh_g[k][t] = acc[k];
  __syncthreads();
  if (ty == 0 && x < g.nx) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < DY; ++k) {
      a += sh_s[0][k][tx];
      b += sh_s[1][k][tx];
    }
    slices[((long long)blockIdx.y * g.nx + x) * 2 + 0] = a;
    slices[((long long)blockIdx.y * g.nx + x) * 2 + 1] = b;
  }
  for (int s = DX * DY / 2; s > 0; s >>= 1) {
    if (t < s) {
#pragma unroll
      for (int k = 0; k < 6; ++k) sh_g[k][t] += sh_g[k][t + s];
      sh_g[6][t] = fmax(sh_g[6][t], sh_g[6][t + s]);
      sh_g[7][t] = fmin(sh_g[7][t], sh_g[7][t + s]);
      sh_g[8][t] = fmax(sh_g[8][t], sh_g[8][t + s]);
      sh_g[9][t] = fmax(sh_g[9][t], sh_g[9][t + s]);
    }
    __syncthreads();
  }
  if (t == 0) {
    const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
#pragma unroll
    for (int k = 0; k < NG; ++k) blocks[b * NG + k] = sh_g[k][0];
  }
}

constexpr int FT = 256;

__global__ void __launch_bounds__(FT) diag_final_kernel(Geom g, int nblocks, int row_blocks,
                                                       const double* slices, const double* blocks,
                                                       double* out) {
  __shared__ double sg[NG][FT];
  __shared__ double smin_w[FT], smin_n[FT];
  __shared__ int smin_x[FT];
  const int t = threadIdx.x;
  double acc[NG];
#pragma unroll
  for (int k = 0; k < NG; ++k) acc[k] = 0.0;
  acc[7] = 1e300;
  acc[8] = -1e300;
  for (int b = t; b < nblocks; b += FT) {
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] += blocks[(long long)b * NG + k];
    acc[6] = fmax(acc[6], blocks[(long long)b * NG + 6]);
    acc[7] = fmin(acc[7], blocks[(long long)b * NG + 7]);
    acc[8] = fmax(acc[8], blocks[(long long)b * NG + 8]);
    acc[9] = fmax(acc[9], blocks[(long long)b * NG + 9]);
  }
  // per-slice totals and their minima (first x on ties)
  double mw = 1e300, mn = 1e300;
  int mx = 0x7fffffff;
  for (int x = t; x < g.nx; x += FT) {
    double a = 0.0, c = 0.0;
    for (int rb = 0; rb < row_blocks; ++rb) {
      a += slices[((long long)rb * g.nx + x) * 2 + 0];
      c += slices[((long long)rb * g.nx + x) * 2 + 1];
    }
    if (a < mw) mw = a;
    if (c < mn) {
      mn = c;
      mx = x;
    }
  }
#pragma unroll
  for (int k = 0; k < NG; ++k) sg[k][t] = acc[k];
  smin_w[t] = mw;
  smin_n[t] = mn;
  smin_x[t] = mx;
  __syncthreads();
  for (int s = FT / 2; s > 0; s >>= 1) {
    if (t < s) {
#pragma unroll
      for (int k = 0; k < 6; ++k) sg[k][t] += sg[k][t + s];
      sg[6][t] = fmax(sg[6][t], sg[6][t + s]);
      sg[7][t] = fmin(sg[7][t], sg[7][t + s]);
      sg[8][t] = fmax(sg[8][t], sg[8][t + s]);
      sg[9][t] = fmax(sg[9][t], sg[9][t + s]);
      smin_w[t] = fmin(smin_w[t], smin_w[t + s]);
      const double on = smin_n[t + s];
      const int ox = smin_x[t + s];
      if (on < smin_n[t] || (on == smin_n[t] && ox < smin_x[t])) {
        smin_n[t] = on;
        smin_x[t] = ox;
      }
    }
    __syncthreads();
  }
  if (t == 0) {
    out[0] = sg[0][0];
    out[1] = sg[1][0];
    out[2] = sg[2][0];
    out[3] = sg[3][0];
    out[4] = sg[4][0];
    out[5] = sg[5][0];
    out[6] = smin_w[0];
    out[7] = smin_n[0];
    out[8] = (double)smin_x[0];
    out[9] = sg[6][0];
    out[10] = sg[7][0];
    out[11] = sg[8][0];
    out[12] = sg[9][0] > 0.0 ? 0.0 : 1.0;
  }
}

// ---------------------------------------------------------------------------
// Connected components of the liquid (rho > threshold), 6-connectivity,
// periodic: lock-free union-find on int labels.  Every label points to a
// node of smaller or equal index, so each root search and each union retry
// strictly decreases an index and ends within N iterations.  As a guard the
// loops still stop after kMaxHops steps and raise an error flag (out[3]).
// ---------------------------------------------------------------------------
constexpr long long kMaxHops = 1ll << 31;

__device__ __forceinline__ int find_root(const int* L, int i, long long& hops) {
  int p = L[i];
  while (p != i && hops < kMaxHops) {
    i = p;
    p = L[i];
    ++hops;
  }
  return i;
}

__device__ __forceinline__ void unite(int* L, int a, int b, unsigned long long* err) {
  long long hops = 0;
  while (hops < kMaxHops) {
    a = find_root(L, a, hops);
    b = find_root(L, b, hops);
    if (a == b) return;
    ++hops;
    if (a < b) {
      const int old = atomicMin(&L[b], a);
      if (old == b) return;
      b = old;
    } else {
      const int old = atomicMin(&L[a], b);
      if (old == a) return;
      a = old;
    }
  }
  atomicOr(err, 1ull);
}

template <int P>
__global__ void ccl_init_kernel(Geom g, Phys ph, int layout, const typename Prec<P>::T* f,
                                double thr, int* L, int* sizes) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  int x, y, z;
  coords(g, i, x, y, z);
  Nbr nb;
  nb.make(g, x, y, z);
  typename Prec<P>::C rho, j[3];
  node_rho_j<P>(g, ph, layout, f, nb, rho, j);
  L[i] = ((double)rho > thr) ? (int)i : -1;
  sizes[i] = 0;
}

__global__ void ccl_union_kernel(Geom g, int* L, unsigned long long* err) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N || L[i] < 0) return;
  int x, y, z;
  coords(g, i, x, y, z);
  Nbr nb;
  nb.make(g, x, y, z);
  const long long n[3] = {nb.idx(1, 0, 0), nb.idx(0, 1, 0), nb.idx(0, 0, 1)};
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (L[n[k]] >= 0) unite(L, (int)i, (int)n[k], err);
}

__global__ void ccl_compress_kernel(Geom g, int* L, int* sizes, unsigned long long* err) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N || L[i] < 0) return;
  long long hops = 0;
  const int r = find_root(L, (int)i, hops);
  if (hops >= kMaxHops) atomicOr(err, 1ull);
  atomicAdd(&sizes[r], 1);
}

__global__ void ccl_count_kernel(Geom g, const int* L, const int* sizes, unsigned long long* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N || L[i] != (int)i) return;
  atomicAdd(&out[0], 1ull);
  if (sizes[i] >= 8) atomicAdd(&out[1], 1ull);
  atomicMax(&out[2], (unsigned long long)sizes[i]);
}

inline unsigned blocks_for(long long n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <int P>
cudaError_t init_t(const Geom& g, const Phys& ph, const InitSpec& sp, void* f, cudaStream_t s) {
  init_kernel<P><<<blocks_for(g.N, 256), 256, 0, s>>>(g, ph, sp, (typename Prec<P>::T*)f);
  return cudaGetLastError();
}
template <int P>
cudaError_t get_t(int layout, const Geom& g, const Phys& ph, const void* f, int a, double* out,
                  cudaStream_t s) {
  get_plane_kernel<P><<<blocks_for(g.N, 256), 256, 0, s>>>(g, ph, layout,
                                                           (const typename Prec<P>::T*)f, a, out);
  return cudaGetLastError();
}
template <int P>
cudaError_t set_t(int layout, const Geom& g, const Phys& ph, void* f, int a, const double* in,
                  cudaStream_t s) {
  set_plane_kernel<P><<<blocks_for(g.N, 256), 256, 0, s>>>(g, ph, layout,
                                                           (typename Prec<P>::T*)f, a, in);
  return cudaGetLastError();
}
template <int P>
cudaError_t moments_t(int layout, const Geom& g, const Phys& ph, const void* f, const void* psi,
                      double* r, double* ux, double* uy, double* uz, cudaStream_t s) {
  moments_kernel<P><<<blocks_for(g.N, 256), 256, 0, s>>>(
      g, ph, layout, (const typename Prec<P>::T*)f, (const typename Prec<P>::C*)psi, r, ux, uy, uz);
  return cudaGetLastError();
}
template <int P>
cudaError_t diag_t(int layout, const Geom& g, const Phys& ph, const void* f, double rho_l,
                   double rho_v, double* scratch, double* out, cudaStream_t s) {
  const int rb = diag_row_blocks(g);
  const int gx = (g.nx + DX - 1) / DX;
  double* slices = scratch;
  double* blocks = scratch + (size_t)rb * g.nx * 2;
  diag_partial_kernel<P><<<dim3(gx, rb), dim3(DX, DY), 0, s>>>(
      g, ph, layout, (const typename Prec<P>::T*)f, rho_l, rho_v, slices, blocks);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<1, FT, 0, s>>>(g, gx * rb, rb, slices, blocks, out);
  return cudaGetLastError();
}
template <int P>
cudaError_t ccl_t(int layout, const Geom& g, const Phys& ph, const void* f, double thr, int* L,
                  int* sizes, long long* out3, cudaStream_t s) {
  const unsigned nb = blocks_for(g.N, 256);
  cudaError_t e = cudaMemsetAsync(out3, 0, 4 * sizeof(long long), s);
  if (e != cudaSuccess) return e;
  unsigned long long* err = (unsigned long long*)out3 + 3;
  ccl_init_kernel<P><<<nb, 256, 0, s>>>(g, ph, layout, (const typename Prec<P>::T*)f, thr, L, sizes);
  ccl_union_kernel<<<nb, 256, 0, s>>>(g, L, err);
  ccl_compress_kernel<<<nb, 256, 0, s>>>(g, L, sizes, err);
  ccl_count_kernel<<<nb, 256, 0, s>>>(g, L, sizes, (unsigned long long*)out3);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_init(int precision, const Geom& g, const Phys& ph, const InitSpec& spec, void* f,
                        cudaStream_t s) {
  switch (precision) {
    case LBM_F64: return init_t<LBM_F64>(g, ph, spec, f, s);
    case LBM_F32: return init_t<LBM_F32>(g, ph, spec, f, s);
    case LBM_F16DEV: return init_t<LBM_F16DEV>(g, ph, spec, f, s);
    case LBM_BF16DEV: return init_t<LBM_BF16DEV>(g, ph, spec, f, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_get_plane(int precision, int layout, const Geom& g, const Phys& ph, const void* f,
                             int a, double* out, cudaStream_t s) {
  switch (precision) {
    case LBM_F64: return get_t<LBM_F64>(layout, g, ph, f, a, out, s);
    case LBM_F32: return get_t<LBM_F32>(layout, g, ph, f, a, out, s);
    case LBM_F16DEV: return get_t<LBM_F16DEV>(layout, g, ph, f, a, out, s);
    case LBM_BF16DEV: return get_t<LBM_BF16DEV>(layout, g, ph, f, a, out, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_set_plane(int precision, int layout, const Geom& g, const Phys& ph, void* f, int a,
                             const double* in, cudaStream_t s) {
  switch (precision) {
    case LBM_F64: return set_t<LBM_F64>(layout, g, ph, f, a, in, s);
    case LBM_F32: return set_t<LBM_F32>(layout, g, ph, f, a, in, s);
    case LBM_F16DEV: return set_t<LBM_F16DEV>(layout, g, ph, f, a, in, s);
    case LBM_BF16DEV: return set_t<LBM_BF16DEV>(layout, g, ph, f, a, in, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_moments(int precision, int layout, const Geom& g, const Phys& ph, const void* f,
                           const void* psi, double* rho, double* ux, double* uy, double* uz,
                           cudaStream_t s) {
  switch (precision) {
    case LBM_F64: return moments_t<LBM_F64>(layout, g, ph, f, psi, rho, ux, uy, uz, s);
    case LBM_F32: return moments_t<LBM_F32>(layout, g, ph, f, psi, rho, ux, uy, uz, s);
    case LBM_F16DEV: return moments_t<LBM_F16DEV>(layout, g, ph, f, psi, rho, ux, uy, uz, s);
    case LBM_BF16DEV: return moments_t<LBM_BF16DEV>(layout, g, ph, f, psi, rho, ux, uy, uz, s);
  }
  return cudaErrorInvalidValue;
}

size_t diag_scratch_doubles(const Geom& g) {
  const int rb = diag_row_blocks(g);
  const int gx = (g.nx + DX - 1) / DX;
  return (size_t)rb * g.nx * 2 + (size_t)gx * rb * NG;
}

cudaError_t launch_diagnostics(int precision, int layout, const Geom& g, const Phys& ph, const void* f,
                               double rho_l, double rho_v, double* scratch, double* out,
                               cudaStream_t s) {
  switch (precision) {
    case LBM_F64: return diag_t<LBM_F64>(layout, g, ph, f, rho_l, rho_v, scratch, out, s);
    case LBM_F32: return diag_t<LBM_F32>(layout, g, ph, f, rho_l, rho_v, scratch, out, s);
    case LBM_F16DEV: return diag_t<LBM_F16DEV>(layout, g, ph, f, rho_l, rho_v, scratch, out, s);
    case LBM_BF16DEV: return diag_t<LBM_BF16DEV>(layout, g, ph, f, rho_l, rho_v, scratch, out, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_ccl(int precision, int layout, const Geom& g, const Phys& ph, const void* f,
                       double threshold, int* labels, int* sizes, long long* out3, cudaStream_t s) {
  switch (precision) {
    case LBM_F64: return ccl_t<LBM_F64>(layout, g, ph, f, threshold, labels, sizes, out3, s);
    case LBM_F32: return ccl_t<LBM_F32>(layout, g, ph, f, threshold, labels, sizes, out3, s);
    case LBM_F16DEV: return ccl_t<LBM_F16DEV>(layout, g, ph, f, threshold, labels, sizes, out3, s);
    case LBM_BF16DEV: return ccl_t<LBM_BF16DEV>(layout, g, ph, f, threshold, labels, sizes, out3, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
