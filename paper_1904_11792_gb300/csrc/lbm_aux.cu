// Kernels around the time step: ligament initial condition, canonical
// population export/import, macroscopic fields, FP64 diagnostics and the
// connected-component labelling of the liquid (droplet count).
#include "lbm_internal.h"

namespace lbm {

namespace {

template <int P>
__device__ __forceinline__ double shift_d(int a, double rho_ref) {
  return Prec<P>::dev ? (double)storage_shift<P>(a, rho_ref) : 0.0;
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
  C v[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) v[a] = Prec<P>::load(f + slot_index(g, layout, a, nb), (C)shift_d<P>(a, ph.rho_ref));
  rho = rho_of<C>(v);
  mom_of<C>(v, j[0], j[1], j[2]);
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
// With WRITE_PSI the partial kernel is also the psi pass of the step: it
// writes psi(rho) of every node and raises the numeric flag, so diagnostics
// on a time step cost no extra pass over the populations.
// ---------------------------------------------------------------------------
constexpr int DX = 32, DY = 8;
constexpr int NG = DIAG_NG;  // global partial slots per block
// slots: 0 mass, 1-3 momentum, 4 volume_w, 5 count, 6 max_u, 7 rho_min,
// 8 rho_max, 9 bad, 10-11 unused

// Row-blocks of the partial kernel: enough blocks to fill the GPU (about 16
// per SM) while the per-slice partials (row-blocks x nx x 2 doubles) stay
// small; each thread then walks rows / (8 row-blocks) rows.
int diag_row_blocks(const Geom& g) {
  const long long rows = (long long)g.ny * g.nz;
  const long long gx = (g.nx + DX - 1) / DX;
  long long want = (16 * 152 + gx - 1) / gx;
  const long long cap = (2ll << 20) / (2ll * g.nx);  // slices <= 2 Mi doubles
  if (want > cap) want = cap;
  long long rb = (rows + DY - 1) / DY;
  if (rb > want) rb = want;
  if (rb < 1) rb = 1;
  return (int)rb;
}

// Each node's momentum and liquid fraction are computed in the compute
// precision (FP32 except in FP64 mode), its density as that sum plus its
// rounding error (rho_of_x); the per-thread sums over the thread's rows are
// DSum accumulators (an error-free FP32 pair, exact to FP64 level), the warp
// shuffle tree and the block sums of mass, momentum and the weighted liquid
// volume are FP64, so the totals carry no reduction error above FP64
// rounding, whatever the storage precision.  Counts, extrema and the
// numeric flag are exact in any precision.
template <int P, bool WRITE_PSI, int LAYOUT>
__global__ void __launch_bounds__(DX* DY, 2) diag_partial_kernel(Geom g, Phys ph,
                                                              const typename Prec<P>::T* f,
                                                              double rho_l, double rho_v,
                                                              double* slices, double* blocks,
                                                              typename Prec<P>::C* psi, int* flag) {
  using C = typename Prec<P>::C;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = blockIdx.x * DX + tx;
  const long long rows = (long long)g.ny * g.nz;
  const C thr = (C)(0.5 * (rho_l + rho_v)), inv = (C)(1.0 / (rho_l - rho_v)), rv = (C)rho_v;
  DSum<C> s_mass, s_jx, s_jy, s_jz, s_vol;
  C umax = 0, rmin = (C)3.0e38, rmax = (C)-3.0e38;
  int cnt = 0;
  bool bad = false;
  const C s0 = (C)shift_d<P>(0, ph.rho_ref);
  const C s1 = (C)shift_d<P>(1, ph.rho_ref);
  const C s2 = (C)shift_d<P>(7, ph.rho_ref);
  if (x < g.nx) {
#pragma unroll 2
    for (long long r = (long long)blockIdx.y * DY + ty; r < rows; r += (long long)DY * gridDim.y) {
      const int i = x + g.nx * (int)r;
      C fv[Q];
      if constexpr (LAYOUT == LAYOUT_LOCAL) {
#pragma unroll
        for (int a = 0; a < Q; ++a)
          fv[a] = Prec<P>::load(f + (long long)a * g.N + i, a == 0 ? s0 : (a <= 6 ? s1 : s2));
      } else {
        Nbr nb;
        nb.make(g, x, (int)(r % g.ny), (int)(r / g.ny));
#pragma unroll
        for (int a = 0; a < Q; ++a)
          fv[a] = Prec<P>::load(f + (long long)opp(a) * g.N + nb.idx(-cx(a), -cy(a), -cz(a)),
                                a == 0 ? s0 : (a <= 6 ? s1 : s2));
      }
      C rho_lo;
      const C rho = rho_of_x(fv, rho_lo);   // rho_of bitwise, plus its rounding error
      C jx, jy, jz;
      mom_of<C>(fv, jx, jy, jz);
      if constexpr (WRITE_PSI) psi[i] = psi_of<C>(rho, ph);
      s_mass.add(rho, rho_lo);
      s_jx.add(jx);
      s_jy.add(jy);
      s_jz.add(jz);
      C phi = (rho - rv) * inv;
      phi = phi < (C)0 ? (C)0 : (phi > (C)1 ? (C)1 : phi);
      s_vol.add(phi);
      cnt += rho > thr;
      const C u = sqrt(xfma(jz, jz, xfma(jy, jy, xmul(jx, jx)))) / rho;
      umax = u > umax ? u : umax;
      rmin = rho < rmin ? rho : rmin;
      rmax = rho > rmax ? rho : rmax;
      bad |= !(rho > (C)0) || !(rho <= (C)3.0e38);
    }
  }
  if constexpr (WRITE_PSI) raise_flag(bad, flag);
  // per-slice sums over the block's 8 row groups (FP64, fixed order)
  __shared__ double sh_s[2][DY][DX];
  sh_s[0][ty][tx] = s_vol.value();
  sh_s[1][ty][tx] = (double)cnt;
  // block totals: a fixed FP64 shuffle tree within each warp, then the 8
  // warp results in FP64 in warp order
  double v[5] = {s_mass.value(), s_jx.value(), s_jy.value(), s_jz.value(), s_vol.value()};
  float c_f = (float)cnt;  // exact below 2^24 nodes per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    c_f += __shfl_down_sync(0xffffffffu, c_f, o);
    const C um = __shfl_down_sync(0xffffffffu, umax, o);
    const C mn = __shfl_down_sync(0xffffffffu, rmin, o);
    const C mx = __shfl_down_sync(0xffffffffu, rmax, o);
    umax = um > umax ? um : umax;
    rmin = mn < rmin ? mn : rmin;
    rmax = mx > rmax ? mx : rmax;
  }
  const int anybad = __any_sync(0xffffffffu, bad);
  __shared__ double sh_w[NG][DY];
  if (tx == 0) {
    sh_w[0][ty] = v[0];
    sh_w[1][ty] = v[1];
    sh_w[2][ty] = v[2];
    sh_w[3][ty] = v[3];
    sh_w[4][ty] = v[4];
    sh_w[5][ty] = (double)c_f;
    sh_w[6][ty] = (double)umax;
    sh_w[7][ty] = (double)rmin;
    sh_w[8][ty] = (double)rmax;
    sh_w[9][ty] = anybad ? 1.0 : 0.0;
  }
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
  if (ty == 0 && tx < NG) {
    double r;
    if (tx < 6) {
      r = 0.0;
      for (int k = 0; k < DY; ++k) r += sh_w[tx][k];
    } else if (tx == 7) {
      r = 1e300;
      for (int k = 0; k < DY; ++k) r = fmin(r, sh_w[tx][k]);
    } else if (tx < 10) {
      r = -1e300;
      for (int k = 0; k < DY; ++k) r = fmax(r, sh_w[tx][k]);
    } else {
      r = 0.0;
    }
    blocks[((long long)blockIdx.y * gridDim.x + blockIdx.x) * NG + tx] = r;
  }
}

constexpr int FT = 256;

// Per-slice totals: one warp per slice x; lane l sums row-blocks l, l + 32,
// ... with four independent accumulators (loads in flight), then a fixed
// shuffle tree.  tot[2x] = liquid area A_w(x), tot[2x + 1] = liquid nodes.
__global__ void __launch_bounds__(256) diag_slices_kernel(Geom g, int row_blocks,
                                                         const double* __restrict__ slices,
                                                         double* __restrict__ tot) {
  const int lane = threadIdx.x & 31;
  const int x = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (x >= g.nx) return;
  double a[4] = {0.0, 0.0, 0.0, 0.0}, c[4] = {0.0, 0.0, 0.0, 0.0};
  int rb = lane;
  for (; rb + 96 < row_blocks; rb += 128) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k] += slices[((long long)(rb + 32 * k) * g.nx + x) * 2 + 0];
      c[k] += slices[((long long)(rb + 32 * k) * g.nx + x) * 2 + 1];
    }
  }
  for (; rb < row_blocks; rb += 32) {
    a[0] += slices[((long long)rb * g.nx + x) * 2 + 0];
    c[0] += slices[((long long)rb * g.nx + x) * 2 + 1];
  }
  double sa = (a[0] + a[1]) + (a[2] + a[3]), sc = (c[0] + c[1]) + (c[2] + c[3]);
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_down_sync(0xffffffffu, sa, o);
    sc += __shfl_down_sync(0xffffffffu, sc, o);
  }
  if (lane == 0) {
    tot[2 * x] = sa;
    tot[2 * x + 1] = sc;
  }
}

// Writes the DIAG_OUT results to out, or, with a ring counter, to record
// slot (counter++ mod ring_cap) of the ring at out (DIAG_STRIDE doubles per
// record).
// First stage for many block partials (the fused step writes one per block):
// block j folds the records [j chunk, (j + 1) chunk) into record j chunk, in
// a fixed order, so the final kernel reads nblocks / chunk records.
__global__ void __launch_bounds__(FT) diag_blocks_kernel(int nblocks, int chunk, double* blocks) {
  __shared__ double sg[NG][FT];
  const int t = threadIdx.x;
  const long long b0 = (long long)blockIdx.x * chunk;
  const long long b1 = min((long long)nblocks, b0 + chunk);
  double acc[NG];
#pragma unroll
  for (int k = 0; k < NG; ++k) acc[k] = 0.0;
  acc[7] = 1e300;
  acc[8] = -1e300;
  for (long long b = b0 + t; b < b1; b += FT) {
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] += blocks[b * NG + k];
    acc[6] = fmax(acc[6], blocks[b * NG + 6]);
    acc[7] = fmin(acc[7], blocks[b * NG + 7]);
    acc[8] = fmax(acc[8], blocks[b * NG + 8]);
    acc[9] = fmax(acc[9], blocks[b * NG + 9]);
  }
#pragma unroll
  for (int k = 0; k < NG; ++k) sg[k][t] = acc[k];
  __syncthreads();
  for (int s = FT / 2; s > 0; s >>= 1) {
    if (t < s) {
#pragma unroll
      for (int k = 0; k < 6; ++k) sg[k][t] += sg[k][t + s];
      sg[6][t] = fmax(sg[6][t], sg[6][t + s]);
      sg[7][t] = fmin(sg[7][t], sg[7][t + s]);
      sg[8][t] = fmax(sg[8][t], sg[8][t + s]);
      sg[9][t] = fmax(sg[9][t], sg[9][t + s]);
    }
    __syncthreads();
  }
  if (t < NG) blocks[b0 * NG + t] = t < 10 ? sg[t][0] : 0.0;
}

// Final reduction: the nblocks block records, stride records apart, and the
// slice totals.
__global__ void __launch_bounds__(FT) diag_final_kernel(Geom g, int nblocks, int stride,
                                                       const double* slice_tot, const double* blocks,
                                                       double* out, unsigned long long* ring_count,
                                                       int ring_cap) {
  __shared__ double sg[NG][FT];
  __shared__ double smin_w[FT], smin_n[FT];
  __shared__ int smin_x[FT];
  const int t = threadIdx.x;
  double acc[NG];
#pragma unroll
  for (int k = 0; k < NG; ++k) acc[k] = 0.0;
  acc[7] = 1e300;
  acc[8] = -1e300;
#pragma unroll 4
  for (int b = t; b < nblocks; b += FT) {
    const double* r = blocks + (long long)b * stride * NG;
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] += r[k];
    acc[6] = fmax(acc[6], r[6]);
    acc[7] = fmin(acc[7], r[7]);
    acc[8] = fmax(acc[8], r[8]);
    acc[9] = fmax(acc[9], r[9]);
  }
  // minima over the slice totals (first x on ties)
  double mw = 1e300, mn = 1e300;
  int mx = 0x7fffffff;
  for (int x = t; x < g.nx; x += FT) {
    const double a = slice_tot[2 * x], c = slice_tot[2 * x + 1];
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
    if (ring_count) {
      const unsigned long long n = *ring_count;
      *ring_count = n + 1;
      out += (n % (unsigned long long)ring_cap) * DIAG_STRIDE;
      out[DIAG_OUT] = (double)n;
      out[DIAG_CCL + 0] = out[DIAG_CCL + 1] = out[DIAG_CCL + 2] = -1.0;
      out[DIAG_CCL + 3] = 0.0;
    }
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

// After the unions every tree is final, so pointing a node straight at its
// root (the smallest index of its component) leaves every concurrent root
// search valid.
__global__ void ccl_compress_kernel(Geom g, int* L, int* sizes, unsigned long long* err) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N || L[i] < 0) return;
  long long hops = 0;
  const int r = find_root(L, (int)i, hops);
  if (hops >= kMaxHops) atomicOr(err, 1ull);
  L[i] = r;
  atomicAdd(&sizes[r], 1);
}

__global__ void ccl_count_kernel(Geom g, const int* L, const int* sizes, unsigned long long* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N || L[i] != (int)i) return;
  atomicAdd(&out[0], 1ull);
  if (sizes[i] >= 8) atomicAdd(&out[1], 1ull);
  atomicMax(&out[2], (unsigned long long)sizes[i]);
}

// Copies the droplet counts of the CCL just run into the ring record the
// diagnostics of the same step appended (slot counter - 1).
__global__ void ccl_ring_kernel(const long long* out4, double* ring, const unsigned long long* ring_count,
                                int ring_cap) {
  const unsigned long long n = *ring_count - 1;
  double* rec = ring + (n % (unsigned long long)ring_cap) * DIAG_STRIDE;
  rec[DIAG_CCL + 0] = (double)out4[0];
  rec[DIAG_CCL + 1] = (double)out4[1];
  rec[DIAG_CCL + 2] = (double)out4[2];
  rec[DIAG_CCL + 3] = (double)out4[3];
}

// ---------------------------------------------------------------------------
// Per-droplet statistics (after launch_ccl): every root takes a record slot;
// every liquid node adds to its droplet's record
//   [root, nodes, sum phi, sum rho, cos/sin sums of 2 pi x/nx, y, z]
// and sets the bit of its x slice in the droplet's x-occupancy mask.  The
// FP64 sums are atomic (their order, and so the last bits, vary run to run).
// ---------------------------------------------------------------------------
__global__ void droplet_slot_kernel(Geom g, const int* L, int* slot_of, double* rec, unsigned* nslot,
                                    int cap) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N || L[i] != (int)i) return;
  const unsigned k = atomicAdd(nslot, 1u);
  slot_of[i] = k < (unsigned)cap ? (int)k : -1;
  if (k < (unsigned)cap) rec[(size_t)k * DROP_REC] = (double)i;
}

template <int P>
__global__ void droplet_stats_kernel(Geom g, Phys ph, int layout, const typename Prec<P>::T* f, double rho_l,
                                     double rho_v, const int* L, const int* slot_of, double* rec, unsigned* xbits,
                                     int words) {
  using C = typename Prec<P>::C;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int k = -1, x = 0;
  double v[DROP_REC - 1];
#pragma unroll
  for (int m = 0; m < DROP_REC - 1; ++m) v[m] = 0.0;
  if (i < g.N && L[i] >= 0) {
    k = slot_of[L[i]];
    if (k >= 0) {
      int y, z;
      coords(g, i, x, y, z);
      Nbr nb;
      nb.make(g, x, y, z);
      C rc, j[3];
      node_rho_j<P>(g, ph, layout, f, nb, rc, j);
      const double rho = (double)rc;
      v[0] = 1.0;
      v[1] = fmin(fmax((rho - rho_v) / (rho_l - rho_v), 0.0), 1.0);
      v[2] = rho;
      sincospi(2.0 * x / g.nx, &v[4], &v[3]);
      sincospi(2.0 * y / g.ny, &v[6], &v[5]);
      sincospi(2.0 * z / g.nz, &v[8], &v[7]);
    }
  }
  // one set of atomics per warp when all its liquid lanes share a droplet
  // (the common case: the warp covers 32 consecutive nodes of a row)
  const int kmax = __reduce_max_sync(0xffffffffu, k);
  const bool uniform = __all_sync(0xffffffffu, k < 0 || k == kmax);
  if (uniform) {
    if (kmax < 0) return;
#pragma unroll
    for (int m = 0; m < DROP_REC - 1; ++m)
      for (int o = 16; o > 0; o >>= 1) v[m] += __shfl_xor_sync(0xffffffffu, v[m], o);
    if ((threadIdx.x & 31) == 0) {
      double* r = rec + (size_t)kmax * DROP_REC + 1;
#pragma unroll
      for (int m = 0; m < DROP_REC - 1; ++m) atomicAdd(r + m, v[m]);
    }
  } else if (k >= 0) {
    double* r = rec + (size_t)k * DROP_REC + 1;
#pragma unroll
    for (int m = 0; m < DROP_REC - 1; ++m) atomicAdd(r + m, v[m]);
  }
  if (k >= 0) {
    unsigned* w = xbits + (size_t)k * words + (x >> 5);
    const unsigned bit = 1u << (x & 31);
    if (!(*(volatile unsigned*)w & bit)) atomicOr(w, bit);
  }
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
                   double rho_v, double* scratch, double* out, void* psi, int* flag,
                   unsigned long long* ring_count, int ring_cap, cudaStream_t s) {
  const int rb = diag_row_blocks(g);
  const int gx = (g.nx + DX - 1) / DX;
  double* slices = scratch;
  double* blocks = scratch + (size_t)rb * g.nx * 2;
  double* slice_tot = blocks + (size_t)gx * rb * NG;
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  const dim3 grid(gx, rb), block(DX, DY);
  if (psi) {
    if (layout == LAYOUT_LOCAL)
      diag_partial_kernel<P, true, LAYOUT_LOCAL><<<grid, block, 0, s>>>(
          g, ph, (const T*)f, rho_l, rho_v, slices, blocks, (C*)psi, flag);
    else
      diag_partial_kernel<P, true, LAYOUT_GATHER><<<grid, block, 0, s>>>(
          g, ph, (const T*)f, rho_l, rho_v, slices, blocks, (C*)psi, flag);
  } else {
    if (layout == LAYOUT_LOCAL)
      diag_partial_kernel<P, false, LAYOUT_LOCAL><<<grid, block, 0, s>>>(
          g, ph, (const T*)f, rho_l, rho_v, slices, blocks, nullptr, nullptr);
    else
      diag_partial_kernel<P, false, LAYOUT_GATHER><<<grid, block, 0, s>>>(
          g, ph, (const T*)f, rho_l, rho_v, slices, blocks, nullptr, nullptr);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_slices_kernel<<<(g.nx + 7) / 8, 256, 0, s>>>(g, rb, slices, slice_tot);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<1, FT, 0, s>>>(g, gx * rb, 1, slice_tot, blocks, out, ring_count, ring_cap);
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

template <int P>
cudaError_t droplets_t(int layout, const Geom& g, const Phys& ph, const void* f, double rho_l, double rho_v,
                       const int* L, int* slot_of, double* rec, unsigned* xbits, unsigned* nslot, int cap,
                       cudaStream_t s) {
  const unsigned nb = blocks_for(g.N, 256);
  const int words = (g.nx + 31) / 32;
  cudaError_t e = cudaMemsetAsync(rec, 0, sizeof(double) * DROP_REC * (size_t)cap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(xbits, 0, sizeof(unsigned) * words * (size_t)cap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(nslot, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  droplet_slot_kernel<<<nb, 256, 0, s>>>(g, L, slot_of, rec, nslot, cap);
  droplet_stats_kernel<P><<<nb, 256, 0, s>>>(g, ph, layout, (const typename Prec<P>::T*)f, rho_l, rho_v, L,
                                             slot_of, rec, xbits, words);
  return cudaGetLastError();
}

}  // namespace

// Stochastic-rounding step salt: set it (mode 1), advance it by one (mode
// 0, after each time step's collision) or by `value` (mode 2, after a launch
// that ran `value` steps).
__global__ void salt_kernel(unsigned* salt, int mode, unsigned value) {
  *salt = mode == 1 ? value : *salt + (mode == 2 ? value : 1u);
}

cudaError_t launch_salt(unsigned* salt, bool set, unsigned value, cudaStream_t s) {
  salt_kernel<<<1, 1, 0, s>>>(salt, set ? 1 : 0, value);
  return cudaGetLastError();
}

cudaError_t launch_salt_add(unsigned* salt, unsigned n, cudaStream_t s) {
  salt_kernel<<<1, 1, 0, s>>>(salt, 2, n);
  return cudaGetLastError();
}

cudaError_t launch_diag_reduce(const Geom& g, int row_blocks, int nblocks, const double* slices,
                               double* blocks, double* slice_tot, double* out,
                               unsigned long long* ring_count, int ring_cap, cudaStream_t s) {
  diag_slices_kernel<<<(g.nx + 7) / 8, 256, 0, s>>>(g, row_blocks, slices, slice_tot);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // many records (one per block of the fused step): a parallel first stage
  // folds runs of kChunk records in place (a single block reading 131072
  // records of the 1024x512x512 lattice took 0.44 ms)
  constexpr int kChunk = 256;
  int stride = 1, n = nblocks;
  if (nblocks > 4 * kChunk) {
    n = (nblocks + kChunk - 1) / kChunk;
    diag_blocks_kernel<<<n, FT, 0, s>>>(nblocks, kChunk, blocks);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stride = kChunk;
  }
  diag_final_kernel<<<1, FT, 0, s>>>(g, n, stride, slice_tot, blocks, out, ring_count, ring_cap);
  return cudaGetLastError();
}

cudaError_t launch_ccl_ring(const long long* out4, double* ring, const unsigned long long* ring_count,
                            int ring_cap, cudaStream_t s) {
  ccl_ring_kernel<<<1, 1, 0, s>>>(out4, ring, ring_count, ring_cap);
  return cudaGetLastError();
}

cudaError_t launch_droplets(int precision, int layout, const Geom& g, const Phys& ph, const void* f,
                            double rho_l, double rho_v, const int* labels, int* sizes, double* rec,
                            unsigned* xbits, unsigned* nslot, int cap, cudaStream_t s) {
  switch (precision) {
    case LBM_F64: return droplets_t<LBM_F64>(layout, g, ph, f, rho_l, rho_v, labels, sizes, rec, xbits, nslot, cap, s);
    case LBM_F32: return droplets_t<LBM_F32>(layout, g, ph, f, rho_l, rho_v, labels, sizes, rec, xbits, nslot, cap, s);
    case LBM_F16DEV:
      return droplets_t<LBM_F16DEV>(layout, g, ph, f, rho_l, rho_v, labels, sizes, rec, xbits, nslot, cap, s);
    case LBM_BF16DEV:
      return droplets_t<LBM_BF16DEV>(layout, g, ph, f, rho_l, rho_v, labels, sizes, rec, xbits, nslot, cap, s);
  }
  return cudaErrorInvalidValue;
}

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
  return (size_t)rb * g.nx * 2 + (size_t)gx * rb * NG + (size_t)g.nx * 2;
}

cudaError_t launch_diagnostics(int precision, int layout, const Geom& g, const Phys& ph, const void* f,
                               double rho_l, double rho_v, double* scratch, double* out, void* psi,
                               int* flag, unsigned long long* ring_count, int ring_cap,
                               cudaStream_t s) {
  switch (precision) {
    case LBM_F64:
      return diag_t<LBM_F64>(layout, g, ph, f, rho_l, rho_v, scratch, out, psi, flag, ring_count, ring_cap, s);
    case LBM_F32:
      return diag_t<LBM_F32>(layout, g, ph, f, rho_l, rho_v, scratch, out, psi, flag, ring_count, ring_cap, s);
    case LBM_F16DEV:
      return diag_t<LBM_F16DEV>(layout, g, ph, f, rho_l, rho_v, scratch, out, psi, flag, ring_count, ring_cap, s);
    case LBM_BF16DEV:
      return diag_t<LBM_BF16DEV>(layout, g, ph, f, rho_l, rho_v, scratch, out, psi, flag, ring_count, ring_cap, s);
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
