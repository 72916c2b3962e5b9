// Per-node bodies of the two time-step kernels, shared by the single-lattice
// kernels (lbm_step.cu) and the batched kernels (lbm_batch.cu) so that a
// batched instance computes bitwise what a standalone lattice computes.
//
//   psi pass      rho = sum_a f_a (Eq. 4) and psi(rho) of a node.  The force
//                 of Eq. 5 needs psi of all 18 neighbours at the same time
//                 level, so psi exists for the whole lattice before any
//                 collision starts.
//   collide       moments (Eq. 4), Shan-Chen force from the neighbour psi
//                 (Eq. 5), velocity shift u' = (j + tau F)/rho (Eq. 6),
//                 second-order equilibrium (Eq. 2, with the leading 1), BGK
//                 relaxation (Eq. 3) and streaming to x + c_a.
//
// Each comes in a one-node form and a two-node form (x and x + 1, x even)
// that loads and stores pairs of populations as one 2-element vector where
// the addresses allow it.  Both forms call the same arithmetic
// (collide_math, psi_math), so their results are identical.
#pragma once

#include "lbm_internal.h"
#include "lbm_mrt.cuh"

namespace lbm {

// The deviation shift of population a in storage P (the FP32 form the host
// set in ph: storage_shift of ph.rho_ref).
template <int P>
__device__ __forceinline__ typename Prec<P>::C shift_of(int a, const Phys& ph) {
  using C = typename Prec<P>::C;
  if constexpr (Prec<P>::dev) {
    return (C)ph.shift_f[a == 0 ? 0 : (a <= 6 ? 1 : 2)];
  } else {
    return (C)0;
  }
}

// Two adjacent stored populations (x, x + 1) as one vector access.
template <int P> struct Pair;
template <> struct Pair<LBM_F64> {
  using V = double2;
  __device__ static __forceinline__ void unpack(V v, double& a, double& b) { a = v.x; b = v.y; }
  __device__ static __forceinline__ V pack(double a, double b) { return make_double2(a, b); }
  __device__ static __forceinline__ V pack_sr(double a, double b, unsigned, unsigned) { return make_double2(a, b); }
};
template <> struct Pair<LBM_F32> {
  using V = float2;
  __device__ static __forceinline__ void unpack(V v, float& a, float& b) { a = v.x; b = v.y; }
  __device__ static __forceinline__ V pack(float a, float b) { return make_float2(a, b); }
  __device__ static __forceinline__ V pack_sr(float a, float b, unsigned, unsigned) { return make_float2(a, b); }
};
template <> struct Pair<LBM_F16DEV> {
  using V = __half2;
  __device__ static __forceinline__ void unpack(V v, float& a, float& b) {
    a = __low2float(v);
    b = __high2float(v);
  }
  __device__ static __forceinline__ V pack(float a, float b) {
    return __halves2half2(__float2half_rn(a), __float2half_rn(b));
  }
  __device__ static __forceinline__ V pack_sr(float a, float b, unsigned ra, unsigned rb) {
    const unsigned d = cvt_rs_f16x2(b, a, (rb << 16) | (ra & 0xFFFFu));   // x + 1 high, x low
    V v;
    memcpy(&v, &d, 4);
    return v;
  }
};
template <> struct Pair<LBM_BF16DEV> {
  using V = __nv_bfloat162;
  __device__ static __forceinline__ void unpack(V v, float& a, float& b) {
    a = __low2float(v);
    b = __high2float(v);
  }
  __device__ static __forceinline__ V pack(float a, float b) {
    return __halves2bfloat162(__float2bfloat16_rn(a), __float2bfloat16_rn(b));
  }
  __device__ static __forceinline__ V pack_sr(float a, float b, unsigned ra, unsigned rb) {
    const unsigned d = cvt_rs_bf16x2(b, a, (rb << 16) | (ra & 0xFFFFu));
    V v;
    memcpy(&v, &d, 4);
    return v;
  }
};

// Stored value to compute precision plus the deviation shift.  For 2-byte
// storage one widening add (add.rn.f32.f16 / .bf16, sm_100 and later) does
// both: the conversion is exact, so the result is the FP32 sum of the
// converted value and the shift rounded once to nearest, the bits of the
// conversion-then-add of the two-kernel step.
__device__ __forceinline__ float add_wide(__half h, float c) {
  float d;
  asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(__half_as_ushort(h)), "f"(c));
  return d;
}
__device__ __forceinline__ float add_wide(__nv_bfloat16 h, float c) {
  float d;
  asm("add.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(__bfloat16_as_ushort(h)), "f"(c));
  return d;
}
template <int P>
__device__ __forceinline__ void unpack_shifted(typename Pair<P>::V v, float sh, float& a, float& b) {
  if constexpr (P == LBM_F16DEV) {
    a = add_wide(__low2half(v), sh);
    b = add_wide(__high2half(v), sh);
  } else if constexpr (P == LBM_BF16DEV) {
    a = add_wide(__low2bfloat16(v), sh);
    b = add_wide(__high2bfloat16(v), sh);
  } else {
    Pair<P>::unpack(v, a, b);   // full precision: no shift
  }
}
// Two FP32 values to a packed 2-byte pair with stochastic rounding: hi takes
// the random bits rbits[31:16], lo rbits[15:0].
template <int P>
__device__ __forceinline__ unsigned cvt_pair_sr(float hi, float lo, unsigned rbits) {
  if constexpr (P == LBM_BF16DEV)
    return cvt_rs_bf16x2(hi, lo, rbits);
  else
    return cvt_rs_f16x2(hi, lo, rbits);
}
template <int P>
__device__ __forceinline__ float load_shifted(const typename Prec<P>::T* p, float sh) {
  if constexpr (Prec<P>::dev)
    return add_wide(*p, sh);
  else
    return *p;
}

// Loads populations x and x + 1 (RO: read-only path; else a plain load for
// in-place updates) and adds the deviation shift.  Full-precision storage has
// no shift and skips the add (x + 0 is not x for x = -0, so the compiler
// keeps it otherwise), as Prec<P>::load does.
template <int P, bool RO>
__device__ __forceinline__ void load_pair(const typename Prec<P>::T* p, typename Prec<P>::C sh,
                                          typename Prec<P>::C& a, typename Prec<P>::C& b) {
  using V = typename Pair<P>::V;
  V v;
  if constexpr (RO)
    v = __ldg(reinterpret_cast<const V*>(p));
  else
    v = *reinterpret_cast<const V*>(p);
  Pair<P>::unpack(v, a, b);
  if constexpr (Prec<P>::dev) {
    a += sh;
    b += sh;
  }
}

template <int P>
__device__ __forceinline__ void store_pair(typename Prec<P>::T* p, typename Prec<P>::C a,
                                           typename Prec<P>::C b, typename Prec<P>::C sh) {
  using V = typename Pair<P>::V;
  *reinterpret_cast<V*>(p) = Pair<P>::pack(a - sh, b - sh);
}

template <int P>
__device__ __forceinline__ void store_pair_sr(typename Prec<P>::T* p, typename Prec<P>::C a,
                                              typename Prec<P>::C b, typename Prec<P>::C sh,
                                              unsigned ra, unsigned rb) {
  using V = typename Pair<P>::V;
  *reinterpret_cast<V*>(p) = Pair<P>::pack_sr(a - sh, b - sh, ra, rb);
}

// Store of population a of a node with seed s: nearest, or stochastic when
// the lattice asks for it (reduced-precision storage only).
template <int P>
__device__ __forceinline__ void store_pop(const Phys& ph, typename Prec<P>::T* p,
                                          typename Prec<P>::C v, typename Prec<P>::C sh, unsigned s,
                                          int a) {
  if (Prec<P>::dev && ph.sr)
    Prec<P>::store_sr(p, v, sh, sr_bits(s, a));
  else
    Prec<P>::store(p, v, sh);
}

// ---------------------------------------------------------------------------
// arithmetic of one node
// ---------------------------------------------------------------------------

// Correctly rounded reciprocal: the bits of 1 / x (IEEE division) without
// the division's general path.
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }

// Lane-wise correctly rounded reciprocal of a pair.
__device__ __forceinline__ float2 rcp_rn(float2 x) { return make_float2(__frcp_rn(x.x), __frcp_rn(x.y)); }

// c_a . u for odd a, whose first nonzero velocity component is +1: sums of
// the velocity components only (no 0 + u_x, which the compiler must keep
// for a -0 operand).
static_assert(cx(9) == 1 && cx(13) == 1 && cy(17) == 1 && cy(15) == 1 && cx(1) == 1 && cy(3) == 1 &&
                  cz(5) == 1 && cx(7) == 1 && cx(11) == 1,
              "odd directions lead with a +1 component");
template <typename C>
__device__ __forceinline__ C cdotu(int a, C ux, C uy, C uz) {
  if (cx(a)) {
    C cu = ux;
    if (cy(a)) cu = cy(a) > 0 ? vadd(cu, uy) : vsub(cu, uy);
    if (cz(a)) cu = cz(a) > 0 ? vadd(cu, uz) : vsub(cu, uz);
    return cu;
  }
  if (cy(a)) return cz(a) ? (cz(a) > 0 ? vadd(uy, uz) : vsub(uy, uz)) : uy;
  return uz;
}

// Post-collision populations fs of a node with populations f, density rho
// (= rho_of(f), passed in where the caller has it already), momentum (jx,
// jy, jz) = mom_of(f) (Eq. 4), psi(x) = pc and the link sums of its
// neighbour values (link_sums).  C = float2 computes two nodes, lane by lane
// with the bits of C = float.
template <typename C>
__device__ __forceinline__ void collide_math_ls(const Phys& ph, const C f[Q], C rho, C jx, C jy, C jz, C pc, C ax,
                                                C ay, C az, C dx, C dy, C dz, C fs[Q]) {
  using S = typename Lane<C>::S;
  // Eq. 5: sum_a w_a psi(x + c_a) c_a, split by weight class.  Products and
  // sums below go through xmul / xfma / vadd / vsub (round to nearest, fused
  // only where written), so every kernel that inlines this function computes
  // the same bits whatever the compiler's contraction choices around it.
  const C w1 = splat<C>((S)(1.0 / 18.0)), w2 = splat<C>((S)(1.0 / 36.0));
  // the constants in the arithmetic's precision (FP32: the host's
  // conversions, read from the kernel parameters)
  S G_s, tau_s, omega_s;
  if constexpr (sizeof(S) == 4) {
    G_s = ph.G_f, tau_s = ph.tau_f, omega_s = ph.omega_f;
  } else {
    G_s = (S)ph.G, tau_s = (S)ph.tau, omega_s = (S)1 / tau_s;
  }
  const C gp = xmul(splat<C>(-G_s), pc);
  const C Fx = xmul(gp, xfma(w1, ax, xmul(w2, dx)));
  const C Fy = xmul(gp, xfma(w1, ay, xmul(w2, dy)));
  const C Fz = xmul(gp, xfma(w1, az, xmul(w2, dz)));
  // Eq. 6
  const C tau = splat<C>(tau_s);
  const C inv_rho = rcp_rn(rho);
  const C ux = xmul(xfma(tau, Fx, jx), inv_rho);
  const C uy = xmul(xfma(tau, Fy, jy), inv_rho);
  const C uz = xmul(xfma(tau, Fz, jz), inv_rho);
  const C usq = xmul(splat<C>((S)1.5), xfma(uz, uz, xfma(uy, uy, xmul(ux, ux))));
  // Eq. 2 and Eq. 3 as f* = (1 - omega) f + omega f_eq.  For the pair a, b =
  // opp(a) of weight w, with q = omega w rho and cu = c_a . u':
  //   omega f_eq_a = A + B,  omega f_eq_b = A - B,
  //   A = q (1 - 3/2 u'.u') + (9/2) q cu^2,  B = 3 q cu,
  // and q, 9/2 q, 3 q of the diagonal class are exactly half those of the
  // axis class (w2 = w1 / 2).  The rest population takes omega f_eq_0 =
  // omega rho - 2 sum_pairs A, which equals Eq. 2's omega w_0 rho (1 - 3/2
  // u'.u') for the exact weights (sum_{a>=1} w_a = 2/3, sum_{a>=1} w_a
  // (c_a.u')^2 = u'.u'/3) and keeps sum_a f* = rho up to unbiased rounding
  // (with weights rounded to the arithmetic's precision the direct form of
  // Eq. 2 creates mass of relative order 1e-8 per FP32 collision in one
  // direction).
  const C om1 = splat<C>((S)1 - omega_s);
  const C orho = xmul(splat<C>(omega_s), rho);
  const C q1 = xmul(orho, w1);
  const C E1 = xmul(q1, vsub(splat<C>((S)1), usq)), M1 = xmul(splat<C>((S)4.5), q1),
          T1 = xmul(splat<C>((S)3), q1);
  const C half = splat<C>((S)0.5);
  const C E2 = xmul(half, E1), M2 = xmul(half, M1), T2 = xmul(half, T1);
  C sumA = splat<C>((S)0);
#pragma unroll
  for (int a = 1; a < Q; a += 2) {
    const int b = a + 1;  // opp(a)
    const bool axis = a <= 6;
    const C cu = cdotu<C>(a, ux, uy, uz);
    const C A = xfma(xmul(axis ? M1 : M2, cu), cu, axis ? E1 : E2);
    const C B = xmul(axis ? T1 : T2, cu);
    sumA = a == 1 ? A : vadd(sumA, A);
    fs[a] = xfma(om1, f[a], vadd(A, B));
    fs[b] = xfma(om1, f[b], vsub(A, B));
  }
  fs[0] = xfma(om1, f[0], xfma(splat<C>((S)-2), sumA, orho));
}

// The same from the neighbour values pn[a] = psi(x + c_a) (a = 1..18).
template <typename C>
__device__ __forceinline__ void collide_math_r(const Phys& ph, const C f[Q], C rho, C pc, const C pn[Q],
                                               C fs[Q]) {
  // (the link sums first: with the momentum first the batched collide-stream
  // kernel, compiled to 64 - 80 registers, ran 6 % slower)
  C jx, jy, jz, ax, ay, az, dx, dy, dz;
  link_sums<C>(pn, ax, ay, az, dx, dy, dz);
  mom_of<C>(f, jx, jy, jz);
  collide_math_ls<C>(ph, f, rho, jx, jy, jz, pc, ax, ay, az, dx, dy, dz, fs);
}

template <typename C>
__device__ __forceinline__ void collide_math(const Phys& ph, const C f[Q], C pc, const C pn[Q], C fs[Q]) {
  collide_math_r<C>(ph, f, rho_of<C>(f), pc, pn, fs);
}

// The collision of two x-adjacent nodes (x, x + 1) as the lanes of float2,
// with the bits of collide_math_r<float> per node: f their populations,
// rho their densities, q[dy + 1][dz + 1][i] psi at x - 1 + i of the row (y +
// dy, z + dz).  The link differences of the directions with c_x = 0 are one
// paired difference of the pair's own two values, those of the x-shifted
// directions two scalar differences (their results pair up freely).
__device__ __forceinline__ void collide_pair_math(const Phys& ph, const float2 f[Q], float2 rho,
                                                  const float (&q)[3][3][4], float2 fs[Q]) {
  float2 e[Q];
#pragma unroll
  for (int a = 1; a < Q; a += 2) {
    const int b = a + 1;
    const float* qa = q[cy(a) + 1][cz(a) + 1];
    const float* qb = q[cy(b) + 1][cz(b) + 1];
    if (cx(a) == 0)
      e[a] = vsub(make_float2(qa[1], qa[2]), make_float2(qb[1], qb[2]));
    else
      e[a] = make_float2(qa[1 + cx(a)] - qb[1 + cx(b)], qa[2 + cx(a)] - qb[2 + cx(b)]);
  }
  float2 ax, ay, az, dx, dy, dz, jx, jy, jz;
  link_combine<float2>(e, ax, ay, az, dx, dy, dz);
  mom_of<float2>(f, jx, jy, jz);
  collide_math_ls<float2>(ph, f, rho, jx, jy, jz, make_float2(q[1][1][1], q[1][1][2]), ax, ay, az, dx, dy, dz, fs);
}

// A non-positive, NaN or infinite density (the numeric flag's condition).
template <typename C>
__device__ __forceinline__ bool bad_rho(C rho) {
  return !(rho > (C)0) || !(rho <= (C)3.0e38);
}

template <typename C>
__device__ __forceinline__ void psi_math(const Phys& ph, C rho, C* out, int* flag) {
  *out = psi_of<C>(rho, ph);
  raise_flag(bad_rho(rho), flag);
}

// ---------------------------------------------------------------------------
// psi pass
// ---------------------------------------------------------------------------

// LAYOUT_LOCAL reads slot a at x; LAYOUT_GATHER (AA before an odd step)
// reads slot opp(a) at x - c_a.
template <int P, int LAYOUT>
__device__ __forceinline__ void psi_node(const Geom& g, const Phys& ph,
                                         const typename Prec<P>::T* f,
                                         typename Prec<P>::C* __restrict__ psi,
                                         int* __restrict__ flag, long long i) {
  using C = typename Prec<P>::C;
  const C s0 = shift_of<P>(0, ph), s1 = shift_of<P>(1, ph),
          s2 = shift_of<P>(7, ph);
  C fv[Q];
  if constexpr (LAYOUT == LAYOUT_LOCAL) {
#pragma unroll
    for (int a = 0; a < Q; ++a)
      fv[a] = Prec<P>::load(f + (long long)a * g.N + i, a == 0 ? s0 : (a <= 6 ? s1 : s2));
  } else {
    const int x = (int)(i % g.nx);
    const long long r = i / g.nx;
    const int y = (int)(r % g.ny), z = (int)(r / g.ny);
    Nbr nb;
    nb.make(g, x, y, z);
#pragma unroll
    for (int a = 0; a < Q; ++a)
      fv[a] = Prec<P>::load(f + (long long)opp(a) * g.N + nb.idx(-cx(a), -cy(a), -cz(a)),
                            a == 0 ? s0 : (a <= 6 ? s1 : s2));
  }
  psi_math<C>(ph, rho_of<C>(fv), psi + i, flag);
}

// Two nodes i, i + 1 (i even, nx even), vector loads where the addresses
// allow (all of LAYOUT_LOCAL; the c_x = 0 slots of LAYOUT_GATHER) and a
// vector store of the two psi values.
template <int P, int LAYOUT>
__device__ __forceinline__ void psi_pair(const Geom& g, const Phys& ph, const typename Prec<P>::T* f,
                                         typename Prec<P>::C* __restrict__ psi,
                                         int* __restrict__ flag, long long i) {
  using C = typename Prec<P>::C;
  const C s0 = shift_of<P>(0, ph), s1 = shift_of<P>(1, ph),
          s2 = shift_of<P>(7, ph);
  C f0[Q], f1[Q];
  if constexpr (LAYOUT == LAYOUT_LOCAL) {
#pragma unroll
    for (int a = 0; a < Q; ++a)
      load_pair<P, true>(f + (long long)a * g.N + i, a == 0 ? s0 : (a <= 6 ? s1 : s2), f0[a], f1[a]);
  } else {
    const int x0 = (int)(i % g.nx);
    const long long r = i / g.nx;
    const int y = (int)(r % g.ny), z = (int)(r / g.ny);
    const int xm = x0 == 0 ? g.nx - 1 : x0 - 1, xp = x0 + 2 == g.nx ? 0 : x0 + 2;
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
    const int yv[3] = {ym, y, yp}, zv[3] = {zm, z, zp};
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      // slot opp(a) at x - c_a
      const int row = g.nx * (yv[1 - cy(a)] + g.ny * zv[1 - cz(a)]);
      const typename Prec<P>::T* base = f + (long long)opp(a) * g.N + row;
      const C sh = a == 0 ? s0 : (a <= 6 ? s1 : s2);
      if (cx(a) == 0) {
        load_pair<P, true>(base + x0, sh, f0[a], f1[a]);
      } else if (cx(a) > 0) {  // from x0 - 1 and x0
        f0[a] = Prec<P>::load(base + xm, sh);
        f1[a] = Prec<P>::load(base + x0, sh);
      } else {                 // from x0 + 1 and x0 + 2
        f0[a] = Prec<P>::load(base + x0 + 1, sh);
        f1[a] = Prec<P>::load(base + xp, sh);
      }
    }
  }
  if constexpr (sizeof(C) == 4) {
    // the two nodes as float2 lanes (paired FP32 instructions, the bits of
    // the scalar form)
    float2 fp[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) fp[a] = make_float2(f0[a], f1[a]);
    const float2 rho = rho_of<float2>(fp);
    raise_flag(bad_rho(rho.x) | bad_rho(rho.y), flag);
    *reinterpret_cast<float2*>(psi + i) = psi_of2(rho, ph);
  } else {
    C p0, p1;
    psi_math<C>(ph, rho_of<C>(f0), &p0, flag);
    psi_math<C>(ph, rho_of<C>(f1), &p1, flag);
    *reinterpret_cast<double2*>(psi + i) = make_double2(p0, p1);
  }
}

// The four populations of slot `a` at x0 .. x0 + 3 of a row (x0 % 4 == 0,
// 16-byte (FP32) or 8-byte (2-byte) aligned), unpacked and shifted.
template <int P>
__device__ __forceinline__ void load_quad(const typename Prec<P>::T* p, float sh, float v[4]) {
  if constexpr (P == LBM_F32) {
    const float4 w = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = w.x;
    v[1] = w.y;
    v[2] = w.z;
    v[3] = w.w;
  } else {
    const uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
    typename Pair<P>::V lo, hi;
    memcpy(&lo, &raw.x, 4);
    memcpy(&hi, &raw.y, 4);
    Pair<P>::unpack(lo, v[0], v[1]);
    Pair<P>::unpack(hi, v[2], v[3]);
    v[0] += sh;
    v[1] += sh;
    v[2] += sh;
    v[3] += sh;
  }
}

// Four nodes i .. i + 3 (i % 4 == 0, nx % 4 == 0, LAYOUT_LOCAL): one 16-byte
// (FP32) or 8-byte (FP16/BF16) load per population, one 16-byte psi store.
template <int P>
__device__ __forceinline__ void psi_quad(const Geom& g, const Phys& ph, const typename Prec<P>::T* f,
                                         typename Prec<P>::C* __restrict__ psi,
                                         int* __restrict__ flag, long long i) {
  static_assert(P != LBM_F64, "four-node psi pass is for 4- and 2-byte storage");
  const float s0 = shift_of<P>(0, ph), s1 = shift_of<P>(1, ph),
              s2 = shift_of<P>(7, ph);
  float fv[4][Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    float v[4];
    load_quad<P>(f + (long long)a * g.N + i, a == 0 ? s0 : (a <= 6 ? s1 : s2), v);
#pragma unroll
    for (int k = 0; k < 4; ++k) fv[k][a] = v[k];
  }
  // nodes (0, 1) and (2, 3) as float2 lanes (paired FP32 instructions, the
  // bits of the scalar form)
  float2 pa[Q], pb[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) pa[a] = make_float2(fv[0][a], fv[1][a]), pb[a] = make_float2(fv[2][a], fv[3][a]);
  const float2 ra = rho_of<float2>(pa), rb = rho_of<float2>(pb);
  raise_flag(bad_rho(ra.x) | bad_rho(ra.y) | bad_rho(rb.x) | bad_rho(rb.y), flag);
  const float2 qa = psi_of2(ra, ph), qb = psi_of2(rb, ph);
  *reinterpret_cast<float4*>(psi + i) = make_float4(qa.x, qa.y, qb.x, qb.y);
}

// Four nodes i .. i + 3 in the gather layout (AA before an odd step: slot
// opp(a) at x - c_a; i % 4 == 0, nx % 4 == 0), for every lane of a warp
// (live: i < N; the others compute on a valid quad and store nothing).  Per
// direction one aligned vector load of the quad at x0 in the source row;
// for c_x = +1 the node x0 - 1 comes from the lane below (its quad's last
// node), for c_x = -1 the node x0 + 4 from the lane above (its first),
// except where that lane holds another row or none (lanes 0 and 31, row
// ends), which load it.  The same values, and psi, as psi_pair.
template <int P>
__device__ __forceinline__ void psi_quad_gather(const Geom& g, const Phys& ph, const typename Prec<P>::T* f,
                                                typename Prec<P>::C* __restrict__ psi, int* __restrict__ flag,
                                                long long i, bool live) {
  static_assert(P != LBM_F64, "four-node psi pass is for 4- and 2-byte storage");
  const float s0 = shift_of<P>(0, ph), s1 = shift_of<P>(1, ph),
              s2 = shift_of<P>(7, ph);
  const int lane = threadIdx.x & 31;
  const int x0 = (int)(i % g.nx);
  const long long r = i / g.nx;
  const int y = (int)(r % g.ny), z = (int)(r / g.ny);
  const int yv[3] = {y == 0 ? g.ny - 1 : y - 1, y, y == g.ny - 1 ? 0 : y + 1};
  const int zv[3] = {z == 0 ? g.nz - 1 : z - 1, z, z == g.nz - 1 ? 0 : z + 1};
  const bool own_lo = lane == 0 || x0 == 0;            // loads x0 - 1 itself
  const bool own_hi = lane == 31 || x0 + 4 == g.nx;    // loads x0 + 4 itself
  const int xlo = x0 == 0 ? g.nx - 1 : x0 - 1, xhi = x0 + 4 == g.nx ? 0 : x0 + 4;
  float fv[4][Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const float sh = a == 0 ? s0 : (a <= 6 ? s1 : s2);
    const typename Prec<P>::T* base = f + (long long)opp(a) * g.N + (long long)g.nx * (yv[1 - cy(a)] + g.ny * zv[1 - cz(a)]);
    float v[4];
    load_quad<P>(base + x0, sh, v);
    if (cx(a) == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) fv[k][a] = v[k];
    } else if (cx(a) > 0) {   // x0 - 1 .. x0 + 2
      float e = __shfl_up_sync(0xffffffffu, v[3], 1);
      if (own_lo) e = load_shifted<P>(base + xlo, sh);
      fv[0][a] = e;
      fv[1][a] = v[0];
      fv[2][a] = v[1];
      fv[3][a] = v[2];
    } else {                  // x0 + 1 .. x0 + 4
      float e = __shfl_down_sync(0xffffffffu, v[0], 1);
      if (own_hi) e = load_shifted<P>(base + xhi, sh);
      fv[0][a] = v[1];
      fv[1][a] = v[2];
      fv[2][a] = v[3];
      fv[3][a] = e;
    }
  }
  float2 pa[Q], pb[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) pa[a] = make_float2(fv[0][a], fv[1][a]), pb[a] = make_float2(fv[2][a], fv[3][a]);
  const float2 ra = rho_of<float2>(pa), rb = rho_of<float2>(pb);
  if (!live) return;
  raise_flag(bad_rho(ra.x) | bad_rho(ra.y) | bad_rho(rb.x) | bad_rho(rb.y), flag);
  const float2 qa = psi_of2(ra, ph), qb = psi_of2(rb, ph);
  *reinterpret_cast<float4*>(psi + i) = make_float4(qa.x, qa.y, qb.x, qb.y);
}

// ---------------------------------------------------------------------------
// collide + stream
// ---------------------------------------------------------------------------

// One node.
template <int P, int MODE, int COLL = COLL_SRT>
__device__ __forceinline__ void collide_node(const Geom& g, const Phys& ph,
                                             const typename Prec<P>::T* src,
                                             typename Prec<P>::T* dst,
                                             const typename Prec<P>::C* __restrict__ psi, int x,
                                             int y, int z) {
  using C = typename Prec<P>::C;
  Nbr nb;
  nb.make(g, x, y, z);
  const int i = nb.idx(0, 0, 0);
  const long long N = g.N;
  const C s0 = shift_of<P>(0, ph), s1 = shift_of<P>(1, ph),
          s2 = shift_of<P>(7, ph);
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
  C pn[Q];
  pn[0] = 0;
#pragma unroll
  for (int a = 1; a < Q; ++a) pn[a] = __ldg(psi + nb.idx(cx(a), cy(a), cz(a)));
  C fs[Q];
  if constexpr (COLL == COLL_MRT)
    collide_math_mrt<C>(ph, f, __ldg(psi + i), pn, fs);
  else
    collide_math<C>(ph, f, __ldg(psi + i), pn, fs);
  const unsigned seed = (Prec<P>::dev && ph.sr) ? sr_seed(i, fs[0], salt_of(ph)) : 0u;
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const C sh = a == 0 ? s0 : (a <= 6 ? s1 : s2);
    long long d;  // 64-bit: plane offset a * N plus the in-plane index
    if constexpr (MODE == MODE_AA_EVEN)
      d = (long long)opp(a) * N + i;
    else
      d = (long long)a * N + nb.idx(cx(a), cy(a), cz(a));
    store_pop<P>(ph, dst + d, fs[a], sh, seed, a);
  }
}

// Two nodes x0, x0 + 1 of one row (x0 even, nx even).  Populations whose
// address pair is contiguous and aligned (x unchanged) move as one vector;
// those shifted along x (c_x != 0 on a gather or scatter) move one by one.
template <int P, int MODE, int COLL = COLL_SRT>
__device__ __forceinline__ void collide_pair(const Geom& g, const Phys& ph,
                                             const typename Prec<P>::T* src,
                                             typename Prec<P>::T* dst,
                                             const typename Prec<P>::C* __restrict__ psi, int x0,
                                             int y, int z) {
  using C = typename Prec<P>::C;
  const int xm = x0 == 0 ? g.nx - 1 : x0 - 1;      // left of node 0
  const int xp = x0 + 2 == g.nx ? 0 : x0 + 2;      // right of node 1
  const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
  const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
  const int yv[3] = {ym, y, yp}, zv[3] = {zm, z, zp};
  int rows[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) rows[i][k] = g.nx * (yv[i] + g.ny * zv[k]);
  // x of node k (0, 1) moved by d (-1, 0, 1)
  auto xof = [&](int k, int d) -> int {
    return k == 0 ? (d < 0 ? xm : (d > 0 ? x0 + 1 : x0)) : (d < 0 ? x0 : (d > 0 ? xp : x0 + 1));
  };
  const int i0 = x0 + rows[1][1];
  const long long N = g.N;
  const C s0 = shift_of<P>(0, ph), s1 = shift_of<P>(1, ph),
          s2 = shift_of<P>(7, ph);

  C f0[Q], f1[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const C sh = a == 0 ? s0 : (a <= 6 ? s1 : s2);
    if constexpr (MODE == MODE_AB) {
      load_pair<P, true>(src + (long long)a * N + i0, sh, f0[a], f1[a]);
    } else if constexpr (MODE == MODE_AA_EVEN) {
      load_pair<P, false>(src + (long long)a * N + i0, sh, f0[a], f1[a]);
    } else {
      const int r = rows[1 - cy(a)][1 - cz(a)];
      const typename Prec<P>::T* base = src + (long long)opp(a) * N + r;
      if (cx(a) == 0) {
        load_pair<P, false>(base + x0, sh, f0[a], f1[a]);
      } else {
        f0[a] = Prec<P>::load_rw(base + xof(0, -cx(a)), sh);
        f1[a] = Prec<P>::load_rw(base + xof(1, -cx(a)), sh);
      }
    }
  }

  // psi along the 9 rows (y + dy, z + dz): q[..][0] = x0 - 1, [1] = x0,
  // [2] = x0 + 1, [3] = x0 + 2 (periodic); only the elements some direction
  // of that row needs are loaded.
  C q[3][3][4];
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
      const C* row = psi + rows[dy + 1][dz + 1];
      C c0, c1;
      if constexpr (sizeof(C) == 4) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(row + x0));
        c0 = v.x;
        c1 = v.y;
      } else {
        const double2 v = __ldg(reinterpret_cast<const double2*>(row + x0));
        c0 = v.x;
        c1 = v.y;
      }
      q[dy + 1][dz + 1][1] = c0;
      q[dy + 1][dz + 1][2] = c1;
      // rows holding a direction with c_x != 0: (0,0), (+-1,0), (0,+-1)
      if (dy == 0 || dz == 0) {
        q[dy + 1][dz + 1][0] = __ldg(row + xm);
        q[dy + 1][dz + 1][3] = __ldg(row + xp);
      } else {
        q[dy + 1][dz + 1][0] = 0;
        q[dy + 1][dz + 1][3] = 0;
      }
    }
  C pn0[Q], pn1[Q];
  pn0[0] = pn1[0] = 0;
#pragma unroll
  for (int a = 1; a < Q; ++a) {
    pn0[a] = q[cy(a) + 1][cz(a) + 1][1 + cx(a)];
    pn1[a] = q[cy(a) + 1][cz(a) + 1][2 + cx(a)];
  }
  C fs0[Q], fs1[Q];
  if constexpr (COLL == COLL_MRT) {
    collide_math_mrt<C>(ph, f0, q[1][1][1], pn0, fs0);
    collide_math_mrt<C>(ph, f1, q[1][1][2], pn1, fs1);
  } else if constexpr (sizeof(C) == 4) {
    float2 fp[Q], fs[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) fp[a] = make_float2(f0[a], f1[a]);
    collide_pair_math(ph, fp, rho_of<float2>(fp), q, fs);
#pragma unroll
    for (int a = 0; a < Q; ++a) fs0[a] = fs[a].x, fs1[a] = fs[a].y;
  } else {
    collide_math<C>(ph, f0, q[1][1][1], pn0, fs0);
    collide_math<C>(ph, f1, q[1][1][2], pn1, fs1);
  }
  const bool sr = Prec<P>::dev && ph.sr;
  const unsigned salt = sr ? salt_of(ph) : 0u;
  const unsigned seed0 = sr ? sr_seed(i0, fs0[0], salt) : 0u, seed1 = sr ? sr_seed(i0 + 1, fs1[0], salt) : 0u;

#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const C sh = a == 0 ? s0 : (a <= 6 ? s1 : s2);
    if constexpr (MODE == MODE_AA_EVEN) {
      if (sr)
        store_pair_sr<P>(dst + (long long)opp(a) * N + i0, fs0[a], fs1[a], sh, sr_bits(seed0, a),
                         sr_bits(seed1, a));
      else
        store_pair<P>(dst + (long long)opp(a) * N + i0, fs0[a], fs1[a], sh);
    } else {
      typename Prec<P>::T* base = dst + (long long)a * N + rows[1 + cy(a)][1 + cz(a)];
      if (cx(a) == 0) {
        if (sr)
          store_pair_sr<P>(base + x0, fs0[a], fs1[a], sh, sr_bits(seed0, a), sr_bits(seed1, a));
        else
          store_pair<P>(base + x0, fs0[a], fs1[a], sh);
      } else {
        store_pop<P>(ph, base + xof(0, cx(a)), fs0[a], sh, seed0, a);
        store_pop<P>(ph, base + xof(1, cx(a)), fs1[a], sh, seed1, a);
      }
    }
  }
}

// Grid-wide barrier of a cooperative launch: counter ctr (zero before the
// launch) reaches `target` = gridDim.x per barrier passed.  Thread 0 of each
// block releases the block's writes, arrives and polls with acquire loads,
// for at most kGridWaitNs of wall time (then it raises bit 2 of the flag and
// the barrier reports failure); the block barrier and an acquire fence in
// every thread then order all later loads of the block, through L1
// included, after every block's writes before the barrier.
constexpr unsigned long long kGridWaitNs = 2000000000ull;
__device__ __forceinline__ unsigned long long gsm_global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool grid_barrier(unsigned* ctr, unsigned target, int* flag,
                                             unsigned long long limit_ns) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    atomicAdd(ctr, 1u);
    const unsigned long long t0 = gsm_global_ns();
    for (;;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
      if (v >= target) break;
      if (gsm_global_ns() - t0 > limit_ns) {
        atomicOr(flag, 2);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
  }
  ok = __syncthreads_and(ok);
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  return ok != 0;
}

}  // namespace lbm
