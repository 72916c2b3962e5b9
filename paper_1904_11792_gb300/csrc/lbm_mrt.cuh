// Multiple-relaxation-time collision arithmetic of one node (used by the
// collide-stream bodies of lbm_node.cuh when the lattice selects it).
#pragma once

#include <utility>

#include "lbm_internal.h"

namespace lbm {

// ---------------------------------------------------------------------------
// Multiple-relaxation-time collision (the operator the conclusions name as
// the next step; not specified in the paper).  D3Q19 moments of d'Humieres,
// Ginzburg, Krafczyk, Lallemand and Luo (2002), rows as polynomials of the
// velocity c, and the forcing of Guo, Zheng and Shi (2002) in moment space:
//   m* = m - S (m - m_eq(rho, u)) + (I - S/2) M F_guo,  u = (j + F/2)/rho,
//   f* = M^-1 m* = M^T diag(1/|row|^2) m*.
// m_eq and M F_guo are the moments of Eq. 2's equilibrium and of Guo's
// forcing populations, in closed form.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int mrt_coef(int k, int a) {
  const int x = cx(a), y = cy(a), z = cz(a), c2 = x * x + y * y + z * z;
  switch (k) {
    case 0: return 1;
    case 1: return 19 * c2 - 30;
    case 2: return (21 * c2 * c2 - 53 * c2 + 24) / 2;
    case 3: return x;
    case 4: return (5 * c2 - 9) * x;
    case 5: return y;
    case 6: return (5 * c2 - 9) * y;
    case 7: return z;
    case 8: return (5 * c2 - 9) * z;
    case 9: return 3 * x * x - c2;
    case 10: return (3 * c2 - 5) * (3 * x * x - c2);
    case 11: return y * y - z * z;
    case 12: return (3 * c2 - 5) * (y * y - z * z);
    case 13: return x * y;
    case 14: return y * z;
    case 15: return x * z;
    case 16: return (y * y - z * z) * x;
    case 17: return (z * z - x * x) * y;
    default: return (x * x - y * y) * z;
  }
}
__host__ __device__ constexpr int mrt_norm(int k) {
  int n = 0;
  for (int a = 0; a < Q; ++a) n += mrt_coef(k, a) * mrt_coef(k, a);
  return n;
}

// v (+)= c * x with c a compile-time integer (0, +-1 and other values).
template <int Cf, typename C>
__device__ __forceinline__ void mrt_fma(C& v, C x) {
  if constexpr (Cf == 1) v += x;
  else if constexpr (Cf == -1) v -= x;
  else if constexpr (Cf != 0) v = xfma((C)Cf, x, v);
}
// m[K] = sum_a M[K][a] f[a] and f[A] = sum_k M[k][A] w[k], expanded at compile
// time so that only the non-zero integer coefficients cost instructions.
template <typename C, int K, int... A>
__device__ __forceinline__ C mrt_row(const C* f, std::integer_sequence<int, A...>) {
  C v = 0;
  (mrt_fma<mrt_coef(K, A)>(v, f[A]), ...);
  return v;
}
template <typename C, int A, int... K>
__device__ __forceinline__ C mrt_col(const C* w, std::integer_sequence<int, K...>) {
  C v = 0;
  (mrt_fma<mrt_coef(K, A)>(v, w[K]), ...);
  return v;
}
template <typename C, int... K>
__device__ __forceinline__ void mrt_forward(const C* f, C* m, std::integer_sequence<int, K...>) {
  ((m[K] = mrt_row<C, K>(f, std::make_integer_sequence<int, Q>{})), ...);
}
template <typename C, int... K>
__device__ __forceinline__ void mrt_scale(C* m, std::integer_sequence<int, K...>) {
  ((m[K] = xmul(m[K], (C)(1.0 / (double)mrt_norm(K)))), ...);
}
template <typename C, int... A>
__device__ __forceinline__ void mrt_backward(const C* w, C* fs, std::integer_sequence<int, A...>) {
  ((fs[A + 1] = mrt_col<C, A + 1>(w, std::make_integer_sequence<int, Q>{})), ...);
}

template <typename C>
__device__ __forceinline__ void collide_math_mrt(const Phys& ph, const C f[Q], C pc, const C pn[Q],
                                                 C fs[Q]) {
  // Eq. 4 and Eq. 5, as in collide_math
  const C rho = rho_of<C>(f);
  C jx, jy, jz;
  mom_of<C>(f, jx, jy, jz);
  C ax, ay, az, dx, dy, dz;
  link_sums<C>(pn, ax, ay, az, dx, dy, dz);
  const C w1 = (C)(1.0 / 18.0), w2 = (C)(1.0 / 36.0);
  // products through xmul / xfma: the same bits in every kernel (see
  // collide_math)
  const C gp = xmul(-(C)ph.G, pc);
  const C Fx = xmul(gp, xfma(w1, ax, xmul(w2, dx)));
  const C Fy = xmul(gp, xfma(w1, ay, xmul(w2, dy)));
  const C Fz = xmul(gp, xfma(w1, az, xmul(w2, dz)));
  // Guo's velocity
  const C inv_rho = (C)1 / rho;
  const C ux = xmul(xfma((C)0.5, Fx, jx), inv_rho);
  const C uy = xmul(xfma((C)0.5, Fy, jy), inv_rho);
  const C uz = xmul(xfma((C)0.5, Fz, jz), inv_rho);
  // moments m = M f
  C m[Q];
  mrt_forward<C>(f, m, std::make_integer_sequence<int, Q>{});
  // equilibrium and forcing moments
  const C ux2 = xmul(ux, ux), uy2 = xmul(uy, uy), uz2 = xmul(uz, uz);
  const C uu = ux2 + uy2 + uz2;
  const C uF = xfma(uz, Fz, xfma(uy, Fy, xmul(ux, Fx)));
  const C pxx = xfma((C)2, ux2, -uy2) - uz2, pww = uy2 - uz2;
  const C fyy = xmul(Fy, uy), fzz = xmul(Fz, uz);
  const C fxx = xmul((C)2, xfma((C)2, xmul(Fx, ux), -fyy) - fzz), fww = xmul((C)2, fyy - fzz);
  const C se = (C)ph.s_e, seps = (C)ph.s_eps, sq = (C)ph.s_q, spi = (C)ph.s_pi, sm = (C)ph.s_m;
  const C snu = (C)1 / (C)ph.tau;
  auto relax = [](C mk, C meq, C s, C src) {
    return xfma(xfma((C)-0.5, s, (C)1), src, xfma(-s, mk - meq, mk));
  };
  C ms[Q];
  ms[0] = rho;
  ms[3] = jx + Fx;
  ms[5] = jy + Fy;
  ms[7] = jz + Fz;
  ms[1] = relax(m[1], xmul(rho, xfma((C)19, uu, (C)-11)), se, xmul((C)38, uF));
  ms[2] = relax(m[2], xmul(rho, xfma((C)-5.5, uu, (C)3)), seps, xmul((C)-11, uF));
  const C mtwo3 = (C)(-2.0 / 3.0);
  const C mr = xmul(mtwo3, rho);
  ms[4] = relax(m[4], xmul(mr, ux), sq, xmul(mtwo3, Fx));
  ms[6] = relax(m[6], xmul(mr, uy), sq, xmul(mtwo3, Fy));
  ms[8] = relax(m[8], xmul(mr, uz), sq, xmul(mtwo3, Fz));
  const C rpxx = xmul(rho, pxx), rpww = xmul(rho, pww);
  ms[9] = relax(m[9], rpxx, snu, fxx);
  ms[10] = relax(m[10], xmul((C)-0.5, rpxx), spi, xmul((C)-0.5, fxx));
  ms[11] = relax(m[11], rpww, snu, fww);
  ms[12] = relax(m[12], xmul((C)-0.5, rpww), spi, xmul((C)-0.5, fww));
  ms[13] = relax(m[13], xmul(xmul(rho, ux), uy), snu, xfma(Fy, ux, xmul(Fx, uy)));
  ms[14] = relax(m[14], xmul(xmul(rho, uy), uz), snu, xfma(Fz, uy, xmul(Fy, uz)));
  ms[15] = relax(m[15], xmul(xmul(rho, ux), uz), snu, xfma(Fz, ux, xmul(Fx, uz)));
  ms[16] = xfma(-sm, m[16], m[16]);
  ms[17] = xfma(-sm, m[17], m[17]);
  ms[18] = xfma(-sm, m[18], m[18]);
  // f* = M^T diag(1/|row|^2) m*; the rest population takes the remainder of
  // the density so that each collision conserves mass up to one rounding
  mrt_scale<C>(ms, std::make_integer_sequence<int, Q>{});
  mrt_backward<C>(ms, fs, std::make_integer_sequence<int, Q - 1>{});
  C rest = rho;
#pragma unroll
  for (int a = 1; a < Q; ++a) rest -= fs[a];
  fs[0] = rest;
}

}  // namespace lbm
