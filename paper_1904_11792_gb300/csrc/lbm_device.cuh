// Device-side definitions shared by the kernels of liblbm.so: the D3Q19
// lattice, the storage-precision traits and the periodic index helper.
//
// D3Q19 (paper, section "Numerical model": 19 velocities, weights
// normalised to unity): c_0 = 0 with w = 1/3, the six +-e_i with w = 1/18,
// the twelve +-e_i +- e_j with w = 1/36, cs^2 = 1/3.  Directions are in the
// library's canonical order (rest, +x,-x,+y,-y,+z,-z, then opposite pairs of
// diagonals), so opp(a) = a + 1 for odd a and a - 1 for even a > 0.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm.h"

namespace lbm {

constexpr int Q = 19;

// Components of c_a.  Written as constexpr functions so that, inside fully
// unrolled loops over a, every use folds to an immediate.
__host__ __device__ constexpr int cx(int a) {
  return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1
         : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int a) {
  return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1
         : (a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int a) {
  return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1
         : (a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }
__host__ __device__ constexpr double wgt(int a) {
  return a == 0 ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// Stochastic rounding of the reduced-precision stores.  Round-to-nearest of
// the same value at every node of a uniform region, step after step, biases
// the stored mass in one direction; rounding up with probability equal to
// the discarded fraction removes the bias.  The random bits come from a
// counter-free hash of the node index and the bits of the node's
// post-collision rest population (which changes from step to step wherever
// the flow changes), so results stay deterministic and independent of the
// kernel variant, the streaming pattern and batching.
__device__ __forceinline__ unsigned mix32(unsigned h) {
  // integer finaliser with full avalanche (multiply-xorshift, two rounds)
  h ^= h >> 16;
  h *= 0x7feb352dU;
  h ^= h >> 15;
  h *= 0x846ca68bU;
  h ^= h >> 16;
  return h;
}
// Seed of a node's stochastic-rounding bits in one time step: the node
// index, the bits of its post-collision rest population and the step salt
// (a per-step counter; without it a node whose state no longer changes would
// round the same way every step and its rounding error would grow linearly
// in time instead of averaging out).
__device__ __forceinline__ unsigned sr_seed(long long node, float rest, unsigned salt) {
  return mix32((unsigned)node * 0x9E3779B9u ^ (unsigned)(node >> 32) ^ __float_as_uint(rest) ^
               mix32(salt + 0x6A09E667u));
}
__device__ __forceinline__ unsigned sr_seed(long long node, double rest, unsigned salt) {
  return sr_seed(node, (float)rest, salt);
}
// 32 random bits shared by the opposite directions 2j - 1 and 2j of a node
// with (well mixed) seed s (j = 1..9; j = 0: the rest population).  The
// product w = s K_j (mod 2^32) with a distinct odd constant per pair is a
// bijection of s, and its high half is well mixed: it gives the high 16 bits.
// Its low half depends on the low half of s only (the same for every pair),
// so the low 16 bits are that half xor the high one.  (The high word of the
// 64-bit product is no use here: it is uniform on [0, K_j) only.)
__device__ __forceinline__ unsigned sr_word(unsigned s, int j) {
  const unsigned w = s * (0x9E3779B1u + 0x6A09E668u * (unsigned)j);
  return w ^ (w >> 16);
}
// 16 random bits for direction a: the high half of its pair's word for odd
// a and the rest population, the low half for even a > 0 (so one conversion
// of the pair (a, a + 1), a odd, takes exactly these bits for each value).
__device__ __forceinline__ unsigned sr_bits(unsigned s, int a) {
  const unsigned w = sr_word(s, (a + 1) >> 1);
  return (a == 0 || (a & 1)) ? w >> 16 : w & 0xFFFFu;
}
// Stochastic rounding by the conversion instruction (cvt.rs, sm_100 and
// later): two FP32 values to a packed FP16 / BF16 pair, each rounded up with
// probability equal to the fraction its kept bits discard.  The first value
// goes to the high half and draws its random bits from rbits[31:16], the
// second to the low half with rbits[15:0] (checked on the GPU: unbiased, also
// for FP16 subnormals).
__device__ __forceinline__ unsigned cvt_rs_f16x2(float hi, float lo, unsigned rbits) {
  unsigned d;
  asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}
__device__ __forceinline__ unsigned cvt_rs_bf16x2(float hi, float lo, unsigned rbits) {
  unsigned d;
  asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
  return d;
}
// One value with 16 random bits r16: the low half of a pair conversion, so a
// value rounds the same alone or as the low or high half of a pair given the
// same bits.
__device__ __forceinline__ __half half_sr(float x, unsigned r16) {
  return __ushort_as_half((unsigned short)(cvt_rs_f16x2(0.0f, x, r16 & 0xFFFFu) & 0xFFFFu));
}
__device__ __forceinline__ __nv_bfloat16 bf16_sr(float x, unsigned r16) {
  return __ushort_as_bfloat16((unsigned short)(cvt_rs_bf16x2(0.0f, x, r16 & 0xFFFFu) & 0xFFFFu));
}

// Round-to-nearest product and fused multiply-add that the compiler does not
// contract or split: arithmetic written with them gives the same bits in every
// kernel that inlines it.
__device__ __forceinline__ float xmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double xmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float xfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double xfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Two FP32 lanes in one value (the nodes x and x + 1 of a thread of the
// single-pass step).  Blackwell's paired FP32 instructions (add / mul / fma
// .f32x2) compute both lanes in one issue slot, each lane rounded to nearest
// exactly like the scalar instruction, so the node arithmetic below, written
// once over C = float, double or float2, gives per lane the bits of the
// scalar form.  vadd / vsub are the plain operators on scalars (what the
// kernels always wrote); the paired difference is fma(b, -1, a), which is a
// - b rounded once.
__device__ __forceinline__ float2 xmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 xfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
// lane type, and a lane value in every lane
template <typename C> struct Lane { using S = C; };
template <> struct Lane<float2> { using S = float; };
template <typename C>
__device__ __forceinline__ C splat(typename Lane<C>::S x) {
  if constexpr (sizeof(C) == 2 * sizeof(typename Lane<C>::S))
    return make_float2(x, x);
  else
    return x;
}

// Moments of one node's populations, and the link sums of the force, in one
// fixed order shared by every kernel: opposite populations a, a + 1 (a odd)
// are combined first, then short trees, so the dependency chains are 5 adds
// deep instead of 18 and the momentum needs 21 adds instead of 30.
static_assert(cx(1) == 1 && cx(7) == 1 && cy(7) == 1 && cx(9) == 1 && cy(9) == -1 && cx(11) == 1 &&
                  cz(11) == 1 && cx(13) == 1 && cz(13) == -1 && cy(15) == 1 && cz(15) == 1 &&
                  cy(17) == 1 && cz(17) == -1 && cy(3) == 1 && cz(5) == 1,
              "direction order of the moment sums");
template <typename C>
__device__ __forceinline__ C rho_of(const C f[Q]) {
  const C s1 = vadd(f[1], f[2]), s3 = vadd(f[3], f[4]), s5 = vadd(f[5], f[6]), s7 = vadd(f[7], f[8]),
          s9 = vadd(f[9], f[10]), s11 = vadd(f[11], f[12]), s13 = vadd(f[13], f[14]), s15 = vadd(f[15], f[16]),
          s17 = vadd(f[17], f[18]);
  return vadd(vadd(vadd(f[0], s1), vadd(s3, s5)),
              vadd(vadd(vadd(s7, s9), vadd(s11, s13)), vadd(s15, s17)));
}
// Density with its rounding error, for the FP64 mass diagnostics: the same
// tree as rho_of, each add done as Knuth's error-free TwoSum (s = a + b
// rounded, e = (a - (s - (s - a))) + (b - (s - a)) exactly, in round to
// nearest), so hi equals rho_of bitwise and hi + lo is the exact sum of the
// 19 values to within the FP32 rounding of the 18 small error terms (about
// 2^-44 of rho).  The mass of FP32 and 2-byte states then reaches the FP64
// reduction without the per-node rounding of rho, which in a uniform
// region is the same at every node and does not average out.  FP64
// storage: lo = 0.
// C = float, or float2 for two nodes at once (paired instructions, each lane
// the bits of the scalar form: the paired difference is a - b rounded once).
// The scalar adds are the round-to-nearest intrinsics, which the compiler
// neither contracts nor reassociates.
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float2 radd(float2 a, float2 b) { return vadd(a, b); }
__device__ __forceinline__ float2 rsub(float2 a, float2 b) { return vsub(a, b); }
template <typename C>
__device__ __forceinline__ C two_sum(C a, C b, C& e) {
  const C s = radd(a, b);
  const C bp = rsub(s, a);
  const C ap = rsub(s, bp);
  e = radd(rsub(a, ap), rsub(b, bp));
  return s;
}
template <typename C>
__device__ __forceinline__ C rho_of_x(const C f[Q], C& lo) {
  C e[18];
  const C s1 = two_sum(f[1], f[2], e[0]), s3 = two_sum(f[3], f[4], e[1]), s5 = two_sum(f[5], f[6], e[2]),
          s7 = two_sum(f[7], f[8], e[3]), s9 = two_sum(f[9], f[10], e[4]), s11 = two_sum(f[11], f[12], e[5]),
          s13 = two_sum(f[13], f[14], e[6]), s15 = two_sum(f[15], f[16], e[7]), s17 = two_sum(f[17], f[18], e[8]);
  const C a = two_sum(two_sum(f[0], s1, e[9]), two_sum(s3, s5, e[10]), e[11]);
  const C b = two_sum(two_sum(s7, s9, e[12]), two_sum(s11, s13, e[13]), e[14]);
  const C c = two_sum(b, two_sum(s15, s17, e[15]), e[16]);
  const C hi = two_sum(a, c, e[17]);
  lo = radd(radd(radd(radd(e[0], e[1]), radd(e[2], e[3])), radd(radd(e[4], e[5]), radd(e[6], e[7]))),
            radd(radd(radd(radd(e[8], e[9]), radd(e[10], e[11])), radd(radd(e[12], e[13]), radd(e[14], e[15]))),
                 radd(e[16], e[17])));
  return hi;
}
__device__ __forceinline__ double rho_of_x(const double f[Q], double& lo) {
  lo = 0.0;
  return rho_of<double>(f);
}

// Per-thread accumulator of the FP64 diagnostics sums.  For FP32
// arithmetic it is an unevaluated FP32 pair hi + lo: each added value goes
// through TwoSum into hi, the rounding error into lo, so after n adds hi + lo
// is the exact sum to about n 2^-48 (lo's own rounding), as close as an FP64
// sum; value() hands it to the FP64 warp and block stages.  GB300's FP64
// pipe runs at about 1/64 of the FP32 rate: an FP64 conversion and add per
// value of every node made the diagnostic step of the 1024x512x512 lattice
// 6.5 ms (100 %) longer, the pair costs FP32 operations only.  FP64
// arithmetic: a plain double.
template <typename C> struct DSum;
template <> struct DSum<float> {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float x) {
    float e;
    hi = two_sum(hi, x, e);
    lo = __fadd_rn(lo, e);
  }
  // x plus a small correction (the rounding error of x itself)
  __device__ __forceinline__ void add(float x, float xlo) {
    float e;
    hi = two_sum(hi, x, e);
    lo = __fadd_rn(lo, __fadd_rn(e, xlo));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
template <> struct DSum<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ void add(double x, double xlo) { v += x + xlo; }
  __device__ __forceinline__ double value() const { return v; }
};

template <typename C>
__device__ __forceinline__ void mom_of(const C f[Q], C& jx, C& jy, C& jz) {
  const C d1 = vsub(f[1], f[2]), d3 = vsub(f[3], f[4]), d5 = vsub(f[5], f[6]), d7 = vsub(f[7], f[8]),
          d9 = vsub(f[9], f[10]), d11 = vsub(f[11], f[12]), d13 = vsub(f[13], f[14]), d15 = vsub(f[15], f[16]),
          d17 = vsub(f[17], f[18]);
  jx = vadd(vadd(d1, vadd(d7, d9)), vadd(d11, d13));
  jy = vadd(vadd(d3, vsub(d7, d9)), vadd(d15, d17));
  jz = vadd(vadd(d5, vsub(d11, d13)), vsub(d15, d17));
}
// sum over the axis links of p(x + c_a) c_a (a, b, c) and over the diagonal
// links (d, e, f): from the link differences e_a = p[a] - p[a + 1] (a odd) of
// the neighbour values p[1..18], and from those values
template <typename C>
__device__ __forceinline__ void link_combine(const C e[Q], C& ax, C& ay, C& az, C& dx, C& dy, C& dz) {
  ax = e[1];
  ay = e[3];
  az = e[5];
  dx = vadd(vadd(e[7], e[9]), vadd(e[11], e[13]));
  dy = vadd(vsub(e[7], e[9]), vadd(e[15], e[17]));
  dz = vadd(vsub(e[11], e[13]), vsub(e[15], e[17]));
}
template <typename C>
__device__ __forceinline__ void link_sums(const C p[Q], C& ax, C& ay, C& az, C& dx, C& dy, C& dz) {
  ax = vsub(p[1], p[2]);
  ay = vsub(p[3], p[4]);
  az = vsub(p[5], p[6]);
  const C e7 = vsub(p[7], p[8]), e9 = vsub(p[9], p[10]), e11 = vsub(p[11], p[12]), e13 = vsub(p[13], p[14]),
          e15 = vsub(p[15], p[16]), e17 = vsub(p[17], p[18]);
  dx = vadd(vadd(e7, e9), vadd(e11, e13));
  dy = vadd(vsub(e7, e9), vadd(e15, e17));
  dz = vadd(vsub(e11, e13), vsub(e15, e17));
}

// Storage traits.  T = stored type, C = compute type.  The *DEV forms store
// the deviation g_a = f_a - w_a rho_ref and add it back on load.  load()
// goes through the read-only data path and is only used on arrays the kernel
// does not write; load_rw() is a plain load for in-place (AA) updates.
template <int P> struct Prec;
template <> struct Prec<LBM_F64> {
  using T = double;
  using C = double;
  static constexpr bool dev = false;
  __device__ static __forceinline__ C load(const T* p, C) { return __ldg(p); }
  __device__ static __forceinline__ C load_rw(const T* p, C) { return *p; }
  __device__ static __forceinline__ void store(T* p, C v, C) { *p = v; }
  __device__ static __forceinline__ void store_sr(T* p, C v, C, unsigned) { *p = v; }
};
template <> struct Prec<LBM_F32> {
  using T = float;
  using C = float;
  static constexpr bool dev = false;
  __device__ static __forceinline__ C load(const T* p, C) { return __ldg(p); }
  __device__ static __forceinline__ C load_rw(const T* p, C) { return *p; }
  __device__ static __forceinline__ void store(T* p, C v, C) { *p = v; }
  __device__ static __forceinline__ void store_sr(T* p, C v, C, unsigned) { *p = v; }
};
template <> struct Prec<LBM_F16DEV> {
  using T = __half;
  using C = float;
  static constexpr bool dev = true;
  __device__ static __forceinline__ C load(const T* p, C shift) {
    return __half2float(__ldg(p)) + shift;
  }
  __device__ static __forceinline__ C load_rw(const T* p, C shift) {
    return __half2float(*p) + shift;
  }
  __device__ static __forceinline__ void store(T* p, C v, C shift) {
    *p = __float2half_rn(v - shift);
  }
  __device__ static __forceinline__ void store_sr(T* p, C v, C shift, unsigned r16) {
    *p = half_sr(v - shift, r16);
  }
};
template <> struct Prec<LBM_BF16DEV> {
  using T = __nv_bfloat16;
  using C = float;
  static constexpr bool dev = true;
  __device__ static __forceinline__ C load(const T* p, C shift) {
    return __bfloat162float(__ldg(p)) + shift;
  }
  __device__ static __forceinline__ C load_rw(const T* p, C shift) {
    return __bfloat162float(*p) + shift;
  }
  __device__ static __forceinline__ void store(T* p, C v, C shift) {
    *p = __float2bfloat16_rn(v - shift);
  }
  __device__ static __forceinline__ void store_sr(T* p, C v, C shift, unsigned r16) {
    *p = bf16_sr(v - shift, r16);
  }
};

// Deviation shift w_a rho_ref of population a in storage P, rounded to the
// storage precision.  With the shift on the storage grid, both the store
// (f - shift, FP32) and the reload (deviation + shift, FP32) are exact for
// the populations of liquid and vapour regions: a shift carrying all 24 bits
// of FP32 made both round, and in a nearly uniform region, where the values
// sit on a few levels, those rounding errors repeat step after step instead
// of averaging out (a uniform liquid at rest lost mass at 1.7e-7 per step in
// FP16 with stochastic rounding).
template <int P>
__device__ __forceinline__ float storage_shift(int a, double rho_ref) {
  const float v = (float)(wgt(a) * rho_ref);
  if constexpr (P == LBM_F16DEV)
    return __half2float(__float2half_rn(v));
  else if constexpr (P == LBM_BF16DEV)
    return __bfloat162float(__float2bfloat16_rn(v));
  else
    return 0.0f;
}

// Per-lattice constants handed to every kernel by value.
struct Geom {
  int nx, ny, nz;
  long long N;  // nx * ny * nz
};

struct Phys {
  double tau, G, rho0, rho_ref;
  int psi_form;
  int sr;    // stochastic rounding of reduced-precision stores (deviation forms)
  int coll;  // collision operator: COLL_SRT (the paper's) or COLL_MRT
  // MRT relaxation rates of the energy, energy-square, heat-flux, the two
  // fourth-order stress and the third-order moments (shear moments relax
  // at 1/tau)
  double s_e, s_eps, s_q, s_pi, s_m;
  // 1 / rho0 (FP32 psi multiplies by it instead of dividing by rho0: the
  // same bits for rho0 = 1, within one rounding otherwise); set by whoever
  // builds a Phys (no default member initializers: Phys stays a trivial
  // aggregate, which shared-memory copies of it need)
  double inv_rho0;
  // stochastic-rounding step salt in device memory (read at each collision);
  // nullptr reads as 0
  const unsigned* salt;
  // where the collision kernel of a step writes the next step's salt (the
  // other word of a pair; nullptr: a separate one-thread kernel advances it)
  unsigned* salt_next;
  // FP32 forms of the constants above for kernels that compute in FP32, set
  // by phys_finalize on the host whenever a Phys is built or changed: as
  // kernel parameters they sit in the constant bank and enter FP32
  // instructions as operands.  Converting the doubles in device code puts
  // each conversion on the FP64 pipe (1/64 of the FP32 rate on GB300), and
  // register-bound kernels repeat them in the step loop.  The values are
  // the device's conversions bit for bit (IEEE round to nearest on both
  // sides).
  float G_f, tau_f, omega_f;   // G, tau, 1 / tau (FP32 division)
  float rho0_f, ninv_rho0_f;   // rho0, -(1 / rho0)
  float shift_f[3];            // storage shifts of the rest, axis and diagonal classes (deviation forms)
};
enum Collision { COLL_SRT = 0, COLL_MRT = 1 };
// Sets the FP32 fields of ph from its doubles, for storage `precision`.
__host__ inline void phys_finalize(Phys& ph, int precision) {
  ph.G_f = (float)ph.G;
  ph.tau_f = (float)ph.tau;
  ph.omega_f = 1.0f / ph.tau_f;
  ph.rho0_f = (float)ph.rho0;
  ph.ninv_rho0_f = -(float)ph.inv_rho0;
  const int lead[3] = {0, 1, 7};
  for (int c = 0; c < 3; ++c) {
    const float v = (float)(wgt(lead[c]) * ph.rho_ref);
    ph.shift_f[c] = precision == LBM_F16DEV    ? __half2float(__float2half_rn(v))
                    : precision == LBM_BF16DEV ? __bfloat162float(__float2bfloat16_rn(v))
                                               : 0.0f;
  }
}
__device__ __forceinline__ unsigned salt_of(const Phys& ph) { return ph.salt ? __ldg(ph.salt) : 0u; }
// One thread of a step's collision kernel writes salt + 1 for the next step
// into the other word of the pair, which nothing of this step reads.
__device__ __forceinline__ void advance_salt(const Phys& ph) {
  if (ph.salt_next && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 &&
      threadIdx.y == 0 && threadIdx.z == 0)
    *ph.salt_next = salt_of(ph) + 1u;
}

// Neighbour index table of one node: x-1, x, x+1 and the 9 row offsets of
// (y + dy, z + dz), all periodic.  idx(cxa, cya, cza) is the flat index of
// the node x + c.  Indices within one plane are 32-bit (N < 2^31 is checked
// at creation); plane offsets a * N are formed in 64 bits by the caller.
struct Nbr {
  int xs[3];
  int rows[3][3];
  __device__ __forceinline__ void make(const Geom& g, int x, int y, int z) {
    const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
    xs[0] = xm;
    xs[1] = x;
    xs[2] = xp;
    const int yv[3] = {ym, y, yp}, zv[3] = {zm, z, zp};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) rows[i][k] = g.nx * (yv[i] + g.ny * zv[k]);
  }
  __device__ __forceinline__ int idx(int dx, int dy, int dz) const {
    return xs[dx + 1] + rows[dy + 1][dz + 1];
  }
};

// Raises *flag when any active lane of the warp has bad != 0, with at most
// one atomic per warp (a lattice that has gone non-finite everywhere must not
// serialise on the flag).
__device__ __forceinline__ void raise_flag(bool bad, int* flag) {
  const unsigned m = __ballot_sync(__activemask(), bad);
  if (m) {
    unsigned lane;
    asm("mov.u32 %0, %%laneid;" : "=r"(lane));
    // once set, later warps only read the flag
    if (lane == (unsigned)(__ffs(m) - 1) && *(volatile int*)flag == 0) atomicOr(flag, 1);
  }
}

// psi(rho) (definition after Eq. 5).
template <typename C>
__device__ __forceinline__ C psi_of(C rho, const Phys& ph) {
  if (ph.psi_form == LBM_PSI_RHO) return rho;
  if constexpr (sizeof(C) == 8) {
    return ph.rho0 * (1.0 - exp(-rho / ph.rho0));
  } else {
    // products and the difference through the non-contracted forms: the
    // bits of psi_of2 below (a product fused into 1 - e would differ)
    return __fmul_rn(ph.rho0_f, __fsub_rn(1.0f, expf(__fmul_rn(rho, ph.ninv_rho0_f))));
  }
}
// psi of two FP32 lanes: per lane the bits of psi_of<float> ((-rho) c is rho
// (-c), 1 - e is fma(e, -1, 1) rounded once)
__device__ __forceinline__ float2 psi_of2(float2 rho, const Phys& ph) {
  if (ph.psi_form == LBM_PSI_RHO) return rho;
  const float2 t = xmul(rho, splat<float2>(ph.ninv_rho0_f));
  const float2 e = make_float2(expf(t.x), expf(t.y));
  return xmul(splat<float2>(ph.rho0_f), vsub(splat<float2>(1.0f), e));
}

}  // namespace lbm
