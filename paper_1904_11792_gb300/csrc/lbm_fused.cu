// Fused time step: one kernel, one pass over the populations per step.
//
// The two-kernel step reads every population twice (the psi pass needs rho of
// every node before any collision, because the force of Eq. 5 at x needs psi
// at all 18 neighbours).  Here each block owns a 32 x 8 tile of (x, y) and a
// run of z planes.  For every plane of its tile plus a one-node halo it
// stages the 19 populations in shared memory, computes psi of that footprint,
// and collides and streams the interior of the plane below once psi of the
// plane above is known:
//
//   plane p = z0 - 1, z0, ..., z1 (periodic):  stage f(p)            (TMA)
//                                              psi(p) of the footprint -> ring
//                                              collide + stream plane p - 1
//
// Staging is Blackwell TMA: one thread issues three cp.async.bulk.tensor
// copies per plane (the 32 x 8 x 19 interior box and the two halo rows, from
// a 4-D tensor map [19][nz][ny][nx]) that complete on an mbarrier; only the
// two halo columns (periodic in x) use per-thread cp.async.  Four plane
// buffers keep two planes in flight while one is collided.  Populations leave
// DRAM once per step (halo rows and the boundary planes of a z run are read
// by neighbouring blocks at about the same time and hit L2) and psi never
// goes to DRAM.  The arithmetic is psi_math and collide_math of lbm_node.cuh,
// so the results equal the two-kernel step bitwise.  A-B streaming; lattices
// with nx % 32 == 0 and ny % 8 == 0.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <tuple>

#include "lbm_node.cuh"

namespace lbm {

namespace {

constexpr int FX = 32;   // tile along x (one warp per row)
constexpr int FY = 8;    // tile along y (eight warps)
constexpr int FZ = 16;   // z planes per block
constexpr int FT = FX * FY;
constexpr int NB = 4;    // staged planes: psi, collide, two in flight
constexpr int FH = FY + 2;
constexpr int PW = FX + 2;
constexpr long long kWaitLimit = 1ll << 22;  // bounded mbarrier polls (seconds)

__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) & ~size_t(127); }

template <int P> struct FusedShape {
  using T = typename Prec<P>::T;
  static constexpr int E = sizeof(T);
  static constexpr int U = E == 2 ? 2 : 1;               // elements per halo-column copy
  static constexpr int UNIT = U * E;                      // bytes per halo-column copy
  static constexpr size_t int_bytes = (size_t)Q * FY * FX * E;   // TMA box (32, 8, 1, 19)
  static constexpr size_t row_bytes = (size_t)Q * FX * E;        // TMA box (32, 1, 1, 19)
  static constexpr size_t col_bytes = (size_t)Q * FH * U * E;
  static constexpr size_t off_int = 0;
  static constexpr size_t off_top = align128(off_int + int_bytes);
  static constexpr size_t off_bot = align128(off_top + row_bytes);
  static constexpr size_t off_xl = align128(off_bot + row_bytes);
  static constexpr size_t off_xr = align128(off_xl + col_bytes);
  static constexpr size_t plane = align128(off_xr + col_bytes);
  static constexpr size_t off_ring = NB * plane;
  static constexpr size_t ring_bytes = align128(3ull * FH * PW * sizeof(typename Prec<P>::C));
  static constexpr size_t off_bar = off_ring + ring_bytes;
  static constexpr size_t smem = off_bar + NB * sizeof(unsigned long long);
  static constexpr unsigned tx_bytes = (unsigned)(int_bytes + 2 * row_bytes);
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_addr(smem_dst)), "l"(gmem_src),
               "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Polls the barrier at most kWaitLimit times; false if it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  for (long long it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];\n" ::"r"(smem_addr(dst)),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

template <int P>
__global__ void __launch_bounds__(FT, 2) fused_kernel(const __grid_constant__ CUtensorMap tm_int,
                                                      const __grid_constant__ CUtensorMap tm_row, Geom g,
                                                      Phys ph, const typename Prec<P>::T* src,
                                                      typename Prec<P>::T* dst, int* flag, int ntx,
                                                      int nchunks) {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  using S = FusedShape<P>;
  extern __shared__ __align__(128) unsigned char smem[];
  C* ring = reinterpret_cast<C*>(smem + S::off_ring);  // [3][FH][PW]
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem + S::off_bar);

  const int u = blockIdx.x;
  const int chunk = u % nchunks, xy = u / nchunks;
  const int x0 = (xy % ntx) * FX, y0 = (xy / ntx) * FY;
  const int z0 = chunk * FZ, z1 = min(z0 + FZ, g.nz);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long N = g.N;
  const int ym = y0 == 0 ? g.ny - 1 : y0 - 1, yp = y0 + FY == g.ny ? 0 : y0 + FY;
  const C s0 = shift_of<P>(0, ph.rho_ref), s1 = shift_of<P>(1, ph.rho_ref),
          s2 = shift_of<P>(7, ph.rho_ref);

  auto part = [&](int b, size_t off) { return reinterpret_cast<T*>(smem + b * S::plane + off); };

  if (tid == 0) {
    for (int b = 0; b < NB; ++b) mbar_init(bar + b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();

  // Stage plane p (periodic) of the footprint into buffer b.
  auto issue = [&](int p, int b) {
    const int zz = p < 0 ? p + g.nz : (p >= g.nz ? p - g.nz : p);
    if (tid == 0) {
      // order earlier generic-proxy reads of this buffer before the TMA writes
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_expect_tx(bar + b, S::tx_bytes);
      tma_load_4d(part(b, S::off_int), &tm_int, x0, y0, zz, 0, bar + b);
      tma_load_4d(part(b, S::off_top), &tm_row, x0, ym, zz, 0, bar + b);
      tma_load_4d(part(b, S::off_bot), &tm_row, x0, yp, zz, 0, bar + b);
    }
    // the two halo columns x0 - 1 and x0 + 32 (periodic), rows y0 - 1 .. y0 + 8
    for (int job = tid; job < 2 * Q * FH; job += FT) {
      const int side = job >= Q * FH;
      const int rem = job - side * Q * FH;
      const int a = rem / FH, r = rem - a * FH;
      int yy = y0 - 1 + r;
      yy = yy < 0 ? yy + g.ny : (yy >= g.ny ? yy - g.ny : yy);
      int xx = side ? x0 + FX : x0 - S::U;
      xx = xx < 0 ? xx + g.nx : (xx >= g.nx ? xx - g.nx : xx);
      T* d = part(b, side ? S::off_xr : S::off_xl) + (a * FH + r) * S::U;
      cp_async<S::UNIT>(d, src + (long long)a * N + (long long)g.nx * (yy + (long long)g.ny * zz) + xx);
    }
    cp_async_commit();
  };

  // population a of footprint cell (r, c), r in [0, FH), c in [0, PW)
  auto fp = [&](int b, int a, int r, int c) -> C {
    const C sh = a == 0 ? s0 : (a <= 6 ? s1 : s2);
    const T* q;
    if (c == 0)
      q = part(b, S::off_xl) + (a * FH + r) * S::U + (S::U - 1);
    else if (c == PW - 1)
      q = part(b, S::off_xr) + (a * FH + r) * S::U;
    else if (r == 0)
      q = part(b, S::off_top) + a * FX + c - 1;
    else if (r == FH - 1)
      q = part(b, S::off_bot) + a * FX + c - 1;
    else
      q = part(b, S::off_int) + (a * FY + r - 1) * FX + c - 1;
    return Prec<P>::load_rw(q, sh);
  };

  // psi of the footprint of the plane in buffer b into ring slot rs: the
  // interior (one cell per thread) and the 84 halo cells
  auto psi_plane = [&](int b, int rs) {
    {
      const T* q = part(b, S::off_int) + warp * FX + lane;
      C fv[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a)
        fv[a] = Prec<P>::load_rw(q + a * FY * FX, a == 0 ? s0 : (a <= 6 ? s1 : s2));
      psi_math<C>(ph, rho_of<C>(fv), ring + (rs * FH + warp + 1) * PW + lane + 1, flag);
    }
    // halo cell h = warp * 11 + lane (lane < 11): every warp takes the same
    // share of the 84 cells
    const int h = warp * 11 + lane;
    if (lane < 11 && h < 2 * FX + 2 * FH) {
      int r, c;
      if (h < FX) {
        r = 0;
        c = h + 1;
      } else if (h < 2 * FX) {
        r = FH - 1;
        c = h - FX + 1;
      } else if (h < 2 * FX + FH) {
        r = h - 2 * FX;
        c = 0;
      } else {
        r = h - 2 * FX - FH;
        c = PW - 1;
      }
      C fv[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) fv[a] = fp(b, a, r, c);
      psi_math<C>(ph, rho_of<C>(fv), ring + (rs * FH + r) * PW + c, flag);
    }
  };

  // collide + stream this thread's interior node on plane z (populations in
  // buffer fb; psi of planes z - 1, z, z + 1 in ring slots bm, bz, bp)
  auto collide_plane = [&](int z, int fb, int bm, int bz, int bp) {
    const int tx = lane, ty = warp;
    const int x = x0 + tx, y = y0 + ty;
    const T* q = part(fb, S::off_int) + ty * FX + tx;
    C f[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) f[a] = Prec<P>::load_rw(q + a * FY * FX, a == 0 ? s0 : (a <= 6 ? s1 : s2));
    const int slot[3] = {bm, bz, bp};
    C pn[Q];
    pn[0] = 0;
#pragma unroll
    for (int a = 1; a < Q; ++a)
      pn[a] = ring[(slot[cz(a) + 1] * FH + ty + 1 + cy(a)) * PW + tx + 1 + cx(a)];
    const C pc = ring[(bz * FH + ty + 1) * PW + tx + 1];
    C fs[Q];
    collide_math<C>(ph, f, pc, pn, fs);
    Nbr nb;
    nb.make(g, x, y, z);
    const unsigned seed = (Prec<P>::dev && ph.sr) ? sr_seed(nb.idx(0, 0, 0), fs[0]) : 0u;
#pragma unroll
    for (int a = 0; a < Q; ++a)
      store_pop<P>(ph, dst + (long long)a * N + nb.idx(cx(a), cy(a), cz(a)), fs[a],
                   a == 0 ? s0 : (a <= 6 ? s1 : s2), seed, a);
  };

  // planes P0 .. z1; plane P0 + k sits in buffer k % NB (barrier phase
  // k / NB) and its psi in ring slot k % 3.
  const int P0 = z0 - 1;
  const int np = (z1 - z0) + 2;
  for (int k = 0; k < NB - 1 && k < np; ++k) issue(P0 + k, k);
  for (int k = 0; k < np; ++k) {
    const int b = k % NB;
    const int ahead = np - 1 - k;
    if (ahead >= 2) cp_async_wait<2>();
    else if (ahead == 1) cp_async_wait<1>();
    else cp_async_wait<0>();
    const bool ok = mbar_wait_bounded(bar + b, (unsigned)((k / NB) & 1));
    if (__syncthreads_or(!ok)) {
      // a staged plane never arrived: report and leave after the copies
      // still in flight have had a bounded chance to land
      if (tid == 0) {
        atomicOr(flag, 2);
        for (int j = 0; j < NB; ++j) mbar_wait_bounded(bar + j, 0u);
      }
      cp_async_wait<0>();
      __syncthreads();
      return;
    }
    psi_plane(b, k % 3);
    __syncthreads();
    if (k >= 2) collide_plane(P0 + k - 1, (k - 1) % NB, (k - 2) % 3, (k - 1) % 3, k % 3);
    __syncthreads();
    if (k + NB - 1 < np) issue(P0 + k + NB - 1, (k + NB - 1) % NB);
  }
}

// ---- tensor maps ------------------------------------------------------------

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

CUtensorMapDataType tma_type(int precision) {
  switch (precision) {
    case LBM_F64: return CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    case LBM_F32: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    case LBM_F16DEV: return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    default: return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  }
}

// The 4-D view [19][nz][ny][nx] of a population array with box (32, rows, 1, 19).
cudaError_t make_map(CUtensorMap* tm, int precision, const Geom& g, const void* base, int rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const size_t e = elem_size(precision);
  const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)Q};
  const cuuint64_t strides[3] = {(cuuint64_t)g.nx * e, (cuuint64_t)g.nx * g.ny * e, (cuuint64_t)g.N * e};
  const cuuint32_t box[4] = {(cuuint32_t)FX, (cuuint32_t)rows, 1u, (cuuint32_t)Q};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  const CUresult r = fn(tm, tma_type(precision), 4, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

struct MapPair {
  CUtensorMap interior, row;
};

// Tensor maps are pure host-side descriptors; they are cached per array.
cudaError_t maps_for(int precision, const Geom& g, const void* base, MapPair* out) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int, int, int>, MapPair> cache;
  const auto key = std::make_tuple(base, precision, g.nx, g.ny, g.nz);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it == cache.end()) {
    MapPair m;
    cudaError_t e = make_map(&m.interior, precision, g, base, FY);
    if (e == cudaSuccess) e = make_map(&m.row, precision, g, base, 1);
    if (e != cudaSuccess) return e;
    it = cache.emplace(key, m).first;
  }
  *out = it->second;
  return cudaSuccess;
}

template <int P>
cudaError_t fused_t(const Geom& g, const Phys& ph, const void* src, void* dst, int* flag, cudaStream_t s) {
  using T = typename Prec<P>::T;
  using S = FusedShape<P>;
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(fused_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::smem);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  MapPair m;
  cudaError_t e = maps_for(P, g, src, &m);
  if (e != cudaSuccess) return e;
  const int ntx = g.nx / FX, nty = g.ny / FY, nchunks = (g.nz + FZ - 1) / FZ;
  const long long blocks = (long long)ntx * nty * nchunks;
  fused_kernel<P><<<(unsigned)blocks, FT, S::smem, s>>>(m.interior, m.row, g, ph, (const T*)src, (T*)dst, flag,
                                                        ntx, nchunks);
  return cudaGetLastError();
}

}  // namespace

bool fused_applicable(const Geom& g) { return g.nx % FX == 0 && g.ny % FY == 0 && g.nz >= 3; }

cudaError_t launch_fused(int precision, const Geom& g, const Phys& ph, const void* src, void* dst, int* flag,
                         cudaStream_t s) {
  if (!fused_applicable(g)) return cudaErrorInvalidValue;
  switch (precision) {
    case LBM_F64: return fused_t<LBM_F64>(g, ph, src, dst, flag, s);
    case LBM_F32: return fused_t<LBM_F32>(g, ph, src, dst, flag, s);
    case LBM_F16DEV: return fused_t<LBM_F16DEV>(g, ph, src, dst, flag, s);
    case LBM_BF16DEV: return fused_t<LBM_BF16DEV>(g, ph, src, dst, flag, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm
