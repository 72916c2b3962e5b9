// Single-pass time step for lattices of any size (the batched sweep).
//
// The TMA fused step (lbm_fused_kernel.cuh) needs rows of a 16-byte multiple
// and nx % 64 == 0; the ligaments of a sweep have arbitrary lengths.  This
// kernel does the same single pass with plain coalesced loads: a block owns
// a GX x GY tile of (x, y), one node per thread (a warp per row), possibly
// cut short at the lattice's edge, and marches through a run of z planes:
//
//   iteration k, plane p = z0 - 1 + k (periodic; odd runs march downwards):
//     load the 19 populations of the thread's node of plane p, rho and psi
//     -> centre of psi ring slot k % 4; threads 0 .. RINGN - 1 load one node
//     each of the tile's one-node ring of plane p -> ring
//     barrier
//     collide + stream plane p - 1 from the populations kept in registers
//     since the last iteration and psi of planes p - 2 .. p
//
// Populations leave DRAM once per step (the ring nodes and the two planes
// around a run are read by the neighbouring blocks about when they read
// them, and hit L2), psi never goes to DRAM.  The arithmetic is psi_of,
// rho_of, collide_math_r and the stores of collide_node, so every instance
// evolves bitwise as a standalone lattice of its size.  A-B streaming, the
// paper's SRT collision, any storage precision.
#pragma once

#include "lbm_node.cuh"

namespace lbm {

constexpr int GX = 32;                          // tile along x: one node per lane
constexpr int GY = 8;                           // tile along y: one warp per row
constexpr int GNT = GX * GY;
constexpr int GRX = GX + 2, GRY = GY + 2;       // tile with its one-node ring
constexpr int RINGN = 2 * GRX + 2 * GY;         // ring nodes of a plane
constexpr int GNR = 4;                          // psi ring slots
static_assert(RINGN <= GNT, "one thread per ring node");

// One lattice as the single-pass batched kernel sees it (a trivial
// aggregate: kernels copy it).
struct GInst {
  Geom g;
  Phys ph;
  long long off_f;    // element offset of the instance's first array in the pool
  int block0;         // first block of the instance
  int ntx, nty;       // tiles along x and y
  int nchunks, fz;    // z runs and their length
};

template <int P> constexpr int gfused_minb() { return P == LBM_F64 ? 1 : 2; }

// Populations of 4 and 8 bytes reach shared memory by per-thread cp.async
// copies issued two planes ahead (each thread later reads only the slots it
// copied, so no barrier guards them); 2-byte populations (no 2-byte
// cp.async) are plain loads at the plane's turn.  Either way a thread keeps
// its node's populations in registers from the psi step to the collision
// in the next iteration (re-reading them from shared memory instead was 4 %
// slower on the 48-ligament sweep: the shared-memory queue is the kernel's
// top stall).
template <int P> struct GShape {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  static constexpr bool async = sizeof(T) >= 4;
  static constexpr int NBUF = 3;                   // own populations: planes k - 1, k, k + 1
  static constexpr int RPAD = (RINGN + 31) / 32 * 32;
  static constexpr size_t own_bytes = async ? (size_t)NBUF * Q * GNT * sizeof(T) : 0;
  static constexpr size_t ring_pop_bytes = async ? (size_t)2 * Q * RPAD * sizeof(T) : 0;
  static constexpr size_t psi_bytes = (size_t)GNR * GRY * GRX * sizeof(C);
  static constexpr size_t smem = own_bytes + ring_pop_bytes + psi_bytes;
};

__device__ __forceinline__ unsigned gsmem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  static_assert(B == 4 || B == 8, "cp.async of 4 or 8 bytes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(gsmem_addr(dst)), "l"(src), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Instance of a block: largest k with block0[k] <= b.
__device__ __forceinline__ int gfind(const GInst* __restrict__ inst, int count, int b) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].block0 <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int P>
__global__ void __launch_bounds__(GNT, gfused_minb<P>())
    gfused_kernel(const GInst* __restrict__ inst, int count, typename Prec<P>::T* pool_f, int cur, int* flag) {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  using S = GShape<P>;
  extern __shared__ __align__(16) unsigned char gsm[];
  T* own = reinterpret_cast<T*>(gsm);                                  // [NBUF][Q][GNT]
  T* rpop = reinterpret_cast<T*>(gsm + S::own_bytes);                  // [2][Q][RPAD]
  C(*ring)[GRY][GRX] = reinterpret_cast<C(*)[GRY][GRX]>(gsm + S::own_bytes + S::ring_pop_bytes);

  const GInst& I = inst[gfind(inst, count, blockIdx.x)];
  const Geom g = I.g;
  const Phys ph = I.ph;
  const long long N = g.N;
  const T* src = pool_f + I.off_f + (long long)cur * Q * N;
  T* dst = pool_f + I.off_f + (long long)(cur ^ 1) * Q * N;
  // block -> (z run, tile x, tile y), the run fastest: the runs of a tile and
  // the tiles of a row of tiles are launched together and share planes and
  // ring rows in L2
  const int u = blockIdx.x - I.block0;
  const int chunk = u % I.nchunks, xy = u / I.nchunks;
  const int x0 = (xy % I.ntx) * GX, y0 = (xy / I.ntx) * GY;
  const int w = min(GX, g.nx - x0), h = min(GY, g.ny - y0);   // tile extent (cut at the edge)
  const int z0 = chunk * I.fz, z1 = min(z0 + I.fz, g.nz);
  const int np = (z1 - z0) + 2;
  const int dir = (chunk & 1) ? -1 : 1;
  const int tid = threadIdx.x, lane = tid & 31, wy = tid >> 5;
  auto zwrap = [&](int p) { return p < 0 ? p + g.nz : (p >= g.nz ? p - g.nz : p); };
  auto zplane = [&](int k) { return zwrap(dir > 0 ? z0 - 1 + k : z1 - k); };
  auto xwrap = [&](int x) { return x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x); };
  auto ywrap = [&](int y) { return y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y); };

  // this thread's node (interior) and ring node
  const bool act = lane < w && wy < h;
  const int x = x0 + lane, y = y0 + wy;
  int rx = -1, ry = -1;
  if (tid < 2 * GRX) {                         // the rows y0 - 1 and y0 + h
    rx = tid % GRX;
    ry = tid < GRX ? 0 : h + 1;
    if (rx > w + 1) rx = -1;
  } else if (tid < RINGN) {                    // the columns x0 - 1 and x0 + w
    const int r = tid - 2 * GRX;
    ry = 1 + r % GY;
    rx = r < GY ? 0 : w + 1;
    if (ry > h) rx = -1;
  }
  const bool ract = rx >= 0;
  const int rxg = ract ? xwrap(x0 - 1 + rx) : 0, ryg = ract ? ywrap(y0 - 1 + ry) : 0;
  const int rrow = rxg + g.nx * ryg;           // in-plane index of the ring node, less the plane
  const int orow = x + g.nx * y;               // in-plane index of the own node, less the plane
  const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x + 1 == g.nx ? 0 : x + 1;
  const int yv[3] = {y == 0 ? g.ny - 1 : y - 1, y, y + 1 == g.ny ? 0 : y + 1};
  const int xs[3] = {xm, x, xp};

  const C s0 = shift_of<P>(0, ph.rho_ref), s1 = shift_of<P>(1, ph.rho_ref), s2 = shift_of<P>(7, ph.rho_ref);
  auto shift = [&](int a) { return a == 0 ? s0 : (a <= 6 ? s1 : s2); };
  const unsigned salt = (Prec<P>::dev && ph.sr) ? salt_of(ph) : 0u;
  const long long plane_n = (long long)g.nx * g.ny;

  // copies of plane zplane(k) (own node into buffer k % 3, ring node into
  // ring buffer k % 2), one commit group per plane, empty past the run
  auto issue = [&](int k) {
    if constexpr (S::async) {
      if (k < np) {
        const long long zo = plane_n * zplane(k);
        if (act) {
          T* d = own + (size_t)(k % S::NBUF) * Q * GNT + tid;
#pragma unroll
          for (int a = 0; a < Q; ++a) cp_async<sizeof(T)>(d + a * GNT, src + (long long)a * N + zo + orow);
        }
        if (ract) {
          T* d = rpop + (size_t)(k % 2) * Q * S::RPAD + tid;
#pragma unroll
          for (int a = 0; a < Q; ++a) cp_async<sizeof(T)>(d + a * S::RPAD, src + (long long)a * N + zo + rrow);
        }
      }
      cp_async_commit();
    }
  };
  issue(0);
  issue(1);

  bool nbad = false;
  C prev[Q], prho = 0;
  for (int k = 0; k < np; ++k) {
    const int zk = zplane(k);
    C(*slot)[GRX] = ring[k % GNR];
    C f[Q];
    C rho = 0;
    if constexpr (S::async) cp_async_wait_one();   // this thread's copies of plane k have landed
    if (act) {
      if constexpr (S::async) {
        const T* o = own + (size_t)(k % S::NBUF) * Q * GNT + tid;
#pragma unroll
        for (int a = 0; a < Q; ++a) f[a] = (C)o[a * GNT];
      } else {
        const long long i = orow + plane_n * zk;
#pragma unroll
        for (int a = 0; a < Q; ++a) f[a] = Prec<P>::load(src + (long long)a * N + i, shift(a));
      }
      rho = rho_of<C>(f);
      nbad |= bad_rho(rho);
      slot[wy + 1][lane + 1] = psi_of<C>(rho, ph);
    }
    if (ract) {
      C fr[Q];
      if constexpr (S::async) {
        const T* o = rpop + (size_t)(k % 2) * Q * S::RPAD + tid;
#pragma unroll
        for (int a = 0; a < Q; ++a) fr[a] = (C)o[a * S::RPAD];
      } else {
        const long long i = rrow + plane_n * zk;
#pragma unroll
        for (int a = 0; a < Q; ++a) fr[a] = Prec<P>::load(src + (long long)a * N + i, shift(a));
      }
      const C rr = rho_of<C>(fr);
      nbad |= bad_rho(rr);
      slot[ry][rx] = psi_of<C>(rr, ph);
    }
    // every psi of plane zk is in the ring
    __syncthreads();
    if (k >= 2 && act) {
      // collide + stream this thread's node of plane z = zplane(k - 1); plane
      // z + dz sits in ring slot (k - 1 + dir dz) % 4
      const int z = zplane(k - 1);
      const int zv[3] = {z == 0 ? g.nz - 1 : z - 1, z, z + 1 == g.nz ? 0 : z + 1};
      C fp[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) fp[a] = prev[a];
      C pn[Q];
      pn[0] = 0;
#pragma unroll
      for (int a = 1; a < Q; ++a) pn[a] = ring[(k - 1 + dir * cz(a) + GNR) % GNR][wy + 1 + cy(a)][lane + 1 + cx(a)];
      const C pc = ring[(k - 1) % GNR][wy + 1][lane + 1];
      C fs[Q];
      collide_math_r<C>(ph, fp, prho, pc, pn, fs);
      const int i = x + g.nx * (y + g.ny * z);
      const unsigned seed = (Prec<P>::dev && ph.sr) ? sr_seed(i, fs[0], salt) : 0u;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const int d = xs[1 + cx(a)] + g.nx * (yv[1 + cy(a)] + g.ny * zv[1 + cz(a)]);
        store_pop<P>(ph, dst + (long long)a * N + d, fs[a], shift(a), seed, a);
      }
    }
    // the buffers of plane k - 1 (own) and k (ring) are read out by this
    // thread: plane k + 2 goes there
    issue(k + 2);
    if (act) {
#pragma unroll
      for (int a = 0; a < Q; ++a) prev[a] = f[a];
      prho = rho;
    }
  }
  raise_flag(nbad, flag);
}


// ---------------------------------------------------------------------------
// Bulk-copy form (4- and 2-byte storage), the batch's default for them.
//
// The per-element copies above put ~88 shared- and global-memory operations
// on every node (the shared-memory queue and the barrier bound them at 53 %
// of HBM).  Here a block owns a 64 x 4 tile (two nodes per thread, as the
// TMA fused step) and a plane reaches shared memory as one 1-D bulk copy
// (cp.async.bulk, completing on the buffer's mbarrier) per direction and
// tile row (the tile's rows and its two halo rows): a bulk copy must start
// on a 16-byte boundary, so each copy starts at the boundary at or below the
// row's element x0 - 1 and is BW elements long, and a reader finds element x
// of that row at x - x0 + 1 + (the start's remainder).  Where the halo column
// wraps around the lattice (x0 = 0 on the left, x0 + w = nx on the right)
// its element comes from a separate 16-byte copy.  The pool of a batch has
// kBulkPad elements of padding before and after its arrays, so a copy's
// rounded-down start and its full length stay inside the allocation.  The
// rest follows the TMA fused step: psi of the tile and its one-node ring into
// a four-plane psi ring, one barrier per plane, the collision of the plane
// below from registers, odd runs marching downwards, waits bounded in time.
// ---------------------------------------------------------------------------
constexpr int BX = 64, BY = 4, BNT = 32 * BY;   // tile (two nodes per lane, one warp per row), threads
constexpr int BRH = BY + 2;                     // rows copied per direction: the tile's and its two halo rows
constexpr int BRW = BX + 4;                     // psi ring row: position x - x0 + 2 (pairs 8-byte aligned)
constexpr int BNB = 2;                          // plane buffers
constexpr int BNR = 4;                          // psi ring slots
constexpr int kBulkPad = 128;                   // pool padding before and after the arrays, elements
constexpr unsigned long long kBulkWaitNs = 2000000000ull;   // a wait on a plane gives up after 2 s

__host__ __device__ constexpr size_t bal128(size_t b) { return (b + 127) & ~size_t(127); }

template <int P> struct BShape {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  static constexpr int E = sizeof(T);
  static constexpr int CW = 16 / E;                                  // elements per 16 bytes
  static constexpr int BW = (BX + 2 + CW - 1 + CW - 1) / CW * CW;     // copy length: x0 - 1 .. x0 + 64 and the remainder
  static_assert(BW <= kBulkPad, "padding covers a copy");
  static constexpr size_t main_bytes = (size_t)Q * BRH * BW * E;     // [a][row][BW]
  static constexpr size_t side_bytes = (size_t)Q * BRH * 2 * CW * E; // [a][row][left/right][CW]
  static constexpr size_t buf = bal128(main_bytes + side_bytes);
  static constexpr size_t off_ring = BNB * buf;
  static constexpr size_t ring_bytes = bal128((size_t)BNR * BRH * BRW * sizeof(C));
  static constexpr size_t off_bar = off_ring + ring_bytes;
  static constexpr size_t smem = off_bar + BNB * sizeof(unsigned long long);
};

__device__ __forceinline__ void gb_mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(gsmem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void gb_mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(gsmem_addr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool gb_mbar_try(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(gsmem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gb_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Polls until the barrier's phase completes or limit_ns of wall time pass.
__device__ __forceinline__ bool gb_mbar_wait(unsigned long long* bar, unsigned parity) {
  if (gb_mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gb_ns();
  for (;;) {
    if (gb_mbar_try(bar, parity)) return true;
    if (gb_ns() - t0 > kBulkWaitNs) return false;
  }
}
// 1-D bulk copy of `bytes` (a multiple of 16) from a 16-byte aligned global
// address to a 16-byte aligned shared address, completing on `bar`.
__device__ __forceinline__ void gb_bulk(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   gsmem_addr(dst)),
               "l"(src), "r"(bytes), "r"(gsmem_addr(bar))
               : "memory");
}

template <int P>
__global__ void __launch_bounds__(BNT, Prec<P>::dev ? 3 : 2)
    gbulk_kernel(const GInst* __restrict__ inst, int count, typename Prec<P>::T* pool_f, int cur, int* flag) {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  using V = typename Pair<P>::V;
  using S = BShape<P>;
  static_assert(P != LBM_F64, "bulk-copy form for 4- and 2-byte storage");
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + S::off_bar);
  C* ring = reinterpret_cast<C*>(smem + S::off_ring);

  const GInst& I = inst[gfind(inst, count, blockIdx.x)];
  const Geom g = I.g;
  const Phys ph = I.ph;
  const long long N = g.N;
  const long long sbase = I.off_f + (long long)cur * Q * N;          // source array, element index in the pool
  const long long dbase = I.off_f + (long long)(cur ^ 1) * Q * N;    // destination array
  T* dst = pool_f + dbase;
  const int u = blockIdx.x - I.block0;
  const int chunk = u % I.nchunks, xy = u / I.nchunks;
  const int x0 = (xy % I.ntx) * BX, y0 = (xy / I.ntx) * BY;
  const int w = min(BX, g.nx - x0), h = min(BY, g.ny - y0);          // tile extent (cut at the edges)
  const bool ledge = x0 == 0, redge = x0 + w == g.nx;               // halo columns that wrap around
  const int z0 = chunk * I.fz, z1 = min(z0 + I.fz, g.nz);
  const int np = (z1 - z0) + 2;
  const int dir = (chunk & 1) ? -1 : 1;
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  auto zwrap = [&](int p) { return p < 0 ? p + g.nz : (p >= g.nz ? p - g.nz : p); };
  auto zplane = [&](int k) { return zwrap(dir > 0 ? z0 - 1 + k : z1 - k); };
  auto ywrap = [&](int y) { return y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y); };
  constexpr unsigned CM = S::CW - 1;

  // copies: thread t < Q (h + 2) issues direction t / (h + 2), row t % (h + 2)
  const int nrows = h + 2;
  const bool copier = tid < Q * nrows;
  const int ca = copier ? tid / nrows : 0, cr = copier ? tid % nrows : 0;
  const long long crow = (long long)ca * N + (long long)ywrap(y0 - 1 + cr) * g.nx;   // less the plane
  const unsigned plane_bytes =
      (unsigned)(nrows * Q) * (unsigned)(S::BW * S::E + ((ledge ? 1 : 0) + (redge ? 1 : 0)) * 16);
  auto issue = [&](int k) {
    if (copier) {
      unsigned char* b = smem + (size_t)(k % BNB) * S::buf;
      const long long rowbase = sbase + crow + (long long)zplane(k) * g.ny * g.nx;
      const long long start = rowbase + x0 - 1;
      const long long e0 = start & ~(long long)CM;
      // earlier generic-proxy reads of this buffer come before the async writes
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      gb_bulk(b + (size_t)(ca * BRH + cr) * S::BW * S::E, pool_f + e0, S::BW * S::E, full + (k % BNB));
      T* side = reinterpret_cast<T*>(b + S::main_bytes) + (size_t)(ca * BRH + cr) * 2 * S::CW;
      if (ledge) gb_bulk(side, pool_f + ((rowbase + g.nx - 1) & ~(long long)CM), 16, full + (k % BNB));
      if (redge) gb_bulk(side + S::CW, pool_f + (rowbase & ~(long long)CM), 16, full + (k % BNB));
    }
  };
  // element x (x0 - 1 <= x <= x0 + w) of direction a, tile row r (0 .. h + 1) of
  // the plane in buffer b; rrow = element index of (a = 0, row r, x = 0)
  auto elem = [&](const unsigned char* b, int a, int r, long long rrow, int x) -> T {
    const unsigned rb = (unsigned)rrow + (unsigned)a * (unsigned)N;     // low bits of the row's base
    const T* side = reinterpret_cast<const T*>(b + S::main_bytes) + (size_t)(a * BRH + r) * 2 * S::CW;
    if (x < x0 && ledge) return side[(rb + g.nx - 1) & CM];
    if (x >= x0 + w && redge) return side[S::CW + (rb & CM)];
    const T* m = reinterpret_cast<const T*>(b) + (size_t)(a * BRH + r) * S::BW;
    return m[x - x0 + 1 + ((rb + x0 - 1) & CM)];
  };

  __shared__ int s_abort;
  if (tid == 0) {
    s_abort = (*(volatile int*)flag & 2) != 0;   // a wait of an earlier launch gave up: skip the work
    for (int b = 0; b < BNB; ++b) gb_mbar_init(full + b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (s_abort) return;
  if (tid == 0)
    for (int k = 0; k < BNB && k < np; ++k) gb_mbar_expect(full + k, plane_bytes);
  __syncthreads();
  for (int k = 0; k < BNB && k < np; ++k) issue(k);

  // this thread's nodes x0 + 2 lane, + 1 of row y0 + ty
  const int x = x0 + 2 * lane, y = y0 + ty;
  const bool v0 = 2 * lane < w && ty < h, v1 = 2 * lane + 1 < w && ty < h;
  // halo cells (as the TMA fused step): warps 0 and 1 the rows y0 - 1 and
  // y0 + h as node pairs over x0 .. x0 + 63, warp 2 the four corners and the
  // 2 h column cells, one per lane
  const int hrow = ty == 0 ? 0 : h + 1;
  int sx = 0, sr = -1;   // scalar halo cell: x and tile row
  if (ty == 2 && lane < 4 + 2 * h) {
    if (lane < 4) {
      sx = (lane & 1) ? x0 + w : x0 - 1;
      sr = (lane >> 1) ? h + 1 : 0;
    } else {
      const int i = lane - 4, side = i >= h;
      sx = side ? x0 + w : x0 - 1;
      sr = 1 + (side ? i - h : i);
    }
  }
  const C s0 = shift_of<P>(0, ph.rho_ref), s1 = shift_of<P>(1, ph.rho_ref), s2 = shift_of<P>(7, ph.rho_ref);
  auto shift = [&](int a) { return a == 0 ? s0 : (a <= 6 ? s1 : s2); };
  auto widen = [&](T t, int a) -> C {
    if constexpr (Prec<P>::dev) return (C)(float)t + shift(a);
    else return (C)t;
  };
  const unsigned salt = (Prec<P>::dev && ph.sr) ? salt_of(ph) : 0u;
  const long long plane_n = (long long)g.nx * g.ny;
  const int xm = x == 0 ? g.nx - 1 : x - 1, xp1 = x + 1 == g.nx ? 0 : x + 1, xp2 = x + 2 >= g.nx ? x + 2 - g.nx : x + 2;
  const int yv[3] = {y == 0 ? g.ny - 1 : y - 1, y, y + 1 == g.ny ? 0 : y + 1};

  bool nbad = false;
  C prev0[Q], prev1[Q], prho0 = 0, prho1 = 0;
  int k = 0;
  for (; k < np; ++k) {
    const int b = k % BNB;
    const bool ok = gb_mbar_wait(full + b, (unsigned)((k / BNB) & 1));
    const unsigned char* buf = smem + (size_t)b * S::buf;
    const long long zoff = sbase + (long long)zplane(k) * plane_n;   // element index of (a = 0, plane, row 0, x 0)
    C* slot = ring + (k % BNR) * BRH * BRW;
    // psi of this thread's two nodes
    C f0[Q], f1[Q];
    const long long orow = zoff + (long long)y * g.nx;
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      f0[a] = widen(elem(buf, a, ty + 1, orow, x), a);
      f1[a] = widen(elem(buf, a, ty + 1, orow, x + 1), a);
    }
    const C r0 = rho_of<C>(f0), r1 = rho_of<C>(f1);
    if (v0) nbad |= bad_rho(r0);
    if (v1) nbad |= bad_rho(r1);
    // positions past the tile's edge belong to the halo column and corner
    // cells (written below by warp 2): only this thread's valid nodes write
    if (v0) slot[(ty + 1) * BRW + 2 * lane + 2] = psi_of<C>(r0, ph);
    if (v1) slot[(ty + 1) * BRW + 2 * lane + 3] = psi_of<C>(r1, ph);
    // psi of this thread's halo cells
    if (ty < 2) {
      const long long hr = zoff + (long long)ywrap(y0 - 1 + hrow) * g.nx;
      C fa[Q], fb[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        fa[a] = widen(elem(buf, a, hrow, hr, x), a);
        fb[a] = widen(elem(buf, a, hrow, hr, x + 1), a);
      }
      const C ra = rho_of<C>(fa), rb = rho_of<C>(fb);
      if (2 * lane < w) nbad |= bad_rho(ra);
      if (2 * lane + 1 < w) nbad |= bad_rho(rb);
      if (2 * lane < w) slot[hrow * BRW + 2 * lane + 2] = psi_of<C>(ra, ph);
      if (2 * lane + 1 < w) slot[hrow * BRW + 2 * lane + 3] = psi_of<C>(rb, ph);
    } else if (sr >= 0) {
      const long long hr = zoff + (long long)ywrap(y0 - 1 + sr) * g.nx;
      C fv[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) fv[a] = widen(elem(buf, a, sr, hr, sx), a);
      const C rv = rho_of<C>(fv);
      nbad |= bad_rho(rv);
      slot[sr * BRW + (sx - x0 + 2)] = psi_of<C>(rv, ph);
    }
    if (tid == 0 && k + BNB < np) gb_mbar_expect(full + b, plane_bytes);   // before any copy into b
    // every psi of plane zplane(k) is in the ring and buffer b is read out
    if (__syncthreads_or(!ok)) break;
    if (k + BNB < np) issue(k + BNB);

    if (k >= 2 && (v0 || v1)) {
      // collide + stream the nodes of plane z = zplane(k - 1); plane z + dz
      // has march index k - 1 + dir dz
      const int z = zplane(k - 1);
      const int zv[3] = {z == 0 ? g.nz - 1 : z - 1, z, z == g.nz - 1 ? 0 : z + 1};
      C q[3][3][4];
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
          const C* row = ring + ((k - 1 + dir * dz) % BNR) * BRH * BRW + (ty + 1 + dy) * BRW + 2 * lane + 2;
#pragma unroll
          for (int c = 0; c < 4; ++c) q[dy + 1][dz + 1][c] = (dy == 0 || dz == 0 || (c == 1 || c == 2)) ? row[c - 1] : (C)0;
        }
      C pn0[Q], pn1[Q];
      pn0[0] = pn1[0] = 0;
#pragma unroll
      for (int a = 1; a < Q; ++a) {
        pn0[a] = q[cy(a) + 1][cz(a) + 1][1 + cx(a)];
        pn1[a] = q[cy(a) + 1][cz(a) + 1][2 + cx(a)];
      }
      C fs0[Q], fs1[Q];
      collide_math_r<C>(ph, prev0, prho0, q[1][1][1], pn0, fs0);
      collide_math_r<C>(ph, prev1, prho1, q[1][1][2], pn1, fs1);
      const int i0 = x + g.nx * (y + g.ny * z);
      const bool srd = Prec<P>::dev && ph.sr;
      const unsigned seed0 = srd ? sr_seed(i0, fs0[0], salt) : 0u;
      const unsigned seed1 = srd ? sr_seed(i0 + 1, fs1[0], salt) : 0u;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const C sh = shift(a);
        const long long row = (long long)a * N + (long long)g.nx * (yv[1 + cy(a)] + g.ny * zv[1 + cz(a)]);
        if (cx(a) == 0 && v1 && (((unsigned)dbase + (unsigned)row + (unsigned)x) & 1u) == 0) {
          // both nodes, an aligned pair: one vector store
          if (srd)
            store_pair_sr<P>(dst + row + x, fs0[a], fs1[a], sh, sr_bits(seed0, a), sr_bits(seed1, a));
          else
            store_pair<P>(dst + row + x, fs0[a], fs1[a], sh);
        } else {
          const int t0 = cx(a) > 0 ? xp1 : (cx(a) < 0 ? xm : x);
          const int t1 = cx(a) > 0 ? xp2 : (cx(a) < 0 ? x : xp1);
          if (v0) store_pop<P>(ph, dst + row + t0, fs0[a], sh, seed0, a);
          if (v1) store_pop<P>(ph, dst + row + t1, fs1[a], sh, seed1, a);
        }
      }
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      prev0[a] = f0[a];
      prev1[a] = f1[a];
    }
    prho0 = r0;
    prho1 = r1;
  }
  raise_flag(nbad, flag);
  if (k < np && tid == 0) {
    // a wait gave up: record it, and let the copies already issued land
    // before the block's shared memory is released
    atomicOr(flag, 2);
    for (int j = k; j < k + BNB && j < np; ++j) gb_mbar_wait(full + j % BNB, (unsigned)((j / BNB) & 1));
  }
}

}  // namespace lbm
