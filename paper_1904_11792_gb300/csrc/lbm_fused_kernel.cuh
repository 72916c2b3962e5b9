// Fused time step: one kernel, one pass over the populations per step.
//
// The two-kernel step reads every population twice (the psi pass needs rho of
// every node before any collision, because the force of Eq. 5 at x needs psi
// at all 18 neighbours).  Here a block owns a 64 x TY tile of (x, y) (32
// lanes x two nodes per row, one warp per row) and a run of z planes, and
// marches through the run:
//
//   iteration k, plane p = z0 - 1 + k (periodic; odd runs march downwards):
//     psi of plane p over the tile and its one-node ring  -> psi ring slot
//     barrier
//     collide + stream plane p - 1 (psi of planes p - 2 .. p now known)
//
// Populations reach shared memory by Blackwell TMA: per plane nine
// cp.async.bulk.tensor copies from 4-D tensor maps [19][nz][ny][nx] (the
// 64 x TY interior, the two halo rows, the two halo columns and the four
// corners as 16-byte wide boxes, every box at in-range coordinates so the
// periodic wrap needs no fill), completing on the buffer's mbarrier.  Two
// plane buffers: the copies of plane p + 2 start as soon as psi of plane p
// has been read out of its buffer, a full iteration ahead.  A thread keeps
// the stored populations of its two nodes in registers from the psi step of
// plane p to their collision in the next iteration, so a buffer is free
// after the psi step.  The psi values of four planes sit in a ring (the
// collision of plane p - 1 reads slots p - 2 .. p while faster warps already
// write p + 1), so one block barrier per plane suffices.  Populations leave
// DRAM once per step (halo boxes and the two boundary planes of a run are
// read by neighbouring blocks at about the same time and mostly hit L2),
// psi never goes to DRAM.  The arithmetic is psi_of and collide_math of
// lbm_node.cuh, computed for the thread's two nodes at once in paired FP32
// instructions (float2 lanes, each rounded like the scalar instruction), and
// the stores are those of collide_pair, so the results equal the two-kernel
// step bitwise.  A-B streaming, 4- and 2-byte storage, lattices with
// nx % 64 == 0 and ny % 4 == 0 (8 for 2-byte storage); bfused_kernel runs
// the same body over the instances of a batch, of any size, whose rows the
// batch pads to 16-byte multiples, on 64-wide tiles or on 32-wide ones (two
// rows of 16 lanes x two nodes per warp, twice as many rows per tile).
//
// This header holds the kernel and its device helpers; lbm_fused.cu holds
// the host side (tensor maps, launch shape, launches).  Include it from one
// translation unit only: its definitions have internal linkage.
#pragma once

#include <cuda.h>

#include "lbm_node.cuh"

namespace lbm {

namespace {

constexpr int TX = 64;   // tile along x: 32 lanes x 2 nodes
constexpr int NB = 2;    // plane buffers
constexpr int NR = 4;    // psi ring slots
constexpr unsigned long long kWaitNs = 2000000000ull;   // a wait on a plane gives up after 2 s

__host__ __device__ constexpr size_t align128(size_t b) { return (b + 127) & ~size_t(127); }

// Tile rows (one warp each): 4 for 4-byte storage, 8 for 2-byte storage,
// whose smaller plane buffers leave room for the taller tile (less halo psi
// per node: the ring of a 64 x 8 tile is 148 nodes for 512, of a 64 x 4 tile
// 140 for 256; and the three warps of halo work are three of eight instead
// of three of four, which the per-plane barrier waited for).
// W = 32 (the batched step's tiles, of lattices of any length, which waste
// fewer lanes at their x ends): a warp takes two rows of 16 lanes x 2 nodes,
// so the same threads cover a 32 x 8 (FP32) or 32 x 16 (2-byte) tile.
template <int P, int W = TX> struct FusedShape {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  static_assert(W == 64 || W == 32, "tiles 64 or 32 nodes wide");
  static constexpr int TXW = W;                     // tile along x
  static constexpr int NT = 32 * (Prec<P>::dev ? 8 : 4);
  static constexpr int TY = W == 64 ? NT / 32 : 2 * (NT / 32);   // tile along y: one (W 64) or two rows per warp
  static constexpr int RWW = W + 4;                 // ring row: position x - x0 + 2 (pairs start 8-byte aligned)
  static constexpr int RH = TY + 2;                 // psi ring rows
  static constexpr int E = sizeof(T);
  static constexpr int CW = 16 / E;                               // one 16-byte TMA unit along x
  static constexpr size_t int_bytes = (size_t)Q * TY * W * E;     // box (W, TY, 1, 19)
  static constexpr size_t row_bytes = (size_t)Q * W * E;          // box (W, 1, 1, 19)
  static constexpr size_t col_bytes = (size_t)Q * TY * CW * E;    // box (CW, TY, 1, 19)
  static constexpr size_t cor_bytes = (size_t)Q * CW * E;         // box (CW, 1, 1, 19)
  static constexpr size_t off_int = 0;
  static constexpr size_t off_top = align128(off_int + int_bytes);
  static constexpr size_t off_bot = align128(off_top + row_bytes);
  static constexpr size_t off_lft = align128(off_bot + row_bytes);
  static constexpr size_t off_rgt = align128(off_lft + col_bytes);
  static constexpr size_t off_cor = align128(off_rgt + col_bytes);  // 4 corners, cor_stride apart
  static constexpr size_t cor_stride = align128(cor_bytes);
  static constexpr size_t plane = align128(off_cor + 4 * cor_stride);
  static constexpr size_t off_ring = NB * plane;
  static constexpr size_t ring_bytes = align128((size_t)NR * RH * RWW * sizeof(C));
  static constexpr size_t off_bar = off_ring + ring_bytes;
  static constexpr size_t smem = off_bar + (NB + 1) * sizeof(unsigned long long);   // + the test barrier
  static constexpr unsigned tx_bytes = (unsigned)(int_bytes + 2 * row_bytes + 2 * col_bytes + 4 * cor_bytes);
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

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
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Polls the barrier until its phase completes or limit_ns of wall time have
// passed (the global nanosecond timer); false if it did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned long long limit_ns = kWaitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];\n" ::"r"(smem_addr(dst)),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(0), "r"(smem_addr(bar))
      : "memory");
}

struct Maps {
  CUtensorMap interior, row, col, cor;
};

// Start of each direction's slab in the destination array (dst + a N) of
// the single-lattice step, set by the host: a kernel parameter, so the
// store address arithmetic takes each base from the constant bank (the
// batched step, whose destination depends on the block's instance, keeps
// them in shared memory).
template <typename T> struct DirBases {
  T* p[Q];
};

// Issues the nine copies of plane zz into buffer b (one thread).
template <int P, int W = TX>
__device__ __forceinline__ void issue_plane(unsigned char* smem, const Maps& m, int b, int x0, int y0, int xl,
                                            int xr, int ym, int yp, int zz, unsigned long long* bar) {
  using S = FusedShape<P, W>;
  unsigned char* base = smem + (size_t)b * S::plane;
  // order earlier generic-proxy reads of this buffer before the async writes
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  mbar_expect_tx(bar, S::tx_bytes);
  tma_load_4d(base + S::off_int, &m.interior, x0, y0, zz, bar);
  tma_load_4d(base + S::off_top, &m.row, x0, ym, zz, bar);
  tma_load_4d(base + S::off_bot, &m.row, x0, yp, zz, bar);
  tma_load_4d(base + S::off_lft, &m.col, xl, y0, zz, bar);
  tma_load_4d(base + S::off_rgt, &m.col, xr, y0, zz, bar);
  tma_load_4d(base + S::off_cor + 0 * S::cor_stride, &m.cor, xl, ym, zz, bar);
  tma_load_4d(base + S::off_cor + 1 * S::cor_stride, &m.cor, xr, ym, zz, bar);
  tma_load_4d(base + S::off_cor + 2 * S::cor_stride, &m.cor, xl, yp, zz, bar);
  tma_load_4d(base + S::off_cor + 3 * S::cor_stride, &m.cor, xr, yp, zz, bar);
}

// Diagnostics of the step's starting state, reduced in the same pass (DIAG):
// every thread sums the nodes of the planes its block owns (the run z0 ..
// z1 - 1, not the two halo planes): each node's momentum, liquid fraction
// and density (with its rounding error, rho_of_x) into DSum accumulators
// (exact to FP64 level), then an FP64 warp shuffle tree and FP64 block
// sums; the block writes FP64 partials in the layout the diagnostics
// reduction reads: slice sums [row block][x][2] with one row block per
// (tile row, z run), and block totals [block][DIAG_NG].
struct DiagOut {
  double rho_l, rho_v;
  double* slices;
  double* blocks;
  // test hook (the timeout path of the bounded waits): > 0 makes every block
  // also wait, for at most this many ns, on a barrier nothing completes
  unsigned long long stall_test_ns;
  // the liquid threshold (rho_l + rho_v) / 2, 1 / (rho_l - rho_v) and rho_v in
  // FP32, computed on the host (diag_out): derived in device code they cost
  // FP64-pipe operations (a division among them), which the register-bound
  // diagnostic step repeated in its plane loop
  float thr_f, inv_f, rv_f;
};
// DiagOut with its FP32 thresholds (host).
__host__ inline DiagOut diag_out(double rho_l, double rho_v, double* slices, double* blocks,
                                 unsigned long long stall_test_ns) {
  // the device's own FP64 expressions, bit for bit (IEEE on both sides)
  return DiagOut{rho_l, rho_v, slices, blocks, stall_test_ns, (float)(0.5 * (rho_l + rho_v)),
                 (float)(1.0 / (rho_l - rho_v)), (float)rho_v};
}

// Blocks per SM the register budget must allow: 3 of 128 threads for 4-byte
// storage (its 73 KB of shared memory allow no more), 2 of 256 threads for
// 2-byte storage (71 KB each), the diagnostic variants included (no spills
// at 168 and 128 registers).
template <int P, bool DIAG, int COLL = COLL_SRT>
constexpr int fused_minb() {
  return Prec<P>::dev ? 2 : 3;
}

// The step of one block: work item u of a lattice (a tile and z run) among
// tiles of ntx columns, tensor maps `maps` of its source array, destination
// array dst with rows of px elements and dstride elements per direction.
// BATCH: the lattice is an
// instance of the batched sweep of any size - tiles are cut at its x and y
// edges (the tensor maps read zeros past them, and nodes there neither
// store nor write psi), its rows are padded to a 16-byte multiple, and the
// halo column at x = nx - 1 comes from the 16-byte box that contains it.
// W: the tile width (32 only for BATCH).
template <int P, bool DIAG, int COLL, bool BATCH, int W = TX, bool SALT_GIVEN = false>
__device__ __forceinline__ void fused_body(const Maps& maps, const Geom& g, const Phys& ph,
                                           typename Prec<P>::T* dst, int* flag, int ntx, int nchunks, int fz,
                                           int grp, const DiagOut& dg, int u, int px, long long dstride,
                                           const DirBases<typename Prec<P>::T>* db, unsigned salt_given = 0u) {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  using V = typename Pair<P>::V;
  using S = FusedShape<P, W>;
  constexpr int TY = S::TY, RH = S::RH, RW = S::RWW;
  static_assert(!DIAG || 2 * TY * TX * sizeof(double) + 10 * TY * sizeof(double) <= S::ring_bytes,
                "the diagnostics reduction reuses the psi ring");
  static_assert(!(BATCH && (DIAG || COLL != COLL_SRT)), "the batched step is the plain SRT step");
  static_assert(W == TX || BATCH, "32-wide tiles for the batched step only");
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + S::off_bar);
  C* ring = reinterpret_cast<C*>(smem + S::off_ring);

  advance_salt(ph);
  // Block order: z runs in groups of grp consecutive runs; inside a group
  // the run index varies fastest, then the tile x, then the tile y.  Blocks
  // that share planes (the two runs either side of a run boundary, x- and
  // y-neighbour tiles) are then launched close together, so the planes and
  // halo rows they share are still in L2 when the second one reads them.
  const int tiles = ntx * (BATCH ? (g.ny + TY - 1) / TY : g.ny / TY);
  const int zg = u / (grp * tiles), r = u - zg * grp * tiles;
  const int gs = min(grp, nchunks - zg * grp);   // runs in this group
  const int chunk = zg * grp + r % gs, xy = r / gs;
  const int x0 = (xy % ntx) * W, y0 = (xy / ntx) * TY;
  // tile extent (BATCH: cut at the lattice's edges)
  const int w = BATCH ? min(W, g.nx - x0) : W, h = BATCH ? min(TY, g.ny - y0) : TY;
  const int z0 = chunk * fz, z1 = min(z0 + fz, g.nz);
  const int tid = threadIdx.x, lane = tid & 31, ty = tid >> 5;
  // the thread's nodes: x0 + 2 xi, x0 + 2 xi + 1 of tile row tr
  const int xi = W == TX ? lane : (lane & 15), tr = W == TX ? ty : 2 * ty + (lane >> 4);
  const int np = (z1 - z0) + 2;        // planes z0 - 1 .. z1, march index k in buffer k % NB
  // Even runs march up (z0 - 1 first), odd runs down (z1 first), so the plane
  // two neighbouring runs share is read by both near the same time (at the
  // start of both, or at the end of both) and the second read hits L2.
  const int dir = (chunk & 1) ? -1 : 1;
  const long long N = dstride;
  const int ym = y0 == 0 ? g.ny - 1 : y0 - 1, yp = y0 + h == g.ny ? 0 : y0 + h;
  // the left halo column x0 - 1 (nx - 1 for the first tile) is element lofs
  // of the 16-byte box at xl; the right one, x0 + w, starts a box
  const int xl = x0 == 0 ? (BATCH ? (g.nx - 1) / S::CW * S::CW : g.nx - S::CW) : x0 - S::CW;
  const int lofs = BATCH && x0 == 0 ? g.nx - 1 - xl : S::CW - 1;
  const int xr = x0 + w == g.nx ? 0 : x0 + W;
  auto zwrap = [&](int p) { return p < 0 ? p + g.nz : (p >= g.nz ? p - g.nz : p); };
  auto zplane = [&](int k) { return zwrap(dir > 0 ? z0 - 1 + k : z1 - k); };   // plane of march index k

  // psi of the halo ring of a plane: warps 0 and 1 take the rows y0 - 1 and
  // y0 + TY over x0 .. x0 + TX - 1 as x pairs (like the interior, in paired
  // FP32 arithmetic), warp 2 the four corners and the 2 TY column cells, one
  // per lane.  A pass costs a warp the same instructions whatever its active
  // lanes.  (With scalar arithmetic the 8-row tile spread its halo rows one
  // node per lane over warps 0 - 3, with the scalar cells on warp 4; with
  // paired arithmetic the pair pass is cheaper: 0.9 % faster FP16 step.)
  // 32-wide tiles: warp 0 takes both rows (16 lanes each), warps 1 (and 2)
  // the scalar cells.
  // h_off: element offset in a plane buffer (-1: no cell), h_str: stride
  // between directions (one-node cells), h_ring: ring position.
  constexpr int SC = 4 + 2 * TY;                      // corner and column cells
  constexpr int SW = W == TX ? 2 : 1;                 // the first warp that takes them
  static_assert(W == TX ? (TY == 4 || TY == 8) && SC <= 32 : (TY == 8 || TY == 16) && SC <= 64,
                "halo split for 64 x 4, 64 x 8, 32 x 8 and 32 x 16 tiles");
  const bool hrow = W == TX ? ty < 2 : ty == 0;       // a thread of the halo rows
  int h_off = -1, h_str = 0, h_ring = 0;
  if (hrow) {
    const int side = W == TX ? ty : lane >> 4;       // 0: row y0 - 1, 1: row y0 + h
    h_off = (int)((side ? S::off_bot : S::off_top) / S::E) + 2 * xi;
    h_ring = (side ? h + 1 : 0) * RW + 2 * xi + 2;
  } else if (ty >= SW && (ty - SW) * 32 + lane < SC) {
    const int c = (ty - SW) * 32 + lane;
    if (c < 4) {
      const int side = c >> 1, right = c & 1;   // corners in the copy order of issue_plane
      h_off = (int)((S::off_cor + c * S::cor_stride) / S::E) + (right ? 0 : lofs);
      h_str = S::CW;
      h_ring = (side ? h + 1 : 0) * RW + (right ? w + 2 : 1);
    } else {
      const int i = c - 4, side = i >= TY, r = i - side * TY;   // side 0: column x0 - 1, 1: x0 + w
      h_off = (int)((side ? S::off_rgt : S::off_lft) / S::E) + r * S::CW + (side ? 0 : lofs);
      h_str = TY * S::CW;
      h_ring = (r + 1) * RW + (side ? w + 2 : 1);
      if (BATCH && r >= h) h_off = -1;   // below the lattice's last row
    }
  }
  // BATCH: this thread's nodes x0 + 2 lane (+1) of row y0 + ty lie in the
  // lattice (act: the first, act1: both)
  const bool act = !BATCH || (tr < h && 2 * xi < w);
  const bool act1 = !BATCH || (tr < h && 2 * xi + 1 < w);
  // the halo row cells x0 + 2 xi (+1) of rows y0 - 1 and y0 + h
  const bool hact = !BATCH || 2 * xi < w, hact1 = !BATCH || 2 * xi + 1 < w;

  // dst + a N, the start of direction a in the destination array: the
  // stores address a direction by this base and a 32-bit offset in it (N <
  // 2^31).  Single lattice: the bases are kernel parameters (db).  Batched
  // step with 2-byte storage (bound by instruction issue): in shared memory,
  // which saves the 64-bit arithmetic per direction and plane (measured: 1.4 %
  // faster; a latency-bound FP32 step was 3 % slower this way).
  __shared__ T* s_dir[Q];
  if (BATCH && Prec<P>::dev && tid < Q) s_dir[tid] = dst + (long long)tid * N;
  __shared__ int s_abort;
  // the deviation shifts, staged through shared memory so that they live in
  // registers: the widening adds of the 2-byte loads take no constant-bank
  // operand (read from the kernel parameters directly, the FP16 step was 4 %
  // slower)
  __shared__ float s_shift[3];
  if (Prec<P>::dev && tid < 3) s_shift[tid] = ph.shift_f[tid];
  if (tid == 0) {
    // bit 2 of the flag: a block (of this launch or an earlier one) gave up
    // on a wait, the result is void; skip the work
    s_abort = (*(volatile int*)flag & 2) != 0;
    for (int b = 0; b < NB + 1; ++b) mbar_init(full + b, 1);   // full[NB]: the test barrier
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (s_abort) return;
  const C s0 = Prec<P>::dev ? (C)s_shift[0] : (C)0, s1 = Prec<P>::dev ? (C)s_shift[1] : (C)0,
          s2 = Prec<P>::dev ? (C)s_shift[2] : (C)0;
  if (tid == 0)
    for (int k = 0; k < NB && k < np; ++k)
      issue_plane<P, W>(smem, maps, k, x0, y0, xl, xr, ym, yp, zplane(k), full + k);

  // the step's stochastic-rounding salt (SALT_GIVEN: by the caller, which
  // runs several steps in one launch)
  const unsigned salt = (Prec<P>::dev && ph.sr) ? (SALT_GIVEN ? salt_given : salt_of(ph)) : 0u;
  // a non-positive or non-finite density met by this thread's psi
  // evaluations (raised on the flag once, after the run: the host reads the
  // flag only after the kernel)
  bool nbad = false;
  V prev[Q];   // stored populations of this thread's two nodes, previous plane
  C prho[2];   // their densities (rho_of of the unpacked values, from the psi step)
  // diagnostics sums (DIAG): block totals and the two x columns of the thread
  DSum<C> d_mass, d_jx, d_jy, d_jz, d_vol, col_w[2];
  C d_umax = 0, d_rmin = (C)3.0e38, d_rmax = (C)-3.0e38;
  C col_n[2] = {0, 0};
  bool d_bad = false;
  const C d_thr = (C)dg.thr_f, d_inv = (C)dg.inv_f, d_rv = (C)dg.rv_f;
  int k = 0;
  for (; k < np; ++k) {
    const int b = k % NB;
    bool ok = mbar_wait_bounded(full + b, (unsigned)((k / NB) & 1));
    if (k == 0 && dg.stall_test_ns) ok = ok && mbar_wait_bounded(full + NB, 0u, dg.stall_test_ns);
    const T* buf = reinterpret_cast<const T*>(smem + (size_t)b * S::plane);
    C* slot = ring + (k % NR) * RH * RW;
    // psi of this thread's two nodes of plane zplane(k), the two nodes as the
    // lanes of one float2 (paired FP32 arithmetic, the bits of the scalar
    // form per lane)
    V cur[Q];
    float2 fp[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      cur[a] = *reinterpret_cast<const V*>(buf + (a * TY + tr) * W + 2 * xi);
      unpack_shifted<P>(cur[a], a == 0 ? s0 : (a <= 6 ? s1 : s2), fp[a].x, fp[a].y);
    }
    const float2 rr = rho_of<float2>(fp);
    const float2 pp = psi_of2(rr, ph);
    const C r0 = rr.x, r1 = rr.y, p0 = pp.x, p1 = pp.y;
    nbad |= (act && bad_rho(r0)) | (act1 && bad_rho(r1));
    if constexpr (DIAG) {
      // momentum of the two nodes (the summation order of the two-kernel
      // diagnostics)
      C jv[2][3], lo[2];
      float2 jx2, jy2, jz2;
      mom_of<float2>(fp, jx2, jy2, jz2);
      jv[0][0] = jx2.x, jv[0][1] = jy2.x, jv[0][2] = jz2.x;
      jv[1][0] = jx2.y, jv[1][1] = jy2.y, jv[1][2] = jz2.y;
      if (k >= 1 && k <= np - 2) {
        // the rounding error of each density (rho_of_x's high part is r0,
        // r1): both nodes in paired instructions for 4-byte storage; one
        // node at a time for 2-byte storage, whose 128-register budget the
        // paired form's error terms exceed (spills)
        if constexpr (Prec<P>::dev) {
          C f0[Q], f1[Q];
#pragma unroll
          for (int a = 0; a < Q; ++a) f0[a] = fp[a].x, f1[a] = fp[a].y;
          rho_of_x(f0, lo[0]);
          rho_of_x(f1, lo[1]);
        } else {
          float2 lo2;
          rho_of_x<float2>(fp, lo2);
          lo[0] = lo2.x;
          lo[1] = lo2.y;
        }
#pragma unroll
        for (int n = 0; n < 2; ++n) {
          const C rho = n ? r1 : r0;
          const C jx = jv[n][0], jy = jv[n][1], jz = jv[n][2];
          d_mass.add(rho, lo[n]);
          d_jx.add(jx);
          d_jy.add(jy);
          d_jz.add(jz);
          C phi = (rho - d_rv) * d_inv;
          phi = phi < (C)0 ? (C)0 : (phi > (C)1 ? (C)1 : phi);
          d_vol.add(phi);
          col_w[n].add(phi);
          col_n[n] += rho > d_thr ? (C)1 : (C)0;
          const C um = sqrt(xfma(jz, jz, xfma(jy, jy, xmul(jx, jx)))) / rho;
          d_umax = um > d_umax ? um : d_umax;
          d_rmin = rho < d_rmin ? rho : d_rmin;
          d_rmax = rho > d_rmax ? rho : d_rmax;
          d_bad |= !(rho > (C)0) || !(rho <= (C)3.0e38);
        }
      }
    }
    if constexpr (BATCH) {
      if (act1)
        *reinterpret_cast<float2*>(slot + (tr + 1) * RW + 2 * xi + 2) = make_float2(p0, p1);
      else if (act)
        slot[(tr + 1) * RW + 2 * xi + 2] = p0;   // the right halo column follows
    } else if constexpr (sizeof(C) == 4) {
      *reinterpret_cast<float2*>(slot + (tr + 1) * RW + 2 * xi + 2) = make_float2(p0, p1);
    } else {
      *reinterpret_cast<double2*>(slot + (tr + 1) * RW + 2 * xi + 2) = make_double2(p0, p1);
    }
    // psi of this thread's halo cells
    if (hrow) {
      float2 fh[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        unpack_shifted<P>(*reinterpret_cast<const V*>(buf + h_off + a * W), a == 0 ? s0 : (a <= 6 ? s1 : s2),
                          fh[a].x, fh[a].y);
      }
      const float2 rh = rho_of<float2>(fh);
      nbad |= (hact && bad_rho(rh.x)) | (hact1 && bad_rho(rh.y));
      const float2 ph2 = psi_of2(rh, ph);
      if (!BATCH || hact1)
        *reinterpret_cast<float2*>(slot + h_ring) = ph2;
      else if (hact)
        slot[h_ring] = ph2.x;
    } else if (h_off >= 0) {
      C fv[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a)
        fv[a] = load_shifted<P>(buf + h_off + a * h_str, a == 0 ? s0 : (a <= 6 ? s1 : s2));
      const C rv = rho_of<C>(fv);
      slot[h_ring] = psi_of<C>(rv, ph);
      nbad |= bad_rho(rv);
    }
    // every psi of plane zplane(k) is in the ring and buffer b is read out
    if (__syncthreads_or(!ok)) break;
    if (tid == 0 && k + NB < np)
      issue_plane<P, W>(smem, maps, b, x0, y0, xl, xr, ym, yp, zplane(k + NB), full + b);

    if (k >= 2 && act) {
      // collide + stream the two nodes (x0 + 2 xi, y0 + tr) of plane z =
      // zplane(k - 1); plane z + dz has march index k - 1 + dir dz
      const int z = zplane(k - 1);
      const int x = x0 + 2 * xi, y = y0 + tr;
      const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x + 2 == g.nx ? 0 : x + 2;
      // right of node 0 (BATCH: x + 1 may be past the lattice's last column)
      const int xr0 = BATCH ? (x + 1 == g.nx ? 0 : x + 1) : x + 1;
      const int rowp = BATCH ? px : g.nx;   // elements per stored row
      const int yv[3] = {y == 0 ? g.ny - 1 : y - 1, y, y == g.ny - 1 ? 0 : y + 1};
      const int zv[3] = {z == 0 ? g.nz - 1 : z - 1, z, z == g.nz - 1 ? 0 : z + 1};
      C q[3][3][4];
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
          const C* row = ring + ((k - 1 + dir * dz) % NR) * RH * RW + (tr + 1 + dy) * RW + 2 * xi + 2;
          if constexpr (sizeof(C) == 4) {
            const float2 v = *reinterpret_cast<const float2*>(row);
            q[dy + 1][dz + 1][1] = v.x;
            q[dy + 1][dz + 1][2] = v.y;
          } else {
            const double2 v = *reinterpret_cast<const double2*>(row);
            q[dy + 1][dz + 1][1] = v.x;
            q[dy + 1][dz + 1][2] = v.y;
          }
          if (dy == 0 || dz == 0) {
            q[dy + 1][dz + 1][0] = row[-1];
            q[dy + 1][dz + 1][3] = row[2];
          } else {
            q[dy + 1][dz + 1][0] = 0;
            q[dy + 1][dz + 1][3] = 0;
          }
        }
      float2 g2[Q];
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        unpack_shifted<P>(prev[a], a == 0 ? s0 : (a <= 6 ? s1 : s2), g2[a].x, g2[a].y);
      }
      C fs0[Q], fs1[Q];
      if constexpr (COLL == COLL_MRT) {
        C g0[Q], g1[Q], pn0[Q], pn1[Q];
        pn0[0] = pn1[0] = 0;
#pragma unroll
        for (int a = 0; a < Q; ++a) g0[a] = g2[a].x, g1[a] = g2[a].y;
#pragma unroll
        for (int a = 1; a < Q; ++a) {
          pn0[a] = q[cy(a) + 1][cz(a) + 1][1 + cx(a)];
          pn1[a] = q[cy(a) + 1][cz(a) + 1][2 + cx(a)];
        }
        collide_math_mrt<C>(ph, g0, q[1][1][1], pn0, fs0);
        collide_math_mrt<C>(ph, g1, q[1][1][2], pn1, fs1);
      } else {
        float2 fs2[Q];
        collide_pair_math(ph, g2, make_float2(prho[0], prho[1]), q, fs2);
#pragma unroll
        for (int a = 0; a < Q; ++a) fs0[a] = fs2[a].x, fs1[a] = fs2[a].y;
      }
      const int i0 = x + g.nx * (y + g.ny * z);
      const bool sr = Prec<P>::dev && ph.sr;
      const unsigned seed0 = sr ? sr_seed(i0, fs0[0], salt) : 0u, seed1 = sr ? sr_seed(i0 + 1, fs1[0], salt) : 0u;
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const C sh = a == 0 ? s0 : (a <= 6 ? s1 : s2);
        const int row = rowp * (yv[1 + cy(a)] + g.ny * zv[1 + cz(a)]);
        if constexpr (Prec<P>::dev) {
          T* const base = BATCH ? s_dir[a] : db->p[a];
          // the shift comes off both nodes in one paired difference
          const float2 sh2 = splat<float2>(sh);
          if (cx(a) == 0) {
            if (BATCH && !act1) {
              store_pop<P>(ph, base + (row + x), fs0[a], sh, seed0, a);   // alone: its bits as in the pair
            } else if (sr) {
              const float2 d = vsub(make_float2(fs0[a], fs1[a]), sh2);   // node x low, x + 1 high
              *reinterpret_cast<unsigned*>(base + (row + x)) =
                  cvt_pair_sr<P>(d.y, d.x, (sr_bits(seed1, a) << 16) | (sr_bits(seed0, a) & 0xFFFFu));
            } else {
              store_pair<P>(base + (row + x), fs0[a], fs1[a], sh);
            }
          } else if (!sr) {
            store_pop<P>(ph, base + (row + (cx(a) > 0 ? xr0 : xm)), fs0[a], sh, seed0, a);
            if (act1) store_pop<P>(ph, base + (row + (cx(a) > 0 ? xp : x)), fs1[a], sh, seed1, a);
          } else if (a & 1) {
            // a and its opposite a + 1 (c_x != 0, the same weight and shift):
            // one conversion per node rounds both with the bits sr_bits gives
            // them (the high half a, the low half a + 1), so the stored values
            // equal those of the one-value conversions of the two-kernel step
            T* const base_b = BATCH ? s_dir[a + 1] : db->p[a + 1];
            const int row_b = rowp * (yv[1 + cy(a + 1)] + g.ny * zv[1 + cz(a + 1)]);
            const unsigned j = (unsigned)(a + 1) >> 1;
            const float2 da = vsub(make_float2(fs0[a], fs1[a]), sh2);
            const float2 db = vsub(make_float2(fs0[a + 1], fs1[a + 1]), sh2);
            const unsigned d0 = cvt_pair_sr<P>(da.x, db.x, sr_word(seed0, j));
            const unsigned d1 = cvt_pair_sr<P>(da.y, db.y, sr_word(seed1, j));
            unsigned short* const pa = reinterpret_cast<unsigned short*>(base + row);
            unsigned short* const pb = reinterpret_cast<unsigned short*>(base_b + row_b);
            pa[cx(a) > 0 ? xr0 : xm] = (unsigned short)(d0 >> 16);
            if (act1) pa[cx(a) > 0 ? xp : x] = (unsigned short)(d1 >> 16);
            pb[cx(a + 1) > 0 ? xr0 : xm] = (unsigned short)d0;
            if (act1) pb[cx(a + 1) > 0 ? xp : x] = (unsigned short)d1;
          }
          // even a with c_x != 0 under stochastic rounding: stored with a - 1
        } else {
          T* base = (BATCH ? dst + (long long)a * N : db->p[a]) + row;
          if (cx(a) == 0) {
            if (act1)
              store_pair<P>(base + x, fs0[a], fs1[a], sh);
            else
              store_pop<P>(ph, base + x, fs0[a], sh, seed0, a);
          } else {
            store_pop<P>(ph, base + (cx(a) > 0 ? xr0 : xm), fs0[a], sh, seed0, a);
            if (act1) store_pop<P>(ph, base + (cx(a) > 0 ? xp : x), fs1[a], sh, seed1, a);
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) prev[a] = cur[a];
    prho[0] = r0;
    prho[1] = r1;
  }
  raise_flag(nbad, flag);
  if (k < np) {
    // a wait gave up: record it, and let the copies already issued land
    // before the block's shared memory is released
    if (tid == 0) {
      atomicOr(flag, 2);
      for (int j = k; j < k + NB && j < np; ++j) mbar_wait_bounded(full + j % NB, (unsigned)((j / NB) & 1));
    }
  }
  if constexpr (DIAG) {
    // the psi ring is free now: it holds the FP64 reduction (TY x 64 x 2
    // slice values, DIAG_NG x TY warp totals)
    __syncthreads();
    double* sh_col = reinterpret_cast<double*>(ring);
    double* sh_w = sh_col + 2 * TY * TX;
#pragma unroll
    for (int n = 0; n < 2; ++n) {
      sh_col[(ty * TX + 2 * lane + n) * 2 + 0] = col_w[n].value();
      sh_col[(ty * TX + 2 * lane + n) * 2 + 1] = (double)col_n[n];
    }
    // warp totals: a fixed FP64 shuffle tree
    double v[5] = {d_mass.value(), d_jx.value(), d_jy.value(), d_jz.value(), d_vol.value()};
    float c_f = 0.0f;
#pragma unroll
    for (int n = 0; n < 2; ++n) c_f += (float)col_n[n];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int i = 0; i < 5; ++i) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
      c_f += __shfl_down_sync(0xffffffffu, c_f, o);
      const C um = __shfl_down_sync(0xffffffffu, d_umax, o);
      const C mn = __shfl_down_sync(0xffffffffu, d_rmin, o);
      const C mx = __shfl_down_sync(0xffffffffu, d_rmax, o);
      d_umax = um > d_umax ? um : d_umax;
      d_rmin = mn < d_rmin ? mn : d_rmin;
      d_rmax = mx > d_rmax ? mx : d_rmax;
    }
    const int anybad = __any_sync(0xffffffffu, d_bad);
    if (lane == 0) {
      sh_w[0 * TY + ty] = v[0];
      sh_w[1 * TY + ty] = v[1];
      sh_w[2 * TY + ty] = v[2];
      sh_w[3 * TY + ty] = v[3];
      sh_w[4 * TY + ty] = v[4];
      sh_w[5 * TY + ty] = (double)c_f;
      sh_w[6 * TY + ty] = (double)d_umax;
      sh_w[7 * TY + ty] = (double)d_rmin;
      sh_w[8 * TY + ty] = (double)d_rmax;
      sh_w[9 * TY + ty] = anybad ? 1.0 : 0.0;
    }
    __syncthreads();
    const long long rb = (long long)(xy / ntx) * nchunks + chunk;
    if (tid < TX) {
      double a = 0.0, c = 0.0;
      for (int r = 0; r < TY; ++r) {
        a += sh_col[(r * TX + tid) * 2 + 0];
        c += sh_col[(r * TX + tid) * 2 + 1];
      }
      dg.slices[(rb * g.nx + x0 + tid) * 2 + 0] = a;
      dg.slices[(rb * g.nx + x0 + tid) * 2 + 1] = c;
    } else if (tid < TX + DIAG_NG) {
      const int i = tid - TX;
      double r;
      if (i < 6) {
        r = 0.0;
        for (int w = 0; w < TY; ++w) r += sh_w[i * TY + w];
      } else if (i == 7) {
        r = 1e300;
        for (int w = 0; w < TY; ++w) r = fmin(r, sh_w[i * TY + w]);
      } else if (i < 10) {
        r = -1e300;
        for (int w = 0; w < TY; ++w) r = fmax(r, sh_w[i * TY + w]);
      } else {
        r = 0.0;
      }
      dg.blocks[(long long)blockIdx.x * DIAG_NG + i] = r;
    }
  }
}

template <int P, bool DIAG, int COLL>
__global__ void __launch_bounds__(FusedShape<P>::NT, fused_minb<P, DIAG, COLL>())
    fused_kernel(const __grid_constant__ Maps maps, Geom g, Phys ph, typename Prec<P>::T* dst, int* flag, int ntx,
                 int nchunks, int fz, int grp, DiagOut dg, const __grid_constant__ DirBases<typename Prec<P>::T> db) {
  fused_body<P, DIAG, COLL, false>(maps, g, ph, dst, flag, ntx, nchunks, fz, grp, dg, blockIdx.x, g.nx, g.N, &db);
}

// One instance of the batched TMA step (device table built by the host).
struct BTInst {
  Geom g;
  Phys ph;
  long long off_f;     // element offset of the instance's array 0 in the padded pool
  long long dstride;   // elements per direction: px ny nz
  const Maps* maps;    // tensor maps of its arrays 0 and 1 (device memory, 64-byte aligned)
  int px;              // elements per row (nx padded to a 16-byte multiple)
  int block0;          // first work item of the instance
  int ntx, nchunks, fz, grp;
};

// The instance of work item w: the largest block0 <= w.
__device__ __forceinline__ const BTInst& find_inst(const BTInst* __restrict__ inst, int count, int w) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].block0 <= w) lo = mid;
    else hi = mid - 1;
  }
  return inst[lo];
}

__device__ __forceinline__ void acquire_maps(const Maps& m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&m.interior) : "memory");
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&m.row) : "memory");
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&m.col) : "memory");
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&m.cor) : "memory");
}

// Work item u of instance I, arrays cur -> cur ^ 1.
template <int P, int W, bool SALT_GIVEN>
__device__ __forceinline__ void batch_item(const BTInst& I, int u, typename Prec<P>::T* pool, int cur, int* flag,
                                           unsigned salt) {
  typename Prec<P>::T* dst = pool + I.off_f + (long long)(cur ^ 1) * Q * I.dstride;
  const DiagOut none{0.0, 0.0, nullptr, nullptr, 0ull, 0.0f, 0.0f, 0.0f};
  const Maps& m = I.maps[cur];
  if (threadIdx.x == 0) acquire_maps(m);
  fused_body<P, false, COLL_SRT, true, W, SALT_GIVEN>(m, I.g, I.ph, dst, flag, I.ntx, I.nchunks, I.fz, I.grp, none,
                                                      u, I.px, I.dstride, nullptr, salt);
}

// The single-pass step of a batch of lattices of any size, their rows
// padded to 16-byte multiples: one launch, each block finds its instance
// and runs fused_body on its work item with that instance's tensor maps,
// which live in global memory (ordered before their use by the tensor-map
// proxy fence).  W: the tile width the table was built for.
template <int P, int W>
__global__ void __launch_bounds__(FusedShape<P, W>::NT, fused_minb<P, false, COLL_SRT>())
    bfused_kernel(const BTInst* __restrict__ inst, int count, typename Prec<P>::T* pool, int cur, int* flag) {
  const BTInst& I = find_inst(inst, count, (int)blockIdx.x);
  batch_item<P, W, false>(I, (int)blockIdx.x - I.block0, pool, cur, flag, 0u);
}

// nsteps steps of the batched TMA step in one cooperative launch of
// persistent blocks: in each step a block takes the next work item (from
// tickets[s], zero before the launch) until none is left and runs fused_body
// on it (its mbarriers invalidated after each item, the next item
// initialises them again); grid barriers on *bar
// separate the steps (bounded: a barrier that waits too long raises the
// timeout bit and the block returns).  Step s runs arrays cur0 ^ (s & 1) ->
// the other with salt salt0 + s, salt0 the salt word at the launch (the host
// advances the word by nsteps after it): the results of nsteps launches of
// bfused_kernel.  stall_test_ns > 0 (a test hook of the failure path):
// block 0 skips the first barrier, the others give up on it after
// stall_test_ns.
template <int P, int W>
__global__ void __launch_bounds__(FusedShape<P, W>::NT, fused_minb<P, false, COLL_SRT>())
    bpersist_kernel(const BTInst* __restrict__ inst, int count, typename Prec<P>::T* pool, int cur0, int nsteps,
                    int items, unsigned* bar, unsigned* tickets, int* flag, unsigned long long stall_test_ns) {
  using S = FusedShape<P, W>;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + S::off_bar);
  __shared__ int s_item;
  const Phys& ph0 = inst[0].ph;   // every instance shares the salt word
  unsigned salt0 = 0u;
  if (Prec<P>::dev && ph0.sr) salt0 = *(const volatile unsigned*)ph0.salt;
  const unsigned long long limit = stall_test_ns ? stall_test_ns : kGridWaitNs;
  for (int s = 0; s < nsteps; ++s) {
    // one read of the flag for the whole block: every thread returns or none
    if (__syncthreads_or(threadIdx.x == 0 && (*(volatile int*)flag & 2) != 0)) return;
    const int cur = cur0 ^ (s & 1);
    for (;;) {
      if (threadIdx.x == 0) s_item = (int)atomicAdd(tickets + s, 1u);
      __syncthreads();
      const int w = s_item;
      if (w >= items) break;
      const BTInst& I = find_inst(inst, count, w);
      batch_item<P, W, true>(I, w - I.block0, pool, cur, flag, salt0 + (unsigned)s);
      __syncthreads();   // the item's shared memory, barriers and s_item are done with
      if (threadIdx.x == 0)
        for (int b = 0; b < NB + 1; ++b)
          asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(full + b)) : "memory");
      __syncthreads();
    }
    if (s + 1 < nsteps) {
      if (stall_test_ns && s == 0 && blockIdx.x == 0) return;
      if (!grid_barrier(bar, (unsigned)(s + 1) * gridDim.x, flag, limit)) return;
    }
  }
}

}  // namespace

}  // namespace lbm
