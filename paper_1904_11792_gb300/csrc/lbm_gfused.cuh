// Single-pass time step for lattices of any size, on the batch's unpadded
// pool (the batched sweep's per-element form: FP64, instances too large for
// the padded TMA form of lbm_fused_kernel.cuh, and the persistent launch).
//
// The TMA fused step needs rows of a 16-byte multiple, which the ligaments
// of a sweep (arbitrary lengths) have only in the batch's padded pool.  This
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

// One work item of the step: block index blk of the tile table (a tile and
// z run of one instance), A-B arrays cur -> cur ^ 1, stochastic-rounding salt
// `salt` (read by the caller), shared memory gsm of GShape<P>::smem bytes.
template <int P>
__device__ __forceinline__ void gfused_item(const GInst* __restrict__ inst, int count,
                                            typename Prec<P>::T* pool_f, int cur, int* flag, int blk,
                                            unsigned salt, unsigned char* gsm) {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  using S = GShape<P>;
  T* own = reinterpret_cast<T*>(gsm);                                  // [NBUF][Q][GNT]
  T* rpop = reinterpret_cast<T*>(gsm + S::own_bytes);                  // [2][Q][RPAD]
  C(*ring)[GRY][GRX] = reinterpret_cast<C(*)[GRY][GRX]>(gsm + S::own_bytes + S::ring_pop_bytes);

  const GInst& I = inst[gfind(inst, count, blk)];
  const Geom g = I.g;
  const Phys ph = I.ph;
  // element offsets within an instance are 32-bit: 19 N < 2^31 (the host
  // sends larger instances to the two-kernel step)
  const int N = (int)g.N;
  const T* src = pool_f + I.off_f + (long long)cur * Q * N;
  T* dst = pool_f + I.off_f + (long long)(cur ^ 1) * Q * N;
  // block -> (z run, tile x, tile y), the run fastest: the runs of a tile and
  // the tiles of a row of tiles are launched together and share planes and
  // ring rows in L2
  const int u = blk - I.block0;
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
  const int yrow[3] = {g.nx * yv[0], g.nx * yv[1], g.nx * yv[2]};   // row offsets of y - 1, y, y + 1

  const C s0 = shift_of<P>(0, ph), s1 = shift_of<P>(1, ph), s2 = shift_of<P>(7, ph);
  auto shift = [&](int a) { return a == 0 ? s0 : (a <= 6 ? s1 : s2); };
  const int plane_n = g.nx * g.ny;

  // copies of plane zplane(k) (own node into buffer k % 3, ring node into
  // ring buffer k % 2), one commit group per plane, empty past the run
  auto issue = [&](int k) {
    if constexpr (S::async) {
      if (k < np) {
        const int zo = plane_n * zplane(k);
        if (act) {
          T* d = own + (size_t)(k % S::NBUF) * Q * GNT + tid;
#pragma unroll
          for (int a = 0; a < Q; ++a) cp_async<sizeof(T)>(d + a * GNT, src + (a * N + zo + orow));
        }
        if (ract) {
          T* d = rpop + (size_t)(k % 2) * Q * S::RPAD + tid;
#pragma unroll
          for (int a = 0; a < Q; ++a) cp_async<sizeof(T)>(d + a * S::RPAD, src + (a * N + zo + rrow));
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
        const int i = orow + plane_n * zk;
#pragma unroll
        for (int a = 0; a < Q; ++a) f[a] = Prec<P>::load(src + (a * N + i), shift(a));
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
        const int i = rrow + plane_n * zk;
#pragma unroll
        for (int a = 0; a < Q; ++a) fr[a] = Prec<P>::load(src + (a * N + i), shift(a));
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
      if constexpr (Prec<P>::dev) {
        // collide_math_r with the momentum before the link sums: that order
        // keeps the 2-byte forms of this kernel within 128 registers (the
        // other order spills; for FP32 it is 1.8 % faster)
        C jx, jy, jz, ax, ay, az, dx, dy, dz;
        mom_of<C>(fp, jx, jy, jz);
        link_sums<C>(pn, ax, ay, az, dx, dy, dz);
        collide_math_ls<C>(ph, fp, prho, jx, jy, jz, pc, ax, ay, az, dx, dy, dz, fs);
      } else {
        collide_math_r<C>(ph, fp, prho, pc, pn, fs);
      }
      const int i = x + g.nx * (y + g.ny * z);
      const unsigned seed = (Prec<P>::dev && ph.sr) ? sr_seed(i, fs[0], salt) : 0u;
      // destination offsets: x + row of y + plane of z, and a N
      const int pz[3] = {plane_n * zv[0], plane_n * zv[1], plane_n * zv[2]};
#pragma unroll
      for (int a = 0; a < Q; ++a) {
        const int d = xs[1 + cx(a)] + yrow[1 + cy(a)] + pz[1 + cz(a)];
        store_pop<P>(ph, dst + (a * N + d), fs[a], shift(a), seed, a);
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

// The step of the whole batch: one block per work item.
template <int P>
__global__ void __launch_bounds__(GNT, gfused_minb<P>())
    gfused_kernel(const GInst* __restrict__ inst, int count, typename Prec<P>::T* pool_f, int cur, int* flag) {
  extern __shared__ __align__(16) unsigned char gsm[];
  const Phys& ph = inst[0].ph;   // every instance shares the salt word
  const unsigned salt = (Prec<P>::dev && ph.sr) ? salt_of(ph) : 0u;
  gfused_item<P>(inst, count, pool_f, cur, flag, blockIdx.x, salt, gsm);
}

// nsteps steps of the whole batch in one cooperative launch of persistent
// blocks (each takes the next work item of the step until none is left:
// tickets[s], zero before the launch, hands them out), the steps separated
// by grid barriers on *bar.  Step s runs
// arrays cur0 ^ (s & 1) -> the other with salt salt0 + s, salt0 the value of
// the salt word at the launch (the host advances the word by nsteps after
// it), so the results are those of nsteps launches of gfused_kernel.  A block
// returns at once if bit 2 of the flag is set (a barrier of this launch or
// an earlier one gave up).  stall_test_ns > 0 (a test hook of the failure
// path): block 0 does not arrive at the first barrier, every other block
// gives up on it after stall_test_ns.
template <int P>
__global__ void __launch_bounds__(GNT, gfused_minb<P>())
    gpersist_kernel(const GInst* __restrict__ inst, int count, typename Prec<P>::T* pool_f, int cur0, int nsteps,
                    int items, unsigned* bar, unsigned* tickets, int* flag, unsigned long long stall_test_ns) {
  extern __shared__ __align__(16) unsigned char gsm[];
  __shared__ int s_item;
  const Phys& ph = inst[0].ph;
  unsigned salt0 = 0u;
  if (Prec<P>::dev && ph.sr) salt0 = *(const volatile unsigned*)ph.salt;
  const unsigned long long limit = stall_test_ns ? stall_test_ns : kGridWaitNs;
  for (int s = 0; s < nsteps; ++s) {
    // one read of the flag for the whole block: every thread returns or none
    if (__syncthreads_or(threadIdx.x == 0 && (*(volatile int*)flag & 2) != 0)) return;
    const int cur = cur0 ^ (s & 1);
    // work items in launch order, each to the next block that asks
    // (tickets[s] counts the items handed out in step s; asking for the next
    // one while working on the current one was 7 % slower: a block then holds
    // an item that idle blocks could take at the end of the step)
    for (;;) {
      if (threadIdx.x == 0) s_item = (int)atomicAdd(tickets + s, 1u);
      __syncthreads();
      const int w = s_item;
      if (w >= items) break;
      gfused_item<P>(inst, count, pool_f, cur, flag, w, salt0 + (unsigned)s, gsm);
      __syncthreads();   // the item's shared memory and s_item are read out before the next item
    }
    if (s + 1 < nsteps) {
      if (stall_test_ns && s == 0 && blockIdx.x == 0) return;
      if (!grid_barrier(bar, (unsigned)(s + 1) * gridDim.x, flag, limit)) return;
    }
  }
}

}  // namespace lbm
