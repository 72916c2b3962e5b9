// Batched form: many independent periodic lattices of uneven size (a sweep of
// ligaments) advanced together.  Every time step is two launches for the
// whole batch - one psi pass and one collide-stream kernel - whose blocks
// find their lattice in a tile table, and lbm_batch_step replays those
// launches from a captured CUDA graph.  The per-node code is the one the
// single-lattice kernels run (lbm_node.cuh), so each instance evolves
// bitwise as it would alone.  lbm_batch_step_sequential is the plain
// alternative: per instance, its own two launches per step.
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_gfused.cuh"
#include "lbm_node.cuh"

namespace lbm {

// One lattice of a batch, as the kernels see it.
struct BatchInst {
  Geom g;
  Phys ph;
  long long off_f;    // element offset of the instance's first array in the pool
  long long off_psi;  // element offset of its psi
  int tile0;          // first collide-stream block of the instance
  int psi_block0;     // first psi-pass block of the instance
  int vec;            // two nodes per thread (nx even and the batch allows it)
};
// The collide kernel keeps a block's descriptor in shared memory, which
// takes only trivially constructible types (a descriptor that needs dynamic
// initialization there made the batched step 30-45 % slower).
static_assert(std::is_trivially_default_constructible<BatchInst>::value &&
                  std::is_trivially_copyable<BatchInst>::value,
              "BatchInst (and Phys, Geom) must stay trivial aggregates");

namespace {

// Chunks of blockDim.x nodes (node pairs) a collide-stream block covers, one
// after the other: the block's instance lookup is paid once per chunks.
constexpr int kChunks = 4;

// Instance of a block: largest k with start[k] <= b (binary search over the
// batch's cumulative tile starts, kept in the descriptors).
__device__ __forceinline__ int find_inst(const BatchInst* __restrict__ inst, int count, int b,
                                         bool psi_blocks) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int start = psi_blocks ? inst[mid].psi_block0 : inst[mid].tile0;
    if (start <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int P>
__global__ void __launch_bounds__(256) batch_psi_kernel(const BatchInst* __restrict__ inst, int count,
                                                        const typename Prec<P>::T* pool_f, int cur,
                                                        typename Prec<P>::C* pool_psi, int* flag) {
  const int k = find_inst(inst, count, blockIdx.x, true);
  const BatchInst I = inst[k];
  const long long t = (long long)(blockIdx.x - I.psi_block0) * blockDim.x + threadIdx.x;
  const typename Prec<P>::T* f = pool_f + I.off_f + (long long)cur * Q * I.g.N;
  if (I.vec) {
    if (2 * t >= I.g.N) return;
    psi_pair<P, LAYOUT_LOCAL>(I.g, I.ph, f, pool_psi + I.off_psi, flag, 2 * t);
  } else {
    if (t >= I.g.N) return;
    psi_node<P, LAYOUT_LOCAL>(I.g, I.ph, f, pool_psi + I.off_psi, flag, t);
  }
}

// Collide-stream over the batch.  A block covers kChunks x blockDim.x
// consecutive nodes (or node pairs) of one instance in linear order, blockDim.x
// at a time, so a warp reads and
// writes 32 (or 64) consecutive x of a plane, rows continuing across the end
// of a row, and lattices of any size waste no lanes except at their end.
// Every thread looks up the block's instance (the same few cached loads).
template <int P, int MINB>
__global__ void __launch_bounds__(256, MINB) batch_collide_kernel(const BatchInst* __restrict__ inst,
                                                                  int count,
                                                                  typename Prec<P>::T* pool_f, int cur,
                                                                  const typename Prec<P>::C* pool_psi) {
  // every thread finds the block's instance itself (a few cached loads):
  // sharing one thread's lookup through shared memory put the whole block
  // behind a barrier for the length of that lookup
  const BatchInst& I = inst[find_inst(inst, count, blockIdx.x, false)];
  const long long plane = (long long)Q * I.g.N;
  const typename Prec<P>::T* src = pool_f + I.off_f + (long long)cur * plane;
  typename Prec<P>::T* dst = pool_f + I.off_f + (long long)(cur ^ 1) * plane;
  for (int c = 0; c < kChunks; ++c) {
    const long long t = ((long long)(blockIdx.x - I.tile0) * kChunks + c) * blockDim.x + threadIdx.x;
    const long long i = I.vec ? 2 * t : t;   // first node of the thread (x even when paired)
    if (i >= I.g.N) return;
    // 32-bit index arithmetic (N < 2^31)
    const int ii = (int)i;
    const int row = ii / I.g.nx;
    const int x = ii - row * I.g.nx;
    const int z = row / I.g.ny, y = row - z * I.g.ny;
    // the branch is uniform over a block (one instance per block)
    if (I.vec)
      collide_pair<P, MODE_AB>(I.g, I.ph, src, dst, pool_psi + I.off_psi, x, y, z);
    else
      collide_node<P, MODE_AB>(I.g, I.ph, src, dst, pool_psi + I.off_psi, x, y, z);
  }
}

template <int P>
cudaError_t batch_launch_t(const BatchInst* d_inst, int count, int psi_blocks, int tiles, void* pool_f,
                           int cur, void* pool_psi, int* flag, dim3 block, int minb, cudaStream_t s) {
  using T = typename Prec<P>::T;
  using C = typename Prec<P>::C;
  batch_psi_kernel<P><<<psi_blocks, 256, 0, s>>>(d_inst, count, (const T*)pool_f, cur, (C*)pool_psi, flag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned threads = block.x * block.y * block.z;
  switch (minb) {
    case 2:
      batch_collide_kernel<P, 2><<<tiles, threads, 0, s>>>(d_inst, count, (T*)pool_f, cur, (const C*)pool_psi);
      break;
    case 3:
      batch_collide_kernel<P, 3><<<tiles, threads, 0, s>>>(d_inst, count, (T*)pool_f, cur, (const C*)pool_psi);
      break;
    default:
      batch_collide_kernel<P, 4><<<tiles, threads, 0, s>>>(d_inst, count, (T*)pool_f, cur, (const C*)pool_psi);
      break;
  }
  return cudaGetLastError();
}

// The single-pass step's kernels may take more than 48 KB of dynamic shared
// memory; set once per layout (on the current device, outside any capture).
template <int P>
cudaError_t batch_fused_prepare_p() {
  cudaError_t e = cudaFuncSetAttribute(gfused_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)GShape<P>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gpersist_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)GShape<P>::smem);
  return e;
}
cudaError_t batch_fused_prepare(int precision) {
  switch (precision) {
    case LBM_F64: return batch_fused_prepare_p<LBM_F64>();
    case LBM_F32: return batch_fused_prepare_p<LBM_F32>();
    case LBM_F16DEV: return batch_fused_prepare_p<LBM_F16DEV>();
    default: return batch_fused_prepare_p<LBM_BF16DEV>();
  }
}

// nsteps single-pass steps of the whole batch as one cooperative launch of
// persistent blocks (as many as fit on the GPU at once, at most one per work
// item), grid barriers on *bar between the steps.
template <int P>
cudaError_t batch_persist_launch_p(const GInst* d_ginst, int count, int items, void* pool_f, int cur, int nsteps,
                                   unsigned* bar, unsigned* tickets, int* flag, unsigned long long stall_ns,
                                   cudaStream_t s) {
  using T = typename Prec<P>::T;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gpersist_kernel<P>, GNT, GShape<P>::smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  const int grid = std::min(items, per_sm * sms);
  e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tickets, 0, sizeof(unsigned) * (size_t)nsteps, s);
  if (e != cudaSuccess) return e;
  T* pf = (T*)pool_f;
  void* args[] = {(void*)&d_ginst, (void*)&count, (void*)&pf, (void*)&cur, (void*)&nsteps,
                  (void*)&items, (void*)&bar, (void*)&tickets, (void*)&flag, (void*)&stall_ns};
  return cudaLaunchCooperativeKernel((const void*)gpersist_kernel<P>, dim3(grid), dim3(GNT), args,
                                     GShape<P>::smem, s);
}
cudaError_t batch_persist_launch(int precision, const GInst* d_ginst, int count, int items, void* pool_f, int cur,
                                 int nsteps, unsigned* bar, unsigned* tickets, int* flag,
                                 unsigned long long stall_ns, cudaStream_t s) {
  switch (precision) {
    case LBM_F64:
      return batch_persist_launch_p<LBM_F64>(d_ginst, count, items, pool_f, cur, nsteps, bar, tickets, flag,
                                             stall_ns, s);
    case LBM_F32:
      return batch_persist_launch_p<LBM_F32>(d_ginst, count, items, pool_f, cur, nsteps, bar, tickets, flag,
                                             stall_ns, s);
    case LBM_F16DEV:
      return batch_persist_launch_p<LBM_F16DEV>(d_ginst, count, items, pool_f, cur, nsteps, bar, tickets, flag,
                                                stall_ns, s);
    default:
      return batch_persist_launch_p<LBM_BF16DEV>(d_ginst, count, items, pool_f, cur, nsteps, bar, tickets, flag,
                                                 stall_ns, s);
  }
}

// The single-pass step of the whole batch: one launch.
cudaError_t batch_fused_launch(int precision, const GInst* d_ginst, int count, int blocks, void* pool_f, int cur,
                               int* flag, cudaStream_t s) {
  switch (precision) {
    case LBM_F64:
      gfused_kernel<LBM_F64><<<blocks, GNT, GShape<LBM_F64>::smem, s>>>(d_ginst, count, (double*)pool_f, cur, flag);
      break;
    case LBM_F32:
      gfused_kernel<LBM_F32><<<blocks, GNT, GShape<LBM_F32>::smem, s>>>(d_ginst, count, (float*)pool_f, cur, flag);
      break;
    case LBM_F16DEV:
      gfused_kernel<LBM_F16DEV><<<blocks, GNT, GShape<LBM_F16DEV>::smem, s>>>(d_ginst, count, (__half*)pool_f,
                                                                              cur, flag);
      break;
    default:
      gfused_kernel<LBM_BF16DEV><<<blocks, GNT, GShape<LBM_BF16DEV>::smem, s>>>(
          d_ginst, count, (__nv_bfloat16*)pool_f, cur, flag);
      break;
  }
  return cudaGetLastError();
}

cudaError_t batch_launch(int precision, const BatchInst* d_inst, int count, int psi_blocks, int tiles,
                         void* pool_f, int cur, void* pool_psi, int* flag, dim3 block, int minb,
                         cudaStream_t s) {
  switch (precision) {
    case LBM_F64:
      return batch_launch_t<LBM_F64>(d_inst, count, psi_blocks, tiles, pool_f, cur, pool_psi, flag, block, minb, s);
    case LBM_F32:
      return batch_launch_t<LBM_F32>(d_inst, count, psi_blocks, tiles, pool_f, cur, pool_psi, flag, block, minb, s);
    case LBM_F16DEV:
      return batch_launch_t<LBM_F16DEV>(d_inst, count, psi_blocks, tiles, pool_f, cur, pool_psi, flag, block, minb, s);
    case LBM_BF16DEV:
      return batch_launch_t<LBM_BF16DEV>(d_inst, count, psi_blocks, tiles, pool_f, cur, pool_psi, flag, block, minb, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_batch_ctx {
  int count = 0;
  int precision = LBM_F32;
  std::vector<lbm_instance> spec;
  std::vector<BatchInst> inst;
  BatchInst* d_inst = nullptr;
  GInst* d_ginst = nullptr;        // single-pass step: per-instance tile table
  int gblocks = 0;
  bool fused = true;               // option "fused": the single-pass step
  int gfz = 16;                    // its z run length (option "fused_fz")
  int ggrp = 0;                    // runs per block-order group of the padded form (option "fused_group")
  int tma_w = 0;                   // tile width of the padded form, 32 or 64, 0: by storage (option "tile_width")
  bool tma = true;                 // option "fused" = 2 (the default): the single pass on padded rows (TMA)
  // its own pool, rows padded to 16 bytes, which holds the state while that
  // form steps (the state moves between the pools by 2-D copies)
  void* pool_p = nullptr;
  std::vector<long long> off_p;
  std::vector<int> px;
  void* d_ttable = nullptr;        // its tensor maps and block table
  BatchTmaPlan tplan{};            // its launch
  bool ttable_ok = false;
  bool padded = false;             // the current state lives in pool_p
  std::vector<char> contig_ok;     // while padded: instance k's unpadded copy is current too
  bool persistent = false;         // option "persistent": n steps per cooperative launch
  unsigned* d_tickets = nullptr;   // its per-step work-item counters
  int tickets_n = 0;
  double persist_stall_ms = 0.0;   // option "persistent_stall_test" (test hook)
  void* pool_f = nullptr;
  size_t pool_f_bytes = 0;
  void* pool_psi = nullptr;
  size_t pool_psi_bytes = 0;
  int* d_flag = nullptr;
  double* d_small = nullptr;
  double* d_scratch = nullptr;
  size_t scratch_doubles = 0;
  int* d_labels = nullptr;
  size_t labels_ints = 0;
  double* d_plane = nullptr;
  long long max_nodes = 0, total_nodes = 0;
  int tiles = 0, psi_blocks = 0;
  dim3 block{32, 8, 1};
  int minb = 2;
  bool vec = true;
  int cur = 0;
  long long step = 0;
  bool initialized = false;
  bool use_graph = true;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  // the persistent form's graphs: one cooperative launch of m steps from
  // array `cur`, with its counter resets and the salt advance
  struct PersistGraph {
    int cur, m;
    cudaGraphExec_t exec;
  };
  std::vector<PersistGraph> pgraphs;
  cudaStream_t stream = nullptr, own_stream = nullptr;
};

namespace {

thread_local std::string b_err;

int bfail(int status, const std::string& m);
int bcuda(cudaError_t e, const char* where);

#define BCK(call)                                    \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return bcuda(e_, #call);  \
  } while (0)

void drop_graphs(lbm_batch_ctx* b) {
  for (auto& g : b->graph)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
  for (auto& pg : b->pgraphs) cudaGraphExecDestroy(pg.exec);
  b->pgraphs.clear();
}

// Recomputes the block table for the current block size and uploads it.
int layout_tiles(lbm_batch_ctx* b) {
  long long tiles = 0, psi_blocks = 0;
  const int threads = (int)(b->block.x * b->block.y * b->block.z);
  for (auto& I : b->inst) {
    I.vec = (b->vec && I.g.nx % 2 == 0) ? 1 : 0;
    const long long units = I.vec ? I.g.N / 2 : I.g.N;
    I.tile0 = (int)tiles;
    tiles += (units + (long long)threads * kChunks - 1) / ((long long)threads * kChunks);
    I.psi_block0 = (int)psi_blocks;
    psi_blocks += (units + 255) / 256;
  }
  if (tiles > 0x7fffffffLL || psi_blocks > 0x7fffffffLL) return bfail(LBM_ERR_ARG, "batch too large for one grid");
  b->tiles = (int)tiles;
  b->psi_blocks = (int)psi_blocks;
  // the single-pass step: GX x GY tiles in x-y, z runs of gfz planes
  std::vector<GInst> gi(b->count);
  long long gblocks = 0;
  for (int k = 0; k < b->count; ++k) {
    const BatchInst& I = b->inst[k];
    GInst& G = gi[k];
    std::memset(&G, 0, sizeof(G));
    G.g = I.g;
    G.ph = I.ph;
    G.off_f = I.off_f;
    G.ntx = (I.g.nx + GX - 1) / GX;
    G.nty = (I.g.ny + GY - 1) / GY;
    G.fz = std::min(b->gfz, I.g.nz);
    G.nchunks = (I.g.nz + G.fz - 1) / G.fz;
    G.block0 = (int)gblocks;
    gblocks += (long long)G.ntx * G.nty * G.nchunks;
  }
  if (gblocks > 0x7fffffffLL) return bfail(LBM_ERR_ARG, "batch too large for one grid");
  b->gblocks = (int)gblocks;
  b->ttable_ok = false;
  BCK(batch_fused_prepare(b->precision));
  BCK(cudaMemcpyAsync(b->d_ginst, gi.data(), sizeof(GInst) * b->count, cudaMemcpyHostToDevice, b->stream));
  BCK(cudaMemcpyAsync(b->d_inst, b->inst.data(), sizeof(BatchInst) * b->count, cudaMemcpyHostToDevice,
                      b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  drop_graphs(b);
  return LBM_OK;
}

// The single pass on padded rows applies to 4- and 2-byte storage whose
// padded instances keep 32-bit in-plane offsets.
bool tma_applicable(const lbm_batch_ctx* b) {
  if (b->precision == LBM_F64) return false;
  const int al = batch_tma_row_align(b->precision);
  for (const auto& I : b->inst)
    if ((long long)((I.g.nx + al - 1) / al * al) * I.g.ny * I.g.nz > 0x7fffffffLL) return false;
  return true;
}

bool tma_form(const lbm_batch_ctx* b) { return b->fused && b->tma && tma_applicable(b); }

// Copies the current array of instance k between the pools.
int copy_instance(lbm_batch_ctx* b, int k, bool to_padded) {
  const size_t e = elem_size(b->precision);
  const BatchInst& I = b->inst[k];
  const size_t w = (size_t)I.g.nx * e, rows = (size_t)Q * I.g.ny * I.g.nz;
  char* c = (char*)b->pool_f + (size_t)(I.off_f + (long long)b->cur * Q * I.g.N) * e;
  char* p = (char*)b->pool_p + (size_t)(b->off_p[k] + (long long)b->cur * Q * b->px[k] * I.g.ny * I.g.nz) * e;
  const size_t pp = (size_t)b->px[k] * e;
  if (to_padded)
    BCK(cudaMemcpy2DAsync(p, pp, c, w, w, rows, cudaMemcpyDeviceToDevice, b->stream));
  else
    BCK(cudaMemcpy2DAsync(c, w, p, pp, w, rows, cudaMemcpyDeviceToDevice, b->stream));
  return LBM_OK;
}

// Instance k's current state in the unpadded pool, for a call that reads
// it (diagnostics, populations); the padded pool stays the state's home.
int ensure_contig_instance(lbm_batch_ctx* b, int k) {
  if (!b->padded || b->contig_ok[k]) return LBM_OK;
  if (int rc = copy_instance(b, k, false)) return rc;
  b->contig_ok[k] = 1;
  return LBM_OK;
}

// The state back in the unpadded pool (every step form but the padded
// single pass).
int ensure_contig(lbm_batch_ctx* b) {
  if (!b->padded) return LBM_OK;
  for (int k = 0; k < b->count; ++k)
    if (int rc = ensure_contig_instance(b, k)) return rc;
  b->padded = false;
  return LBM_OK;
}


// Tile width of the padded form: 64 for FP32 storage, 32 for 2-byte
// storage (on the 48-ligament sweep on GB300, 32-wide tiles leave fewer
// lanes idle at the instances' x ends, 3 % faster for FP16, but their
// narrower rows cost the bandwidth-bound FP32 step more DRAM traffic and
// bandwidth: 16 % slower).
int table_width(const lbm_batch_ctx* b) { return b->tma_w ? b->tma_w : (b->precision == LBM_F32 ? 64 : 32); }

// The padded pool, its tensor maps and block tables, and the state in it.
int ensure_padded(lbm_batch_ctx* b) {
  const size_t e = elem_size(b->precision);
  if (!b->pool_p) {
    const int al = batch_tma_row_align(b->precision);
    long long off = 0;
    b->off_p.resize(b->count);
    b->px.resize(b->count);
    for (int k = 0; k < b->count; ++k) {
      const Geom& g = b->inst[k].g;
      b->px[k] = (g.nx + al - 1) / al * al;
      b->off_p[k] = off;
      off += 2LL * Q * b->px[k] * g.ny * g.nz;   // a multiple of al: every instance starts on 16 bytes
    }
    if (alloc_over_cap((size_t)off * e)) return bfail(LBM_ERR_OOM, "the padded pool exceeds LBM_ALLOC_CAP_BYTES");
    BCK(cudaMalloc(&b->pool_p, (size_t)off * e));
    b->ttable_ok = false;
  }
  if (!b->d_ttable) {
    BCK(cudaMalloc(&b->d_ttable, batch_tma_table_bytes(b->count)));
    b->ttable_ok = false;
  }
  if (!b->ttable_ok) {
    std::vector<BatchTmaInst> t(b->count);
    for (int k = 0; k < b->count; ++k) {
      t[k].g = b->inst[k].g;
      t[k].ph = b->inst[k].ph;
      t[k].off_f = b->off_p[k];
      t[k].px = b->px[k];
    }
    BCK(batch_tma_build(b->precision, table_width(b), t.data(), b->count, b->gfz, b->ggrp, b->pool_p,
                        b->d_ttable, &b->tplan, b->stream));
    b->ttable_ok = true;
  }
  if (!b->padded) {
    for (int k = 0; k < b->count; ++k)
      if (int rc = copy_instance(b, k, true)) return rc;
    b->padded = true;
    b->contig_ok.assign(b->count, 1);   // both copies current until the next step
  }
  return LBM_OK;
}

bool batch_sr(const lbm_batch_ctx* b) {
  return (b->precision == LBM_F16DEV || b->precision == LBM_BF16DEV) && !b->inst.empty() && b->inst[0].ph.sr;
}

int enqueue_batch_step(lbm_batch_ctx* b, cudaStream_t s, int cur) {
  // the single-pass kernel addresses an instance's populations by 32-bit
  // offsets: instances of 113 M nodes or more take the two kernels
  const bool fused_fits = 19LL * b->max_nodes <= 0x7fffffffLL;
  if (tma_form(b))
    BCK(batch_tma_launch(b->precision, b->d_ttable, b->tplan, b->pool_p, cur, b->d_flag, s));
  // (the caller marks the unpadded copies stale: lbm_batch_step)
  else if (b->fused && fused_fits)
    BCK(batch_fused_launch(b->precision, b->d_ginst, b->count, b->gblocks, b->pool_f, cur, b->d_flag, s));
  else
    BCK(batch_launch(b->precision, b->d_inst, b->count, b->psi_blocks, b->tiles, b->pool_f, cur, b->pool_psi,
                     b->d_flag, b->block, b->minb, s));
  if (batch_sr(b)) BCK(launch_salt((unsigned*)(b->d_flag + 2), false, 0u, s));
  return LBM_OK;
}

int capture_pair(lbm_batch_ctx* b, int phase) {
  cudaStream_t cs;
  BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int rc = LBM_OK;
  if (e == cudaSuccess) {
    rc = enqueue_batch_step(b, cs, phase);
    if (rc == LBM_OK) rc = enqueue_batch_step(b, cs, phase ^ 1);
    e = cudaStreamEndCapture(cs, &g);
  }
  cudaStreamDestroy(cs);
  if (rc != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) return bcuda(e, "batch graph capture");
  e = cudaGraphInstantiate(&b->graph[phase], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph[phase] = nullptr;
    return bcuda(e, "cudaGraphInstantiate");
  }
  return LBM_OK;
}

// A single-lattice view (geometry, physics, current array) of instance k.
struct View {
  Geom g;
  Phys ph;
  void* f;
  void* psi;
};

View view_of(lbm_batch_ctx* b, int k) {
  const BatchInst& I = b->inst[k];
  const size_t e = elem_size(b->precision);
  const size_t pe = b->precision == LBM_F64 ? 8 : 4;
  View v;
  v.g = I.g;
  v.ph = I.ph;
  v.f = (char*)b->pool_f + (I.off_f + (long long)b->cur * Q * I.g.N) * e;
  v.psi = (char*)b->pool_psi + I.off_psi * pe;
  return v;
}

int bfail(int status, const std::string& m) {
  b_err = m;
  // surface through the single-lattice error channel as well
  return status;
}

int bcuda(cudaError_t e, const char* where) {
  b_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

// Steps of one persistent launch, and the graph of them.
constexpr int kPersistSteps = 1024;

// The counter resets, the cooperative launch of m steps from array cur and
// the salt advance, on stream s.
int enqueue_persist(lbm_batch_ctx* b, cudaStream_t s, int cur, int m) {
  const unsigned long long stall_ns = (unsigned long long)(b->persist_stall_ms * 1e6);
  if (tma_form(b))
    BCK(batch_tma_persist_launch(b->precision, b->d_ttable, b->tplan, b->pool_p, cur, m,
                                 (unsigned*)(b->d_flag + 4), b->d_tickets, b->d_flag, stall_ns, s));
  else
    BCK(batch_persist_launch(b->precision, b->d_ginst, b->count, b->gblocks, b->pool_f, cur, m,
                             (unsigned*)(b->d_flag + 4), b->d_tickets, b->d_flag, stall_ns, s));
  if (batch_sr(b)) BCK(launch_salt_add((unsigned*)(b->d_flag + 2), (unsigned)m, s));
  return LBM_OK;
}

int capture_persist(lbm_batch_ctx* b, int cur, int m, cudaGraphExec_t* out) {
  cudaStream_t cs;
  BCK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int rc = LBM_OK;
  if (e == cudaSuccess) {
    rc = enqueue_persist(b, cs, cur, m);
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (rc == LBM_OK) e = e2;
  }
  cudaStreamDestroy(cs);
  if (rc != LBM_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    (void)cudaGetLastError();
    return rc != LBM_OK ? rc : bcuda(e, "persistent batch graph capture (option graph 0 launches it directly)");
  }
  cudaGraphExec_t ge = nullptr;
  e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return bcuda(e, "cudaGraphInstantiate (persistent batch)");
  if (b->pgraphs.size() >= 8) {   // calls of many step counts: keep the newest graphs
    cudaGraphExecDestroy(b->pgraphs.front().exec);
    b->pgraphs.erase(b->pgraphs.begin());
  }
  b->pgraphs.push_back({cur, m, ge});
  *out = ge;
  return LBM_OK;
}

}  // namespace

extern "C" {

const char* lbm_batch_last_error(void) { return b_err.c_str(); }

void lbm_batch_destroy(lbm_batch b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  cudaFree(b->d_inst);
  cudaFree(b->d_ginst);
  cudaFree(b->pool_f);
  cudaFree(b->pool_psi);
  cudaFree(b->d_flag);
  cudaFree(b->d_tickets);
  cudaFree(b->pool_p);
  cudaFree(b->d_ttable);
  cudaFree(b->d_small);
  cudaFree(b->d_scratch);
  cudaFree(b->d_labels);
  cudaFree(b->d_plane);
  if (b->own_stream) cudaStreamDestroy(b->own_stream);
  delete b;
}

lbm_batch lbm_batch_create(const lbm_instance* inst, int count, int precision, int psi_form, double rho0,
                           void* stream) {
  if (!inst || count < 1 || count > 1 << 20) {
    bfail(LBM_ERR_ARG, "need 1 <= count <= 2^20 instances");
    return nullptr;
  }
  if (precision < LBM_F64 || precision > LBM_BF16DEV || (psi_form != LBM_PSI_EXP && psi_form != LBM_PSI_RHO) ||
      !(rho0 > 0.0) || !std::isfinite(rho0)) {
    bfail(LBM_ERR_ARG, "bad precision, psi_form or rho0");
    return nullptr;
  }
  lbm_batch_ctx* b = new (std::nothrow) lbm_batch_ctx();
  if (!b) {
    bfail(LBM_ERR_OOM, "host allocation failed");
    return nullptr;
  }
  b->count = count;
  b->precision = precision;
  b->spec.assign(inst, inst + count);
  long long off_f = 0, off_psi = 0;
  for (int k = 0; k < count; ++k) {
    const lbm_instance& s = inst[k];
    const long long N = (long long)s.nx * s.ny * s.nz;
    if (s.nx < 3 || s.ny < 3 || s.nz < 3 || N > 0x7fffffffLL || !(s.tau > 0.5) || !std::isfinite(s.tau) ||
        !std::isfinite(s.G) || !(s.rho_l > s.rho_v) || !(s.rho_v > 0.0) || !(s.width > 0.0) || !(s.lambda > 0.0)) {
      bfail(LBM_ERR_ARG, "instance " + std::to_string(k) + ": bad size or parameters");
      delete b;
      return nullptr;
    }
    BatchInst I;
    std::memset(&I, 0, sizeof(I));
    I.g = Geom{s.nx, s.ny, s.nz, N};
    I.ph = Phys{s.tau, s.G, rho0, precision >= LBM_F16DEV ? s.rho_v : 0.0, psi_form,
                precision >= LBM_F16DEV ? 1 : 0};
    I.ph.inv_rho0 = 1.0 / rho0;
    phys_finalize(I.ph, precision);
    I.off_f = off_f;
    I.off_psi = off_psi;
    // every instance's arrays start on a multiple of 8 elements (64 bytes in
    // FP64): the vector kernels move node pairs (and four-node groups) as one
    // 2- or 4-element access, which an odd N before them would misalign
    off_f += (2 * (long long)Q * N + 7) / 8 * 8;
    off_psi += (N + 7) / 8 * 8;
    b->inst.push_back(I);
    b->max_nodes = N > b->max_nodes ? N : b->max_nodes;
    b->total_nodes += N;
  }
  const size_t e = elem_size(precision);
  b->pool_f_bytes = (size_t)off_f * e;
  b->pool_psi_bytes = (size_t)off_psi * (precision == LBM_F64 ? 8 : 4);
  cudaError_t err = cudaSuccess;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    err = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking);
    b->stream = b->own_stream;
  }
  if (err == cudaSuccess) err = cudaMalloc(&b->d_inst, sizeof(BatchInst) * count);
  if (err == cudaSuccess) err = cudaMalloc(&b->d_ginst, sizeof(GInst) * count);
  if (err == cudaSuccess && alloc_over_cap(b->pool_f_bytes + b->pool_psi_bytes)) {
    bfail(LBM_ERR_OOM, "the batch's pools exceed LBM_ALLOC_CAP_BYTES");
    lbm_batch_destroy(b);
    return nullptr;
  }
  if (err == cudaSuccess) err = cudaMalloc(&b->pool_f, b->pool_f_bytes);
  if (err == cudaSuccess) err = cudaMalloc(&b->pool_psi, b->pool_psi_bytes);
  // d_flag[0] the numeric flag, [2] the stochastic-rounding salt, [4] the
  // grid-barrier counter of the persistent step
  if (err == cudaSuccess) err = cudaMalloc(&b->d_flag, sizeof(int) * 8);
  if (err == cudaSuccess) err = cudaMalloc(&b->d_small, sizeof(double) * 64);
  if (err == cudaSuccess) err = cudaMemsetAsync(b->d_flag, 0, sizeof(int) * 8, b->stream);
  // d_flag[2] is the stochastic-rounding step salt of every instance
  if (err == cudaSuccess)
    for (auto& I : b->inst) I.ph.salt = (const unsigned*)(b->d_flag + 2);
  if (err == cudaSuccess) err = cudaMemsetAsync(b->pool_f, 0, b->pool_f_bytes, b->stream);
  if (err != cudaSuccess) {
    bcuda(err, "lbm_batch_create");
    lbm_batch_destroy(b);
    return nullptr;
  }
  if (layout_tiles(b) != LBM_OK) {
    lbm_batch_destroy(b);
    return nullptr;
  }
  return b;
}

int lbm_batch_set_stream(lbm_batch b, void* stream) {
  if (!b) return bfail(LBM_ERR_ARG, "null batch");
  BCK(cudaStreamSynchronize(b->stream));
  b->stream = stream ? (cudaStream_t)stream : b->own_stream;
  if (!b->stream) {
    BCK(cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking));
    b->stream = b->own_stream;
  }
  return LBM_OK;
}

int lbm_batch_set_option(lbm_batch b, const char* key, double v) {
  if (!b || !key) return bfail(LBM_ERR_ARG, "null argument");
  const std::string k(key);
  if (k == "graph") {
    b->use_graph = v != 0.0;
    return LBM_OK;
  }
  if (k == "stochastic_rounding") {
    for (auto& I : b->inst) I.ph.sr = v != 0.0 ? 1 : 0;
    return layout_tiles(b);
  }
  if (k == "vector") {
    b->vec = v != 0.0;
    return layout_tiles(b);
  }
  if (k == "fused") {
    if (v != 0.0 && v != 1.0 && v != 2.0) return bfail(LBM_ERR_ARG, "fused must be 0, 1 or 2");
    b->fused = v != 0.0;
    b->tma = v == 2.0;
    drop_graphs(b);
    return LBM_OK;
  }
  if (k == "persistent") {
    b->persistent = v != 0.0;
    return LBM_OK;
  }
  if (k == "persistent_stall_test") {
    if (!(v >= 0.0 && v <= 10.0)) return bfail(LBM_ERR_ARG, "persistent_stall_test must be in 0..10 ms");
    b->persist_stall_ms = v;
    drop_graphs(b);   // the hook is an argument of the captured launches
    return LBM_OK;
  }
  if (k == "tile_width") {
    if (v != 0.0 && v != 32.0 && v != 64.0) return bfail(LBM_ERR_ARG, "tile_width must be 0, 32 or 64");
    b->tma_w = (int)v;
    return layout_tiles(b);
  }
  if (k == "fused_group") {
    const long long n = (long long)v;
    if (n < 0 || n > 1 << 20 || (double)n != v) return bfail(LBM_ERR_ARG, "fused_group must be a non-negative integer");
    b->ggrp = (int)n;
    return layout_tiles(b);
  }
  if (k == "fused_fz") {
    const long long n = (long long)v;
    if (n < 1 || n > 1 << 20 || (double)n != v) return bfail(LBM_ERR_ARG, "fused_fz must be a positive integer");
    b->gfz = (int)n;
    return layout_tiles(b);
  }
  if (k == "occupancy") {
    if (v != 2.0 && v != 3.0 && v != 4.0) return bfail(LBM_ERR_ARG, "occupancy must be 2, 3 or 4");
    b->minb = (int)v;
    drop_graphs(b);
    return LBM_OK;
  }
  if (k == "block_x" || k == "block_y" || k == "block_z") {
    const long long n = (long long)v;
    if (n < 1 || n > 256 || (double)n != v) return bfail(LBM_ERR_ARG, "block size must be an integer in 1..256");
    dim3 nb = b->block;
    if (k == "block_x") nb.x = (unsigned)n;
    if (k == "block_y") nb.y = (unsigned)n;
    if (k == "block_z") nb.z = (unsigned)n;
    if ((long long)nb.x * nb.y * nb.z > 256 || nb.z > 64) return bfail(LBM_ERR_ARG, "block shape has more than 256 threads");
    b->block = nb;
    return layout_tiles(b);
  }
  return bfail(LBM_ERR_ARG, "unknown option " + k);
}

int lbm_batch_info(lbm_batch b, long long* total_nodes, int* collide_tiles, int* block3) {
  if (!b) return bfail(LBM_ERR_ARG, "null batch");
  if (total_nodes) *total_nodes = b->total_nodes;
  if (collide_tiles) *collide_tiles = b->tiles;
  if (block3) {
    block3[0] = (int)b->block.x;
    block3[1] = (int)b->block.y;
    block3[2] = (int)b->block.z;
  }
  return LBM_OK;
}

int lbm_batch_init(lbm_batch b) {
  if (!b) return bfail(LBM_ERR_ARG, "null batch");
  b->cur = 0;
  b->step = 0;
  b->padded = false;   // the initial condition goes to the unpadded pool
  BCK(launch_salt((unsigned*)(b->d_flag + 2), true, 0u, b->stream));
  for (int k = 0; k < b->count; ++k) {
    const lbm_instance& s = b->spec[k];
    View v = view_of(b, k);
    InitSpec sp{s.R0, s.lambda, s.eps, s.phase, s.rho_l, s.rho_v, s.width, nullptr, 0, 0.0, 1.0};
    BCK(launch_init(b->precision, v.g, v.ph, sp, v.f, b->stream));
  }
  BCK(cudaStreamSynchronize(b->stream));
  b->initialized = true;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch b, int n) {
  if (!b || n < 0) return bfail(LBM_ERR_ARG, "null batch or negative step count");
  if (!b->initialized) return bfail(LBM_ERR_STATE, "batch not initialised");
  if (n > 0) {
    const int rc = tma_form(b) ? ensure_padded(b) : ensure_contig(b);
    if (rc) return rc;
    if (b->padded) b->contig_ok.assign(b->count, 0);   // the steps below change the padded state
  }
  while (n > 0 && b->persistent && b->fused && (tma_form(b) || 19LL * b->max_nodes <= 0x7fffffffLL)) {
    // up to kPersistSteps steps in one cooperative launch of persistent
    // blocks, replayed from a graph (option graph, default on)
    const int m = std::min(n, kPersistSteps);
    if (!b->d_tickets) {
      BCK(cudaMalloc(&b->d_tickets, sizeof(unsigned) * kPersistSteps));
      b->tickets_n = kPersistSteps;
    }
    if (b->use_graph) {
      cudaGraphExec_t ge = nullptr;
      for (const auto& pg : b->pgraphs)
        if (pg.cur == b->cur && pg.m == m) ge = pg.exec;
      if (!ge) {
        if (int rc = capture_persist(b, b->cur, m, &ge)) return rc;
      }
      BCK(cudaGraphLaunch(ge, b->stream));
    } else {
      if (int rc = enqueue_persist(b, b->stream, b->cur, m)) return rc;
    }
    b->cur ^= m & 1;
    b->step += m;
    n -= m;
  }
  while (n > 0) {
    if (b->use_graph && n >= 2) {
      if (!b->graph[b->cur]) {
        int rc = capture_pair(b, b->cur);
        if (rc) return rc;
      }
      BCK(cudaGraphLaunch(b->graph[b->cur], b->stream));
      n -= 2;
      b->step += 2;
    } else {
      int rc = enqueue_batch_step(b, b->stream, b->cur);
      if (rc) return rc;
      b->cur ^= 1;
      n -= 1;
      b->step += 1;
    }
  }
  return LBM_OK;
}

int lbm_batch_step_sequential(lbm_batch b, int n) {
  if (!b || n < 0) return bfail(LBM_ERR_ARG, "null batch or negative step count");
  if (!b->initialized) return bfail(LBM_ERR_STATE, "batch not initialised");
  if (int rc = ensure_contig(b)) return rc;
  const size_t e = elem_size(b->precision);
  for (int s = 0; s < n; ++s) {
    for (int k = 0; k < b->count; ++k) {
      View v = view_of(b, k);
      void* dst = (char*)v.f + (b->cur ? -1 : 1) * (long long)Q * v.g.N * (long long)e;
      const bool vec = b->inst[k].vec != 0;
      BCK(launch_psi(b->precision, LAYOUT_LOCAL, vec, v.g, v.ph, v.f, v.psi, b->d_flag, b->stream));
      // as a standalone lattice of this size runs by default
      BCK(launch_collide(b->precision, MODE_AB, 0, vec, v.g, v.ph, v.f, dst, v.psi, default_block(v.g),
                         b->stream));
    }
    if (batch_sr(b)) BCK(launch_salt((unsigned*)(b->d_flag + 2), false, 0u, b->stream));
    b->cur ^= 1;
    b->step += 1;
  }
  return LBM_OK;
}

int lbm_batch_sync(lbm_batch b) {
  if (!b) return bfail(LBM_ERR_ARG, "null batch");
  int flag = 0;
  BCK(cudaMemcpyAsync(&flag, b->d_flag, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (flag) {
    BCK(cudaMemsetAsync(b->d_flag, 0, sizeof(int), b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    if (flag & 2) return bfail(LBM_ERR_TIMEOUT, "a grid barrier of the persistent step gave up; the state is void");
    return bfail(LBM_ERR_NUMERIC, "a density became non-positive or non-finite");
  }
  return LBM_OK;
}

int lbm_batch_get_populations(lbm_batch b, int k, double* host) {
  if (!b || !host || k < 0 || k >= b->count) return bfail(LBM_ERR_ARG, "bad batch, instance or buffer");
  if (int rc = ensure_contig_instance(b, k)) return rc;
  if (!b->d_plane) BCK(cudaMalloc(&b->d_plane, sizeof(double) * b->max_nodes));
  View v = view_of(b, k);
  for (int a = 0; a < Q; ++a) {
    BCK(launch_get_plane(b->precision, LAYOUT_LOCAL, v.g, v.ph, v.f, a, b->d_plane, b->stream));
    BCK(cudaMemcpyAsync(host + (size_t)a * v.g.N, b->d_plane, sizeof(double) * v.g.N, cudaMemcpyDeviceToHost,
                        b->stream));
  }
  BCK(cudaStreamSynchronize(b->stream));
  return LBM_OK;
}

int lbm_batch_diagnostics(lbm_batch b, int k, lbm_diag* out, int want_ccl) {
  if (!b || !out || k < 0 || k >= b->count) return bfail(LBM_ERR_ARG, "bad batch, instance or output");
  if (int rc = ensure_contig_instance(b, k)) return rc;
  View v = view_of(b, k);
  const size_t need = diag_scratch_doubles(v.g);
  if (need > b->scratch_doubles) {
    cudaFree(b->d_scratch);
    b->d_scratch = nullptr;
    BCK(cudaMalloc(&b->d_scratch, sizeof(double) * need));
    b->scratch_doubles = need;
  }
  const lbm_instance& s = b->spec[k];
  BCK(launch_diagnostics(b->precision, LAYOUT_LOCAL, v.g, v.ph, v.f, s.rho_l, s.rho_v, b->d_scratch, b->d_small,
                         nullptr, nullptr, nullptr, 0, b->stream));
  double r[DIAG_OUT];
  long long c4[4] = {-1, -1, -1, 0};
  if (want_ccl) {
    if ((size_t)(2 * v.g.N) > b->labels_ints) {
      cudaFree(b->d_labels);
      b->d_labels = nullptr;
      BCK(cudaMalloc(&b->d_labels, sizeof(int) * 2 * b->max_nodes));
      b->labels_ints = 2 * b->max_nodes;
    }
    long long* d4 = (long long*)(b->d_small + 32);
    BCK(launch_ccl(b->precision, LAYOUT_LOCAL, v.g, v.ph, v.f, 0.5 * (s.rho_l + s.rho_v), b->d_labels,
                   b->d_labels + v.g.N, d4, b->stream));
    BCK(cudaMemcpyAsync(c4, d4, sizeof(c4), cudaMemcpyDeviceToHost, b->stream));
  }
  BCK(cudaMemcpyAsync(r, b->d_small, sizeof(r), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (want_ccl && c4[3]) return bfail(LBM_ERR_TIMEOUT, "connected-component labelling guard tripped");
  std::memset(out, 0, sizeof(*out));
  out->step = b->step;
  out->mass = r[0];
  out->mom[0] = r[1];
  out->mom[1] = r[2];
  out->mom[2] = r[3];
  out->liquid_volume_w = r[4];
  out->liquid_count = (long long)r[5];
  out->min_slice_area_w = r[6];
  out->min_slice_count = (long long)r[7];
  out->min_slice_x = (int)r[8];
  out->neck_radius = std::sqrt(r[6] / 3.14159265358979323846);
  out->max_u = r[9];
  out->rho_min = r[10];
  out->rho_max = r[11];
  out->numeric_ok = (int)r[12];
  out->droplets = (int)c4[0];
  out->droplets_min8 = (int)c4[1];
  out->largest_droplet = c4[2];
  return LBM_OK;
}

}  // extern "C"
