// Fused time step, host side: the tensor maps of the population arrays, the
// launch shape (z-run length, runs per block-order group, blocks) and the
// launches of the kernel in lbm_fused_kernel.cuh.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "lbm_fused_kernel.cuh"

namespace lbm {

namespace {

// Tile rows of the fused step for a storage precision (FusedShape<P>::TY).
int fused_tile_rows(int precision) {
  return precision == LBM_F16DEV ? FusedShape<LBM_F16DEV>::TY
                                 : (precision == LBM_BF16DEV ? FusedShape<LBM_BF16DEV>::TY : FusedShape<LBM_F32>::TY);
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

// The 4-D view [19][nz][ny][nx] of a population array with box (bx, by, 1, 19),
// rows px elements apart (px = nx, or nx padded for the batched step).
cudaError_t make_map(CUtensorMap* tm, int precision, const Geom& g, const void* base, int bx, int by, int px = 0) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const size_t e = elem_size(precision);
  const cuuint64_t p = px > 0 ? (cuuint64_t)px : (cuuint64_t)g.nx;
  const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)Q};
  const cuuint64_t strides[3] = {p * e, p * g.ny * e, p * g.ny * g.nz * e};
  const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1u, (cuuint32_t)Q};
  const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
  const CUresult r = fn(tm, tma_type(precision), 4, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor maps are pure host-side descriptors; they are cached per array.
cudaError_t maps_for(int precision, const Geom& g, const void* base, Maps* out) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, int, int, int>, Maps> cache;
  const auto key = std::make_tuple(base, precision, g.nx, g.ny, g.nz);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it == cache.end()) {
    const int cw = 16 / (int)elem_size(precision);
    Maps m;
    const int ty = fused_tile_rows(precision);
    cudaError_t e = make_map(&m.interior, precision, g, base, TX, ty);
    if (e == cudaSuccess) e = make_map(&m.row, precision, g, base, TX, 1);
    if (e == cudaSuccess) e = make_map(&m.col, precision, g, base, cw, ty);
    if (e == cudaSuccess) e = make_map(&m.cor, precision, g, base, cw, 1);
    if (e != cudaSuccess) return e;
    it = cache.emplace(key, m).first;
  }
  *out = it->second;
  return cudaSuccess;
}

// z planes per block.  Each block also loads the two planes around its run,
// and a grid that leaves SMs idle in its last wave wastes their bandwidth:
// the cost of a run length is waves x planes loaded per block, times
// (1 + fz/256) for long runs.  On grids of many waves long runs cost more
// than that (measured on GB300, 1024x512x512 in groups of runs: 12-, 16-,
// 19-, 24- and 32-plane runs take 6.5, 6.4-7.8, 7.0, 7.7 and 8.2 ms per
// step: the longer a block lives, the further apart in time neighbouring
// tiles read the rows they share; with the current kernel, 8-plane runs in
// groups of 4 take 6.44 ms and 12-plane runs 6.99 ms), so on lattices with
// more tiles than resident blocks runs stop at 8 planes (cap); small grids (256x128x128:
// 1.96 waves of 19-plane runs, 0.114 ms, against 0.126 ms for 16-plane runs
// in 2.25 waves) keep the wave count low instead.  2-byte storage, bound by
// instruction issue and with half the bytes per plane in L2, has no cap, and
// on lattices with more tiles than resident blocks long runs cost it little
// (1 + fz/2048: 1024x512x512 FP16, 1 run per group, 27-, 32-, 48-, 64-,
// 86-, 128-, 256- and 512-plane runs take 4.598, 4.567, 4.524, 4.485, 4.506,
// 4.491, 4.614 and 4.700 ms; BF16 is best at 64 too, 4.519 ms); on smaller
// lattices 1 + fz/256 keeps the best shape (512x256x256: 20-plane runs
// 0.5975 ms, 32 0.604, 64 0.604; 256x128x128: 15-plane runs 0.0894 ms, 32
// 0.0933).
int choose_fz(const Geom& g, long long tiles, long long slots, bool cap) {
  int best = g.nz;
  double best_cost = -1.0;
  const double k = (!cap && tiles > slots) ? 2048.0 : 256.0;   // the long-run factor 1 + fz / k
  for (int fz = 4; fz <= g.nz; ++fz) {
    const long long chunks = (g.nz + fz - 1) / fz;
    const long long waves = (tiles * chunks + slots - 1) / slots;
    if (cap && fz > 8 && tiles > slots) continue;
    const double cost = (double)waves * (fz + 2) * (1.0 + fz / k);
    if (best_cost < 0.0 || cost < best_cost) {
      best_cost = cost;
      best = fz;
    }
  }
  return best;
}

// Per device and storage type: the kernels' shared-memory limit is set and
// the SM count and resident blocks per SM of the step kernel are read on
// the first call with that device current (under a lock: several threads,
// or several devices, may make their first calls at once).
template <int P>
cudaError_t fused_device_info(int* slots_per_sm, int* sms) {
  using S = FusedShape<P>;
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static int slots_of[kMaxDev] = {}, sms_of[kMaxDev] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!slots_of[dev]) {
    for (const void* k : {(const void*)fused_kernel<P, false, COLL_SRT>, (const void*)fused_kernel<P, true, COLL_SRT>,
                          (const void*)fused_kernel<P, false, COLL_MRT>, (const void*)fused_kernel<P, true, COLL_MRT>})
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
    for (const void* k : {(const void*)bfused_kernel<P, TX>, (const void*)bpersist_kernel<P, TX>})
      if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
    for (const void* k : {(const void*)bfused_kernel<P, 32>, (const void*)bpersist_kernel<P, 32>})
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FusedShape<P, 32>::smem);
    int n_sm = 0, slots = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&slots, fused_kernel<P, false, COLL_SRT>, S::NT, S::smem);
    if (e != cudaSuccess) return e;
    if (slots < 1) return cudaErrorInvalidConfiguration;
    sms_of[dev] = n_sm;
    slots_of[dev] = slots;
  }
  *slots_per_sm = slots_of[dev];
  *sms = sms_of[dev];
  return cudaSuccess;
}

// Grid of the fused step: z run length, runs per tile column, blocks.
template <int P>
cudaError_t fused_grid(const Geom& g, int fz_req, int grp_req, int* fz, int* nchunks, int* grp,
                       long long* blocks) {
  int slots_per_sm = 0, sms = 0;
  cudaError_t e = fused_device_info<P>(&slots_per_sm, &sms);
  if (e != cudaSuccess) return e;
  const long long tiles = (long long)(g.nx / TX) * (g.ny / FusedShape<P>::TY);
  *fz = fz_req > 0 ? std::min(fz_req, g.nz) : choose_fz(g, tiles, (long long)slots_per_sm * sms, !Prec<P>::dev);
  *nchunks = (g.nz + *fz - 1) / *fz;
  *blocks = tiles * *nchunks;
  // runs per group (a tile's y neighbours are ntx x grp blocks apart in the
  // launch order).  Measured on GB300 (FP32, A-B): 256x128x128 is fastest
  // with one run per group (0.117 ms against 0.127 ms with all 7 runs of a
  // tile together), 512x256x256 within 2 % for 1 to 4, 1024x512x512 with
  // 12-plane runs in groups of 4 (6.5 ms and 21.8 GB of DRAM reads in every
  // launch; 16-plane runs in pairs took 6.4 to 7.8 ms, reading 22 to 29 GB):
  // one run per 4 tile columns (2-byte storage: one run per group, 32-plane
  // runs in ones 6.20 ms on 1024x512x512 FP16, in pairs 6.33 ms)
  const int ntx = g.nx / TX;
  *grp = std::min(grp_req > 0 ? grp_req : (Prec<P>::dev ? 1 : std::max(1, ntx / 4)), *nchunks);
  return *blocks > 0x7fffffffLL ? cudaErrorInvalidConfiguration : cudaSuccess;
}

template <int P>
cudaError_t fused_t(const Geom& g, const Phys& ph, const void* src, void* dst, int* flag, int fz_req,
                    int grp_req, const FusedDiag* diag, unsigned long long stall_ns, cudaStream_t s) {
  using S = FusedShape<P>;
  int fz = 0, nchunks = 0, grp = 0;
  long long blocks = 0;
  cudaError_t e = fused_grid<P>(g, fz_req, grp_req, &fz, &nchunks, &grp, &blocks);
  if (e != cudaSuccess) return e;
  Maps m;
  e = maps_for(P, g, src, &m);
  if (e != cudaSuccess) return e;
  const int ntx = g.nx / TX;
  using T = typename Prec<P>::T;
  DirBases<T> db;
  for (int a = 0; a < Q; ++a) db.p[a] = (T*)dst + (long long)a * g.N;
  if (!diag) {
    const DiagOut none = diag_out(0.0, 0.0, nullptr, nullptr, stall_ns);
    if (ph.coll == COLL_MRT)
      fused_kernel<P, false, COLL_MRT><<<(unsigned)blocks, S::NT, S::smem, s>>>(m, g, ph, (T*)dst, flag, ntx, nchunks,
                                                                             fz, grp, none, db);
    else
      fused_kernel<P, false, COLL_SRT><<<(unsigned)blocks, S::NT, S::smem, s>>>(m, g, ph, (T*)dst, flag, ntx, nchunks,
                                                                             fz, grp, none, db);
    return cudaGetLastError();
  }
  const long long row_blocks = (long long)(g.ny / S::TY) * nchunks;
  const size_t need = (size_t)row_blocks * g.nx * 2 + (size_t)blocks * DIAG_NG + (size_t)g.nx * 2;
  if (need > diag->scratch_doubles) return cudaErrorInvalidValue;
  double* slices = diag->scratch;
  double* bl = slices + (size_t)row_blocks * g.nx * 2;
  double* slice_tot = bl + (size_t)blocks * DIAG_NG;
  const DiagOut dg = diag_out(diag->rho_l, diag->rho_v, slices, bl, stall_ns);
  if (ph.coll == COLL_MRT)
    fused_kernel<P, true, COLL_MRT><<<(unsigned)blocks, S::NT, S::smem, s>>>(m, g, ph, (T*)dst, flag, ntx, nchunks,
                                                                          fz, grp, dg, db);
  else
    fused_kernel<P, true, COLL_SRT><<<(unsigned)blocks, S::NT, S::smem, s>>>(m, g, ph, (T*)dst, flag, ntx, nchunks,
                                                                          fz, grp, dg, db);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_diag_reduce(g, (int)row_blocks, (int)blocks, slices, bl, slice_tot, diag->out, diag->ring_count,
                            diag->ring_cap, s);
}

template <int P>
size_t fused_scratch_t(const Geom& g, int fz_req) {
  int fz = 0, nchunks = 0, grp = 0;
  long long blocks = 0;
  if (fused_grid<P>(g, fz_req, 0, &fz, &nchunks, &grp, &blocks) != cudaSuccess) return 0;
  return (size_t)(g.ny / FusedShape<P>::TY) * nchunks * g.nx * 2 + (size_t)blocks * DIAG_NG + (size_t)g.nx * 2;
}

}  // namespace

cudaError_t fused_launch_shape(int precision, const Geom& g, int fz_req, int grp_req, int* fz, int* grp) {
  int nchunks = 0;
  long long blocks = 0;
  switch (precision) {
    case LBM_F32: return fused_grid<LBM_F32>(g, fz_req, grp_req, fz, &nchunks, grp, &blocks);
    case LBM_F16DEV: return fused_grid<LBM_F16DEV>(g, fz_req, grp_req, fz, &nchunks, grp, &blocks);
    case LBM_BF16DEV: return fused_grid<LBM_BF16DEV>(g, fz_req, grp_req, fz, &nchunks, grp, &blocks);
  }
  return cudaErrorInvalidValue;
}

bool fused_applicable(const Geom& g, int precision) {
  return precision != LBM_F64 && g.nx % TX == 0 && g.ny % fused_tile_rows(precision) == 0 && g.nz >= 3;
}

cudaError_t launch_fused(int precision, const Geom& g, const Phys& ph, const void* src, void* dst, int* flag,
                         int fz, int grp, const FusedDiag* diag, unsigned long long stall_ns, cudaStream_t s) {
  if (!fused_applicable(g, precision)) return cudaErrorInvalidValue;
  switch (precision) {
    case LBM_F32: return fused_t<LBM_F32>(g, ph, src, dst, flag, fz, grp, diag, stall_ns, s);
    case LBM_F16DEV: return fused_t<LBM_F16DEV>(g, ph, src, dst, flag, fz, grp, diag, stall_ns, s);
    case LBM_BF16DEV: return fused_t<LBM_BF16DEV>(g, ph, src, dst, flag, fz, grp, diag, stall_ns, s);
  }
  return cudaErrorInvalidValue;
}

// ---- batched single-pass step on padded rows --------------------------------

namespace {

template <int P, int W>
cudaError_t batch_tma_build_t(const BatchTmaInst* in, int count, int fz_req, int grp_req, const void* pool,
                              void* d_table, BatchTmaPlan* plan, cudaStream_t s) {
  using S = FusedShape<P, W>;
  int slots_per_sm = 0, sms = 0;
  cudaError_t e = fused_device_info<P>(&slots_per_sm, &sms);   // the kernels' shared-memory limit
  if (e != cudaSuccess) return e;
  const size_t es = elem_size(P);
  const size_t inst_bytes = align128(sizeof(BTInst) * (size_t)count);
  std::vector<unsigned char> host(inst_bytes + sizeof(Maps) * 2 * (size_t)count);
  BTInst* ti = reinterpret_cast<BTInst*>(host.data());
  Maps* tm = reinterpret_cast<Maps*>(host.data() + inst_bytes);
  const Maps* d_maps = reinterpret_cast<const Maps*>((const unsigned char*)d_table + inst_bytes);
  const int cw = 16 / (int)es;
  long long blocks = 0;
  for (int k = 0; k < count; ++k) {
    const BatchTmaInst& b = in[k];
    if (b.px % cw || b.off_f % cw || b.px < b.g.nx) return cudaErrorInvalidValue;
    BTInst& t = ti[k];
    std::memset(&t, 0, sizeof(t));
    t.g = b.g;
    t.ph = b.ph;
    t.off_f = b.off_f;
    t.px = b.px;
    t.dstride = (long long)b.px * b.g.ny * b.g.nz;
    t.maps = d_maps + 2 * k;
    t.ntx = (b.g.nx + W - 1) / W;
    const int nty = (b.g.ny + S::TY - 1) / S::TY;
    t.fz = std::min(fz_req > 0 ? fz_req : 16, b.g.nz);
    t.nchunks = (b.g.nz + t.fz - 1) / t.fz;
    // runs per block-order group (0: a tile's z runs one after another)
    t.grp = grp_req > 0 ? std::min(grp_req, t.nchunks) : t.nchunks;
    t.block0 = (int)blocks;
    blocks += (long long)t.ntx * nty * t.nchunks;
    for (int arr = 0; arr < 2; ++arr) {
      const void* base = (const unsigned char*)pool + (size_t)(b.off_f + (long long)arr * Q * t.dstride) * es;
      Maps& m = tm[2 * k + arr];
      e = make_map(&m.interior, P, b.g, base, W, S::TY, b.px);
      if (e == cudaSuccess) e = make_map(&m.row, P, b.g, base, W, 1, b.px);
      if (e == cudaSuccess) e = make_map(&m.col, P, b.g, base, cw, S::TY, b.px);
      if (e == cudaSuccess) e = make_map(&m.cor, P, b.g, base, cw, 1, b.px);
      if (e != cudaSuccess) return e;
    }
  }
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  plan->width = W;
  plan->count = count;
  plan->blocks = (int)blocks;
  e = cudaMemcpyAsync(d_table, host.data(), host.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host table goes out of scope
  return e;
}

template <int P>
cudaError_t batch_tma_build_w(int tile_w, const BatchTmaInst* insts, int count, int fz, int grp, const void* pool,
                              void* d_table, BatchTmaPlan* plan, cudaStream_t s) {
  if (tile_w == 32) return batch_tma_build_t<P, 32>(insts, count, fz, grp, pool, d_table, plan, s);
  if (tile_w == TX) return batch_tma_build_t<P, TX>(insts, count, fz, grp, pool, d_table, plan, s);
  return cudaErrorInvalidValue;
}

template <int P, int W>
void batch_tma_launch_t(const void* d_table, const BatchTmaPlan& plan, void* pool, int cur, int* flag,
                        cudaStream_t s) {
  using S = FusedShape<P, W>;
  bfused_kernel<P, W><<<plan.blocks, S::NT, S::smem, s>>>(reinterpret_cast<const BTInst*>(d_table), plan.count,
                                                          (typename Prec<P>::T*)pool, cur, flag);
}

template <int P>
cudaError_t batch_tma_launch_w(const void* d_table, const BatchTmaPlan& plan, void* pool, int cur, int* flag,
                               cudaStream_t s) {
  if (plan.width == 32)
    batch_tma_launch_t<P, 32>(d_table, plan, pool, cur, flag, s);
  else if (plan.width == TX)
    batch_tma_launch_t<P, TX>(d_table, plan, pool, cur, flag, s);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <int P, int W>
cudaError_t batch_tma_persist_t(const void* d_table, const BatchTmaPlan& plan, void* pool, int cur, int nsteps,
                                unsigned* bar, unsigned* tickets, int* flag, unsigned long long stall_ns,
                                cudaStream_t s) {
  using S = FusedShape<P, W>;
  using T = typename Prec<P>::T;
  int slots_per_sm = 0, sms = 0, per_sm = 0;
  cudaError_t e = fused_device_info<P>(&slots_per_sm, &sms);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bpersist_kernel<P, W>, S::NT, S::smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  int items = plan.blocks, count = plan.count;
  const int grid = std::min(items, per_sm * sms);
  e = cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(tickets, 0, sizeof(unsigned) * (size_t)nsteps, s);
  if (e != cudaSuccess) return e;
  const BTInst* t = reinterpret_cast<const BTInst*>(d_table);
  T* pf = (T*)pool;
  void* args[] = {(void*)&t, (void*)&count, (void*)&pf, (void*)&cur, (void*)&nsteps,
                  (void*)&items, (void*)&bar, (void*)&tickets, (void*)&flag, (void*)&stall_ns};
  return cudaLaunchCooperativeKernel((const void*)bpersist_kernel<P, W>, dim3(grid), dim3(S::NT), args, S::smem, s);
}

template <int P>
cudaError_t batch_tma_persist_w(const void* d_table, const BatchTmaPlan& plan, void* pool, int cur, int nsteps,
                                unsigned* bar, unsigned* tickets, int* flag, unsigned long long stall_ns,
                                cudaStream_t s) {
  if (plan.width == 32)
    return batch_tma_persist_t<P, 32>(d_table, plan, pool, cur, nsteps, bar, tickets, flag, stall_ns, s);
  if (plan.width == TX)
    return batch_tma_persist_t<P, TX>(d_table, plan, pool, cur, nsteps, bar, tickets, flag, stall_ns, s);
  return cudaErrorInvalidValue;
}

}  // namespace

size_t batch_tma_table_bytes(int count) {
  return align128(sizeof(BTInst) * (size_t)count) + sizeof(Maps) * 2 * (size_t)count;
}

int batch_tma_row_align(int precision) { return 16 / (int)elem_size(precision); }

cudaError_t batch_tma_build(int precision, int tile_w, const BatchTmaInst* insts, int count, int fz, int grp,
                            const void* pool, void* d_table, BatchTmaPlan* plan, cudaStream_t s) {
  switch (precision) {
    case LBM_F32: return batch_tma_build_w<LBM_F32>(tile_w, insts, count, fz, grp, pool, d_table, plan, s);
    case LBM_F16DEV: return batch_tma_build_w<LBM_F16DEV>(tile_w, insts, count, fz, grp, pool, d_table, plan, s);
    case LBM_BF16DEV: return batch_tma_build_w<LBM_BF16DEV>(tile_w, insts, count, fz, grp, pool, d_table, plan, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t batch_tma_launch(int precision, const void* d_table, const BatchTmaPlan& plan, void* pool, int cur,
                             int* flag, cudaStream_t s) {
  switch (precision) {
    case LBM_F32: return batch_tma_launch_w<LBM_F32>(d_table, plan, pool, cur, flag, s);
    case LBM_F16DEV: return batch_tma_launch_w<LBM_F16DEV>(d_table, plan, pool, cur, flag, s);
    case LBM_BF16DEV: return batch_tma_launch_w<LBM_BF16DEV>(d_table, plan, pool, cur, flag, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t batch_tma_persist_launch(int precision, const void* d_table, const BatchTmaPlan& plan, void* pool,
                                     int cur, int nsteps, unsigned* bar, unsigned* tickets, int* flag,
                                     unsigned long long stall_ns, cudaStream_t s) {
  switch (precision) {
    case LBM_F32:
      return batch_tma_persist_w<LBM_F32>(d_table, plan, pool, cur, nsteps, bar, tickets, flag, stall_ns, s);
    case LBM_F16DEV:
      return batch_tma_persist_w<LBM_F16DEV>(d_table, plan, pool, cur, nsteps, bar, tickets, flag, stall_ns, s);
    case LBM_BF16DEV:
      return batch_tma_persist_w<LBM_BF16DEV>(d_table, plan, pool, cur, nsteps, bar, tickets, flag, stall_ns, s);
  }
  return cudaErrorInvalidValue;
}

size_t fused_diag_scratch_doubles(const Geom& g, int precision, int fz) {
  if (!fused_applicable(g, precision)) return 0;
  switch (precision) {
    case LBM_F32: return fused_scratch_t<LBM_F32>(g, fz);
    case LBM_F16DEV: return fused_scratch_t<LBM_F16DEV>(g, fz);
    case LBM_BF16DEV: return fused_scratch_t<LBM_BF16DEV>(g, fz);
  }
  return 0;
}

}  // namespace lbm
