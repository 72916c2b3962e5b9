// Host runtime and C ABI of liblbm.so (declared in include/lbm.h): handle
// life cycle, device memory, the stream, CUDA-graph replay of the time step,
// kernel timing, checkpoints and the host side of diagnostics.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "lbm_internal.h"

using namespace lbm;

namespace lbm {
inline bool Prec_dev(int precision) { return precision == LBM_F16DEV || precision == LBM_BF16DEV; }

// Default collide-stream block: 256 threads, as long along x (the
// contiguous axis) as the lattice allows; with two nodes per thread (nx
// even) block.x counts node pairs.
dim3 default_block(const Geom& g) {
  const int ux = g.nx % 2 == 0 ? g.nx / 2 : g.nx;
  const unsigned bx = ux >= 256 ? 256 : (ux >= 128 ? 128 : (ux >= 64 ? 64 : 32));
  return dim3(bx, 256 / bx, 1);
}
}  // namespace lbm

namespace {

thread_local std::string g_last_error;

int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

int cuda_fail(cudaError_t e, const char* where) {
  g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

#define CK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// Device allocation with an optional cap (environment LBM_ALLOC_CAP_BYTES)
// so that out-of-memory handling can be exercised without exhausting a GPU.
size_t g_alloc_total = 0;

int dev_alloc(void** p, size_t bytes, const char* what) {
  const char* cap = std::getenv("LBM_ALLOC_CAP_BYTES");
  if (cap && *cap) {
    const unsigned long long c = std::strtoull(cap, nullptr, 10);
    if (g_alloc_total + bytes > c)
      return fail(LBM_ERR_OOM, std::string("allocation of ") + what + " exceeds LBM_ALLOC_CAP_BYTES");
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, what);
  }
  g_alloc_total += bytes;
  return LBM_OK;
}

void dev_free(void* p, size_t bytes) {
  if (p) {
    cudaFree(p);
    g_alloc_total -= bytes;
  }
}

int validate(const lbm_config* c) {
  if (!c) return fail(LBM_ERR_ARG, "null config");
  if (c->nx < 3 || c->ny < 3 || c->nz < 3)
    return fail(LBM_ERR_ARG, "every lattice dimension must be >= 3");
  const long long N = (long long)c->nx * c->ny * c->nz;
  if (N > 0x7fffffffLL) return fail(LBM_ERR_ARG, "lattice has more than 2^31-1 nodes");
  if (!std::isfinite(c->tau) || !(c->tau > 0.5)) return fail(LBM_ERR_ARG, "tau must be finite and > 1/2");
  if (!std::isfinite(c->G)) return fail(LBM_ERR_ARG, "G must be finite");
  if (c->psi_form != LBM_PSI_EXP && c->psi_form != LBM_PSI_RHO) return fail(LBM_ERR_ARG, "unknown psi_form");
  if (!std::isfinite(c->rho0) || !(c->rho0 > 0.0)) return fail(LBM_ERR_ARG, "rho0 must be finite and > 0");
  if (c->precision < LBM_F64 || c->precision > LBM_BF16DEV) return fail(LBM_ERR_ARG, "unknown precision");
  if (c->pattern != LBM_AB && c->pattern != LBM_AA) return fail(LBM_ERR_ARG, "unknown pattern");
  if (!std::isfinite(c->rho_ref)) return fail(LBM_ERR_ARG, "rho_ref must be finite");
  const int bx = c->block_x, by = c->block_y, bz = c->block_z;
  if (bx < 0 || by < 0 || bz < 0) return fail(LBM_ERR_ARG, "negative block size");
  if ((bx || by || bz) && (bx == 0 || by == 0 || bz == 0 || (long long)bx * by * bz > 256 || bz > 64))
    return fail(LBM_ERR_ARG, "block shape must be all zero or have 1..256 threads (bz <= 64)");
  return LBM_OK;
}

void sizes_for(const lbm_config* c, size_t* state, size_t* psi) {
  const size_t N = (size_t)c->nx * c->ny * c->nz;
  const size_t e = elem_size(c->precision);
  const size_t arrays = c->pattern == LBM_AB ? 2 : 1;
  *state = arrays * Q * N * e;
  *psi = N * (c->precision == LBM_F64 ? 8 : 4);
}


// ---- per-handle helpers -----------------------------------------------------

void* array_ptr(lbm_ctx* h, int k) {
  const size_t one = (size_t)Q * h->g.N * elem_size(h->cfg.precision);
  return (char*)h->state + (size_t)k * one;
}

void* cur_array(lbm_ctx* h) { return h->cfg.pattern == LBM_AB ? array_ptr(h, h->cur) : h->state; }

int cur_layout(const lbm_ctx* h) {
  return (h->cfg.pattern == LBM_AA && (h->step & 1)) ? LAYOUT_GATHER : LAYOUT_LOCAL;
}

void drop_graphs(lbm_ctx* h) {
  for (auto& ge : h->graph)
    if (ge) {
      cudaGraphExecDestroy(ge);
      ge = nullptr;
    }
}

cudaEvent_t take_event(lbm_ctx* h) {
  if (!h->ev_free.empty()) {
    cudaEvent_t e = h->ev_free.back();
    h->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// The word of the salt pair step `step` reads: the A-B array index, or the
// step parity for AA (whose graph chunks hold an even number of steps).
int salt_word(const lbm_ctx* h, long long step, int cur) {
  return h->cfg.pattern == LBM_AA ? (int)(step & 1) : (cur & 1);
}

// Default register budget of the collide-stream kernel (blocks of 256
// threads per SM), as measured on the 1024x512x512 lattice: 3 for the
// one-node kernel and for the AA even step's two-node kernel (local loads
// and stores: no spills at 80 registers); for the AA odd step's two-node
// kernel 3 with 2-byte storage (6.93 ms per FP16 AA step against 7.65 with
// 2, although it spills a little at 80 registers) and 2 otherwise (FP32:
// 9.11 ms against 9.84); 2 for the A-B step's two-node kernel (no spills at
// <= 128 registers).
int auto_minb(bool vec, int mode, int precision) {
  if (!vec || mode == MODE_AA_EVEN) return 3;
  if (mode == MODE_AA_ODD && (precision == LBM_F16DEV || precision == LBM_BF16DEV)) return 3;
  return 2;
}

// Enqueues one time step on stream s.  `phase` is the step parity (AA) or
// the index of the current array (A-B).  With timing on, each kernel is
// bracketed by events on s.
int enqueue_step(lbm_ctx* h, cudaStream_t s, long long step, int cur, bool timed) {
  const int prec = h->cfg.precision;
  const bool aa = h->cfg.pattern == LBM_AA;
  const int layout = (aa && (step & 1)) ? LAYOUT_GATHER : LAYOUT_LOCAL;
  const void* src = aa ? h->state : array_ptr(h, cur);
  void* dst = aa ? h->state : array_ptr(h, cur ^ 1);
  const int mode = aa ? ((step & 1) ? MODE_AA_ODD : MODE_AA_EVEN) : MODE_AB;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  const bool diag_step = h->diag_interval > 0 && step % h->diag_interval == 0;
  const bool fused = h->fused && !aa && fused_applicable(h->g, prec);
  // stochastic-rounding salt: a pair of words, read and advanced by the
  // step's collision kernel; the word a step reads follows the A-B array
  // (AA: the step parity), so graph replays and eager steps agree
  Phys ph = h->ph;
  if (Prec_dev(prec) && h->ph.sr) {
    const int w = salt_word(h, step, cur);
    ph.salt = (const unsigned*)(h->d_flag + 2 + w);
    ph.salt_next = (unsigned*)(h->d_flag + 2 + (w ^ 1));
  }
  // a diagnostic step runs fused too when the scratch holds its partials
  const bool fused_diag =
      fused && diag_step && h->d_scratch && fused_diag_scratch_doubles(h->g, prec, h->fused_fz) <= h->scratch_doubles;
  if (fused && (!diag_step || fused_diag)) {
    // single pass: psi of each tile is computed from the staged populations
    if (timed) {
      e0 = take_event(h);
      e1 = take_event(h);
      CK(cudaEventRecord(e0, s));
    }
    if (diag_step) {
      const FusedDiag fd{h->rho_l, h->rho_v, h->d_scratch, h->scratch_doubles, h->d_ring, h->d_ring_count,
                         lbm_ctx::kRing};
      CK(launch_fused(prec, h->g, ph, src, dst, h->d_flag, h->fused_fz, h->fused_group, &fd, h->fused_stall_test_ns, s));
    } else {
      CK(launch_fused(prec, h->g, ph, src, dst, h->d_flag, h->fused_fz, h->fused_group, nullptr, h->fused_stall_test_ns, s));
    }
    if (timed) {
      CK(cudaEventRecord(e1, s));
      h->pending.push_back({2, e0, e1});
    }
    if (diag_step && h->diag_ccl) {
      long long* d4 = (long long*)(h->d_small + 32);
      CK(launch_ccl(prec, layout, h->g, h->ph, src, 0.5 * (h->rho_l + h->rho_v), h->d_labels,
                    h->d_labels + h->g.N, d4, s));
      CK(launch_ccl_ring(d4, h->d_ring, h->d_ring_count, lbm_ctx::kRing, s));
    }
    return LBM_OK;
  }
  if (timed) {
    e0 = take_event(h);
    e1 = take_event(h);
    e2 = take_event(h);
    CK(cudaEventRecord(e0, s));
  }
  if (diag_step) {
    CK(launch_diagnostics(prec, layout, h->g, h->ph, src, h->rho_l, h->rho_v, h->d_scratch, h->d_ring,
                          h->psi, h->d_flag, h->d_ring_count, lbm_ctx::kRing, s));
    if (h->diag_ccl) {
      long long* d4 = (long long*)(h->d_small + 32);
      CK(launch_ccl(prec, layout, h->g, h->ph, src, 0.5 * (h->rho_l + h->rho_v), h->d_labels,
                    h->d_labels + h->g.N, d4, s));
      CK(launch_ccl_ring(d4, h->d_ring, h->d_ring_count, lbm_ctx::kRing, s));
    }
  } else {
    CK(launch_psi(prec, layout, h->vec, h->g, h->ph, src, h->psi, h->d_flag, s));
  }
  if (timed) CK(cudaEventRecord(e1, s));
  const bool vec = h->vec && (h->g.nx % 2 == 0);
  const int minb = h->minb ? h->minb : auto_minb(vec, mode, prec);
  if (h->ph.coll == COLL_MRT)
    CK(launch_collide_mrt(prec, mode, vec, h->g, ph, src, dst, h->psi, h->block, s));
  else
    CK(launch_collide(prec, mode, minb, vec, h->g, ph, src, dst, h->psi, h->block, s));
  if (timed) {
    CK(cudaEventRecord(e2, s));
    h->pending.push_back({0, e0, e1});
    h->pending.push_back({1, e1, e2});
  }
  return LBM_OK;
}

int settle_timing(lbm_ctx* h) {
  if (h->pending.empty()) return LBM_OK;
  CK(cudaStreamSynchronize(h->stream));
  // events shared between consecutive kernels are returned once
  std::vector<cudaEvent_t> seen;
  for (auto& p : h->pending) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p.a, p.b));
    h->t_launches[p.k] += 1;
    h->t_ms[p.k] += ms;
    seen.push_back(p.a);
    seen.push_back(p.b);
  }
  h->pending.clear();
  for (size_t i = 0; i < seen.size(); ++i) {
    bool dup = false;
    for (size_t k = 0; k < i; ++k) dup |= seen[k] == seen[i];
    for (auto e : h->ev_free) dup |= e == seen[i];
    if (!dup) h->ev_free.push_back(seen[i]);
  }
  return LBM_OK;
}

// Steps per captured graph: 2 without in-loop diagnostics; with them, the
// diagnostic interval k (2k for AA when k is odd, so every chunk starts on
// an even step).  Chunks are replayed only from steps that are multiples of
// the chunk length, so the diagnostic steps inside a chunk are fixed.
int chunk_len(const lbm_ctx* h) {
  const int k = h->diag_interval;
  if (k <= 0) return 2;
  if (h->cfg.pattern == LBM_AA && (k & 1)) return 2 * k;
  return k;
}

// Captures chunk_len() consecutive steps starting at array `phase` (A-B; 0
// for AA) into an executable graph.  Capture runs on a private stream
// (capture is not allowed on the legacy default stream); the graph is
// launched on the handle's stream.
int capture_chunk(lbm_ctx* h, int phase) {
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  int rc = LBM_OK;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    return cuda_fail(e, "cudaStreamBeginCapture");
  }
  const int C = chunk_len(h);
  for (int k = 0; k < C && rc == LBM_OK; ++k) {
    // step numbers relative to a chunk start (a multiple of C): the same
    // parity and the same diagnostic steps as every replay
    rc = enqueue_step(h, cs, k, phase ^ (k & 1), false);
  }
  e = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  if (rc != LBM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->graph[phase], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    h->graph[phase] = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  return LBM_OK;
}

// Diagnostics partials: room for the two-kernel reduction and, where the
// fused step applies, for the fused step's (which depends on its z runs).
int ensure_scratch(lbm_ctx* h) {
  size_t need = diag_scratch_doubles(h->g);
  if (h->fused && h->cfg.pattern == LBM_AB)
    need = std::max(need, fused_diag_scratch_doubles(h->g, h->cfg.precision, h->fused_fz));
  if (h->d_scratch && h->scratch_doubles >= need) return LBM_OK;
  if (h->d_scratch) dev_free(h->d_scratch, h->scratch_doubles * sizeof(double));
  h->d_scratch = nullptr;
  h->scratch_doubles = 0;
  int rc = dev_alloc((void**)&h->d_scratch, need * sizeof(double), "diagnostics scratch");
  if (rc == LBM_OK) h->scratch_doubles = need;
  return rc;
}

int ensure_labels(lbm_ctx* h) {
  if (h->d_labels) return LBM_OK;
  return dev_alloc((void**)&h->d_labels, (size_t)h->g.N * 2 * sizeof(int), "labels");
}

int ensure_ring(lbm_ctx* h) {
  if (h->d_ring) return LBM_OK;
  int rc = dev_alloc((void**)&h->d_ring, sizeof(double) * DIAG_STRIDE * lbm_ctx::kRing, "diagnostics ring");
  if (rc) return rc;
  rc = dev_alloc((void**)&h->d_ring_count, sizeof(unsigned long long), "ring counter");
  if (rc) return rc;
  CK(cudaMemsetAsync(h->d_ring_count, 0, sizeof(unsigned long long), h->stream));
  return LBM_OK;
}

void fill_diag(lbm_diag* out, const double* r, long long step) {
  out->step = step;
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
  out->droplets = -1;
  out->droplets_min8 = -1;
  out->largest_droplet = -1;
}

// One FP64 plane of N doubles for host transfers (moments, populations).
int with_plane(lbm_ctx* h, double** plane) {
  return dev_alloc((void**)plane, (size_t)h->g.N * sizeof(double), "transfer plane");
}

struct StateHeader {
  char magic[8];
  int version, precision, pattern, nx, ny, nz, cur, pad;
  long long step;
  double rho_l, rho_v;
};

}  // namespace

extern "C" {

void lbm_config_default(lbm_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->nx = c->ny = c->nz = 3;
  c->tau = 1.0;
  c->G = 0.0;
  c->psi_form = LBM_PSI_EXP;
  c->rho0 = 1.0;
  c->precision = LBM_F32;
  c->pattern = LBM_AB;
  c->rho_ref = 0.0;
}

int lbm_required_bytes(const lbm_config* cfg, size_t* state_bytes, size_t* psi_bytes) {
  int rc = validate(cfg);
  if (rc) return rc;
  size_t s, p;
  sizes_for(cfg, &s, &p);
  if (state_bytes) *state_bytes = s;
  if (psi_bytes) *psi_bytes = p;
  return LBM_OK;
}

const char* lbm_last_error(void) { return g_last_error.c_str(); }

const char* lbm_strerror(int status) {
  switch (status) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_OOM: return "out of device memory";
    case LBM_ERR_NUMERIC: return "non-positive or non-finite density";
    case LBM_ERR_TIMEOUT: return "bounded device wait timed out";
    case LBM_ERR_STATE: return "invalid state for this call";
  }
  return "unknown status";
}

int lbm_lattice(int* c, double* w) {
  for (int a = 0; a < Q; ++a) {
    if (c) {
      c[3 * a] = cx(a);
      c[3 * a + 1] = cy(a);
      c[3 * a + 2] = cz(a);
    }
    if (w) w[a] = wgt(a);
  }
  return LBM_OK;
}

void lbm_destroy(lbm_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  drop_graphs(h);
  for (auto& p : h->pending) {
    h->ev_free.push_back(p.a);
    h->ev_free.push_back(p.b);
  }
  std::vector<cudaEvent_t> uniq;
  for (auto e : h->ev_free) {
    bool dup = false;
    for (auto u : uniq) dup |= u == e;
    if (!dup) uniq.push_back(e);
  }
  for (auto e : uniq) cudaEventDestroy(e);
  if (h->own_state) dev_free(h->state, h->state_bytes);
  if (h->own_psi) dev_free(h->psi, h->psi_bytes);
  dev_free(h->d_flag, sizeof(int) * 4);
  dev_free(h->d_small, sizeof(double) * 64);
  dev_free(h->d_scratch, h->scratch_doubles * sizeof(double));
  dev_free(h->d_labels, (size_t)h->g.N * 2 * sizeof(int));
  dev_free(h->d_drop, h->drop_bytes);
  dev_free(h->d_ring, sizeof(double) * DIAG_STRIDE * lbm_ctx::kRing);
  dev_free(h->d_ring_count, sizeof(unsigned long long));
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
}

lbm_handle lbm_create_ex(const lbm_config* cfg) {
  if (validate(cfg) != LBM_OK) return nullptr;
  lbm_ctx* h = new (std::nothrow) lbm_ctx();
  if (!h) {
    fail(LBM_ERR_OOM, "host allocation failed");
    return nullptr;
  }
  h->cfg = *cfg;
  h->g = Geom{cfg->nx, cfg->ny, cfg->nz, (long long)cfg->nx * cfg->ny * cfg->nz};
  // stochastic rounding is on by default for the reduced-precision forms
  h->ph = Phys{cfg->tau, cfg->G, cfg->rho0, cfg->rho_ref, cfg->psi_form,
               cfg->precision >= LBM_F16DEV ? 1 : 0, COLL_SRT, 1.19, 1.4, 1.2, 1.4, 1.98};
  h->ph.inv_rho0 = 1.0 / cfg->rho0;
  phys_finalize(h->ph, cfg->precision);
  h->block = (cfg->block_x && cfg->block_y && cfg->block_z)
                 ? dim3(cfg->block_x, cfg->block_y, cfg->block_z)
                 : default_block(h->g);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) {
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, dev);
    if (e == cudaSuccess && !(prop.major == 10 && prop.minor == 3)) {
      fail(LBM_ERR_CUDA, "liblbm.so is built for sm_103a (GB300); device has compute capability " +
                             std::to_string(prop.major) + "." + std::to_string(prop.minor));
      delete h;
      return nullptr;
    }
  }
  if (e != cudaSuccess) {
    cuda_fail(e, "cudaGetDevice");
    delete h;
    return nullptr;
  }
  h->device = dev;
  sizes_for(cfg, &h->state_bytes, &h->psi_bytes);
  int rc = LBM_OK;
  if (cfg->stream) {
    h->stream = (cudaStream_t)cfg->stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaStreamCreate");
    h->stream = h->own_stream;
  }
  if (rc == LBM_OK) {
    if (cfg->ext_state) {
      if (cfg->ext_state_bytes < h->state_bytes)
        rc = fail(LBM_ERR_ARG, "ext_state_bytes smaller than required");
      h->state = cfg->ext_state;
    } else {
      rc = dev_alloc(&h->state, h->state_bytes, "populations");
      h->own_state = rc == LBM_OK;
    }
  }
  if (rc == LBM_OK) {
    if (cfg->ext_psi) {
      if (cfg->ext_psi_bytes < h->psi_bytes) rc = fail(LBM_ERR_ARG, "ext_psi_bytes smaller than required");
      h->psi = cfg->ext_psi;
    } else {
      rc = dev_alloc(&h->psi, h->psi_bytes, "psi");
      h->own_psi = rc == LBM_OK;
    }
  }
  if (rc == LBM_OK) rc = dev_alloc((void**)&h->d_flag, sizeof(int) * 4, "flag");
  if (rc == LBM_OK) h->ph.salt = (const unsigned*)(h->d_flag + 2);
  if (rc == LBM_OK) rc = dev_alloc((void**)&h->d_small, sizeof(double) * 64, "results");
  if (rc == LBM_OK) {
    e = cudaMemsetAsync(h->d_flag, 0, sizeof(int) * 4, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->state, 0, h->state_bytes, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "initial clear");
  }
  if (rc != LBM_OK) {
    std::string msg = g_last_error;
    lbm_destroy(h);
    g_last_error = msg;
    return nullptr;
  }
  return h;
}

lbm_handle lbm_create(int nx, int ny, int nz, double tau, double G, int psi_form) {
  lbm_config c;
  lbm_config_default(&c);
  c.nx = nx;
  c.ny = ny;
  c.nz = nz;
  c.tau = tau;
  c.G = G;
  c.psi_form = psi_form;
  return lbm_create_ex(&c);
}

int lbm_set_stream(lbm_handle h, void* stream) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  CK(cudaStreamSynchronize(h->stream));
  h->stream = stream ? (cudaStream_t)stream : h->own_stream;
  if (!h->stream) {
    CK(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
    h->stream = h->own_stream;
  }
  return LBM_OK;
}

int lbm_set_option(lbm_handle h, const char* key, double v) {
  if (!h || !key) return fail(LBM_ERR_ARG, "null handle or key");
  const std::string k(key);
  if (!std::isfinite(v)) return fail(LBM_ERR_ARG, "option value must be finite");
  if (k == "tau") {
    if (!(v > 0.5)) return fail(LBM_ERR_ARG, "tau must be > 1/2");
    h->ph.tau = h->cfg.tau = v;
    phys_finalize(h->ph, h->cfg.precision);
    drop_graphs(h);
  } else if (k == "G") {
    h->ph.G = h->cfg.G = v;
    phys_finalize(h->ph, h->cfg.precision);
    drop_graphs(h);
  } else if (k == "rho_l") {
    h->rho_l = v;
    drop_graphs(h);   // the in-loop diagnostics capture the densities
  } else if (k == "rho_v") {
    h->rho_v = v;
    drop_graphs(h);
  } else if (k == "graph") {
    h->use_graph = v != 0.0;
  } else if (k == "stochastic_rounding") {
    h->ph.sr = v != 0.0 ? 1 : 0;
    drop_graphs(h);
  } else if (k == "collision") {
    if (v != 0.0 && v != 1.0) return fail(LBM_ERR_ARG, "collision must be 0 (SRT) or 1 (MRT)");
    h->ph.coll = v != 0.0 ? COLL_MRT : COLL_SRT;
    drop_graphs(h);
  } else if (k == "mrt_s_e" || k == "mrt_s_eps" || k == "mrt_s_q" || k == "mrt_s_pi" || k == "mrt_s_m") {
    if (!(v > 0.0 && v < 2.0)) return fail(LBM_ERR_ARG, "MRT relaxation rates must lie in (0, 2)");
    if (k == "mrt_s_e") h->ph.s_e = v;
    if (k == "mrt_s_eps") h->ph.s_eps = v;
    if (k == "mrt_s_q") h->ph.s_q = v;
    if (k == "mrt_s_pi") h->ph.s_pi = v;
    if (k == "mrt_s_m") h->ph.s_m = v;
    drop_graphs(h);
  } else if (k == "fused") {
    h->fused = v != 0.0;
    drop_graphs(h);
    if (h->diag_interval > 0) {
      int rc = ensure_scratch(h);
      if (rc) return rc;
    }
  } else if (k == "fused_stall_test") {
    if (!(v >= 0.0 && v <= 10.0)) return fail(LBM_ERR_ARG, "fused_stall_test must be in 0..10 ms");
    h->fused_stall_test_ns = (unsigned long long)(v * 1e6);
    drop_graphs(h);
  } else if (k == "fused_group") {
    const long long gr = (long long)v;
    if (gr < 0 || gr > (1LL << 20) || (double)gr != v)
      return fail(LBM_ERR_ARG, "fused_group must be a non-negative integer");
    h->fused_group = (int)gr;
    drop_graphs(h);
  } else if (k == "fused_fz") {
    const long long z = (long long)v;
    if (z < 0 || z > h->g.nz || (double)z != v) return fail(LBM_ERR_ARG, "fused_fz must be an integer in 0..nz");
    h->fused_fz = (int)z;
    drop_graphs(h);
    if (h->diag_interval > 0) {
      int rc = ensure_scratch(h);
      if (rc) return rc;
    }
  } else if (k == "vector") {
    h->vec = v != 0.0;
    drop_graphs(h);
  } else if (k == "occupancy") {
    if (v != 0.0 && v != 2.0 && v != 3.0 && v != 4.0) return fail(LBM_ERR_ARG, "occupancy must be 0 (auto), 2, 3 or 4");
    h->minb = (int)v;
    drop_graphs(h);
  } else if (k == "diag_interval") {
    const long long d = (long long)v;
    if (d < 0 || d > 1000000 || (double)d != v) return fail(LBM_ERR_ARG, "diag_interval must be an integer in 0..1e6");
    if (d > 0) {
      int rc = ensure_scratch(h);
      if (rc == LBM_OK) rc = ensure_ring(h);
      if (rc) return rc;
    }
    h->diag_interval = (int)d;
    drop_graphs(h);
  } else if (k == "diag_ccl") {
    if (v != 0.0) {
      int rc = ensure_labels(h);
      if (rc) return rc;
    }
    h->diag_ccl = v != 0.0;
    drop_graphs(h);
  } else if (k == "kernel_timing") {
    if (v != 0.0 && !h->kernel_timing) {
      int rc = settle_timing(h);
      if (rc) return rc;
      for (int c = 0; c < 3; ++c) {
        h->t_launches[c] = 0;
        h->t_ms[c] = 0.0;
      }
    }
    h->kernel_timing = v != 0.0;
  } else if (k == "block_x" || k == "block_y" || k == "block_z") {
    const long long b = (long long)v;
    if (b < 1 || b > 256 || (double)b != v) return fail(LBM_ERR_ARG, "block size must be an integer in 1..256");
    dim3 nb = h->block;
    if (k == "block_x") nb.x = (unsigned)b;
    if (k == "block_y") nb.y = (unsigned)b;
    if (k == "block_z") nb.z = (unsigned)b;
    if ((long long)nb.x * nb.y * nb.z > 256 || nb.z > 64)
      return fail(LBM_ERR_ARG, "block shape has more than 256 threads");
    h->block = nb;
    drop_graphs(h);
  } else {
    return fail(LBM_ERR_ARG, "unknown option " + k);
  }
  return LBM_OK;
}

int lbm_get_option(lbm_handle h, const char* key, double* v) {
  if (!h || !key || !v) return fail(LBM_ERR_ARG, "null argument");
  const std::string k(key);
  if (k == "tau") *v = h->ph.tau;
  else if (k == "G") *v = h->ph.G;
  else if (k == "rho_l") *v = h->rho_l;
  else if (k == "rho_v") *v = h->rho_v;
  else if (k == "graph") *v = h->use_graph;
  else if (k == "diag_interval") *v = h->diag_interval;
  else if (k == "diag_ccl") *v = h->diag_ccl;
  else if (k == "occupancy")
    *v = h->minb ? h->minb
                 : auto_minb(h->vec && h->g.nx % 2 == 0, h->cfg.pattern == LBM_AA ? MODE_AA_ODD : MODE_AB,
                             h->cfg.precision);
  else if (k == "vector") *v = h->vec && (h->g.nx % 2 == 0);
  else if (k == "stochastic_rounding") *v = h->ph.sr;
  else if (k == "fused")
    *v = h->fused && h->cfg.pattern == LBM_AB && fused_applicable(h->g, h->cfg.precision);
  else if (k == "fused_fz") *v = h->fused_fz;
  else if (k == "fused_group") *v = h->fused_group;
  else if (k == "fused_fz_used" || k == "fused_group_used") {
    int fz = 0, grp = 0;
    if (fused_applicable(h->g, h->cfg.precision)) {
      const cudaError_t e = fused_launch_shape(h->cfg.precision, h->g, h->fused_fz, h->fused_group, &fz, &grp);
      if (e != cudaSuccess) return cuda_fail(e, "fused launch shape");
    }
    *v = k == "fused_fz_used" ? fz : grp;
  }
  else if (k == "fused_stall_test") *v = h->fused_stall_test_ns * 1e-6;
  else if (k == "collision") *v = h->ph.coll;
  else if (k == "mrt_s_e") *v = h->ph.s_e;
  else if (k == "mrt_s_eps") *v = h->ph.s_eps;
  else if (k == "mrt_s_q") *v = h->ph.s_q;
  else if (k == "mrt_s_pi") *v = h->ph.s_pi;
  else if (k == "mrt_s_m") *v = h->ph.s_m;
  else if (k == "kernel_timing") *v = h->kernel_timing;
  else if (k == "block_x") *v = h->block.x;
  else if (k == "block_y") *v = h->block.y;
  else if (k == "block_z") *v = h->block.z;
  else if (k == "step") *v = (double)h->step;
  else if (k == "nx") *v = h->g.nx;
  else if (k == "ny") *v = h->g.ny;
  else if (k == "nz") *v = h->g.nz;
  else if (k == "precision") *v = h->cfg.precision;
  else if (k == "pattern") *v = h->cfg.pattern;
  else return fail(LBM_ERR_ARG, "unknown option " + k);
  return LBM_OK;
}

static int init_common(lbm_handle h, const InitSpec& sp) {
  h->step = 0;
  h->cur = 0;
  CK(launch_salt((unsigned*)(h->d_flag + 2), true, 0u, h->stream));
  drop_graphs(h);   // the in-loop diagnostics capture the densities
  CK(launch_init(h->cfg.precision, h->g, h->ph, sp, array_ptr(h, 0), h->stream));
  h->initialized = true;
  return LBM_OK;
}

int lbm_init_ligament(lbm_handle h, double R0, double lambda, double eps, double phase, double rho_l,
                      double rho_v, double width) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  for (double v : {R0, lambda, eps, phase, rho_l, rho_v, width})
    if (!std::isfinite(v)) return fail(LBM_ERR_ARG, "non-finite ligament parameter");
  if (!(rho_l > rho_v) || !(rho_v > 0.0)) return fail(LBM_ERR_ARG, "need rho_l > rho_v > 0");
  if (!(width > 0.0) || !(lambda > 0.0) || !(R0 >= 0.0)) return fail(LBM_ERR_ARG, "need width, lambda > 0, R0 >= 0");
  InitSpec sp{R0, lambda, eps, phase, rho_l, rho_v, width, nullptr, 0, 0.0, 1.0};
  h->rho_l = rho_l;
  h->rho_v = rho_v;
  return init_common(h, sp);
}

int lbm_init_profile(lbm_handle h, double R0, double lambda, double eps, double phase, const double* prof,
                     int n, double d0, double dd) {
  if (!h || !prof) return fail(LBM_ERR_ARG, "null argument");
  if (n < 2 || !(dd > 0.0) || !std::isfinite(d0) || !std::isfinite(dd) || !(lambda > 0.0))
    return fail(LBM_ERR_ARG, "need n >= 2, dd > 0, lambda > 0");
  double lo = prof[0], hi = prof[0];
  for (int k = 0; k < n; ++k) {
    if (!std::isfinite(prof[k]) || !(prof[k] > 0.0)) return fail(LBM_ERR_ARG, "profile must be finite and > 0");
    lo = prof[k] < lo ? prof[k] : lo;
    hi = prof[k] > hi ? prof[k] : hi;
  }
  double* dprof = nullptr;
  int rc = dev_alloc((void**)&dprof, sizeof(double) * n, "profile");
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(dprof, prof, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) {
    dev_free(dprof, sizeof(double) * n);
    return cuda_fail(e, "profile upload");
  }
  InitSpec sp{R0, lambda, eps, phase, hi, lo, 1.0, dprof, n, d0, dd};
  h->rho_l = hi;
  h->rho_v = lo;
  rc = init_common(h, sp);
  e = cudaStreamSynchronize(h->stream);
  dev_free(dprof, sizeof(double) * n);
  if (rc == LBM_OK && e != cudaSuccess) rc = cuda_fail(e, "init_profile");
  return rc;
}

int lbm_step(lbm_handle h, int n) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (n < 0) return fail(LBM_ERR_ARG, "negative step count");
  if (!h->initialized) return fail(LBM_ERR_STATE, "lattice not initialised");
  const bool aa = h->cfg.pattern == LBM_AA;
  const int C = chunk_len(h);
  const int k = h->diag_interval;
  if (h->graph_chunk != C) {
    drop_graphs(h);
    h->graph_chunk = C;
  }
  while (n > 0) {
    if (h->use_graph && !h->kernel_timing && n >= C && h->step % C == 0) {
      const int phase = aa ? 0 : h->cur;
      if (!h->graph[phase]) {
        int rc = capture_chunk(h, phase);
        if (rc) return rc;
      }
      CK(cudaGraphLaunch(h->graph[phase], h->stream));
      if (k > 0)
        for (long long t = h->step; t < h->step + C; t += k) h->diag_steps.push_back(t);
      if (!aa && (C & 1)) h->cur ^= 1;
      h->step += C;
      n -= C;
    } else {
      int rc = enqueue_step(h, h->stream, h->step, h->cur, h->kernel_timing);
      if (rc) return rc;
      if (k > 0 && h->step % k == 0) h->diag_steps.push_back(h->step);
      if (!aa) h->cur ^= 1;
      h->step += 1;
      n -= 1;
    }
  }
  return LBM_OK;
}

int lbm_diag_history(lbm_handle h, lbm_diag* out, int max_records, int* count) {
  if (!h || !count || max_records < 0 || (max_records > 0 && !out)) return fail(LBM_ERR_ARG, "bad argument");
  *count = 0;
  const long long total = (long long)h->diag_steps.size();
  if (!h->d_ring || total == h->diag_fetched) {
    CK(cudaStreamSynchronize(h->stream));
    return LBM_OK;
  }
  unsigned long long dev_total = 0;
  CK(cudaMemcpyAsync(&dev_total, h->d_ring_count, sizeof(dev_total), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if ((long long)dev_total != total) return fail(LBM_ERR_STATE, "diagnostics ring out of step with the host log");
  long long first = h->diag_fetched;
  if (total - first > lbm_ctx::kRing) first = total - lbm_ctx::kRing;  // older records were overwritten
  if (total - first > max_records) first = total - max_records;
  std::vector<double> rec(DIAG_STRIDE);
  int n = 0;
  for (long long r = first; r < total; ++r) {
    const long long slot = r % lbm_ctx::kRing;
    CK(cudaMemcpy(rec.data(), h->d_ring + slot * DIAG_STRIDE, sizeof(double) * DIAG_STRIDE,
                  cudaMemcpyDeviceToHost));
    fill_diag(&out[n], rec.data(), h->diag_steps[(size_t)r]);
    if (rec[DIAG_CCL + 3] != 0.0) return fail(LBM_ERR_TIMEOUT, "connected-component labelling guard tripped");
    out[n].droplets = (int)rec[DIAG_CCL];
    out[n].droplets_min8 = (int)rec[DIAG_CCL + 1];
    out[n].largest_droplet = (long long)rec[DIAG_CCL + 2];
    ++n;
  }
  h->diag_fetched = total;
  *count = n;
  return LBM_OK;
}

int lbm_sync(lbm_handle h) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (flag) {
    CK(cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (flag & 2) return fail(LBM_ERR_TIMEOUT, "a staged copy of the fused step did not complete in time");
    return fail(LBM_ERR_NUMERIC, "a density became non-positive or non-finite");
  }
  return LBM_OK;
}

int lbm_moments(lbm_handle h, double* rho, double* ux, double* uy, double* uz) {
  if (!h) return fail(LBM_ERR_ARG, "null handle");
  if (!h->initialized) return fail(LBM_ERR_STATE, "lattice not initialised");
  const int layout = cur_layout(h);
  const void* f = cur_array(h);
  CK(launch_psi(h->cfg.precision, layout, h->vec, h->g, h->ph, f, h->psi, h->d_flag, h->stream));
  double* plane = nullptr;
  int rc = with_plane(h, &plane);
  if (rc) return rc;
  double* outs[4] = {rho, ux, uy, uz};
  for (int k = 0; k < 4 && rc == LBM_OK; ++k) {
    if (!outs[k]) continue;
    cudaError_t e = launch_moments(h->cfg.precision, layout, h->g, h->ph, f, h->psi, k == 0 ? plane : nullptr,
                                   k == 1 ? plane : nullptr, k == 2 ? plane : nullptr,
                                   k == 3 ? plane : nullptr, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(outs[k], plane, sizeof(double) * h->g.N, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "moments");
  }
  cudaStreamSynchronize(h->stream);
  dev_free(plane, sizeof(double) * h->g.N);
  return rc;
}

int lbm_diagnostics(lbm_handle h, lbm_diag* out, int want_ccl) {
  if (!h || !out) return fail(LBM_ERR_ARG, "null argument");
  if (!h->initialized) return fail(LBM_ERR_STATE, "lattice not initialised");
  int rc = ensure_scratch(h);
  if (rc) return rc;
  const int layout = cur_layout(h);
  const void* f = cur_array(h);
  CK(launch_diagnostics(h->cfg.precision, layout, h->g, h->ph, f, h->rho_l, h->rho_v, h->d_scratch,
                        h->d_small, nullptr, nullptr, nullptr, 0, h->stream));
  double r[DIAG_OUT];
  long long c4[4] = {-1, -1, -1, 0};
  if (want_ccl) {
    rc = ensure_labels(h);
    if (rc) return rc;
    long long* d4 = (long long*)(h->d_small + 32);
    CK(launch_ccl(h->cfg.precision, layout, h->g, h->ph, f, 0.5 * (h->rho_l + h->rho_v), h->d_labels,
                  h->d_labels + h->g.N, d4, h->stream));
    CK(cudaMemcpyAsync(c4, d4, sizeof(c4), cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaMemcpyAsync(r, h->d_small, sizeof(r), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (want_ccl && c4[3]) return fail(LBM_ERR_TIMEOUT, "connected-component labelling guard tripped");
  fill_diag(out, r, h->step);
  out->droplets = (int)c4[0];
  out->droplets_min8 = (int)c4[1];
  out->largest_droplet = c4[2];
  return LBM_OK;
}

int lbm_droplets(lbm_handle h, lbm_droplet* out, int max_droplets, int* count) {
  if (!h || !count || max_droplets < 0 || (max_droplets > 0 && !out)) return fail(LBM_ERR_ARG, "bad argument");
  if (!h->initialized) return fail(LBM_ERR_STATE, "lattice not initialised");
  *count = 0;
  int rc = ensure_labels(h);
  if (rc) return rc;
  const int layout = cur_layout(h);
  const void* f = cur_array(h);
  long long* d4 = (long long*)(h->d_small + 32);
  int* L = h->d_labels;
  int* sizes = h->d_labels + h->g.N;
  CK(launch_ccl(h->cfg.precision, layout, h->g, h->ph, f, 0.5 * (h->rho_l + h->rho_v), L, sizes, d4, h->stream));
  long long c4[4];
  CK(cudaMemcpyAsync(c4, d4, sizeof(c4), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (c4[3]) return fail(LBM_ERR_TIMEOUT, "connected-component labelling guard tripped");
  const long long nd = c4[0];
  *count = (int)nd;
  if (nd == 0) return LBM_OK;
  const int words = (h->g.nx + 31) / 32;
  const size_t rec_bytes = sizeof(double) * DROP_REC * (size_t)nd;
  const size_t need = rec_bytes + sizeof(unsigned) * ((size_t)words * nd + 1);
  if (need > h->drop_bytes) {
    dev_free(h->d_drop, h->drop_bytes);
    h->d_drop = nullptr;
    h->drop_bytes = 0;
    rc = dev_alloc((void**)&h->d_drop, need, "droplet records");
    if (rc) return rc;
    h->drop_bytes = need;
  }
  double* rec = h->d_drop;
  unsigned* xbits = (unsigned*)((char*)h->d_drop + rec_bytes);
  unsigned* nslot = xbits + (size_t)words * nd;
  CK(launch_droplets(h->cfg.precision, layout, h->g, h->ph, f, h->rho_l, h->rho_v, L, sizes, rec, xbits, nslot,
                     (int)nd, h->stream));
  std::vector<double> hr((size_t)DROP_REC * nd);
  std::vector<unsigned> hb((size_t)words * nd);
  unsigned ns = 0;
  CK(cudaMemcpyAsync(hr.data(), rec, rec_bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(hb.data(), xbits, sizeof(unsigned) * hb.size(), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&ns, nslot, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if ((long long)ns != nd) return fail(LBM_ERR_STATE, "droplet roots differ from the component count");
  std::vector<lbm_droplet> d((size_t)nd);
  const double two_pi = 6.283185307179586476925286766559;
  const int dims[3] = {h->g.nx, h->g.ny, h->g.nz};
  for (long long k = 0; k < nd; ++k) {
    const double* r = &hr[(size_t)k * DROP_REC];
    lbm_droplet& o = d[(size_t)k];
    o.first_node = (long long)r[0];
    o.nodes = (long long)r[1];
    o.volume_w = r[2];
    o.mass = r[3];
    for (int a = 0; a < 3; ++a) {
      const double c = r[4 + 2 * a], sn = r[5 + 2 * a];
      double t = std::atan2(sn, c);
      if (t < 0.0) t += two_pi;
      double pos = t / two_pi * dims[a];
      if (pos >= dims[a]) pos -= dims[a];
      o.centroid[a] = pos;
      o.resultant[a] = std::sqrt(c * c + sn * sn) / r[1];
    }
    int xs = 0;
    for (int w = 0; w < words; ++w) xs += __builtin_popcount(hb[(size_t)k * words + w]);
    o.x_slices = xs;
    o.reserved = 0;
  }
  std::sort(d.begin(), d.end(), [](const lbm_droplet& a, const lbm_droplet& b) {
    return a.nodes != b.nodes ? a.nodes > b.nodes : a.first_node < b.first_node;
  });
  const long long n = std::min<long long>(nd, max_droplets);
  for (long long k = 0; k < n; ++k) out[k] = d[(size_t)k];
  return LBM_OK;
}

int lbm_get_populations(lbm_handle h, double* host) {
  if (!h || !host) return fail(LBM_ERR_ARG, "null argument");
  double* plane = nullptr;
  int rc = with_plane(h, &plane);
  if (rc) return rc;
  const int layout = cur_layout(h);
  for (int a = 0; a < Q && rc == LBM_OK; ++a) {
    cudaError_t e = launch_get_plane(h->cfg.precision, layout, h->g, h->ph, cur_array(h), a, plane, h->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(host + (size_t)a * h->g.N, plane, sizeof(double) * h->g.N, cudaMemcpyDeviceToHost,
                          h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "get_populations");
  }
  cudaStreamSynchronize(h->stream);
  dev_free(plane, sizeof(double) * h->g.N);
  return rc;
}

int lbm_set_populations(lbm_handle h, const double* host) {
  if (!h || !host) return fail(LBM_ERR_ARG, "null argument");
  double* plane = nullptr;
  int rc = with_plane(h, &plane);
  if (rc) return rc;
  const int layout = cur_layout(h);
  for (int a = 0; a < Q && rc == LBM_OK; ++a) {
    cudaError_t e = cudaMemcpyAsync(plane, host + (size_t)a * h->g.N, sizeof(double) * h->g.N,
                                    cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
      e = launch_set_plane(h->cfg.precision, layout, h->g, h->ph, cur_array(h), a, plane, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "set_populations");
  }
  cudaStreamSynchronize(h->stream);
  dev_free(plane, sizeof(double) * h->g.N);
  if (rc == LBM_OK) h->initialized = true;
  return rc;
}

int lbm_state_bytes(lbm_handle h, size_t* bytes) {
  if (!h || !bytes) return fail(LBM_ERR_ARG, "null argument");
  *bytes = sizeof(StateHeader) + (size_t)Q * h->g.N * elem_size(h->cfg.precision);
  return LBM_OK;
}

int lbm_save_state(lbm_handle h, void* host, size_t bytes) {
  size_t need = 0;
  int rc = lbm_state_bytes(h, &need);
  if (rc) return rc;
  if (!host || bytes < need) return fail(LBM_ERR_ARG, "buffer too small for the state");
  StateHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, "LBMD3Q19", 8);
  hd.version = 1;
  hd.precision = h->cfg.precision;
  hd.pattern = h->cfg.pattern;
  hd.nx = h->g.nx;
  hd.ny = h->g.ny;
  hd.nz = h->g.nz;
  hd.cur = 0;
  hd.step = h->step;
  hd.rho_l = h->rho_l;
  hd.rho_v = h->rho_v;
  std::memcpy(host, &hd, sizeof(hd));
  CK(cudaMemcpyAsync((char*)host + sizeof(hd), cur_array(h), need - sizeof(hd), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_load_state(lbm_handle h, const void* host, size_t bytes) {
  size_t need = 0;
  int rc = lbm_state_bytes(h, &need);
  if (rc) return rc;
  if (!host || bytes < need) return fail(LBM_ERR_ARG, "buffer too small for the state");
  StateHeader hd;
  std::memcpy(&hd, host, sizeof(hd));
  if (std::memcmp(hd.magic, "LBMD3Q19", 8) != 0 || hd.version != 1)
    return fail(LBM_ERR_ARG, "not a saved lattice state");
  if (hd.precision != h->cfg.precision || hd.pattern != h->cfg.pattern || hd.nx != h->g.nx || hd.ny != h->g.ny ||
      hd.nz != h->g.nz)
    return fail(LBM_ERR_ARG, "saved state has another size, precision or pattern");
  h->cur = 0;
  h->step = hd.step;
  CK(launch_salt((unsigned*)(h->d_flag + 2 + salt_word(h, h->step, h->cur)), true, (unsigned)hd.step, h->stream));
  h->rho_l = hd.rho_l;
  h->rho_v = hd.rho_v;
  CK(cudaMemcpyAsync(array_ptr(h, 0), (const char*)host + sizeof(hd), need - sizeof(hd),
                     cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->initialized = true;
  return LBM_OK;
}

int lbm_kernel_time(lbm_handle h, int k, long long* launches, double* ms) {
  if (!h || k < 0 || k > 2) return fail(LBM_ERR_ARG, "bad handle or kernel class");
  int rc = settle_timing(h);
  if (rc) return rc;
  if (launches) *launches = h->t_launches[k];
  if (ms) *ms = h->t_ms[k];
  return LBM_OK;
}

}  // extern "C"

namespace lbm {
// The allocation cap of LBM_ALLOC_CAP_BYTES for one request of `bytes`
// (the batched form's pools; the single lattice also counts what it holds).
bool alloc_over_cap(size_t bytes) {
  const char* cap = std::getenv("LBM_ALLOC_CAP_BYTES");
  return cap && *cap && bytes > std::strtoull(cap, nullptr, 10);
}
}  // namespace lbm

