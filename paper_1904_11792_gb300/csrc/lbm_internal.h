// Host-side internals of liblbm.so: the handle and the kernel launchers each
// translation unit provides.  Not part of the public ABI (include/lbm.h).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_device.cuh"

namespace lbm {

// Streaming modes of one time step.
enum Mode {
  MODE_AB = 0,      // A-B push: read f_a(x) from src, write f*_a to dst at x + c_a
  MODE_AA_EVEN = 1, // AA even step: read slot a at x, write f*_a to slot opp(a) at x
  MODE_AA_ODD = 2   // AA odd step: read slot opp(a) at x - c_a, write f*_a to slot a at x + c_a
};

// Where the pre-collision population a of node x lives for a given state
// layout: LOCAL = slot a at x (A-B, and AA before an even step); GATHER =
// slot opp(a) at x - c_a (AA before an odd step).
enum Layout { LAYOUT_LOCAL = 0, LAYOUT_GATHER = 1 };

size_t elem_size(int precision);

// ---- launchers (lbm_step.cu) ---------------------------------------------
// psi pass: psi[i] = psi(rho_i) for all nodes; flag |= 1 on a non-positive
// or non-finite density.
// vec: two nodes per thread with vector accesses (used when nx is even).
cudaError_t launch_psi(int precision, int layout, bool vec, const Geom& g, const Phys& ph,
                       const void* f, void* psi, int* flag, cudaStream_t s);
// fused force + collision + streaming of one step; block has at most 256
// threads (with vec, block.x counts node pairs); minb (2, 3, 4) = blocks per
// SM the register budget must allow.
cudaError_t launch_collide(int precision, int mode, int minb, bool vec, const Geom& g,
                           const Phys& ph, const void* src, void* dst, const void* psi, dim3 block,
                           cudaStream_t s);

// Default collide-stream block shape of a lattice (lbm_api.cu).
dim3 default_block(const Geom& g);

// force + collision + streaming with the MRT collision (lbm_mrt.cu); the
// same modes and layouts as launch_collide
cudaError_t launch_collide_mrt(int precision, int mode, bool vec, const Geom& g, const Phys& ph,
                               const void* src, void* dst, const void* psi, dim3 block, cudaStream_t s);

// ---- fused single-pass step (lbm_fused.cu) ----------------------------------
// One kernel per A-B step (psi of each tile and its ring computed in shared
// memory); 4- and 2-byte storage, nx % 64 == 0, ny % 4 == 0, nz >= 3.
bool fused_applicable(const Geom& g, int precision);
// fz: z planes per block (0: chosen from the lattice and the GPU).  diag
// (nullable): also reduce the diagnostics of the starting state in the same
// pass and append the record to the ring (or write out[0..DIAG_OUT)); the
// scratch must hold fused_diag_scratch_doubles(g, precision, fz) doubles.
struct FusedDiag {
  double rho_l, rho_v;
  double* scratch;
  size_t scratch_doubles;
  double* out;
  unsigned long long* ring_count;
  int ring_cap;
};
// stall_ns > 0 (test hook): every block also waits that long, bounded, on a
// barrier nothing completes, so the launch takes its timeout path.
// The run length and runs per group the fused step launches with for the
// requested values (0 = automatic).
cudaError_t fused_launch_shape(int precision, const Geom& g, int fz_req, int grp_req, int* fz, int* grp);
// fz: z planes per block (0 = automatic); grp: z runs per group of the
// block order (0 = automatic).
cudaError_t launch_fused(int precision, const Geom& g, const Phys& ph, const void* src, void* dst,
                         int* flag, int fz, int grp, const FusedDiag* diag, unsigned long long stall_ns,
                         cudaStream_t s);
size_t fused_diag_scratch_doubles(const Geom& g, int precision, int fz);

// ---- auxiliary kernels (lbm_aux.cu) ---------------------------------------
struct InitSpec {
  double R0, lambda, eps, phase, rho_l, rho_v, width;
  const double* prof;  // device table, or nullptr for the tanh profile
  int n;
  double d0, dd;
};
cudaError_t launch_init(int precision, const Geom& g, const Phys& ph, const InitSpec& spec,
                        void* f, cudaStream_t s);
// canonical FP64 plane a <-> storage (layout-aware)
cudaError_t launch_get_plane(int precision, int layout, const Geom& g, const Phys& ph,
                             const void* f, int a, double* out, cudaStream_t s);
cudaError_t launch_set_plane(int precision, int layout, const Geom& g, const Phys& ph, void* f,
                             int a, const double* in, cudaStream_t s);
// rho and u = (j + F/2)/rho into four FP64 device arrays (psi must be current)
cudaError_t launch_moments(int precision, int layout, const Geom& g, const Phys& ph,
                           const void* f, const void* psi, double* rho, double* ux, double* uy,
                           double* uz, cudaStream_t s);

// Diagnostics reduction.  scratch must hold diag_scratch_doubles(g) doubles.
size_t diag_scratch_doubles(const Geom& g);
// Results: DIAG_OUT doubles, 0 mass, 1-3 momentum, 4 liquid volume (phi),
// 5 liquid count, 6 min slice area (phi), 7 min slice count, 8 its x,
// 9 max |j|/rho, 10 min rho, 11 max rho, 12 numeric ok (1/0).  A ring
// record holds them plus, at DIAG_OUT, its sequence number and, from
// DIAG_CCL, the droplet counts of a step that also ran the labelling
// (components, components >= 8 nodes, largest, guard error; -1 if it did not).
constexpr int DIAG_OUT = 13;
constexpr int DIAG_NG = 12;   // partial slots per block of the diagnostics reduction
constexpr int DIAG_CCL = 14;
constexpr int DIAG_STRIDE = 20;
// psi (nullable): also write psi of every node and raise flag on a bad
// density (the psi pass of a diagnostic step).  ring_count (nullable):
// append the record to the ring at out instead of writing out[0..12].
cudaError_t launch_diagnostics(int precision, int layout, const Geom& g, const Phys& ph,
                               const void* f, double rho_l, double rho_v, double* scratch,
                               double* out, void* psi, int* flag,
                               unsigned long long* ring_count, int ring_cap, cudaStream_t s);

// Stochastic-rounding step salt (Phys::salt): set to value, or advance by one.
cudaError_t launch_salt(unsigned* salt, bool set, unsigned value, cudaStream_t s);
// Advances the salt word by n (after a launch that ran n steps).
cudaError_t launch_salt_add(unsigned* salt, unsigned n, cudaStream_t s);

// Second and third stage of the diagnostics reduction from partials
// slices[row_blocks][nx][2] and blocks[nblocks][DIAG_NG] (slice_tot: 2 nx
// doubles of scratch; with many block records they are folded in place, so
// blocks is overwritten); arguments after slice_tot as launch_diagnostics.
cudaError_t launch_diag_reduce(const Geom& g, int row_blocks, int nblocks, const double* slices,
                               double* blocks, double* slice_tot, double* out,
                               unsigned long long* ring_count, int ring_cap, cudaStream_t s);

// Connected components of the liquid mask.  labels: N ints; sizes: N ints;
// out3 (device, 4 long long): components, components with >= 8 nodes,
// largest size, error flag (a union-find guard tripped).
cudaError_t launch_ccl(int precision, int layout, const Geom& g, const Phys& ph, const void* f,
                       double threshold, int* labels, int* sizes, long long* out3,
                       cudaStream_t s);

// Appends the counts of the last launch_ccl (out4, device) to the newest
// ring record (fields DIAG_CCL ..).
cudaError_t launch_ccl_ring(const long long* out4, double* ring, const unsigned long long* ring_count,
                            int ring_cap, cudaStream_t s);

// Per-droplet statistics after launch_ccl on the same state: records of
// DROP_REC doubles [root, nodes, sum phi, sum rho, cos/sin sums of the
// angles 2 pi x/nx, 2 pi y/ny, 2 pi z/nz] for the first cap roots met, and
// x-occupancy bit masks of (nx + 31)/32 words per record.  sizes is the CCL
// sizes array (overwritten with record slots); nslot receives the number of
// roots.
constexpr int DROP_REC = 10;
cudaError_t launch_droplets(int precision, int layout, const Geom& g, const Phys& ph, const void* f,
                            double rho_l, double rho_v, const int* labels, int* sizes, double* rec,
                            unsigned* xbits, unsigned* nslot, int cap, cudaStream_t s);


// ---- batched single-pass step on padded rows (lbm_fused.cu) ----------------
// One instance: geometry, physics, element offset of its array 0 in the
// padded pool (arrays 0 and 1 are Q px ny nz elements each) and its row
// pitch px (nx rounded up to batch_tma_row_align elements, 16 bytes).
struct BatchTmaInst {
  Geom g;
  Phys ph;
  long long off_f;
  int px;
};
int batch_tma_row_align(int precision);
// The launch of one step: tile width (32 or 64), instance records, blocks.
struct BatchTmaPlan {
  int width, count, blocks;
};
// Bytes of the device table (instance records and their tensor maps).
size_t batch_tma_table_bytes(int count);
// Encodes the tensor maps, builds the block table for tiles tile_w (32 or
// 64) nodes wide and z runs of fz planes in groups of grp runs (0: all runs
// of a tile one after another), and copies it to d_table (device,
// batch_tma_table_bytes).  FP32, FP16-dev, BF16-dev.  Synchronises s.
cudaError_t batch_tma_build(int precision, int tile_w, const BatchTmaInst* insts, int count, int fz, int grp,
                            const void* pool, void* d_table, BatchTmaPlan* plan, cudaStream_t s);
// One step of every instance: padded pool arrays cur -> cur ^ 1.
cudaError_t batch_tma_launch(int precision, const void* d_table, const BatchTmaPlan& plan, void* pool, int cur,
                             int* flag, cudaStream_t s);
// nsteps such steps in one cooperative launch of persistent blocks: grid
// barriers on *bar (zeroed here), per-step work tickets tickets[nsteps]
// (zeroed here); stall_ns > 0 is the barrier-timeout test hook.
cudaError_t batch_tma_persist_launch(int precision, const void* d_table, const BatchTmaPlan& plan, void* pool,
                                     int cur, int nsteps, unsigned* bar, unsigned* tickets, int* flag,
                                     unsigned long long stall_ns, cudaStream_t s);

// True if LBM_ALLOC_CAP_BYTES is set and a device allocation of `bytes`
// exceeds it (out-of-memory handling without exhausting a GPU).
bool alloc_over_cap(size_t bytes);

}  // namespace lbm

// ---- the handle -------------------------------------------------------------
struct lbm_ctx {
  lbm_config cfg;
  lbm::Geom g;
  lbm::Phys ph;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  int device = 0;

  void* state = nullptr;  // populations: A-B = two arrays, AA = one
  size_t state_bytes = 0;
  bool own_state = false;
  void* psi = nullptr;
  size_t psi_bytes = 0;
  bool own_psi = false;
  int cur = 0;            // A-B: index of the current array
  long long step = 0;
  bool initialized = false;
  double rho_l = 1.0, rho_v = 0.0;

  int* d_flag = nullptr;          // [0] numeric / timeout flag, [2] stochastic-rounding step salt
  double* d_small = nullptr;      // small result buffer (diagnostics out etc.)
  double* d_scratch = nullptr;    // diagnostics partials
  size_t scratch_doubles = 0;
  int* d_labels = nullptr;        // CCL labels and sizes (2 N ints)
  bool diag_ccl = false;          // label droplets at every in-loop diagnostic step
  double* d_drop = nullptr;       // droplet records and x masks (lbm_droplets)
  size_t drop_bytes = 0;

  // CUDA graphs of one chunk of steps, keyed by the A-B array they start on
  // (AA chunks always start on an even step)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_chunk = 0;            // steps per captured chunk
  bool use_graph = true;
  dim3 block{0, 0, 0};
  int minb = 0;                   // collide kernel register budget variant (0 = auto)
  bool vec = true;                // two nodes per thread (when nx is even)
  bool fused = true;              // single-pass fused step on non-diagnostic A-B steps (where it applies)
  int fused_fz = 0;               // z planes per block of the fused step (0 = automatic)
  int fused_group = 0;            // z runs per group of its block order (0 = automatic)
  unsigned long long fused_stall_test_ns = 0;   // test hook of the fused step's timeout path

  // diagnostics inside the time loop: every diag_interval steps the psi
  // pass also reduces the diagnostics into a device ring of records
  int diag_interval = 0;
  static constexpr int kRing = 1024;
  double* d_ring = nullptr;                 // kRing * DIAG_STRIDE doubles
  unsigned long long* d_ring_count = nullptr;
  std::vector<long long> diag_steps;        // step of every record launched
  long long diag_fetched = 0;               // records already returned

  // kernel timing
  bool kernel_timing = false;
  std::vector<cudaEvent_t> ev_free;
  struct Pending {
    int k;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  long long t_launches[3] = {0, 0, 0};
  double t_ms[3] = {0.0, 0.0, 0.0};
};
