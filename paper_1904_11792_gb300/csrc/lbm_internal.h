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
cudaError_t launch_psi(int precision, int layout, const Geom& g, const Phys& ph, const void* f,
                       void* psi, int* flag, cudaStream_t s);
// fused force + collision + streaming of one step.
cudaError_t launch_collide(int precision, int mode, const Geom& g, const Phys& ph, const void* src,
                           void* dst, const void* psi, dim3 block, cudaStream_t s);

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
// out (device) receives DIAG_OUT doubles in the order of the oracle's
// diagnostics; see lbm_aux.cu.
constexpr int DIAG_OUT = 13;
cudaError_t launch_diagnostics(int precision, int layout, const Geom& g, const Phys& ph,
                               const void* f, double rho_l, double rho_v, double* scratch,
                               double* out, cudaStream_t s);

// Connected components of the liquid mask.  labels: N ints; sizes: N ints;
// out3 (device, 4 long long): components, components with >= 8 nodes,
// largest size, error flag (a union-find guard tripped).
cudaError_t launch_ccl(int precision, int layout, const Geom& g, const Phys& ph, const void* f,
                       double threshold, int* labels, int* sizes, long long* out3,
                       cudaStream_t s);

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

  int* d_flag = nullptr;          // numeric flag
  double* d_small = nullptr;      // small result buffer (diagnostics out etc.)
  double* d_scratch = nullptr;    // diagnostics partials
  size_t scratch_doubles = 0;
  int* d_labels = nullptr;        // CCL labels and sizes (2 N ints)

  // CUDA graphs of one A-B/AA step pair, keyed by the phase they start on
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool use_graph = true;
  dim3 block{0, 0, 0};

  // kernel timing
  bool kernel_timing = false;
  std::vector<cudaEvent_t> ev_free;
  struct Pending {
    int k;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  long long t_launches[2] = {0, 0};
  double t_ms[2] = {0.0, 0.0};
};
