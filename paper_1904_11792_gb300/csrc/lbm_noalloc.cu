// Diagnostics of a population array without any device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need the
// diagnostics: code running while a CUDA graph is being captured on another
// stream of the process (an allocation there can synchronise the device or
// invalidate the capture), code inside a custom allocator or memory-pool
// callback (re-entering the allocator), and embedding hosts that forbid the
// library from growing device memory on its own after start-up.  For them
// lbm_diagnostics_noalloc reduces the diagnostics with the same kernels as
// lbm_diagnostics, but the reduction's partial sums live in a fixed
// statically allocated device array instead of a buffer the handle allocates.
#include <mutex>
#include <string>

#include "lbm_internal.h"

using namespace lbm;

namespace {

// Scratch for the block and per-slice partial sums: 4 MiB per device that
// loads the library, held until the process exits.
constexpr size_t kNoallocScratchDoubles = 524288;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};
thread_local std::string g_err;

int nfail(int status, const std::string& m) {
  g_err = m;
  return status;
}

}  // namespace

extern "C" {

const char* lbm_noalloc_last_error(void) { return g_err.c_str(); }

size_t lbm_diagnostics_noalloc_max_scratch(void) { return kNoallocScratchDoubles; }

int lbm_diagnostics_noalloc(const void* f, int nx, int ny, int nz, int precision, double rho_ref,
                            double rho_l, double rho_v, double* out, void* stream) {
  if (!f || !out) return nfail(LBM_ERR_ARG, "null populations or output pointer");
  if (nx < 3 || ny < 3 || nz < 3) return nfail(LBM_ERR_ARG, "every lattice dimension must be >= 3");
  if ((long long)nx * ny * nz > 0x7fffffffLL) return nfail(LBM_ERR_ARG, "lattice has more than 2^31-1 nodes");
  if (precision < LBM_F64 || precision > LBM_BF16DEV) return nfail(LBM_ERR_ARG, "unknown precision");
  if (!(rho_l > rho_v)) return nfail(LBM_ERR_ARG, "need rho_l > rho_v");
  const Geom g{nx, ny, nz, (long long)nx * ny * nz};
  const size_t need = diag_scratch_doubles(g);
  if (need > kNoallocScratchDoubles)
    return nfail(LBM_ERR_ARG, "lattice needs " + std::to_string(need) +
                                  " scratch doubles, more than the static maximum of " +
                                  std::to_string(kNoallocScratchDoubles));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(LBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return nfail(LBM_ERR_ARG, "device ordinal beyond 63");
  double* scratch = nullptr;
  {
    // set-up, once per device, with that device current: the device address
    // of the static array (its name in host code is only a host-side stand-in)
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return nfail(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = (double*)p;
    }
    scratch = g_scratch_ptr[dev];
  }
  // The partial kernel writes every slot the final kernel reads, so nothing
  // in the scratch has to start at zero.
  Phys ph{1.0, 0.0, 1.0, rho_ref, LBM_PSI_EXP, 0};
  ph.inv_rho0 = 1.0;
  phys_finalize(ph, precision);
  e = launch_diagnostics(precision, LAYOUT_LOCAL, g, ph, f, rho_l, rho_v, scratch, out, nullptr,
                         nullptr, nullptr, 0, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    // the cached address may belong to a context that no longer exists (a
    // device reset): look it up again on the next call
    std::lock_guard<std::mutex> lock(g_mu);
    g_scratch_ptr[dev] = nullptr;
    return nfail(LBM_ERR_CUDA, std::string("diagnostics launch: ") + cudaGetErrorString(e));
  }
  return LBM_OK;
}

}  // extern "C"
