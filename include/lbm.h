/*
 * lbm.h - C ABI of the GB300 (sm_103a) D3Q19 pseudo-potential lattice
 * Boltzmann library, liblbm.so.
 *
 * The library advances the single-relaxation-time D3Q19 lattice Boltzmann
 * equation with single-belt Shan-Chen forcing on a periodic Cartesian
 * lattice, as defined in Chiappini, Xue, Falcucci, Sbragaglia, "Ligament
 * break-up simulation through pseudo-potential Lattice Boltzmann Method"
 * (arXiv:1904.11792), section "Numerical model":
 *   Eq. 4   rho = sum_a f_a,  rho u = sum_a c_a f_a
 *   psi(rho) = rho0 (1 - exp(-rho / rho0))   (definition after Eq. 5)
 *   Eq. 5   F = -G psi(x) sum_a w_a psi(x + c_a) c_a
 *   Eq. 6   u' = u + tau F / rho
 *   Eq. 2   f_eq(rho, u') = w_a rho [1 + c.u'/cs2 + (c.u')^2/(2 cs2^2) - u'.u'/(2 cs2)]
 *           (the leading 1 is missing in the paper's print; cs2 = 1/3)
 *   Eq. 3   f_a(x + c_a, t + 1) = f_a - (f_a - f_eq_a) / tau   (force only via Eq. 6)
 * The test case is the perturbed liquid ligament of section "Ligament
 * set-up" (Plateau-Rayleigh break-up).
 *
 * Conventions
 *  - Every call returns an int status (LBM_OK = 0 on success) except the
 *    constructors, which return a handle or NULL; after NULL (or any error)
 *    lbm_last_error() gives a message (per host thread).
 *  - No C++ exception crosses this interface.
 *  - Node index i = x + nx * (y + ny * z), x fastest.  N = nx * ny * nz.
 *  - Canonical population arrays (lbm_get/set_populations) are float64,
 *    19 * N values, direction-major: f[a * N + i], holding the
 *    pre-collision populations of the current time step.
 *  - Canonical direction order (a = 0..18): rest; +x, -x, +y, -y, +z, -z;
 *    then opposite pairs (+x+y, -x-y), (+x-y, -x+y), (+x+z, -x-z),
 *    (+x-z, -x+z), (+y+z, -y-z), (+y-z, -y+z).  Weights 1/3, 1/18, 1/36.
 *  - Host arrays are owned by the caller and must hold the sizes stated.
 *    The library owns all device memory it allocates; buffers passed in
 *    lbm_config.ext_* stay owned by the caller and must outlive the handle.
 *  - A handle is not thread-safe.  All its GPU work goes to one CUDA
 *    stream (lbm_set_stream); calls that return host data synchronise it.
 *  - The library runs only on a CUDA device of compute capability 10.3
 *    (built for sm_103a); there is no CPU fallback.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_Q 19

/* Status codes. */
enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,      /* invalid argument (sizes, tau <= 1/2, non-finite values ...) */
    LBM_ERR_CUDA = 2,     /* a CUDA runtime call failed; see lbm_last_error()              */
    LBM_ERR_OOM = 3,      /* device allocation failed (or exceeded LBM_ALLOC_CAP_BYTES)    */
    LBM_ERR_NUMERIC = 4,  /* a density became non-positive or non-finite                   */
    LBM_ERR_TIMEOUT = 5,  /* a bounded device wait gave up                                 */
    LBM_ERR_STATE = 6     /* call not valid in the current state (e.g. no init yet)        */
};

/* Pseudo-potential functional psi(rho). */
enum {
    LBM_PSI_EXP = 0, /* psi = rho0 (1 - exp(-rho / rho0)), the paper's choice (after Eq. 5) */
    LBM_PSI_RHO = 1  /* psi = rho (a test functional)                                       */
};

/* Storage precision of the populations.  Arithmetic is FP64 for LBM_F64
 * and FP32 otherwise.  The *DEV forms store g_a = f_a - s_a with the shift
 * s_a = w_a rho_ref rounded to the storage precision (FP16 or BF16), which
 * keeps the shift's subtraction and addition exact in FP32 for liquid and
 * vapour populations. */
enum { LBM_F64 = 0, LBM_F32 = 1, LBM_F16DEV = 2, LBM_BF16DEV = 3 };

/* Streaming pattern: two arrays (A-B, push), or one array updated in place
 * with alternating even/odd steps (AA). */
enum { LBM_AB = 0, LBM_AA = 1 };

typedef struct lbm_ctx *lbm_handle;

typedef struct {
    int nx, ny, nz;        /* lattice size, each >= 3                               */
    double tau;            /* relaxation time, > 1/2 (Eq. 3)                         */
    double G;              /* interaction strength of Eq. 5 (signed; < 0 attracts)   */
    int psi_form;          /* LBM_PSI_EXP or LBM_PSI_RHO                             */
    double rho0;           /* reference density of psi, > 0 (paper: 1)               */
    int precision;         /* LBM_F64, LBM_F32, LBM_F16DEV, LBM_BF16DEV              */
    int pattern;           /* LBM_AB or LBM_AA                                       */
    double rho_ref;        /* deviation reference density of the *DEV storage forms  */
    int block_x, block_y, block_z; /* collide-stream block shape (<= 256 threads), 0 = default */
    void *ext_state;       /* optional caller device buffer for the populations      */
    size_t ext_state_bytes;
    void *ext_psi;         /* optional caller device buffer for psi                  */
    size_t ext_psi_bytes;
    void *stream;          /* cudaStream_t to use (cudaStreamLegacy = (void*)1 for the
                              legacy default stream); NULL = a new non-blocking stream */
} lbm_config;

/* Diagnostics of the current state, all sums in FP64 with a fixed
 * reduction order (bitwise reproducible).  Liquid means
 * rho > (rho_l + rho_v) / 2 with the densities given at initialisation
 * (or set by lbm_set_option "rho_l"/"rho_v"); phi = clamp((rho - rho_v) /
 * (rho_l - rho_v), 0, 1) is the weighted liquid fraction. */
typedef struct {
    long long step;            /* time steps done                                  */
    double mass;               /* sum_i rho_i                                      */
    double mom[3];             /* sum_i j_i (bare momentum, Eq. 4)                 */
    double liquid_volume_w;    /* sum_i phi_i                                      */
    long long liquid_count;    /* number of liquid nodes                           */
    double min_slice_area_w;   /* min over x of sum_{y,z} phi                      */
    long long min_slice_count; /* min over x of the liquid nodes of slice x        */
    int min_slice_x;           /* first x where min_slice_count is reached         */
    double neck_radius;        /* sqrt(min_slice_area_w / pi)                      */
    double max_u;              /* max_i |j_i| / rho_i                              */
    double rho_min, rho_max;
    int droplets;              /* connected liquid components (6-conn., periodic),
                                  -1 when not requested                            */
    int droplets_min8;         /* components with at least 8 nodes, -1 if not run  */
    long long largest_droplet; /* node count of the largest component, -1 if not run */
    int numeric_ok;            /* 1 if every rho is finite and positive            */
} lbm_diag;

/* Fills cfg with defaults: F32, AB, psi form EXP, rho0 = 1, rho_ref = 0,
 * default block shape, no external buffers, library stream. */
void lbm_config_default(lbm_config *cfg);

/* Device bytes the populations and psi need for cfg (for ext_* buffers). */
int lbm_required_bytes(const lbm_config *cfg, size_t *state_bytes, size_t *psi_bytes);

/* Creates a lattice.  lbm_create is lbm_create_ex with the defaults above
 * (FP32, A-B).  The populations are zero until an init call.  Returns NULL
 * on error (LBM_ERR_ARG / CUDA / OOM in lbm_last_error()). */
lbm_handle lbm_create(int nx, int ny, int nz, double tau, double G, int psi_form);
lbm_handle lbm_create_ex(const lbm_config *cfg);
void lbm_destroy(lbm_handle h);

const char *lbm_last_error(void);
const char *lbm_strerror(int status);

/* The canonical direction table: c[a * 3 + k] (k = x, y, z) and w[a]. */
int lbm_lattice(int *c, double *w);

/* Uses the given cudaStream_t (NULL = the library's own stream;
 * (void*)1 = cudaStreamLegacy). */
int lbm_set_stream(lbm_handle h, void *stream);

/* Named options (value as double): "tau", "G", "rho_l", "rho_v",
 * "graph" (0/1: replay captured CUDA graphs in lbm_step, default 1),
 * "diag_interval" (k >= 0: every step t with t % k == 0 the psi pass also
 * reduces the diagnostics of the state at t into a device ring, read with
 * lbm_diag_history; 0 = off, the default),
 * "kernel_timing" (0/1: record CUDA events around every kernel of lbm_step;
 * disables graphs), "block_x", "block_y", "block_z" (collide-stream block
 * shape, at most 256 threads), "occupancy" (2, 3 or 4: 256-thread blocks
 * per SM the collide-stream kernel's register budget allows; 0 = auto,
 * the default: 3 for the one-node kernel and the AA even step's two-node
 * kernel, 3 for the AA odd step's with 2-byte storage and 2 otherwise, 2
 * for the A-B step's two-node kernel; get answers the odd step's (AA) or
 * the A-B step's value),
 * "vector" (0/1, default 1: when nx is even each thread updates two
 * neighbouring nodes with 2-element vector loads and stores; block_x then
 * counts node pairs), "fused" (0/1, default 1: A-B steps run as one
 * single-pass kernel that computes psi per tile in shared memory, reading
 * the populations once per step, with a variant that also reduces the
 * in-loop diagnostics on diagnostic steps; applies to FP32,
 * FP16-dev and BF16-dev storage when nx % 64 == 0 and ny % 4 == 0 (FP32) or
 * ny % 8 == 0 (2-byte storage), other
 * lattices take the two-kernel step; results equal the two-kernel step
 * bitwise; lbm_get_option answers whether it applies), "fused_fz" (z planes
 * each block of the fused step marches through; 0 = chosen from the lattice
 * size and the GPU, the default), "fused_group" (the fused step launches
 * its blocks in groups of this many consecutive z runs, the run varying
 * fastest inside a group, then the tile x, then the tile y; 0 = one run
 * per 4 tile columns of 64 nodes (FP32; one run for 2-byte storage), at
 * least one, the default; any value
 * gives the same results), "fused_fz_used" and "fused_group_used" (get
 * only: the run length and runs per group the fused step launches with for
 * the current options; 0 where the fused step does not apply),
 * "fused_stall_test" (a test hook of the
 * failure path, in ms, 0..10, default 0: while > 0 every block of the fused
 * step also waits that long on a barrier that nothing completes, so its
 * bounded wait gives up, the step's result is void and lbm_sync returns
 * LBM_ERR_TIMEOUT; the waits on real copies give up after 2 s),
 * "stochastic_rounding" (0/1, default 1 for LBM_F16DEV / LBM_BF16DEV: the
 * stored deviations are rounded up or down with probability given by the
 * discarded fraction, from a hash of the node index and its post-collision
 * rest population, instead of to nearest; removes the mass bias of
 * round-to-nearest in uniform regions; deterministic), "diag_ccl" (0/1,
 * default 0: every in-loop diagnostic step also labels the liquid
 * components on the GPU, so the records of lbm_diag_history carry the
 * droplet counts; needs 8 N bytes of labels), "collision" (0 = the paper's
 * single-relaxation-time collision with the velocity shift of Eq. 6, the
 * default; 1 = multiple-relaxation-time collision, the operator the
 * paper's conclusions name as its next step: D3Q19 moments of d'Humieres et
 * al. 2002, the Shan-Chen force of Eq. 5 entered by Guo's forcing with
 * u = (j + F/2)/rho; shear moments relax at 1/tau, so nu = (tau - 1/2)/3;
 * the fused step and the two-kernel step both have it), "mrt_s_e",
 * "mrt_s_eps", "mrt_s_q",
 * "mrt_s_pi", "mrt_s_m" (its other rates, each in (0, 2); defaults 1.19,
 * 1.4, 1.2, 1.4, 1.98).  lbm_get_option also answers "step", "nx", "ny", "nz",
 * "precision", "pattern". */
int lbm_set_option(lbm_handle h, const char *key, double value);
int lbm_get_option(lbm_handle h, const char *key, double *value);

/* Ligament initial condition (section "Ligament set-up", Fig. 1):
 * R(x) = R0 (1 + eps cos(2 pi x / lambda + phase)), axis at
 * ((ny-1)/2, (nz-1)/2), rho = rho_v + (rho_l - rho_v)/2 [1 - tanh(2 (r - R(x)) / width)],
 * f_a = w_a rho (zero velocity).  Resets the step count to 0.
 * Requires rho_l > rho_v > 0, width > 0, lambda > 0. */
int lbm_init_ligament(lbm_handle h, double R0, double lambda, double eps, double phase,
                      double rho_l, double rho_v, double width);

/* Same geometry, rho = prof(r - R(x)) from n >= 2 samples prof[k] at
 * d0 + k dd (linear interpolation, clamped).  prof is a host array; rho_l
 * and rho_v (thresholds of the diagnostics) are set to prof's largest and
 * smallest value. */
int lbm_init_profile(lbm_handle h, double R0, double lambda, double eps, double phase,
                     const double *prof, int n, double d0, double dd);

/* Enqueues n >= 0 time steps on the handle's stream and returns without
 * waiting.  Each step computes psi (definition after Eq. 5), the force of
 * Eq. 5, the velocity shift of Eq. 6, the equilibrium of Eq. 2, the BGK
 * relaxation of Eq. 3 and streaming.  Where option "fused" applies (A-B
 * streaming, FP32 or 2-byte storage, nx % 64 == 0, ny % 4 == 0 for FP32 or
 * ny % 8 == 0 for 2-byte storage; the
 * default) a step is one single-pass kernel that computes psi per tile in
 * shared memory (its diagnostic-step variant also reduces the in-loop
 * diagnostics); otherwise it is a psi pass followed by one kernel of force,
 * collision and streaming.  Steps are replayed from captured CUDA graphs
 * unless option "kernel_timing" is on. */
int lbm_step(lbm_handle h, int n);

/* Diagnostics recorded inside lbm_step (option "diag_interval"), oldest
 * first: up to max_records of the records not returned before (the device
 * ring keeps the last 1024).  droplets* are -1 unless option "diag_ccl"
 * was on when the record's step ran.
 * *count receives the number written.  Synchronises. */
int lbm_diag_history(lbm_handle h, lbm_diag *out, int max_records, int *count);

/* Waits for the handle's stream; LBM_ERR_NUMERIC if any psi pass since
 * the last check met a non-positive or non-finite density, LBM_ERR_TIMEOUT
 * if a bounded device wait of the fused step gave up. */
int lbm_sync(lbm_handle h);

/* Macroscopic fields of the current state into host arrays of N doubles:
 * rho (Eq. 4) and u = (j + F/2) / rho with F of Eq. 5.  Any pointer may
 * be NULL.  Synchronises. */
int lbm_moments(lbm_handle h, double *rho, double *ux, double *uy, double *uz);

/* Diagnostics (see lbm_diag); want_ccl != 0 also labels the liquid
 * components on the GPU.  Synchronises. */
int lbm_diagnostics(lbm_handle h, lbm_diag *out, int want_ccl);

/* One droplet: a connected liquid component (6-connectivity, periodic;
 * liquid as in lbm_diag), the droplets and satellites of the break-up
 * study (section "Results": the main drop and the satellite droplets left
 * after the ligament pinches off). */
typedef struct {
    long long first_node;   /* smallest linear index x + nx (y + ny z) in it          */
    long long nodes;        /* node count                                             */
    double volume_w;        /* sum of phi over its nodes                              */
    double mass;            /* sum of rho over its nodes                              */
    double centroid[3];     /* circular mean of its node coordinates on the periodic
                               box, each in [0, n)                                   */
    double resultant[3];    /* length of the mean unit vector per axis, in [0, 1];
                               near 0 the centroid along that axis is undefined
                               (the droplet fills the axis)                          */
    int x_slices;           /* x slices holding one of its nodes (nx: it wraps)       */
    int reserved;
} lbm_droplet;

/* Labels the liquid of the current state on the GPU and returns per-droplet
 * statistics, largest first (ties: smaller first_node first): *count
 * receives the number of droplets, out the first min(*count, max_droplets)
 * of them (out may be NULL when max_droplets is 0).  The FP64 sums are
 * accumulated with atomics, so their last bits may differ between calls.
 * Device scratch: 8 N bytes of labels plus (80 + 4 ceil(nx/32)) bytes per
 * droplet.  Synchronises.  LBM_ERR_TIMEOUT if the labelling guard tripped. */
int lbm_droplets(lbm_handle h, lbm_droplet *out, int max_droplets, int *count);

/* Canonical populations (see Conventions), host arrays of 19 * N doubles.
 * set converts to the storage precision (round to nearest even). */
int lbm_get_populations(lbm_handle h, double *host);
int lbm_set_populations(lbm_handle h, const double *host);

/* Raw checkpoint: the storage bytes plus a small header (layout, size,
 * step count).  lbm_load_state restores it bitwise into a handle of the
 * same size, precision and pattern. */
int lbm_state_bytes(lbm_handle h, size_t *bytes);
int lbm_save_state(lbm_handle h, void *host, size_t bytes);
int lbm_load_state(lbm_handle h, const void *host, size_t bytes);

/* Kernel timing (option "kernel_timing"): launches and summed device time
 * in ms of kernel class k since the option was set, k = 0 psi pass,
 * 1 collide-stream, 2 fused single-pass step.  Synchronises. */
int lbm_kernel_time(lbm_handle h, int k, long long *launches, double *ms);

/* ---- batched form ---------------------------------------------------------
 * A batch advances many independent periodic lattices of uneven size (e.g.
 * a sweep of ligaments) together: every time step is one single-pass launch
 * for the whole batch (option "fused", the default; or one psi-pass launch
 * and one collide-stream launch), whose blocks find their lattice in a tile
 * table, replayed from a captured CUDA graph.  The per-node
 * arithmetic is that of a single lattice, so each instance evolves bitwise
 * as it would alone.  A-B streaming; all instances share the precision. */
typedef struct lbm_batch_ctx *lbm_batch;

typedef struct {
    int nx, ny, nz;                   /* lattice size, each >= 3                  */
    double tau, G;                    /* as in lbm_config                        */
    double R0, lambda, eps, phase;    /* ligament of lbm_init_ligament            */
    double rho_l, rho_v, width;       /* densities and interface width            */
} lbm_instance;

/* Creates a batch of count instances (host array, copied).  The *DEV
 * precisions use rho_ref = rho_v of each instance.  NULL on error, message
 * in lbm_batch_last_error(). */
lbm_batch lbm_batch_create(const lbm_instance *inst, int count, int precision, int psi_form,
                           double rho0, void *stream);
void lbm_batch_destroy(lbm_batch b);
const char *lbm_batch_last_error(void);
int lbm_batch_set_stream(lbm_batch b, void *stream);
/* "fused" (0, 1 or 2; default 2: every step of the whole batch is one
 * single-pass kernel - blocks own tiles of an instance's x-y plane, cut
 * short at its edges, march through a run of z planes and compute psi of
 * the tile and its one-node ring in shared memory, so the populations are
 * read once per step (Eqs. 2-6 as in lbm_step).  2: the TMA-staged step of
 * lbm_step on 64 x 4 (FP32) or 32 x 16 (2-byte) tiles (option "tile_width"),
 * for which the batch
 * keeps a second pool with every row padded to a 16-byte multiple and moves
 * the state there and back by 2-D copies when the step form changes (a
 * read of one instance - diagnostics, populations - copies that instance
 * out, and the padded pool stays current); FP64 and instances whose padded planes pass 2^31
 * elements take form 1.  1: blocks of 32 x 8 nodes, one per thread, copying
 * the populations element by element (instances up to 113 M nodes, larger
 * ones take the two kernels).  0: a psi pass and a collide-stream kernel per
 * step), "persistent" (0/1, default 0: with a single-pass form (1 or 2),
 * every lbm_batch_step call runs its n steps (up to 1024 per launch) as one
 * cooperative launch of persistent blocks - as many as the GPU holds at once,
 * each taking several tiles and z runs per step - separated by grid-wide
 * barriers, replayed from a CUDA graph captured on the first call with that
 * step count (option "graph" 0: launched directly); the same results as one
 * launch per step; a barrier
 * that waits more than 2 s gives up, the launch returns and lbm_batch_sync
 * reports LBM_ERR_TIMEOUT with the state void), "persistent_stall_test" (a
 * test hook of that failure path, in ms, 0..10: one block skips the first
 * barrier and the others give up after this long), "fused_fz" (z planes
 * per block of the single-pass step, default 16), "fused_group" (form 2:
 * z runs per block-order group, as lbm_set_option's; 0, the default: all
 * runs of a tile one after another), "tile_width" (form 2: 64 - tiles of
 * 64 x 4 (FP32) or 64 x 8 (2-byte) nodes -, 32 - tiles of 32 x 8 or 32 x
 * 16 -, or 0, the default: 64 for FP32, 32 for 2-byte storage; the same
 * results), "graph" (0/1),
 * "stochastic_rounding" (0/1, as lbm_set_option), and for the two-kernel
 * step "occupancy" (2, 3, 4; default 2), "vector" (0/1, default 1:
 * instances with even nx update two nodes per thread), "block_x",
 * "block_y", "block_z" (<= 256 threads in all: the batched collide-stream
 * kernel runs block_x * block_y * block_z threads per block over that many
 * consecutive nodes, or node pairs, of one instance in linear order; the
 * per-instance launches of lbm_batch_step_sequential use the shape). */
int lbm_batch_set_option(lbm_batch b, const char *key, double value);
/* Total nodes, collide-stream blocks of one launch, block shape (int[3]);
 * any pointer may be NULL. */
int lbm_batch_info(lbm_batch b, long long *total_nodes, int *collide_tiles, int *block3);
/* Ligament initial condition of every instance; resets the step count. */
int lbm_batch_init(lbm_batch b);
/* n steps of every instance: two launches per step for the whole batch. */
int lbm_batch_step(lbm_batch b, int n);
/* n steps, each instance with its own two launches per step (the plain
 * per-lattice path, for comparison). */
int lbm_batch_step_sequential(lbm_batch b, int n);
/* Waits; LBM_ERR_NUMERIC if a density of any instance went bad,
 * LBM_ERR_TIMEOUT if a grid barrier of the persistent step gave up (the
 * state is then void: re-initialise).  Clears the flag it reports. */
int lbm_batch_sync(lbm_batch b);
/* Canonical FP64 populations of instance k (19 * N_k doubles). */
int lbm_batch_get_populations(lbm_batch b, int k, double *host);
/* Diagnostics of instance k (as lbm_diagnostics). */
int lbm_batch_diagnostics(lbm_batch b, int k, lbm_diag *out, int want_ccl);

/* ---- diagnostics without device allocation ------------------------------
 * The paper has no counterpart of this entry point.  It serves callers that
 * cannot allocate device memory at the moment they need the diagnostics:
 * code running while another stream of the process is capturing a CUDA
 * graph (an allocation there can synchronise the device or break the
 * capture), code inside an allocator or memory-pool callback (re-entering
 * the allocator), and hosts that forbid the library to grow its device
 * memory after start-up.  It computes what lbm_diagnostics computes (not the
 * droplet count) from a population array the caller owns, with the same
 * kernels, but keeps the reduction's partial sums in one static device array
 * of lbm_diagnostics_noalloc_max_scratch() doubles (4 MiB) that every GPU
 * loading the library holds until the process exits.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   f:       device populations of an nx x ny x nz lattice in the library's
 *            storage layout with slot a of node i at f[a * N + i] (the current
 *            array of an A-B lattice, or an AA lattice after an even number of
 *            steps); for the *DEV precisions the stored deviations from
 *            the shifts s_a (w_a * rho_ref rounded to the storage precision).
 *   out:     device array of 13 doubles: mass, momentum x, y, z, liquid volume
 *            (sum of phi), liquid node count, minimum slice area (phi), minimum
 *            slice node count, its x, max |j|/rho, min rho, max rho, 1 if every
 *            density is finite and positive else 0 (definitions as lbm_diag).
 *   stream:  cudaStream_t the kernels run on (NULL = the legacy default stream).
 * Asynchronous: out holds the results once the stream reaches them.  The
 * first call on a device looks up the device address of the static array
 * (cudaGetSymbolAddress, with that device current) and keeps it for later
 * calls; make that first call before any stream capture.  A device reset
 * (cudaDeviceReset) between calls ends the context that held the array, and
 * the kept address with it: the first call after it fails with
 * LBM_ERR_CUDA and forgets the address, and the next call looks it up
 * again.  Every call shares the array and leaves its last
 * contents there (nothing in it needs to start at zero: the kernels write
 * every partial before reading it); calls that overlap on the GPU (streams
 * without an ordering between them) race and give wrong results.  A lattice
 * whose reduction needs more partial sums than the array holds (very large
 * nx) is rejected with LBM_ERR_ARG; the message is in
 * lbm_noalloc_last_error(). */
int lbm_diagnostics_noalloc(const void *f, int nx, int ny, int nz, int precision, double rho_ref,
                            double rho_l, double rho_v, double *out, void *stream);
size_t lbm_diagnostics_noalloc_max_scratch(void);
const char *lbm_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
