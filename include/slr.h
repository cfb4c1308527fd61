/*
 * slr.h -- C ABI of the GB300 (sm_103a) semi-Lagrangian level-set surface
 * reconstruction library (libslr.so).
 *
 * Method: Preda & Semplice, "Surface reconstruction from point cloud using a
 * semi-Lagrangian scheme with local interpolator" (arXiv 2410.22205). The
 * calls follow the paper's statement of the problem, Algorithm 1: build a
 * Cartesian grid around the cloud, compute the distance d to the cloud
 * (§3.4), set the initial level set φ^0 (§3.6), then loop { narrow band
 * (§3.8), energy E_p (§3.5), SL update (§3.1) with the Q1 or WENO
 * interpolator (§3.2), cut (§3.8) } until the stopping criterion of §4.
 *
 * Conventions
 *  - Every call returns an slr_status; nothing aborts or throws across the
 *    ABI. On failure, slr_last_error(ctx) holds a one-line message.
 *  - Host arrays passed in are read during the call and not retained; the
 *    caller keeps ownership. Output arrays are caller buffers with a stated
 *    capacity; SLR_E_CAPACITY reports the count that would be needed.
 *  - Device memory comes from the allocator given to slr_create (NULL: the
 *    library uses cudaMalloc/cudaFree). All work is enqueued on the stream
 *    given to slr_create (NULL: a non-blocking stream the context creates
 *    and owns; the legacy default stream cannot hold the captured iteration
 *    graphs). Calls that return host data synchronise that stream.
 *  - A context is not thread-safe: one host thread at a time per context.
 *    Different contexts may be used from different threads.
 *  - Grid layout: node (i,j,k), 0 <= i < n[0] ..., has linear index
 *    i + n[0]*(j + n[1]*k) (x fastest); in 2-D n[2] must be 1. Node
 *    coordinates are lo[a] + i*h with h = (hi[0]-lo[0])/(n[0]-1), which must
 *    be the same on every axis (§3: one mesh width Δx).
 *  - Calling out of order (e.g. slr_step before slr_init_u) returns
 *    SLR_E_STATE.
 */
#ifndef SLR_H
#define SLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slr_ctx slr_ctx;

typedef enum {
    SLR_OK = 0,
    SLR_E_INVALID = 1,  /* bad argument or configuration */
    SLR_E_NOMEM = 2,    /* the allocator returned NULL */
    SLR_E_CUDA = 3,     /* a CUDA runtime call failed */
    SLR_E_TIMEOUT = 4,  /* a bounded wait inside a kernel gave up (the grid barrier between
                           the planes of the cooperative fast sweeping, §3.4 / §3.6) */
    SLR_E_STATE = 5,    /* call out of order, or a device-side consistency check failed */
    SLR_E_CAPACITY = 6  /* output buffer too small; the needed count is returned */
} slr_status;

/* Device allocator. alloc returns device memory of at least `bytes` bytes
 * (NULL on failure); free releases a pointer alloc returned. `user` is passed
 * through unchanged. */
typedef struct {
    void* (*alloc)(size_t bytes, void* user);
    void (*free)(void* ptr, void* user);
    void* user;
} slr_allocator;

/* Run configuration. slr_config_default fills the paper's defaults. */
typedef struct {
    int dim;            /* 2 or 3 */
    int64_t n[3];       /* nodes per axis (n[2] = 1 in 2-D); at most 2^31-1 nodes in total */
    double lo[3];       /* box corner of node (0,0,0) */
    double hi[3];       /* box corner of the last node; equal h on every axis */
    int precision;      /* 32 or 64: storage and arithmetic type of u, d and the SL step */
    int interp;         /* 0 = Q1 (§3.2 eq. IQ1), 1 = WENO (§3.2 eq. IWENO) */
    double p;           /* energy exponent p (§2 eq. energy), default 2 */
    double delta;       /* curvature weight δ (§2 eq. levelset:pde), default 1 */
    double dt;          /* time step; 0 -> h/4 (§4 eq. dxdt) */
    int band;           /* 0 = update the whole grid; 1 = narrow band of §3.8 */
    double gamma;       /* band half-width γ; 0 -> 4h (2-D) / 6h (3-D) (§3.8) */
    double beta;        /* cut-off inner radius β; 0 -> 2h (2-D) / 3h (3-D) (§3.8 eq. cutoff) */
    double c_sing;      /* singular-gradient test constant C (§3.1 eq. SL:2), default 1e-3 */
    double alpha;       /* singular-gradient test exponent α, default 1 */
    int energy_R;       /* 3-D energy subcells per axis R (§3.5), default 5, 1..8 */
    double stop_tol;    /* Δ_E threshold (§4 eq. deltaEn), default 1e-4 */
    int stop_k;         /* running-mean window k_max, default 10, at most 1023 */
    int min_iters;      /* default 10 */
    int max_iters;      /* default 100 */
    int reinit;         /* 1: the reinitialisation of Algorithm 1 (§3.7) on the band and its
                         * first neighbours after every SL step (needs band = 1); 0: off (default) */
    int reinit_sweeps;  /* pseudo-time sweeps of eq. reinit; 0 -> 4(γ/h + 1) */
    double reinit_dtau; /* pseudo-time step Δτ; 0 -> h/2 (at most h/sqrt(dim)) */
    int step_kind;      /* SL step of a 3-D run without reinitialisation: 1 = on bricks staged in shared memory,
                         * 2 = on the band list (the only kind in 2-D and with reinitialisation); 0 (default) =
                         * by the rule measured on GB300: the list step for a band run with the Q1 interpolator
                         * on a grid whose rows are not a multiple of 16 bytes (no TMA staging), bricks
                         * otherwise. The kind changes timing only within the tolerances of the step. */
} slr_config;

void slr_config_default(slr_config* cfg);

/* Create a context for one reconstruction job. Validates cfg (equal h on
 * all axes, at least 4 nodes per active axis, precision 32|64, ...) and
 * allocates the dense fields u (two buffers), d and argmin plus the band and
 * reduction buffers. alloc may be NULL (cudaMalloc/cudaFree); stream is a
 * cudaStream_t or NULL (the context then owns a stream of its own). The
 * context binds to the device current at this call. */
slr_status slr_create(const slr_config* cfg, const slr_allocator* alloc, void* cuda_stream, slr_ctx** out);

/* Copy the point cloud S = {Q_1..Q_N} (§2) to the device. xyz: host array of
 * n_points rows of `dim` FP64 coordinates, row-major. n_points >= 1. */
slr_status slr_load_cloud(slr_ctx* ctx, const double* xyz, int64_t n_points);

/* Algorithm 1, §3.4: d(x_j) = min_Q |x_j - Q| on every node, exact,
 * with argmin (the lowest point index on ties). Needs slr_load_cloud. The
 * minimiser is decided in FP64; d is stored in the configured precision. */
slr_status slr_build_distance(slr_ctx* ctx);

/* §3.4 as the paper builds the distance grid: the exact d of
 * slr_build_distance on the nodes of a box of 4 grid points per axis around
 * each point (per axis the nodes i0-1 .. i0+2, i0 = floor((Q_a - lo_a)/h),
 * clipped to the grid), then the fast sweeping method (Zhao 2005: Godunov
 * upwind solution of |∇d| = 1, Gauss-Seidel sweeps in the 2^dim orderings,
 * two rounds, box nodes kept) on every other node, started at +inf. FP64
 * throughout, rounded to the storage precision at the end; argmin is the
 * exact minimiser on box nodes and -1 elsewhere. Needs slr_load_cloud.
 * SLR_E_INVALID when no point lies within a cell of the grid (no box node). */
slr_status slr_build_distance_fsm(slr_ctx* ctx);

/* Set d from a host FP64 array of all nodes (e.g. an analytic distance);
 * argmin is set to -1. Rounded to the storage precision. */
slr_status slr_set_distance(slr_ctx* ctx, const double* d_host);

/* Cloud resolution h_S of §4 (eq. dxdt): the mean, over the listed sample of
 * the cloud (0-based point indices, distinct; the paper draws 10% of the
 * points at random), of the distance from each sampled point to its nearest
 * other point of the cloud (a duplicate counts, at distance 0). Needs the
 * cloud (slr_load_cloud) and at least two points; sample is a host array of
 * m indices. Exact distances (FP64), summed in sample order. */
slr_status slr_cloud_spacing(slr_ctx* ctx, const int64_t* sample, int64_t m, double* h_s);

/* Algorithm 1, §3.6: initial level set φ^0.
 *  kind 0 (sphere): params = {cx, cy, cz, r}; φ^0 = |x - c| - r (FP64, rounded to storage);
 *  kind 1 (array):  u0_host = FP64 values of all nodes;
 *  kind 2 (§3.6, from the cloud): params = {γ_S}: nodes on the grid boundary
 *    are external, the marking spreads along the grid lines (one round of
 *    sweeps +x, -x, +y, -y, +z, -z) through nodes with d >= γ_S; φ^0 = d - γ_S
 *    on external nodes, and the fast sweeping method (|∇φ| = 1, Godunov
 *    local solver, two rounds of 2^dim orderings) fills the other nodes, whose
 *    sign is then reversed: a signed distance whose zero set encloses the
 *    cloud at about γ_S from it. The paper takes γ_S = K_S h_S, h_S the mean
 *    nearest-neighbour spacing of the cloud and K_S = 2. Computed in FP64
 *    (slr_init_u holds N doubles and N bytes of scratch while it runs).
 * In band mode the cut of eq. cut is applied, so |φ^0| <= γ holds before the
 * first step; the band G̃^0 (eq. subgrid, |φ| < γ) and the list of cells the
 * energy quadrature may visit are built here. Resets the iteration count and
 * the diagnostics. Needs d (build or set) first. */
slr_status slr_init_u(slr_ctx* ctx, int kind, const double* params, const double* u0_host);

/* Run n_steps iterations of Algorithm 1 (band, SL update §3.1, cut)
 * without the stopping test, each followed by the FP64 energy of the new
 * state. energy_override >= 0 uses that value as E_p in the scale factor
 * (d/E_p)^(p-1) of every step; < 0 uses the computed E_p(φ^n). */
slr_status slr_step(slr_ctx* ctx, int n_steps, double energy_override);

/* As slr_step, but only enqueues the iterations on the context's stream and
 * returns without waiting (no host synchronisation, no status read). Errors
 * raised by the device's own checks (SLR_E_STATE) are reported by the next
 * synchronous call. For overlapping host work or other jobs with the iterations. */
slr_status slr_step_async(slr_ctx* ctx, int n_steps, double energy_override);

/* Iterate until the stopping criterion of §4 (eq. deltaEn: Δ_E < stop_tol
 * after at least min_iters iterations, or max_iters). The test and the
 * iteration count live on the device; the host reads a 4-byte status every
 * few iterations. iters_out / converged_out may be NULL. */
slr_status slr_evolve(slr_ctx* ctx, int* iters_out, int* converged_out);

/* Batched form of slr_evolve for independent jobs on one device: each
 * launch of one CUDA graph advances every job by `chunk` iterations (1..64,
 * 0 -> 8; < 0: autotuned, see below), the jobs as parallel branches, so that the iterations of many
 * small and large reconstructions overlap on the GPU instead of running one
 * job after another. A job whose stop test (§4) has fired turns the rest of
 * its branch into no-ops. Returns when every job has stopped. Every job must
 * have been initialised (slr_init_u) on the current device; jobs keep their
 * own streams and memory; `cuda_stream` (NULL: the first job's stream) orders
 * the batch launches. iters_out / converged_out: n_jobs entries each, may be
 * NULL. The jobs' contexts must not be used by other threads meanwhile. */
slr_status slr_batch_evolve(slr_ctx* const* jobs, int n_jobs, int chunk, void* cuda_stream, int* iters_out,
                            int* converged_out);

/* The chunk of the last slr_batch_evolve whose first job was first_job. With
 * chunk < 0 the batch autotunes it: the first launches try 32, 16, 8 and 4
 * iterations per launch once each, timed on the device, and the rest of the
 * batch keeps the one with the least time per iteration. The iterations do
 * not depend on the chunk, so the results are the same as with any fixed
 * chunk. 0 before any batch. */
int slr_batch_chunk(const slr_ctx* first_job);

/* Batched form of slr_evolve in one persistent kernel (the batching of many
 * reconstructions on one GPU stands in for the paper's ranks advancing
 * subdomains together, §3.3; each job runs the loop of Algorithm 1 (§3)
 * without the reinitialisation). One cooperative launch, captured in a CUDA
 * graph, advances every job iteration by iteration: its blocks take work
 * items (a brick of a 3-D job's band, a group of band-list tiles of a 2-D
 * job, a slot of candidate cells of the energy of §3.5, a slice of a job's
 * record and stop test of §4 eq. deltaEn) from one ticket counter, in three
 * phases per iteration separated by grid barriers. A job whose stop test has
 * fired contributes no items; the launch ends when every job has stopped.
 * Each job's state, iteration count and history are bit-identical to those
 * of slr_evolve on that job alone.
 * Jobs: initialised (slr_init_u) on the current device, narrow band on,
 * reinitialisation off, energy_R = 5 in 3-D (else SLR_E_INVALID: use
 * slr_batch_evolve, which takes any job); FP32 and FP64 jobs run as separate
 * launches, at most 64 jobs per launch. autotune != 0: the first launches
 * time seven launch shapes (128 threads at two register budgets with one,
 * two or four bricks per step item, 256 threads with one; one iteration
 * each, twice) and the rest of the batch keeps the fastest; 0: the first
 * shape (128 threads, one brick per item). `cuda_stream`
 * (NULL: the first job's stream) orders the launches; every job's own stream
 * is synchronised first. iters_out / converged_out: n_jobs entries each, may
 * be NULL. SLR_E_TIMEOUT if a grid barrier waited longer than its poll limit
 * (~0.3 s); SLR_E_STATE if a job's device-side check failed. Contexts must
 * not be used by other threads meanwhile. */
slr_status slr_batch_run(slr_ctx* const* jobs, int n_jobs, int autotune, void* cuda_stream, int* iters_out,
                         int* converged_out);

/* The last slr_batch_run whose first job was first_job: the launch shape
 * it ran with (threads per block, resident blocks per SM, bricks of a 3-D
 * job per step item), whether its launches ran as captured CUDA graphs (1)
 * or were enqueued directly where capture was refused (0), and the
 * autotuner's best trial time in ms (0 without autotuning). Any pointer may
 * be NULL. */
slr_status slr_batch_run_info(const slr_ctx* first_job, int* threads, int* blocks_per_sm, int* bricks_per_item,
                              int* graph, float* tuned_ms);

/* Nodes with |φ| < width, in ascending linear index (the reconstructed zero
 * level set's neighbourhood). idx/u: caller buffers of `cap` entries (either
 * may be NULL to query the count). *n_out = number of such nodes; returns
 * SLR_E_CAPACITY if it exceeds cap (nothing written then). */
slr_status slr_extract(slr_ctx* ctx, double width, int64_t* idx, double* u, int64_t cap, int64_t* n_out);

enum { SLR_FIELD_U = 0, SLR_FIELD_D = 1, SLR_FIELD_ARGMIN = 2 };

/* Copy a whole field to the host: U and D as FP64 (widened from storage),
 * ARGMIN as int32. cap = number of entries host_out holds (>= nodes). */
slr_status slr_get_field(slr_ctx* ctx, int which, void* host_out, int64_t cap);

/* Current narrow band G̃ (ascending node indices), as int64. In whole-grid
 * mode the band is every node and *n_out = nodes (idx may be NULL). */
slr_status slr_get_band(slr_ctx* ctx, int64_t* idx, int64_t cap, int64_t* n_out);

/* §3.5 energy of the current state computed now: E_p with the given p and,
 * separately, the raw sum Σ|d|^p·measure. Either output may be NULL. */
slr_status slr_energy(slr_ctx* ctx, double p, double* E_out, double* sum_out);

/* Per-iteration history since slr_init_u: e2_hist[i] = E_2(φ^i) for
 * i = 0..iters, dphi_hist[i] = Δ_φ (§4, h^dim Σ|φ^{i+1}-φ^i|) and
 * band_hist[i] = band size of iteration i for i < iters. Arrays may be NULL;
 * each holds `cap` entries (entries beyond cap are dropped). *n_out = iters.
 * err_cloud (may be NULL): Err_S of §4 eq. errCloud for the current state,
 * needs the cloud. */
slr_status slr_diagnostics(slr_ctx* ctx, double* e2_hist, double* dphi_hist, int64_t* band_hist, int cap,
                           int* n_out, double* err_cloud);

/* Checkpoint: serialise u, d, argmin, the band, the iteration count and the
 * energy history into buf (host, cap bytes). buf NULL or too small ->
 * SLR_E_CAPACITY with *n_out = bytes needed. slr_import_state restores a
 * state exported from a context with the same configuration; continuing
 * from it reproduces an uninterrupted run bit for bit. */
slr_status slr_export_state(slr_ctx* ctx, void* buf, int64_t cap, int64_t* n_out);
slr_status slr_import_state(slr_ctx* ctx, const void* buf, int64_t n);

/* Opt-in timing of the kernels of one iteration: with on != 0 the captured
 * iteration graph also records CUDA events between its phases (SL step with
 * band compaction, reinitialisation when on, energy quadrature, record/stop).
 * After an iteration has run, slr_last_iteration_times synchronises the
 * stream and writes the durations of the SL step, energy and record phases of
 * the most recent iteration in milliseconds; slr_last_iteration_phases writes
 * the same with the reinitialisation phase: ms[0] step, ms[1]
 * reinitialisation (0 when off), ms[2] energy, ms[3] record. */
slr_status slr_set_profiling(slr_ctx* ctx, int on);
slr_status slr_last_iteration_times(slr_ctx* ctx, float ms[3]);
slr_status slr_last_iteration_phases(slr_ctx* ctx, float ms[4]);

/* Number of kernels this context has launched so far (for launch accounting). */
int64_t slr_kernel_launches(const slr_ctx* ctx);

/* Launch shape of the brick-staged 3-D step (every 3-D context without the
 * reinitialisation runs its SL step, §3.1 eq. SL3d, on 8x8x8-node bricks
 * whose u and d are staged in shared memory). slr_init_u times each candidate
 * shape on φ^0 and keeps the fastest; every shape gives identical results.
 * *threads: threads per block; *stages: 2 when the next brick is prefetched
 * by TMA while one is computed, else 1; *trial_ms: the chosen shape's trial
 * time. Any output may be NULL. SLR_E_STATE for 2-D contexts, contexts with
 * the reinitialisation, or before slr_init_u. */
slr_status slr_brick_shape(const slr_ctx* ctx, int* threads, int* stages, float* trial_ms);

/* Force the brick step's launch shape (threads 128 or 256, stages 1 or 2;
 * where TMA does not stage the boxes, stages 2 runs as 1) in place of the
 * autotuner's choice, until the next slr_init_u. Results do not change.
 * SLR_E_INVALID for another shape, SLR_E_STATE as slr_brick_shape. */
slr_status slr_brick_shape_set(slr_ctx* ctx, int threads, int stages);

/* Distance grid for callers that cannot allocate device memory.
 *
 * The paper has no counterpart to this call; it exists for users of this
 * library that may not call cudaMalloc: code running while another framework
 * owns the device memory through its own pool, real-time loops that must not
 * allocate once running, or plug-ins that are handed pre-allocated buffers
 * only. It computes exactly what slr_build_distance computes (d and argmin,
 * the lowest point index on ties, d rounded to `precision`), but from
 * caller-owned device buffers and without a context, and it allocates
 * nothing: no cudaMalloc, cudaFree or allocating library routine. Its
 * scratch (point codes, bin counts, sorted points, box hierarchy, leaf
 * cylinders) is one fixed array of about 2.5 MB in the library's device
 * memory, present on every GPU that loads the library until the process
 * exits.
 *
 *  dim, n, lo, h: the grid (as in slr_config; node coordinates lo + i*h;
 *                 n[2] = 1 in 2-D); at most 2^31-1 nodes.
 *  pts_dev:       device array of n_points rows of `dim` FP64 coordinates;
 *                 1 <= n_points <= 65536 (larger clouds: SLR_E_INVALID,
 *                 use slr_build_distance).
 *  d_dev:         device output, one float (precision 32) or double (64) per node.
 *  argmin_dev:    device output, one int32 per node.
 *  cuda_stream:   stream for the work (NULL: the legacy default stream). The
 *                 call returns after the stream has finished the work.
 *
 * The call is synchronous: it reads the cloud's bounding box and a status
 * word back to the host and waits on cuda_stream, so it cannot be recorded
 * into a CUDA graph; call it on a stream that is not capturing (a capturing
 * stream gives SLR_E_INVALID, with nothing enqueued). The first call on each device also looks up that
 * device's address of the scratch array (cudaGetSymbolAddress, with that
 * device current). All calls share the one array and it
 * keeps the last call's contents (what must start at zero is cleared at the
 * start of each call): calls that overlap on the GPU, from different threads
 * or streams, race. Errors are described by slr_last_error(NULL). */
slr_status slr_distance_grid_noalloc(int dim, const int64_t n[3], const double lo[3], double h, int precision,
                                     const double* pts_dev, int64_t n_points, void* d_dev, int32_t* argmin_dev,
                                     void* cuda_stream);

/* Last error message of the context (never NULL; "" when none). With
 * ctx == NULL: the reason of the last failed slr_create or
 * slr_distance_grid_noalloc on this thread. */
const char* slr_last_error(const slr_ctx* ctx);

/* FMA throughput of the current device (the paper has no counterpart: the
 * benchmark's ALU roofline divides by it). Launches 8 blocks of 256 threads
 * per SM, each thread running 8 independent chains of `trips` x 8 FMAs in
 * `precision` (32 or 64), twice, and times the second launch with CUDA events
 * on the legacy default stream. *tflops_out = 2 flops x FMAs / time;
 * *ms_out = that launch's time. Allocates a few bytes of device memory.
 * SLR_E_INVALID for another precision, trips < 1 or a NULL output. */
slr_status slr_probe_fma(int precision, int64_t trips, double* tflops_out, double* ms_out);

/* Release all device memory of the context and the context itself. NULL is a no-op. */
void slr_destroy(slr_ctx* ctx);

/* Failure-detection check of the bounded waits (the paper has no
 * counterpart), on the current device. unreachable = 0: the grid barrier
 * that the cooperative fast-sweeping kernel uses between planes, alone in a
 * two-block cooperative launch, SLR_OK. unreachable = 1: a barrier that no
 * block completes; every wait gives up after its poll limit (about 0.3 s)
 * and the call returns SLR_E_TIMEOUT, the device staying usable.
 * unreachable = 2: the batched kernel's per-job dependency wait (slr_batch_run)
 * on a counter that no work item completes, SLR_E_TIMEOUT after its poll
 * limit. SLR_E_INVALID for another mode; SLR_E_CUDA when cooperative launch
 * is unavailable; slr_last_error(NULL) gives the reason. */
slr_status slr_selftest_barrier(int unreachable);

/* §4: the L^1 norm of the error against an exact signed distance,
 * Δx^dim Σ_j |c(φ_j) - c(φ*_j)| over every node, with c the cut of eq. cut
 * at the band half-width γ in band mode (the identity in full-grid mode),
 * in FP64. kind 0: φ* = |x - c| - r, params = {cx, cy, cz, r} (cz unused in
 * 2-D), evaluated on the device in FP64; kind 1: φ* from exact_host, one FP64
 * value per node. Needs slr_init_u. */
slr_status slr_l1_error(slr_ctx* ctx, int kind, const double* params, const double* exact_host, double* l1_out);

/* ---------------------------------------------------------------------------
 * Several runs from coarse to fine (§4: eq. dxdt and Tab. param).
 *
 * h_S, the cloud's resolution, comes from a sample of the points
 * (slr_cloud_spacing). Run r works on a grid of width Δx(r) = h_S / 2^(r-1)
 * over the cloud's bounding box widened by 8 Δx(r) on every side, plus
 * γ_S = K_S h_S in the first run (this reproduces the grids of the paper's
 * circle test, 42^2, 58^2, 99^2, 181^2 and 344^2), with (p, δ) = (1, 0),
 * (2, 0), then (2, 1), and with the reinitialisation of §3.7. φ^0 of the
 * first run is the §3.6 initial data at γ_S; each later run starts from the
 * previous run's steady state, interpolated (Q1) at its nodes and cut. A run
 * whose grid would exceed max_nodes is coarsened until it fits
 * (report->coarsened); a coarsened first run takes γ_S = K_S Δx(1), so that
 * the marked shell around the cloud stays closed on its grid. The sample is a Bernoulli draw with probability
 * sample_frac per point from the counter-based splitmix64 stream of `seed`
 * (point i is drawn when splitmix64(seed + (i+1)·0x9E3779B97F4A7C15) <
 * sample_frac·2^64).
 *
 * At the end of each run the report holds the quantities of the paper's
 * tables: the grid, E_2 of the run's final state, Err_S (eq. errCloud) and,
 * when an exact signed distance is given, the L^1 error of slr_l1_error.
 * ------------------------------------------------------------------------- */
#define SLR_MAX_RUNS 8

typedef struct {
    int dim;             /* 2 or 3 */
    int precision;       /* 32 or 64 */
    int interp;          /* 0 = Q1, 1 = WENO */
    int runs;            /* runs of Algorithm 1, 1..SLR_MAX_RUNS, default 3 */
    double K_s;          /* γ_S = K_S h_S for the initial data, default 2;
                            K_S Δx(1) when the first grid is coarsened */
    double sample_frac;  /* fraction of the points sampled for h_S, default 0.1 */
    uint64_t seed;       /* sample stream, default 1 */
    int64_t max_nodes;   /* node budget of one run, default 2^27 */
    int max_iters;       /* iterations per run (§4), default 100 */
    int distance_fsm;    /* 1: every run's d by slr_build_distance_fsm (§3.4);
                            0 (default): exact d (slr_build_distance) */
    int exact_sphere;    /* 1: report the L^1 error against |x - c| - r */
    double sphere[4];    /* {cx, cy, cz, r} for exact_sphere */
} slr_multirun_config;

typedef struct {
    double h_s;                        /* the cloud's resolution */
    int64_t sample_size;               /* points in the h_S sample */
    int runs_done;
    int coarsened;                     /* a run was coarsened to fit max_nodes */
    double run_dx[SLR_MAX_RUNS];       /* grid width of each run */
    int64_t run_n[SLR_MAX_RUNS][3];    /* nodes per axis of each run */
    double run_lo[SLR_MAX_RUNS][3];    /* node (0,0,0) of each run's grid */
    int run_iters[SLR_MAX_RUNS];       /* iterations of each run */
    int run_converged[SLR_MAX_RUNS];   /* the Δ_E test stopped the run */
    double run_energy[SLR_MAX_RUNS];   /* E_2 of the run's final state */
    double run_err_cloud[SLR_MAX_RUNS];/* Err_S (eq. errCloud) of the final state */
    double run_l1_err[SLR_MAX_RUNS];   /* L^1 error (exact_sphere), else NaN */
} slr_multirun_report;

void slr_multirun_default(slr_multirun_config* mc);

/* Reconstruct from xyz (host, n_points rows of dim FP64 coordinates) with the
 * runs above. On success *out is the context of the last run (the caller
 * destroys it): its field, band and diagnostics are the result. report may be
 * NULL. alloc and cuda_stream as for slr_create. */
slr_status slr_reconstruct(const slr_multirun_config* mc, const double* xyz, int64_t n_points,
                           const slr_allocator* alloc, void* cuda_stream, slr_ctx** out,
                           slr_multirun_report* report);

/* ------------------------------------------------------------------------
 * Serving: a continuous-batching request loop (the paper has no counterpart;
 * it reconstructs one cloud at a time). Requests are admitted in order while
 * an active slot (max_active) and enough of the device-memory budget are
 * free; each admitted job gets its own context and stream, its exact
 * distance grid and φ^0 (a sphere), and then joins the round-robin of
 * iterations of all running jobs, which overlap on the GPU. A finished job's
 * context stays with the server until released; the client reads results
 * from it with slr_extract / slr_get_field / slr_diagnostics meanwhile.
 * Thread-safe: any thread may submit, poll and release.
 * ------------------------------------------------------------------------ */
typedef struct slr_server slr_server;

/* hbm_budget: device bytes the server may hold for admitted jobs (a job is
 * admitted alone even if its estimate exceeds the budget); max_active: jobs
 * admitted at once; setup_threads (1..64): threads that set admitted jobs up
 * (context, distance grid, φ^0) at the same time, each on its job's stream;
 * alloc: allocator for the jobs' contexts (NULL: cudaMalloc). Binds to the
 * current device; starts the setup and iteration threads. */
slr_status slr_server_create(size_t hbm_budget, int max_active, int setup_threads, const slr_allocator* alloc,
                             slr_server** out);

/* Admission order of queued requests (the paper has no counterpart): 0 (the
 * default) the oldest first; 1 the least estimated set-up time less the time
 * the request has waited, so that small requests pass a large one whose
 * distance grid would hold the set-up threads, and a large request still gets
 * its turn once it has waited about its estimate (4 ns per grid node plus
 * 20 ns per point). Either way a request is admitted only while a slot and
 * its share of the HBM budget are free. SLR_E_INVALID for another value. */
slr_status slr_server_set_policy(slr_server* s, int policy);

/* Queue one reconstruction: cfg as for slr_create, the cloud (host, copied),
 * φ^0 = |x - c| - r with sphere = {cx, cy, cz, r}; the job then runs to the
 * stopping criterion of §4. *ticket identifies it. */
slr_status slr_server_submit(slr_server* s, const slr_config* cfg, const double* xyz, int64_t n_points,
                             const double sphere[4], uint64_t* ticket);

/* *state: 0 queued, 1 running, 2 done, 3 failed (then SLR_E_CUDA and
 * slr_server_last_error). result (may be NULL): the job's context once done,
 * owned by the server. latency_ms (may be NULL): submit-to-finish time once
 * done or failed, else -1. */
slr_status slr_server_poll(slr_server* s, uint64_t ticket, int* state, slr_ctx** result, double* latency_ms);

/* Where a finished (done or failed) job's latency went, in milliseconds:
 * queue_ms from submission to admission, setup_ms from admission to its first
 * iteration (context, cloud copy, distance grid, φ^0), iterate_ms from then to
 * the stop test's end. Any output may be NULL. SLR_E_STATE while the job is
 * queued or running; SLR_E_INVALID for an unknown or released ticket. */
slr_status slr_server_timing(slr_server* s, uint64_t ticket, double* queue_ms, double* setup_ms,
                             double* iterate_ms);

/* Destroy a finished (done or failed) job's context and return its budget
 * share; SLR_E_STATE while it is queued or running. */
slr_status slr_server_release(slr_server* s, uint64_t ticket);

const char* slr_server_last_error(const slr_server* s);

/* Stop the threads (running jobs are abandoned after their queued work
 * drains) and destroy every context the server still holds. */
void slr_server_destroy(slr_server* s);

#ifdef __cplusplus
}
#endif
#endif
