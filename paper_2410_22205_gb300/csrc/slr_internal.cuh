// Internal declarations of libslr: context, device state, launch wrappers
// and the device-side numerics shared by the kernels (centred differences,
// cut-off, tangent directions, Q1 and WENO interpolation).
//
// Method: Preda & Semplice, arXiv 2410.22205 (§3 numerical scheme).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/slr.h"

namespace slr {

// ---------------------------------------------------------------------------
// sizes
// ---------------------------------------------------------------------------
constexpr int kHist = 4096;          // ring size of the per-iteration history
constexpr int kStepBlock = 256;      // threads per block of the SL step kernels
constexpr int kStepTile = 128;       // band entries per warp ticket (4 per lane)
constexpr int kMaxR = 8;             // largest supported energy subcell count per axis
constexpr int kRecordBlocks = 32;    // blocks of the record kernel (slices of the tile counts)
constexpr int kMaxStopK = 1023;      // bound on the stop window k_max (staged in shared memory)
constexpr int kErrBandOffset = 1;    // DevState::error: a band-list write fell outside the list
constexpr int kErrBarrier = 2;       // a grid-wide barrier of a cooperative kernel waited too long
constexpr int kErrStage = 4;         // a shared-memory staging wait of the brick step gave up
constexpr long long kBarrierSpinLimit = 1ll << 22;  // polls of one barrier wait (~0.3 s with the sleeps)

// Programmatic dependent launch (griddepcontrol): pdl_trigger lets the next
// kernel of the stream, launched with the programmatic-serialization
// attribute, be scheduled once every block of this grid has started;
// pdl_wait returns once the previous kernel has completed and its writes are
// visible. Both are no-ops for a kernel launched without the attribute.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
#endif

// Grid-wide barrier of a cooperative launch (every block co-resident).
// bar[0] counts the arrivals, bar[1] is the generation; both start at 0.
// Writes before the barrier are visible to loads after it that bypass L1
// (__ldcg). A wait longer than the poll limit sets kErrBarrier in *err and
// makes every block of the caller see false, so the kernel can return.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
        if (atomicAdd(bar, 1u) == nb - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long polls = 0;
            while (*vgen == gen) {
                if (++polls > kBarrierSpinLimit || (*(volatile int*)err & kErrBarrier)) {
                    ok = 0;
                    atomicOr(err, kErrBarrier);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// device-resident state of one job (one allocation)
// ---------------------------------------------------------------------------
struct DevState {
    int n;               // iterations completed since init
    int stop;            // nonzero: step kernels return at entry
    int converged;       // the Δ_E test stopped the loop
    int error;           // kErr* bits set by device code
    int band_count[2];   // [n & 1]: scan domain L^{n-1}; [(n+1) & 1]: band L^n written by step n
    unsigned ticket;     // tile ticket of the fused step kernel (reset by the record kernel)
    unsigned record_done;  // blocks of the record kernel done (reset by its last block)
    unsigned eticket[2];   // [1]: slot ticket of the energy kernel; [0] unused (both reset by the record kernel)
    int band_next;       // size of the band the next step writes (sum of the tile counts)
    int band_sl;         // with reinitialisation: band nodes the SL step of this iteration updated
    int n_ecells_dyn;    // with reinitialisation: candidate cells of the energy pass
    int band_brick;      // brick step: band nodes of this iteration (summed by the bricks, reset by the record kernel)
    int band_base[kRecordBlocks];  // exclusive prefix of the tile counts per record-block slice
    double Ep;           // E_p(φ^n) used by step n
    double e2_hist[kHist];
    double dphi_hist[kHist];
    long long band_hist[kHist];
};

// grid and scheme parameters passed by value to the kernels
template <typename T>
struct Params {
    int n0, n1, n2;        // nodes per axis
    long long s1, s2;      // strides of axes 1 and 2
    int is1, is2;          // the same strides as 32-bit values (fewer than 2^31 nodes)
    T h;                   // mesh width
    T inv_h;               // 1/h
    T inv_2h;              // 1/(2h)
    T h4;                  // h^4 (WENO: ε = h^2 folded into the weights)
    T dt;
    T delta, p, inv_p;
    T gamma, beta, inv_gb3;  // γ, β, 1/(γ-β)^3
    T sing_thr;            // C Δt^α of the singular-gradient test
    int band;              // narrow band on
    int p_kind;            // 1: p == 1, 2: p == 2, 0: general
};

// ---------------------------------------------------------------------------
// host-side context
// ---------------------------------------------------------------------------
struct Buffer {
    void* ptr = nullptr;
    size_t bytes = 0;
};

// the brick-staged 3-D step (slr_brick.cu): bricks of 8x8x8 nodes
struct BrickState {
    int nb[3] = {0, 0, 0};      // bricks per axis
    long long ntotal = 0;       // bricks of the grid
    long long nbricks = 0;      // active bricks (listed at init)
    int* list = nullptr;        // active brick ids, ascending
    int* cnt = nullptr;         // per brick id: band count of the previous iteration
    double* part = nullptr;     // per brick id: Δ_φ partial
    int tma = 0;                // stage by TMA tile loads (else cp.async copies)
    int occ[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // resident blocks per SM of each launch shape
    int shape = 0;              // launch shape chosen by the autotuner
    float tuned_ms = 0.f;       // its trial time
    long long list_iter = -1;   // iteration whose band the band list holds (after import), else -1
    CUtensorMap tm_u[2];        // u buffers, 24x16x16 boxes
    CUtensorMap tm_d;           // d, 24x10x10 boxes
};

}  // namespace slr

struct slr_ctx {
    slr_config cfg;
    slr_allocator al;
    bool default_alloc = true;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int num_sms = 0;
    double h = 0, dt = 0, gamma = 0, beta = 0;
    long long N = 0;          // nodes
    long long ncells_all = 0; // cells of the whole grid
    size_t tsize = 4;         // bytes of the storage type

    void* u[2] = {nullptr, nullptr};
    void* d = nullptr;
    int* argmin = nullptr;
    double* pts = nullptr;
    long long npts = 0;

    int* band[2] = {nullptr, nullptr};  // band lists (capacity band_cap)
    long long band_cap = 0;
    int* ecells = nullptr;     // candidate cells of the energy quadrature (lower-corner node index)
    long long n_ecells = 0;
    double* part_dphi = nullptr;   // one per step tile
    long long n_tiles_cap = 0;
    double* part_e = nullptr;      // two per energy block, plus a two-value report slot
    long long n_echunks = 0;       // candidate chunks of 32 cells (sizes part_e)
    int* tile_off = nullptr;       // per 128-entry tile of the step's input band: count, then offset in its slice
    // reinitialisation (cfg.reinit): scratch field, row-padded bitmasks, flags
    void* rw = nullptr;                  // W: sweep ping-pong partner of the output φ buffer
    unsigned* bits_band = nullptr;       // band G̃^n
    unsigned* bits_gbar = nullptr;       // Ḡ^n
    unsigned* bits_cell = nullptr;       // candidate cells
    int* rblk = nullptr;                 // per-block counts of the two compactions
    unsigned char* rflags = nullptr;     // per Ḡ position: fixed, sign
    double* part_dphi_r = nullptr;       // Δ_φ partials of the final reinitialisation kernel
    slr::DevState* ds = nullptr;
    int* host_pinned_flags = nullptr;  // pinned host words for status readback

    bool have_cloud = false, have_d = false, have_u = false;
    int batch_chunk = 0;  // chunk of the last slr_batch_evolve this context led (autotuned or given)
    // slr_batch_run: this job's iterations and stop reason; as the first job,
    // the block size, graph use and autotuning trial time of the run it led
    int batch_iters = 0, batch_converged = 0;
    int batch_threads = 0, batch_blocks = 0, batch_bpi = 0, batch_graph = 0;
    float batch_tuned_ms = 0.f;
    std::string err;
    long long launches = 0;

    cudaGraphExec_t g_evolve = nullptr;
    cudaGraphExec_t g_step = nullptr;
    double g_step_override = -2.0;
    bool profiling = false;
    cudaEvent_t pev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    slr::BrickState brick;
};

namespace slr {

// allocation through the context's allocator
void* dev_alloc(slr_ctx* c, size_t bytes);
void dev_free(slr_ctx* c, void* p);

// kernel launch wrappers (defined in the .cu files); each returns the CUDA
// error of the launch and adds the number of kernels it launched to *launches
cudaError_t launch_init_u(slr_ctx* c, int kind, const double* params, const double* u0_dev);
cudaError_t launch_count_band(slr_ctx* c, long long* count_out);
cudaError_t launch_build_band(slr_ctx* c);
cudaError_t launch_build_ecells(slr_ctx* c, long long* count_out, bool write);
cudaError_t launch_step(slr_ctx* c, double energy_override, int evolve_mode);
// brick-staged 3-D step (every 3-D run without reinitialisation); see slr_brick.cu
bool brick_mode(const slr_ctx* c);
cudaError_t bricks_init(slr_ctx* c, const void* u);
void bricks_free(slr_ctx* c);
cudaError_t launch_step_brick(slr_ctx* c, double energy_override);
cudaError_t bricks_autotune(slr_ctx* c);
void brick_shape_of(const slr_ctx* c, int* threads, int* stages, float* trial_ms);
int brick_shape_index(int threads, int stages);
cudaError_t band_of_field(slr_ctx* c, const void* u, int* out, long long* count);
cudaError_t launch_energy(slr_ctx* c, int offset, double p_override, int record_mode, int evolve_mode,
                          cudaEvent_t between = nullptr);
cudaError_t launch_extract(slr_ctx* c, double width, long long* idx_dev, double* u_dev, long long* count_out,
                           bool write);
// the rest of slr_init_u once both φ buffers hold φ^0 (e: status of writing them)
slr_status init_after_u(slr_ctx* c, cudaError_t e);
// §3.6 initial data into an FP64 device field (ext: N bytes of scratch); see slr_initdata.cu
cudaError_t launch_init_marking(slr_ctx* c, double gamma_s, double* phi_dev, unsigned char* ext_dev);
// the reinitialisation of Algorithm 1 (§3.7) after launch_step; see slr_reinit.cu
cudaError_t launch_reinit(slr_ctx* c);
int reinit_grid(const slr_ctx* c);
int reinit_sweeps(const slr_ctx* c);
double reinit_dtau(const slr_ctx* c);
size_t reinit_bit_words(const slr_ctx* c);
int reinit_scan_blocks(const slr_ctx* c);
cudaError_t launch_err_cloud(slr_ctx* c, double* out_dev);
cudaError_t launch_to_double(slr_ctx* c, const void* src, double* dst, long long n);
cudaError_t launch_from_double(slr_ctx* c, const double* src, void* dst, long long n);
cudaError_t build_distance(slr_ctx* c);
// exact distance (FP64) and argmin on the nodes with mask[j] != 0; others untouched
cudaError_t distance_on_marked(slr_ctx* c, const unsigned char* mask, double* dout);
// §3.4: exact on the 4^dim node box around each point, fast sweeping elsewhere
// (cudaErrorInvalidValue: no point within a cell of the grid)
cudaError_t build_distance_fsm(slr_ctx* c);
// the grid barrier alone on the current device (unreachable: one that no
// block completes); *err_out receives the kernel's error bits
cudaError_t barrier_selftest(int device, int unreachable, int* err_out);
// per-block partial sums of |c(u_j) - c(φ*_j)| (kind 0: sphere prm = {cx, cy,
// cz, r}; kind 1: exact_dev) into part[0..blocks)
cudaError_t launch_l1_error(slr_ctx* c, const void* u, int kind, const double* prm, const double* exact_dev,
                            double* part, int blocks);
long long energy_blocks(const slr_ctx* c);
// Message of the last failed call without a context on this thread
// (slr_create, slr_selftest_barrier, slr_distance_grid_noalloc,
// slr_reconstruct before its first context exists): each of these clears it
// on entry and sets it on failure; slr_last_error(NULL) returns it.
void ctxless_error_clear();
slr_status ctxless_error_set(slr_status s, const std::string& msg);
const char* ctxless_error();
long long full_step_blocks(const slr_ctx* c);
// evolve building blocks for schedulers: capture the iteration graph if
// needed and clear the stop flags; enqueue one iteration (no host wait)
slr_status evolve_prepare(slr_ctx* c);
slr_status evolve_launch(slr_ctx* c);
cudaError_t launch_gather_status(slr_ctx* c, DevState* const* states, int n, int* out, cudaStream_t st);
// a failed CUDA call of a context's operation: the message goes to the
// context, the status is SLR_E_CUDA (slr_api.cu)
slr_status cuda_status(slr_ctx* c, cudaError_t e, const char* where);
// the batched persistent kernel (slr_batch.cuh) for one group of at most 64
// jobs of one storage type: shape_io in/out (-1: autotune); out: graph use,
// the autotuner's best trial time, and the shape's threads per block,
// resident blocks per SM and bricks per item
slr_status batch_run_f32(slr_ctx* const* jobs, int n, int tune, cudaStream_t st, int* shape_io, int* graph_out,
                         float* tuned_ms, int* threads, int* blocks, int* bpi);
slr_status batch_run_f64(slr_ctx* const* jobs, int n, int tune, cudaStream_t st, int* shape_io, int* graph_out,
                         float* tuned_ms, int* threads, int* blocks, int* bpi);
// the batched kernel's dependency wait on a counter that nothing completes
// (slr_batch_f32.cu); *err_out receives its error bits
cudaError_t batch_wait_selftest(int* err_out);

// ---------------------------------------------------------------------------
// device numerics
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

// Global loads of the fields read by the numerics below. A per-job kernel
// reads data that no block writes during its launch, through the read-only
// path. The batched persistent kernel reads fields that other blocks wrote
// earlier in the same launch, before a grid barrier; its translation unit
// defines SLR_COHERENT_LOADS, and the loads become plain cached loads
// (ld.global.ca), which the barrier's acquire orders after those writes.
#ifdef SLR_COHERENT_LOADS
template <typename T>
__device__ __forceinline__ T ld(const T* p) {
    return __ldca(p);
}
#else
template <typename T>
__device__ __forceinline__ T ld(const T* p) {
    return __ldg(p);
}
#endif

// §3: centred difference along one axis; one-sided first order on the
// domain boundary (the paper is silent there).
template <typename T>
__device__ __forceinline__ T diff_axis(const T* __restrict__ v, long long idx, int i, int n, long long stride,
                                       T inv_2h, T inv_h) {
    if (i > 0 && i < n - 1) return (ld(v + idx + stride) - ld(v + idx - stride)) * inv_2h;
    if (i == 0) return (ld(v + idx + stride) - ld(v + idx)) * inv_h;
    return (ld(v + idx) - ld(v + idx - stride)) * inv_h;
}

// §3.8 eq. cutoff
template <typename T>
__device__ __forceinline__ T cutoff(const Params<T>& P, T u) {
    T a = fabs(u);
    if (a <= P.beta) return T(1);
    if (a <= P.gamma) {
        T m = a - P.gamma;
        return m * m * (T(2) * a + P.gamma - T(3) * P.beta) * P.inv_gb3;
    }
    return T(0);
}

template <typename T>
__device__ __forceinline__ T fast_div(T a, T b) {
    return a / b;
}
template <>
__device__ __forceinline__ float fast_div<float>(float a, float b) {
    return __fdividef(a, b);
}

// cell index and local coordinate along one axis for a foot at node index
// `i` plus a displacement `r` in units of h; the index-space coordinate is
// clamped to [0, n-1] and the cell to [0, n-2].
template <typename T>
__device__ __forceinline__ void locate_rel(int i, T r, int n, int& c, T& t) {
    const T big = T(4) * T(n) + T(8);
    r = fmin(fmax(r, -big), big);
    T f = floor(r);
    c = i + (int)f;
    t = r - f;
    if (c < 0) {
        c = 0;
        t = T(0);
    } else if (c >= n - 1) {
        c = n - 2;
        t = T(1);
    }
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Per-axis WENO coefficients at local coordinate θ: linear weights
// C_L = (2-θ)/3, C_R = (1+θ)/3 (eq. ckgamma) and q = θ(θ-1)/2.
template <typename T>
struct WenoAxis {
    T th, q, rho;  // θ, θ(θ-1)/2, C_L/C_R
    // C_L = (2-θ)/3, C_R = (1+θ)/3; set() divides with the fast reciprocal,
    // set_exact() with a correctly rounded division (folded at compile time
    // for a constant θ)
    __device__ __forceinline__ void set(T t) {
        th = t;
        q = T(0.5) * t * (t - T(1));
        rho = fast_div(T(2) - t, T(1) + t);
    }
    __device__ __forceinline__ void set_exact(T t) {
        th = t;
        q = T(0.5) * t * (t - T(1));
        rho = (T(2) - t) / (T(1) + t);
    }
};

// One-dimensional third-order WENO of §3.2 (eq. IWENO, n = 2) on the cell
// [x_j, x_{j+1}] with data v0..v3 = v_{j-1}..v_{j+2}. Algebraically equal to
// Σ w_k P_k with α_k = C_k/(I_k + h^2)^2 and I_k = D_k^2/h^2 (the quadratic
// forms A_L, A_R give the squared second differences D_L, D_R):
//   P_k(θ) = v_j + θ (v_{j+1} - v_j) + D_k θ(θ-1)/2,
//   w_L = ρ s_R^2 / (ρ s_R^2 + s_L^2),  s_k = D_k^2 + h^4,  ρ = C_L/C_R,
//   Σ w_k P_k = v_j + θ (v_{j+1} - v_j) + (D_R + w_L (D_L - D_R)) θ(θ-1)/2.
template <typename T>
__device__ __forceinline__ T weno1(T v0, T v1, T v2, T v3, const WenoAxis<T>& w, T h4) {
    const T dl = fma(T(-2), v1, v0 + v2);
    const T dr = fma(T(-2), v2, v1 + v3);
    const T sl = fma(dl, dl, h4), sr = fma(dr, dr, h4);
    const T gl = w.rho * (sr * sr);
    const T wl = fast_div(gl, fma(sl, sl, gl));
    return fma(w.q, fma(wl, dl - dr, dr), fma(w.th, v2 - v1, v1));
}

// Two-wide values for evaluating two interpolation lines at once. FP32 pairs
// use the packed two-wide add, multiply and FMA of sm_100 and later (each lane
// rounded to nearest, as the scalar operation), which halves the issued
// arithmetic; FP64 pairs are two scalar operations. a - b is written
// fma(-1, b, a), which rounds identically.
template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};
template <typename T>
using V2 = typename Vec2<T>::type;
__device__ __forceinline__ float2 v2_make(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 v2_make(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 v2_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 v2_add(double2 a, double2 b) { return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)); }
__device__ __forceinline__ float2 v2_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 v2_mul(double2 a, double2 b) { return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)); }
__device__ __forceinline__ float2 v2_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 v2_fma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
template <typename T>
__device__ __forceinline__ V2<T> v2_div(V2<T> a, V2<T> b) {
    return v2_make(fast_div(a.x, b.x), fast_div(a.y, b.y));
}

// Two lines at once (same axis, same θ): each result equals weno1 of its own
// data bit for bit.
template <typename T>
__device__ __forceinline__ void weno_pair(T a0, T a1, T a2, T a3, T b0, T b1, T b2, T b3, const WenoAxis<T>& w,
                                          T h4, T& ra, T& rb) {
    const V2<T> v0 = v2_make(a0, b0), v1 = v2_make(a1, b1), v2 = v2_make(a2, b2), v3 = v2_make(a3, b3);
    const V2<T> m2 = v2_make(T(-2), T(-2)), m1 = v2_make(T(-1), T(-1)), hh = v2_make(h4, h4);
    const V2<T> dl = v2_fma(m2, v1, v2_add(v0, v2));
    const V2<T> dr = v2_fma(m2, v2, v2_add(v1, v3));
    const V2<T> sl = v2_fma(dl, dl, hh), sr = v2_fma(dr, dr, hh);
    const V2<T> gl = v2_mul(v2_make(w.rho, w.rho), v2_mul(sr, sr));
    const V2<T> wl = v2_div<T>(gl, v2_fma(sl, sl, gl));
    const V2<T> t1 = v2_fma(wl, v2_fma(m1, dr, dl), dr);
    const V2<T> t2 = v2_fma(v2_make(w.th, w.th), v2_fma(m1, v1, v2), v1);
    const V2<T> res = v2_fma(v2_make(w.q, w.q), t1, t2);
    ra = res.x;
    rb = res.y;
}

// eq. IQ1 at node (i,j,k) + displacement r (units of h): multilinear
// interpolation in the cell holding the foot, along x, then y, then z.
template <typename T, int DIM>
__device__ __forceinline__ T interp_q1(const Params<T>& P, const T* __restrict__ u, int i, int j, int k,
                                       const T r[3]) {
    int cx, cy, cz = 0;
    T tx, ty, tz = T(0);
    locate_rel(i, r[0], P.n0, cx, tx);
    locate_rel(j, r[1], P.n1, cy, ty);
    if (DIM == 3) locate_rel(k, r[2], P.n2, cz, tz);
    long long b = (long long)cx + P.s1 * cy + P.s2 * cz;
    T v00 = ld(u + b), v10 = ld(u + b + 1), v01 = ld(u + b + P.s1), v11 = ld(u + b + P.s1 + 1);
    // lerps written as explicit FMAs, so that every kernel rounds them alike
    T a0 = fma(tx, v10 - v00, v00);
    T a1 = fma(tx, v11 - v01, v01);
    T s0 = fma(ty, a1 - a0, a0);
    if (DIM == 2) return s0;
    long long b2 = b + P.s2;
    T w00 = ld(u + b2), w10 = ld(u + b2 + 1), w01 = ld(u + b2 + P.s1), w11 = ld(u + b2 + P.s1 + 1);
    T c0 = fma(tx, w10 - w00, w00);
    T c1 = fma(tx, w11 - w01, w01);
    T s1 = fma(ty, c1 - c0, c0);
    return fma(tz, s1 - s0, s0);
}

// §3.2 WENO by dimension splitting: 16 lines along z, then 4 along y, then
// 1 along x (2-D: 4 along y, then 1 along x). Stencil nodes outside the grid
// repeat the edge node.
template <typename T, int DIM>
__device__ __forceinline__ T interp_weno(const Params<T>& P, const T* __restrict__ u, int i, int j, int k,
                                         const T r[3]) {
    int cx, cy, cz = 0;
    T tx, ty, tz = T(0);
    locate_rel(i, r[0], P.n0, cx, tx);
    locate_rel(j, r[1], P.n1, cy, ty);
    if (DIM == 3) locate_rel(k, r[2], P.n2, cz, tz);
    WenoAxis<T> wx, wy, wz;
    wx.set(tx);
    wy.set(ty);
    if (DIM == 3) wz.set(tz);
    const bool interior = cx >= 1 && cx <= P.n0 - 3 && cy >= 1 && cy <= P.n1 - 3 &&
                          (DIM == 2 || (cz >= 1 && cz <= P.n2 - 3));
    if (interior) {
        // whole stencil inside the grid: one base pointer, rows of four
        // consecutive x-values at 32-bit offsets (the grid holds fewer than
        // 2^31 nodes), z-lines evaluated in pairs as their rows arrive
        const T* base = u + ((cx - 1) + P.is1 * (cy - 1) + (DIM == 3 ? P.is2 * (cz - 1) : 0));
        T yv[4][4];  // [a][b]: z-line (DIM 3) or node value (DIM 2) at column a, row b
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            if (DIM == 3) {
                T r[4][4];  // [c][a]
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const T* row = base + (P.is1 * b + P.is2 * c);
#pragma unroll
                    for (int a = 0; a < 4; ++a) r[c][a] = ld(row + a);
                }
                weno_pair(r[0][0], r[1][0], r[2][0], r[3][0], r[0][1], r[1][1], r[2][1], r[3][1], wz, P.h4, yv[0][b],
                          yv[1][b]);
                weno_pair(r[0][2], r[1][2], r[2][2], r[3][2], r[0][3], r[1][3], r[2][3], r[3][3], wz, P.h4, yv[2][b],
                          yv[3][b]);
            } else {
                const T* row = base + P.is1 * b;
#pragma unroll
                for (int a = 0; a < 4; ++a) yv[a][b] = ld(row + a);
            }
        }
        T xv[4];
        weno_pair(yv[0][0], yv[0][1], yv[0][2], yv[0][3], yv[1][0], yv[1][1], yv[1][2], yv[1][3], wy, P.h4, xv[0], xv[1]);
        weno_pair(yv[2][0], yv[2][1], yv[2][2], yv[2][3], yv[3][0], yv[3][1], yv[3][2], yv[3][3], wy, P.h4, xv[2], xv[3]);
        return weno1(xv[0], xv[1], xv[2], xv[3], wx, P.h4);
    }
    int ox[4], oy[4], oz[4] = {0, 0, 0, 0};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        ox[a] = clampi(cx - 1 + a, 0, P.n0 - 1);
        oy[a] = P.is1 * clampi(cy - 1 + a, 0, P.n1 - 1);
        if (DIM == 3) oz[a] = P.is2 * clampi(cz - 1 + a, 0, P.n2 - 1);
    }
    T xv[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        T yv[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const T* col = u + (ox[a] + oy[b]);
            if (DIM == 3) {
                yv[b] = weno1(ld(col + oz[0]), ld(col + oz[1]), ld(col + oz[2]), ld(col + oz[3]), wz, P.h4);
            } else {
                yv[b] = ld(col);
            }
        }
        xv[a] = weno1(yv[0], yv[1], yv[2], yv[3], wy, P.h4);
    }
    return weno1(xv[0], xv[1], xv[2], xv[3], wx, P.h4);
}

template <typename T, int DIM, int INTERP>
__device__ __forceinline__ T interp_at(const Params<T>& P, const T* __restrict__ u, int i, int j, int k,
                                       const T r[3]) {
    if (INTERP == 1) return interp_weno<T, DIM>(P, u, i, j, k, r);
    return interp_q1<T, DIM>(P, u, i, j, k, r);
}

// §3.1: SL update of band node idx = (i,j,k) with value uc, before the cut.
// Scale factor C = (d_j/E_p)^(p-1) (1 for p = 1, 0 when E_p <= 0), times the
// cut-off c(φ_j) in band mode; feet x_j + C Δt ∇d + sqrt(C δ d Δt / p) σ λ
// (eq. SL2d / SL3d, σ of eq. sigma2d, ν1 ν2 of eq. sigma3d with the
// regularisation of §3.1); eq. SL:2 when |∇φ| < C_sing Δt^α.
template <typename T, int DIM, int INTERP>
__device__ T sl_update(const Params<T>& P, const T* __restrict__ u, const T* __restrict__ d, T Ep, int i, int j,
                       int k, long long idx, T uc) {
    T gx = diff_axis(u, idx, i, P.n0, 1ll, P.inv_2h, P.inv_h);
    T gy = diff_axis(u, idx, j, P.n1, P.s1, P.inv_2h, P.inv_h);
    T gz = DIM == 3 ? diff_axis(u, idx, k, P.n2, P.s2, P.inv_2h, P.inv_h) : T(0);
    T gn = sqrt(gx * gx + gy * gy + gz * gz);
    if (gn < P.sing_thr) {
        // eq. SL:2: mean of the face neighbours inside the grid (-x,+x,-y,+y,-z,+z)
        T s = T(0);
        int cnt = 0;
        if (i > 0) { s += ld(u + idx - 1); ++cnt; }
        if (i < P.n0 - 1) { s += ld(u + idx + 1); ++cnt; }
        if (j > 0) { s += ld(u + idx - P.s1); ++cnt; }
        if (j < P.n1 - 1) { s += ld(u + idx + P.s1); ++cnt; }
        if (DIM == 3) {
            if (k > 0) { s += ld(u + idx - P.s2); ++cnt; }
            if (k < P.n2 - 1) { s += ld(u + idx + P.s2); ++cnt; }
        }
        return s / T(cnt);
    }
    T dj = ld(d + idx);
    T C;
    if (P.p_kind == 1)
        C = T(1);
    else if (!(Ep > T(0)))
        C = T(0);
    else if (P.p_kind == 2)
        C = dj / Ep;
    else
        C = pow(dj / Ep, P.p - T(1));
    if (P.band) C *= cutoff(P, uc);
    T ddx = diff_axis(d, idx, i, P.n0, 1ll, P.inv_2h, P.inv_h);
    T ddy = diff_axis(d, idx, j, P.n1, P.s1, P.inv_2h, P.inv_h);
    T ddz = DIM == 3 ? diff_axis(d, idx, k, P.n2, P.s2, P.inv_2h, P.inv_h) : T(0);
    // displacements in units of h
    T adv = C * P.dt * P.inv_h;
    T bx = adv * ddx, by = adv * ddy, bz = adv * ddz;
    T s = sqrt(C * P.delta * dj * P.dt * P.inv_p) * P.inv_h;
    if (DIM == 2) {
        if (s == T(0)) {
            // δ = 0 (or C d = 0): the feet coincide; the same sum of equal terms
            const T r[3] = {bx, by, T(0)};
            const T f = interp_at<T, DIM, INTERP>(P, u, i, j, k, r);
            return (f + f) * T(0.5);
        }
        T sx = gy / gn, sy = -gx / gn;  // eq. sigma2d
        T r0[3] = {bx - s * sx, by - s * sy, T(0)};
        T r1[3] = {bx + s * sx, by + s * sy, T(0)};
        T a = interp_at<T, DIM, INTERP>(P, u, i, j, k, r0);
        T b = interp_at<T, DIM, INTERP>(P, u, i, j, k, r1);
        return (a + b) * T(0.5);
    }
    T n1x, n1y, n1z, n2x, n2y, n2z;
    if (gx == T(0) && gz == T(0)) {
        n1x = T(1); n1y = T(0); n1z = T(0);
        n2x = T(0); n2y = T(0); n2z = T(1);
    } else {
        T rr = sqrt(gx * gx + gz * gz);
        n1x = -gz / rr; n1y = T(0); n1z = gx / rr;
        T ig = T(1) / gn;
        n2x = ig * (-gx * gy / rr);
        n2y = ig * rr;
        n2z = ig * (-gy * gz / rr);
    }
    // δ = 0 (or C d = 0): the four feet coincide, so one interpolation
    // serves all of them, summed as in the general case
    const int nfeet = s == T(0) ? 1 : 4;
    T acc = T(0), last = T(0);
#pragma unroll 1
    for (int f = 0; f < nfeet; ++f) {
        T l1 = (f & 2) ? T(1) : T(-1);
        T l2 = (f & 1) ? T(1) : T(-1);
        T r[3] = {bx + s * (l1 * n1x + l2 * n2x), by + s * (l1 * n1y + l2 * n2y), bz + s * (l1 * n1z + l2 * n2z)};
        last = interp_at<T, DIM, INTERP>(P, u, i, j, k, r);
        acc += last;
    }
    if (nfeet == 1) acc = ((last + last) + last) + last;
    return acc * T(0.25);
}

// ordered block compaction helpers --------------------------------------------

// inclusive-exclusive prefix of one flag per thread across the block.
// Returns the exclusive offset of this thread; *total receives the block sum.
template <int BLOCK>
__device__ __forceinline__ int block_exclusive_flag(int flag, int* smem_warp, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned m = __ballot_sync(0xffffffffu, flag);
    int within = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) smem_warp[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < BLOCK / 32; ++w) {
            int c = smem_warp[w];
            smem_warp[w] = run;
            run += c;
        }
        smem_warp[BLOCK / 32] = run;
    }
    __syncthreads();
    *total = smem_warp[BLOCK / 32];
    return smem_warp[warp] + within;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// fixed-order block sum (result valid in thread 0); with warp_done the
// value of lane 0 of each warp is already that warp's sum
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v, double* smem, bool warp_done = false) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (!warp_done) v = warp_sum(v);
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < BLOCK / 32; ++w) r += smem[w];
    __syncthreads();
    return r;
}

#endif  // __CUDACC__

}  // namespace slr
