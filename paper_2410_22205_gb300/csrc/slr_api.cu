// C ABI of libslr (declared in include/slr.h): context lifecycle, argument
// validation, device memory through the injected allocator, and the
// per-iteration loop. One iteration (fused band+SL step, energy pass,
// record/stop kernel) is captured once as a CUDA graph and replayed; the
// iteration counter, the stop flag and the energy history live on the
// device, and the host reads a few status words every kChunk iterations.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "slr_internal.cuh"

using namespace slr;

namespace {

constexpr int kChunk = 8;  // graph replays between status reads in slr_evolve
constexpr uint32_t kStateMagic = 0x534c5231u;  // "SLR1"
thread_local std::string g_ctxless_error;  // see ctxless_error_clear()

slr_status fail(slr_ctx* c, slr_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

slr_status cuda_fail(slr_ctx* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return fail(c, SLR_E_CUDA, m);
}

#define CK(call, where)                                  \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return cuda_fail(c, _e, where); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

void free_graphs(slr_ctx* c) {
    if (c->g_evolve) cudaGraphExecDestroy(c->g_evolve);
    if (c->g_step) cudaGraphExecDestroy(c->g_step);
    c->g_evolve = nullptr;
    c->g_step = nullptr;
    c->g_step_override = -2.0;
}

void release(slr_ctx* c, void*& p) {
    dev_free(c, p);
    p = nullptr;
}

template <typename P>
void release_t(slr_ctx* c, P*& p) {
    void* v = (void*)p;
    dev_free(c, v);
    p = nullptr;
}

// capture one iteration into a graph template (not instantiated)
slr_status capture_step_graph(slr_ctx* c, double ov, int evolve, cudaGraph_t* out) {
    cudaGraph_t g = nullptr;
    long long l0 = c->launches;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    cudaError_t e1 = launch_step(c, ov, evolve);
    if (e1 == cudaSuccess && c->cfg.reinit) e1 = launch_reinit(c);
    cudaError_t e2 = e1 == cudaSuccess ? launch_energy(c, 1, -1.0, 1, evolve) : e1;
    cudaError_t e3 = cudaStreamEndCapture(c->stream, &g);
    c->launches = l0;
    if (e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e2, "capture of one iteration");
    }
    if (e3 != cudaSuccess) return cuda_fail(c, e3, "cudaStreamEndCapture");
    *out = g;
    return SLR_OK;
}

// capture one iteration as a graph
slr_status capture_step(slr_ctx* c, double ov, int evolve, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    long long l0 = c->launches;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    // external event-record nodes: recorded again at every replay
    cudaError_t e1 = c->profiling ? cudaEventRecordWithFlags(c->pev[0], c->stream, cudaEventRecordExternal) : cudaSuccess;
    if (e1 == cudaSuccess) e1 = launch_step(c, ov, evolve);
    if (e1 == cudaSuccess && c->profiling) e1 = cudaEventRecordWithFlags(c->pev[1], c->stream, cudaEventRecordExternal);
    if (e1 == cudaSuccess && c->cfg.reinit) e1 = launch_reinit(c);
    if (e1 == cudaSuccess && c->profiling) e1 = cudaEventRecordWithFlags(c->pev[2], c->stream, cudaEventRecordExternal);
    // launch_energy enqueues the front-cell, energy and record kernels
    cudaError_t e2 = e1 == cudaSuccess ? launch_energy(c, 1, -1.0, 1, evolve, c->profiling ? c->pev[3] : nullptr) : e1;
    if (e2 == cudaSuccess && c->profiling) e2 = cudaEventRecordWithFlags(c->pev[4], c->stream, cudaEventRecordExternal);
    cudaError_t e3 = cudaStreamEndCapture(c->stream, &g);
    c->launches = l0;  // captured kernels are counted per replay
    if (e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e2, "capture of one iteration");
    }
    if (e3 != cudaSuccess) return cuda_fail(c, e3, "cudaStreamEndCapture");
    cudaError_t e4 = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e4 != cudaSuccess) return cuda_fail(c, e4, "cudaGraphInstantiate");
    return SLR_OK;
}

// kernels of one iteration: step, front cells, energy, record, plus the
// reinitialisation stage (10 kernels and the sweeps) when it is on
long long kernels_per_iteration(const slr_ctx* c) {
    return 3 + (c->cfg.reinit ? 10 + reinit_sweeps(c) : 0);
}

slr_status read_status(slr_ctx* c, int* stop, int* error, int* n) {
    int* hp = c->host_pinned_flags;
    CK(cudaMemcpyAsync(hp + 0, &c->ds->stop, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status read");
    CK(cudaMemcpyAsync(hp + 1, &c->ds->error, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status read");
    CK(cudaMemcpyAsync(hp + 2, &c->ds->n, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status read");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (stop) *stop = hp[0];
    if (error) *error = hp[1];
    if (n) *n = hp[2];
    return SLR_OK;
}

slr_status check_device_error(slr_ctx* c) {
    int err = 0;
    slr_status s = read_status(c, nullptr, &err, nullptr);
    if (s != SLR_OK) return s;
    if (err & kErrBandOffset) return fail(c, SLR_E_STATE, "band-list offsets inconsistent with the band");
    if (err & kErrStage) return fail(c, SLR_E_TIMEOUT, "a shared-memory staging wait of the step gave up");
    if (err) return fail(c, SLR_E_STATE, "a device-side check failed");
    return SLR_OK;
}

// allocate the per-band buffers for a band of `count` nodes and the energy
// partials for `ncells` candidate cells
slr_status size_band_buffers(slr_ctx* c, long long count) {
    long long cap = count > 0 ? count : 1;
    release_t(c, c->band[0]);
    release_t(c, c->band[1]);
    release_t(c, c->part_dphi);
    release_t(c, c->tile_off);
    c->band[0] = (int*)dev_alloc(c, sizeof(int) * cap);
    c->band[1] = (int*)dev_alloc(c, sizeof(int) * cap);
    long long tiles = (cap + kStepTile - 1) / kStepTile + 1;
    c->part_dphi = (double*)dev_alloc(c, sizeof(double) * tiles);
    c->tile_off = (int*)dev_alloc(c, sizeof(int) * tiles);
    if (!c->band[0] || !c->band[1] || !c->part_dphi || !c->tile_off)
        return fail(c, SLR_E_NOMEM, "allocation of the band buffers failed");
    c->band_cap = cap;
    c->n_tiles_cap = tiles;
    return SLR_OK;
}

slr_status size_energy_buffers(slr_ctx* c, long long ncells) {
    release_t(c, c->part_e);
    c->n_echunks = (ncells + 31) / 32;
    c->part_e = (double*)dev_alloc(c, sizeof(double) * (2 * c->n_echunks + 2 + 3 * kRecordBlocks));  // + record blocks
    if (!c->part_e) return fail(c, SLR_E_NOMEM, "allocation of the energy buffers failed");
    return SLR_OK;
}

// the reinitialisation stage's scratch (cfg.reinit): field W, three
// bitmasks, compaction counts, per-node flags, Δ_φ partials
slr_status size_reinit_buffers(slr_ctx* c) {
    release(c, c->rw);
    release_t(c, c->bits_band);
    release_t(c, c->bits_gbar);
    release_t(c, c->bits_cell);
    release_t(c, c->rblk);
    release_t(c, c->rflags);
    release_t(c, c->part_dphi_r);
    const size_t words = reinit_bit_words(c);
    c->rw = dev_alloc(c, c->tsize * c->N);
    c->bits_band = (unsigned*)dev_alloc(c, sizeof(unsigned) * words);
    c->bits_gbar = (unsigned*)dev_alloc(c, sizeof(unsigned) * words);
    c->bits_cell = (unsigned*)dev_alloc(c, sizeof(unsigned) * words);
    c->rblk = (int*)dev_alloc(c, sizeof(int) * 2 * ((size_t)reinit_scan_blocks(c) + 1));
    c->rflags = (unsigned char*)dev_alloc(c, (size_t)c->N);
    c->part_dphi_r = (double*)dev_alloc(c, sizeof(double) * (size_t)reinit_grid(c));
    if (!c->rw || !c->bits_band || !c->bits_gbar || !c->bits_cell || !c->rblk || !c->rflags || !c->part_dphi_r)
        return fail(c, SLR_E_NOMEM, "allocation of the reinitialisation buffers failed");
    return SLR_OK;
}

bool same_config(const slr_config& a, const slr_config& b) { return memcmp(&a, &b, sizeof(slr_config)) == 0; }

}  // namespace

namespace slr {

slr_status evolve_prepare(slr_ctx* c) {
    if (!c->have_u) return fail(c, SLR_E_STATE, "evolve: initial level set not set");
    if (!c->g_evolve) {
        slr_status s = capture_step(c, -1.0, 1, &c->g_evolve);
        if (s != SLR_OK) return s;
    }
    CK(cudaMemsetAsync(&c->ds->stop, 0, sizeof(int), c->stream), "evolve");
    CK(cudaMemsetAsync(&c->ds->converged, 0, sizeof(int), c->stream), "evolve");
    return SLR_OK;
}

slr_status evolve_launch(slr_ctx* c) {
    CK(cudaGraphLaunch(c->g_evolve, c->stream), "cudaGraphLaunch");
    c->launches += kernels_per_iteration(c);
    return SLR_OK;
}

}  // namespace slr

namespace slr {

// the rest of slr_init_u once u[0] and u[1] hold φ^0 (write status e):
// device state, band list, candidate cells, the first energy
slr_status init_after_u(slr_ctx* c, cudaError_t e) {
    DeviceGuard g(c->device);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ds, 0, sizeof(DevState), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "init_u");
    if (c->cfg.band) {
        // with reinitialisation the band can grow: lists and cells get the
        // capacity of the whole grid, and the candidate-cell count lives on
        // the device
        const bool rei = c->cfg.reinit != 0;
        long long cnt = 0;
        CK(launch_count_band(c, &cnt), "init_u band count");
        slr_status s = size_band_buffers(c, rei ? c->N : cnt);
        if (s != SLR_OK) return s;
        CK(launch_build_band(c), "init_u band list");
        int ci = (int)cnt;
        CK(cudaMemcpyAsync(&c->ds->band_count[0], &ci, sizeof(int), cudaMemcpyHostToDevice, c->stream), "init_u");
        long long nc = 0;
        CK(launch_build_ecells(c, &nc, false), "init_u cell count");
        release_t(c, c->ecells);
        const long long ecap = rei ? c->ncells_all : nc;
        c->ecells = (int*)dev_alloc(c, sizeof(int) * (ecap > 0 ? ecap : 1));
        if (!c->ecells) return fail(c, SLR_E_NOMEM, "init_u: cell list allocation failed");
        c->n_ecells = ecap;
        CK(launch_build_ecells(c, &nc, true), "init_u cell list");
        s = size_energy_buffers(c, c->n_ecells);
        if (s != SLR_OK) return s;
        if (rei) {
            int nci = (int)nc;
            CK(cudaMemcpyAsync(&c->ds->n_ecells_dyn, &nci, sizeof(int), cudaMemcpyHostToDevice, c->stream), "init_u");
            CK(cudaMemcpyAsync(c->rw, c->u[0], c->tsize * c->N, cudaMemcpyDeviceToDevice, c->stream), "init_u");
        }
    }
    if (brick_mode(c)) {
        cudaError_t eb = bricks_init(c, c->u[0]);
        if (eb == cudaErrorMemoryAllocation) return fail(c, SLR_E_NOMEM, "init_u: brick lists allocation failed");
        CK(eb, "init_u bricks");
    }
    CK(launch_energy(c, 0, -1.0, 0, 0), "init_u energy");
    if (brick_mode(c)) CK(bricks_autotune(c), "init_u brick autotune");
    CK(cudaStreamSynchronize(c->stream), "init_u sync");
    c->have_u = true;
    return SLR_OK;
}

}  // namespace slr

namespace slr {
void ctxless_error_clear() { g_ctxless_error.clear(); }
slr_status ctxless_error_set(slr_status s, const std::string& msg) {
    g_ctxless_error = msg;
    return s;
}
const char* ctxless_error() { return g_ctxless_error.c_str(); }
}  // namespace slr

namespace slr {
slr_status cuda_status(slr_ctx* c, cudaError_t e, const char* where) { return cuda_fail(c, e, where); }
}  // namespace slr

extern "C" {

void slr_config_default(slr_config* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->dim = 3;
    cfg->n[0] = cfg->n[1] = cfg->n[2] = 64;
    for (int a = 0; a < 3; ++a) {
        cfg->lo[a] = -1.0;
        cfg->hi[a] = 1.0;
    }
    cfg->precision = 32;
    cfg->interp = 1;
    cfg->p = 2.0;
    cfg->delta = 1.0;
    cfg->dt = 0.0;
    cfg->band = 1;
    cfg->gamma = 0.0;
    cfg->beta = 0.0;
    cfg->c_sing = 1e-3;
    cfg->alpha = 1.0;
    cfg->energy_R = 5;
    cfg->stop_tol = 1e-4;
    cfg->stop_k = 10;
    cfg->min_iters = 10;
    cfg->max_iters = 100;
    cfg->reinit = 0;
    cfg->reinit_sweeps = 0;
    cfg->reinit_dtau = 0.0;
    cfg->step_kind = 0;
}

slr_status slr_create(const slr_config* cfg, const slr_allocator* alloc, void* cuda_stream, slr_ctx** out) {
    ctxless_error_clear();
    if (!cfg || !out) return ctxless_error_set(SLR_E_INVALID, "create: null argument");
    *out = nullptr;
    slr_ctx* c = new slr_ctx();
    c->cfg = *cfg;
    slr_config& k = c->cfg;
    auto bad = [&](const char* m) {
        ctxless_error_set(SLR_E_INVALID, m);
        delete c;
        return SLR_E_INVALID;
    };
    if (k.dim != 2 && k.dim != 3) return bad("dim must be 2 or 3");
    if (k.dim == 2) {
        if (k.n[2] != 1) return bad("n[2] must be 1 in 2-D");
        k.lo[2] = k.hi[2] = 0.0;
    }
    for (int a = 0; a < k.dim; ++a)
        if (k.n[a] < 4) return bad("need at least 4 nodes per axis");
    // every factor is positive here; bound each one before multiplying, so
    // the product cannot overflow
    long long N = 1;
    for (int a = 0; a < 3; ++a) {
        if (k.n[a] > 2147483647ll / N) return bad("at most 2^31-1 nodes");
        N *= k.n[a];
    }
    double h = (k.hi[0] - k.lo[0]) / (double)(k.n[0] - 1);
    if (!(h > 0.0) || !isfinite(h)) return bad("hi must exceed lo");
    for (int a = 1; a < k.dim; ++a) {
        double ha = (k.hi[a] - k.lo[a]) / (double)(k.n[a] - 1);
        if (!(fabs(ha - h) <= 1e-12 * h)) return bad("mesh width must be equal on every axis");
    }
    if (k.precision != 32 && k.precision != 64) return bad("precision must be 32 or 64");
    if (k.interp != 0 && k.interp != 1) return bad("interp must be 0 (Q1) or 1 (WENO)");
    if (!(k.p >= 1.0) || !isfinite(k.p)) return bad("p must be >= 1");
    if (!(k.delta >= 0.0)) return bad("delta must be >= 0");
    if (!(k.dt >= 0.0)) return bad("dt must be >= 0");
    if (k.band != 0 && k.band != 1) return bad("band must be 0 or 1");
    if (k.energy_R < 1 || k.energy_R > kMaxR) return bad("energy_R must be in 1..8");
    if (k.stop_k < 1 || k.stop_k > kMaxStopK || k.max_iters < 1 || k.min_iters < 0) return bad("bad stop parameters");
    if (k.max_iters >= kHist - 1) return bad("max_iters too large");
    if (!(k.c_sing >= 0.0)) return bad("c_sing must be >= 0");
    if (k.reinit != 0 && k.reinit != 1) return bad("reinit must be 0 or 1");
    if (k.reinit && !k.band) return bad("reinit needs the narrow band (band = 1)");
    if (k.reinit_sweeps < 0 || k.reinit_sweeps > 10000) return bad("reinit_sweeps must be in 0..10000");
    if (!(k.reinit_dtau >= 0.0) || !(k.reinit_dtau <= h / sqrt((double)k.dim) * (1.0 + 1e-12)))
        return bad("reinit_dtau must be in [0, h/sqrt(dim)]");
    if (k.step_kind < 0 || k.step_kind > 2) return bad("step_kind must be 0, 1 or 2");
    if (k.step_kind == 1 && (k.dim != 3 || k.reinit))
        return bad("step_kind 1 (bricks) needs a 3-D run without reinitialisation");
    c->h = h;
    c->dt = k.dt > 0.0 ? k.dt : h / 4.0;
    c->gamma = k.gamma > 0.0 ? k.gamma : (k.dim == 2 ? 4.0 : 6.0) * h;
    c->beta = k.beta > 0.0 ? k.beta : (k.dim == 2 ? 2.0 : 3.0) * h;
    if (!(c->beta < c->gamma)) return bad("beta must be smaller than gamma");
    c->N = N;
    c->ncells_all = (k.n[0] - 1) * (k.n[1] - 1) * (k.dim == 3 ? (k.n[2] - 1) : 1);
    c->tsize = k.precision == 32 ? 4 : 8;
    if (alloc && alloc->alloc && alloc->free) {
        c->al = *alloc;
        c->default_alloc = false;
    }
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return SLR_E_CUDA;
    }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (c->num_sms <= 0) c->num_sms = 1;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
        c->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return SLR_E_CUDA;
        }
        c->own_stream = true;
    }
    if (cudaMallocHost((void**)&c->host_pinned_flags, 64) != cudaSuccess) {
        cudaGetLastError();
        slr_destroy(c);
        return SLR_E_CUDA;
    }
    c->u[0] = dev_alloc(c, c->tsize * N);
    c->u[1] = dev_alloc(c, c->tsize * N);
    c->d = dev_alloc(c, c->tsize * N);
    c->argmin = (int*)dev_alloc(c, sizeof(int) * N);
    c->ds = (DevState*)dev_alloc(c, sizeof(DevState));
    if (!c->u[0] || !c->u[1] || !c->d || !c->argmin || !c->ds) {
        slr_destroy(c);
        return SLR_E_NOMEM;
    }
    if (cudaMemsetAsync(c->ds, 0, sizeof(DevState), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->argmin, 0xff, sizeof(int) * N, c->stream) != cudaSuccess) {
        cudaGetLastError();
        slr_destroy(c);
        return SLR_E_CUDA;
    }
    if (k.reinit && size_reinit_buffers(c) != SLR_OK) {
        slr_destroy(c);
        return SLR_E_NOMEM;
    }
    if (!k.band) {
        long long tiles = (N + kStepBlock - 1) / kStepBlock;
        c->part_dphi = (double*)dev_alloc(c, sizeof(double) * tiles);
        c->n_tiles_cap = tiles;
        if (!c->part_dphi || size_energy_buffers(c, c->ncells_all) != SLR_OK) {
            slr_destroy(c);
            return SLR_E_NOMEM;
        }
    }
    *out = c;
    return SLR_OK;
}

slr_status slr_load_cloud(slr_ctx* c, const double* xyz, int64_t n_points) {
    if (!c) return SLR_E_INVALID;
    if (!xyz || n_points < 1) return fail(c, SLR_E_INVALID, "load_cloud: need at least one point");
    if (n_points > 2147483647ll) return fail(c, SLR_E_INVALID, "load_cloud: at most 2^31-1 points");
    DeviceGuard g(c->device);
    release_t(c, c->pts);
    size_t bytes = sizeof(double) * (size_t)c->cfg.dim * (size_t)n_points;
    c->pts = (double*)dev_alloc(c, bytes);
    if (!c->pts) return fail(c, SLR_E_NOMEM, "load_cloud: allocation failed");
    CK(cudaMemcpyAsync(c->pts, xyz, bytes, cudaMemcpyHostToDevice, c->stream), "load_cloud copy");
    CK(cudaStreamSynchronize(c->stream), "load_cloud sync");
    c->npts = n_points;
    c->have_cloud = true;
    return SLR_OK;
}

slr_status slr_build_distance(slr_ctx* c) {
    if (!c) return SLR_E_INVALID;
    if (!c->have_cloud) return fail(c, SLR_E_STATE, "build_distance: no cloud loaded");
    DeviceGuard g(c->device);
    cudaError_t e = build_distance(c);
    if (e == cudaErrorInvalidValue) return fail(c, SLR_E_INVALID, "build_distance: non-finite point coordinates");
    if (e == cudaErrorMemoryAllocation) return fail(c, SLR_E_NOMEM, "build_distance: scratch allocation failed");
    if (e != cudaSuccess) return cuda_fail(c, e, "build_distance");
    c->have_d = true;
    return SLR_OK;
}

slr_status slr_build_distance_fsm(slr_ctx* c) {
    if (!c) return SLR_E_INVALID;
    if (!c->have_cloud) return fail(c, SLR_E_STATE, "build_distance_fsm: no cloud loaded");
    DeviceGuard g(c->device);
    cudaError_t e = build_distance_fsm(c);
    if (e == cudaErrorInvalidValue)
        return fail(c, SLR_E_INVALID, "build_distance_fsm: no point within a cell of the grid, or non-finite points");
    if (e == cudaErrorMemoryAllocation) return fail(c, SLR_E_NOMEM, "build_distance_fsm: scratch allocation failed");
    if (e == cudaErrorLaunchTimeout)
        return fail(c, SLR_E_TIMEOUT, "build_distance_fsm: a grid barrier of the fast sweeping waited too long");
    if (e != cudaSuccess) return cuda_fail(c, e, "build_distance_fsm");
    c->have_d = true;
    return SLR_OK;
}

slr_status slr_set_distance(slr_ctx* c, const double* d_host) {
    if (!c) return SLR_E_INVALID;
    if (!d_host) return fail(c, SLR_E_INVALID, "set_distance: null array");
    DeviceGuard g(c->device);
    double* tmp = (double*)dev_alloc(c, sizeof(double) * c->N);
    if (!tmp) return fail(c, SLR_E_NOMEM, "set_distance: staging allocation failed");
    cudaError_t e = cudaMemcpyAsync(tmp, d_host, sizeof(double) * c->N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_from_double(c, tmp, c->d, c->N);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->argmin, 0xff, sizeof(int) * c->N, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "set_distance");
    c->have_d = true;
    return SLR_OK;
}

slr_status slr_init_u(slr_ctx* c, int kind, const double* params, const double* u0_host) {
    if (!c) return SLR_E_INVALID;
    if (!c->have_d) return fail(c, SLR_E_STATE, "init_u: distance field not set");
    if (kind == 0 && !params) return fail(c, SLR_E_INVALID, "init_u: sphere needs {cx,cy,cz,r}");
    if (kind == 1 && !u0_host) return fail(c, SLR_E_INVALID, "init_u: array needs u0_host");
    if (kind == 2 && !(params && params[0] > 0.0))
        return fail(c, SLR_E_INVALID, "init_u: external marking needs {gamma_s > 0}");
    if (kind < 0 || kind > 2) return fail(c, SLR_E_INVALID, "init_u: kind must be 0, 1 or 2");
    DeviceGuard g(c->device);
    free_graphs(c);
    c->have_u = false;
    double* tmp = nullptr;
    double prm[4] = {0, 0, 0, 0};
    if (kind == 0)
        for (int a = 0; a < 4; ++a) prm[a] = params[a];
    if (kind == 1) {
        tmp = (double*)dev_alloc(c, sizeof(double) * c->N);
        if (!tmp) return fail(c, SLR_E_NOMEM, "init_u: staging allocation failed");
        cudaError_t e = cudaMemcpyAsync(tmp, u0_host, sizeof(double) * c->N, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) {
            dev_free(c, tmp);
            return cuda_fail(c, e, "init_u copy");
        }
    }
    if (kind == 2) {
        // §3.6: φ0 from d by external marking and fast sweeping (FP64), then
        // the array path (storage type, cut)
        tmp = (double*)dev_alloc(c, sizeof(double) * c->N);
        unsigned char* ext = (unsigned char*)dev_alloc(c, (size_t)c->N);
        cudaError_t e = (tmp && ext) ? launch_init_marking(c, params[0], tmp, ext) : cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        dev_free(c, ext);
        if (e != cudaSuccess) {
            dev_free(c, tmp);
            if (e == cudaErrorMemoryAllocation) return fail(c, SLR_E_NOMEM, "init_u: marking buffers");
            if (e == cudaErrorLaunchTimeout)
                return fail(c, SLR_E_TIMEOUT, "init_u: a grid barrier of the fast sweeping waited too long");
            return cuda_fail(c, e, "init_u marking");
        }
    }
    cudaError_t e = launch_init_u(c, kind == 2 ? 1 : kind, prm, tmp);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, tmp);
    return slr::init_after_u(c, e);
}

slr_status slr_step(slr_ctx* c, int n_steps, double energy_override) {
    if (!c) return SLR_E_INVALID;
    if (!c->have_u) return fail(c, SLR_E_STATE, "step: initial level set not set");
    if (n_steps < 0) return fail(c, SLR_E_INVALID, "step: negative step count");
    DeviceGuard g(c->device);
    double ov = energy_override >= 0.0 ? energy_override : -1.0;
    if (!c->g_step || c->g_step_override != ov) {
        if (c->g_step) cudaGraphExecDestroy(c->g_step);
        c->g_step = nullptr;
        slr_status s = capture_step(c, ov, 0, &c->g_step);
        if (s != SLR_OK) return s;
        c->g_step_override = ov;
    }
    CK(cudaMemsetAsync(&c->ds->stop, 0, sizeof(int), c->stream), "step");
    for (int i = 0; i < n_steps; ++i) {
        CK(cudaGraphLaunch(c->g_step, c->stream), "cudaGraphLaunch");
        c->launches += kernels_per_iteration(c);
    }
    CK(cudaStreamSynchronize(c->stream), "step sync");
    return check_device_error(c);
}

slr_status slr_batch_evolve(slr_ctx* const* jobs, int n_jobs, int chunk, void* cuda_stream, int* iters_out,
                            int* converged_out) {
    if (!jobs || n_jobs < 1) return SLR_E_INVALID;
    if (chunk == 0) chunk = 8;
    const bool tune = chunk < 0;
    if (!tune && chunk > 64) return fail(jobs[0], SLR_E_INVALID, "batch_evolve: chunk must be in 1..64 (or <= 0)");
    int dev = -1;
    for (int j = 0; j < n_jobs; ++j) {
        slr_ctx* c = jobs[j];
        if (!c) return SLR_E_INVALID;
        if (!c->have_u) return fail(c, SLR_E_STATE, "batch_evolve: a job has no initial level set");
        if (dev < 0) dev = c->device;
        if (c->device != dev) return fail(c, SLR_E_INVALID, "batch_evolve: jobs on different devices");
    }
    slr_ctx* c0 = jobs[0];
    DeviceGuard g(dev);
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c0->stream;
    // the batch graphs: per job a chain of `chunk` copies of its iteration
    // graph; with autotuning one graph per candidate chunk
    static const int kCand[] = {4, 8, 16, 32};
    constexpr int kNCand = 4;
    cudaGraphExec_t execs[kNCand] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<cudaGraph_t> tmpl(n_jobs, nullptr);
    slr_status status = SLR_OK;
    DevState** dstates = nullptr;
    int* dstop = nullptr;
    int* hstop = nullptr;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    auto cleanup = [&]() {
        for (auto& x : execs)
            if (x) cudaGraphExecDestroy(x);
        for (auto t : tmpl)
            if (t) cudaGraphDestroy(t);
        if (dstates) dev_free(c0, dstates);
        if (dstop) dev_free(c0, dstop);
        if (hstop) cudaFreeHost(hstop);
        for (auto x : ev)
            if (x) cudaEventDestroy(x);
    };
    for (int j = 0; j < n_jobs && status == SLR_OK; ++j) status = capture_step_graph(jobs[j], -1.0, 1, &tmpl[j]);
    if (status != SLR_OK) {
        cleanup();
        return status;
    }
    auto build = [&](int ch, cudaGraphExec_t* out) -> cudaError_t {
        cudaGraph_t parent = nullptr;
        cudaError_t e = cudaGraphCreate(&parent, 0);
        for (int j = 0; j < n_jobs && e == cudaSuccess; ++j) {
            cudaGraphNode_t prev = nullptr;
            for (int r = 0; r < ch && e == cudaSuccess; ++r) {
                cudaGraphNode_t node;
                e = cudaGraphAddChildGraphNode(&node, parent, prev ? &prev : nullptr, prev ? 1 : 0, tmpl[j]);
                prev = node;
            }
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(out, parent, 0);
        if (parent) cudaGraphDestroy(parent);
        return e;
    };
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < (tune ? kNCand : 1) && e == cudaSuccess; ++k) e = build(tune ? kCand[k] : chunk, &execs[k]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    // stop flags of all jobs gathered by one kernel into one array
    if (e == cudaSuccess) {
        dstates = (DevState**)dev_alloc(c0, sizeof(DevState*) * n_jobs);
        dstop = (int*)dev_alloc(c0, sizeof(int) * 4 * n_jobs);
        if (!dstates || !dstop) {
            cleanup();
            return fail(c0, SLR_E_NOMEM, "batch_evolve: allocation failed");
        }
        e = cudaMallocHost((void**)&hstop, sizeof(int) * 4 * n_jobs);
    }
    if (e == cudaSuccess) {
        std::vector<DevState*> hs(n_jobs);
        for (int j = 0; j < n_jobs; ++j) hs[j] = jobs[j]->ds;
        e = cudaMemcpyAsync(dstates, hs.data(), sizeof(DevState*) * n_jobs, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    // every job's own stream must be idle before the batch stream takes over
    for (int j = 0; j < n_jobs && e == cudaSuccess; ++j) e = cudaStreamSynchronize(jobs[j]->stream);
    for (int j = 0; j < n_jobs && e == cudaSuccess; ++j) {
        e = cudaMemsetAsync(&jobs[j]->ds->stop, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(&jobs[j]->ds->converged, 0, sizeof(int), st);
    }
    int max_iters = 0;
    for (int j = 0; j < n_jobs; ++j) max_iters = jobs[j]->cfg.max_iters > max_iters ? jobs[j]->cfg.max_iters : max_iters;
    // autotuning: the first launches try each candidate once (largest first)
    // and keep the one with the least device time per iteration and per node
    // of the jobs still running when the launch starts (jobs that stop within
    // a chunk are charged for its no-op iterations, the cost of a large
    // chunk); the iterations themselves do not depend on the chunk, so
    // neither do the results
    int cur = 0, tried = 0;
    float best_ms = 0.f;
    std::vector<char> running(n_jobs, 1);
    int best = 0;
    if (tune) cur = kNCand - 1;
    long long advanced = 0;
    int rounds = 0;
    while (e == cudaSuccess) {
        const int ch = tune ? kCand[cur] : chunk;
        const bool timing = tune && tried < kNCand;
        if (timing) e = cudaEventRecord(ev[0], st);
        if (e == cudaSuccess) e = cudaGraphLaunch(execs[tune ? cur : 0], st);
        if (e == cudaSuccess && timing) e = cudaEventRecord(ev[1], st);
        for (int j = 0; j < n_jobs; ++j) jobs[j]->launches += (long long)ch * kernels_per_iteration(jobs[j]);
        advanced += ch;
        if (e == cudaSuccess) e = launch_gather_status(c0, dstates, n_jobs, dstop, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hstop, dstop, sizeof(int) * 4 * n_jobs, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        ++rounds;
        if (timing) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (e != cudaSuccess) break;
            double work = 0.0;
            for (int j = 0; j < n_jobs; ++j)
                if (running[j]) work += (double)jobs[j]->N;
            const float per = work > 0.0 ? (float)(ms / ((double)ch * work)) : ms / (float)ch;
            if (tried == 0 || per < best_ms) {
                best_ms = per;
                best = cur;
            }
            ++tried;
            cur = tried < kNCand ? kNCand - 1 - tried : best;
        }
        bool all = true, err = false;
        for (int j = 0; j < n_jobs; ++j) {
            all = all && hstop[4 * j + 0];
            err = err || hstop[4 * j + 3];
            running[j] = !hstop[4 * j + 0];
        }
        if (err) {
            cleanup();
            return fail(c0, SLR_E_STATE, "batch_evolve: a device-side check failed in a job");
        }
        if (all) break;
        if (advanced > (long long)max_iters + 2 * 64) {
            cleanup();
            return fail(c0, SLR_E_STATE, "batch_evolve: stop flags never set");
        }
    }
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(c0, e, "batch_evolve");
    }
    c0->batch_chunk = tune ? kCand[best] : chunk;
    for (int j = 0; j < n_jobs; ++j) {
        if (iters_out) iters_out[j] = hstop[4 * j + 1];
        if (converged_out) converged_out[j] = hstop[4 * j + 2];
    }
    cleanup();
    return SLR_OK;
}

int slr_batch_chunk(const slr_ctx* first_job) { return first_job ? first_job->batch_chunk : 0; }


slr_status slr_batch_run(slr_ctx* const* jobs, int n_jobs, int autotune, void* cuda_stream, int* iters_out,
                         int* converged_out) {
    if (!jobs || n_jobs < 1) return SLR_E_INVALID;
    int dev = -1;
    for (int j = 0; j < n_jobs; ++j) {
        slr_ctx* c = jobs[j];
        if (!c) return SLR_E_INVALID;
        if (!c->have_u) return fail(c, SLR_E_STATE, "batch_run: a job has no initial level set");
        if (dev < 0) dev = c->device;
        if (c->device != dev) return fail(c, SLR_E_INVALID, "batch_run: jobs on different devices");
        if (!c->cfg.band)
            return fail(c, SLR_E_INVALID, "batch_run: a job runs on the whole grid (slr_batch_evolve takes it)");
        if (c->cfg.reinit)
            return fail(c, SLR_E_INVALID, "batch_run: a job runs the reinitialisation (slr_batch_evolve takes it)");
        if (c->cfg.dim == 3 && c->cfg.energy_R != 5)
            return fail(c, SLR_E_INVALID, "batch_run: a 3-D job's energy_R is not 5 (slr_batch_evolve takes it)");
        for (int i = 0; i < j; ++i)
            if (jobs[i] == c) return fail(c, SLR_E_INVALID, "batch_run: a job is listed twice");
    }
    slr_ctx* c0 = jobs[0];
    DeviceGuard g(dev);
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : c0->stream;
    // groups of one storage type and at most 64 jobs, in the caller's order
    int shape = -1, graph = 1, threads = 0, blocks = 0, bpi = 0;
    float tuned = 0.f;
    for (int prec : {32, 64}) {
        std::vector<slr_ctx*> grp;
        for (int j = 0; j < n_jobs; ++j)
            if (jobs[j]->cfg.precision == prec) grp.push_back(jobs[j]);
        for (size_t b = 0; b < grp.size(); b += 64) {
            const int m = (int)std::min<size_t>(64, grp.size() - b);
            int sh = autotune ? -1 : 0, gr = 0, th = 0, bl = 0, bp = 0;
            float tm = 0.f;
            const slr_status s = prec == 32
                                     ? batch_run_f32(grp.data() + b, m, autotune != 0, st, &sh, &gr, &tm, &th, &bl, &bp)
                                     : batch_run_f64(grp.data() + b, m, autotune != 0, st, &sh, &gr, &tm, &th, &bl, &bp);
            if (s == SLR_E_TIMEOUT) return fail(c0, s, "batch_run: a grid barrier of the batched kernel waited too long");
            if (s == SLR_E_STATE) return fail(c0, s, "batch_run: a device-side check failed in a job");
            if (s == SLR_E_NOMEM) return fail(c0, s, "batch_run: allocation failed");
            if (s != SLR_OK) {
                if (grp[b] != c0 && !grp[b]->err.empty()) c0->err = grp[b]->err;
                return s;
            }
            if (shape < 0) {
                shape = sh;
                tuned = tm;
                threads = th;
                blocks = bl;
                bpi = bp;
            }
            graph = graph && gr;
        }
    }
    c0->batch_threads = threads;
    c0->batch_blocks = blocks;
    c0->batch_bpi = bpi;
    c0->batch_graph = graph;
    c0->batch_tuned_ms = tuned;
    for (int j = 0; j < n_jobs; ++j) {
        if (iters_out) iters_out[j] = jobs[j]->batch_iters;
        if (converged_out) converged_out[j] = jobs[j]->batch_converged;
    }
    return SLR_OK;
}

slr_status slr_batch_run_info(const slr_ctx* first_job, int* threads, int* blocks_per_sm, int* bricks_per_item,
                              int* graph, float* tuned_ms) {
    if (!first_job) return SLR_E_INVALID;
    if (threads) *threads = first_job->batch_threads;
    if (blocks_per_sm) *blocks_per_sm = first_job->batch_blocks;
    if (bricks_per_item) *bricks_per_item = first_job->batch_bpi;
    if (graph) *graph = first_job->batch_graph;
    if (tuned_ms) *tuned_ms = first_job->batch_tuned_ms;
    return SLR_OK;
}

slr_status slr_step_async(slr_ctx* c, int n_steps, double energy_override) {
    if (!c) return SLR_E_INVALID;
    if (!c->have_u) return fail(c, SLR_E_STATE, "step_async: initial level set not set");
    if (n_steps < 0) return fail(c, SLR_E_INVALID, "step_async: negative step count");
    DeviceGuard g(c->device);
    double ov = energy_override >= 0.0 ? energy_override : -1.0;
    if (!c->g_step || c->g_step_override != ov) {
        if (c->g_step) cudaGraphExecDestroy(c->g_step);
        c->g_step = nullptr;
        slr_status s = capture_step(c, ov, 0, &c->g_step);
        if (s != SLR_OK) return s;
        c->g_step_override = ov;
    }
    CK(cudaMemsetAsync(&c->ds->stop, 0, sizeof(int), c->stream), "step_async");
    for (int i = 0; i < n_steps; ++i) {
        CK(cudaGraphLaunch(c->g_step, c->stream), "cudaGraphLaunch");
        c->launches += kernels_per_iteration(c);
    }
    return SLR_OK;
}

slr_status slr_set_profiling(slr_ctx* c, int on) {
    if (!c) return SLR_E_INVALID;
    DeviceGuard g(c->device);
    bool want = on != 0;
    if (want && !c->pev[0])
        for (int i = 0; i < 5; ++i) CK(cudaEventCreate(&c->pev[i]), "cudaEventCreate");
    if (want != c->profiling) free_graphs(c);
    c->profiling = want;
    return SLR_OK;
}

slr_status slr_last_iteration_times(slr_ctx* c, float ms[3]) {
    if (!c || !ms) return SLR_E_INVALID;
    if (!c->profiling) return fail(c, SLR_E_STATE, "last_iteration_times: profiling is off");
    DeviceGuard g(c->device);
    CK(cudaStreamSynchronize(c->stream), "last_iteration_times");
    // events: 0 before the step, 1 after it, 2 after the reinitialisation, 3 between energy and record, 4 after
    CK(cudaEventElapsedTime(&ms[0], c->pev[0], c->pev[1]), "cudaEventElapsedTime");
    CK(cudaEventElapsedTime(&ms[1], c->pev[2], c->pev[3]), "cudaEventElapsedTime");
    CK(cudaEventElapsedTime(&ms[2], c->pev[3], c->pev[4]), "cudaEventElapsedTime");
    return SLR_OK;
}

slr_status slr_last_iteration_phases(slr_ctx* c, float ms[4]) {
    if (!c || !ms) return SLR_E_INVALID;
    if (!c->profiling) return fail(c, SLR_E_STATE, "last_iteration_phases: profiling is off");
    DeviceGuard g(c->device);
    CK(cudaStreamSynchronize(c->stream), "last_iteration_phases");
    for (int i = 0; i < 4; ++i) CK(cudaEventElapsedTime(&ms[i], c->pev[i], c->pev[i + 1]), "cudaEventElapsedTime");
    return SLR_OK;
}

slr_status slr_evolve(slr_ctx* c, int* iters_out, int* converged_out) {
    if (!c) return SLR_E_INVALID;
    if (!c->have_u) return fail(c, SLR_E_STATE, "evolve: initial level set not set");
    DeviceGuard g(c->device);
    if (!c->g_evolve) {
        slr_status s = capture_step(c, -1.0, 1, &c->g_evolve);
        if (s != SLR_OK) return s;
    }
    CK(cudaMemsetAsync(&c->ds->stop, 0, sizeof(int), c->stream), "evolve");
    CK(cudaMemsetAsync(&c->ds->converged, 0, sizeof(int), c->stream), "evolve");
    int stop = 0, err = 0, n = 0;
    int guard = 0;
    while (!stop) {
        for (int i = 0; i < kChunk; ++i) {
            CK(cudaGraphLaunch(c->g_evolve, c->stream), "cudaGraphLaunch");
            c->launches += kernels_per_iteration(c);
        }
        slr_status s = read_status(c, &stop, &err, &n);
        if (s != SLR_OK) return s;
        if (err) return fail(c, SLR_E_STATE, "a device-side check failed (band-list offsets)");
        guard += kChunk;
        if (guard > c->cfg.max_iters + 2 * kChunk && !stop)
            return fail(c, SLR_E_STATE, "evolve: stop flag never set");
    }
    int conv = 0;
    CK(cudaMemcpyAsync(c->host_pinned_flags + 3, &c->ds->converged, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
       "evolve");
    CK(cudaStreamSynchronize(c->stream), "evolve sync");
    conv = c->host_pinned_flags[3];
    if (iters_out) *iters_out = n;
    if (converged_out) *converged_out = conv;
    return SLR_OK;
}

slr_status slr_extract(slr_ctx* c, double width, int64_t* idx, double* u, int64_t cap, int64_t* n_out) {
    if (!c) return SLR_E_INVALID;
    if (!c->have_u) return fail(c, SLR_E_STATE, "extract: no level set");
    if (!(width > 0.0)) return fail(c, SLR_E_INVALID, "extract: width must be > 0");
    DeviceGuard g(c->device);
    long long cnt = 0;
    CK(launch_extract(c, width, nullptr, nullptr, &cnt, false), "extract count");
    if (n_out) *n_out = cnt;
    if (!idx && !u) return SLR_OK;
    if (cnt > cap) return fail(c, SLR_E_CAPACITY, "extract: buffer too small");
    if (cnt == 0) return SLR_OK;
    long long* di = (long long*)dev_alloc(c, sizeof(long long) * cnt);
    double* dv = (double*)dev_alloc(c, sizeof(double) * cnt);
    if (!di || !dv) {
        dev_free(c, di);
        dev_free(c, dv);
        return fail(c, SLR_E_NOMEM, "extract: allocation failed");
    }
    cudaError_t e = launch_extract(c, width, di, dv, &cnt, true);
    if (e == cudaSuccess && idx)
        e = cudaMemcpyAsync(idx, di, sizeof(long long) * cnt, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, dv, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, di);
    dev_free(c, dv);
    if (e != cudaSuccess) return cuda_fail(c, e, "extract");
    return SLR_OK;
}

slr_status slr_get_field(slr_ctx* c, int which, void* host_out, int64_t cap) {
    if (!c) return SLR_E_INVALID;
    if (!host_out) return fail(c, SLR_E_INVALID, "get_field: null buffer");
    if (cap < c->N) return fail(c, SLR_E_CAPACITY, "get_field: buffer smaller than the grid");
    DeviceGuard g(c->device);
    if (which == SLR_FIELD_ARGMIN) {
        CK(cudaMemcpyAsync(host_out, c->argmin, sizeof(int) * c->N, cudaMemcpyDeviceToHost, c->stream), "get_field");
        CK(cudaStreamSynchronize(c->stream), "get_field");
        return SLR_OK;
    }
    if (which != SLR_FIELD_U && which != SLR_FIELD_D) return fail(c, SLR_E_INVALID, "get_field: unknown field");
    const void* src = c->d;
    if (which == SLR_FIELD_U) {
        int n = 0;
        slr_status s = read_status(c, nullptr, nullptr, &n);
        if (s != SLR_OK) return s;
        src = c->u[n & 1];
    }
    double* tmp = (double*)dev_alloc(c, sizeof(double) * c->N);
    if (!tmp) return fail(c, SLR_E_NOMEM, "get_field: staging allocation failed");
    cudaError_t e = launch_to_double(c, src, tmp, c->N);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, tmp, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_field");
    return SLR_OK;
}

slr_status slr_selftest_barrier(int unreachable) {
    ctxless_error_clear();
    if (unreachable < 0 || unreachable > 2) return ctxless_error_set(SLR_E_INVALID, "selftest_barrier: mode 0, 1 or 2");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return ctxless_error_set(SLR_E_CUDA, "selftest_barrier: no usable current device");
    }
    int err = 0;
    cudaError_t e = unreachable == 2 ? batch_wait_selftest(&err) : barrier_selftest(dev, unreachable, &err);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ctxless_error_set(SLR_E_CUDA, std::string("selftest_barrier: ") + cudaGetErrorString(e));
    }
    if (err & kErrBarrier)
        return ctxless_error_set(SLR_E_TIMEOUT, unreachable == 2 ? "selftest_barrier: the batched kernel's wait ran out"
                                                                 : "selftest_barrier: the barrier's wait ran out");
    return SLR_OK;
}

slr_status slr_l1_error(slr_ctx* c, int kind, const double* params, const double* exact_host, double* l1_out) {
    if (!c) return SLR_E_INVALID;
    if (!l1_out) return fail(c, SLR_E_INVALID, "l1_error: null output");
    if (kind == 0 && !(params && params[3] >= 0.0 && std::isfinite(params[0]) && std::isfinite(params[1]) &&
                       std::isfinite(params[2]) && std::isfinite(params[3])))
        return fail(c, SLR_E_INVALID, "l1_error: a sphere needs finite {cx, cy, cz, r >= 0}");
    if (kind == 1 && !exact_host) return fail(c, SLR_E_INVALID, "l1_error: null exact array");
    if (kind < 0 || kind > 1) return fail(c, SLR_E_INVALID, "l1_error: kind must be 0 or 1");
    if (!c->have_u) return fail(c, SLR_E_STATE, "l1_error: no level set");
    DeviceGuard g(c->device);
    int n = 0;
    slr_status s = read_status(c, nullptr, nullptr, &n);
    if (s != SLR_OK) return s;
    const int blocks = c->num_sms * 4;
    const size_t pbytes = (sizeof(double) * (size_t)blocks + 255) & ~size_t(255);
    char* tmp = (char*)dev_alloc(c, pbytes + (kind == 1 ? sizeof(double) * (size_t)c->N : 0));
    if (!tmp) return fail(c, SLR_E_NOMEM, "l1_error: scratch allocation failed");
    double* part = (double*)tmp;
    double* ex = kind == 1 ? (double*)(tmp + pbytes) : nullptr;
    std::vector<double> hp((size_t)blocks);
    cudaError_t e = cudaSuccess;
    if (kind == 1) e = cudaMemcpyAsync(ex, exact_host, sizeof(double) * (size_t)c->N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_l1_error(c, c->u[n & 1], kind, params, ex, part, blocks);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * (size_t)blocks, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "l1_error");
    double sum = 0.0;
    for (int b = 0; b < blocks; ++b) sum += hp[(size_t)b];
    double vol = c->h * c->h;
    if (c->cfg.dim == 3) vol *= c->h;
    *l1_out = sum * vol;
    return SLR_OK;
}

slr_status slr_get_band(slr_ctx* c, int64_t* idx, int64_t cap, int64_t* n_out) {
    if (!c) return SLR_E_INVALID;
    if (!c->have_u) return fail(c, SLR_E_STATE, "get_band: no level set");
    DeviceGuard g(c->device);
    if (!c->cfg.band) {
        if (n_out) *n_out = c->N;
        if (!idx) return SLR_OK;
        if (cap < c->N) return fail(c, SLR_E_CAPACITY, "get_band: buffer too small");
        for (long long i = 0; i < c->N; ++i) idx[i] = i;
        return SLR_OK;
    }
    int n = 0;
    slr_status s = read_status(c, nullptr, nullptr, &n);
    if (s != SLR_OK) return s;
    int cnt = 0;
    int* list = c->band[n & 1];
    if (brick_mode(c) && c->brick.list_iter != n) {
        // the brick step keeps no list: the band the last step updated is
        // {|u| < γ} of that step's input (φ^0 before any step)
        long long lc = 0;
        list = c->band[0];
        CK(band_of_field(c, c->u[n >= 1 ? ((n - 1) & 1) : 0], list, &lc), "get_band");
        cnt = (int)lc;
    } else {
        if (brick_mode(c)) list = c->band[0];
        CK(cudaMemcpyAsync(&cnt, &c->ds->band_count[n & 1], sizeof(int), cudaMemcpyDeviceToHost, c->stream),
           "get_band");
        CK(cudaStreamSynchronize(c->stream), "get_band");
    }
    if (n_out) *n_out = cnt;
    if (!idx) return SLR_OK;
    if (cnt > cap) return fail(c, SLR_E_CAPACITY, "get_band: buffer too small");
    int* tmp = (int*)malloc(sizeof(int) * (cnt > 0 ? cnt : 1));
    if (!tmp) return fail(c, SLR_E_NOMEM, "get_band: host allocation failed");
    cudaError_t e = cudaMemcpyAsync(tmp, list, sizeof(int) * cnt, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess)
        for (int i = 0; i < cnt; ++i) idx[i] = tmp[i];
    free(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "get_band");
    return SLR_OK;
}

slr_status slr_energy(slr_ctx* c, double p, double* E_out, double* sum_out) {
    if (!c) return SLR_E_INVALID;
    if (!c->have_u) return fail(c, SLR_E_STATE, "energy: no level set");
    if (!(p >= 1.0)) return fail(c, SLR_E_INVALID, "energy: p must be >= 1");
    DeviceGuard g(c->device);
    CK(launch_energy(c, 0, p, 2, 0), "energy");
    double rep[2] = {0, 0};
    CK(cudaMemcpyAsync(rep, c->part_e + 2 * c->n_echunks, sizeof(rep), cudaMemcpyDeviceToHost, c->stream), "energy");
    CK(cudaStreamSynchronize(c->stream), "energy");
    if (sum_out) *sum_out = rep[0];
    if (E_out) *E_out = pow(rep[0], 1.0 / p);
    return SLR_OK;
}

slr_status slr_diagnostics(slr_ctx* c, double* e2_hist, double* dphi_hist, int64_t* band_hist, int cap, int* n_out,
                           double* err_cloud) {
    if (!c) return SLR_E_INVALID;
    if (!c->have_u) return fail(c, SLR_E_STATE, "diagnostics: no level set");
    DeviceGuard g(c->device);
    DevState* h = (DevState*)malloc(sizeof(DevState));
    if (!h) return fail(c, SLR_E_NOMEM, "diagnostics: host allocation failed");
    cudaError_t e = cudaMemcpyAsync(h, c->ds, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free(h);
        return cuda_fail(c, e, "diagnostics");
    }
    int n = h->n;
    if (n_out) *n_out = n;
    int first = n + 1 > kHist ? n + 1 - kHist : 0;
    for (int i = 0; i <= n && i - first < cap; ++i) {
        if (i < first) continue;
        if (e2_hist) e2_hist[i - first] = h->e2_hist[i % kHist];
        if (i < n) {
            if (dphi_hist) dphi_hist[i - first] = h->dphi_hist[i % kHist];
            if (band_hist) band_hist[i - first] = h->band_hist[i % kHist];
        }
    }
    free(h);
    if (err_cloud) {
        if (!c->have_cloud) return fail(c, SLR_E_STATE, "diagnostics: Err_S needs the cloud");
        double* dv = (double*)dev_alloc(c, sizeof(double));
        if (!dv) return fail(c, SLR_E_NOMEM, "diagnostics: allocation failed");
        cudaError_t e2 = launch_err_cloud(c, dv);
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(err_cloud, dv, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(c->stream);
        dev_free(c, dv);
        if (e2 != cudaSuccess) return cuda_fail(c, e2, "Err_S");
    }
    return SLR_OK;
}

// checkpoint layout: header, config, DevState, band list, cell list, u, d, argmin
struct StateHeader {
    uint32_t magic;
    uint32_t tsize;
    int64_t N;
    int64_t band_count;
    int64_t n_ecells;
};

slr_status slr_export_state(slr_ctx* c, void* buf, int64_t cap, int64_t* n_out) {
    if (!c) return SLR_E_INVALID;
    if (!c->have_u) return fail(c, SLR_E_STATE, "export_state: no level set");
    DeviceGuard g(c->device);
    int n = 0;
    slr_status s = read_status(c, nullptr, nullptr, &n);
    if (s != SLR_OK) return s;
    int cnt = 0;
    int* list = c->band[n & 1];
    const bool bricked = brick_mode(c);
    if (c->cfg.band && bricked) {
        // the band the last step updated (see slr_get_band), rebuilt into band[0]
        long long lc = 0;
        list = c->band[0];
        if (c->brick.list_iter != n)
            CK(band_of_field(c, c->u[n >= 1 ? ((n - 1) & 1) : 0], list, &lc), "export");
        else {
            CK(cudaMemcpyAsync(&cnt, &c->ds->band_count[n & 1], sizeof(int), cudaMemcpyDeviceToHost, c->stream),
               "export");
            CK(cudaStreamSynchronize(c->stream), "export");
            lc = cnt;
        }
        cnt = (int)lc;
    } else if (c->cfg.band) {
        CK(cudaMemcpyAsync(&cnt, &c->ds->band_count[n & 1], sizeof(int), cudaMemcpyDeviceToHost, c->stream), "export");
        CK(cudaStreamSynchronize(c->stream), "export");
    }
    long long ncell = c->cfg.band ? c->n_ecells : 0;
    if (c->cfg.reinit) {
        int nd = 0;
        CK(cudaMemcpyAsync(&nd, &c->ds->n_ecells_dyn, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "export");
        CK(cudaStreamSynchronize(c->stream), "export");
        ncell = nd;
    }
    StateHeader hd{kStateMagic, (uint32_t)c->tsize, c->N, cnt, ncell};
    size_t need = sizeof(hd) + sizeof(slr_config) + sizeof(DevState) + sizeof(int) * (size_t)cnt +
                  sizeof(int) * (size_t)hd.n_ecells + c->tsize * 2 * c->N + sizeof(int) * c->N;
    if (n_out) *n_out = (int64_t)need;
    if (!buf || cap < (int64_t)need) return fail(c, SLR_E_CAPACITY, "export_state: buffer too small");
    char* p = (char*)buf;
    memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    memcpy(p, &c->cfg, sizeof(slr_config));
    p += sizeof(slr_config);
    CK(cudaMemcpyAsync(p, c->ds, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "export");
    p += sizeof(DevState);
    if (cnt) CK(cudaMemcpyAsync(p, list, sizeof(int) * cnt, cudaMemcpyDeviceToHost, c->stream), "export");
    p += sizeof(int) * cnt;
    if (hd.n_ecells)
        CK(cudaMemcpyAsync(p, c->ecells, sizeof(int) * hd.n_ecells, cudaMemcpyDeviceToHost, c->stream), "export");
    p += sizeof(int) * hd.n_ecells;
    CK(cudaMemcpyAsync(p, c->u[n & 1], c->tsize * c->N, cudaMemcpyDeviceToHost, c->stream), "export");
    p += c->tsize * c->N;
    CK(cudaMemcpyAsync(p, c->d, c->tsize * c->N, cudaMemcpyDeviceToHost, c->stream), "export");
    p += c->tsize * c->N;
    CK(cudaMemcpyAsync(p, c->argmin, sizeof(int) * c->N, cudaMemcpyDeviceToHost, c->stream), "export");
    CK(cudaStreamSynchronize(c->stream), "export");
    return SLR_OK;
}

slr_status slr_import_state(slr_ctx* c, const void* buf, int64_t nbytes) {
    if (!c) return SLR_E_INVALID;
    if (!buf || nbytes < (int64_t)(sizeof(StateHeader) + sizeof(slr_config)))
        return fail(c, SLR_E_INVALID, "import_state: buffer too small");
    DeviceGuard g(c->device);
    const char* p = (const char*)buf;
    StateHeader hd;
    memcpy(&hd, p, sizeof(hd));
    p += sizeof(hd);
    slr_config cfg;
    memcpy(&cfg, p, sizeof(cfg));
    p += sizeof(cfg);
    if (hd.magic != kStateMagic || hd.tsize != c->tsize || hd.N != c->N || !same_config(cfg, c->cfg))
        return fail(c, SLR_E_INVALID, "import_state: state of a different configuration");
    size_t need = sizeof(hd) + sizeof(slr_config) + sizeof(DevState) + sizeof(int) * (size_t)hd.band_count +
                  sizeof(int) * (size_t)hd.n_ecells + c->tsize * 2 * c->N + sizeof(int) * c->N;
    if (nbytes < (int64_t)need) return fail(c, SLR_E_INVALID, "import_state: truncated buffer");
    free_graphs(c);
    DevState* hds = (DevState*)malloc(sizeof(DevState));
    if (!hds) return fail(c, SLR_E_NOMEM, "import_state: host allocation failed");
    memcpy(hds, p, sizeof(DevState));
    p += sizeof(DevState);
    const int n = hds->n;
    if (c->cfg.band) {
        const bool rei = c->cfg.reinit != 0;
        slr_status s = size_band_buffers(c, rei ? c->N : hd.band_count);
        if (s == SLR_OK) {
            release_t(c, c->ecells);
            const long long ecap = rei ? c->ncells_all : hd.n_ecells;
            c->ecells = (int*)dev_alloc(c, sizeof(int) * (ecap > 0 ? ecap : 1));
            c->n_ecells = ecap;
            if (!c->ecells) s = fail(c, SLR_E_NOMEM, "import_state: allocation failed");
        }
        if (s == SLR_OK) s = size_energy_buffers(c, c->n_ecells);
        if (s != SLR_OK) {
            free(hds);
            return s;
        }
    }
    cudaError_t e = cudaMemcpyAsync(c->ds, hds, sizeof(DevState), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    free(hds);
    if (e != cudaSuccess) return cuda_fail(c, e, "import_state");
    const bool bricked = brick_mode(c);
    if (hd.band_count)
        CK(cudaMemcpyAsync(c->band[bricked ? 0 : (n & 1)], p, sizeof(int) * hd.band_count, cudaMemcpyHostToDevice,
                           c->stream),
           "import");
    if (bricked) {
        // the band count sits where slr_get_band reads it until the next step
        int bc = (int)hd.band_count;
        CK(cudaMemcpyAsync(&c->ds->band_count[n & 1], &bc, sizeof(int), cudaMemcpyHostToDevice, c->stream), "import");
    }
    p += sizeof(int) * hd.band_count;
    if (hd.n_ecells)
        CK(cudaMemcpyAsync(c->ecells, p, sizeof(int) * hd.n_ecells, cudaMemcpyHostToDevice, c->stream), "import");
    p += sizeof(int) * hd.n_ecells;
    CK(cudaMemcpyAsync(c->u[0], p, c->tsize * c->N, cudaMemcpyHostToDevice, c->stream), "import");
    CK(cudaMemcpyAsync(c->u[1], p, c->tsize * c->N, cudaMemcpyHostToDevice, c->stream), "import");
    p += c->tsize * c->N;
    CK(cudaMemcpyAsync(c->d, p, c->tsize * c->N, cudaMemcpyHostToDevice, c->stream), "import");
    p += c->tsize * c->N;
    CK(cudaMemcpyAsync(c->argmin, p, sizeof(int) * c->N, cudaMemcpyHostToDevice, c->stream), "import");
    if (c->cfg.reinit)
        CK(cudaMemcpyAsync(c->rw, c->u[0], c->tsize * c->N, cudaMemcpyDeviceToDevice, c->stream), "import");
    if (bricked) {
        // active bricks of the imported state; both buffers hold it, and the
        // Δ_φ partials are keyed by brick id, so an uninterrupted run and the
        // resumed one sum the same partials in the same order
        cudaError_t eb = bricks_init(c, c->u[0]);
        if (eb == cudaErrorMemoryAllocation) return fail(c, SLR_E_NOMEM, "import_state: brick lists allocation failed");
        CK(eb, "import bricks");
        c->brick.list_iter = c->cfg.band ? n : -1;
    }
    // an energy pass in report mode recomputes the band-tile offsets the
    // next step reads (the history and E_p stay as imported)
    CK(launch_energy(c, 0, c->cfg.p, 2, 0), "import energy pass");
    if (bricked) CK(bricks_autotune(c), "import brick autotune");
    CK(cudaStreamSynchronize(c->stream), "import");
    c->have_d = true;
    c->have_u = true;
    return SLR_OK;
}

int64_t slr_kernel_launches(const slr_ctx* c) { return c ? c->launches : 0; }

slr_status slr_brick_shape_set(slr_ctx* c, int threads, int stages) {
    if (!c) return SLR_E_INVALID;
    if (!brick_mode(c) || !c->have_u) return fail(c, SLR_E_STATE, "brick_shape_set: no brick-staged step");
    const int sh = brick_shape_index(threads, stages);
    if (sh < 0) return fail(c, SLR_E_INVALID, "brick_shape_set: threads must be 128 or 256 and stages 1 or 2");
    free_graphs(c);  // the captured iteration holds the old launch
    c->brick.shape = sh;
    return SLR_OK;
}

slr_status slr_brick_shape(const slr_ctx* c, int* threads, int* stages, float* trial_ms) {
    if (!c) return SLR_E_INVALID;
    if (!brick_mode(c) || !c->have_u) return SLR_E_STATE;
    brick_shape_of(c, threads, stages, trial_ms);
    return SLR_OK;
}

const char* slr_last_error(const slr_ctx* c) {
    if (c) return c->err.c_str();
    return g_ctxless_error.c_str();
}

void slr_destroy(slr_ctx* c) {
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_graphs(c);
    release(c, c->u[0]);
    release(c, c->u[1]);
    release(c, c->d);
    release_t(c, c->argmin);
    release_t(c, c->pts);
    release_t(c, c->band[0]);
    release_t(c, c->band[1]);
    release_t(c, c->ecells);
    release_t(c, c->part_dphi);
    release_t(c, c->part_e);
    release_t(c, c->tile_off);
    release(c, c->rw);
    release_t(c, c->bits_band);
    release_t(c, c->bits_gbar);
    release_t(c, c->bits_cell);
    release_t(c, c->rblk);
    release_t(c, c->rflags);
    release_t(c, c->part_dphi_r);
    bricks_free(c);
    release_t(c, c->ds);
    if (c->host_pinned_flags) cudaFreeHost(c->host_pinned_flags);
    for (int i = 0; i < 5; ++i)
        if (c->pev[i]) cudaEventDestroy(c->pev[i]);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    delete c;
}

}  // extern "C"
