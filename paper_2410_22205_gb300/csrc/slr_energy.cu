// Energy functional, stopping criterion and diagnostics (arXiv 2410.22205,
// §3.5 and §4), all on the device with FP64 accumulation.
//
// Energy: the candidate cells (every cell in whole-grid mode; in band mode
// the cells touching the initial band or crossing the front at init) are
// checked 1024 per block slot for a sign change (front cells, vertices of
// both signs, zero counted as positive), which the block then processes:
//   2-D: edge crossings by linear interpolation of φ, d interpolated along
//        the edge, trapezoid rule on the segment(s) (eq. energyApprox);
//   3-D: R^3 subcells (eq. energyApproxFiner); φ at the subcell centres by
//        the active interpolator — for WENO the dimension splitting shares
//        work across the regular R×R×R lattice (16R z-evaluations, then 4R^2
//        along y, then R^3 along x, all with the same arithmetic as a single
//        point evaluation); d by Q1; a subcell counts when
//        |φ(x')| < (√3/2)Δx' and adds |d(x')|^p (Δx')^2.
// Each block writes one FP64 partial per sum and one block reduces the
// partials in a fixed order, so results are bit-reproducible.
#include "slr_energy.cuh"
#include "slr_internal.cuh"

namespace slr {

template <typename T>
Params<T> make_params(const slr_ctx* c);

// grid of the energy pass: one block per 1024 candidate cells (one partial
// pair per block)
// slots of 1024 candidate cells (the capacity of the list with the
// reinitialisation on), and the energy kernels' grid, which takes slots from
// a ticket
long long energy_slots(const slr_ctx* c) {
    long long ncells = c->cfg.band ? c->n_ecells : c->ncells_all;
    return (ncells + 1023) / 1024;
}

long long energy_blocks(const slr_ctx* c) {
    long long b = energy_slots(c);
    const long long cap = (long long)c->num_sms * 6;
    if (b > cap) b = cap;
    return b < 1 ? 1 : b;
}


// Energy pass of one job, one launch. Blocks take slots of kEnergyCand
// candidate cells from a ticket; per slot the block collects the front cells
// (vertices of both signs, zero counted as positive) in candidate order and
// runs their quadrature (energy_slot). In band mode with the list step its
// warps first count, per tile of kStepTile entries of the band list the next
// step reads, the members |φ| < γ; the record kernel turns the counts into
// offsets. No ordering across blocks is needed, and the block scheduler
// evens out the uneven slot sizes.
template <typename T, int DIM, int INTERP, int RC>
__global__ void __launch_bounds__(kEnergyThreads, (DIM == 3 && sizeof(T) == 4) ? 4 : 1) k_energy(Params<T> P, const T* ub0, const T* ub1,
                                                           const T* __restrict__ d, const int* __restrict__ cells,
                                                           long long ncells_host,
                                                           const int* ncells_dev, EnergyArgs<T> E, int offset,
                                                           double* part, const int* L0, const int* L1,
                                                           int* __restrict__ tile_cnt, DevState* ds, int check_stop) {
    constexpr int W = kEnergyThreads / 32;
    __shared__ EnergyWs<T> ws;
    __shared__ long long s_sb;
    if (check_stop && ds->stop) return;
    const int sel = (ds->n + offset) & 1;
    const T* __restrict__ u = sel ? ub1 : ub0;
    if (tile_cnt) {
        const int nb = ds->band_count[sel];
        const int* Lb = sel ? L1 : L0;
        const int ntb = (nb + kStepTile - 1) / kStepTile;
        const int nw = gridDim.x * W;
        for (int t = blockIdx.x * W + (threadIdx.x >> 5); t < ntb; t += nw) tile_count<T>(P, u, Lb, nb, t, tile_cnt);
    }
    energy_setup<T, RC>(ws, E.R);
    __syncthreads();
    const long long ncells = ncells_dev ? (long long)*ncells_dev : ncells_host;
    const long long nslots = (ncells + kEnergyCand - 1) / kEnergyCand;
    for (;;) {
        if (threadIdx.x == 0) s_sb = (long long)atomicAdd(&ds->eticket[1], 1u);
        __syncthreads();
        const long long sb = s_sb;
        __syncthreads();
        if (sb >= nslots) break;
        energy_slot<T, DIM, INTERP, RC, kEnergyThreads>(P, u, d, cells, ncells, sb, E, part, ws);
    }
}

// Reduction of the step and energy partials and the bookkeeping of one
// iteration (record_slice): kRecordBlocks blocks, one slice each.
__global__ void __launch_bounds__(kRecordThreads) k_record(RecordArgs A, DevState* ds) {
    __shared__ RecordWs ws;
    record_slice<kRecordThreads>(A, ds, blockIdx.x, gridDim.x, ws);
}

template <typename T>
EnergyArgs<T> energy_args(const slr_ctx* c, double p, int p_kind) {
    EnergyArgs<T> E;
    E.R = c->cfg.energy_R;
    E.h = c->h;
    E.p = p;
    E.p_kind = p_kind;
    const double hp = c->h / c->cfg.energy_R;
    E.thr = (T)(0.8660254037844386 * hp);
    E.hp2 = (T)(hp * hp);
    E.pT = (T)p;
    return E;
}
template EnergyArgs<float> energy_args<float>(const slr_ctx*, double, int);
template EnergyArgs<double> energy_args<double>(const slr_ctx*, double, int);

template <typename T, int DIM, int INTERP>
static cudaError_t energy_t(slr_ctx* c, int offset, double p, int p_kind, int check_stop) {
    Params<T> P = make_params<T>(c);
    const int* cells = c->cfg.band ? c->ecells : nullptr;
    long long ncells = c->cfg.band ? c->n_ecells : c->ncells_all;
    const int blocks = (int)energy_blocks(c);
    const EnergyArgs<T> E = energy_args<T>(c, p, p_kind);
    const int* ncells_dev = c->cfg.reinit ? &c->ds->n_ecells_dyn : nullptr;  // the list changes every iteration
    // the list step reads per-tile counts of the band list; the brick step does not
    int* tile_cnt = (c->cfg.band && !brick_mode(c)) ? c->tile_off : nullptr;
    if (DIM == 3 && c->cfg.energy_R == 5)
        k_energy<T, DIM, INTERP, 5><<<blocks, kEnergyThreads, 0, c->stream>>>(
            P, (const T*)c->u[0], (const T*)c->u[1], (const T*)c->d, cells, ncells, ncells_dev, E, offset, c->part_e,
            c->band[0], c->band[1], tile_cnt, c->ds, check_stop);
    else
        k_energy<T, DIM, INTERP, 0><<<blocks, kEnergyThreads, 0, c->stream>>>(
            P, (const T*)c->u[0], (const T*)c->u[1], (const T*)c->d, cells, ncells, ncells_dev, E, offset, c->part_e,
            c->band[0], c->band[1], tile_cnt, c->ds, check_stop);
    c->launches += 1;
    return cudaGetLastError();
}

static cudaError_t energy_dispatch(slr_ctx* c, int offset, double p, int p_kind, int check_stop) {
    const bool f32 = c->cfg.precision == 32;
    const int dim = c->cfg.dim, ip = c->cfg.interp;
    if (f32) {
        if (dim == 2) return ip ? energy_t<float, 2, 1>(c, offset, p, p_kind, check_stop)
                                : energy_t<float, 2, 0>(c, offset, p, p_kind, check_stop);
        return ip ? energy_t<float, 3, 1>(c, offset, p, p_kind, check_stop)
                  : energy_t<float, 3, 0>(c, offset, p, p_kind, check_stop);
    }
    if (dim == 2) return ip ? energy_t<double, 2, 1>(c, offset, p, p_kind, check_stop)
                            : energy_t<double, 2, 0>(c, offset, p, p_kind, check_stop);
    return ip ? energy_t<double, 3, 1>(c, offset, p, p_kind, check_stop)
              : energy_t<double, 3, 0>(c, offset, p, p_kind, check_stop);
}

// the record kernel's arguments for one job (record_mode: 0 init, 1 step,
// 2 report)
RecordArgs record_args(slr_ctx* c, int record_mode, int evolve_mode, double p, int p_kind) {
    RecordArgs A;
    const bool bricked = brick_mode(c);
    A.part_dphi = bricked ? c->brick.part : (c->cfg.reinit ? c->part_dphi_r : c->part_dphi);
    A.bricked = bricked;
    A.part_e = c->part_e;
    A.nchunks = energy_slots(c);
    A.ncells_dev = c->cfg.reinit ? &c->ds->n_ecells_dyn : nullptr;
    A.n_dphi_full = bricked ? c->brick.ntotal : (c->cfg.reinit ? reinit_grid(c) : full_step_blocks(c));
    A.N = c->N;
    A.full_grid = !c->cfg.band;
    A.reinit = c->cfg.reinit;
    A.mode = record_mode;
    A.evolve = evolve_mode;
    A.h_dim = c->cfg.dim == 3 ? c->h * c->h * c->h : c->h * c->h;
    A.p = p;
    A.p_kind = p_kind;
    A.stop_tol = c->cfg.stop_tol;
    A.stop_k = c->cfg.stop_k;
    A.min_iters = c->cfg.min_iters;
    A.max_iters = c->cfg.max_iters;
    A.tile_off = (c->cfg.band && !bricked) ? c->tile_off : nullptr;
    A.offset = record_mode == 1 ? 1 : 0;
    A.report = c->part_e + 2 * c->n_echunks;          // two spare doubles after the partials
    A.block_part = c->part_e + 2 * c->n_echunks + 2;  // then three per record block
    return A;
}

// record_mode: 0 init, 1 step, 2 report (p_override used, result in ds report slot)
cudaError_t launch_energy(slr_ctx* c, int offset, double p_override, int record_mode, int evolve_mode,
                          cudaEvent_t between) {
    double p = record_mode == 2 ? p_override : c->cfg.p;
    int p_kind = p == 1.0 ? 1 : (p == 2.0 ? 2 : 0);
    cudaError_t e = energy_dispatch(c, offset, p, p_kind, record_mode == 1);
    if (e != cudaSuccess) return e;
    if (between) {
        e = cudaEventRecordWithFlags(between, c->stream, cudaEventRecordExternal);
        if (e != cudaSuccess) return e;
    }
    const RecordArgs A = record_args(c, record_mode, evolve_mode, p, p_kind);
    k_record<<<kRecordBlocks, kRecordThreads, 0, c->stream>>>(A, c->ds);
    c->launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// extract (ordered) and Err_S
// ---------------------------------------------------------------------------
}  // namespace slr

#include "slr_compact.cuh"

namespace slr {

template <typename T>
struct WidthPred {
    const T* u;
    double w;
    __device__ bool operator()(long long i) const { return fabs((double)u[i]) < w; }
};

template <typename T>
struct EmitExtract {
    const T* u;
    long long* idx;
    double* val;
    __device__ void operator()(long long pos, long long i) const {
        if (idx) idx[pos] = i;
        if (val) val[pos] = (double)u[i];
    }
};

template <typename T>
static cudaError_t extract_t(slr_ctx* c, double width, long long* idx, double* val, long long* count, bool write) {
    int cur = 0;
    cudaError_t e = cudaMemcpyAsync(&cur, &c->ds->n, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return e;
    const T* u = (const T*)c->u[cur & 1];
    WidthPred<T> pr{u, width};
    if (!write) return compact_count(c, pr, c->N, count);
    return compact_write(c, pr, EmitExtract<T>{u, idx, val}, c->N);
}

cudaError_t launch_extract(slr_ctx* c, double width, long long* idx_dev, double* u_dev, long long* count_out,
                           bool write) {
    return c->cfg.precision == 32 ? extract_t<float>(c, width, idx_dev, u_dev, count_out, write)
                                  : extract_t<double>(c, width, idx_dev, u_dev, count_out, write);
}

// §4 eq. errCloud: mean over the cloud of |I[φ](Q)|, active interpolator
template <typename T, int DIM, int INTERP>
__global__ void k_err_cloud(Params<T> P, const T* ub0, const T* ub1, const double* pts, long long npts, double lo0,
                            double lo1, double lo2, double inv_h, double* part, DevState* ds) {
    __shared__ double s_red[8];
    const T* u = (ds->n & 1) ? ub1 : ub0;
    double acc = 0.0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < npts; q += (long long)gridDim.x * blockDim.x) {
        // index-space coordinate relative to node (0,0,0)
        T r[3];
        r[0] = (T)((pts[q * DIM + 0] - lo0) * inv_h);
        r[1] = (T)((pts[q * DIM + 1] - lo1) * inv_h);
        r[2] = DIM == 3 ? (T)((pts[q * DIM + 2] - lo2) * inv_h) : T(0);
        T v = interp_at<T, DIM, INTERP>(P, u, 0, 0, 0, r);
        acc += fabs((double)v);
    }
    double s = block_sum<256>(acc, s_red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_sum_parts(const double* part, int n, double scale, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s * scale;
    }
}

template <typename T, int DIM, int INTERP>
static cudaError_t err_t(slr_ctx* c, double* out) {
    Params<T> P = make_params<T>(c);
    int blocks = (int)((c->npts + 255) / 256);
    if (blocks > c->num_sms * 4) blocks = c->num_sms * 4;
    if (blocks < 1) blocks = 1;
    double* part = (double*)dev_alloc(c, sizeof(double) * blocks);
    if (!part) return cudaErrorMemoryAllocation;
    k_err_cloud<T, DIM, INTERP><<<blocks, 256, 0, c->stream>>>(P, (const T*)c->u[0], (const T*)c->u[1], c->pts,
                                                               c->npts, c->cfg.lo[0], c->cfg.lo[1], c->cfg.lo[2],
                                                               1.0 / c->h, part, c->ds);
    k_sum_parts<<<1, 32, 0, c->stream>>>(part, blocks, 1.0 / (double)c->npts, out);
    c->launches += 2;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, part);
    return e;
}

cudaError_t launch_err_cloud(slr_ctx* c, double* out) {
    const bool f32 = c->cfg.precision == 32;
    const int dim = c->cfg.dim, ip = c->cfg.interp;
    if (f32) {
        if (dim == 2) return ip ? err_t<float, 2, 1>(c, out) : err_t<float, 2, 0>(c, out);
        return ip ? err_t<float, 3, 1>(c, out) : err_t<float, 3, 0>(c, out);
    }
    if (dim == 2) return ip ? err_t<double, 2, 1>(c, out) : err_t<double, 2, 0>(c, out);
    return ip ? err_t<double, 3, 1>(c, out) : err_t<double, 3, 0>(c, out);
}

}  // namespace slr
