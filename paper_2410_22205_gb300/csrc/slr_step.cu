// Per-iteration kernels of Algorithm 1 (arXiv 2410.22205, §3): the fused
// narrow-band rebuild + semi-Lagrangian update + cut, the whole-grid SL
// update, and the initial-data kernels.
//
// Fused band step (one launch per iteration, persistent grid):
//   input  L^{n-1}  (sorted node list, scan domain) and u^n;
//   for every entry j: j is in the band G̃^n iff |u^n_j| < γ (eq. subgrid,
//   decided in the storage precision); band nodes get the SL update of §3.1
//   followed by the cut of eq. cut, the others are copied unchanged into
//   u^{n+1} (they sit at ±γ since the initial cut); G̃^n is written as a
//   sorted list at offsets prepared before the step (per-tile member counts
//   from the energy kernel, their prefix from the record kernel); per-tile
//   FP64 partial sums of |u^{n+1} - u^n| feed Δ_φ.
// Without reinitialisation a node outside the band keeps |u| = γ and can
// never re-enter, so G̃^n ⊆ G̃^{n-1} and scanning L^{n-1} finds the whole band.
#include "slr_compact.cuh"
#include "slr_internal.cuh"
#include "slr_step.cuh"

namespace slr {

// fused band rebuild + SL update + cut (band mode). Work is handed out per
// warp: a ticket is a tile of kStepTile consecutive entries of L^{n-1} (four
// per lane). The count of band members of every tile and their prefix were
// computed after the previous step (front-cell kernel and record kernel), so
// a tile knows its output offset at once: it ballots band membership, writes
// its part of G̃^n, and runs the SL arithmetic. No warp waits on another.
template <typename T, int DIM, int INTERP>
__global__ void __launch_bounds__(kStepBlock, (INTERP == 1 ? (sizeof(T) == 8 ? 2 : 3) : (sizeof(T) == 8 ? 3 : 8))) k_step_band(Params<T> P, T* ub0, T* ub1, const T* __restrict__ d,
                                                          int* L0, int* L1, const int* __restrict__ tile_off,
                                                          int band_cap, double* part_dphi, DevState* ds,
                                                          double ep_override) {
    if (ds->stop) return;
    const int lane = threadIdx.x & 31;
    const int n = ds->n;
    const int cnt_in = ds->band_count[n & 1];
    const T* __restrict__ uin = (n & 1) ? ub1 : ub0;
    T* __restrict__ uout = (n & 1) ? ub0 : ub1;
    const int* __restrict__ Lin = (n & 1) ? L1 : L0;
    int* __restrict__ Lout = (n & 1) ? L0 : L1;
    const T Ep = ep_override >= 0.0 ? (T)ep_override : (T)ds->Ep;
    const int ntiles = (cnt_in + kStepTile - 1) / kStepTile;
    if (blockIdx.x == 0 && threadIdx.x == 0) ds->band_count[(n + 1) & 1] = ntiles ? ds->band_next : 0;
    if (ntiles == 0) return;
    const int per = (ntiles + kRecordBlocks - 1) / kRecordBlocks;  // tiles per record-block slice
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(&ds->ticket, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        band_tile<T, DIM, INTERP>(P, uin, uout, d, Lin, Lout, tile_off, ds->band_base, band_cap, cnt_in, per, t, Ep,
                                  part_dphi, ds);
    }
}

// whole-grid SL update (band off: c ≡ 1, no cut), static tiles
template <typename T, int DIM, int INTERP>
__global__ void __launch_bounds__(kStepBlock, (INTERP == 1 ? (sizeof(T) == 8 ? 2 : 3) : (sizeof(T) == 8 ? 3 : 4))) k_step_full(Params<T> P, T* ub0, T* ub1, const T* __restrict__ d,
                                                          long long N, double* part_dphi, DevState* ds,
                                                          double ep_override) {
    __shared__ double s_red[kStepBlock / 32];
    if (ds->stop) return;
    const int n = ds->n;
    const T* __restrict__ uin = (n & 1) ? ub1 : ub0;  // whole-grid tiles: 256 consecutive nodes
    T* __restrict__ uout = (n & 1) ? ub0 : ub1;
    const T Ep = ep_override >= 0.0 ? (T)ep_override : (T)ds->Ep;
    const long long ntiles = (N + kStepBlock - 1) / kStepBlock;
    double acc = 0.0;  // lane 0 of each warp: sum of the warp's per-tile sums
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long idx = t * kStepBlock + threadIdx.x;
        T dabs = T(0);
        if (idx < N) {
            int i, j, k;
            decode(P, idx, i, j, k);
            const T v = uin[idx];
            const T out = sl_update<T, DIM, INTERP>(P, uin, d, Ep, i, j, k, idx, v);
            uout[idx] = out;
            dabs = fabs(out - v);
        }
        acc += (double)warp_sum(dabs);
    }
    const double bs = block_sum<kStepBlock>(acc, s_red, true);
    if (threadIdx.x == 0) part_dphi[blockIdx.x] = bs;
}

// ---------------------------------------------------------------------------
// initial data
// ---------------------------------------------------------------------------

// φ^0 = |x - c| - r in FP64 without contraction (x = lo + i*h), rounded to
// the storage type, then cut to [-γ, γ] in band mode; written to both buffers
template <typename T>
__global__ void k_init_sphere(Params<T> P, T* ub0, T* ub1, long long N, double lo0, double lo1, double lo2, double h,
                              double cx, double cy, double cz, double r, int dim, int band) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N) return;
    int i, j, k;
    decode(P, idx, i, j, k);
    double x = __dadd_rn(lo0, __dmul_rn((double)i, h));
    double y = __dadd_rn(lo1, __dmul_rn((double)j, h));
    double dx = __dsub_rn(x, cx), dy = __dsub_rn(y, cy);
    double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    if (dim == 3) {
        double z = __dadd_rn(lo2, __dmul_rn((double)k, h));
        double dz = __dsub_rn(z, cz);
        s = __dadd_rn(s, __dmul_rn(dz, dz));
    }
    T v = (T)__dsub_rn(__dsqrt_rn(s), r);
    if (band) v = fmin(fmax(v, -P.gamma), P.gamma);
    ub0[idx] = v;
    ub1[idx] = v;
}

template <typename T>
__global__ void k_init_array(Params<T> P, T* ub0, T* ub1, const double* src, long long N, int band) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N) return;
    T v = (T)src[idx];
    if (band) v = fmin(fmax(v, -P.gamma), P.gamma);
    ub0[idx] = v;
    ub1[idx] = v;
}

// predicates and emitters of the init compactions
template <typename T>
struct BandPred {
    const T* u;
    T gamma;
    __device__ bool operator()(long long i) const { return fabs(u[i]) < gamma; }
};

struct EmitInt {
    int* out;
    __device__ void operator()(long long pos, long long i) const { out[pos] = (int)i; }
};

// candidate cells of the energy quadrature: cells with a vertex in the
// initial band, or with a sign change at init. Only band nodes ever change,
// so no other cell can become a front cell later.
template <typename T, int DIM>
struct CellPred {
    const T* u;
    T gamma;
    int n0, n1, n2;
    long long s1, s2;
    __device__ bool operator()(long long c) const {
        int cn0 = n0 - 1, cn1 = n1 - 1;
        long long q = c / cn0;
        int i = (int)(c - q * cn0);
        int j = (int)(q % cn1);
        int k = (int)(q / cn1);
        long long base = i + s1 * j + s2 * k;
        bool neg = false, pos = false, inb = false;
#pragma unroll
        for (int dz = 0; dz < (DIM == 3 ? 2 : 1); ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    T v = u[base + dx + s1 * dy + s2 * dz];
                    if (v < T(0))
                        neg = true;
                    else
                        pos = true;
                    if (fabs(v) < gamma) inb = true;
                }
        return inb || (neg && pos);
    }
};

template <typename T, int DIM>
struct EmitCell {
    int* out;
    int n0, n1;
    long long s1, s2;
    __device__ void operator()(long long pos, long long c) const {
        int cn0 = n0 - 1, cn1 = n1 - 1;
        long long q = c / cn0;
        int i = (int)(c - q * cn0);
        int j = (int)(q % cn1);
        int k = (int)(q / cn1);
        out[pos] = (int)(i + s1 * j + s2 * k);
    }
};

// ---------------------------------------------------------------------------
// host wrappers
// ---------------------------------------------------------------------------
template <typename T>
Params<T> make_params(const slr_ctx* c) {
    Params<T> P;
    P.n0 = (int)c->cfg.n[0];
    P.n1 = (int)c->cfg.n[1];
    P.n2 = (int)c->cfg.n[2];
    P.s1 = c->cfg.n[0];
    P.s2 = c->cfg.n[0] * c->cfg.n[1];
    P.is1 = (int)P.s1;
    P.is2 = (int)P.s2;
    P.h = (T)c->h;
    P.inv_h = (T)(1.0 / c->h);
    P.inv_2h = (T)(1.0 / (2.0 * c->h));
    P.h4 = (T)(c->h * c->h * c->h * c->h);
    P.dt = (T)c->dt;
    P.delta = (T)c->cfg.delta;
    P.p = (T)c->cfg.p;
    P.inv_p = (T)(1.0 / c->cfg.p);
    P.gamma = (T)c->gamma;
    P.beta = (T)c->beta;
    double gb = c->gamma - c->beta;
    P.inv_gb3 = (T)(1.0 / (gb * gb * gb));
    P.sing_thr = (T)(c->cfg.c_sing * pow(c->dt, c->cfg.alpha));
    P.band = c->cfg.band;
    P.p_kind = c->cfg.p == 1.0 ? 1 : (c->cfg.p == 2.0 ? 2 : 0);
    return P;
}
template Params<float> make_params<float>(const slr_ctx*);
template Params<double> make_params<double>(const slr_ctx*);

static int grid_blocks(const slr_ctx* c, int per_sm) { return c->num_sms * per_sm; }

// fixed grid of the whole-grid step (one Δ_φ partial per block)
long long full_step_blocks(const slr_ctx* c) {
    long long ntiles = (c->N + kStepBlock - 1) / kStepBlock;
    long long nb = (long long)c->num_sms * 8;
    return nb < ntiles ? nb : ntiles;
}

template <typename T, int DIM, int INTERP>
static cudaError_t step_t(slr_ctx* c, double ov) {
    Params<T> P = make_params<T>(c);
    T* u0 = (T*)c->u[0];
    T* u1 = (T*)c->u[1];
    if (c->cfg.band) {
        // enough blocks for one round of tickets over the largest band (it only shrinks)
        long long per_block = (long long)kStepTile * (kStepBlock / 32);
        long long nb = (c->band_cap + per_block - 1) / per_block;
        if (nb > grid_blocks(c, 8)) nb = grid_blocks(c, 8);
        if (nb < 1) nb = 1;
        k_step_band<T, DIM, INTERP><<<(int)nb, kStepBlock, 0, c->stream>>>(
            P, u0, u1, (const T*)c->d, c->band[0], c->band[1], c->tile_off, (int)c->band_cap, c->part_dphi, c->ds,
            ov);
    } else {
        long long nb = full_step_blocks(c);
        k_step_full<T, DIM, INTERP><<<(int)nb, kStepBlock, 0, c->stream>>>(P, u0, u1, (const T*)c->d, c->N,
                                                                          c->part_dphi, c->ds, ov);
    }
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_step(slr_ctx* c, double ov, int /*evolve_mode*/) {
    if (brick_mode(c)) return launch_step_brick(c, ov);
    const bool f32 = c->cfg.precision == 32;
    const int dim = c->cfg.dim, ip = c->cfg.interp;
    if (f32) {
        if (dim == 2) return ip ? step_t<float, 2, 1>(c, ov) : step_t<float, 2, 0>(c, ov);
        return ip ? step_t<float, 3, 1>(c, ov) : step_t<float, 3, 0>(c, ov);
    }
    if (dim == 2) return ip ? step_t<double, 2, 1>(c, ov) : step_t<double, 2, 0>(c, ov);
    return ip ? step_t<double, 3, 1>(c, ov) : step_t<double, 3, 0>(c, ov);
}

template <typename T>
static cudaError_t init_t(slr_ctx* c, int kind, const double* prm, const double* u0_dev) {
    Params<T> P = make_params<T>(c);
    int blocks = (int)((c->N + 255) / 256);
    if (kind == 0) {
        k_init_sphere<T><<<blocks, 256, 0, c->stream>>>(P, (T*)c->u[0], (T*)c->u[1], c->N, c->cfg.lo[0], c->cfg.lo[1],
                                                        c->cfg.lo[2], c->h, prm[0], prm[1], prm[2], prm[3],
                                                        c->cfg.dim, c->cfg.band);
    } else {
        k_init_array<T><<<blocks, 256, 0, c->stream>>>(P, (T*)c->u[0], (T*)c->u[1], u0_dev, c->N, c->cfg.band);
    }
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_init_u(slr_ctx* c, int kind, const double* params, const double* u0_dev) {
    return c->cfg.precision == 32 ? init_t<float>(c, kind, params, u0_dev) : init_t<double>(c, kind, params, u0_dev);
}

template <typename T>
static cudaError_t band_t(slr_ctx* c, long long* count, bool write) {
    BandPred<T> pr{(const T*)c->u[0], (T)c->gamma};
    if (!write) return compact_count(c, pr, c->N, count);
    return compact_write(c, pr, EmitInt{c->band[0]}, c->N);
}

cudaError_t launch_count_band(slr_ctx* c, long long* count_out) {
    return c->cfg.precision == 32 ? band_t<float>(c, count_out, false) : band_t<double>(c, count_out, false);
}

cudaError_t launch_build_band(slr_ctx* c) {
    long long dummy = 0;
    return c->cfg.precision == 32 ? band_t<float>(c, &dummy, true) : band_t<double>(c, &dummy, true);
}

template <typename T, int DIM>
static cudaError_t ecells_t(slr_ctx* c, long long* count, bool write) {
    CellPred<T, DIM> pr{(const T*)c->u[0], (T)c->gamma, (int)c->cfg.n[0], (int)c->cfg.n[1], (int)c->cfg.n[2],
                        c->cfg.n[0], c->cfg.n[0] * c->cfg.n[1]};
    if (!write) return compact_count(c, pr, c->ncells_all, count);
    EmitCell<T, DIM> em{c->ecells, (int)c->cfg.n[0], (int)c->cfg.n[1], c->cfg.n[0], c->cfg.n[0] * c->cfg.n[1]};
    return compact_write(c, pr, em, c->ncells_all);
}

cudaError_t launch_build_ecells(slr_ctx* c, long long* count_out, bool write) {
    if (c->cfg.precision == 32)
        return c->cfg.dim == 2 ? ecells_t<float, 2>(c, count_out, write) : ecells_t<float, 3>(c, count_out, write);
    return c->cfg.dim == 2 ? ecells_t<double, 2>(c, count_out, write) : ecells_t<double, 3>(c, count_out, write);
}

}  // namespace slr
