// Device code of the energy functional and the per-iteration bookkeeping
// (arXiv 2410.22205, §3.5 eqs. energyApprox and energyApproxFiner, §4 eq.
// deltaEn): the front cells of a slot of candidate cells and their
// quadrature, the band-member count of one tile of the band list, and one
// slice of the record reduction with the stop test. Shared by the per-job
// kernels (slr_energy.cu) and the batched persistent kernel (slr_batch.cuh);
// both translation units are compiled without implicit FMA contraction, so
// a slot or slice computes the same bits in either. The reductions keep the
// summation tree of kEnergyThreads (kRecordThreads) threads whatever the
// block size NT: a block of fewer threads runs the missing threads' shares
// as extra rounds, in the same order.
#pragma once

#include "slr_internal.cuh"

namespace slr {

__device__ __forceinline__ double pow_abs(double v, double p, int p_kind) {
    double a = fabs(v);
    if (p_kind == 2) return a * a;
    if (p_kind == 1) return a;
    return pow(a, p);
}

template <typename T, int DIM>
__device__ __forceinline__ void cell_of(const Params<T>& P, const int* cells, long long e, int& i, int& j, int& k) {
    if (cells) {
        long long node = cells[e];
        long long q = node / P.n0;
        i = (int)(node - q * P.n0);
        k = (int)(q / P.n1);
        j = (int)(q - (long long)k * P.n1);
    } else {
        int cn0 = P.n0 - 1, cn1 = P.n1 - 1;
        long long q = e / cn0;
        i = (int)(e - q * cn0);
        j = (int)(q % cn1);
        k = (int)(q / cn1);
    }
}

// 2-D front cell of eq. energyApprox, evaluated in FP64 from the stored values
template <typename T>
__device__ double energy_cell_2d(const Params<T>& P, const T* __restrict__ u, const T* __restrict__ d, int i, int j,
                                 double h, double p, int p_kind, double* acc2) {
    long long b = i + P.s1 * j;
    long long id[4] = {b, b + 1, b + 1 + P.s1, b + P.s1};  // corners 00, 10, 11, 01
    const double cx[4] = {0, 1, 1, 0}, cy[4] = {0, 0, 1, 1};
    double uv[4], dv[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        uv[c] = (double)ld(u + id[c]);
        dv[c] = (double)ld(d + id[c]);
    }
    double px[4], py[4], pd[4];
    int has[4], nc = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        int a = e, bb = (e + 1) & 3;
        has[e] = (uv[a] < 0.0) != (uv[bb] < 0.0);
        if (has[e]) {
            double t = uv[a] / (uv[a] - uv[bb]);
            px[e] = (cx[a] + t * (cx[bb] - cx[a])) * h;
            py[e] = (cy[a] + t * (cy[bb] - cy[a])) * h;
            pd[e] = dv[a] + t * (dv[bb] - dv[a]);
            ++nc;
        } else {
            px[e] = py[e] = pd[e] = 0.0;
        }
    }
    int pr[2][2], np;
    if (nc == 2) {
        int kk = 0;
        for (int e = 0; e < 4; ++e)
            if (has[e]) pr[0][kk++] = e;
        np = 1;
    } else if (nc == 4) {
        double mean = (uv[0] + uv[1] + uv[2] + uv[3]) / 4.0;
        if ((mean < 0.0) == (uv[0] < 0.0)) {
            pr[0][0] = 0; pr[0][1] = 1; pr[1][0] = 2; pr[1][1] = 3;
        } else {
            pr[0][0] = 3; pr[0][1] = 0; pr[1][0] = 1; pr[1][1] = 2;
        }
        np = 2;
    } else {
        return 0.0;
    }
    double s = 0.0, s2 = 0.0;
    for (int q = 0; q < np; ++q) {
        int e1 = pr[q][0], e2 = pr[q][1];
        double dx = px[e1] - px[e2], dy = py[e1] - py[e2];
        double len = sqrt(dx * dx + dy * dy);
        s += len * (pow_abs(pd[e1], p, p_kind) + pow_abs(pd[e2], p, p_kind)) / 2.0;
        s2 += len * (pd[e1] * pd[e1] + pd[e2] * pd[e2]) / 2.0;
    }
    *acc2 += s2;
    return s;
}

// Data-only part of one WENO evaluation (the squared second differences and
// their h^4-shifted squares); evaluations of the same four values at several
// θ share it.
template <typename T>
struct WenoInd {
    T v1, dv, dr, ddf, sl2, sr2;
    __device__ __forceinline__ void set(T v0, T a1, T v2, T v3, T h4) {
        v1 = a1;
        dv = v2 - a1;
        const T dl = fma(T(-2), a1, v0 + v2);
        dr = fma(T(-2), v2, a1 + v3);
        const T sl = fma(dl, dl, h4), sr = fma(dr, dr, h4);
        sl2 = sl * sl;
        sr2 = sr * sr;
        ddf = dl - dr;
    }
    // weno1() at this θ (the weight's denominator rounded once more)
    __device__ __forceinline__ T eval(const WenoAxis<T>& w) const {
        const T gl = w.rho * sr2;
        const T wl = fast_div(gl, sl2 + gl);
        return fma(w.q, fma(wl, ddf, dr), fma(w.th, dv, v1));
    }
};

constexpr int kEnergyThreads = 256;

template <typename T, int DIM>
__device__ __forceinline__ bool is_front(const Params<T>& P, const T* __restrict__ u, int node) {
    bool neg = false, pos = false;
#pragma unroll
    for (int dz = 0; dz < (DIM == 3 ? 2 : 1); ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                T v = ld(u + (node + dx + P.is1 * dy + P.is2 * dz));
                if (v < T(0))
                    neg = true;
                else
                    pos = true;
            }
    return neg && pos;
}

// Energy pass, one launch (k_energy). Blocks take slots of kEnergyCand
// candidate cells from a ticket; for slot b a block first collects, in
// candidate order and in shared memory, the front cells among candidates
// [b·kEnergyCand, (b+1)·kEnergyCand) (sign change, zero counted as
// positive), then processes them:
//   3-D: one thread per (front cell, subcell layer c along z): the 16 z-lines
//        of the 4x4x4 stencil at θ_z(c), the 4 y-lines at the R θ_y, the R
//        x-lines at the R θ_x (WENO; the data-only part of each y- and x-line
//        indicator is computed once and reused for its R points), or the
//        trilinear interpolant (Q1); d by Q1, linear along each x-line. A
//        subcell counts when |φ(x')| < (√3/2)Δx' and adds |d(x')|^p Δx'^2.
//   2-D: one thread per front cell (segments, FP64).
//        In band mode its warps first count, per tile of kStepTile entries of
//        the band list the next step reads, the members |φ| < γ (the step
//        kernel's own test); the record kernel turns the counts into offsets.
// No ordering across blocks is needed, and the block scheduler evens out the
// uneven slot sizes. 3-D sums per work item, per thread and per warp in the
// storage type, then per block in FP64 (2-D: FP64 throughout), in a fixed
// order (one partial pair per block).
constexpr int kEnergyCand = 1024;  // candidate cells per slot (4 per thread)

// The front cells of slot sb: the candidate cells [sb·kEnergyCand,
// (sb+1)·kEnergyCand) with vertices of both signs (zero counted as
// positive), in candidate order, into out[] (block-wide: all NT threads of
// the block call it; thread t checks the kEnergyCand/NT consecutive
// candidates from sb·kEnergyCand + t·kEnergyCand/NT). Returns their count.
template <typename T, int DIM, int NT>
__device__ __forceinline__ int front_of_slot(const Params<T>& P, const T* __restrict__ u, const int* __restrict__ cells,
                                             long long ncells, long long sb, int* out, int* s_warp) {
    constexpr int W = NT / 32;
    constexpr int PER = kEnergyCand / NT;
    static_assert(PER % 4 == 0, "whole 16-byte loads of the cell list per thread");
    const long long e0 = sb * kEnergyCand + PER * threadIdx.x;
    int node[PER];
    if (cells && e0 + PER <= ncells) {
#pragma unroll
        for (int v = 0; v < PER / 4; ++v) {
            const int4 c4 = *reinterpret_cast<const int4*>(cells + e0 + 4 * v);  // slot starts are multiples of 1024
            node[4 * v + 0] = c4.x;
            node[4 * v + 1] = c4.y;
            node[4 * v + 2] = c4.z;
            node[4 * v + 3] = c4.w;
        }
    } else {
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            node[r] = 0;
            if (e0 + r < ncells) {
                int i, j, k;
                cell_of<T, DIM>(P, cells, e0 + r, i, j, k);
                node[r] = i + P.is1 * j + P.is2 * k;
            }
        }
    }
    bool fl[PER];
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        fl[r] = e0 + r < ncells && is_front<T, DIM>(P, u, node[r]);
        cnt += fl[r];
    }
    // block exclusive scan of the per-thread counts (candidate order kept)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < W; ++w) {
            const int c = s_warp[w];
            s_warp[w] = run;
            run += c;
        }
        s_warp[W] = run;
    }
    __syncthreads();
    int off = s_warp[warp] + incl - cnt;
#pragma unroll
    for (int r = 0; r < PER; ++r)
        if (fl[r]) out[off++] = node[r];
    const int nf = s_warp[W];
    __syncthreads();
    return nf;
}

// Shared-memory workspace of the energy pass (one slot at a time)
template <typename T>
struct EnergyWs {
    T th[kMaxR];                        // θ_m of the subcell centres (general R)
    WenoAxis<T> wa[kMaxR];              // WENO constants at θ_m (general R)
    double a[kEnergyThreads / 32];      // per-warp partial sums
    double b[kEnergyThreads / 32];
    int front[kEnergyCand];             // this slot's front cells
    int warp[kEnergyThreads / 32 + 1];  // scan of the front-cell counts
};

// Per-launch set-up of the subcell centres for a run-time R (RC = 0)
template <typename T, int RC>
__device__ __forceinline__ void energy_setup(EnergyWs<T>& ws, int R) {
    if (RC == 0 && threadIdx.x < R) {
        T t = ((T)threadIdx.x + (T)0.5) / (T)R;  // subcell centre θ_m = (m + 1/2)/R
        ws.th[threadIdx.x] = t;
        ws.wa[threadIdx.x].set_exact(t);
    }
}

// Scalars of the quadrature (computed on the host): thr = (√3/2)Δx',
// hp2 = Δx'^2, pT = p in the storage type; p, p_kind, h for the 2-D FP64 path
template <typename T>
struct EnergyArgs {
    int R;
    double h, p;
    int p_kind;
    T thr, hp2, pT;
};

// Slot sb of the candidate cells: its front cells (front_of_slot), then the
// quadrature of eq. energyApprox (2-D) or energyApproxFiner (3-D), into the
// partial pair part[2 sb], part[2 sb + 1] (sum of |d|^p and of d^2 terms).
// All NT threads of the block call it; the sums follow the tree of
// kEnergyThreads threads (item it to thread it mod kEnergyThreads, thread
// sums in the storage type (3-D) or FP64 (2-D), warp sums, the warps' sums
// in order).
template <typename T, int DIM, int INTERP, int RC, int NT>
__device__ __forceinline__ void energy_slot(const Params<T>& P, const T* __restrict__ u, const T* __restrict__ d,
                                            const int* __restrict__ cells, long long ncells, long long sb,
                                            const EnergyArgs<T>& E, double* part, EnergyWs<T>& ws) {
    static_assert(kEnergyThreads % NT == 0, "the block size divides kEnergyThreads");
    constexpr int V = kEnergyThreads / NT;  // rounds of the kEnergyThreads-thread tree per thread
    constexpr int VW = kEnergyThreads / 32;
    const int R = RC > 0 ? RC : E.R;
    constexpr double RD = RC > 0 ? (double)RC : 1.0;
    const T thr = E.thr, hp2 = E.hp2, pT = E.pT;
    const int p_kind = E.p_kind;
    const int nf = front_of_slot<T, DIM, NT>(P, u, cells, ncells, sb, ws.front, ws.warp);
    const int* s_list = ws.front;
    // subcell centre θ_m = (m + 1/2)/R (folded at compile time for RC > 0)
    auto TH = [&](int m) -> T { return RC > 0 ? (T)m * (T)(1.0 / RD) + (T)(0.5 / RD) : ws.th[m]; };
    // WENO constants at θ_m (storage-type arithmetic; folded at compile
    // time where m is a constant)
    auto WA = [&](int m) -> WenoAxis<T> {
        if (RC > 0) {
            WenoAxis<T> w;
            w.set_exact(TH(m));
            return w;
        }
        return ws.wa[m];
    };
    auto contrib = [&](T uu, T dd, T& cp, T& c2) {
        const T a = fabs(dd);
        const T d2 = a * a;
        const T keep = fabs(uu) < thr ? hp2 : T(0);
        cp = fma(p_kind == 2 ? d2 : (p_kind == 1 ? a : (T)pow(a, pT)), keep, cp);
        c2 = fma(d2, keep, c2);
    };
    const int lane = threadIdx.x & 31;
#pragma unroll 1
    for (int r = 0; r < V; ++r) {
        const int vt = threadIdx.x + r * NT;  // thread of the kEnergyThreads tree
        double ap = 0.0, a2 = 0.0;
        if (DIM == 2) {
            for (int fi = vt; fi < nf; fi += kEnergyThreads) {
                const int nd = s_list[fi];
                const int q = nd / P.n0;
                double s2 = 0.0;
                ap += energy_cell_2d<T>(P, u, d, nd - q * P.n0, q, E.h, E.p, p_kind, &s2);
                a2 += s2;
            }
            ap = warp_sum(ap);
            a2 = warp_sum(a2);
        } else {
            // sums over this thread's items in the storage type, widened once
            T tp = T(0), t2 = T(0);
            const int items = nf * R;
            for (int it = vt; it < items; it += kEnergyThreads) {
                const int fi = it / R, cz = it - fi * R;
                const int nd = s_list[fi];
                const int q = nd / P.n0;
                const int i = nd - q * P.n0;
                const int k = q / P.n1;
                const int j = q - k * P.n1;
                const T tz = TH(cz);
                T dc[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) dc[c] = ld(d + (nd + (c & 1) + P.is1 * ((c >> 1) & 1) + P.is2 * (c >> 2)));
                // d on the layer z = θ_z: bilinear in (x, y) from the two z-faces
                T dz[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) dz[c] = fma(tz, dc[c + 4] - dc[c], dc[c]);
                T cp = T(0), c2 = T(0);
                if (INTERP == 1) {
                    const WenoAxis<T> wz = WA(cz);
                    int ox[4], oy[4], oz[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        ox[a] = clampi(i - 1 + a, 0, P.n0 - 1);
                        oy[a] = P.is1 * clampi(j - 1 + a, 0, P.n1 - 1);
                        oz[a] = P.is2 * clampi(k - 1 + a, 0, P.n2 - 1);
                    }
                    WenoInd<T> iy[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        T zl[4];
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const T* col = u + (ox[a] + oy[b]);
                            zl[b] = weno1(ld(col + oz[0]), ld(col + oz[1]), ld(col + oz[2]), ld(col + oz[3]), wz, P.h4);
                        }
                        iy[a].set(zl[0], zl[1], zl[2], zl[3], P.h4);
                    }
#pragma unroll
                    for (int by = 0; by < (RC > 0 ? RC : kMaxR); ++by) {
                        if (RC == 0 && by >= R) break;
                        const WenoAxis<T> wy = WA(by);
                        const T ty = TH(by);
                        WenoInd<T> ix;
                        ix.set(iy[0].eval(wy), iy[1].eval(wy), iy[2].eval(wy), iy[3].eval(wy), P.h4);
                        const T d0 = fma(ty, dz[2] - dz[0], dz[0]), d1 = fma(ty, dz[3] - dz[1], dz[1]);
#pragma unroll
                        for (int ax = 0; ax < (RC > 0 ? RC : kMaxR); ++ax) {
                            if (RC == 0 && ax >= R) break;
                            const T tx = TH(ax);
                            contrib(ix.eval(WA(ax)), fma(tx, d1 - d0, d0), cp, c2);
                        }
                    }
                } else {
                    T uc[8];
#pragma unroll
                    for (int c = 0; c < 8; ++c) uc[c] = ld(u + (nd + (c & 1) + P.is1 * ((c >> 1) & 1) + P.is2 * (c >> 2)));
                    T uz[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) uz[c] = fma(tz, uc[c + 4] - uc[c], uc[c]);
                    for (int by = 0; by < R; ++by) {
                        const T ty = TH(by);
                        const T u0 = fma(ty, uz[2] - uz[0], uz[0]), u1 = fma(ty, uz[3] - uz[1], uz[1]);
                        const T d0 = fma(ty, dz[2] - dz[0], dz[0]), d1 = fma(ty, dz[3] - dz[1], dz[1]);
                        for (int ax = 0; ax < R; ++ax) {
                            const T tx = TH(ax);
                            contrib(fma(tx, u1 - u0, u0), fma(tx, d1 - d0, d0), cp, c2);
                        }
                    }
                }
                tp += cp;
                t2 += c2;
            }
            // warp sums in the storage type, per-warp sums widened
            tp = warp_sum(tp);
            t2 = warp_sum(t2);
            ap = (double)tp;
            a2 = (double)t2;
        }
        if (lane == 0) {
            ws.a[vt >> 5] = ap;
            ws.b[vt >> 5] = a2;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < VW; ++w) {
            x += ws.a[w];
            y += ws.b[w];
        }
        part[2 * sb] = x;
        part[2 * sb + 1] = y;
    }
    __syncthreads();
}

// Band mode with the list step: the members (|φ| < γ, the step's own test)
// of tile t of kStepTile entries of the band list Lb (nb entries) that the
// next step reads, into tile_cnt[t]. One warp.
template <typename T>
__device__ __forceinline__ void tile_count(const Params<T>& P, const T* __restrict__ u, const int* Lb, int nb, int t,
                                           int* tile_cnt) {
    const int lane = threadIdx.x & 31;
    int c = 0;
#pragma unroll
    for (int h = 0; h < kStepTile / 32; ++h) {
        const int e = t * kStepTile + h * 32 + lane;
        const bool in = e < nb && fabs(ld(u + ld(Lb + e))) < P.gamma;
        c += __popc(__ballot_sync(0xffffffffu, in));
    }
    if (lane == 0) tile_cnt[t] = c;
}

// Reduction of the step and energy partials and the bookkeeping of one
// iteration. kRecordBlocks blocks each sum a fixed slice of the partials
// (FP64, fixed order) into one triple; the last block to finish sums the
// triples in block order and does the bookkeeping:
//  mode 0 (init):   E_2(φ^0) into the history, E_p for the first step
//  mode 1 (step):   Δ_φ, band size, n += 1, E_2(φ^{n}), E_p; with evolve
//                   set, the stop test of §4 eq. deltaEn
//  mode 2 (report): sums of the energy pass into report[0..1] only
// The slices depend on the sizes alone, so the result does not depend on
// which block finishes last.
static_assert(kRecordBlocks <= 32, "the last record block combines one value per lane");
constexpr int kRecordThreads = 256;

struct RecordArgs {
    const int* ncells_dev; // reinitialisation: candidate cells counted on the device (energy slots of 1024)
    int* tile_off;         // band mode: tile counts in, offsets within the slice out
    int offset;            // 1 after a step (the band the next step reads has parity n+1), else 0
    const double* part_dphi;
    const double* part_e;
    double* block_part;    // 3 per record block
    long long nchunks;     // number of energy partial pairs (energy blocks)
    long long n_dphi_full; // number of Δ_φ partials in whole-grid mode (step blocks)
    long long N;
    int full_grid;
    int reinit;            // Δ_φ partials from the reinitialisation stage; band size from band_sl
    int bricked;           // brick step: n_dphi_full partials, one per brick; band size from band_brick
    int mode;
    int evolve;
    double h_dim;  // h^dim
    double p;
    int p_kind;
    double stop_tol;
    int stop_k, min_iters, max_iters;
    double* report;
};

// Shared-memory workspace of one record slice
struct RecordWs {
    double a[kRecordThreads / 32], b[kRecordThreads / 32], c[kRecordThreads / 32];
    double hist[kMaxStopK + 1];
    int scan[kRecordThreads / 32];
    int last;
};

// Slice blk of the G = kRecordBlocks slices of one job's record reduction
// (all NT threads of the block calling), then, in the block that finishes
// the job's last slice, the bookkeeping. The FP64 sums follow the tree of
// kRecordThreads threads whatever NT; the tile offsets are integers.
// Returns true in the block that did the bookkeeping.
template <int NT>
__device__ __forceinline__ bool record_slice(const RecordArgs& A, DevState* ds, int blk, int G, RecordWs& ws) {
    static_assert(kRecordThreads % NT == 0 && NT >= 64, "the block size divides kRecordThreads");
    constexpr int V = kRecordThreads / NT;
    constexpr int VW = kRecordThreads / 32;
    if (A.mode == 1 && ds->stop) return false;
    const int n = ds->n;
    long long ntiles = 0;
    if (A.mode == 1) {
        ntiles = (A.full_grid || A.reinit || A.bricked) ? A.n_dphi_full
                                           : ((long long)ds->band_count[n & 1] + kStepTile - 1) / kStepTile;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long nch = A.ncells_dev ? ((long long)*A.ncells_dev + 1023) / 1024 : A.nchunks;
#pragma unroll 1
    for (int r = 0; r < V; ++r) {
        const int vt = threadIdx.x + r * NT;  // thread of the kRecordThreads tree
        double a = 0.0, b = 0.0, cc = 0.0;
        {
            const long long per = (ntiles + G - 1) / G;
            const long long beg = blk * per, end = beg + per < ntiles ? beg + per : ntiles;
            for (long long i = beg + vt; i < end; i += kRecordThreads) a += __ldcg(A.part_dphi + i);
        }
        {
            const double2* pe = reinterpret_cast<const double2*>(A.part_e);
            const long long per = (nch + G - 1) / G;
            const long long beg = blk * per, end = beg + per < nch ? beg + per : nch;
            for (long long i = beg + vt; i < end; i += kRecordThreads) {
                const double2 v = __ldcg(pe + i);
                b += v.x;
                cc += v.y;
            }
        }
        a = warp_sum(a);
        b = warp_sum(b);
        cc = warp_sum(cc);
        if (lane == 0) {
            ws.a[vt >> 5] = a;
            ws.b[vt >> 5] = b;
            ws.c[vt >> 5] = cc;
        }
    }
    if (A.tile_off) {
        // exclusive scan of this slice of tile counts (in place); the slice
        // total goes to band_base[blk] for the last block
        const int nb = ds->band_count[(n + A.offset) & 1];
        const int ntb = (nb + kStepTile - 1) / kStepTile;
        const int per = (ntb + G - 1) / G;
        const int beg = blk * per, end = beg + per < ntb ? beg + per : ntb;
        const int len = end > beg ? end - beg : 0;
        const int q = (len + NT - 1) / NT;  // contiguous run per thread
        const int rb = beg + (int)threadIdx.x * q, re = rb + q < end ? rb + q : end;
        int sum = 0;
        for (int i = rb; i < re; ++i) sum += __ldcg(A.tile_off + i);
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) ws.scan[w] = incl;
        __syncthreads();
        int run = incl - sum;
        for (int i = 0; i < w; ++i) run += ws.scan[i];
        for (int i = rb; i < re; ++i) {
            const int c = __ldcg(A.tile_off + i);
            A.tile_off[i] = run;
            run += c;
        }
        if (threadIdx.x == NT - 1) {
            ds->band_base[blk] = run;  // slice total
            __threadfence();
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0, z = 0.0;
        for (int i = 0; i < VW; ++i) {
            x += ws.a[i];
            y += ws.b[i];
            z += ws.c[i];
        }
        A.block_part[3 * blk + 0] = x;
        A.block_part[3 * blk + 1] = y;
        A.block_part[3 * blk + 2] = z;
        __threadfence();
        const unsigned prev = atomicAdd(&ds->record_done, 1u);
        ws.last = prev == (unsigned)G - 1;
    }
    __syncthreads();
    const bool last = ws.last != 0;
    __syncthreads();  // ws is reused by the caller's next item
    if (!last) return false;
    __threadfence();
    // the stop test's window of earlier energies:
    // hist[t] = E_2 at iteration (nn - k) + t for t < k (nn, k as below)
    const int nn = A.mode == 1 ? n + 1 : n;
    const int kwin = nn < A.stop_k ? nn : A.stop_k;
    if (A.mode == 1 && A.evolve)
        for (int t = threadIdx.x; t < kwin; t += NT) ws.hist[t] = __ldcg(ds->e2_hist + (nn - kwin + t) % kHist);
    if (A.tile_off && w == 1) {
        // slice totals -> exclusive slice bases; their sum is the next band size
        int tot = lane < G ? __ldcg(ds->band_base + lane) : 0;
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane < G) ds->band_base[lane] = incl - tot;
        if (lane == 31) ds->band_next = incl;
    }
    if (w == 0) {
        // slice triples in slice order (a fixed shuffle tree over lanes)
        double x = 0.0, y = 0.0, z = 0.0;
        if (lane < G) {
            x = __ldcg(A.block_part + 3 * lane + 0);
            y = __ldcg(A.block_part + 3 * lane + 1);
            z = __ldcg(A.block_part + 3 * lane + 2);
        }
        x = warp_sum(x);
        y = warp_sum(y);
        z = warp_sum(z);
        if (lane == 0) {
            ws.a[0] = x;
            ws.b[0] = y;
            ws.c[0] = z;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ds->record_done = 0u;
        ds->eticket[0] = 0u;
        ds->eticket[1] = 0u;
        const double dphi = ws.a[0], sp = ws.b[0], s2 = ws.c[0];
        if (A.mode == 2) {
            A.report[0] = sp;
            A.report[1] = s2;
        } else {
            if (A.mode == 1) {
                ds->dphi_hist[n % kHist] = dphi * A.h_dim;
                ds->band_hist[n % kHist] =
                    A.full_grid ? A.N
                                : (A.bricked ? (long long)ds->band_brick
                                             : (A.reinit ? (long long)ds->band_sl
                                                         : (long long)ds->band_count[(n + 1) & 1]));
                ds->n = nn;
            }
            ds->band_brick = 0;
            double E2 = sqrt(s2);
            ds->e2_hist[nn % kHist] = E2;
            ds->Ep = A.p_kind == 2 ? E2 : (A.p_kind == 1 ? 1.0 : pow(sp, 1.0 / A.p));
            if (A.mode == 1) {
                ds->ticket = 0u;
                if (A.evolve) {
                    // §4 eq. deltaEn with k = min(n, k_max) for both running
                    // means: en over iterations nn-k+1..nn, em over nn-k..nn-1,
                    // summed in increasing iteration order
                    const int k = kwin;
                    double en = 0.0, em = 0.0;
                    for (int i = 1; i < k; ++i) en += ws.hist[i];
                    en += E2;
                    for (int i = 0; i < k; ++i) em += ws.hist[i];
                    en /= (double)k;
                    em /= (double)k;
                    double delta = en > 0.0 ? fabs(em - en) / en : (em == en ? 0.0 : INFINITY);
                    int conv = (nn >= A.min_iters) && (delta < A.stop_tol);
                    if (conv || nn >= A.max_iters) {
                        ds->stop = 1;
                        ds->converged = conv;
                    }
                }
            }
        }
    }
    __syncthreads();  // ws is reused by the caller's next item
    return true;
}

// host side (slr_energy.cu): the quadrature scalars and the record
// arguments of one job, and its number of energy slots
template <typename T>
EnergyArgs<T> energy_args(const slr_ctx* c, double p, int p_kind);
RecordArgs record_args(slr_ctx* c, int record_mode, int evolve_mode, double p, int p_kind);
long long energy_slots(const slr_ctx* c);

}  // namespace slr
