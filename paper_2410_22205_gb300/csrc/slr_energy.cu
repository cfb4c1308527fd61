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
        uv[c] = (double)u[id[c]];
        dv[c] = (double)d[id[c]];
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
// positive), in candidate order, into out[] (block-wide: every thread of the
// block calls it). Returns their count.
template <typename T, int DIM>
__device__ __forceinline__ int front_of_slot(const Params<T>& P, const T* __restrict__ u, const int* __restrict__ cells,
                                             long long ncells, long long sb, int* out, int* s_warp) {
    constexpr int W = kEnergyThreads / 32;
    constexpr int PER = kEnergyCand / kEnergyThreads;
    static_assert(PER == 4, "four candidates per thread (one 16-byte load of the cell list)");
    // thread t checks the candidates e0 .. e0+3, e0 = slot start + 4t
    const long long e0 = sb * kEnergyCand + PER * threadIdx.x;
    int node[PER];
    if (cells && e0 + PER <= ncells) {
        const int4 c4 = *reinterpret_cast<const int4*>(cells + e0);  // slot starts are multiples of 1024
        node[0] = c4.x;
        node[1] = c4.y;
        node[2] = c4.z;
        node[3] = c4.w;
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

template <typename T, int DIM, int INTERP, int RC>
__global__ void __launch_bounds__(kEnergyThreads, (INTERP == 1 && sizeof(T) == 4) ? 4 : 1) k_energy(Params<T> P, const T* ub0, const T* ub1,
                                                           const T* __restrict__ d, const int* __restrict__ cells,
                                                           long long ncells_host,
                                                           const int* ncells_dev, int R_run, double h,
                                                           double p, int p_kind, T thr, T hp2, T pT, int offset,
                                                           double* part, const int* L0, const int* L1,
                                                           int* __restrict__ tile_cnt, DevState* ds, int check_stop) {
    constexpr int W = kEnergyThreads / 32;
    const int R = RC > 0 ? RC : R_run;
    constexpr double RD = RC > 0 ? (double)RC : 1.0;
    __shared__ T s_th[kMaxR];
    __shared__ WenoAxis<T> s_wa[kMaxR];
    __shared__ double s_a[W], s_b[W];
    __shared__ int s_front[kEnergyCand];  // this slot's front cells
    __shared__ int s_warp[W + 1];
    if (check_stop && ds->stop) return;
    const int sel = (ds->n + offset) & 1;
    const T* __restrict__ u = sel ? ub1 : ub0;
    if (tile_cnt) {
        // band mode: members (|φ| < γ, the step kernel's test) of each tile
        // of kStepTile entries of the band list the next step reads
        const int nb = ds->band_count[sel];
        const int* __restrict__ Lb = sel ? L1 : L0;
        const int ntb = (nb + kStepTile - 1) / kStepTile;
        const int lane = threadIdx.x & 31;
        const int nw = gridDim.x * W;
        for (int t = blockIdx.x * W + (threadIdx.x >> 5); t < ntb; t += nw) {
            int c = 0;
#pragma unroll
            for (int h = 0; h < kStepTile / 32; ++h) {
                const int e = t * kStepTile + h * 32 + lane;
                const bool in = e < nb && fabs(u[Lb[e]]) < P.gamma;
                c += __popc(__ballot_sync(0xffffffffu, in));
            }
            if (lane == 0) tile_cnt[t] = c;
        }
    }
    if (RC == 0 && threadIdx.x < R) {
        T t = ((T)threadIdx.x + (T)0.5) / (T)R;  // subcell centre θ_m = (m + 1/2)/R
        s_th[threadIdx.x] = t;
        s_wa[threadIdx.x].set_exact(t);
    }
    __syncthreads();
    const long long ncells = ncells_dev ? (long long)*ncells_dev : ncells_host;
    const long long nslots = (ncells + kEnergyCand - 1) / kEnergyCand;
    __shared__ long long s_sb;
    for (;;) {
        if (threadIdx.x == 0) s_sb = (long long)atomicAdd(&ds->eticket[1], 1u);
        __syncthreads();
        const long long sb = s_sb;
        __syncthreads();
        if (sb >= nslots) break;
        const int nf = front_of_slot<T, DIM>(P, u, cells, ncells, sb, s_front, s_warp);
        const int* s_list = s_front;
        // thr = (√3/2) Δx', hp2 = Δx'^2, pT = p: computed on the host
        auto TH = [&](int m) -> T { return RC > 0 ? (T)m * (T)(1.0 / RD) + (T)(0.5 / RD) : s_th[m]; };
        // WENO constants at θ_m (storage-type arithmetic; folded at compile
        // time where m is a constant)
        auto WA = [&](int m) -> WenoAxis<T> {
            if (RC > 0) {
                WenoAxis<T> w;
                w.set_exact(TH(m));
                return w;
            }
            return s_wa[m];
        };
        auto contrib = [&](T uu, T dd, T& cp, T& c2) {
            const T a = fabs(dd);
            const T d2 = a * a;
            const T keep = fabs(uu) < thr ? hp2 : T(0);
            cp += (p_kind == 2 ? d2 : (p_kind == 1 ? a : (T)pow(a, pT))) * keep;
            c2 += d2 * keep;
        };
        double ap = 0.0, a2 = 0.0;
        if (DIM == 2) {
            for (int fi = threadIdx.x; fi < nf; fi += kEnergyThreads) {
                const int nd = s_list[fi];
                const int q = nd / P.n0;
                double s2 = 0.0;
                ap += energy_cell_2d<T>(P, u, d, nd - q * P.n0, q, h, p, p_kind, &s2);
                a2 += s2;
            }
        } else {
            // sums over this thread's items in the storage type, widened once
            T tp = T(0), t2 = T(0);
            const int items = nf * R;
            for (int it = threadIdx.x; it < items; it += kEnergyThreads) {
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
                for (int c = 0; c < 4; ++c) dz[c] = dc[c] + tz * (dc[c + 4] - dc[c]);
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
                        const T d0 = dz[0] + ty * (dz[2] - dz[0]), d1 = dz[1] + ty * (dz[3] - dz[1]);
    #pragma unroll
                        for (int ax = 0; ax < (RC > 0 ? RC : kMaxR); ++ax) {
                            if (RC == 0 && ax >= R) break;
                            const T tx = TH(ax);
                            contrib(ix.eval(WA(ax)), d0 + tx * (d1 - d0), cp, c2);
                        }
                    }
                } else {
                    T uc[8];
    #pragma unroll
                    for (int c = 0; c < 8; ++c) uc[c] = ld(u + (nd + (c & 1) + P.is1 * ((c >> 1) & 1) + P.is2 * (c >> 2)));
                    T uz[4];
    #pragma unroll
                    for (int c = 0; c < 4; ++c) uz[c] = uc[c] + tz * (uc[c + 4] - uc[c]);
                    for (int by = 0; by < R; ++by) {
                        const T ty = TH(by);
                        const T u0 = uz[0] + ty * (uz[2] - uz[0]), u1 = uz[1] + ty * (uz[3] - uz[1]);
                        const T d0 = dz[0] + ty * (dz[2] - dz[0]), d1 = dz[1] + ty * (dz[3] - dz[1]);
                        for (int ax = 0; ax < R; ++ax) {
                            const T tx = TH(ax);
                            contrib(u0 + tx * (u1 - u0), d0 + tx * (d1 - d0), cp, c2);
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
        if (DIM == 2) {
            ap = warp_sum(ap);
            a2 = warp_sum(a2);
        }
        const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
        if (lane == 0) {
            s_a[wib] = ap;
            s_b[wib] = a2;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double x = 0.0, y = 0.0;
            for (int w = 0; w < W; ++w) {
                x += s_a[w];
                y += s_b[w];
            }
            part[2 * sb] = x;
            part[2 * sb + 1] = y;
        }
        __syncthreads();
    }
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

__global__ void __launch_bounds__(kRecordThreads) k_record(RecordArgs A, DevState* ds) {
    constexpr int W = kRecordThreads / 32;
    __shared__ double s_a[W], s_b[W], s_c[W];
    __shared__ double s_hist[kMaxStopK + 1];
    __shared__ int s_scan[W];
    __shared__ int s_last;
    if (A.mode == 1 && ds->stop) return;
    const int n = ds->n;
    long long ntiles = 0;
    if (A.mode == 1) {
        ntiles = (A.full_grid || A.reinit || A.bricked) ? A.n_dphi_full
                                           : ((long long)ds->band_count[n & 1] + kStepTile - 1) / kStepTile;
    }
    const long long G = gridDim.x;
    double a = 0.0, b = 0.0, cc = 0.0;
    {
        const long long per = (ntiles + G - 1) / G;
        const long long beg = blockIdx.x * per, end = beg + per < ntiles ? beg + per : ntiles;
        for (long long i = beg + threadIdx.x; i < end; i += kRecordThreads) a += A.part_dphi[i];
    }
    {
        const double2* pe = reinterpret_cast<const double2*>(A.part_e);
        const long long nch = A.ncells_dev ? ((long long)*A.ncells_dev + 1023) / 1024 : A.nchunks;
        const long long per = (nch + G - 1) / G;
        const long long beg = blockIdx.x * per, end = beg + per < nch ? beg + per : nch;
        for (long long i = beg + threadIdx.x; i < end; i += kRecordThreads) {
            const double2 v = pe[i];
            b += v.x;
            cc += v.y;
        }
    }
    a = warp_sum(a);
    b = warp_sum(b);
    cc = warp_sum(cc);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s_a[w] = a;
        s_b[w] = b;
        s_c[w] = cc;
    }
    if (A.tile_off) {
        // exclusive scan of this block's slice of tile counts (in place);
        // the slice total goes to band_base[block] for the last block
        const int nb = ds->band_count[(n + A.offset) & 1];
        const int ntb = (nb + kStepTile - 1) / kStepTile;
        const int per = (ntb + (int)G - 1) / (int)G;
        const int beg = (int)blockIdx.x * per, end = beg + per < ntb ? beg + per : ntb;
        const int len = end > beg ? end - beg : 0;
        const int q = (len + kRecordThreads - 1) / kRecordThreads;  // contiguous run per thread
        const int rb = beg + (int)threadIdx.x * q, re = rb + q < end ? rb + q : end;
        int sum = 0;
        for (int i = rb; i < re; ++i) sum += A.tile_off[i];
        int incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) s_scan[w] = incl;
        __syncthreads();
        int run = incl - sum;
        for (int i = 0; i < w; ++i) run += s_scan[i];
        for (int i = rb; i < re; ++i) {
            const int c = A.tile_off[i];
            A.tile_off[i] = run;
            run += c;
        }
        if (threadIdx.x == kRecordThreads - 1) {
            ds->band_base[blockIdx.x] = run;  // slice total
            __threadfence();
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0, y = 0.0, z = 0.0;
        for (int i = 0; i < W; ++i) {
            x += s_a[i];
            y += s_b[i];
            z += s_c[i];
        }
        A.block_part[3 * blockIdx.x + 0] = x;
        A.block_part[3 * blockIdx.x + 1] = y;
        A.block_part[3 * blockIdx.x + 2] = z;
        __threadfence();
        const unsigned prev = atomicAdd(&ds->record_done, 1u);
        s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the stop test's window of earlier energies:
    // s_hist[t] = E_2 at iteration (nn - k) + t for t < k (nn, k as below)
    const int nn = A.mode == 1 ? n + 1 : n;
    const int kwin = nn < A.stop_k ? nn : A.stop_k;
    if (A.mode == 1 && A.evolve)
        for (int t = threadIdx.x; t < kwin; t += kRecordThreads) s_hist[t] = ds->e2_hist[(nn - kwin + t) % kHist];
    if (A.tile_off && w == 1) {
        // slice totals -> exclusive slice bases; their sum is the next band size
        int tot = lane < (int)gridDim.x ? __ldcg(ds->band_base + lane) : 0;
        int incl = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane < (int)gridDim.x) ds->band_base[lane] = incl - tot;
        if (lane == 31) ds->band_next = incl;
    }
    if (w == 0) {
        // block triples in block order (a fixed shuffle tree over lanes)
        double x = 0.0, y = 0.0, z = 0.0;
        if (lane < (int)gridDim.x) {
            x = __ldcg(A.block_part + 3 * lane + 0);
            y = __ldcg(A.block_part + 3 * lane + 1);
            z = __ldcg(A.block_part + 3 * lane + 2);
        }
        x = warp_sum(x);
        y = warp_sum(y);
        z = warp_sum(z);
        if (lane == 0) {
            s_a[0] = x;
            s_b[0] = y;
            s_c[0] = z;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    ds->record_done = 0u;
    ds->eticket[0] = 0u;
    ds->eticket[1] = 0u;
    const double dphi = s_a[0], sp = s_b[0], s2 = s_c[0];
    if (A.mode == 2) {
        A.report[0] = sp;
        A.report[1] = s2;
        return;
    }
    if (A.mode == 1) {
        ds->dphi_hist[n % kHist] = dphi * A.h_dim;
        ds->band_hist[n % kHist] =
            A.full_grid ? A.N
                        : (A.bricked ? (long long)ds->band_brick
                                     : (A.reinit ? (long long)ds->band_sl : (long long)ds->band_count[(n + 1) & 1]));
        ds->n = nn;
    }
    if (A.mode != 2) ds->band_brick = 0;
    double E2 = sqrt(s2);
    ds->e2_hist[nn % kHist] = E2;
    ds->Ep = A.p_kind == 2 ? E2 : (A.p_kind == 1 ? 1.0 : pow(sp, 1.0 / A.p));
    if (A.mode == 1) {
        ds->ticket = 0u;
        if (A.evolve) {
            // §4 eq. deltaEn with k = min(n, k_max) for both running means:
            // en over iterations nn-k+1..nn, em over nn-k..nn-1, summed in
            // increasing iteration order
            const int k = kwin;
            double en = 0.0, em = 0.0;
            for (int i = 1; i < k; ++i) en += s_hist[i];
            en += E2;
            for (int i = 0; i < k; ++i) em += s_hist[i];
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

template <typename T, int DIM, int INTERP>
static cudaError_t energy_t(slr_ctx* c, int offset, double p, int p_kind, int check_stop) {
    Params<T> P = make_params<T>(c);
    const int* cells = c->cfg.band ? c->ecells : nullptr;
    long long ncells = c->cfg.band ? c->n_ecells : c->ncells_all;
    const int blocks = (int)energy_blocks(c);
    const double hp = c->h / c->cfg.energy_R;
    const T thr = (T)(0.8660254037844386 * hp), hp2 = (T)(hp * hp), pT = (T)p;
    const int* ncells_dev = c->cfg.reinit ? &c->ds->n_ecells_dyn : nullptr;  // the list changes every iteration
    // the list step reads per-tile counts of the band list; the brick step does not
    int* tile_cnt = (c->cfg.band && !brick_mode(c)) ? c->tile_off : nullptr;
    if (DIM == 3 && c->cfg.energy_R == 5)
        k_energy<T, DIM, INTERP, 5><<<blocks, kEnergyThreads, 0, c->stream>>>(
            P, (const T*)c->u[0], (const T*)c->u[1], (const T*)c->d, cells, ncells, ncells_dev,
            c->cfg.energy_R, c->h, p, p_kind, thr, hp2, pT, offset, c->part_e, c->band[0], c->band[1], tile_cnt, c->ds,
            check_stop);
    else
        k_energy<T, DIM, INTERP, 0><<<blocks, kEnergyThreads, 0, c->stream>>>(
            P, (const T*)c->u[0], (const T*)c->u[1], (const T*)c->d, cells, ncells, ncells_dev,
            c->cfg.energy_R, c->h, p, p_kind, thr, hp2, pT, offset, c->part_e, c->band[0], c->band[1], tile_cnt, c->ds,
            check_stop);
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
