// Energy functional, stopping criterion and diagnostics (arXiv 2410.22205,
// §3.5 and §4), all on the device with FP64 accumulation.
//
// Energy: the candidate cells (every cell in whole-grid mode; in band mode
// the cells touching the initial band or crossing the front at init) are
// taken 32 at a time by one warp; a ballot finds the front cells (vertices of
// both signs, zero counted as positive) and the warp then works through them
// one by one:
//   2-D: edge crossings by linear interpolation of φ, d interpolated along
//        the edge, trapezoid rule on the segment(s) (eq. energyApprox);
//   3-D: R^3 subcells (eq. energyApproxFiner); φ at the subcell centres by
//        the active interpolator — for WENO the dimension splitting shares
//        work across the regular R×R×R lattice (16R z-evaluations, then 4R^2
//        along y, then R^3 along x, all with the same arithmetic as a single
//        point evaluation); d by Q1; a subcell counts when
//        |φ(x')| < (√3/2)Δx' and adds |d(x')|^p (Δx')^2.
// Each warp writes FP64 partial sums per chunk; one block reduces them in a
// fixed order, so results are bit-reproducible.
#include "slr_internal.cuh"

namespace slr {

template <typename T>
Params<T> make_params(const slr_ctx* c);

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

template <typename T, int DIM, int INTERP>
__global__ void __launch_bounds__(kEnergyBlock) k_energy(Params<T> P, const T* ub0, const T* ub1,
                                                         const T* __restrict__ d, const int* __restrict__ cells,
                                                         long long ncells, long long nchunks, int R, double h,
                                                         double p, int p_kind, int offset, double* part,
                                                         DevState* ds, int check_stop) {
    constexpr int W = kEnergyBlock / 32;
    __shared__ T s_sv[W][64];
    __shared__ T s_zv[W][16 * kMaxR];
    __shared__ T s_yv[W][4 * kMaxR * kMaxR];
    __shared__ T s_dc[W][8];
    if (check_stop && ds->stop) return;
    const T* __restrict__ u = ((ds->n + offset) & 1) ? ub1 : ub0;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long gw = (long long)blockIdx.x * W + wib;
    const long long nw = (long long)gridDim.x * W;
    const T hp = (T)(h / R);
    const T thr = (T)(0.8660254037844386 * (h / R));  // (√3/2) Δx'
    const double hp2 = (h / R) * (h / R);
    T* sv = s_sv[wib];
    T* zv = s_zv[wib];
    T* yv = s_yv[wib];
    T* dc = s_dc[wib];
    (void)hp;
    for (long long c = gw; c < nchunks; c += nw) {
        const long long e = c * 32 + lane;
        int ci = 0, cj = 0, ck = 0;
        bool front = false;
        if (e < ncells) {
            cell_of<T, DIM>(P, cells, e, ci, cj, ck);
            long long b = ci + P.s1 * cj + P.s2 * ck;
            bool neg = false, pos = false;
#pragma unroll
            for (int dz = 0; dz < (DIM == 3 ? 2 : 1); ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                    for (int dx = 0; dx < 2; ++dx) {
                        T v = u[b + dx + P.s1 * dy + P.s2 * dz];
                        if (v < T(0))
                            neg = true;
                        else
                            pos = true;
                    }
            front = neg && pos;
        }
        unsigned m = __ballot_sync(0xffffffffu, front);
        double accp = 0.0, acc2 = 0.0;
        if (DIM == 2) {
            if (front) accp = energy_cell_2d<T>(P, u, d, ci, cj, h, p, p_kind, &acc2);
        } else {
            while (m) {
                const int f = __ffs(m) - 1;
                m &= m - 1;
                const int i = __shfl_sync(0xffffffffu, ci, f);
                const int j = __shfl_sync(0xffffffffu, cj, f);
                const int k = __shfl_sync(0xffffffffu, ck, f);
                const long long b = i + P.s1 * j + P.s2 * k;
                if (lane < 8) dc[lane] = d[b + (lane & 1) + P.s1 * ((lane >> 1) & 1) + P.s2 * (lane >> 2)];
                if (INTERP == 1) {
                    for (int q = lane; q < 64; q += 32) {
                        int a = q & 3, bb = (q >> 2) & 3, cz = q >> 4;
                        long long id = clampi(i - 1 + a, 0, P.n0 - 1) + P.s1 * clampi(j - 1 + bb, 0, P.n1 - 1) +
                                       P.s2 * clampi(k - 1 + cz, 0, P.n2 - 1);
                        sv[q] = u[id];
                    }
                    __syncwarp();
                    // z-lines: zv[(a*4+b)*R + c] at θ_z = (c + 1/2)/R
                    for (int q = lane; q < 16 * R; q += 32) {
                        int line = q / R, cz = q - line * R;
                        int a = line >> 2, bb = line & 3;
                        WenoAxis<T> wz;
                        wz.set((T)((cz + 0.5) / R));
                        const T* s = sv + a + 4 * bb;
                        zv[q] = weno1(s[0], s[16], s[32], s[48], wz, P.h4);
                    }
                    __syncwarp();
                    // y-lines: yv[(a*R + c)*R + b'] at θ_y = (b' + 1/2)/R
                    for (int q = lane; q < 4 * R * R; q += 32) {
                        int a = q / (R * R), rem = q - a * R * R;
                        int cz = rem / R, by = rem - cz * R;
                        WenoAxis<T> wy;
                        wy.set((T)((by + 0.5) / R));
                        yv[q] = weno1(zv[(a * 4 + 0) * R + cz], zv[(a * 4 + 1) * R + cz], zv[(a * 4 + 2) * R + cz],
                                      zv[(a * 4 + 3) * R + cz], wy, P.h4);
                    }
                    __syncwarp();
                } else {
                    if (lane < 8) sv[lane] = u[b + (lane & 1) + P.s1 * ((lane >> 1) & 1) + P.s2 * (lane >> 2)];
                    __syncwarp();
                }
                // x pass (WENO) or trilinear (Q1), d by Q1, accumulate
                for (int q = lane; q < R * R * R; q += 32) {
                    int cz = q / (R * R), rem = q - cz * R * R;
                    int by = rem / R, ax = rem - by * R;
                    T tx = (T)((ax + 0.5) / R), ty = (T)((by + 0.5) / R), tz = (T)((cz + 0.5) / R);
                    T uu;
                    if (INTERP == 1) {
                        WenoAxis<T> wx;
                        wx.set(tx);
                        const int RR = R * R;
                        uu = weno1(yv[cz * R + by], yv[RR + cz * R + by], yv[2 * RR + cz * R + by],
                                   yv[3 * RR + cz * R + by], wx, P.h4);
                    } else {
                        T a0 = sv[0] + tx * (sv[1] - sv[0]);
                        T a1 = sv[2] + tx * (sv[3] - sv[2]);
                        T a2 = sv[4] + tx * (sv[5] - sv[4]);
                        T a3 = sv[6] + tx * (sv[7] - sv[6]);
                        T b0 = a0 + ty * (a1 - a0);
                        T b1 = a2 + ty * (a3 - a2);
                        uu = b0 + tz * (b1 - b0);
                    }
                    T e0 = dc[0] + tx * (dc[1] - dc[0]);
                    T e1 = dc[2] + tx * (dc[3] - dc[2]);
                    T e2 = dc[4] + tx * (dc[5] - dc[4]);
                    T e3 = dc[6] + tx * (dc[7] - dc[6]);
                    T f0 = e0 + ty * (e1 - e0);
                    T f1 = e2 + ty * (e3 - e2);
                    double dd = (double)(f0 + tz * (f1 - f0));
                    if (fabs(uu) < thr) {
                        accp += pow_abs(dd, p, p_kind) * hp2;
                        acc2 += dd * dd * hp2;
                    }
                }
                __syncwarp();
            }
        }
        accp = warp_sum(accp);
        acc2 = warp_sum(acc2);
        if (lane == 0) {
            part[2 * c] = accp;
            part[2 * c + 1] = acc2;
        }
    }
}

// Reduction of the step and energy partials and the bookkeeping of one
// iteration (single block, fixed summation order).
//  mode 0 (init):   E_2(φ^0) into the history, E_p for the first step
//  mode 1 (step):   Δ_φ, band size, n += 1, E_2(φ^{n}), E_p; with evolve
//                   set, the stop test of §4 eq. deltaEn
//  mode 2 (report): sums of the energy pass into report[0..1] only
struct RecordArgs {
    const double* part_dphi;
    const double* part_e;
    long long nchunks;
    long long N;
    int full_grid;
    int mode;
    int evolve;
    double h_dim;  // h^dim
    double p;
    int p_kind;
    double stop_tol;
    int stop_k, min_iters, max_iters;
    double* report;
};

__global__ void __launch_bounds__(1024) k_record(RecordArgs A, DevState* ds) {
    __shared__ double s_a[32], s_b[32], s_c[32];
    if (A.mode == 1 && ds->stop) return;
    const int n = ds->n;
    long long ntiles = 0;
    if (A.mode == 1) {
        long long cnt = A.full_grid ? A.N : (long long)ds->band_count[n & 1];
        ntiles = (cnt + kStepTile - 1) / kStepTile;
    }
    double a = 0.0, b = 0.0, cc = 0.0;
    for (long long t = threadIdx.x; t < ntiles; t += blockDim.x) a += A.part_dphi[t];
    for (long long t = threadIdx.x; t < A.nchunks; t += blockDim.x) {
        b += A.part_e[2 * t];
        cc += A.part_e[2 * t + 1];
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
    __syncthreads();
    if (threadIdx.x != 0) return;
    double dphi = 0.0, sp = 0.0, s2 = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) {
        dphi += s_a[i];
        sp += s_b[i];
        s2 += s_c[i];
    }
    if (A.mode == 2) {
        A.report[0] = sp;
        A.report[1] = s2;
        return;
    }
    int nn = n;
    if (A.mode == 1) {
        ds->dphi_hist[nn % kHist] = dphi * A.h_dim;
        ds->band_hist[nn % kHist] = A.full_grid ? A.N : (long long)ds->band_count[(nn + 1) & 1];
        nn += 1;
        ds->n = nn;
    }
    double E2 = sqrt(s2);
    ds->e2_hist[nn % kHist] = E2;
    ds->Ep = A.p_kind == 2 ? E2 : (A.p_kind == 1 ? 1.0 : pow(sp, 1.0 / A.p));
    if (A.mode == 1) {
        ds->ticket = 0u;
        ds->epoch = ds->epoch + 1u;
        if (A.evolve) {
            // §4 eq. deltaEn with k = min(n, k_max) for both running means
            int k = nn < A.stop_k ? nn : A.stop_k;
            double en = 0.0, em = 0.0;
            for (int i = nn - k + 1; i <= nn; ++i) en += ds->e2_hist[i % kHist];
            for (int i = nn - k; i <= nn - 1; ++i) em += ds->e2_hist[i % kHist];
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
    long long nchunks = (ncells + 31) / 32;
    long long blocks = (nchunks + kEnergyBlock / 32 - 1) / (kEnergyBlock / 32);
    long long cap = (long long)c->num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k_energy<T, DIM, INTERP><<<(int)blocks, kEnergyBlock, 0, c->stream>>>(
        P, (const T*)c->u[0], (const T*)c->u[1], (const T*)c->d, cells, ncells, nchunks, c->cfg.energy_R, c->h, p,
        p_kind, offset, c->part_e, c->ds, check_stop);
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
cudaError_t launch_energy(slr_ctx* c, int offset, double p_override, int record_mode, int evolve_mode) {
    double p = record_mode == 2 ? p_override : c->cfg.p;
    int p_kind = p == 1.0 ? 1 : (p == 2.0 ? 2 : 0);
    cudaError_t e = energy_dispatch(c, offset, p, p_kind, record_mode == 1);
    if (e != cudaSuccess) return e;
    RecordArgs A;
    A.part_dphi = c->part_dphi;
    A.part_e = c->part_e;
    A.nchunks = c->n_echunks;
    A.N = c->N;
    A.full_grid = !c->cfg.band;
    A.mode = record_mode;
    A.evolve = evolve_mode;
    A.h_dim = c->cfg.dim == 3 ? c->h * c->h * c->h : c->h * c->h;
    A.p = p;
    A.p_kind = p_kind;
    A.stop_tol = c->cfg.stop_tol;
    A.stop_k = c->cfg.stop_k;
    A.min_iters = c->cfg.min_iters;
    A.max_iters = c->cfg.max_iters;
    A.report = c->part_e + 2 * c->n_echunks;  // two spare doubles after the partials
    k_record<<<1, 1024, 0, c->stream>>>(A, c->ds);
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
