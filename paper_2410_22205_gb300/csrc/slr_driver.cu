// Several runs of Algorithm 1 from coarse to fine (§4: eq. dxdt and Tab.
// param), every step on the device:
//  - h_S, the cloud's resolution, from a sample of the points (slr_cloud_spacing);
//  - run r on a grid of width Δx(r) = h_S / 2^(r-1) over the cloud's bounding
//    box widened by 8 Δx(r), plus γ_S in the first run, with
//    (p, δ) = (1, 0), (2, 0), (2, 1), (2, 1), ...;
//  - φ^0 of the first run by external marking and fast sweeping at
//    γ_S = K_S Δx(1) (§3.6; K_S h_S unless the first grid was coarsened), of
//    the later runs by Q1 interpolation of the previous run's
//    steady state at the new nodes, then cut;
//  - Algorithm 1 with the reinitialisation of §3.7 to the stop test of §4;
//  - at the end of each run, the quantities of the paper's tables: E_2, Err_S
//    (eq. errCloud) and the L^1 error against an exact signed distance.
// Readings (the paper leaves them open): the sample is a Bernoulli draw with
// probability sample_frac per point, from a counter-based splitmix64 stream
// (Steele, Lea and Flood 2014); the margin of the box is the one that gives
// the grids printed for the circle test (42, 58, 99, 181 and 344 nodes per
// axis); a run whose grid would exceed max_nodes is coarsened to fit (Δx
// grows by the dim-th root of the excess); d is exact unless distance_fsm
// asks for the §3.4 construction.
#include <cuda_runtime.h>

#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "slr_internal.cuh"

namespace slr {

namespace {

// Q1 value of the coarse field (storage type T) at the nodes of the fine grid,
// FP64 with correctly rounded operations: index coordinate (x - lo)/h clamped
// to [0, n-1], cell clamped to [0, n-2], linear along x, then y, then z
struct GridGeom {
    int n[3];
    double lo[3];
    double h;
    int dim;
};

template <typename T>
__global__ void k_resample_q1(const T* __restrict__ uc, GridGeom C, GridGeom F, double* __restrict__ out, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += stride) {
        long long q = j;
        int fi[3] = {0, 0, 0};
        fi[0] = (int)(q % F.n[0]);
        q /= F.n[0];
        fi[1] = (int)(q % F.n[1]);
        fi[2] = (int)(q / F.n[1]);
        long long c[3] = {0, 0, 0};
        double t[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < C.dim; ++a) {
            const double x = __dadd_rn(F.lo[a], __dmul_rn((double)fi[a], F.h));
            double xi = __ddiv_rn(__dsub_rn(x, C.lo[a]), C.h);
            const double top = (double)(C.n[a] - 1);
            if (xi < 0.0) xi = 0.0;
            if (xi > top) xi = top;
            long long cc = (long long)floor(xi);
            if (cc > C.n[a] - 2) cc = C.n[a] - 2;
            c[a] = cc;
            t[a] = __dsub_rn(xi, (double)cc);
        }
        const long long s1 = C.n[0], s2 = (long long)C.n[0] * C.n[1];
        double vz[2] = {0.0, 0.0};
        const int nz = C.dim == 3 ? 2 : 1;
        for (int dz = 0; dz < nz; ++dz) {
            double vy[2];
            for (int dy = 0; dy < 2; ++dy) {
                const long long b = c[0] + s1 * (c[1] + dy) + s2 * (c[2] + dz);
                const double v0 = (double)uc[b], v1 = (double)uc[b + 1];
                vy[dy] = __dadd_rn(__dmul_rn(__dsub_rn(1.0, t[0]), v0), __dmul_rn(t[0], v1));
            }
            vz[dz] = __dadd_rn(__dmul_rn(__dsub_rn(1.0, t[1]), vy[0]), __dmul_rn(t[1], vy[1]));
        }
        out[j] = C.dim == 2 ? vz[0] : __dadd_rn(__dmul_rn(__dsub_rn(1.0, t[2]), vz[0]), __dmul_rn(t[2], vz[1]));
    }
}

uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// partial sums of |c(φ_j) - c(φ*_j)| per block (FP64); kind 0: φ* the
// signed distance to a sphere, from correctly rounded FP64 operations
constexpr int kL1Block = 256;

template <typename T>
__global__ void __launch_bounds__(kL1Block) k_l1_error(const T* __restrict__ u, GridGeom G, int kind, double cx,
                                                       double cy, double cz, double r,
                                                       const double* __restrict__ exact, int band, double gamma,
                                                       long long N, double* __restrict__ part) {
    __shared__ double s_sum[kL1Block / 32];
    double acc = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += stride) {
        double ex;
        if (kind == 0) {
            const long long q = j / G.n[0];
            const int i0 = (int)(j - q * G.n[0]);
            const int i1 = (int)(q % G.n[1]), i2 = (int)(q / G.n[1]);
            const double x = __dsub_rn(__dadd_rn(G.lo[0], __dmul_rn((double)i0, G.h)), cx);
            const double y = __dsub_rn(__dadd_rn(G.lo[1], __dmul_rn((double)i1, G.h)), cy);
            double s2 = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
            if (G.dim == 3) {
                const double z = __dsub_rn(__dadd_rn(G.lo[2], __dmul_rn((double)i2, G.h)), cz);
                s2 = __dadd_rn(s2, __dmul_rn(z, z));
            }
            ex = __dsub_rn(__dsqrt_rn(s2), r);
        } else {
            ex = exact[j];
        }
        double v = (double)u[j];
        if (band) {
            v = fmin(fmax(v, -gamma), gamma);
            ex = fmin(fmax(ex, -gamma), gamma);
        }
        acc += fabs(v - ex);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kL1Block / 32; ++w) t += s_sum[w];
        part[blockIdx.x] = t;
    }
}

GridGeom geom_of(const slr_config& k) {
    GridGeom g;
    g.dim = k.dim;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = (int)k.n[a];
        g.lo[a] = k.lo[a];
    }
    g.h = (k.hi[0] - k.lo[0]) / (double)(k.n[0] - 1);
    return g;
}

}  // namespace

cudaError_t launch_l1_error(slr_ctx* c, const void* u, int kind, const double* prm, const double* exact_dev,
                            double* part, int blocks) {
    const GridGeom G = geom_of(c->cfg);
    const double cx = kind == 0 ? prm[0] : 0.0, cy = kind == 0 ? prm[1] : 0.0;
    const double cz = kind == 0 && c->cfg.dim == 3 ? prm[2] : 0.0, r = kind == 0 ? prm[3] : 0.0;
    if (c->cfg.precision == 32)
        k_l1_error<float><<<blocks, kL1Block, 0, c->stream>>>((const float*)u, G, kind, cx, cy, cz, r, exact_dev,
                                                              c->cfg.band, c->gamma, c->N, part);
    else
        k_l1_error<double><<<blocks, kL1Block, 0, c->stream>>>((const double*)u, G, kind, cx, cy, cz, r, exact_dev,
                                                               c->cfg.band, c->gamma, c->N, part);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace slr

using namespace slr;

extern "C" {

void slr_multirun_default(slr_multirun_config* mc) {
    if (!mc) return;
    memset(mc, 0, sizeof(*mc));
    mc->dim = 3;
    mc->precision = 32;
    mc->interp = 1;
    mc->runs = 3;
    mc->K_s = 2.0;
    mc->sample_frac = 0.1;
    mc->seed = 1;
    mc->max_nodes = 1ll << 27;
    mc->max_iters = 100;
    mc->distance_fsm = 0;
    mc->exact_sphere = 0;
}

slr_status slr_reconstruct(const slr_multirun_config* mc, const double* xyz, int64_t n_points,
                           const slr_allocator* alloc, void* cuda_stream, slr_ctx** out,
                           slr_multirun_report* report) {
    if (!mc || !xyz || !out || n_points < 2) return SLR_E_INVALID;
    *out = nullptr;
    const int dim = mc->dim;
    if (dim != 2 && dim != 3) return SLR_E_INVALID;
    if (mc->runs < 1 || mc->runs > SLR_MAX_RUNS || !(mc->K_s > 0.0) || !(mc->sample_frac > 0.0) ||
        !(mc->sample_frac <= 1.0) || mc->max_nodes < 64 || mc->max_iters < 1 ||
        (mc->distance_fsm != 0 && mc->distance_fsm != 1) || (mc->exact_sphere != 0 && mc->exact_sphere != 1) ||
        (mc->exact_sphere && !(mc->sphere[3] >= 0.0 && isfinite(mc->sphere[0]) && isfinite(mc->sphere[1]) &&
                               isfinite(mc->sphere[2]) && isfinite(mc->sphere[3]))))
        return SLR_E_INVALID;
    slr_multirun_report rep;
    memset(&rep, 0, sizeof(rep));
    // bounding box of the cloud
    double bmin[3] = {0, 0, 0}, bmax[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        bmin[a] = INFINITY;
        bmax[a] = -INFINITY;
    }
    for (int64_t i = 0; i < n_points; ++i)
        for (int a = 0; a < dim; ++a) {
            const double v = xyz[i * dim + a];
            if (!isfinite(v)) return SLR_E_INVALID;
            if (v < bmin[a]) bmin[a] = v;
            if (v > bmax[a]) bmax[a] = v;
        }
    // the sample for h_S
    std::vector<int64_t> sample;
    const uint64_t lim = (uint64_t)(mc->sample_frac * 18446744073709551616.0 > 18446744073709549568.0
                                        ? 18446744073709549568.0
                                        : mc->sample_frac * 18446744073709551616.0);
    for (int64_t i = 0; i < n_points; ++i)
        if (mc->sample_frac >= 1.0 || splitmix64_at(mc->seed, (uint64_t)i) < lim) sample.push_back(i);
    if (sample.empty()) sample.push_back(0);
    // h_S on a provisional context (any grid: only the cloud's index is used)
    double hs = 0.0;
    {
        slr_config k;
        slr_config_default(&k);
        k.dim = dim;
        k.n[0] = k.n[1] = 4;
        k.n[2] = dim == 3 ? 4 : 1;
        double ext = 0.0;
        for (int a = 0; a < dim; ++a) ext = fmax(ext, bmax[a] - bmin[a]);
        if (!(ext > 0.0)) ext = 1.0;
        for (int a = 0; a < 3; ++a) {
            k.lo[a] = a < dim ? bmin[a] : 0.0;
            k.hi[a] = a < dim ? bmin[a] + ext : 0.0;
        }
        k.precision = mc->precision;
        slr_ctx* c0 = nullptr;
        slr_status s = slr_create(&k, alloc, cuda_stream, &c0);
        if (s == SLR_OK) s = slr_load_cloud(c0, xyz, n_points);
        if (s == SLR_OK) s = slr_cloud_spacing(c0, sample.data(), (int64_t)sample.size(), &hs);
        if (c0) slr_destroy(c0);
        if (s != SLR_OK) return s;
        if (!(hs > 0.0)) return SLR_E_INVALID;  // every sampled point has a duplicate
    }
    rep.h_s = hs;
    rep.sample_size = (int64_t)sample.size();
    // the box of run r: the cloud's bounding box widened by 8 Δx(r), plus
    // γ_S in the first run; Δx(1) = h_S coarsened until the first grid fits
    auto nodes_for = [&](double dx, double margin, long long nn[3]) {
        double tot = 1.0;
        for (int a = 0; a < 3; ++a) nn[a] = 1;
        for (int a = 0; a < dim; ++a) {
            // clamped far above any grid slr_create accepts, so that the
            // conversion and the product stay finite for any cloud extent
            const double q = fmin(ceil(((bmax[a] - bmin[a]) + 2.0 * margin) / dx) + 1.0, 4e9);
            nn[a] = q < 8.0 ? 8 : (long long)q;
            tot *= (double)nn[a];
        }
        return tot;
    };
    double dx1 = hs;
    {
        long long nn[3];
        for (int it = 0; it < 200; ++it) {
            const double tot = nodes_for(dx1, (mc->K_s + 8.0) * dx1, nn);
            if (tot <= (double)mc->max_nodes) break;
            dx1 *= pow(tot / (double)mc->max_nodes, 1.0 / dim) * 1.0001;
        }
    }
    if (dx1 > hs * 1.000001) rep.coarsened = 1;
    // γ_S = K_S h_S; on a coarsened first grid K_S Δx(1), so that the nodes
    // within γ_S of the cloud still form a closed shell for the marking
    const double gamma_s = mc->K_s * dx1;
    std::vector<double> e2buf((size_t)mc->max_iters + 2);
    slr_ctx* prev = nullptr;
    slr_status status = SLR_OK;
    for (int r = 1; r <= mc->runs && status == SLR_OK; ++r) {
        double dx = dx1 / (double)(1ll << (r - 1));
        long long nn[3];
        for (int it = 0; it < 200; ++it) {
            const double tot = nodes_for(dx, 8.0 * dx + (r == 1 ? gamma_s : 0.0), nn);
            if (tot <= (double)mc->max_nodes) break;
            dx *= pow(tot / (double)mc->max_nodes, 1.0 / dim) * 1.0001;
        }
        if (dx > dx1 / (double)(1ll << (r - 1)) * 1.000001) rep.coarsened = 1;
        const double margin = 8.0 * dx + (r == 1 ? gamma_s : 0.0);
        double lo[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) lo[a] = bmin[a] - margin;
        slr_config k;
        slr_config_default(&k);
        k.dim = dim;
        for (int a = 0; a < 3; ++a) {
            k.n[a] = a < dim ? nn[a] : 1;
            k.lo[a] = a < dim ? lo[a] : 0.0;
            k.hi[a] = a < dim ? lo[a] + (double)(nn[a] - 1) * dx : 0.0;
        }
        k.precision = mc->precision;
        k.interp = mc->interp;
        k.band = 1;
        k.reinit = 1;
        k.p = r == 1 ? 1.0 : 2.0;     // Tab. param
        k.delta = r <= 2 ? 0.0 : 1.0;
        k.max_iters = mc->max_iters;
        slr_ctx* c = nullptr;
        status = slr_create(&k, alloc, cuda_stream, &c);
        if (status == SLR_OK) status = slr_load_cloud(c, xyz, n_points);
        if (status == SLR_OK) status = mc->distance_fsm ? slr_build_distance_fsm(c) : slr_build_distance(c);
        if (status == SLR_OK) {
            if (r == 1) {
                const double prm[4] = {gamma_s, 0, 0, 0};
                status = slr_init_u(c, 2, prm, nullptr);
            } else {
                // previous steady state at the new nodes (Q1), then the array path
                double* tmp = (double*)dev_alloc(c, sizeof(double) * (size_t)c->N);
                if (!tmp) {
                    status = SLR_E_NOMEM;
                } else {
                    int cur = 0;
                    cudaError_t e = cudaMemcpyAsync(&cur, &prev->ds->n, sizeof(int), cudaMemcpyDeviceToHost, prev->stream);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(prev->stream);
                    const GridGeom C = geom_of(prev->cfg), F = geom_of(c->cfg);
                    const int grid = c->num_sms * 8;
                    if (e == cudaSuccess) {
                        if (mc->precision == 32)
                            k_resample_q1<float><<<grid, 256, 0, c->stream>>>((const float*)prev->u[cur & 1], C, F, tmp, c->N);
                        else
                            k_resample_q1<double><<<grid, 256, 0, c->stream>>>((const double*)prev->u[cur & 1], C, F, tmp, c->N);
                        c->launches += 1;
                        e = cudaGetLastError();
                    }
                    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
                    if (e == cudaSuccess) {
                        cudaError_t e2 = launch_init_u(c, 1, nullptr, tmp);
                        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(c->stream);
                        status = init_after_u(c, e2);
                    } else {
                        status = SLR_E_CUDA;
                    }
                    dev_free(c, tmp);
                }
            }
        }
        int iters = 0, conv = 0;
        if (status == SLR_OK) status = slr_evolve(c, &iters, &conv);
        if (status == SLR_OK) {
            rep.runs_done = r;
            rep.run_dx[r - 1] = dx;
            for (int a = 0; a < 3; ++a) rep.run_n[r - 1][a] = k.n[a];
            rep.run_iters[r - 1] = iters;
            rep.run_converged[r - 1] = conv;
            for (int a = 0; a < 3; ++a) rep.run_lo[r - 1][a] = k.lo[a];
            int nit = 0;
            double errc = 0.0;
            status = slr_diagnostics(c, e2buf.data(), nullptr, nullptr, (int)e2buf.size(), &nit, &errc);
            if (status == SLR_OK) {
                rep.run_energy[r - 1] = e2buf[nit < (int)e2buf.size() ? nit : (int)e2buf.size() - 1];
                rep.run_err_cloud[r - 1] = errc;
                rep.run_l1_err[r - 1] = NAN;
                if (mc->exact_sphere) status = slr_l1_error(c, 0, mc->sphere, nullptr, &rep.run_l1_err[r - 1]);
            }
        }
        if (prev) slr_destroy(prev);
        prev = c;
        if (status != SLR_OK) {
            if (c) slr_destroy(c);
            prev = nullptr;
        }
    }
    if (report) *report = rep;
    if (status != SLR_OK) return status;
    *out = prev;
    return SLR_OK;
}

}  // extern "C"
