// §3.6 initial data from the distance field: external marking, then the
// fast sweeping method of Zhao (2005) on the internal nodes, whose sign is
// then reversed. The result is an FP64 field that slr_init_u passes through
// the array path (storage type, eq. cut in band mode).
//
// §3.4 distance grid as the paper builds it (build_distance_fsm): the exact
// distance on the nodes of a box of 4 grid points per axis around each point
// of the cloud, the same fast sweeping on every other node (started at +inf),
// in FP64, rounded to the storage type at the end. argmin is -1 off the boxes.
//
// Readings (the paper describes the steps in words):
//  - every node on the grid boundary is external; then one round of
//    directional sweeps along the grid lines, +x, -x, +y, -y (+z, -z): a sweep
//    in direction +x visits each line in increasing x and marks a node
//    external when the node before it is external and its own d >= γ_S;
//  - φ0 = d - γ_S on external nodes, 1e30 on the others;
//  - fast sweeping on the internal nodes: Gauss-Seidel sweeps in the 2^dim
//    orderings (bit a of the ordering set = axis a decreasing), two rounds,
//    with Godunov's local solution of |∇φ| = 1 and φ_j = min(φ_j, x);
//  - finally φ0 = -φ on the internal nodes.
//
// A sweep in one ordering visits the nodes plane by plane, ii + jj + kk = s
// in the ordering's own coordinates: every upwind neighbour of a node lies on
// an earlier plane and every downwind neighbour on a later one, as in the
// lexicographic order, so the values (and the result) are the same; the nodes
// of one plane are independent and run in parallel. The local solver uses
// explicitly rounded FP64 operations in the order of its definition.
#include "slr_internal.cuh"

namespace slr {

namespace {

constexpr int kIB = 256;

__global__ void k_mark_boundary(unsigned char* ext, int n0, int n1, int n2, int dim, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += stride) {
        const int i = (int)(j % n0);
        const long long q = j / n0;
        const int y = (int)(q % n1), z = (int)(q / n1);
        bool b = i == 0 || i == n0 - 1 || y == 0 || y == n1 - 1;
        if (dim == 3) b = b || z == 0 || z == n2 - 1;
        ext[j] = b ? 1 : 0;
    }
}

// one directional sweep along axis `ax` (dir 0 increasing, 1 decreasing):
// one thread per grid line
template <typename T>
__global__ void k_mark_sweep(unsigned char* ext, const T* __restrict__ d, double gamma_s, int ax, int dir, int n0,
                             int n1, int n2) {
    const int n[3] = {n0, n1, n2};
    const long long st[3] = {1, (long long)n0, (long long)n0 * n1};
    const int o1 = (ax + 1) % 3, o2 = (ax + 2) % 3;
    const long long lines = (long long)n[o1] * n[o2];
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < lines; l += stride) {
        const int q1 = (int)(l % n[o1]), q2 = (int)(l / n[o1]);
        const long long base = q1 * st[o1] + q2 * st[o2];
        unsigned char prev = ext[base + (long long)(dir == 0 ? 0 : n[ax] - 1) * st[ax]];
        for (int t = 1; t < n[ax]; ++t) {
            const long long ic = base + (long long)(dir == 0 ? t : n[ax] - 1 - t) * st[ax];
            unsigned char e = ext[ic];
            if (!e && prev && (double)d[ic] >= gamma_s) {
                e = 1;
                ext[ic] = 1;
            }
            prev = e;
        }
    }
}

template <typename T>
__global__ void k_phi_start(double* phi, const unsigned char* __restrict__ ext, const T* __restrict__ d,
                            double gamma_s, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += stride)
        phi[j] = ext[j] ? __dsub_rn((double)d[j], gamma_s) : 1e30;
}

// Godunov local solution from the per-axis upwind values a[0..m)
__device__ double fsm_solve(double a0, double a1, double a2, int m, double h) {
    double a[3] = {a0, a1, a2};
    for (int i = 1; i < m; ++i)
        for (int j = i; j > 0 && a[j] < a[j - 1]; --j) {
            const double t = a[j];
            a[j] = a[j - 1];
            a[j - 1] = t;
        }
    double x = __dadd_rn(a[0], h);
    if (m > 1 && x > a[1]) {
        const double df = __dsub_rn(a[0], a[1]);
        const double r = __dsub_rn(__dmul_rn(__dmul_rn(2.0, h), h), __dmul_rn(df, df));
        x = __ddiv_rn(__dadd_rn(__dadd_rn(a[0], a[1]), __dsqrt_rn(r)), 2.0);
        if (m > 2 && x > a[2]) {
            const double sm = __dadd_rn(__dadd_rn(a[0], a[1]), a[2]);
            const double q = __dsub_rn(
                __dadd_rn(__dadd_rn(__dmul_rn(a[0], a[0]), __dmul_rn(a[1], a[1])), __dmul_rn(a[2], a[2])),
                __dmul_rn(h, h));
            const double r3 = __dsub_rn(__dmul_rn(sm, sm), __dmul_rn(3.0, q));
            x = __ddiv_rn(__dadd_rn(sm, __dsqrt_rn(r3)), 3.0);
        }
    }
    return x;
}

// the nodes of plane s (ii + jj + kk = s) of ordering `ord`
template <int DIM>
__global__ void k_fsm_plane(double* phi, const unsigned char* __restrict__ ext, int ord, int s, int n0, int n1,
                            int n2, double h) {
    const long long st1 = n0, st2 = (long long)n0 * n1;
    const long long count = DIM == 3 ? (long long)n1 * n2 : (long long)n1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
        const int jj = (int)(t % n1), kk = DIM == 3 ? (int)(t / n1) : 0;
        const int ii = s - jj - kk;
        if (ii < 0 || ii >= n0) continue;
        const int c0 = (ord & 1) ? n0 - 1 - ii : ii;
        const int c1 = (ord & 2) ? n1 - 1 - jj : jj;
        const int c2 = (ord & 4) ? n2 - 1 - kk : kk;
        const long long idx = c0 + st1 * c1 + st2 * c2;
        if (ext[idx]) continue;
        const double inf = __longlong_as_double(0x7ff0000000000000ll);
        double a[3];
        {
            const double lo = c0 > 0 ? phi[idx - 1] : inf, hi = c0 < n0 - 1 ? phi[idx + 1] : inf;
            a[0] = lo < hi ? lo : hi;
        }
        {
            const double lo = c1 > 0 ? phi[idx - st1] : inf, hi = c1 < n1 - 1 ? phi[idx + st1] : inf;
            a[1] = lo < hi ? lo : hi;
        }
        if (DIM == 3) {
            const double lo = c2 > 0 ? phi[idx - st2] : inf, hi = c2 < n2 - 1 ? phi[idx + st2] : inf;
            a[2] = lo < hi ? lo : hi;
        } else {
            a[2] = inf;
        }
        const double x = fsm_solve(a[0], a[1], a[2], DIM, h);
        if (x < phi[idx]) phi[idx] = x;
    }
}

// every plane of every ordering of both rounds in one cooperative launch:
// the blocks cross from one plane to the next through a grid-wide barrier;
// neighbour values come through L2 (__ldcg), where the previous plane's
// writes of the other blocks are visible after the barrier
template <int DIM>
__global__ void __launch_bounds__(kIB) k_fsm_coop(double* phi, const unsigned char* __restrict__ fixed, int n0,
                                                  int n1, int n2, double h, unsigned* bar, int* err) {
    const long long st1 = n0, st2 = (long long)n0 * n1;
    const long long count = DIM == 3 ? (long long)n1 * n2 : (long long)n1;
    const int planes = n0 + n1 + (DIM == 3 ? n2 : 1) - 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    for (int round = 0; round < 2; ++round)
        for (int ord = 0; ord < (1 << DIM); ++ord)
            for (int s = 0; s < planes; ++s) {
                for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
                    const int jj = (int)(t % n1), kk = DIM == 3 ? (int)(t / n1) : 0;
                    const int ii = s - jj - kk;
                    if (ii < 0 || ii >= n0) continue;
                    const int c0 = (ord & 1) ? n0 - 1 - ii : ii;
                    const int c1 = (ord & 2) ? n1 - 1 - jj : jj;
                    const int c2 = (ord & 4) ? n2 - 1 - kk : kk;
                    const long long idx = c0 + st1 * c1 + st2 * c2;
                    if (fixed[idx]) continue;
                    double a[3];
                    {
                        const double lo = c0 > 0 ? __ldcg(phi + idx - 1) : inf;
                        const double hi = c0 < n0 - 1 ? __ldcg(phi + idx + 1) : inf;
                        a[0] = lo < hi ? lo : hi;
                    }
                    {
                        const double lo = c1 > 0 ? __ldcg(phi + idx - st1) : inf;
                        const double hi = c1 < n1 - 1 ? __ldcg(phi + idx + st1) : inf;
                        a[1] = lo < hi ? lo : hi;
                    }
                    if (DIM == 3) {
                        const double lo = c2 > 0 ? __ldcg(phi + idx - st2) : inf;
                        const double hi = c2 < n2 - 1 ? __ldcg(phi + idx + st2) : inf;
                        a[2] = lo < hi ? lo : hi;
                    } else {
                        a[2] = inf;
                    }
                    const double x = fsm_solve(a[0], a[1], a[2], DIM, h);
                    if (x < __ldcg(phi + idx)) __stcg(phi + idx, x);
                }
                if (!grid_barrier(bar, err)) return;
            }
}

__global__ void k_phi_finish(double* phi, const unsigned char* __restrict__ ext, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += stride)
        if (!ext[j]) phi[j] = -phi[j];
}

// two rounds of Gauss-Seidel sweeps in the 2^dim orderings over the nodes
// that are not fixed: one cooperative launch with a grid barrier between
// planes where the device supports it (bar: two zeroed words, err: one
// zeroed word, both device memory), else one launch per plane
cudaError_t fsm_sweeps(slr_ctx* c, double* phi, const unsigned char* fixed, unsigned* bar, int* err) {
    const int n0 = (int)c->cfg.n[0], n1 = (int)c->cfg.n[1], n2 = c->cfg.dim == 3 ? (int)c->cfg.n[2] : 1;
    const int dim = c->cfg.dim;
    const int grid = c->num_sms * 8;
    const long long count = dim == 3 ? (long long)n1 * n2 : (long long)n1;
    const int pgrid = (int)((count + kIB - 1) / kIB < grid ? (count + kIB - 1) / kIB : grid);
    const int planes = n0 + n1 + (dim == 3 ? n2 : 1) - 2;
    int coop = 0, per_sm = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device);
    if (coop) {
        cudaError_t e = dim == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fsm_coop<3>, kIB, 0)
                                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fsm_coop<2>, kIB, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            per_sm = 0;
        }
    }
    if (coop && per_sm > 0) {
        const long long cap = (long long)c->num_sms * per_sm;
        const int cgrid = (int)(cap < (count + kIB - 1) / kIB ? cap : (count + kIB - 1) / kIB);
        double h = c->h;
        void* args[] = {&phi, (void*)&fixed, (void*)&n0, (void*)&n1, (void*)&n2, &h, &bar, &err};
        cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), c->stream);
        if (e == cudaSuccess)
            e = cudaLaunchCooperativeKernel(dim == 3 ? (const void*)k_fsm_coop<3> : (const void*)k_fsm_coop<2>,
                                            dim3(cgrid), dim3(kIB), args, 0, c->stream);
        c->launches += 1;
        return e;
    }
    for (int round = 0; round < 2; ++round)
        for (int ord = 0; ord < (1 << dim); ++ord)
            for (int s = 0; s < planes; ++s) {
                if (dim == 3)
                    k_fsm_plane<3><<<pgrid, kIB, 0, c->stream>>>(phi, fixed, ord, s, n0, n1, n2, c->h);
                else
                    k_fsm_plane<2><<<pgrid, kIB, 0, c->stream>>>(phi, fixed, ord, s, n0, n1, n2, c->h);
            }
    c->launches += 2ll * (1 << dim) * planes;
    return cudaGetLastError();
}

// the sweeps with their barrier words and error word in a small scratch;
// a barrier that waited too long reports cudaErrorLaunchTimeout
cudaError_t sweeps_checked(slr_ctx* c, double* phi, const unsigned char* fixed) {
    void* base = dev_alloc(c, 256);
    if (!base) return cudaErrorMemoryAllocation;
    unsigned* bar = (unsigned*)base;
    int* err = (int*)((char*)base + 64);
    int herr = 0;
    cudaError_t e = fsm_sweeps(c, phi, fixed, bar, err);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, base);
    if (e == cudaSuccess && herr) e = cudaErrorLaunchTimeout;
    return e;
}

struct GridBox {
    double lo[3];
    double h;
    int n[3];
};

template <typename T>
cudaError_t marking_t(slr_ctx* c, double gamma_s, double* phi, unsigned char* ext) {
    const int n0 = (int)c->cfg.n[0], n1 = (int)c->cfg.n[1], n2 = c->cfg.dim == 3 ? (int)c->cfg.n[2] : 1;
    const int dim = c->cfg.dim;
    const int grid = c->num_sms * 8;
    const T* d = (const T*)c->d;
    k_mark_boundary<<<grid, kIB, 0, c->stream>>>(ext, n0, n1, n2, dim, c->N);
    long long launches = 1;
    for (int ax = 0; ax < dim; ++ax)
        for (int dir = 0; dir < 2; ++dir) {
            k_mark_sweep<T><<<grid, kIB, 0, c->stream>>>(ext, d, gamma_s, ax, dir, n0, n1, n2);
            ++launches;
        }
    k_phi_start<T><<<grid, kIB, 0, c->stream>>>(phi, ext, d, gamma_s, c->N);
    ++launches;
    c->launches += launches;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = sweeps_checked(c, phi, ext);
    if (e != cudaSuccess) return e;
    k_phi_finish<<<grid, kIB, 0, c->stream>>>(phi, ext, c->N);
    c->launches += 1;
    return cudaGetLastError();
}

// --- §3.4: the distance grid as the paper builds it ---------------------------

// the box of 4 nodes per axis around each point: i0-1 .. i0+2 with
// i0 = floor((Q_a - lo_a)/h), clipped to the grid
__global__ void k_mark_boxes(const double* __restrict__ pts, long long npts, int dim, GridBox G,
                             unsigned char* fixed) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < npts; q += stride) {
        int b0[3] = {0, 0, 0}, b1[3] = {0, 0, 0};
        bool empty = false;
        for (int a = 0; a < dim; ++a) {
            const double xi = floor(__ddiv_rn(__dsub_rn(pts[q * dim + a], G.lo[a]), G.h));
            if (!isfinite(xi)) {
                empty = true;
                break;
            }
            double l = xi - 1.0, u = xi + 2.0;
            if (l < 0.0) l = 0.0;
            if (u > (double)(G.n[a] - 1)) u = (double)(G.n[a] - 1);
            if (l > u) {
                empty = true;
                break;
            }
            b0[a] = (int)l;
            b1[a] = (int)u;
        }
        if (empty) continue;
        const long long s1 = G.n[0], s2 = (long long)G.n[0] * G.n[1];
        for (int k = b0[2]; k <= b1[2]; ++k)
            for (int j = b0[1]; j <= b1[1]; ++j)
                for (int i = b0[0]; i <= b1[0]; ++i) fixed[i + s1 * j + s2 * k] = 1;
    }
}

__global__ void k_count_fixed(const unsigned char* __restrict__ fixed, long long N, unsigned long long* count) {
    __shared__ unsigned long long s_sum[kIB / 32];
    unsigned long long v = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += stride) v += fixed[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kIB / 32; ++w) t += s_sum[w];
        atomicAdd(count, t);
    }
}

__global__ void k_fill_inf(double* v, long long N) {
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += stride) v[j] = inf;
}

template <typename T>
__global__ void k_store_rounded(const double* __restrict__ v, T* out, long long N) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += stride) out[j] = (T)v[j];
}

}  // namespace

cudaError_t build_distance_fsm(slr_ctx* c) {
    const long long N = c->N;
    const int grid = c->num_sms * 8;
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    char* base = (char*)dev_alloc(c, al(sizeof(double) * N) + al(N) + 256);
    if (!base) return cudaErrorMemoryAllocation;
    double* dv = (double*)base;
    unsigned char* fixed = (unsigned char*)(base + al(sizeof(double) * N));
    unsigned long long* count = (unsigned long long*)(base + al(sizeof(double) * N) + al(N));
    GridBox G;
    for (int a = 0; a < 3; ++a) {
        G.lo[a] = a < c->cfg.dim ? c->cfg.lo[a] : 0.0;
        G.n[a] = (int)c->cfg.n[a];
    }
    G.h = c->h;
    unsigned long long hcount = 0;
    cudaError_t e = cudaMemsetAsync(fixed, 0, (size_t)N, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) {
        const long long pb = (c->npts + kIB - 1) / kIB;
        k_mark_boxes<<<(unsigned)(pb < grid ? pb : grid), kIB, 0, c->stream>>>(c->pts, c->npts, c->cfg.dim, G, fixed);
        k_count_fixed<<<grid, kIB, 0, c->stream>>>(fixed, N, count);
        k_fill_inf<<<grid, kIB, 0, c->stream>>>(dv, N);
        c->launches += 3;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(c->argmin, 0xff, sizeof(int) * (size_t)N, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&hcount, count, sizeof(hcount), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess && hcount == 0) e = cudaErrorInvalidValue;
    if (e == cudaSuccess) e = distance_on_marked(c, fixed, dv);
    if (e == cudaSuccess) e = sweeps_checked(c, dv, fixed);
    if (e == cudaSuccess) {
        if (c->cfg.precision == 32)
            k_store_rounded<float><<<grid, kIB, 0, c->stream>>>(dv, (float*)c->d, N);
        else
            k_store_rounded<double><<<grid, kIB, 0, c->stream>>>(dv, (double*)c->d, N);
        c->launches += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, base);
    return e;
}

// the bounded grid barrier on its own: a barrier that one block cannot
// complete (the arrival count starting at the grid size) makes every wait run
// out, which the caller reads back from err
__global__ void k_barrier_check(unsigned* bar, int* err) { grid_barrier(bar, err); }

cudaError_t barrier_selftest(int device, int unreachable, int* err_out) {
    void* base = nullptr;
    cudaError_t e = cudaMalloc(&base, 256);
    if (e != cudaSuccess) return e;
    unsigned* bar = (unsigned*)base;
    int* err = (int*)((char*)base + 64);
    const unsigned grid = 2;
    unsigned init[2] = {unreachable ? grid : 0u, 0u};
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    e = coop ? cudaSuccess : cudaErrorNotSupported;
    if (e == cudaSuccess) e = cudaMemcpy(bar, init, sizeof(init), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        void* args[] = {&bar, &err};
        e = cudaLaunchCooperativeKernel((const void*)k_barrier_check, dim3(grid), dim3(32), args, 0, 0);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(err_out, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(base);
    return e;
}

cudaError_t launch_init_marking(slr_ctx* c, double gamma_s, double* phi_dev, unsigned char* ext_dev) {
    return c->cfg.precision == 32 ? marking_t<float>(c, gamma_s, phi_dev, ext_dev)
                                  : marking_t<double>(c, gamma_s, phi_dev, ext_dev);
}

}  // namespace slr
