// Small utility kernels: exclusive scan of block counts, type conversions,
// and allocation through the context's allocator.
#include "slr_compact.cuh"
#include "slr_internal.cuh"

namespace slr {

void* dev_alloc(slr_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (c->default_alloc) {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    return c->al.alloc(bytes, c->al.user);
}

void dev_free(slr_ctx* c, void* p) {
    if (!p) return;
    if (c->default_alloc)
        cudaFree(p);
    else
        c->al.free(p, c->al.user);
}

// single block of 1024 threads; nb <= 4 * 1024
__global__ void __launch_bounds__(1024) k_scan_counts(int* counts, int nb, long long* total) {
    __shared__ long long s[1024];
    const int per = (nb + 1023) / 1024;
    const int beg = threadIdx.x * per;
    long long local = 0;
    for (int i = 0; i < per; ++i)
        if (beg + i < nb) local += counts[beg + i];
    s[threadIdx.x] = local;
    __syncthreads();
    // Hillis-Steele inclusive scan over the 1024 thread sums
    for (int off = 1; off < 1024; off <<= 1) {
        long long v = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    long long run = threadIdx.x ? s[threadIdx.x - 1] : 0;
    for (int i = 0; i < per; ++i)
        if (beg + i < nb) {
            int c = counts[beg + i];
            counts[beg + i] = (int)run;
            run += c;
        }
    if (threadIdx.x == 1023) *total = s[1023];
}

template <typename T>
__global__ void k_to_double(const T* src, double* dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

template <typename T>
__global__ void k_from_double(const double* src, T* dst, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (T)src[i];
}

// per job: stop flag, iteration count, converged flag, error bits
__global__ void k_gather_status(DevState* const* states, int n, int* out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const DevState* s = states[j];
    out[4 * j + 0] = s->stop;
    out[4 * j + 1] = s->n;
    out[4 * j + 2] = s->converged;
    out[4 * j + 3] = s->error;
}

cudaError_t launch_gather_status(slr_ctx* c, DevState* const* states, int n, int* out, cudaStream_t st) {
    k_gather_status<<<(n + 127) / 128, 128, 0, st>>>(states, n, out);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_to_double(slr_ctx* c, const void* src, double* dst, long long n) {
    int blocks = c->num_sms * 8;
    if (c->cfg.precision == 32)
        k_to_double<float><<<blocks, 256, 0, c->stream>>>((const float*)src, dst, n);
    else
        k_to_double<double><<<blocks, 256, 0, c->stream>>>((const double*)src, dst, n);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_from_double(slr_ctx* c, const double* src, void* dst, long long n) {
    int blocks = c->num_sms * 8;
    if (c->cfg.precision == 32)
        k_from_double<float><<<blocks, 256, 0, c->stream>>>(src, (float*)dst, n);
    else
        k_from_double<double><<<blocks, 256, 0, c->stream>>>(src, (double*)dst, n);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace slr
