// Small utility kernels: exclusive scan of block counts, type conversions,
// and allocation through the context's allocator.
#include <mutex>

#include "slr_compact.cuh"
#include "slr_internal.cuh"

namespace slr {

// Without an injected allocator, memory comes from the library's own
// stream-ordered pool on the context's stream (cudaMallocFromPoolAsync /
// cudaFreeAsync): neither call waits for the device, so contexts set up from
// several threads (the server) do not stall behind each other's work the way
// cudaFree does. One pool per device, created on first use, keeps freed
// memory for reuse (release threshold: unlimited), as a caching allocator
// would; the process's default pool is left as it is. Everything a context
// allocates is used on its own stream, or after that stream was
// synchronised. Devices without memory pools use cudaMalloc / cudaFree.
namespace {
constexpr int kPoolDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pool[kPoolDevices] = {};
bool g_pool_tried[kPoolDevices] = {};

cudaMemPool_t pool_of(int device) {
    if (device < 0 || device >= kPoolDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    if (!g_pool_tried[device]) {
        g_pool_tried[device] = true;
        int ok = 0;
        if (cudaDeviceGetAttribute(&ok, cudaDevAttrMemoryPoolsSupported, device) == cudaSuccess && ok) {
            cudaMemPoolProps pr = {};
            pr.allocType = cudaMemAllocationTypePinned;
            pr.location.type = cudaMemLocationTypeDevice;
            pr.location.id = device;
            cudaMemPool_t mp = nullptr;
            if (cudaMemPoolCreate(&mp, &pr) == cudaSuccess) {
                unsigned long long thr = ~0ull;
                cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr);
                g_pool[device] = mp;
            }
        }
        cudaGetLastError();
    }
    return g_pool[device];
}
}  // namespace

void* dev_alloc(slr_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (c->default_alloc) {
        void* p = nullptr;
        cudaMemPool_t mp = pool_of(c->device);
        const cudaError_t e = mp ? cudaMallocFromPoolAsync(&p, bytes, mp, c->stream) : cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return p;
    }
    return c->al.alloc(bytes, c->al.user);
}

void dev_free(slr_ctx* c, void* p) {
    if (!p) return;
    if (c->default_alloc) {
        if (pool_of(c->device))
            cudaFreeAsync(p, c->stream);
        else
            cudaFree(p);
    } else {
        c->al.free(p, c->al.user);
    }
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

// ---------------------------------------------------------------------------
// FMA throughput probe (the paper has no counterpart): the ALU roofline of the
// WENO step divides by the device's measured FP32 FMA rate. Every thread runs
// 8 independent FMA chains (enough to cover the FMA latency with 8 warps per
// scheduler), 64 FMAs per loop trip; the result is stored only when it takes
// a value it never takes, so the work cannot be removed.
// ---------------------------------------------------------------------------
namespace slr {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* out, long long trips, T a, T b) {
    T x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x & 31) * T(1e-3) + (T)i;
    for (long long t = 0; t < trips; ++t) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == T(-1.25e30)) out[blockIdx.x] = s;
}

template <typename T>
cudaError_t probe_t(long long trips, double* tflops, double* ms_out) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int blocks = sms * 8;
    T* out = nullptr;
    e = cudaMalloc(&out, sizeof(T) * blocks);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    const T a = T(0.9999999), b = T(1e-7);
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
        e = cudaEventRecord(e0, 0);
        if (e == cudaSuccess) {
            k_fma_probe<T><<<blocks, 256>>>(out, trips, a, b);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return e;
    const double flops = 2.0 * 64.0 * (double)trips * 256.0 * (double)blocks;
    *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    *ms_out = ms;
    return cudaSuccess;
}

}  // namespace
}  // namespace slr

extern "C" slr_status slr_probe_fma(int precision, int64_t trips, double* tflops_out, double* ms_out) {
    using namespace slr;
    if ((precision != 32 && precision != 64) || trips < 1 || !tflops_out || !ms_out) return SLR_E_INVALID;
    cudaError_t e = precision == 32 ? probe_t<float>(trips, tflops_out, ms_out)
                                    : probe_t<double>(trips, tflops_out, ms_out);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? SLR_E_NOMEM : SLR_E_CUDA;
    }
    return SLR_OK;
}
