// Ordered stream compaction used outside the per-step path (initial band,
// energy candidate cells, extract). Two passes over a fixed block/chunk
// partition: count per block, exclusive scan of the block counts in one
// block, then each block re-evaluates its predicate and writes its survivors
// in index order. Deterministic and free of inter-block waits.
#pragma once

#include "slr_internal.cuh"

namespace slr {

constexpr int kCompactBlock = 256;

struct CompactPlan {
    long long M = 0;      // items
    long long chunk = 0;  // items per block (multiple of kCompactBlock)
    int blocks = 0;
};

inline CompactPlan make_plan(long long M) {
    CompactPlan p;
    p.M = M;
    long long nb = (M + kCompactBlock - 1) / kCompactBlock;
    if (nb > 4096) nb = 4096;
    if (nb < 1) nb = 1;
    long long chunk = (M + nb - 1) / nb;
    chunk = ((chunk + kCompactBlock - 1) / kCompactBlock) * kCompactBlock;
    if (chunk < kCompactBlock) chunk = kCompactBlock;
    p.chunk = chunk;
    p.blocks = (int)((M + chunk - 1) / chunk);
    if (p.blocks < 1) p.blocks = 1;
    return p;
}

template <typename Pred>
__global__ void __launch_bounds__(kCompactBlock) k_compact_count(Pred pred, long long M, long long chunk,
                                                                 int* block_counts) {
    __shared__ int s_warp[kCompactBlock / 32 + 1];
    long long beg = (long long)blockIdx.x * chunk;
    long long end = beg + chunk < M ? beg + chunk : M;
    int local = 0;
    for (long long i = beg + threadIdx.x; i < end; i += kCompactBlock) local += pred(i) ? 1 : 0;
    local = warp_sum(local);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = local;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kCompactBlock / 32; ++w) t += s_warp[w];
        block_counts[blockIdx.x] = t;
    }
}

// exclusive scan of nb block counts in place; total written to *total
__global__ void k_scan_counts(int* counts, int nb, long long* total);

template <typename Pred, typename Emit>
__global__ void __launch_bounds__(kCompactBlock) k_compact_write(Pred pred, Emit emit, long long M, long long chunk,
                                                                 const int* block_offsets) {
    __shared__ int s_warp[kCompactBlock / 32 + 1];
    long long beg = (long long)blockIdx.x * chunk;
    long long end = beg + chunk < M ? beg + chunk : M;
    long long base = block_offsets[blockIdx.x];
    for (long long t0 = beg; t0 < end; t0 += kCompactBlock) {
        long long i = t0 + threadIdx.x;
        int f = (i < end) && pred(i);
        int total;
        int off = block_exclusive_flag<kCompactBlock>(f, s_warp, &total);
        if (f) emit(base + off, i);
        base += total;
        __syncthreads();
    }
}

// count survivors (host-synchronous readback of the total); scratch is
// allocated from the context allocator and released before returning
template <typename Pred>
cudaError_t compact_count(slr_ctx* c, Pred pred, long long M, long long* count_out) {
    CompactPlan pl = make_plan(M);
    int* counts = (int*)dev_alloc(c, sizeof(int) * (pl.blocks + 2) + sizeof(long long) * 2);
    if (!counts) return cudaErrorMemoryAllocation;
    long long* tot = (long long*)(counts + ((pl.blocks + 1) & ~1));
    k_compact_count<<<pl.blocks, kCompactBlock, 0, c->stream>>>(pred, M, pl.chunk, counts);
    k_scan_counts<<<1, 1024, 0, c->stream>>>(counts, pl.blocks, tot);
    c->launches += 2;
    cudaError_t e = cudaGetLastError();
    long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, tot, sizeof(long long), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, counts);
    *count_out = h;
    return e;
}

template <typename Pred, typename Emit>
cudaError_t compact_write(slr_ctx* c, Pred pred, Emit emit, long long M) {
    CompactPlan pl = make_plan(M);
    int* counts = (int*)dev_alloc(c, sizeof(int) * (pl.blocks + 2) + sizeof(long long) * 2);
    if (!counts) return cudaErrorMemoryAllocation;
    long long* tot = (long long*)(counts + ((pl.blocks + 1) & ~1));
    k_compact_count<<<pl.blocks, kCompactBlock, 0, c->stream>>>(pred, M, pl.chunk, counts);
    k_scan_counts<<<1, 1024, 0, c->stream>>>(counts, pl.blocks, tot);
    k_compact_write<<<pl.blocks, kCompactBlock, 0, c->stream>>>(pred, emit, M, pl.chunk, counts);
    c->launches += 3;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, counts);
    return e;
}

}  // namespace slr
