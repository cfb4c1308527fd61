// The batched persistent kernel (slr_batch.cuh) for float storage. Fields
// written by other blocks earlier in the same launch are read with coherent
// loads, so ld() is the plain cached load here.
#define SLR_COHERENT_LOADS 1
#include "slr_batch.cuh"

namespace slr {

slr_status batch_run_f32(slr_ctx* const* jobs, int n, int tune, cudaStream_t st, int* shape_io, int* graph_out,
                         float* tuned_ms, int* threads, int* blocks, int* bpi) {
    return batch_run_group<float>(jobs, n, tune, st, shape_io, graph_out, tuned_ms, threads, blocks, bpi);
}

// the batched kernel's dependency wait alone, on a counter that nothing
// completes: *err_out receives the error bits (kErrBarrier once it ran out)
cudaError_t batch_wait_selftest(int* err_out) {
    int* words = nullptr;
    cudaError_t e = cudaMalloc((void**)&words, 3 * sizeof(int));
    if (e != cudaSuccess) return e;
    e = cudaMemset(words, 0, 3 * sizeof(int));  // counter 0, stop flag 0, error bits 0
    if (e == cudaSuccess) {
        k_batch_wait_selftest<<<1, 32>>>(words, words + 2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(err_out, words + 2, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(words);
    return e;
}

}  // namespace slr
