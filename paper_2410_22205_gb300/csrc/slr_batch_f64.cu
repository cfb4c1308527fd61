// The batched persistent kernel (slr_batch.cuh) for double storage. Fields
// written by other blocks earlier in the same launch are read with coherent
// loads, so ld() is the plain cached load here.
#define SLR_COHERENT_LOADS 1
#include "slr_batch.cuh"

namespace slr {

slr_status batch_run_f64(slr_ctx* const* jobs, int n, int tune, cudaStream_t st, int* shape_io, int* graph_out,
                         float* tuned_ms, int* threads, int* blocks, int* bpi) {
    return batch_run_group<double>(jobs, n, tune, st, shape_io, graph_out, tuned_ms, threads, blocks, bpi);
}

}  // namespace slr
