// Batched evolution of many independent reconstructions in one persistent,
// cooperative, graph-captured kernel (k_batch).
//
// Every job is one run of Algorithm 1's loop (arXiv 2410.22205, §3: the
// band, the SL update of §3.1-§3.2 with the band and cut of §3.8, then the energy
// of §3.5 and the stop test of §4 eq. deltaEn), without the
// reinitialisation. One iteration of a job is three phases of work items:
//   0. step:   one item per bpi active bricks of a 3-D job on the brick
//              step (slr_brick.cuh), or per NT/32 tiles of 128 band-list
//              entries of a job on the list step (slr_step.cuh: 2-D, and 3-D
//              where the step-kind rule picks it);
//   1. energy: one item per slot of 1024 candidate cells, after, for a job on
//              the list step, the items that count its tiles' band members;
//   2. record: kRecordBlocks slices; the block that finishes a job's last
//              slice does its bookkeeping and stop test.
// The items of all jobs form one ticket sequence, iteration by iteration and
// phase by phase (jobs in a fixed order inside a phase), and the blocks of
// the launch take tickets from one counter. An item waits only for its own
// job: a step item for the job's record of the previous iteration, an
// energy item for all of the job's step items, a record item for all of its
// energy items (per-job completion counters). Every wait is on items with
// smaller tickets, taken by blocks that are resident (a cooperative launch),
// so the sequence always advances; jobs are at different phases at the same
// time and no grid-wide barrier exists. A wait gives up after a poll limit
// and reports kErrBarrier, which the host returns as SLR_E_TIMEOUT. Items of
// a job whose stop test has fired are no-ops, and the blocks leave once every
// job has stopped.
//
// The per-item device code is the per-job kernels' own (brick_compute,
// band_tile, energy_slot, tile_count, record_slice), compiled like them
// without implicit FMA contraction and with the reductions' summation trees
// kept, so each job's results are bit-identical to its solo run. Fields that
// other blocks wrote before a wait are read with coherent loads
// (SLR_COHERENT_LOADS, L2 loads of the partials, TMA after a proxy fence).
#pragma once

#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "slr_brick.cuh"
#include "slr_energy.cuh"
#include "slr_internal.cuh"
#include "slr_step.cuh"

namespace slr {

template <typename T>
Params<T> make_params(const slr_ctx* c);

namespace {

constexpr int kBatchMaxJobs = 64;  // jobs per launch (kernel-parameter space)

// per-job data read on every work item: kept in kernel-parameter space
template <typename T>
struct BatchHot {
    Params<T> P;
    BrickArgs<T> A;  // 3-D: active bricks, counts, partials, staging mode
    EnergyArgs<T> E;
    T* ub0;
    T* ub1;
    const T* d;
    DevState* ds;
    const int* cells;   // candidate cells of the energy pass
    long long ncells;
    int nslots;         // slots of 1024 candidate cells
    double* part_e;
    int* L0;            // 2-D: band lists, tile counts/offsets, Δ_φ partials
    int* L1;
    int* tile_off;
    double* part_dphi;
    int band_cap;
    int dim, interp;
    int bricked;        // 3-D brick step; else the list step (2-D, or 3-D by the step-kind rule)
    int ntc;            // list step: tile-count items that open its energy phase
};

template <typename T>
struct BatchParams {
    BatchHot<T> job[kBatchMaxJobs];
    int pre[3][kBatchMaxJobs + 1];  // per phase: prefix over jobs of the items of one iteration
    long long per_iter;             // items of one iteration (all phases)
};
static_assert(sizeof(BatchParams<double>) + 64 <= 32764, "batch parameters fit the kernel-parameter space");

// per-job data read rarely: in global memory (CUtensorMap carries its own alignment)
struct BatchCold {
    CUtensorMap tm[3];  // u buffer 0, u buffer 1, d (3-D jobs staged by TMA)
    RecordArgs rec;
};

struct BatchCtl {
    unsigned long long ticket;     // next work item of the launch
    int err;                       // kErrBarrier / kErrStage
    int pad;
    int step_done[kBatchMaxJobs];  // per job: step items completed in this launch
    int energy_done[kBatchMaxJobs];
    int rec_done[kBatchMaxJobs];   // per job: iterations whose record is complete
};

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_tensormap_acquire(const void* p) {
    asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(p) : "memory");
}
template <typename X>
__device__ __forceinline__ X vload(const X* p) {
    return *(const volatile X*)p;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: wait until *cnt >= need (an acquire load: the counted items'
// writes are visible after it), the job has stopped, or another block
// reported an error; false after the poll limit (kErrBarrier is then set
// for every block to see).
__device__ __forceinline__ bool batch_wait(const int* cnt, int need, const int* stop, int* err) {
    long long polls = 0;
    while (ld_acquire(cnt) < need) {
        if (ld_acquire(stop)) return true;
        if (vload(err) & kErrBarrier) return false;
        if (++polls > kBarrierSpinLimit) {
            atomicOr(err, kErrBarrier);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// item words in shared memory (the brick step's ticket area, 32 bytes)
enum {
    kItJob = 0,  // job of the current item
    kItLoc,      // its index within the job's items of the phase
    kItPhIt,     // phase | iteration << 2 (iteration -1: past the launch's end)
    kItFlags,    // kFlOk: wait passed / staged; kFlStop: the job has stopped; kFlPar: staging parity
    kItKey,      // the last (iteration, phase, job) whose wait this block passed
    kItDone,     // completion to publish for the previous item: step j, energy 64 + j, or -1
    kItTk0,      // two ticket slots: the current ticket and the next one, by turns
    kItTk1
};
enum { kFlOk = 1, kFlStop = 2, kFlPar = 4 };

// One launch shape of the batch kernel: NT threads per block, OCC resident
// blocks per SM asked of the register allocator (80 registers at NT = 128,
// OCC = 6 in FP32; 96 at OCC = 5), and bpi bricks per step item of a 3-D job
// (a run-time argument). Thread 0 decodes the current ticket and waits for
// its dependency while thread 32 publishes the previous item's completion
// and thread 64 takes the next ticket, so the three latencies overlap.
template <typename T, int NT, int OCC>
__global__ void __launch_bounds__(NT, OCC)
    k_batch(const __grid_constant__ BatchParams<T> BP, const BatchCold* __restrict__ cold, BatchCtl* ctl, int njobs,
            int max_iters, int bpi) {
    using S = BrickSmem<T, 1>;
    using G = BoxGeom;
    constexpr int W = NT / 32;
    static_assert(NT >= 96, "three threads in distinct warps run the item bookkeeping");
    static_assert(sizeof(EnergyWs<T>) <= S::kBar && sizeof(RecordWs) <= S::kBar, "workspaces fit the brick area");
    static_assert(kItTk1 < 8, "item words fit the ticket area");
    extern __shared__ __align__(128) unsigned char smem[];
    // [0, kBar): one item's scratch (brick boxes and lists, or the energy or
    // record workspace); kBar: the staging barrier; kTicket: the item words
    T* su = reinterpret_cast<T*>(smem);
    T* sd = reinterpret_cast<T*>(smem + G::BoxN * (int)sizeof(T));
    unsigned short* s_list = reinterpret_cast<unsigned short*>(smem + S::kList);
    T* s_abs = reinterpret_cast<T*>(smem + S::kAbs);
    int* s_cnt = reinterpret_cast<int*>(smem + S::kCnt);
    EnergyWs<T>& ews = *reinterpret_cast<EnergyWs<T>*>(smem);
    RecordWs& rws = *reinterpret_cast<RecordWs*>(smem);
    int* s_it = reinterpret_cast<int*>(smem + S::kTicket);
    const unsigned bar = smem_addr(smem + S::kBar);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        for (int j = 0; j < njobs; ++j)
            if (BP.job[j].bricked && BP.job[j].A.tma)
                for (int m = 0; m < 3; ++m) fence_tensormap_acquire(&cold[j].tm[m]);
        s_it[kItFlags] = 0;
        s_it[kItKey] = -1;
        s_it[kItDone] = -1;
        s_it[kItTk0] = (int)atomicAdd(&ctl->ticket, 1u);
    }
    __syncthreads();
    const unsigned end = (unsigned)max_iters * (unsigned)BP.per_iter;  // the host keeps it below 2^31
    int cur_iter = -1;
    for (int slot = 0;; slot ^= 1) {
        if (tid == 0) {
            // ---- decode the current ticket: iteration, phase, job, index ----
            const unsigned t = (unsigned)s_it[kItTk0 + slot];
            int iter = -1, ph = 0, j = 0, r = 0;
            if (t < end) {
                iter = (int)(t / (unsigned)BP.per_iter);
                r = (int)(t - (unsigned)iter * (unsigned)BP.per_iter);
                if (r >= BP.pre[0][njobs]) {
                    r -= BP.pre[0][njobs];
                    ph = 1;
                    if (r >= BP.pre[1][njobs]) {
                        r -= BP.pre[1][njobs];
                        ph = 2;
                    }
                }
                int lo = 0, hi = njobs;  // pre[ph][lo] <= r < pre[ph][hi]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (BP.pre[ph][mid] <= r)
                        lo = mid;
                    else
                        hi = mid;
                }
                j = lo;
                r -= BP.pre[ph][lo];
                // ---- wait for this job's previous phase (once per iteration,
                // phase and job in a block: the job's stop flag cannot change
                // meanwhile) ----
                const int key = (iter * 3 + ph) * kBatchMaxJobs + j;
                int fl = s_it[kItFlags] & kFlPar;
                if (key == s_it[kItKey]) {
                    fl |= kFlOk | (s_it[kItFlags] & kFlStop);
                } else {
                    const DevState* ds = BP.job[j].ds;
                    bool ok;
                    if (ph == 0)
                        ok = iter == 0 || batch_wait(&ctl->rec_done[j], iter, &ds->stop, &ctl->err);
                    else if (ph == 1)
                        ok = batch_wait(&ctl->step_done[j], (iter + 1) * (BP.pre[0][j + 1] - BP.pre[0][j]),
                                        &ds->stop, &ctl->err);
                    else
                        ok = batch_wait(&ctl->energy_done[j], (iter + 1) * (BP.pre[1][j + 1] - BP.pre[1][j]),
                                        &ds->stop, &ctl->err);
                    fl |= (ok ? kFlOk : 0) | (ld_acquire(&ds->stop) ? kFlStop : 0);
                    s_it[kItKey] = ok ? key : -1;
                }
                s_it[kItFlags] = fl;
            }
            s_it[kItPhIt] = ph | (iter << 2);
            s_it[kItJob] = j;
            s_it[kItLoc] = r;
        } else if (tid == 32) {
            // ---- the previous item's completion: its writes ended at the
            // last block barrier; fence, then count it (release) ----
            const int dn = s_it[kItDone];
            if (dn >= 0) {
                __threadfence();
                atomicAdd(dn < kBatchMaxJobs ? &ctl->step_done[dn] : &ctl->energy_done[dn - kBatchMaxJobs], 1);
                s_it[kItDone] = -1;
            }
        } else if (tid == 64) {
            // ---- the next ticket; it depends on nothing the current item
            // produces (waits point to smaller tickets only) ----
            s_it[kItTk0 + (slot ^ 1)] = (int)atomicAdd(&ctl->ticket, 1u);
        }
        __syncthreads();
        const int phit = s_it[kItPhIt];
        const int iter = phit >> 2;
        if (iter < 0) break;  // past the launch's last iteration
        if (iter != cur_iter) {
            // a new iteration for this block: leave if every job has stopped
            cur_iter = iter;
            if (__syncthreads_and(tid >= njobs || vload(&BP.job[tid].ds->stop) != 0)) break;
        }
        if (!(s_it[kItFlags] & kFlOk)) return;
        const int ph = phit & 3, j = s_it[kItJob], loc = s_it[kItLoc];
        const BatchHot<T>& J = BP.job[j];
        DevState* ds = J.ds;
        if (!(s_it[kItFlags] & kFlStop)) {
            const int n = vload(&ds->n);
            if (ph == 0 && J.bricked) {
                // ---- bpi bricks of a 3-D job ----
                const Params<T>& P = J.P;
                const BrickArgs<T>& A = J.A;
                const int b_end = min((loc + 1) * bpi, A.nbricks);
                for (int bq = loc * bpi; bq < b_end; ++bq) {
                    const int b = __ldg(A.bricks + bq);
                    if (__ldcg(A.bcnt + b) == 0) continue;
                    const T* uin = (n & 1) ? J.ub1 : J.ub0;
                    T* uout = (n & 1) ? J.ub0 : J.ub1;
                    const T Ep = (T)vload(&ds->Ep);
                    const T invEp = Ep > T(0) ? T(1) / Ep : T(0);
                    const int bxi = b % A.nbx, q = b / A.nbx;
                    const int ox = bxi * kBX - kHalo, oy = (q % A.nby) * kBY - kHalo, oz = (q / A.nby) * kBZ - kHalo;
                    if (A.tma) {
                        if (tid == 0) {
                            // the boxes' rows were written through the generic proxy
                            // by other blocks before the wait, and this block's
                            // generic accesses of the scratch area ended at the last
                            // block barrier
                            fence_proxy_async_global();
                            fence_proxy_async();
                            mbar_expect_tx(bar, (unsigned)((G::BoxN + G::DBoxN) * sizeof(T)));
                            tma_load_3d(smem_addr(su), &cold[j].tm[n & 1], bar, ox, oy, oz);
                            tma_load_3d(smem_addr(sd), &cold[j].tm[2], bar, ox, oy + kHalo - 1, oz + kHalo - 1);
                            const int fl = s_it[kItFlags];
                            const unsigned par = (fl & kFlPar) ? 1u : 0u;
                            long long w = 0;
                            while (!mbar_try_wait(bar, par) && ++w < kStageWaitLimit) {
                            }
                            const bool staged = w < kStageWaitLimit;
                            if (!staged) {
                                long long w2 = 0;  // the copies in flight: a second bounded wait
                                while (!mbar_try_wait(bar, par) && ++w2 < kStageWaitLimit) {
                                }
                            }
                            s_it[kItFlags] = ((fl ^ kFlPar) & ~kFlOk) | (staged ? kFlOk : 0);
                        }
                    } else {
                        brick_stage_copy<T, NT, false>(P, uin, J.d, su, sd, ox, oy, oz);
                    }
                    __syncthreads();
                    if (!(s_it[kItFlags] & kFlOk)) {
                        if (tid == 0) {
                            atomicOr(&ds->error, kErrStage);
                            atomicOr(&ctl->err, kErrStage | kErrBarrier);  // the waiting blocks leave
                        }
                        return;
                    }
                    if (J.interp)
                        brick_compute<T, 1, 1, NT>(P, A, su, sd, uin, uout, J.d, ds, Ep, invEp, b, ox, oy, oz,
                                                   s_list, s_abs, s_cnt);
                    else
                        brick_compute<T, 0, 1, NT>(P, A, su, sd, uin, uout, J.d, ds, Ep, invEp, b, ox, oy, oz,
                                                   s_list, s_abs, s_cnt);
                    __syncthreads();  // the boxes are free for the next brick
                }
            } else if (ph == 0) {
                // ---- NT/32 tiles of the band list (2-D, or a 3-D job on the
                // list step), one per warp ----
                const Params<T>& P = J.P;
                const int cnt_in = vload(&ds->band_count[n & 1]);
                const int ntiles = (cnt_in + kStepTile - 1) / kStepTile;
                if (loc == 0 && tid == 0) ds->band_count[(n + 1) & 1] = ntiles ? vload(&ds->band_next) : 0;
                const int t = loc * W + warp;
                if (t < ntiles) {
                    const T* uin = (n & 1) ? J.ub1 : J.ub0;
                    T* uout = (n & 1) ? J.ub0 : J.ub1;
                    const int* Lin = (n & 1) ? J.L1 : J.L0;
                    int* Lout = (n & 1) ? J.L0 : J.L1;
                    const T Ep = (T)vload(&ds->Ep);
                    const int per = (ntiles + kRecordBlocks - 1) / kRecordBlocks;
                    if (J.dim == 3) {
                        if (J.interp)
                            band_tile<T, 3, 1>(P, uin, uout, J.d, Lin, Lout, J.tile_off, ds->band_base, J.band_cap,
                                               cnt_in, per, t, Ep, J.part_dphi, ds);
                        else
                            band_tile<T, 3, 0>(P, uin, uout, J.d, Lin, Lout, J.tile_off, ds->band_base, J.band_cap,
                                               cnt_in, per, t, Ep, J.part_dphi, ds);
                    } else if (J.interp) {
                        band_tile<T, 2, 1>(P, uin, uout, J.d, Lin, Lout, J.tile_off, ds->band_base, J.band_cap, cnt_in,
                                           per, t, Ep, J.part_dphi, ds);
                    } else {
                        band_tile<T, 2, 0>(P, uin, uout, J.d, Lin, Lout, J.tile_off, ds->band_base, J.band_cap, cnt_in,
                                           per, t, Ep, J.part_dphi, ds);
                    }
                }
            } else if (ph == 1) {
                // ---- energy slots (after a list-step job's tile counts) on u^{n+1} ----
                const Params<T>& P = J.P;
                const EnergyArgs<T>& E = J.E;
                const int sel = (n + 1) & 1;
                const T* u = sel ? J.ub1 : J.ub0;
                if (loc < J.ntc) {
                    const int nb = vload(&ds->band_count[sel]);
                    const int t = loc * W + warp;
                    if (t < (nb + kStepTile - 1) / kStepTile) tile_count<T>(P, u, sel ? J.L1 : J.L0, nb, t, J.tile_off);
                } else if (J.dim == 3) {
                    if (J.interp)
                        energy_slot<T, 3, 1, 5, NT>(P, u, J.d, J.cells, J.ncells, loc - J.ntc, E, J.part_e, ews);
                    else
                        energy_slot<T, 3, 0, 5, NT>(P, u, J.d, J.cells, J.ncells, loc - J.ntc, E, J.part_e, ews);
                } else if (J.interp) {
                    energy_slot<T, 2, 1, 0, NT>(P, u, J.d, J.cells, J.ncells, loc - J.ntc, E, J.part_e, ews);
                } else {
                    energy_slot<T, 2, 0, 0, NT>(P, u, J.d, J.cells, J.ncells, loc - J.ntc, E, J.part_e, ews);
                }
            } else {
                // ---- a record slice; the last one completes the iteration ----
                const bool last = record_slice<NT>(cold[j].rec, ds, loc, kRecordBlocks, rws);
                if (last && tid == 0) {
                    __threadfence();
                    atomicAdd(&ctl->rec_done[j], 1);
                }
            }
        }
        // this item's completion, published by thread 32 at the top of the
        // next pass (after the barrier below; every way out of the loop
        // passes through that top)
        if (tid == 0) s_it[kItDone] = ph == 0 ? j : (ph == 1 ? kBatchMaxJobs + j : -1);
        __syncthreads();
    }
}

// Failure-detection check of the dependency wait above: one thread waits
// for a counter that nothing increments (no stop flag set), so the wait
// runs out after its poll limit and sets kErrBarrier in *err.
__global__ void k_batch_wait_selftest(const int* words, int* err) {
    if (threadIdx.x == 0 && blockIdx.x == 0) batch_wait(words, 1, words + 1, err);
}

// dynamic shared memory of k_batch
template <typename T>
constexpr int batch_smem() {
    return BrickSmem<T, 1>::kBytes;
}

// ---------------------------------------------------------------------------
// host side: one group of at most kBatchMaxJobs jobs of storage type T
// ---------------------------------------------------------------------------
// Launch shapes the autotuner chooses between: threads per block, resident
// blocks per SM (the register budget: FP32 80 or 96 registers at 128
// threads; FP64 168 or 255), bricks per step item (more bricks per item
// spread the item's bookkeeping; fewer even out the end of a phase)
constexpr int kBatchShapes = 7;
struct BatchShape {
    int nt, inst, bpi;  // inst: 0 = <128, hi occ>, 1 = <128, lo occ>, 2 = <256, ...>
};
constexpr BatchShape kBatchShape[kBatchShapes] = {{128, 0, 1}, {128, 0, 2}, {128, 1, 1}, {128, 1, 2},
                                                   {256, 2, 1}, {128, 0, 4}, {128, 1, 4}};
template <typename T>
struct BatchInstOcc {
    static constexpr int hi = sizeof(T) == 4 ? 6 : 3, lo = sizeof(T) == 4 ? 5 : 2, wide = sizeof(T) == 4 ? 3 : 1;
};
constexpr int kBatchTuneIters = 1;      // iterations of each autotuning launch
constexpr int kBatchChunk = 1 << 20;    // iterations of a launch after autotuning (all jobs stop first)

template <typename T, int NT, int OCC>
cudaError_t batch_kernel_setup(int* occ) {
    auto kern = k_batch<T, NT, OCC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_smem<T>());
    if (e != cudaSuccess) return e;
    int o = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, NT, batch_smem<T>());
    *occ = o;
    return e;
}

template <typename T, int NT, int OCC>
cudaError_t batch_enqueue(const BatchParams<T>& bp, const BatchCold* cold, BatchCtl* ctl, int njobs, int iters,
                          int bpi, int grid, cudaStream_t st) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = batch_smem<T>();
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch<T, NT, OCC>, bp, cold, ctl, njobs, iters, bpi);
}

// Advance jobs[0..n) (band mode, no reinitialisation, 3-D energy R = 5; all
// of storage type T, on one device) until each has stopped. shape_io: -1 to
// autotune the launch shape, else the index into kBatchShape; receives the
// one used. graph_out: 1 if the launches ran as captured graphs; threads,
// resident blocks per SM and bricks per item of the shape used.
template <typename T>
slr_status batch_run_group(slr_ctx* const* jobs, int n, int tune, cudaStream_t st, int* shape_io, int* graph_out,
                           float* tuned_ms, int* threads_out, int* blocks_out, int* bpi_out) {
    slr_ctx* c0 = jobs[0];
    std::vector<int> order(n);
    for (int j = 0; j < n; ++j) order[j] = j;
    // the costliest items first, so that the sequence of one phase ends on
    // small items: 3-D WENO, then 3-D Q1, then 2-D (results do not depend on it)
    auto rank = [&](int j) { return jobs[j]->cfg.dim == 3 ? (jobs[j]->cfg.interp ? 0 : 1) : 2; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rank(a) < rank(b); });
    // one parameter block per launch shape (its item counts depend on the
    // shape: NT/32 tiles per 2-D item, bpi bricks per 3-D item)
    std::vector<BatchParams<T>*> bp(kBatchShapes, nullptr);
    for (auto& x : bp) x = new BatchParams<T>();
    std::vector<BatchCold> hcold(n);
    memset(hcold.data(), 0, sizeof(BatchCold) * n);
    for (int q = 0; q < n; ++q) {
        slr_ctx* c = jobs[order[q]];
        BatchHot<T> J;
        memset(&J, 0, sizeof(J));
        J.P = make_params<T>(c);
        const double p = c->cfg.p;
        const int p_kind = p == 1.0 ? 1 : (p == 2.0 ? 2 : 0);
        J.E = energy_args<T>(c, p, p_kind);
        J.ub0 = (T*)c->u[0];
        J.ub1 = (T*)c->u[1];
        J.d = (const T*)c->d;
        J.ds = c->ds;
        J.cells = c->ecells;
        J.ncells = c->n_ecells;
        J.nslots = (int)energy_slots(c);
        J.part_e = c->part_e;
        J.L0 = c->band[0];
        J.L1 = c->band[1];
        J.tile_off = c->tile_off;
        J.part_dphi = c->part_dphi;
        J.band_cap = (int)c->band_cap;
        J.dim = c->cfg.dim;
        J.interp = c->cfg.interp;
        J.bricked = brick_mode(c) ? 1 : 0;
        if (J.bricked) {
            const BrickState& B = c->brick;
            J.A.nbricks = (int)B.nbricks;
            J.A.bricks = B.list;
            J.A.bcnt = B.cnt;
            J.A.part_dphi = B.part;
            J.A.nbx = B.nb[0];
            J.A.nby = B.nb[1];
            J.A.tma = B.tma;
            J.A.dt_h = (T)(c->dt / c->h);
            J.A.kdiff = (T)(c->cfg.delta * c->dt / (c->cfg.p * c->h * c->h));
            const double thr = c->cfg.c_sing * pow(c->dt, c->cfg.alpha);
            J.A.thr2 = (T)thr * (T)thr;
            hcold[q].tm[0] = B.tm_u[0];
            hcold[q].tm[1] = B.tm_u[1];
            hcold[q].tm[2] = B.tm_d;
        }
        hcold[q].rec = record_args(c, 1, 1, p, p_kind);
        for (int sh = 0; sh < kBatchShapes; ++sh) {
            // items per iteration: the band of a job without reinitialisation
            // only shrinks, so a 2-D job's tiles are bounded by its list capacity
            const int W = kBatchShape[sh].nt / 32, bpi = kBatchShape[sh].bpi;
            BatchHot<T> Js = J;
            const int cap_tiles = (int)((c->band_cap + kStepTile - 1) / kStepTile);
            Js.ntc = J.bricked ? 0 : (cap_tiles + W - 1) / W;
            const int s_items = J.bricked ? (J.A.nbricks + bpi - 1) / bpi : std::max(1, Js.ntc);
            const int e_items = Js.ntc + J.nslots;
            BatchParams<T>& B = *bp[sh];
            B.job[q] = Js;
            B.pre[0][q + 1] = B.pre[0][q] + s_items;
            B.pre[1][q + 1] = B.pre[1][q] + e_items;
            B.pre[2][q + 1] = B.pre[2][q] + kRecordBlocks;
        }
    }
    for (int sh = 0; sh < kBatchShapes; ++sh)
        bp[sh]->per_iter = (long long)bp[sh]->pre[0][n] + bp[sh]->pre[1][n] + bp[sh]->pre[2][n];
    BatchCold* dcold = nullptr;
    BatchCtl* dctl = nullptr;
    DevState** dstates = nullptr;
    int* dstat = nullptr;
    int* hstat = nullptr;
    cudaGraphExec_t gx[kBatchShapes][2] = {};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    auto cleanup = [&]() {
        for (auto& r : gx)
            for (auto& g : r)
                if (g) cudaGraphExecDestroy(g);
        for (auto x : ev)
            if (x) cudaEventDestroy(x);
        if (dcold) dev_free(c0, dcold);
        if (dctl) dev_free(c0, dctl);
        if (dstates) dev_free(c0, dstates);
        if (dstat) dev_free(c0, dstat);
        if (hstat) cudaFreeHost(hstat);
        for (auto b : bp) delete b;
    };
    dcold = (BatchCold*)dev_alloc(c0, sizeof(BatchCold) * n);
    dctl = (BatchCtl*)dev_alloc(c0, sizeof(BatchCtl));
    dstates = (DevState**)dev_alloc(c0, sizeof(DevState*) * n);
    dstat = (int*)dev_alloc(c0, sizeof(int) * (4 * n + 1));
    if (!dcold || !dctl || !dstates || !dstat) {
        cleanup();
        return SLR_E_NOMEM;
    }
    cudaError_t e = cudaMallocHost((void**)&hstat, sizeof(int) * (4 * n + 1));
    std::vector<DevState*> hs(n);
    for (int q = 0; q < n; ++q) hs[q] = jobs[order[q]]->ds;
    if (e == cudaSuccess) e = cudaMemcpyAsync(dcold, hcold.data(), sizeof(BatchCold) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dstates, hs.data(), sizeof(DevState*) * n, cudaMemcpyHostToDevice, st);
    // every job's own stream must be idle before the batch stream takes over
    for (int j = 0; j < n && e == cudaSuccess; ++j) e = cudaStreamSynchronize(jobs[j]->stream);
    for (int j = 0; j < n && e == cudaSuccess; ++j) {
        e = cudaMemsetAsync(&jobs[j]->ds->stop, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(&jobs[j]->ds->converged, 0, sizeof(int), st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    using O = BatchInstOcc<T>;
    int occ[3] = {0, 0, 0};  // resident blocks per SM of each kernel instance
    if (e == cudaSuccess) e = batch_kernel_setup<T, 128, O::hi>(&occ[0]);
    if (e == cudaSuccess) e = batch_kernel_setup<T, 128, O::lo>(&occ[1]);
    if (e == cudaSuccess) e = batch_kernel_setup<T, 256, O::wide>(&occ[2]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_status(c0, e, "batch_run");
    }
    // one launch: reset the control words, the kernel, the jobs' status
    // words gathered into one array and copied to pinned host memory. The
    // tickets are 32-bit: a launch covers at most 2^31 items.
    auto enqueue = [&](int sh, int iters) -> cudaError_t {
        const BatchShape& S = kBatchShape[sh];
        const long long cap = 0x7fffffffll / std::max(1ll, bp[sh]->per_iter);
        iters = (int)std::min<long long>(iters, std::max(1ll, cap));
        cudaError_t r = cudaMemsetAsync(dctl, 0, sizeof(BatchCtl), st);
        const int grid = occ[S.inst] * c0->num_sms;
        if (r == cudaSuccess) {
            if (S.inst == 0)
                r = batch_enqueue<T, 128, O::hi>(*bp[sh], dcold, dctl, n, iters, S.bpi, grid, st);
            else if (S.inst == 1)
                r = batch_enqueue<T, 128, O::lo>(*bp[sh], dcold, dctl, n, iters, S.bpi, grid, st);
            else
                r = batch_enqueue<T, 256, O::wide>(*bp[sh], dcold, dctl, n, iters, S.bpi, grid, st);
        }
        if (r == cudaSuccess) r = launch_gather_status(c0, dstates, n, dstat, st);
        if (r == cudaSuccess) r = cudaMemcpyAsync(dstat + 4 * n, &dctl->err, sizeof(int), cudaMemcpyDeviceToDevice, st);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(hstat, dstat, sizeof(int) * (4 * n + 1), cudaMemcpyDeviceToHost, st);
        return r;
    };
    bool graphs = true;
    // capture the launch sequence as a graph (once per shape and launch
    // length); where capture is refused, the same sequence is enqueued directly
    auto launch = [&](int sh, int li) -> cudaError_t {
        const int iters = li == 0 ? kBatchTuneIters : kBatchChunk;
        if (graphs && !gx[sh][li]) {
            cudaGraph_t g = nullptr;
            cudaError_t r = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (r == cudaSuccess) {
                cudaError_t r1 = enqueue(sh, iters);
                cudaError_t r2 = cudaStreamEndCapture(st, &g);
                r = r1 != cudaSuccess ? r1 : r2;
            }
            if (r == cudaSuccess) r = cudaGraphInstantiate(&gx[sh][li], g, 0);
            if (g) cudaGraphDestroy(g);
            if (r != cudaSuccess) {
                graphs = false;
                cudaGetLastError();
                if (gx[sh][li]) cudaGraphExecDestroy(gx[sh][li]);
                gx[sh][li] = nullptr;
            }
        }
        c0->launches += 2;
        if (graphs) return cudaGraphLaunch(gx[sh][li], st);
        return enqueue(sh, iters);
    };
    int shape = *shape_io >= 0 && *shape_io < kBatchShapes ? *shape_io : 0;
    float best_ms = 0.f;
    bool done = false;
    slr_status status = SLR_OK;
    auto check = [&]() -> bool {
        // after a launch has completed: error words, then whether all stopped
        if (hstat[4 * n] & kErrBarrier) {
            status = SLR_E_TIMEOUT;
            return true;
        }
        bool all = true;
        for (int q = 0; q < n; ++q) {
            if (hstat[4 * q + 3]) {
                status = SLR_E_STATE;
                return true;
            }
            all = all && hstat[4 * q + 0];
        }
        return all;
    };
    if (tune) {
        // each shape twice, kBatchTuneIters iterations per launch, in turns;
        // the least device time per launch wins (the iterations and results
        // do not depend on the shape)
        float ms_of[kBatchShapes];
        for (auto& x : ms_of) x = 1e30f;
        for (int rep = 0; rep < 2 && !done && e == cudaSuccess; ++rep)
            for (int sh = kBatchShapes - 1; sh >= 0 && !done && e == cudaSuccess; --sh) {
                e = cudaEventRecord(ev[0], st);
                if (e == cudaSuccess) e = launch(sh, 0);
                if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
                if (e == cudaSuccess) {
                    done = check();
                    if (ms < ms_of[sh]) ms_of[sh] = ms;
                }
            }
        shape = 0;
        for (int sh = 1; sh < kBatchShapes; ++sh)
            if (ms_of[sh] < ms_of[shape]) shape = sh;
        best_ms = ms_of[shape];
    }
    while (!done && e == cudaSuccess) {
        e = launch(shape, 1);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) done = check();
    }
    if (e != cudaSuccess) {
        cleanup();
        return cuda_status(c0, e, "batch_run");
    }
    for (int q = 0; q < n; ++q) {
        slr_ctx* c = jobs[order[q]];
        c->batch_iters = hstat[4 * q + 1];
        c->batch_converged = hstat[4 * q + 2];
    }
    *shape_io = shape;
    *graph_out = graphs ? 1 : 0;
    *tuned_ms = best_ms;
    *threads_out = kBatchShape[shape].nt;
    *blocks_out = occ[kBatchShape[shape].inst];
    *bpi_out = kBatchShape[shape].bpi;
    cleanup();
    return status;
}

}  // namespace
}  // namespace slr
