// Batched evolution of many independent reconstructions in one persistent,
// cooperative, graph-captured kernel (k_batch).
//
// Every job is one run of Algorithm 1's loop (arXiv 2410.22205, §3: step 4,
// the SL update of §3.1-§3.2 with the band and cut of §3.8, then the energy
// of §3.5 and the stop test of §4 eq. deltaEn), without the
// reinitialisation. The kernel advances all jobs together, iteration by
// iteration, in three phases separated by grid barriers:
//   0. step:   one work item per active brick of a 3-D job (the brick step
//              of slr_brick.cuh) or per NT/32 tiles of 128 band-list
//              entries of a 2-D job (the list step of slr_step.cuh);
//   1. energy: one work item per slot of 1024 candidate cells of every job,
//              plus, for a 2-D job, its tiles' band-member counts;
//   2. record: kRecordBlocks slices per job; the block that finishes a
//              job's last slice does its bookkeeping and stop test.
// Blocks take work items from one ticket counter; a phase's items are the
// concatenation of the running jobs' items (jobs whose stop test has fired
// have none), so large and small jobs share the GPU without one launch per
// job. The barriers give up after a poll limit and report kErrBarrier,
// which the host returns as SLR_E_TIMEOUT.
//
// The per-item device code is the per-job kernels' own (brick_compute,
// band_tile, energy_slot, tile_count, record_slice), compiled like them
// without implicit FMA contraction and with the reductions' summation trees
// kept, so each job's results are bit-identical to its solo run. Fields that
// other blocks wrote before a barrier are read with coherent loads
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
};

template <typename T>
struct BatchParams {
    BatchHot<T> job[kBatchMaxJobs];
};
static_assert(sizeof(BatchParams<double>) + 64 <= 32764, "batch parameters fit the kernel-parameter space");

// per-job data read rarely: in global memory (tensor maps 64-byte aligned)
struct __align__(64) BatchCold {
    CUtensorMap tm[3];  // u buffer 0, u buffer 1, d (3-D jobs staged by TMA)
    RecordArgs rec;
};

struct BatchCtl {
    unsigned bar[2];           // grid barrier: arrivals, generation
    int err;                   // kErrBarrier / kErrStage
    int iters;                 // iterations this launch ran (block 0)
    unsigned long long ticket; // work-item tickets of all phases of the launch
};

// block size x resident blocks per SM the register budget allows
template <typename T, int NT>
struct BatchOcc {
    static constexpr int v = sizeof(T) == 4 ? 768 / NT : (NT == 128 ? 3 : 1);
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

// Grid-wide barrier of the cooperative launch (the protocol of grid_barrier,
// with its result word in dynamic shared memory: the kernel keeps no static
// shared memory, so that six blocks of 128 threads fit an SM). A wait
// longer than the poll limit, or an error bit set by another block, makes
// every block see false.
__device__ __forceinline__ bool batch_barrier(unsigned* bar, int* err, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long polls = 0;
            while (*vgen == gen) {
                if (++polls > kBarrierSpinLimit || (*(volatile int*)err & kErrBarrier)) {
                    ok = 0;
                    atomicOr(err, kErrBarrier);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// work items of job J in phase ph (0 while its stop flag is set)
template <typename T, int NT>
__device__ __forceinline__ int batch_items(const BatchHot<T>& J, int ph) {
    constexpr int W = NT / 32;
    const DevState* ds = J.ds;
    if (vload(&ds->stop)) return 0;
    if (ph == 2) return kRecordBlocks;
    if (J.dim == 3) return ph == 0 ? J.A.nbricks : J.nslots;
    const int n = vload(&ds->n);
    if (ph == 0) {
        // at least one item: item 0 also publishes the size of the band it writes
        const int nt = (vload(&ds->band_count[n & 1]) + kStepTile - 1) / kStepTile;
        const int it = (nt + W - 1) / W;
        return it > 0 ? it : 1;
    }
    const int nt = (vload(&ds->band_count[(n + 1) & 1]) + kStepTile - 1) / kStepTile;
    return (nt + W - 1) / W + J.nslots;
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, BatchOcc<T, NT>::v)
    k_batch(const __grid_constant__ BatchParams<T> BP, const BatchCold* __restrict__ cold, BatchCtl* ctl, int njobs,
            int max_iters) {
    using S = BrickSmem<T, 1>;
    using G = BoxGeom;
    constexpr int W = NT / 32;
    static_assert(sizeof(EnergyWs<T>) <= S::kBar && sizeof(RecordWs) <= S::kBar, "workspaces fit the brick area");
    extern __shared__ __align__(128) unsigned char smem[];
    // [0, kBar): one item's scratch (brick boxes and lists, or the energy or
    // record workspace); kBar: the staging barrier; kTicket: the item (job,
    // index) and the grid barrier's result; kBytes: the prefix of the jobs'
    // item counts
    T* su = reinterpret_cast<T*>(smem);
    T* sd = reinterpret_cast<T*>(smem + G::BoxN * (int)sizeof(T));
    unsigned short* s_list = reinterpret_cast<unsigned short*>(smem + S::kList);
    T* s_abs = reinterpret_cast<T*>(smem + S::kAbs);
    int* s_cnt = reinterpret_cast<int*>(smem + S::kCnt);
    EnergyWs<T>& ews = *reinterpret_cast<EnergyWs<T>*>(smem);
    RecordWs& rws = *reinterpret_cast<RecordWs*>(smem);
    int* s_item = reinterpret_cast<int*>(smem + S::kTicket);
    int* s_pre = reinterpret_cast<int*>(smem + S::kBytes);
    const unsigned bar = smem_addr(smem + S::kBar);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        for (int j = 0; j < njobs; ++j)
            if (BP.job[j].dim == 3 && BP.job[j].A.tma)
                for (int m = 0; m < 3; ++m) fence_tensormap_acquire(&cold[j].tm[m]);
    }
    __syncthreads();
    unsigned long long tbase = 0;  // tickets taken before this phase (the same in every block)
    unsigned tpar = 0;             // thread 0: parity of the staging barrier's next completion
    int it = 0;
    for (; it < max_iters; ++it) {
        bool any = true;
        for (int ph = 0; ph < 3 && any; ++ph) {
            if (tid < njobs) s_pre[tid + 1] = batch_items<T, NT>(BP.job[tid], ph);
            __syncthreads();
            if (tid == 0) {
                s_pre[0] = 0;
                for (int j = 1; j <= njobs; ++j) s_pre[j] += s_pre[j - 1];
            }
            __syncthreads();
            const int total = s_pre[njobs];
            if (ph == 0 && total == 0) {
                any = false;  // every job has stopped (every block sees the same state)
                break;
            }
            for (;;) {
                if (tid == 0) {
                    const long long t = (long long)(atomicAdd(&ctl->ticket, 1ull) - tbase);
                    int jj = -1, loc = 0;
                    if (t < total) {
                        int lo = 0, hi = njobs;  // s_pre[lo] <= t < s_pre[hi]
                        while (hi - lo > 1) {
                            const int mid = (lo + hi) >> 1;
                            if (s_pre[mid] <= t)
                                lo = mid;
                            else
                                hi = mid;
                        }
                        jj = lo;
                        loc = (int)(t - s_pre[lo]);
                    }
                    s_item[0] = jj;
                    s_item[1] = loc;
                }
                __syncthreads();
                const int j = s_item[0], loc = s_item[1];
                if (j < 0) break;
                const BatchHot<T>& J = BP.job[j];
                DevState* ds = J.ds;
                const int n = vload(&ds->n);
                if (ph == 0 && J.dim == 3) {
                    // ---- a brick of a 3-D job ----
                    const Params<T> P = J.P;
                    const BrickArgs<T> A = J.A;
                    const int b = __ldg(A.bricks + loc);
                    if (__ldcg(A.bcnt + b) != 0) {
                        const T* uin = (n & 1) ? J.ub1 : J.ub0;
                        T* uout = (n & 1) ? J.ub0 : J.ub1;
                        const T Ep = (T)vload(&ds->Ep);
                        const T invEp = Ep > T(0) ? T(1) / Ep : T(0);
                        const int bxi = b % A.nbx, q = b / A.nbx;
                        const int ox = bxi * kBX - kHalo, oy = (q % A.nby) * kBY - kHalo, oz = (q / A.nby) * kBZ - kHalo;
                        bool staged = true;
                        if (A.tma) {
                            if (tid == 0) {
                                // the boxes' rows were written through the generic proxy
                                // by other blocks before the last barrier, and this
                                // block's generic accesses of the scratch area ended at
                                // the last block barrier
                                fence_proxy_async_global();
                                fence_proxy_async();
                                mbar_expect_tx(bar, (unsigned)((G::BoxN + G::DBoxN) * sizeof(T)));
                                tma_load_3d(smem_addr(su), &cold[j].tm[n & 1], bar, ox, oy, oz);
                                tma_load_3d(smem_addr(sd), &cold[j].tm[2], bar, ox, oy + kHalo - 1, oz + kHalo - 1);
                                long long w = 0;
                                while (!mbar_try_wait(bar, tpar) && ++w < kStageWaitLimit) {
                                }
                                staged = w < kStageWaitLimit;
                                if (!staged) {
                                    long long w2 = 0;  // the copies in flight: a second bounded wait
                                    while (!mbar_try_wait(bar, tpar) && ++w2 < kStageWaitLimit) {
                                    }
                                }
                                tpar ^= 1u;
                            }
                        } else {
                            brick_stage_copy<T, NT>(P, uin, J.d, su, sd, ox, oy, oz);
                        }
                        if (__syncthreads_or(!staged)) {
                            if (tid == 0) {
                                atomicOr(&ds->error, kErrStage);
                                atomicOr(&ctl->err, kErrStage | kErrBarrier);  // the other blocks leave their barrier
                            }
                            return;
                        }
                        if (J.interp)
                            brick_compute<T, 1, 1, NT>(P, A, su, sd, uin, uout, J.d, ds, Ep, invEp, b, ox, oy, oz,
                                                       s_list, s_abs, s_cnt);
                        else
                            brick_compute<T, 0, 1, NT>(P, A, su, sd, uin, uout, J.d, ds, Ep, invEp, b, ox, oy, oz,
                                                       s_list, s_abs, s_cnt);
                    }
                } else if (ph == 0) {
                    // ---- NT/32 tiles of a 2-D job's band list, one per warp ----
                    const Params<T> P = J.P;
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
                        if (J.interp)
                            band_tile<T, 2, 1>(P, uin, uout, J.d, Lin, Lout, J.tile_off, ds->band_base, J.band_cap,
                                               cnt_in, per, t, Ep, J.part_dphi, ds);
                        else
                            band_tile<T, 2, 0>(P, uin, uout, J.d, Lin, Lout, J.tile_off, ds->band_base, J.band_cap,
                                               cnt_in, per, t, Ep, J.part_dphi, ds);
                    }
                } else if (ph == 1) {
                    // ---- energy slots (and a 2-D job's tile counts) on u^{n+1} ----
                    const Params<T> P = J.P;
                    const EnergyArgs<T> E = J.E;
                    const int sel = (n + 1) & 1;
                    const T* u = sel ? J.ub1 : J.ub0;
                    if (J.dim == 3) {
                        if (J.interp)
                            energy_slot<T, 3, 1, 5, NT>(P, u, J.d, J.cells, J.ncells, loc, E, J.part_e, ews);
                        else
                            energy_slot<T, 3, 0, 5, NT>(P, u, J.d, J.cells, J.ncells, loc, E, J.part_e, ews);
                    } else {
                        const int nb = vload(&ds->band_count[sel]);
                        const int ntb = (nb + kStepTile - 1) / kStepTile;
                        const int ntc = (ntb + W - 1) / W;
                        if (loc < ntc) {
                            const int t = loc * W + warp;
                            if (t < ntb) tile_count<T>(P, u, sel ? J.L1 : J.L0, nb, t, J.tile_off);
                        } else if (J.interp) {
                            energy_slot<T, 2, 1, 0, NT>(P, u, J.d, J.cells, J.ncells, loc - ntc, E, J.part_e, ews);
                        } else {
                            energy_slot<T, 2, 0, 0, NT>(P, u, J.d, J.cells, J.ncells, loc - ntc, E, J.part_e, ews);
                        }
                    }
                } else {
                    // ---- a record slice ----
                    record_slice<NT>(cold[j].rec, ds, loc, kRecordBlocks, rws);
                }
                __syncthreads();
            }
            tbase += (unsigned long long)total + gridDim.x;  // every block took one ticket past the end
            if (!batch_barrier(ctl->bar, &ctl->err, s_item + 2)) return;
        }
        if (!any) break;
    }
    if (blockIdx.x == 0 && tid == 0) ctl->iters = it;
}

// dynamic shared memory of k_batch<T, NT>
template <typename T>
constexpr int batch_smem() {
    return BrickSmem<T, 1>::kBytes + (kBatchMaxJobs + 1) * (int)sizeof(int);
}

// ---------------------------------------------------------------------------
// host side: one group of at most kBatchMaxJobs jobs of storage type T
// ---------------------------------------------------------------------------
constexpr int kBatchShapes = 2;
constexpr int kBatchNT[kBatchShapes] = {128, 256};
constexpr int kBatchTuneIters = 2;      // iterations of each autotuning launch
constexpr int kBatchChunk = 1 << 20;    // iterations of a launch after autotuning (all jobs stop first)

template <typename T, int NT>
cudaError_t batch_kernel_setup(int device, int* occ) {
    auto kern = k_batch<T, NT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, batch_smem<T>());
    if (e != cudaSuccess) return e;
    int o = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kern, NT, batch_smem<T>());
    *occ = o;
    (void)device;
    return e;
}

template <typename T, int NT>
cudaError_t batch_enqueue(const BatchParams<T>& bp, const BatchCold* cold, BatchCtl* ctl, int njobs, int iters,
                          int grid, cudaStream_t st) {
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
    return cudaLaunchKernelEx(&cfg, k_batch<T, NT>, bp, cold, ctl, njobs, iters);
}

// Advance jobs[0..n) (band mode, no reinitialisation, 3-D energy R = 5; all
// of storage type T, on one device) until each has stopped. shape_io: -1 to
// autotune the block size, else the index of kBatchNT to use; receives the
// one used. graph_out: 1 if the launches ran as captured graphs.
template <typename T>
slr_status batch_run_group(slr_ctx* const* jobs, int n, int tune, cudaStream_t st, int* shape_io, int* graph_out,
                           float* tuned_ms) {
    slr_ctx* c0 = jobs[0];
    std::vector<int> order(n);
    for (int j = 0; j < n; ++j) order[j] = j;
    // the costliest items first, so a phase ends on small items: 3-D WENO,
    // then 3-D Q1, then 2-D (the results do not depend on the order)
    auto rank = [&](int j) { return jobs[j]->cfg.dim == 3 ? (jobs[j]->cfg.interp ? 0 : 1) : 2; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rank(a) < rank(b); });
    BatchParams<T>* bp = new BatchParams<T>();
    std::vector<BatchCold> hcold(n);
    memset(hcold.data(), 0, sizeof(BatchCold) * n);
    for (int q = 0; q < n; ++q) {
        slr_ctx* c = jobs[order[q]];
        BatchHot<T>& J = bp->job[q];
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
        memset(&J.A, 0, sizeof(J.A));
        if (c->cfg.dim == 3) {
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
    }
    BatchCold* dcold = nullptr;
    BatchCtl* dctl = nullptr;
    DevState** dstates = nullptr;
    int* dstat = nullptr;
    int* hstat = nullptr;
    cudaGraphExec_t gx[kBatchShapes][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
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
        delete bp;
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
    int occ[kBatchShapes] = {0, 0};
    if (e == cudaSuccess) e = batch_kernel_setup<T, 128>(c0->device, &occ[0]);
    if (e == cudaSuccess) e = batch_kernel_setup<T, 256>(c0->device, &occ[1]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_status(c0, e, "batch_run");
    }
    // one launch: reset the control words, the kernel, the jobs' status
    // words gathered into one array and copied to pinned host memory
    auto enqueue = [&](int sh, int iters) -> cudaError_t {
        cudaError_t r = cudaMemsetAsync(dctl, 0, sizeof(BatchCtl), st);
        const int grid = occ[sh] * c0->num_sms;
        if (r == cudaSuccess)
            r = sh == 0 ? batch_enqueue<T, 128>(*bp, dcold, dctl, n, iters, grid, st)
                        : batch_enqueue<T, 256>(*bp, dcold, dctl, n, iters, grid, st);
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
        // each shape twice, kBatchTuneIters iterations per launch, in
        // alternation; the least device time per launch wins (the iterations
        // and results do not depend on the shape)
        float ms_of[kBatchShapes] = {1e30f, 1e30f};
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
        shape = ms_of[0] <= ms_of[1] ? 0 : 1;
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
    cleanup();
    return status;
}

}  // namespace
}  // namespace slr
