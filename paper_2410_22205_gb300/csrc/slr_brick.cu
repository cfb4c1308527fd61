// Brick-staged semi-Lagrangian step in 3-D (arXiv 2410.22205, §3.1 eq. SL3d
// and eq. sigma3d, §3.2 eqs. IQ1 and IWENO, §3.8 eqs. subgrid, cutoff and
// cut), for the narrow band and for the whole grid.
//
// The grid is cut into bricks of 8x8x8 nodes. At init the bricks that hold a
// node of the band G̃^0 (every brick on the whole grid) form a fixed list.
// Per iteration, one persistent launch hands the bricks out by ticket; for
// each brick a block
//   1. stages u^n on the brick plus a halo of 4 nodes in y and z and of 4
//      (left) and 12 (right) in x (a 24x16x16 box), and d on the brick plus
//      4 and 12 nodes in x and 1 in y and z (24x10x10), into shared memory:
//      one TMA tile load per box when rows are 16-byte aligned, 4- or 8-byte
//      cp.async copies with zero fill otherwise (with two stages the next
//      brick's boxes load while this one is computed);
//   2. compacts the brick's band nodes (|u^n_j| < γ in the storage
//      precision: every node outside the band sits at ±γ since the initial
//      cut, so this is G̃^n) into a shared list, in node order;
//   3. runs the SL update of every listed node from shared memory: gradients
//      of u and d, scale factor and cut-off, tangent basis, four feet. A foot
//      whose interpolation stencil lies inside the box and away from the grid
//      edge is interpolated from shared memory; any other foot takes the
//      global-memory interpolators, which clamp at the edge as the paper's
//      silent cases are read;
//   4. writes u^{n+1} on the band nodes (after the cut) and copies u^n into
//      u^{n+1} on the brick's other nodes, so both buffers agree outside the
//      band; writes the brick's Δ_φ partial (FP64, summed in list order)
//      and its band count.
// A brick whose band count was zero in the previous iteration has both
// buffers equal on all its nodes and is skipped. The launch shape (threads per
// block, stages) is chosen at init by timing each candidate.
//
// This file is compiled with -fmad=false: each launch shape is its own
// template instance, and an implicit a*b + c that the compiler fused in one
// instance and not in another would make results depend on the autotuner's
// choice. Every FMA here is written explicitly.
#include <cuda.h>

#include <mutex>

#include "slr_brick.cuh"
#include "slr_compact.cuh"
#include "slr_internal.cuh"

namespace slr {

template <typename T>
Params<T> make_params(const slr_ctx* c);

namespace {

// One persistent launch over the active bricks. NT threads per block; ST = 2
// prefetches the next brick's boxes by TMA while the current brick is
// computed (the cp.async path stages one brick at a time).
template <typename T, int INTERP, int BAND, int NT, int ST>
__global__ void __launch_bounds__(NT, BrickOcc<T, INTERP, NT>::v)
    k_step_brick(const __grid_constant__ CUtensorMap tm_u0, const __grid_constant__ CUtensorMap tm_u1,
                 const __grid_constant__ CUtensorMap tm_d, Params<T> P, BrickArgs<T> A, T* ub0, T* ub1,
                 const T* __restrict__ d, DevState* ds, double ep_override) {
    using S = BrickSmem<T, ST>;
    using G = BoxGeom;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned short* s_list = reinterpret_cast<unsigned short*>(smem + S::kList);
    T* s_abs = reinterpret_cast<T*>(smem + S::kAbs);
    int* s_cnt = reinterpret_cast<int*>(smem + S::kCnt);
    int* s_tk = reinterpret_cast<int*>(smem + S::kTicket);  // per stage: ticket, brick id, skip
    if (ds->stop) return;
    const int tid = threadIdx.x;
    const int n = ds->n;
    const T* __restrict__ uin = (n & 1) ? ub1 : ub0;
    T* __restrict__ uout = (n & 1) ? ub0 : ub1;
    const CUtensorMap* tmu = (n & 1) ? &tm_u1 : &tm_u0;
    const CUtensorMap* tmd = &tm_d;
    const T Ep = ep_override >= 0.0 ? (T)ep_override : (T)ds->Ep;
    const T invEp = Ep > T(0) ? T(1) / Ep : T(0);
    const bool tma = A.tma != 0;
    const bool pipe = ST == 2 && tma;
    auto stage_u = [&](int st) { return reinterpret_cast<T*>(smem + st * S::kStage); };
    auto stage_d = [&](int st) { return reinterpret_cast<T*>(smem + st * S::kStage + G::BoxN * (int)sizeof(T)); };
    auto bar_of = [&](int st) { return smem_addr(smem + S::kBar + 8 * st); };
    // thread 0: take a ticket into stage st and, by TMA, start its copies
    auto take = [&](int st) {
        const int t = (int)atomicAdd(&ds->ticket, 1u);
        const int b = t < A.nbricks ? A.bricks[t] : 0;
        const int skip = (BAND && t < A.nbricks) ? (A.bcnt[b] == 0) : 0;
        s_tk[4 * st + 0] = t;
        s_tk[4 * st + 1] = b;
        s_tk[4 * st + 2] = skip;
        if (tma && t < A.nbricks && !skip) {
            const int bxi = b % A.nbx, q = b / A.nbx;
            const int ox = bxi * kBX - kHalo, oy = (q % A.nby) * kBY - kHalo, oz = (q / A.nby) * kBZ - kHalo;
            const unsigned bar = bar_of(st);
            fence_proxy_async();
            mbar_expect_tx(bar, (unsigned)((G::BoxN + G::DBoxN) * sizeof(T)));
            tma_load_3d(smem_addr(stage_u(st)), tmu, bar, ox, oy, oz);
            tma_load_3d(smem_addr(stage_d(st)), tmd, bar, ox, oy + kHalo - 1, oz + kHalo - 1);
        }
    };
    if (tma && tid == 0) {
        mbar_init(bar_of(0), 1);
        if (ST == 2) mbar_init(bar_of(1), 1);
        fence_mbar_init();
    }
    unsigned phases = 0u;  // bit s: parity of the next completion of stage s's barrier
    int st = 0;
    if (tid == 0) take(0);
    __syncthreads();
    for (;;) {
        const int t = s_tk[4 * st + 0];
        if (t >= A.nbricks) break;
        const int b = s_tk[4 * st + 1];
        const int skip = s_tk[4 * st + 2];
        // the other stage was released by the barrier that ended the previous brick
        if (pipe && tid == 0) take(st ^ 1);
        if (!skip) {
            T* su = stage_u(st);
            T* sd = stage_d(st);
            const int bxi = b % A.nbx, q = b / A.nbx;
            const int ox = bxi * kBX - kHalo, oy = (q % A.nby) * kBY - kHalo, oz = (q / A.nby) * kBZ - kHalo;
            // ---- 1. stage u (24x16x16 box) and d (24x10x10 box) ----
            bool staged = true;
            if (tma) {
                // one thread polls the barrier; the others wait at the block
                // barrier below without issuing
                if (tid == 0) {
                    const unsigned bar = bar_of(st);
                    long long it = 0;
                    const unsigned par = (phases >> st) & 1u;
                    while (!mbar_try_wait(bar, par) && ++it < kStageWaitLimit) {
                    }
                    staged = it < kStageWaitLimit;
                    if (!staged) {
                        // give the copies in flight a second bounded wait before leaving
                        long long it2 = 0;
                        while (!mbar_try_wait(bar, par) && ++it2 < kStageWaitLimit) {
                        }
                    }
                }
                phases ^= 1u << st;
            } else {
                brick_stage_copy<T, NT, true>(P, uin, d, su, sd, ox, oy, oz);
            }
            if (__syncthreads_or(!staged)) {
                if (tid == 0) atomicOr(&ds->error, kErrStage);
                if (pipe && tid == 0) {
                    // the prefetch of the other stage: a bounded wait, then leave
                    long long it3 = 0;
                    while (!mbar_try_wait(bar_of(st ^ 1), (phases >> (st ^ 1)) & 1u) && ++it3 < kStageWaitLimit) {
                    }
                }
                return;
            }
            // ---- 2.-4. band list, SL update and cut, Δ_φ partial and band count ----
            brick_compute<T, INTERP, BAND, NT>(P, A, su, sd, uin, uout, d, ds, Ep, invEp, b, ox, oy, oz, s_list,
                                               s_abs, s_cnt);
        }
        __syncthreads();
        if (!pipe) {
            // one stage: the next ticket (and its copies) once every thread is done with this brick
            if (tid == 0) take(st);
            __syncthreads();
        } else {
            st ^= 1;
        }
    }
}
// bricks holding a node with |u| < γ (band), or every brick (whole grid)
template <typename T>
struct BrickPred {
    const T* u;
    T gamma;
    int n0, n1, n2, nbx, nby;
    int band;
    __device__ bool operator()(long long b) const {
        if (!band) return true;
        const int bx = (int)(b % nbx), q = (int)(b / nbx);
        const int by = q % nby, bz = q / nby;
        for (int lz = 0; lz < kBZ; ++lz) {
            const int k = bz * kBZ + lz;
            if (k >= n2) break;
            for (int ly = 0; ly < kBY; ++ly) {
                const int j = by * kBY + ly;
                if (j >= n1) break;
                const long long row = (long long)n0 * (j + (long long)n1 * k);
                for (int lx = 0; lx < kBX; ++lx) {
                    const int i = bx * kBX + lx;
                    if (i >= n0) break;
                    if (fabs(u[row + i]) < gamma) return true;
                }
            }
        }
        return false;
    }
};

struct EmitIdx {
    int* out;
    __device__ void operator()(long long pos, long long i) const { out[pos] = (int)i; }
};

__global__ void k_fill_int(int* p, long long n, int v) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once (contexts may be set up
// from several threads at a time, as the server does)
EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    });
    return fn;
}

// tiled tensor map of a dense field (x fastest) with the given box
bool encode_field(CUtensorMap* m, void* base, const slr_ctx* c, unsigned bx, unsigned by, unsigned bz) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)c->cfg.n[0], (cuuint64_t)c->cfg.n[1], (cuuint64_t)c->cfg.n[2]};
    const cuuint64_t strides[2] = {(cuuint64_t)(c->cfg.n[0] * c->tsize),
                                   (cuuint64_t)(c->cfg.n[0] * c->cfg.n[1] * c->tsize)};
    const cuuint32_t box[3] = {bx, by, bz};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUtensorMapDataType dt = c->tsize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    return fn(m, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the launch shapes the autotuner chooses between: threads per block and
// pipeline stages (2: the next brick's boxes prefetched by TMA)
constexpr int kShapes = 4;
constexpr int kShapeNT[kShapes] = {256, 128, 256, 128};
constexpr int kShapeST[kShapes] = {1, 1, 2, 2};

template <typename T, int INTERP, int BAND, int NT, int ST>
cudaError_t brick_launch_t(slr_ctx* c, double ov, int shape) {
    using S = BrickSmem<T, ST>;
    auto kern = k_step_brick<T, INTERP, BAND, NT, ST>;
    BrickState& B = c->brick;
    if (B.occ[shape] == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, S::kBytes);
        if (e != cudaSuccess) return e;
        B.occ[shape] = occ > 0 ? occ : 1;
    }
    Params<T> P = make_params<T>(c);
    BrickArgs<T> A;
    A.nbricks = (int)B.nbricks;
    A.bricks = B.list;
    A.bcnt = B.cnt;
    A.part_dphi = B.part;
    A.nbx = B.nb[0];
    A.nby = B.nb[1];
    A.tma = B.tma;
    A.dt_h = (T)(c->dt / c->h);
    A.kdiff = (T)(c->cfg.delta * c->dt / (c->cfg.p * c->h * c->h));
    const double thr = c->cfg.c_sing * pow(c->dt, c->cfg.alpha);
    A.thr2 = (T)thr * (T)thr;
    long long grid = (long long)c->num_sms * B.occ[shape];
    if (grid > B.nbricks) grid = B.nbricks;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, NT, S::kBytes, c->stream>>>(B.tm_u[0], B.tm_u[1], B.tm_d, P, A, (T*)c->u[0], (T*)c->u[1],
                                                        (const T*)c->d, c->ds, ov);
    c->launches += 1;
    return cudaGetLastError();
}

template <typename T, int INTERP, int BAND>
cudaError_t brick_launch_s(slr_ctx* c, double ov, int shape) {
    switch (shape) {
        case 1: return brick_launch_t<T, INTERP, BAND, 128, 1>(c, ov, 1);
        case 2: return brick_launch_t<T, INTERP, BAND, 256, 2>(c, ov, 2);
        case 3: return brick_launch_t<T, INTERP, BAND, 128, 2>(c, ov, 3);
        default: return brick_launch_t<T, INTERP, BAND, 256, 1>(c, ov, 0);
    }
}

template <typename T>
cudaError_t brick_launch_p(slr_ctx* c, double ov, int shape) {
    const bool band = c->cfg.band != 0;
    if (c->cfg.interp) return band ? brick_launch_s<T, 1, 1>(c, ov, shape) : brick_launch_s<T, 1, 0>(c, ov, shape);
    return band ? brick_launch_s<T, 0, 1>(c, ov, shape) : brick_launch_s<T, 0, 0>(c, ov, shape);
}

cudaError_t brick_launch(slr_ctx* c, double ov, int shape) {
    return c->tsize == 4 ? brick_launch_p<float>(c, ov, shape) : brick_launch_p<double>(c, ov, shape);
}

// the active-brick list from field u (bricks with a node |u| < γ; every
// brick on the whole grid)
template <typename T>
cudaError_t bricks_build_t(slr_ctx* c, const void* u, long long* count, bool write) {
    BrickState& B = c->brick;
    BrickPred<T> pr{(const T*)u, (T)c->gamma, (int)c->cfg.n[0], (int)c->cfg.n[1], (int)c->cfg.n[2],
                    B.nb[0], B.nb[1], c->cfg.band};
    if (!write) return compact_count(c, pr, B.ntotal, count);
    return compact_write(c, pr, EmitIdx{B.list}, B.ntotal);
}

// band nodes {j : |u_j| < γ} of field u
template <typename T>
struct BandOf {
    const T* u;
    T gamma;
    __device__ bool operator()(long long i) const { return fabs(u[i]) < gamma; }
};

}  // namespace

// The brick step for 3-D runs without reinitialisation (where the band cannot
// leave the bricks of G̃^0), by cfg.step_kind. By rule (0): bricks, except a
// band run with the Q1 interpolator on a grid whose rows are not a multiple
// of 16 bytes. Such rows cannot be staged by TMA, and on GB300 the list step
// measured faster there (one iteration at 131^3: 62 against 69 µs; at 189^3:
// 89 against 102 µs), while WENO and TMA-staged grids favour the bricks.
bool brick_mode(const slr_ctx* c) {
    if (c->cfg.dim != 3 || c->cfg.reinit) return false;
    if (c->cfg.step_kind != 0) return c->cfg.step_kind == 1;
    const bool tma_rows = (c->cfg.n[0] * (long long)c->tsize) % 16 == 0;
    return !c->cfg.band || c->cfg.interp == 1 || tma_rows;
}

// Active bricks of field u (normally φ^0 in u[0]), the per-brick counters
// and partials (keyed by brick id over the whole grid, so the Δ_φ sum does
// not depend on which bricks are listed), and the tensor maps of the fields.
cudaError_t bricks_init(slr_ctx* c, const void* u) {
    BrickState& B = c->brick;
    B.ntotal = 1;
    for (int a = 0; a < 3; ++a) {
        const int bs = a == 0 ? kBX : (a == 1 ? kBY : kBZ);
        B.nb[a] = (int)((c->cfg.n[a] + bs - 1) / bs);
        B.ntotal *= B.nb[a];
    }
    bricks_free(c);
    long long cnt = 0;
    cudaError_t e = c->tsize == 4 ? bricks_build_t<float>(c, u, &cnt, false) : bricks_build_t<double>(c, u, &cnt, false);
    if (e != cudaSuccess) return e;
    B.list = (int*)dev_alloc(c, sizeof(int) * (cnt > 0 ? cnt : 1));
    B.cnt = (int*)dev_alloc(c, sizeof(int) * B.ntotal);
    B.part = (double*)dev_alloc(c, sizeof(double) * B.ntotal);
    if (!B.list || !B.cnt || !B.part) return cudaErrorMemoryAllocation;
    B.nbricks = cnt;
    if (cnt > 0) {
        e = c->tsize == 4 ? bricks_build_t<float>(c, u, &cnt, true) : bricks_build_t<double>(c, u, &cnt, true);
        if (e != cudaSuccess) return e;
    }
    // every listed brick runs at the next step; unlisted bricks add 0 to Δ_φ
    k_fill_int<<<(unsigned)((B.ntotal + 255) / 256), 256, 0, c->stream>>>(B.cnt, B.ntotal, 1);
    c->launches += 1;
    e = cudaMemsetAsync(B.part, 0, sizeof(double) * B.ntotal, c->stream);
    if (e != cudaSuccess) return e;
    // TMA needs 16-byte rows and 16-byte aligned bases
    const bool rows = (c->cfg.n[0] * (long long)c->tsize) % 16 == 0;
    const bool al = ((uintptr_t)c->u[0] % 16 == 0) && ((uintptr_t)c->u[1] % 16 == 0) && ((uintptr_t)c->d % 16 == 0);
    B.tma = 0;
    memset(B.tm_u, 0, sizeof(B.tm_u));
    memset(&B.tm_d, 0, sizeof(B.tm_d));
    if (rows && al) {
        const unsigned px = (unsigned)BoxGeom::X;
        bool ok = encode_field(&B.tm_u[0], c->u[0], c, px, kBox, kBox) &&
                  encode_field(&B.tm_u[1], c->u[1], c, px, kBox, kBox) && encode_field(&B.tm_d, c->d, c, px, kDY, kDY);
        B.tma = ok ? 1 : 0;
    }
    B.list_iter = -1;
    for (int i = 0; i < kShapes; ++i) B.occ[i] = 0;
    static_assert(kShapes <= (int)(sizeof(B.occ) / sizeof(B.occ[0])), "occupancy slot per shape");
    return cudaGetLastError();
}

// the launch shape with these threads per block and stages; -1 if none
int brick_shape_index(int threads, int stages) {
    for (int i = 0; i < kShapes; ++i)
        if (kShapeNT[i] == threads && kShapeST[i] == stages) return i;
    return -1;
}

void brick_shape_of(const slr_ctx* c, int* threads, int* stages, float* trial_ms) {
    const int sh = c->brick.shape;
    if (threads) *threads = kShapeNT[sh];
    if (stages) *stages = (kShapeST[sh] == 2 && c->brick.tma) ? 2 : 1;
    if (trial_ms) *trial_ms = c->brick.tuned_ms;
}

void bricks_free(slr_ctx* c) {
    BrickState& B = c->brick;
    if (B.list) dev_free(c, B.list);
    if (B.cnt) dev_free(c, B.cnt);
    if (B.part) dev_free(c, B.part);
    B.list = nullptr;
    B.cnt = nullptr;
    B.part = nullptr;
    B.nbricks = 0;
}

cudaError_t launch_step_brick(slr_ctx* c, double ov) {
    if (c->brick.nbricks <= 0) return cudaSuccess;
    return brick_launch(c, ov, c->brick.shape);
}

// The brick step's autotuner: times each launch shape (threads per block x
// pipeline stages; two stages only where TMA stages the boxes)
// on the current state and keeps the fastest.
// Every shape computes the same u^{n+1}, band count and Δ_φ partials (each
// node's arithmetic does not depend on the shape, and the partials are
// summed in list order), so the choice changes timing only. The trial
// launches write only the output buffer of the next step, which that step
// overwrites on every node they touched; the counters are reset after.
cudaError_t bricks_autotune(slr_ctx* c) {
    BrickState& B = c->brick;
    B.shape = 0;
    if (B.nbricks <= 0) return cudaSuccess;
    // without TMA the two-stage shapes run as one stage: the one-stage shapes only
    static const int kCand[] = {0, 1, 2, 3};
    const int* cand = kCand;
    const int nshapes = B.tma ? 4 : 2;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int ci = 0; ci < nshapes && e == cudaSuccess; ++ci) {
        const int sh = cand[ci];
        float ms = 0.f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            e = cudaMemsetAsync(&c->ds->ticket, 0, sizeof(unsigned), c->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
            if (e == cudaSuccess) e = brick_launch(c, -1.0, sh);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        }
        if (e == cudaSuccess && ms < best) {
            best = ms;
            B.shape = sh;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    c->launches -= 2 * nshapes;  // trial launches are not steps
    // back to the state after init: no ticket taken, every listed brick due, no
    // partials, no band count
    e = cudaMemsetAsync(&c->ds->ticket, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(&c->ds->band_brick, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B.part, 0, sizeof(double) * B.ntotal, c->stream);
    if (e == cudaSuccess) {
        k_fill_int<<<(unsigned)((B.ntotal + 255) / 256), 256, 0, c->stream>>>(B.cnt, B.ntotal, 1);
        e = cudaGetLastError();
    }
    B.tuned_ms = best;
    return e;
}

// {j : |u_j| < γ} of field u, ascending, into out (capacity band_cap); the
// count comes back to the host
cudaError_t band_of_field(slr_ctx* c, const void* u, int* out, long long* count) {
    cudaError_t e;
    if (c->tsize == 4) {
        BandOf<float> pr{(const float*)u, (float)c->gamma};
        e = compact_count(c, pr, c->N, count);
        if (e == cudaSuccess && *count > 0) e = compact_write(c, pr, EmitIdx{out}, c->N);
    } else {
        BandOf<double> pr{(const double*)u, c->gamma};
        e = compact_count(c, pr, c->N, count);
        if (e == cudaSuccess && *count > 0) e = compact_write(c, pr, EmitIdx{out}, c->N);
    }
    return e;
}

}  // namespace slr
