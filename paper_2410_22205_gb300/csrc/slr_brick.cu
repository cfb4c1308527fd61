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

#include "slr_compact.cuh"
#include "slr_internal.cuh"

namespace slr {

template <typename T>
Params<T> make_params(const slr_ctx* c);

namespace {

constexpr int kBX = 8, kBY = 8, kBZ = 8;          // nodes of a brick per axis
constexpr int kBrN = kBX * kBY * kBZ;             // nodes per brick (512)
constexpr int kHalo = 4;                          // staged halo of u per side
constexpr int kBox = kBY + 2 * kHalo;             // u box along y and z (16)
constexpr int kDY = kBY + 2;                      // d box along y and z (10)
constexpr long long kStageWaitLimit = 1ll << 22;  // polls of one staging wait before it gives up

// Box geometry: both boxes are 24 nodes wide along x (kHalo = 4 on the left,
// the brick's 8, and 12 on the right), the row pitch in shared memory. The
// compacted node order puts a warp's 32 nodes in 4 rows of 8 at one z; with a
// pitch of 24 words those rows (and the feet, which move with their nodes)
// fall in 32 distinct banks, where a pitch of 16 would alias rows y and y+2.
// The 16-byte TMA rows need a width that is a multiple of 4 nodes.
struct BoxGeom {
    static constexpr int X = 24;                     // row pitch
    static constexpr int PY = X * kBox;              // u plane pitch
    static constexpr int BoxN = X * kBox * kBox;     // u box
    static constexpr int DPZ = X * kDY;              // d plane pitch
    static constexpr int DBoxN = X * kDY * kDY;      // d box
    static_assert((BoxN * 4) % 128 == 0 && (DBoxN * 4) % 128 == 0, "boxes keep 128-byte alignment");
};

// dynamic shared memory of one block (bytes): ST stages of (u box, d box),
// then the member list, the per-member |Δu|, per-warp counts, the staging
// barriers and the ticket words
template <typename T, int ST>
struct BrickSmem {
    using G = BoxGeom;
    static constexpr int kStage = (G::BoxN + G::DBoxN) * (int)sizeof(T);  // multiple of 128
    static constexpr int kList = ST * kStage;
    static constexpr int kAbs = kList + kBrN * 2;
    static constexpr int kCnt = kAbs + kBrN * (int)sizeof(T);
    static constexpr int kBar = kCnt + 256;
    static constexpr int kTicket = kBar + 16;
    static constexpr int kBytes = kTicket + 32;
};

// node l of a brick: x fastest, then y, then z
__device__ __forceinline__ void brick_local(int l, int& lx, int& ly, int& lz) {
    lx = l & 7;
    ly = (l >> 3) & 7;
    lz = l >> 6;
}
static_assert(kBX == 8 && kBY == 8 && kBZ == 8, "brick_local decodes 8x8x8 bricks");

// ---- staging primitives (inline PTX: mbarrier, TMA tile load, cp.async) ----
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// one tile of a 3-D tensor map into shared memory; x must be a multiple of
// 16 bytes / element size (the box origins here are multiples of 4 nodes)
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, unsigned bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(x), "r"(y), "r"(z)
        : "memory");
}
template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(unsigned dst, const void* src, bool valid) {
    const unsigned n = valid ? BYTES : 0u;  // 0 source bytes: the destination is zero-filled
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(dst), "l"(src), "n"(BYTES), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// FP32 normalisations with the hardware reciprocal square root (relative
// error ~1e-7, far inside the FP32 tolerance of 1e-5 h on u); FP64 keeps
// correctly rounded square roots and divisions
template <typename T>
struct Norm;
template <>
struct Norm<float> {
    static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float root(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
};
template <>
struct Norm<double> {
    static __device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }
    static __device__ __forceinline__ double root(double x) { return sqrt(x); }
};

// §3.2 WENO by dimension splitting (16 z-lines, 4 y-lines, 1 x-line) on a
// stencil that lies inside the staged box; base = node (c_x-1, c_y-1, c_z-1)
template <typename T>
__device__ __forceinline__ T weno_box(const T* __restrict__ base, const WenoAxis<T>& wx, const WenoAxis<T>& wy,
                                      const WenoAxis<T>& wz, T h4) {
    using G = BoxGeom;
    T yv[4][4];  // [column a][row b]: the z-line at (a, b)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        T r[4][4];  // [plane c][column a]
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int a = 0; a < 4; ++a) r[c][a] = base[a + G::X * b + G::PY * c];
        weno_pair(r[0][0], r[1][0], r[2][0], r[3][0], r[0][1], r[1][1], r[2][1], r[3][1], wz, h4, yv[0][b], yv[1][b]);
        weno_pair(r[0][2], r[1][2], r[2][2], r[3][2], r[0][3], r[1][3], r[2][3], r[3][3], wz, h4, yv[2][b], yv[3][b]);
    }
    T xv[4];
    weno_pair(yv[0][0], yv[0][1], yv[0][2], yv[0][3], yv[1][0], yv[1][1], yv[1][2], yv[1][3], wy, h4, xv[0], xv[1]);
    weno_pair(yv[2][0], yv[2][1], yv[2][2], yv[2][3], yv[3][0], yv[3][1], yv[3][2], yv[3][3], wy, h4, xv[2], xv[3]);
    return weno1(xv[0], xv[1], xv[2], xv[3], wx, h4);
}

// eq. IQ1 on a cell inside the staged box (lower corner at base): along x,
// then y, then z
template <typename T>
__device__ __forceinline__ T q1_box(const T* __restrict__ base, T tx, T ty, T tz) {
    using G = BoxGeom;
    const T v00 = base[0], v10 = base[1], v01 = base[G::X], v11 = base[G::X + 1];
    const T w00 = base[G::PY], w10 = base[G::PY + 1], w01 = base[G::PY + G::X], w11 = base[G::PY + G::X + 1];
    const T a0 = fma(tx, v10 - v00, v00);
    const T a1 = fma(tx, v11 - v01, v01);
    const T s0 = fma(ty, a1 - a0, a0);
    const T c0 = fma(tx, w10 - w00, w00);
    const T c1 = fma(tx, w11 - w01, w01);
    const T s1 = fma(ty, c1 - c0, c0);
    return fma(tz, s1 - s0, s0);
}

// centred difference along one axis from a staged box; one-sided first
// order on the domain boundary (the paper is silent there)
template <typename T>
__device__ __forceinline__ T diff_box(const T* __restrict__ s, int idx, int stride, int i, int n, T vc, T inv_2h,
                                      T inv_h) {
    const T up = s[idx + stride], um = s[idx - stride];
    if (i > 0 && i < n - 1) return (up - um) * inv_2h;
    return i == 0 ? (up - vc) * inv_h : (vc - um) * inv_h;
}

template <typename T>
struct BrickArgs {
    int nbricks;          // active bricks
    const int* bricks;    // their brick ids (x fastest over bricks)
    int* bcnt;            // per brick id: band count in the previous iteration
    double* part_dphi;    // per brick id: Δ_φ partial (0 for bricks never listed)
    int nbx, nby;         // bricks along x and y
    int tma;              // stage by TMA (16-byte rows and base addresses)
    T dt_h;               // Δt / h
    T kdiff;              // δ Δt / (p h^2): s^2 = C d kdiff, s the diffusive offset in cells
    T thr2;               // (C_sing Δt^α)^2
};

// §3.1 SL update of one band node from the staged boxes (before the cut).
// (i, j, k): the node; su_i / sd_i: its index in the u and d boxes;
// flo/fhi: per axis, the range of floor(displacement) for which the foot's
// stencil lies in the box and away from the grid edge.
template <typename T, int INTERP, int BAND>
__device__ __forceinline__ T brick_node(const Params<T>& P, const BrickArgs<T>& A, const T* __restrict__ su,
                                        const T* __restrict__ sd, const T* __restrict__ uin,
                                        const T* __restrict__ d, T Ep, T invEp, int i, int j, int k, int su_i,
                                        int sd_i, const T flo[3], const T fhi[3], T uc) {
    using G = BoxGeom;
    const bool inner = i > 0 && i < P.n0 - 1 && j > 0 && j < P.n1 - 1 && k > 0 && k < P.n2 - 1;
    T gx, gy, gz;
    if (inner) {
        gx = (su[su_i + 1] - su[su_i - 1]) * P.inv_2h;
        gy = (su[su_i + G::X] - su[su_i - G::X]) * P.inv_2h;
        gz = (su[su_i + G::PY] - su[su_i - G::PY]) * P.inv_2h;
    } else {
        gx = diff_box(su, su_i, 1, i, P.n0, uc, P.inv_2h, P.inv_h);
        gy = diff_box(su, su_i, G::X, j, P.n1, uc, P.inv_2h, P.inv_h);
        gz = diff_box(su, su_i, G::PY, k, P.n2, uc, P.inv_2h, P.inv_h);
    }
    const T g2 = fma(gx, gx, fma(gy, gy, gz * gz));
    if (g2 < A.thr2) {
        // eq. SL:2: mean of the face neighbours inside the grid (-x,+x,-y,+y,-z,+z)
        T s = T(0);
        int cnt = 0;
        if (i > 0) { s += su[su_i - 1]; ++cnt; }
        if (i < P.n0 - 1) { s += su[su_i + 1]; ++cnt; }
        if (j > 0) { s += su[su_i - G::X]; ++cnt; }
        if (j < P.n1 - 1) { s += su[su_i + G::X]; ++cnt; }
        if (k > 0) { s += su[su_i - G::PY]; ++cnt; }
        if (k < P.n2 - 1) { s += su[su_i + G::PY]; ++cnt; }
        return s / T(cnt);
    }
    const T dj = sd[sd_i];
    T C;
    if (P.p_kind == 1)
        C = T(1);
    else if (!(Ep > T(0)))
        C = T(0);
    else if (P.p_kind == 2)
        C = dj * invEp;
    else
        C = pow(dj / Ep, P.p - T(1));
    if (BAND) C *= cutoff(P, uc);
    T ddx, ddy, ddz;
    if (inner) {
        ddx = (sd[sd_i + 1] - sd[sd_i - 1]) * P.inv_2h;
        ddy = (sd[sd_i + G::X] - sd[sd_i - G::X]) * P.inv_2h;
        ddz = (sd[sd_i + G::DPZ] - sd[sd_i - G::DPZ]) * P.inv_2h;
    } else {
        ddx = diff_box(sd, sd_i, 1, i, P.n0, dj, P.inv_2h, P.inv_h);
        ddy = diff_box(sd, sd_i, G::X, j, P.n1, dj, P.inv_2h, P.inv_h);
        ddz = diff_box(sd, sd_i, G::DPZ, k, P.n2, dj, P.inv_2h, P.inv_h);
    }
    // displacements in cells: advective C Δt ∇d / h, diffusive sqrt(C δ d Δt / p) / h
    const T adv = C * A.dt_h;
    const T bx = adv * ddx, by = adv * ddy, bz = adv * ddz;
    const T s = Norm<T>::root(C * dj * A.kdiff);
    // eq. sigma3d: ν1 = (-φz, 0, φx)/r, ν2 = (-φx φy, r^2, -φy φz)/(r |∇φ|),
    // r = sqrt(φx^2 + φz^2); (1,0,0), (0,0,1) when φx = φz = 0
    T n1x, n1z, n2x, n2y, n2z;
    const T w = fma(gx, gx, gz * gz);
    if (gx == T(0) && gz == T(0)) {
        n1x = T(1); n1z = T(0);
        n2x = T(0); n2y = T(0); n2z = T(1);
    } else {
        const T irr = Norm<T>::rsq(w);
        const T ig = Norm<T>::rsq(g2);
        n1x = -gz * irr;
        n1z = gx * irr;
        const T q = irr * ig;
        n2x = -(gx * gy) * q;
        n2y = (w * irr) * ig;
        n2z = -(gy * gz) * q;
    }
    // δ = 0 (or C d = 0): the four feet coincide, so one interpolation
    // serves all of them, summed as in the general case
    const int nfeet = s == T(0) ? 1 : 4;
    const T ax = s * n1x, az = s * n1z;                 // s ν1 (its y component is 0)
    const T cx = s * n2x, cy = s * n2y, cz = s * n2z;   // s ν2
    T acc = T(0), last = T(0);
#pragma unroll 1
    for (int f = 0; f < nfeet; ++f) {
        // λ in the order (-,-), (-,+), (+,-), (+,+)
        const T l1 = (f & 2) ? T(1) : T(-1);
        const T l2 = (f & 1) ? T(1) : T(-1);
        T r[3] = {bx + (l1 * ax + l2 * cx), by + l2 * cy, bz + (l1 * az + l2 * cz)};
        const T fx = floor(r[0]), fy = floor(r[1]), fz = floor(r[2]);
        const bool fast = fx >= flo[0] && fx <= fhi[0] && fy >= flo[1] && fy <= fhi[1] && fz >= flo[2] &&
                          fz <= fhi[2];
        if (fast) {
            const int off = su_i + (int)fx + G::X * (int)fy + G::PY * (int)fz;
            const T tx = r[0] - fx, ty = r[1] - fy, tz = r[2] - fz;
            if (INTERP == 1) {
                WenoAxis<T> wx, wy, wz;
                wx.set(tx);
                wy.set(ty);
                wz.set(tz);
                last = weno_box<T>(su + (off - 1 - G::X - G::PY), wx, wy, wz, P.h4);
            } else {
                last = q1_box<T>(su + off, tx, ty, tz);
            }
        } else {
            last = interp_at<T, 3, INTERP>(P, uin, i, j, k, r);
        }
        acc += last;
    }
    if (nfeet == 1) acc = ((last + last) + last) + last;
    return acc * T(0.25);
}

// blocks per SM the launch bounds ask for: register budget of the scalar
// type and interpolator, scaled by the block size
template <typename T, int INTERP, int NT>
struct BrickOcc {
    static constexpr int v = (INTERP == 1 ? (sizeof(T) == 8 ? 2 : 3) : (sizeof(T) == 8 ? 3 : 4)) * (256 / NT);
};

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
    constexpr int W = NT / 32;    // warps per block
    constexpr int PER = kBrN / NT;  // nodes per thread in the compaction
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned short* s_list = reinterpret_cast<unsigned short*>(smem + S::kList);
    T* s_abs = reinterpret_cast<T*>(smem + S::kAbs);
    int* s_cnt = reinterpret_cast<int*>(smem + S::kCnt);
    int* s_tk = reinterpret_cast<int*>(smem + S::kTicket);  // per stage: ticket, brick id, skip
    if (ds->stop) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
                for (int e = tid; e < G::BoxN; e += NT) {
                    const int r = e / G::X;
                    const int x = ox + (e - r * G::X), y = oy + (r & 15), z = oz + (r >> 4);
                    const bool in = x >= 0 && x < P.n0 && y >= 0 && y < P.n1 && z >= 0 && z < P.n2;
                    const T* src = in ? uin + (x + P.is1 * y + P.is2 * z) : uin;
                    cp_async_zfill<(int)sizeof(T)>(smem_addr(su + e), src, in);
                }
                for (int e = tid; e < G::DBoxN; e += NT) {
                    const int r = e / G::X;
                    const int x = ox + (e - r * G::X);
                    const int y = oy + kHalo - 1 + r % kDY, z = oz + kHalo - 1 + r / kDY;
                    const bool in = x >= 0 && x < P.n0 && y >= 0 && y < P.n1 && z >= 0 && z < P.n2;
                    const T* src = in ? d + (x + P.is1 * y + P.is2 * z) : d;
                    cp_async_zfill<(int)sizeof(T)>(smem_addr(sd + e), src, in);
                }
                cp_async_wait_all();
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
            // ---- 2. band nodes of the brick, in node order ----
            bool mem[PER];
            T val[PER];
            int gidx[PER];
#pragma unroll
            for (int h = 0; h < PER; ++h) {
                const int l = tid + h * NT;
                int lx, ly, lz;
                brick_local(l, lx, ly, lz);
                const int i = ox + kHalo + lx, j = oy + kHalo + ly, k = oz + kHalo + lz;
                const bool in = i < P.n0 && j < P.n1 && k < P.n2;
                val[h] = su[(lx + kHalo) + G::X * (ly + kHalo) + G::PY * (lz + kHalo)];
                gidx[h] = in ? i + P.is1 * j + P.is2 * k : -1;
                mem[h] = in && (!BAND || fabs(val[h]) < P.gamma);
                const unsigned m = __ballot_sync(0xffffffffu, mem[h]);
                if (lane == 0) s_cnt[h * W + warp] = __popc(m);
            }
            __syncthreads();
            if (tid == 0) {
                int run = 0;
                for (int w = 0; w < kBrN / 32; ++w) {
                    const int c = s_cnt[w];
                    s_cnt[w] = run;
                    run += c;
                }
                s_cnt[kBrN / 32] = run;
            }
            __syncthreads();
#pragma unroll
            for (int h = 0; h < PER; ++h) {
                const unsigned m = __ballot_sync(0xffffffffu, mem[h]);
                if (mem[h]) s_list[s_cnt[h * W + warp] + __popc(m & ((1u << lane) - 1u))] = (unsigned short)(tid + h * NT);
                // nodes of the brick outside the band: u^{n+1} = u^n (both buffers agree there)
                if (BAND && gidx[h] >= 0 && !mem[h]) uout[gidx[h]] = val[h];
            }
            __syncthreads();
            const int count = s_cnt[kBrN / 32];
            // fast-path ranges of floor(displacement) in box coordinates:
            // Q1 needs the cell c, c+1 in the box and c in [0, n-2];
            // WENO needs c-1 .. c+2 in the box and inside the grid
            constexpr int lo_b = INTERP == 1 ? 1 : 0;
            constexpr int hx_b = INTERP == 1 ? G::X - 3 : G::X - 2, hb = INTERP == 1 ? kBox - 3 : kBox - 2;
            const int bx_lo = max(lo_b, lo_b - ox), by_lo = max(lo_b, lo_b - oy), bz_lo = max(lo_b, lo_b - oz);
            const int hx = min(hx_b, (INTERP == 1 ? P.n0 - 3 : P.n0 - 2) - ox);
            const int hy = min(hb, (INTERP == 1 ? P.n1 - 3 : P.n1 - 2) - oy);
            const int hz = min(hb, (INTERP == 1 ? P.n2 - 3 : P.n2 - 2) - oz);
            // ---- 3. the SL update of the band nodes ----
            for (int e = tid; e < count; e += NT) {
                const int l = s_list[e];
                int lx, ly, lz;
                brick_local(l, lx, ly, lz);
                lx += kHalo;
                ly += kHalo;
                lz += kHalo;
                const int i = ox + lx, j = oy + ly, k = oz + lz;
                const int su_i = lx + G::X * ly + G::PY * lz;
                const int sd_i = lx + G::X * (ly - kHalo + 1) + G::DPZ * (lz - kHalo + 1);
                const T uc = su[su_i];
                const T flo[3] = {(T)(bx_lo - lx), (T)(by_lo - ly), (T)(bz_lo - lz)};
                const T fhi[3] = {(T)(hx - lx), (T)(hy - ly), (T)(hz - lz)};
                T out = brick_node<T, INTERP, BAND>(P, A, su, sd, uin, d, Ep, invEp, i, j, k, su_i, sd_i, flo, fhi, uc);
                if (BAND) out = fmin(fmax(out, -P.gamma), P.gamma);  // eq. cut
                uout[i + P.is1 * j + P.is2 * k] = out;
                s_abs[e] = fabs(out - uc);
            }
            __syncthreads();
            // ---- 4. Δ_φ partial (FP64, in list order: independent of NT) and band count ----
            if (warp == 0) {
                double sum = 0.0;
                for (int e = lane; e < count; e += 32) sum += (double)s_abs[e];
                sum = warp_sum(sum);
                if (lane == 0) {
                    A.part_dphi[b] = sum;
                    A.bcnt[b] = count;
                    if (BAND && count) atomicAdd(&ds->band_brick, count);
                }
            }
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

bool brick_mode(const slr_ctx* c) { return c->cfg.dim == 3 && !c->cfg.reinit; }

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
