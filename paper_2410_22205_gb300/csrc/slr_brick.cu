// Brick-staged semi-Lagrangian step in 3-D (arXiv 2410.22205, §3.1 eq. SL3d
// and eq. sigma3d, §3.2 eqs. IQ1 and IWENO, §3.8 eqs. subgrid, cutoff and
// cut), for the narrow band and for the whole grid.
//
// The grid is cut into bricks of 8x8x8 nodes. At init the bricks that hold a
// node of the band G̃^0 (every brick on the whole grid) form a fixed list.
// Per iteration, one persistent launch hands the bricks out by ticket; for
// each brick a block
//   1. stages u^n on the brick plus a halo of 4 nodes (a 16^3 box) and d on
//      the brick plus 1 node in y and z (16x10x10) into shared memory: one
//      TMA tile load per box when rows are 16-byte aligned, 4- or 8-byte
//      cp.async copies with zero fill otherwise;
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
//      band; writes the brick's Δ_φ partial (FP64) and its band count.
// A brick whose band count was zero in the previous iteration has both
// buffers equal on all its nodes and is skipped.
#include <cuda.h>

#include "slr_compact.cuh"
#include "slr_internal.cuh"

namespace slr {

template <typename T>
Params<T> make_params(const slr_ctx* c);

namespace {

constexpr int kBr = 8;                            // nodes per axis of a brick
constexpr int kBrN = kBr * kBr * kBr;             // nodes per brick
constexpr int kHalo = 4;                          // staged halo of u per side
constexpr int kBox = kBr + 2 * kHalo;             // u box per axis (16)
constexpr int kBoxN = kBox * kBox * kBox;         // 4096
constexpr int kDY = kBr + 2;                      // d box along y and z (10); 16 along x (16-byte TMA rows)
constexpr int kDBoxN = kBox * kDY * kDY;          // 1600
constexpr int kBrickThreads = 256;
constexpr long long kStageWaitLimit = 1ll << 22;  // polls of one staging wait before it gives up

// dynamic shared memory of one block (bytes): u box, d box, member list,
// per-warp counts, the staging barrier and the ticket words
template <typename T>
struct BrickSmem {
    static constexpr int kU = 0;
    static constexpr int kD = kU + kBoxN * (int)sizeof(T);
    static constexpr int kList = kD + ((kDBoxN * (int)sizeof(T) + 127) & ~127);
    static constexpr int kCnt = kList + kBrN * 2;
    static constexpr int kRed = kCnt + 128;
    static constexpr int kBar = kRed + 64;
    static constexpr int kTicket = kBar + 16;
    static constexpr int kBytes = kTicket + 16;
};

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
    T yv[4][4];  // [column a][row b]: the z-line at (a, b)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        T r[4][4];  // [plane c][column a]
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int a = 0; a < 4; ++a) r[c][a] = base[a + kBox * b + kBox * kBox * c];
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
    const T v00 = base[0], v10 = base[1], v01 = base[kBox], v11 = base[kBox + 1];
    const T w00 = base[kBox * kBox], w10 = base[kBox * kBox + 1], w01 = base[kBox * kBox + kBox],
            w11 = base[kBox * kBox + kBox + 1];
    const T a0 = v00 + tx * (v10 - v00);
    const T a1 = v01 + tx * (v11 - v01);
    const T s0 = a0 + ty * (a1 - a0);
    const T c0 = w00 + tx * (w10 - w00);
    const T c1 = w01 + tx * (w11 - w01);
    const T s1 = c0 + ty * (c1 - c0);
    return s0 + tz * (s1 - s0);
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
    const T gx = diff_box(su, su_i, 1, i, P.n0, uc, P.inv_2h, P.inv_h);
    const T gy = diff_box(su, su_i, kBox, j, P.n1, uc, P.inv_2h, P.inv_h);
    const T gz = diff_box(su, su_i, kBox * kBox, k, P.n2, uc, P.inv_2h, P.inv_h);
    const T g2 = gx * gx + gy * gy + gz * gz;
    if (g2 < A.thr2) {
        // eq. SL:2: mean of the face neighbours inside the grid (-x,+x,-y,+y,-z,+z)
        T s = T(0);
        int cnt = 0;
        if (i > 0) { s += su[su_i - 1]; ++cnt; }
        if (i < P.n0 - 1) { s += su[su_i + 1]; ++cnt; }
        if (j > 0) { s += su[su_i - kBox]; ++cnt; }
        if (j < P.n1 - 1) { s += su[su_i + kBox]; ++cnt; }
        if (k > 0) { s += su[su_i - kBox * kBox]; ++cnt; }
        if (k < P.n2 - 1) { s += su[su_i + kBox * kBox]; ++cnt; }
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
    const T ddx = diff_box(sd, sd_i, 1, i, P.n0, dj, P.inv_2h, P.inv_h);
    const T ddy = diff_box(sd, sd_i, kBox, j, P.n1, dj, P.inv_2h, P.inv_h);
    const T ddz = diff_box(sd, sd_i, kBox * kDY, k, P.n2, dj, P.inv_2h, P.inv_h);
    // displacements in cells: advective C Δt ∇d / h, diffusive sqrt(C δ d Δt / p) / h
    const T adv = C * A.dt_h;
    const T bx = adv * ddx, by = adv * ddy, bz = adv * ddz;
    const T s = Norm<T>::root(C * dj * A.kdiff);
    // eq. sigma3d: ν1 = (-φz, 0, φx)/r, ν2 = (-φx φy, r^2, -φy φz)/(r |∇φ|),
    // r = sqrt(φx^2 + φz^2); (1,0,0), (0,0,1) when φx = φz = 0
    T n1x, n1z, n2x, n2y, n2z;
    const T w = gx * gx + gz * gz;
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
            const int off = su_i + (int)fx + kBox * (int)fy + kBox * kBox * (int)fz;
            const T tx = r[0] - fx, ty = r[1] - fy, tz = r[2] - fz;
            if (INTERP == 1) {
                WenoAxis<T> wx, wy, wz;
                wx.set(tx);
                wy.set(ty);
                wz.set(tz);
                last = weno_box(su + (off - 1 - kBox - kBox * kBox), wx, wy, wz, P.h4);
            } else {
                last = q1_box(su + off, tx, ty, tz);
            }
        } else {
            last = interp_at<T, 3, INTERP>(P, uin, i, j, k, r);
        }
        acc += last;
    }
    if (nfeet == 1) acc = ((last + last) + last) + last;
    return acc * T(0.25);
}

template <typename T, int INTERP, int BAND>
__global__ void __launch_bounds__(kBrickThreads, (INTERP == 1 ? (sizeof(T) == 8 ? 2 : 3) : (sizeof(T) == 8 ? 3 : 6)))
    k_step_brick(const __grid_constant__ CUtensorMap tm_u0, const __grid_constant__ CUtensorMap tm_u1,
                 const __grid_constant__ CUtensorMap tm_d, Params<T> P, BrickArgs<T> A, T* ub0, T* ub1,
                 const T* __restrict__ d, DevState* ds, double ep_override) {
    using S = BrickSmem<T>;
    extern __shared__ __align__(1024) unsigned char smem[];
    T* su = reinterpret_cast<T*>(smem + S::kU);
    T* sd = reinterpret_cast<T*>(smem + S::kD);
    unsigned short* s_list = reinterpret_cast<unsigned short*>(smem + S::kList);
    int* s_cnt = reinterpret_cast<int*>(smem + S::kCnt);
    int* s_tk = reinterpret_cast<int*>(smem + S::kTicket);
    const unsigned bar = smem_addr(smem + S::kBar);
    if (ds->stop) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = ds->n;
    const T* __restrict__ uin = (n & 1) ? ub1 : ub0;
    T* __restrict__ uout = (n & 1) ? ub0 : ub1;
    const CUtensorMap* tmu = (n & 1) ? &tm_u1 : &tm_u0;
    const T Ep = ep_override >= 0.0 ? (T)ep_override : (T)ds->Ep;
    const T invEp = Ep > T(0) ? T(1) / Ep : T(0);
    if (A.tma && tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    unsigned phase = 0;
    for (;;) {
        if (tid == 0) {
            const int t = (int)atomicAdd(&ds->ticket, 1u);
            s_tk[0] = t;
            s_tk[1] = t < A.nbricks ? A.bricks[t] : 0;
            s_tk[2] = (BAND && t < A.nbricks) ? (A.bcnt[s_tk[1]] == 0) : 0;
        }
        __syncthreads();
        const int t = s_tk[0];
        if (t >= A.nbricks) break;
        if (!s_tk[2]) {
            const int b = s_tk[1];
            const int bxi = b % A.nbx, q = b / A.nbx;
            const int byi = q % A.nby, bzi = q / A.nby;
            const int ox = bxi * kBr - kHalo, oy = byi * kBr - kHalo, oz = bzi * kBr - kHalo;
            // ---- 1. stage u (16^3 box) and d (16x10x10 box) ----
            bool staged = true;
            if (A.tma) {
                if (tid == 0) {
                    fence_proxy_async();
                    mbar_expect_tx(bar, (unsigned)((kBoxN + kDBoxN) * sizeof(T)));
                    tma_load_3d(smem_addr(su), tmu, bar, ox, oy, oz);
                    tma_load_3d(smem_addr(sd), &tm_d, bar, ox, oy + kHalo - 1, oz + kHalo - 1);
                }
                long long it = 0;
                while (!mbar_try_wait(bar, phase) && ++it < kStageWaitLimit) {
                }
                staged = it < kStageWaitLimit;
                if (!staged) {
                    // give the copies in flight a second bounded wait before leaving
                    long long it2 = 0;
                    while (!mbar_try_wait(bar, phase) && ++it2 < kStageWaitLimit) {
                    }
                }
                phase ^= 1u;
            } else {
                for (int e = tid; e < kBoxN; e += kBrickThreads) {
                    const int x = ox + (e & 15), y = oy + ((e >> 4) & 15), z = oz + (e >> 8);
                    const bool in = x >= 0 && x < P.n0 && y >= 0 && y < P.n1 && z >= 0 && z < P.n2;
                    const T* src = in ? uin + (x + P.is1 * y + P.is2 * z) : uin;
                    cp_async_zfill<(int)sizeof(T)>(smem_addr(su + e), src, in);
                }
                for (int e = tid; e < kDBoxN; e += kBrickThreads) {
                    const int x = ox + (e & 15), r = e >> 4;
                    const int y = oy + kHalo - 1 + r % kDY, z = oz + kHalo - 1 + r / kDY;
                    const bool in = x >= 0 && x < P.n0 && y >= 0 && y < P.n1 && z >= 0 && z < P.n2;
                    const T* src = in ? d + (x + P.is1 * y + P.is2 * z) : d;
                    cp_async_zfill<(int)sizeof(T)>(smem_addr(sd + e), src, in);
                }
                cp_async_wait_all();
            }
            if (__syncthreads_or(!staged)) {
                if (tid == 0) atomicOr(&ds->error, kErrStage);
                return;
            }
            // ---- 2. band nodes of the brick, in node order ----
            bool mem[2];
            T val[2];
            int gidx[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int l = tid + h * kBrickThreads;
                const int lx = l & 7, ly = (l >> 3) & 7, lz = l >> 6;
                const int i = ox + kHalo + lx, j = oy + kHalo + ly, k = oz + kHalo + lz;
                const bool in = i < P.n0 && j < P.n1 && k < P.n2;
                val[h] = su[(lx + kHalo) + kBox * (ly + kHalo) + kBox * kBox * (lz + kHalo)];
                gidx[h] = in ? i + P.is1 * j + P.is2 * k : -1;
                mem[h] = in && (!BAND || fabs(val[h]) < P.gamma);
                const unsigned m = __ballot_sync(0xffffffffu, mem[h]);
                if (lane == 0) s_cnt[h * 8 + warp] = __popc(m);
            }
            __syncthreads();
            if (tid == 0) {
                int run = 0;
                for (int w = 0; w < 16; ++w) {
                    const int c = s_cnt[w];
                    s_cnt[w] = run;
                    run += c;
                }
                s_cnt[16] = run;
            }
            __syncthreads();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const unsigned m = __ballot_sync(0xffffffffu, mem[h]);
                if (mem[h]) s_list[s_cnt[h * 8 + warp] + __popc(m & ((1u << lane) - 1u))] = (unsigned short)(tid + h * kBrickThreads);
                // nodes of the brick outside the band: u^{n+1} = u^n (both buffers agree there)
                if (BAND && gidx[h] >= 0 && !mem[h]) uout[gidx[h]] = val[h];
            }
            __syncthreads();
            const int count = s_cnt[16];
            // fast-path ranges of floor(displacement), relative to the node:
            // Q1 needs the cell c, c+1 in the box and c in [0, n-2];
            // WENO needs c-1 .. c+2 in the box and inside the grid
            const int lo_b = INTERP == 1 ? 1 : 0, hi_b = INTERP == 1 ? kBox - 3 : kBox - 2;
            const int lo_g = INTERP == 1 ? 1 : 0;
            const int bx_lo = max(lo_b, lo_g - ox), by_lo = max(lo_b, lo_g - oy), bz_lo = max(lo_b, lo_g - oz);
            const int hx = min(hi_b, (INTERP == 1 ? P.n0 - 3 : P.n0 - 2) - ox);
            const int hy = min(hi_b, (INTERP == 1 ? P.n1 - 3 : P.n1 - 2) - oy);
            const int hz = min(hi_b, (INTERP == 1 ? P.n2 - 3 : P.n2 - 2) - oz);
            // ---- 3. the SL update of the band nodes ----
            T dabs = T(0);
            for (int e = tid; e < count; e += kBrickThreads) {
                const int l = s_list[e];
                const int lx = (l & 7) + kHalo, ly = ((l >> 3) & 7) + kHalo, lz = (l >> 6) + kHalo;
                const int i = ox + lx, j = oy + ly, k = oz + lz;
                const int su_i = lx + kBox * ly + kBox * kBox * lz;
                const int sd_i = lx + kBox * (ly - kHalo + 1) + kBox * kDY * (lz - kHalo + 1);
                const T uc = su[su_i];
                const T flo[3] = {(T)(bx_lo - lx), (T)(by_lo - ly), (T)(bz_lo - lz)};
                const T fhi[3] = {(T)(hx - lx), (T)(hy - ly), (T)(hz - lz)};
                T out = brick_node<T, INTERP, BAND>(P, A, su, sd, uin, d, Ep, invEp, i, j, k, su_i, sd_i, flo, fhi, uc);
                if (BAND) out = fmin(fmax(out, -P.gamma), P.gamma);  // eq. cut
                uout[i + P.is1 * j + P.is2 * k] = out;
                dabs += fabs(out - uc);
            }
            // ---- 4. Δ_φ partial and band count of the brick ----
            dabs = warp_sum(dabs);
            double* s_red = reinterpret_cast<double*>(smem + S::kRed);
            if (lane == 0) s_red[warp] = (double)dabs;
            __syncthreads();
            if (tid == 0) {
                double sum = 0.0;
                for (int w = 0; w < kBrickThreads / 32; ++w) sum += s_red[w];
                A.part_dphi[b] = sum;
                A.bcnt[b] = count;
                if (BAND && count) atomicAdd(&ds->band_brick, count);
            }
        }
        __syncthreads();
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
        for (int lz = 0; lz < kBr; ++lz) {
            const int k = bz * kBr + lz;
            if (k >= n2) break;
            for (int ly = 0; ly < kBr; ++ly) {
                const int j = by * kBr + ly;
                if (j >= n1) break;
                const long long row = (long long)n0 * (j + (long long)n1 * k);
                for (int lx = 0; lx < kBr; ++lx) {
                    const int i = bx * kBr + lx;
                    if (i >= n0) break;
                    if (fabs(u[row + i]) < gamma) return true;
                }
            }
        }
        return false;
    }
};

__global__ void k_fill_int(int* p, long long n, int v) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        else
            cudaGetLastError();
    }
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

template <typename T, int INTERP, int BAND>
cudaError_t brick_launch_t(slr_ctx* c, double ov) {
    using S = BrickSmem<T>;
    auto kern = k_step_brick<T, INTERP, BAND>;
    BrickState& B = c->brick;
    if (B.occ[INTERP][BAND] == 0) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBytes);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBrickThreads, S::kBytes);
        if (e != cudaSuccess) return e;
        B.occ[INTERP][BAND] = occ > 0 ? occ : 1;
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
    long long grid = (long long)c->num_sms * B.occ[INTERP][BAND];
    if (grid > B.nbricks) grid = B.nbricks;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kBrickThreads, S::kBytes, c->stream>>>(B.tm_u[0], B.tm_u[1], B.tm_d, P, A, (T*)c->u[0],
                                                                   (T*)c->u[1], (const T*)c->d, c->ds, ov);
    c->launches += 1;
    return cudaGetLastError();
}

template <typename T>
cudaError_t brick_launch_p(slr_ctx* c, double ov) {
    const bool band = c->cfg.band != 0;
    if (c->cfg.interp) return band ? brick_launch_t<T, 1, 1>(c, ov) : brick_launch_t<T, 1, 0>(c, ov);
    return band ? brick_launch_t<T, 0, 1>(c, ov) : brick_launch_t<T, 0, 0>(c, ov);
}

struct EmitIdx {
    int* out;
    __device__ void operator()(long long pos, long long i) const { out[pos] = (int)i; }
};

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
        B.nb[a] = (int)((c->cfg.n[a] + kBr - 1) / kBr);
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
    memset(&B.tm_u[0], 0, sizeof(CUtensorMap));
    memset(&B.tm_u[1], 0, sizeof(CUtensorMap));
    memset(&B.tm_d, 0, sizeof(CUtensorMap));
    if (rows && al) {
        bool ok = encode_field(&B.tm_u[0], c->u[0], c, kBox, kBox, kBox) &&
                  encode_field(&B.tm_u[1], c->u[1], c, kBox, kBox, kBox) &&
                  encode_field(&B.tm_d, c->d, c, kBox, kDY, kDY);
        B.tma = ok ? 1 : 0;
    }
    B.list_iter = -1;
    return cudaGetLastError();
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
    return c->tsize == 4 ? brick_launch_p<float>(c, ov) : brick_launch_p<double>(c, ov);
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
