// Device code of the brick-staged semi-Lagrangian step in 3-D (arXiv
// 2410.22205, §3.1 eq. SL3d and eq. sigma3d, §3.2 eqs. IQ1 and IWENO, §3.8
// eqs. subgrid, cutoff and cut): box geometry, staging primitives (mbarrier,
// TMA tile load, cp.async), the SL update of one node from the staged boxes,
// and the work of one brick once its boxes are staged. Shared by the
// per-job step kernel (slr_brick.cu) and the batched persistent kernel
// (slr_batch.cuh); both translation units are compiled without implicit FMA
// contraction, so a brick computes the same bits in either.
#pragma once

#include <cuda.h>

#include "slr_internal.cuh"

namespace slr {
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

// Step 1 without TMA: the u box (24x16x16) and the d box (24x10x10) of the
// brick whose u box starts at node (ox, oy, oz), by 4- or 8-byte cp.async
// copies; nodes outside the grid are zero-filled. The boxes are rows of 24
// nodes along x. ROWS: each warp takes whole rows, lanes 0..23 one node each,
// so a row's y/z test and address are computed once per row (the per-job
// step: 6% (WENO) and 13% (Q1) shorter than the flat form on such grids).
// Otherwise the threads take consecutive nodes of the flattened box, all
// lanes busy (the batched kernel, where the row form measured 6% slower).
// Both fill the same shared memory.
template <typename T, int NT, bool ROWS>
__device__ __forceinline__ void brick_stage_copy(const Params<T>& P, const T* uin, const T* __restrict__ d, T* su,
                                                 T* sd, int ox, int oy, int oz) {
    using G = BoxGeom;
    constexpr int W = NT / 32;
    static_assert(G::X == 24 && kBox == 16 && kDY == 10, "row layout of the staged boxes");
    if (ROWS) {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane < G::X) {
            const int x = ox + lane;
            const bool xin = x >= 0 && x < P.n0;
            // u box: row r = y + 16 z (y, z from 0), origin (ox, oy, oz)
            for (int r = warp; r < kBox * kBox; r += W) {
                const int y = oy + (r & 15), z = oz + (r >> 4);
                const bool in = xin && y >= 0 && y < P.n1 && z >= 0 && z < P.n2;
                const T* src = in ? uin + (x + P.is1 * y + P.is2 * z) : uin;
                cp_async_zfill<(int)sizeof(T)>(smem_addr(su + r * G::X + lane), src, in);
            }
            // d box: row r = y + 10 z, origin (ox, oy + kHalo - 1, oz + kHalo - 1)
            for (int r = warp; r < kDY * kDY; r += W) {
                const int ry = r / kDY;
                const int y = oy + kHalo - 1 + (r - ry * kDY), z = oz + kHalo - 1 + ry;
                const bool in = xin && y >= 0 && y < P.n1 && z >= 0 && z < P.n2;
                const T* src = in ? d + (x + P.is1 * y + P.is2 * z) : d;
                cp_async_zfill<(int)sizeof(T)>(smem_addr(sd + r * G::X + lane), src, in);
            }
        }
    } else {
        for (int e = threadIdx.x; e < G::BoxN; e += NT) {
            const int r = e / G::X;
            const int x = ox + (e - r * G::X), y = oy + (r & 15), z = oz + (r >> 4);
            const bool in = x >= 0 && x < P.n0 && y >= 0 && y < P.n1 && z >= 0 && z < P.n2;
            const T* src = in ? uin + (x + P.is1 * y + P.is2 * z) : uin;
            cp_async_zfill<(int)sizeof(T)>(smem_addr(su + e), src, in);
        }
        for (int e = threadIdx.x; e < G::DBoxN; e += NT) {
            const int r = e / G::X;
            const int x = ox + (e - r * G::X);
            const int y = oy + kHalo - 1 + r % kDY, z = oz + kHalo - 1 + r / kDY;
            const bool in = x >= 0 && x < P.n0 && y >= 0 && y < P.n1 && z >= 0 && z < P.n2;
            const T* src = in ? d + (x + P.is1 * y + P.is2 * z) : d;
            cp_async_zfill<(int)sizeof(T)>(smem_addr(sd + e), src, in);
        }
    }
    cp_async_wait_all();
}

// Steps 2-4 for brick b (u box at node (ox, oy, oz), boxes staged in su and
// sd, every thread of the block calling): the band nodes of the brick in
// node order, the SL update and cut of each, u^n copied into u^{n+1} on the
// other nodes, the brick's Δ_φ partial (FP64, in list order, so that it does
// not depend on NT) and its band count. s_list (512 entries), s_abs (512)
// and s_cnt (NT/32 * 512/NT + 1 words) are shared-memory scratch.
template <typename T, int INTERP, int BAND, int NT>
__device__ __forceinline__ void brick_compute(const Params<T>& P, const BrickArgs<T>& A, const T* __restrict__ su,
                                              const T* __restrict__ sd, const T* __restrict__ uin,
                                              T* __restrict__ uout, const T* __restrict__ d, DevState* ds, T Ep,
                                              T invEp, int b, int ox, int oy, int oz, unsigned short* s_list,
                                              T* s_abs, int* s_cnt) {
    using G = BoxGeom;
    constexpr int W = NT / 32;      // warps per block
    constexpr int PER = kBrN / NT;  // nodes per thread in the compaction
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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

}  // namespace
}  // namespace slr
