// Exact distance grid d(x_j) = min_Q |x_j - Q| with argmin (arXiv 2410.22205,
// §2 and §3.4; the paper computes exact values only near the cloud and fast
// sweeping elsewhere — here every node gets the exact value).
//
//  1. bounding box of the cloud (order-preserving integer atomics);
//  2. Morton code of each point's bin on a 2^L-per-axis bin grid over the
//     box, counting sort of the points by code (count, scan, scatter), so
//     consecutive points are spatially close;
//  3. a 32-ary box hierarchy over the sorted points: a leaf box per 32
//     consecutive points, a box per 32 consecutive boxes above, up to a top
//     level of at most 32 boxes; each leaf also gets a bounding cylinder
//     (centre, unit axis along the leaf's least-variance direction,
//     half-height, radius): on a surface cloud a leaf is a thin patch, and
//     the cylinder bounds the distance to it far more tightly than its box;
//  4. one warp per tile of 64 grid nodes (4x4x4 in 3-D, 8x8 in 2-D), two
//     nodes per lane one step apart along the last axis: a depth-first walk
//     of the hierarchy, nearest child first. A child box is pushed only if it
//     lies within the bound of the whole tile and of one of its eight 2x2x2
//     sub-tiles (each sub-tile's bound the largest current best of its
//     nodes); a popped leaf is screened only if, for some node, both its box
//     and its cylinder lie within that node's bound. At a screened leaf each
//     lane first takes the leaf's FP32 minimum for each node (a leaf whose
//     minimum passes no node's screen ends there), then re-checks in FP64 —
//     with the oracle's exact arithmetic, (x-qx)^2 + (y-qy)^2 + (z-qz)^2
//     without contraction — every point whose FP32 distance is within a
//     safety margin of both that minimum and the node's best. Ties go to the
//     lowest point index.
// The FP32 screen only discards points whose true distance exceeds the
// node's best (or the leaf's nearest) by more than the FP32 error bound
// (margin 1.2e-6 x (extent + d), about 6x the worst rounding), so the FP64
// decision is exact.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "slr_compact.cuh"
#include "slr_internal.cuh"

namespace slr {

template <typename T>
Params<T> make_params(const slr_ctx* c);

constexpr int kMaxLevels = 8;
constexpr int kStack = 256;
// widening of the exact search's FP32 screen for its expanded form (about 67 ulp)
constexpr float kWide = 4e-6f;
// block size and resident blocks per SM of the exact search
constexpr int kSearchThreads = 256;
constexpr int kSearchMinBlocks = 4;

__device__ __forceinline__ unsigned long long enc_double(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__host__ __device__ inline double dec_double(unsigned long long e) {
    unsigned long long b = (e >> 63) ? (e & 0x7fffffffffffffffull) : ~e;
    double x;
    memcpy(&x, &b, sizeof(double));
    return x;
}

// bbox[0..2] = min, bbox[3..5] = max (encoded); flag[0] = non-finite seen
__global__ void k_bbox(const double* pts, long long npts, int dim, unsigned long long* bbox, int* flag) {
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
    int bad = 0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < npts; q += (long long)gridDim.x * blockDim.x)
        for (int a = 0; a < dim; ++a) {
            double v = pts[q * dim + a];
            if (!isfinite(v)) {
                bad = 1;
                continue;
            }
            unsigned long long e = enc_double(v);
            mn[a] = e < mn[a] ? e : mn[a];
            mx[a] = e > mx[a] ? e : mx[a];
        }
    // warp reduction first: one atomic per warp instead of one per thread
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long m0 = __shfl_xor_sync(0xffffffffu, mn[a], o);
            const unsigned long long m1 = __shfl_xor_sync(0xffffffffu, mx[a], o);
            mn[a] = m0 < mn[a] ? m0 : mn[a];
            mx[a] = m1 > mx[a] ? m1 : mx[a];
        }
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < dim; ++a) {
            atomicMin(&bbox[a], mn[a]);
            atomicMax(&bbox[3 + a], mx[a]);
        }
        if (bad) atomicOr(flag, 1);
    }
}

__device__ __forceinline__ unsigned spread3(unsigned v) {  // 10 bits -> every third bit
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000FFu;
    v = (v | (v << 8)) & 0x0300F00Fu;
    v = (v | (v << 4)) & 0x030C30C3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__device__ __forceinline__ unsigned spread2(unsigned v) {  // 16 bits -> every second bit
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

struct BinArgs {
    double bmin[3];
    double inv_bin;
    int L;
    int dim;
};

__global__ void k_codes(const double* pts, long long npts, BinArgs B, unsigned* codes, int* counts) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npts) return;
    unsigned b[3] = {0, 0, 0};
    const int top = (1 << B.L) - 1;
    for (int a = 0; a < B.dim; ++a) {
        double t = (pts[q * B.dim + a] - B.bmin[a]) * B.inv_bin;
        int v = (int)floor(t);
        b[a] = (unsigned)(v < 0 ? 0 : (v > top ? top : v));
    }
    unsigned code = B.dim == 3 ? (spread3(b[0]) | (spread3(b[1]) << 1) | (spread3(b[2]) << 2))
                               : (spread2(b[0]) | (spread2(b[1]) << 1));
    codes[q] = code;
    atomicAdd(&counts[code], 1);
}

// exclusive scan of an int array, 4096 items per block
__global__ void __launch_bounds__(1024) k_scan_blocks(int* a, long long M, int* tot) {
    __shared__ int s[1024];
    long long beg = (long long)blockIdx.x * 4096 + threadIdx.x * 4;
    int v[4], local = 0;
    for (int i = 0; i < 4; ++i) {
        v[i] = beg + i < M ? a[beg + i] : 0;
        local += v[i];
    }
    s[threadIdx.x] = local;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        int x = threadIdx.x >= (unsigned)off ? s[threadIdx.x - off] : 0;
        __syncthreads();
        s[threadIdx.x] += x;
        __syncthreads();
    }
    int run = threadIdx.x ? s[threadIdx.x - 1] : 0;
    for (int i = 0; i < 4; ++i) {
        if (beg + i < M) a[beg + i] = run;
        run += v[i];
    }
    if (threadIdx.x == 1023) tot[blockIdx.x] = s[1023];
}

__global__ void k_scan_add(int* a, long long M, const int* tot) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M) a[i] += tot[i / 4096];
}

__global__ void k_scatter(const double* pts, long long npts, int dim, const unsigned* codes, int* offsets,
                          double o0, double o1, double o2, float4* spt) {
    long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= npts) return;
    int pos = atomicAdd(&offsets[codes[q]], 1);
    float4 r;
    r.x = (float)(pts[q * dim + 0] - o0);
    r.y = (float)(pts[q * dim + 1] - o1);
    r.z = dim == 3 ? (float)(pts[q * dim + 2] - o2) : 0.0f;
    r.w = __int_as_float((int)q);
    spt[pos] = r;
}

// one warp per box of level `lvl` (children: points at level 0, boxes above)
__global__ void k_boxes(const float4* spt, long long npts, float4* blo, float4* bhi, long long child_off,
                        long long child_cnt, long long own_off, long long own_cnt, int lvl) {
    long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= own_cnt) return;
    long long ch = w * 32 + lane;
    float lx = INFINITY, ly = INFINITY, lz = INFINITY, hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
    if (lvl == 0) {
        if (ch < npts) {
            float4 p = spt[ch];
            lx = hx = p.x;
            ly = hy = p.y;
            lz = hz = p.z;
        }
    } else if (ch < child_cnt) {
        float4 a = blo[child_off + ch], b = bhi[child_off + ch];
        lx = a.x; ly = a.y; lz = a.z;
        hx = b.x; hy = b.y; hz = b.z;
    }
    for (int o = 16; o > 0; o >>= 1) {
        lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
        ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
        lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
        hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
        hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
        hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
    }
    if (lane == 0) {
        blo[own_off + w] = make_float4(lx, ly, lz, 0.f);
        bhi[own_off + w] = make_float4(hx, hy, hz, 0.f);
    }
}

// One warp per leaf: its bounding cylinder, cyl[2 l] = (centre, half-height),
// cyl[2 l + 1] = (unit axis, radius). The axis is the least-variance
// direction of the leaf's points (any unit vector gives a valid bound; this
// one makes the cylinder thin on a surface patch). Half-height and radius are
// widened by 1e-5 relative plus `slack`, which covers the FP32 rounding of the
// point offsets and of the search's evaluation of the bound.
__global__ void k_leaf_cyl(const float4* spt, long long npts, int dim, long long nleaves, float slack, float4* cyl) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nleaves) return;
    const long long q = w * 32 + lane;
    const long long rem = npts - w * 32;
    const int cnt = rem < 32 ? (int)rem : 32;
    const bool have = lane < cnt;
    float4 p = have ? spt[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    float sx = p.x, sy = p.y, sz = p.z;
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    const float cx = sx / (float)cnt, cy = sy / (float)cnt, cz = dim == 3 ? sz / (float)cnt : 0.f;
    const float wx = have ? p.x - cx : 0.f, wy = have ? p.y - cy : 0.f, wz = have && dim == 3 ? p.z - cz : 0.f;
    float m[6] = {wx * wx, wx * wy, wx * wz, wy * wy, wy * wz, wz * wz};
    for (int k = 0; k < 6; ++k)
        for (int o = 16; o > 0; o >>= 1) m[k] += __shfl_xor_sync(0xffffffffu, m[k], o);
    double ax = 0.0, ay = 0.0, az = 1.0;
    if (lane == 0) {
        const double xx = m[0], xy = m[1], xz = m[2], yy = m[3], yz = m[4], zz = m[5];
        if (dim == 2) {
            // the normal of the 2-D patch: the eigenvector of the smaller
            // eigenvalue of [[xx, xy], [xy, yy]]
            const double hm = 0.5 * (xx + yy), hd = 0.5 * (xx - yy);
            const double lmin = hm - sqrt(hd * hd + xy * xy);
            double ux = xy, uy = lmin - xx, vx = lmin - yy, vy = xy;
            if (ux * ux + uy * uy < vx * vx + vy * vy) {
                ux = vx;
                uy = vy;
            }
            ax = ux;
            ay = uy;
            az = 0.0;
            if (ax * ax + ay * ay == 0.0) {
                ax = 1.0;
                ay = 0.0;
            }
        } else {
            // adj(M) = sum_i (product of the other two eigenvalues) v_i v_i^T:
            // its dominant direction is the least-variance one; its largest
            // column, refined by two products with adj(M)
            const double a00 = yy * zz - yz * yz, a01 = xz * yz - xy * zz, a02 = xy * yz - xz * yy;
            const double a11 = xx * zz - xz * xz, a12 = xy * xz - xx * yz, a22 = xx * yy - xy * xy;
            const double n0 = a00 * a00 + a01 * a01 + a02 * a02, n1 = a01 * a01 + a11 * a11 + a12 * a12,
                         n2 = a02 * a02 + a12 * a12 + a22 * a22;
            if (n0 >= n1 && n0 >= n2) {
                ax = a00; ay = a01; az = a02;
            } else if (n1 >= n2) {
                ax = a01; ay = a11; az = a12;
            } else {
                ax = a02; ay = a12; az = a22;
            }
            for (int it = 0; it < 2; ++it) {
                const double bx = a00 * ax + a01 * ay + a02 * az, by = a01 * ax + a11 * ay + a12 * az,
                             bz = a02 * ax + a12 * ay + a22 * az;
                const double nb = sqrt(bx * bx + by * by + bz * bz);
                if (!(nb > 0.0) || !isfinite(nb)) break;
                ax = bx / nb;
                ay = by / nb;
                az = bz / nb;
            }
            if (!(ax * ax + ay * ay + az * az > 0.0) || !isfinite(ax + ay + az)) {
                // a rank-1 or empty spread: the axis of least extent
                ax = (xx <= yy && xx <= zz) ? 1.0 : 0.0;
                ay = (ax == 0.0 && yy <= zz) ? 1.0 : 0.0;
                az = (ax == 0.0 && ay == 0.0) ? 1.0 : 0.0;
            }
        }
        const double na = sqrt(ax * ax + ay * ay + az * az);
        ax /= na;
        ay /= na;
        az /= na;
    }
    const float nx = (float)__shfl_sync(0xffffffffu, ax, 0), ny = (float)__shfl_sync(0xffffffffu, ay, 0),
                nz = (float)__shfl_sync(0xffffffffu, az, 0);
    float hh = 0.f, rr = 0.f;
    if (have) {
        const float an = fmaf(wx, nx, fmaf(wy, ny, wz * nz));
        const float px = fmaf(-an, nx, wx), py = fmaf(-an, ny, wy), pz = fmaf(-an, nz, wz);
        hh = fabsf(an);
        rr = sqrtf(fmaf(px, px, fmaf(py, py, pz * pz)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        hh = fmaxf(hh, __shfl_xor_sync(0xffffffffu, hh, o));
        rr = fmaxf(rr, __shfl_xor_sync(0xffffffffu, rr, o));
    }
    if (lane == 0) {
        cyl[2 * w] = make_float4(cx, cy, cz, fmaf(hh, 1.00001f, slack));
        cyl[2 * w + 1] = make_float4(nx, ny, nz, fmaf(rr, 1.00001f, slack));
    }
}

struct SearchArgs {
    int n0, n1, n2;
    int tx, ty, tz;        // tiles per axis
    double lo0, lo1, lo2, h;
    const float4* spt;
    const double* pts;
    long long npts;
    const float4* blo;
    const float4* bhi;
    const float4* cyl;     // leaf cylinders (k_leaf_cyl)
    int nlevels;
    long long off[kMaxLevels];
    long long cnt[kMaxLevels];
    double extent;         // coordinate extent used in the FP32 error margin
    int* flag;             // bit 2: traversal stack overflow
    const unsigned char* mask = nullptr;  // nodes to compute (nullptr: every node)
};

__device__ __forceinline__ float box_dist2(float tlx, float tly, float tlz, float thx, float thy, float thz,
                                           float4 lo, float4 hi) {
    float gx = fmaxf(0.f, fmaxf(lo.x - thx, tlx - hi.x));
    float gy = fmaxf(0.f, fmaxf(lo.y - thy, tly - hi.y));
    float gz = fmaxf(0.f, fmaxf(lo.z - thz, tlz - hi.z));
    return gx * gx + gy * gy + gz * gz;
}

__device__ __forceinline__ float tile_box_dist2(const float4* tb, float4 lo, float4 hi) {
    const float4 tl = tb[0], th = tb[1];
    return box_dist2(tl.x, tl.y, tl.z, th.x, th.y, th.z, lo, hi);
}

__device__ __forceinline__ float warp_maxf(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_minf(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sub-tiles of k_dist_search's tile: with 8, lanes that differ only in bits
// 0 and 2 (3-D: 2x2 in x and y) or 0 and 1 (2-D: 4 in x) share one; with 16,
// lanes that differ only in bit 0 (2 in x). kSubSecond is the second bit.
constexpr int kSubTiles = 8;
template <int DIM>
constexpr int kSubSecond = kSubTiles == 16 ? 0 : (DIM == 3 ? 4 : 2);

template <int DIM>
__device__ __forceinline__ int sub_of(int lane) {
    if (kSubTiles == 16) return lane >> 1;
    return DIM == 3 ? (((lane >> 1) & 1) | ((lane >> 2) & 6)) : (lane >> 2);
}

// The two nodes of lane `lane` in tile `tile` of k_dist_search: node a at
// (i, j, k), node b one step further along the last axis (z in 3-D, y in 2-D);
// pa, pb their indices along it. Out-of-grid nodes are clamped onto the grid
// (they only widen the tile) and marked invalid, as are unlisted nodes under a
// mask; idx_a, idx_b are the nodes' linear indices.
template <int DIM>
__device__ __forceinline__ void pair_node(const SearchArgs& A, long long tile, int lane, int& i, int& j, int& k,
                                          int& pa, int& pb, long long& idx_a, long long& idx_b, bool& valid_a,
                                          bool& valid_b) {
    const int ti = (int)(tile % A.tx);
    const long long r = tile / A.tx;
    const int tj = (int)(r % A.ty);
    const int tk = (int)(r / A.ty);
    if (DIM == 3) {
        i = ti * 4 + (lane & 3);
        j = tj * 4 + ((lane >> 2) & 3);
        k = tk * 4 + ((lane >> 4) << 1);
    } else {
        i = ti * 8 + (lane & 7);
        j = tj * 8 + ((lane >> 3) << 1);
        k = 0;
    }
    const int np_ = DIM == 3 ? A.n2 : A.n1;
    const int pa_ = DIM == 3 ? k : j;
    valid_a = i < A.n0 && j < A.n1 && k < A.n2;
    valid_b = valid_a && pa_ + 1 < np_;
    i = i < A.n0 ? i : A.n0 - 1;
    j = j < A.n1 ? j : A.n1 - 1;
    k = k < A.n2 ? k : A.n2 - 1;
    pa = pa_ < np_ ? pa_ : np_ - 1;
    pb = pa + 1 < np_ ? pa + 1 : np_ - 1;
    idx_a = (long long)i + (long long)A.n0 * ((long long)j + (long long)A.n1 * k);
    idx_b = idx_a + (long long)(pb - pa) * (DIM == 3 ? (long long)A.n0 * A.n1 : (long long)A.n0);
    if (A.mask) {
        valid_a = valid_a && A.mask[idx_a];
        valid_b = valid_b && A.mask[idx_b];
    }
}

// Each warp owns a tile of 64 nodes, two per lane: node a and node b one step
// further along the last axis (z in 3-D, y in 2-D). The pair shares its other
// coordinates, so the screen shares two of its three FMAs per point, and one
// walk of the tree, one leaf staging and one stack serve twice the nodes.
template <typename T, int DIM>
__global__ void __launch_bounds__(kSearchThreads, kSearchMinBlocks) k_dist_search(SearchArgs A, T* dout, int* aout) {
    __shared__ int s_stack[kSearchThreads / 32][kStack];
    __shared__ float4 s_leaf[kSearchThreads / 32][32];  // a leaf's points about the leaf centre, |q'|^2 in .w
    __shared__ int s_pid[kSearchThreads / 32][32];      // their input indices
    __shared__ float4 s_tbox[kSearchThreads / 32][2];  // the tile's box (low and high corners)
    // the tile's sub-tiles (kSubTiles): low corner with the largest pruning
    // bound of their nodes in .w, high corner
    __shared__ float4 s_sub[kSearchThreads / 32][kSubTiles][2];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long tile = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (tile >= (long long)A.tx * A.ty * A.tz) return;
    int* stack = s_stack[wib];
    int i, j, k, pa, pb;
    {
        long long idx_a, idx_b;
        bool valid_a, valid_b;
        pair_node<DIM>(A, tile, lane, i, j, k, pa, pb, idx_a, idx_b, valid_a, valid_b);
        // a warp with none of its nodes listed has nothing to do
        if (A.mask && !__any_sync(0xffffffffu, valid_a || valid_b)) return;
    }
    // exact node coordinates (lo + i*h, no contraction): x, the shared second
    // coordinate s (y in 3-D), the pair coordinates za, zb (z in 3-D, y in 2-D);
    // FP32 offsets from lo
    const double loP = DIM == 3 ? A.lo2 : A.lo1;
    const double x = __dadd_rn(A.lo0, __dmul_rn((double)i, A.h));
    const double s = DIM == 3 ? __dadd_rn(A.lo1, __dmul_rn((double)j, A.h)) : 0.0;
    const double za = __dadd_rn(loP, __dmul_rn((double)pa, A.h));
    const double zb = __dadd_rn(loP, __dmul_rn((double)pb, A.h));
    const float xf = (float)(x - A.lo0), sf = DIM == 3 ? (float)(s - A.lo1) : 0.f;
    const float zaf = (float)(za - loP), zbf = (float)(zb - loP);
    // the tile's box in (x, y, z) order, kept in shared memory for the
    // interior nodes' tests (registers are the scarce resource here)
    {
        float tlx, tly, tlz, thx, thy, thz;
        tlx = warp_minf(xf);
        thx = warp_maxf(xf);
        if (DIM == 3) {
            tly = warp_minf(sf);
            thy = warp_maxf(sf);
            tlz = warp_minf(zaf);
            thz = warp_maxf(zbf);
        } else {
            tly = warp_minf(zaf);
            thy = warp_maxf(zbf);
            tlz = thz = 0.f;
        }
        if (lane == 0) {
            s_tbox[wib][0] = make_float4(tlx, tly, tlz, 0.f);
            s_tbox[wib][1] = make_float4(thx, thy, thz, 0.f);
        }
        // the box of this lane's sub-tile
        float slx = fminf(xf, __shfl_xor_sync(0xffffffffu, xf, 1));
        float shx = fmaxf(xf, __shfl_xor_sync(0xffffffffu, xf, 1));
        float sly = DIM == 3 ? sf : zaf, shy = DIM == 3 ? sf : zbf;
        float slz = DIM == 3 ? zaf : 0.f, shz = DIM == 3 ? zbf : 0.f;
        sly = fminf(sly, __shfl_xor_sync(0xffffffffu, sly, 1));
        shy = fmaxf(shy, __shfl_xor_sync(0xffffffffu, shy, 1));
        slz = fminf(slz, __shfl_xor_sync(0xffffffffu, slz, 1));
        shz = fmaxf(shz, __shfl_xor_sync(0xffffffffu, shz, 1));
        constexpr int X2 = kSubSecond<DIM>;
        if (X2) {
            slx = fminf(slx, __shfl_xor_sync(0xffffffffu, slx, X2));
            shx = fmaxf(shx, __shfl_xor_sync(0xffffffffu, shx, X2));
            sly = fminf(sly, __shfl_xor_sync(0xffffffffu, sly, X2));
            shy = fmaxf(shy, __shfl_xor_sync(0xffffffffu, shy, X2));
            slz = fminf(slz, __shfl_xor_sync(0xffffffffu, slz, X2));
            shz = fmaxf(shz, __shfl_xor_sync(0xffffffffu, shz, X2));
        }
        if ((lane & (1 | X2)) == 0) {
            s_sub[wib][sub_of<DIM>(lane)][0] = make_float4(slx, sly, slz, INFINITY);
            s_sub[wib][sub_of<DIM>(lane)][1] = make_float4(shx, shy, shz, 0.f);
        }
        __syncwarp();
    }
    // the FP32 screen's margin, 1.2e-6 (extent + d): the FP32 offsets and
    // squared distances err by ~1e-7 extent, the FP32 square roots of the
    // bounds below by ~1e-7 d; bounds only screen, the decision is FP64
    const float mscale = 1.2e-6f;
    const float extf = (float)A.extent;

    double best_a = INFINITY, best_b = INFINITY;
    int bi_a = 0x7fffffff, bi_b = 0x7fffffff;
    float thr_a = INFINITY, thr_b = INFINITY;  // squared FP32 screens
    float lb_a = INFINITY, lb_b = INFINITY;    // bests plus the error margin (FP32)
    float wb2 = INFINITY;                      // squared warp bound
    float4* leaf = s_leaf[wib];
    int* lpid = s_pid[wib];

    int sp = 0;
    {
        const int top = A.nlevels - 1;
        long long c = lane;
        bool ex = c < A.cnt[top];
        float d2 = ex ? tile_box_dist2(s_tbox[wib], A.blo[A.off[top] + c], A.bhi[A.off[top] + c]) : INFINITY;
        unsigned m = __ballot_sync(0xffffffffu, ex);
        int np = __popc(m);
        int rank = 0;
        for (int s2 = 0; s2 < 32; ++s2) {
            float o = __shfl_sync(0xffffffffu, d2, s2);
            bool oex = (m >> s2) & 1u;
            if (oex && (o < d2 || (o == d2 && s2 < lane))) ++rank;
        }
        if (ex) stack[np - 1 - rank] = (top << 27) | (int)c;
        sp = np;
        __syncwarp();
    }
    while (sp > 0) {
        --sp;
        const int ent = stack[sp];
        __syncwarp();
        const int lvl = ent >> 27;
        const long long id = ent & ((1 << 27) - 1);
        if (lvl == 0) {
            // no tile-box test for a leaf: the per-lane test below implies it,
            // as no lane's bound exceeds the warp bound
            const float4 blo_ = A.blo[A.off[0] + id], bhi_ = A.bhi[A.off[0] + id];
            // per-lane test: skip the leaf when its box, or else its cylinder,
            // is beyond both nodes' own bounds of every lane
            {
                const float loP_ = DIM == 3 ? blo_.z : blo_.y, hiP_ = DIM == 3 ? bhi_.z : bhi_.y;
                const float gx = fmaxf(0.f, fmaxf(blo_.x - xf, xf - bhi_.x));
                const float gs = DIM == 3 ? fmaxf(0.f, fmaxf(blo_.y - sf, sf - bhi_.y)) : 0.f;
                const float gza = fmaxf(0.f, fmaxf(loP_ - zaf, zaf - hiP_));
                const float gzb = fmaxf(0.f, fmaxf(loP_ - zbf, zbf - hiP_));
                const float g2 = fmaf(gx, gx, gs * gs);
                bool need_a = !(fmaf(gza, gza, g2) > lb_a * lb_a);
                bool need_b = !(fmaf(gzb, gzb, g2) > lb_b * lb_b);
                if (!__any_sync(0xffffffffu, need_a || need_b)) continue;
                // the distance to a point of the leaf is at least that to the
                // cylinder: its axial excess over the half-height and its
                // radial excess over the radius, orthogonal components
                const float4 cc = A.cyl[2 * id], cn = A.cyl[2 * id + 1];
                const float ccP = DIM == 3 ? cc.z : cc.y, cnP = DIM == 3 ? cn.z : cn.y;
                const float wx = xf - cc.x, ws = DIM == 3 ? sf - cc.y : 0.f;
                const float cnS = DIM == 3 ? cn.y : 0.f;
                const float wza = zaf - ccP, wzb = zbf - ccP;
                const float ans = fmaf(wx, cn.x, ws * cnS);
                const float ana = fmaf(wza, cnP, ans), anb = fmaf(wzb, cnP, ans);
                const float pxa = fmaf(-ana, cn.x, wx), psa = fmaf(-ana, cnS, ws), pza = fmaf(-ana, cnP, wza);
                const float pxb = fmaf(-anb, cn.x, wx), psb = fmaf(-anb, cnS, ws), pzb = fmaf(-anb, cnP, wzb);
                const float gaa = fmaxf(0.f, fabsf(ana) - cc.w), gab = fmaxf(0.f, fabsf(anb) - cc.w);
                const float gra = fmaxf(0.f, sqrtf(fmaf(pxa, pxa, fmaf(psa, psa, pza * pza))) - cn.w);
                const float grb = fmaxf(0.f, sqrtf(fmaf(pxb, pxb, fmaf(psb, psb, pzb * pzb))) - cn.w);
                need_a = need_a && !(fmaf(gaa, gaa, gra * gra) > lb_a * lb_a);
                need_b = need_b && !(fmaf(gab, gab, grb * grb) > lb_b * lb_b);
                if (!__any_sync(0xffffffffu, need_a || need_b)) continue;
            }
            // The screen works about the leaf centre c: with u = x - c and
            // q' = q - c, |x - q|^2 = |u|^2 + (|q'|^2 - 2 u.q'), three FMAs per
            // point, the pair coordinate's last, so that nodes a and b share
            // the first two. Rounding u, q' and the expanded form moves the
            // squared distance by at most ~16 ulp (|x - q|^2 + e^2), e the
            // diagonal of the leaf's box; the screens widen by 4e-6 (thr + e^2).
            const float cx = 0.5f * (blo_.x + bhi_.x), cy = 0.5f * (blo_.y + bhi_.y), cz = 0.5f * (blo_.z + bhi_.z);
            const float ex_ = bhi_.x - blo_.x, ey_ = bhi_.y - blo_.y, ez_ = bhi_.z - blo_.z;
            const float we2 = kWide * (ex_ * ex_ + ey_ * ey_ + ez_ * ez_);
            const long long base = id * 32;
            long long rem = A.npts - base;
            const int cnt = rem < 32 ? (int)rem : 32;
            // a ragged last leaf is padded with points at infinite distance,
            // which no screen passes, so both passes run over 32 points
            if (lane < cnt) {
                const float4 p = A.spt[base + lane];
                const float qx = p.x - cx, qy = p.y - cy, qz = p.z - cz;
                leaf[lane] = make_float4(qx, qy, qz, fmaf(qx, qx, fmaf(qy, qy, qz * qz)));
                lpid[lane] = __float_as_int(p.w);
            } else {
                leaf[lane] = make_float4(0.f, 0.f, 0.f, INFINITY);
                lpid[lane] = 0x7fffffff;
            }
            __syncwarp();
            const float cP = DIM == 3 ? cz : cy;
            const float ux = xf - cx, us = DIM == 3 ? sf - cy : 0.f, uza = zaf - cP, uzb = zbf - cP;
            const float uxs = fmaf(ux, ux, us * us);
            const float uua = fmaf(uza, uza, uxs), uub = fmaf(uzb, uzb, uxs);
            const float ax = -2.f * ux, as = -2.f * us, aza = -2.f * uza, azb = -2.f * uzb;
            // The leaf's FP32 minimum first: it bounds the distance of the
            // leaf's nearest point, and any point beyond the margin of it is
            // strictly farther than that point, so only points within the
            // margin (and within the node's own best) need the FP64 check,
            // however the leaf's points are ordered.
            float tla, tlb;
            {
                float s2a = INFINITY, s2b = INFINITY;
#pragma unroll 8
                for (int t = 0; t < 32; ++t) {
                    const float4 q = leaf[t];
                    const float qP = DIM == 3 ? q.z : q.y;
                    const float cm = DIM == 3 ? fmaf(ax, q.x, fmaf(as, q.y, q.w)) : fmaf(ax, q.x, q.w);
                    s2a = fminf(s2a, fmaf(aza, qP, cm));
                    s2b = fminf(s2b, fmaf(azb, qP, cm));
                }
                const float m2a = fmaf(fmaxf(0.f, s2a + uua), 1.f + kWide, we2);
                const float m2b = fmaf(fmaxf(0.f, s2b + uub), 1.f + kWide, we2);
                const float mda = sqrtf(m2a), mdb = sqrtf(m2b);
                const float lima = mda + 2.0f * mscale * (extf + mda), limb = mdb + 2.0f * mscale * (extf + mdb);
                // this leaf's screens, moved to the side of the expanded form
                tla = fmaf(fminf(thr_a, lima * lima * 1.000002f), 1.f + kWide, we2) - uua;
                tlb = fmaf(fminf(thr_b, limb * limb * 1.000002f), 1.f + kWide, we2) - uub;
                // the second pass computes the same screen values: when no
                // node's smallest one passes, no point of the leaf does
                if (!__any_sync(0xffffffffu, s2a <= tla || s2b <= tlb)) continue;
            }
#pragma unroll 4
            for (int t = 0; t < 32; ++t) {
                const float4 q = leaf[t];
                const float qP = DIM == 3 ? q.z : q.y;
                const float cm = DIM == 3 ? fmaf(ax, q.x, fmaf(as, q.y, q.w)) : fmaf(ax, q.x, q.w);
                const bool ca = fmaf(aza, qP, cm) <= tla, cb = fmaf(azb, qP, cm) <= tlb;
                if (ca || cb) {
                    const int pid = lpid[t];
                    const double* Q = A.pts + (long long)pid * DIM;
                    const double ex = __dsub_rn(x, Q[0]);
                    const double ex2 = __dmul_rn(ex, ex);
                    double sxy = 0.0;
                    if (DIM == 3) {
                        const double ey = __dsub_rn(s, Q[1]);
                        sxy = __dadd_rn(ex2, __dmul_rn(ey, ey));
                    }
                    const double qz = Q[DIM - 1];
                    if (ca) {
                        const double ez = __dsub_rn(za, qz);
                        const double s2 = DIM == 3 ? __dadd_rn(sxy, __dmul_rn(ez, ez)) : __dadd_rn(ex2, __dmul_rn(ez, ez));
                        if (s2 < best_a || (s2 == best_a && pid < bi_a)) {
                            best_a = s2;
                            bi_a = pid;
                            const float bdist = sqrtf((float)s2);
                            const float lim = bdist + mscale * (extf + bdist);
                            thr_a = lim * lim * 1.000002f;
                            lb_a = lim * 1.000002f;
                            tla = fmaf(thr_a, 1.f + kWide, we2) - uua;
                        }
                    }
                    if (cb) {
                        const double ez = __dsub_rn(zb, qz);
                        const double s2 = DIM == 3 ? __dadd_rn(sxy, __dmul_rn(ez, ez)) : __dadd_rn(ex2, __dmul_rn(ez, ez));
                        if (s2 < best_b || (s2 == best_b && pid < bi_b)) {
                            best_b = s2;
                            bi_b = pid;
                            const float bdist = sqrtf((float)s2);
                            const float lim = bdist + mscale * (extf + bdist);
                            thr_b = lim * lim * 1.000002f;
                            lb_b = lim * 1.000002f;
                            tlb = fmaf(thr_b, 1.f + kWide, we2) - uub;
                        }
                    }
                }
            }
            {
                // the sub-tiles' bounds: the largest of their lanes' own
                constexpr int X2 = kSubSecond<DIM>;
                float v = fmaxf(lb_a, lb_b);
                v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, 1));
                if (X2) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, X2));
                if ((lane & (1 | X2)) == 0) s_sub[wib][sub_of<DIM>(lane)][0].w = v;
            }
            __syncwarp();
            const float wb = warp_maxf(fmaxf(lb_a, lb_b));
            wb2 = wb * wb;
        } else {
            if (tile_box_dist2(s_tbox[wib], A.blo[A.off[lvl] + id], A.bhi[A.off[lvl] + id]) > wb2) continue;
            const int cl = lvl - 1;
            const long long c = id * 32 + lane;
            const bool ex = c < A.cnt[cl];
            const float4 clo = ex ? A.blo[A.off[cl] + c] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 chi = ex ? A.bhi[A.off[cl] + c] : make_float4(0.f, 0.f, 0.f, 0.f);
            float d2 = ex ? tile_box_dist2(s_tbox[wib], clo, chi) : INFINITY;
            bool pass = ex && d2 <= wb2;
            if (pass) {
                // a child is pushed only if it lies within the bound of one of
                // the sub-tiles: no node is nearer to it than its sub-tile's
                // box, and no node's own bound exceeds its sub-tile's
                bool near = false;
#pragma unroll
                for (int t = 0; t < kSubTiles; ++t) {
                    const float4 sl = s_sub[wib][t][0], sh = s_sub[wib][t][1];
                    near = near || !(box_dist2(sl.x, sl.y, sl.z, sh.x, sh.y, sh.z, clo, chi) > sl.w * sl.w);
                }
                pass = near;
            }
            const unsigned m = __ballot_sync(0xffffffffu, pass);
            const int np = __popc(m);
            if (sp + np > kStack) {
                if (lane == 0) atomicOr(A.flag, 4);
                break;
            }
            // each passing child's rank among the passing ones (nearest last
            // on the stack, ties by lane), over the set bits of the ballot only
            int rank = 0;
            for (unsigned mm = m; mm; mm &= mm - 1) {
                const int o = __ffs(mm) - 1;
                const float od = __shfl_sync(0xffffffffu, d2, o);
                if (od < d2 || (od == d2 && o < lane)) ++rank;
            }
            if (pass) stack[sp + np - 1 - rank] = (cl << 27) | (int)c;
            sp += np;
            __syncwarp();
        }
    }
    // the nodes' indices again (cheaper than keeping them through the walk)
    long long idx_a, idx_b;
    bool valid_a, valid_b;
    pair_node<DIM>(A, tile, lane, i, j, k, pa, pb, idx_a, idx_b, valid_a, valid_b);
    if (valid_a) {
        dout[idx_a] = (T)sqrt(best_a);
        aout[idx_a] = bi_a;
    }
    if (valid_b) {
        dout[idx_b] = (T)sqrt(best_b);
        aout[idx_b] = bi_b;
    }
}

template <typename T, int DIM>
static void launch_search(slr_ctx* c, const SearchArgs& A) {
    long long ntiles = (long long)A.tx * A.ty * A.tz;
    long long blocks = (ntiles * 32 + kSearchThreads - 1) / kSearchThreads;
    k_dist_search<T, DIM><<<(unsigned)blocks, kSearchThreads, 0, c->stream>>>(A, (T*)c->d, c->argmin);
    c->launches += 1;
}

// the sorted cloud and its box hierarchy (scratch of one search)
struct CloudIndex {
    char* base = nullptr;  // the context path's allocation (nullptr for fixed scratch)
    int* flag = nullptr;
    float4* spt = nullptr;
    float4* blo = nullptr;
    float4* bhi = nullptr;
    float4* cyl = nullptr;
    int nlevels = 0;
    long long off[kMaxLevels], cnt[kMaxLevels];
    double extent = 0.0;
};

// device buffers of one index build
struct IndexScratch {
    unsigned long long* bbox;  // 6 words: encoded minima, then maxima
    int* flag;                 // error bits (non-finite point: k_bbox; stack overflow: the search)
    unsigned* codes;           // one bin code per point
    int* counts;               // one counter per bin (2^(dim L))
    int* tot;                  // scan partials
    float4* spt;               // sorted points (FP32 offsets from lo, index in w)
    float4* blo;               // box hierarchy: lower corners, then upper corners
    float4* cyl;               // leaf cylinders, two per leaf
};

// Level sizes of the 32-ary box hierarchy over npts points. False when the
// hierarchy would be deeper than kMaxLevels.
static bool hierarchy_sizes(long long npts, long long* cnt, long long* off, int* nlevels, long long* total_boxes) {
    int nl = 0;
    long long tot = 0;
    long long cc = (npts + 31) / 32;
    for (;;) {
        if (nl >= kMaxLevels) return false;
        cnt[nl] = cc;
        off[nl] = tot;
        tot += cc;
        ++nl;
        if (cc <= 32) break;
        cc = (cc + 31) / 32;
    }
    *nlevels = nl;
    *total_boxes = tot;
    return true;
}

// Builds the bin-sorted cloud and its box hierarchy in S, with 2^L bins per
// axis over the cloud's bounding box. X.nlevels/off/cnt must hold the sizes
// from hierarchy_sizes. lo, hi: the grid's corners (they bound the FP32
// offsets the search screens with). Waits on st for the bounding box;
// cudaErrorInvalidValue when a coordinate is not finite. *launches counts the
// kernels launched.
static cudaError_t build_index(const double* pts, long long npts, int dim, int L, const double lo[3],
                               const double hi[3], int num_sms, cudaStream_t st, const IndexScratch& S, CloudIndex& X,
                               long long* launches) {
    const long long nbins = 1ll << (dim * L);
    const long long nscan_blocks = (nbins + 4095) / 4096;
    long long total_boxes = 0;
    for (int l = 0; l < X.nlevels; ++l) total_boxes += X.cnt[l];
    X.flag = S.flag;
    X.spt = S.spt;
    X.blo = S.blo;
    X.bhi = S.blo + total_boxes;
    X.cyl = S.cyl;

    unsigned long long init_bbox[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
    unsigned long long hb[6];
    int hflag = 0;
    cudaError_t e = cudaMemcpyAsync(S.bbox, init_bbox, sizeof(init_bbox), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.flag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.counts, 0, sizeof(int) * nbins, st);
    if (e == cudaSuccess) {
        int blocks = (int)((npts + 255) / 256);
        if (blocks > num_sms * 8) blocks = num_sms * 8;
        k_bbox<<<blocks, 256, 0, st>>>(pts, npts, dim, S.bbox, S.flag);
        *launches += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb, S.bbox, sizeof(hb), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, S.flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (hflag) return cudaErrorInvalidValue;
    BinArgs B;
    double bmin[3] = {0, 0, 0}, bmax[3] = {0, 0, 0}, ext = 0.0;
    for (int a = 0; a < dim; ++a) {
        bmin[a] = dec_double(hb[a]);
        bmax[a] = dec_double(hb[3 + a]);
        ext = fmax(ext, bmax[a] - bmin[a]);
    }
    double bin = ext > 0 ? ext / (double)(1 << L) * (1.0 + 1e-9) : 1.0;
    for (int a = 0; a < 3; ++a) B.bmin[a] = bmin[a];
    B.inv_bin = 1.0 / bin;
    B.L = L;
    B.dim = dim;
    const double o0 = lo[0], o1 = lo[1], o2 = dim == 3 ? lo[2] : 0.0;
    double extent = 0.0;
    for (int a = 0; a < dim; ++a) {
        extent = fmax(extent, fabs(hi[a] - lo[a]));
        extent = fmax(extent, fabs(bmin[a] - lo[a]));
        extent = fmax(extent, fabs(bmax[a] - lo[a]));
    }
    X.extent = extent;
    int blocks = (int)((npts + 255) / 256);
    k_codes<<<blocks, 256, 0, st>>>(pts, npts, B, S.codes, S.counts);
    k_scan_blocks<<<(unsigned)nscan_blocks, 1024, 0, st>>>(S.counts, nbins, S.tot);
    k_scan_counts<<<1, 1024, 0, st>>>(S.tot, (int)nscan_blocks, (long long*)(S.tot + ((nscan_blocks + 2) & ~1ll)));
    k_scan_add<<<(unsigned)((nbins + 255) / 256), 256, 0, st>>>(S.counts, nbins, S.tot);
    k_scatter<<<blocks, 256, 0, st>>>(pts, npts, dim, S.codes, S.counts, o0, o1, o2, S.spt);
    *launches += 5;
    for (int l = 0; l < X.nlevels; ++l) {
        long long own = X.cnt[l];
        long long threads = own * 32;
        k_boxes<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
            S.spt, npts, X.blo, X.bhi, l == 0 ? 0 : X.off[l - 1], l == 0 ? npts : X.cnt[l - 1], X.off[l], own, l);
        *launches += 1;
    }
    // cylinder slack: the FP32 offsets of points and nodes err by ~1.2e-7
    // extent per coordinate, the search's evaluation of the axial and radial
    // components by ~1.5e-6 extent; 8e-6 extent covers both with room
    const float slack = (float)(8e-6 * (extent > 0.0 ? extent : 1.0));
    k_leaf_cyl<<<(unsigned)((X.cnt[0] * 32 + 255) / 256), 256, 0, st>>>(S.spt, npts, dim, X.cnt[0], slack, S.cyl);
    *launches += 1;
    return cudaGetLastError();
}

// bytes of the scan partials for 2^(dim L) bins (the second-level sums go
// after them, 8-byte aligned)
static size_t scan_tot_bytes(long long nbins) { return sizeof(int) * ((nbins + 4095) / 4096 + 2) + 16; }

static cudaError_t build_cloud_index(slr_ctx* c, CloudIndex& X) {
    const int dim = c->cfg.dim;
    const long long npts = c->npts;
    // bit-grid resolution: 2^L bins per axis
    const int L = dim == 3 ? 7 : 10;
    const long long nbins = 1ll << (dim * L);
    long long total_boxes = 0;
    if (!hierarchy_sizes(npts, X.cnt, X.off, &X.nlevels, &total_boxes)) return cudaErrorInvalidValue;
    // scratch layout
    size_t b_bbox = 64, b_flag = 16, b_codes = sizeof(unsigned) * npts, b_counts = sizeof(int) * nbins,
           b_tot = scan_tot_bytes(nbins), b_spt = sizeof(float4) * npts, b_boxes = sizeof(float4) * 2 * total_boxes,
           b_cyl = sizeof(float4) * 2 * X.cnt[0];
    auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
    size_t total =
        al(b_bbox) + al(b_flag) + al(b_codes) + al(b_counts) + al(b_tot) + al(b_spt) + al(b_boxes) + al(b_cyl);
    char* base = (char*)dev_alloc(c, total);
    if (!base) return cudaErrorMemoryAllocation;
    X.base = base;
    IndexScratch S;
    char* p = base;
    S.bbox = (unsigned long long*)p;
    p += al(b_bbox);
    S.flag = (int*)p;
    p += al(b_flag);
    S.codes = (unsigned*)p;
    p += al(b_codes);
    S.counts = (int*)p;
    p += al(b_counts);
    S.tot = (int*)p;
    p += al(b_tot);
    S.spt = (float4*)p;
    p += al(b_spt);
    S.blo = (float4*)p;
    p += al(b_boxes);
    S.cyl = (float4*)p;
    return build_index(c->pts, npts, dim, L, c->cfg.lo, c->cfg.hi, c->num_sms, c->stream, S, X, &c->launches);
}

// search arguments over a grid (n[2] = 1 in 2-D) and a built cloud index
static SearchArgs search_args(int dim, const int64_t n[3], const double lo[3], double h, const double* pts,
                              long long npts, const CloudIndex& X) {
    SearchArgs A;
    A.n0 = (int)n[0];
    A.n1 = (int)n[1];
    A.n2 = dim == 3 ? (int)n[2] : 1;
    // k_dist_search's tiles: 4x4x4 nodes in 3-D, 8x8 in 2-D
    if (dim == 3) {
        A.tx = (A.n0 + 3) / 4;
        A.ty = (A.n1 + 3) / 4;
        A.tz = (A.n2 + 3) / 4;
    } else {
        A.tx = (A.n0 + 7) / 8;
        A.ty = (A.n1 + 7) / 8;
        A.tz = 1;
    }
    A.lo0 = lo[0];
    A.lo1 = lo[1];
    A.lo2 = dim == 3 ? lo[2] : 0.0;
    A.h = h;
    A.spt = X.spt;
    A.pts = pts;
    A.npts = npts;
    A.blo = X.blo;
    A.bhi = X.bhi;
    A.cyl = X.cyl;
    A.nlevels = X.nlevels;
    for (int l = 0; l < kMaxLevels; ++l) {
        A.off[l] = l < X.nlevels ? X.off[l] : 0;
        A.cnt[l] = l < X.nlevels ? X.cnt[l] : 0;
    }
    A.extent = X.extent;
    A.flag = X.flag;
    return A;
}

static SearchArgs search_args(slr_ctx* c, const CloudIndex& X) {
    return search_args(c->cfg.dim, c->cfg.n, c->cfg.lo, c->h, c->pts, c->npts, X);
}

cudaError_t build_distance(slr_ctx* c) {
    const int dim = c->cfg.dim;
    cudaStream_t st = c->stream;
    CloudIndex X;
    cudaError_t e = build_cloud_index(c, X);
    char* base = X.base;
    int* flag = X.flag;
    int hflag = 0;
    if (e == cudaSuccess) {
        SearchArgs A = search_args(c, X);
        if (c->cfg.precision == 32) {
            if (dim == 3) launch_search<float, 3>(c, A);
            else launch_search<float, 2>(c, A);
        } else {
            if (dim == 3) launch_search<double, 3>(c, A);
            else launch_search<double, 2>(c, A);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(c, base);
    if (e == cudaSuccess && (hflag & 4)) return cudaErrorLaunchOutOfResources;
    return e;
}

cudaError_t distance_on_marked(slr_ctx* c, const unsigned char* mask, double* dout) {
    CloudIndex X;
    cudaError_t e = build_cloud_index(c, X);
    int hflag = 0;
    if (e == cudaSuccess) {
        SearchArgs A = search_args(c, X);
        A.mask = mask;
        const long long ntiles = (long long)A.tx * A.ty * A.tz;
        const unsigned blocks = (unsigned)((ntiles * 32 + kSearchThreads - 1) / kSearchThreads);
        if (c->cfg.dim == 3)
            k_dist_search<double, 3><<<blocks, kSearchThreads, 0, c->stream>>>(A, dout, c->argmin);
        else
            k_dist_search<double, 2><<<blocks, kSearchThreads, 0, c->stream>>>(A, dout, c->argmin);
        c->launches += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, X.flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, X.base);
    if (e == cudaSuccess && (hflag & 4)) return cudaErrorLaunchOutOfResources;
    return e;
}

}  // namespace slr

// ---------------------------------------------------------------------------
// Distance grid for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc: code that runs while
// another framework owns all of the device memory through its own pool,
// real-time loops that must not allocate after start-up, or plug-ins handed
// only pre-allocated buffers. slr_distance_grid_noalloc computes the same
// d and argmin as slr_build_distance from caller-owned device buffers and
// keeps its scratch (point codes, bin counts, sorted points, box hierarchy)
// in the fixed array below, which every GPU that loads the library holds
// until the process exits.
// ---------------------------------------------------------------------------
namespace slr {
namespace {

constexpr long long kNoAllocMaxPoints = 1ll << 16;  // 65,536 points
constexpr int kNoAllocL3 = 6;                         // 2^6 bins per axis in 3-D
constexpr int kNoAllocL2 = 9;                         // 2^9 bins per axis in 2-D
constexpr long long kNoAllocBins = 1ll << 18;         // both cases
constexpr long long kNoAllocScanBlocks = (kNoAllocBins + 4095) / 4096;
constexpr size_t al256(size_t v) { return (v + 255) & ~size_t(255); }
constexpr long long kNoAllocBoxes = (kNoAllocMaxPoints + 31) / 32 + (kNoAllocMaxPoints + 1023) / 1024 + 8;
constexpr size_t kOffBbox = 0;
constexpr size_t kOffFlag = kOffBbox + al256(64);
constexpr size_t kOffCodes = kOffFlag + al256(16);
constexpr size_t kOffCounts = kOffCodes + al256(sizeof(unsigned) * kNoAllocMaxPoints);
constexpr size_t kOffTot = kOffCounts + al256(sizeof(int) * kNoAllocBins);
constexpr size_t kOffSpt = kOffTot + al256(sizeof(int) * (kNoAllocScanBlocks + 2) + 16);
constexpr size_t kOffBoxes = kOffSpt + al256(sizeof(float4) * kNoAllocMaxPoints);
constexpr size_t kOffCyl = kOffBoxes + al256(sizeof(float4) * 2 * kNoAllocBoxes);
constexpr size_t kNoAllocScratchBytes = kOffCyl + al256(sizeof(float4) * 2 * ((kNoAllocMaxPoints + 31) / 32));  // ~2.5 MB

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};  // device address of g_noalloc_scratch, per device

slr_status noalloc_fail(slr_status s, const std::string& m) { return ctxless_error_set(s, m); }

}  // namespace

}  // namespace slr

extern "C" slr_status slr_distance_grid_noalloc(int dim, const int64_t n[3], const double lo[3], double h, int precision,
                                                const double* pts_dev, int64_t n_points, void* d_dev,
                                                int32_t* argmin_dev, void* cuda_stream) {
    using namespace slr;
    ctxless_error_clear();
    if (dim != 2 && dim != 3) return noalloc_fail(SLR_E_INVALID, "distance_grid_noalloc: dim must be 2 or 3");
    if (!n || !lo || !pts_dev || !d_dev || !argmin_dev)
        return noalloc_fail(SLR_E_INVALID, "distance_grid_noalloc: null argument");
    if (precision != 32 && precision != 64)
        return noalloc_fail(SLR_E_INVALID, "distance_grid_noalloc: precision must be 32 or 64");
    if (n_points < 1 || n_points > kNoAllocMaxPoints)
        return noalloc_fail(SLR_E_INVALID, "distance_grid_noalloc: n_points must be in 1..65536 (the fixed scratch "
                                           "holds at most 65536 points; use slr_build_distance for larger clouds)");
    long long N = 1;
    for (int a = 0; a < dim; ++a) {
        if (n[a] < 2) return noalloc_fail(SLR_E_INVALID, "distance_grid_noalloc: need at least 2 nodes per axis");
        // bounded before the product, which therefore cannot overflow
        if (n[a] > 2147483647ll / N) return noalloc_fail(SLR_E_INVALID, "distance_grid_noalloc: at most 2^31-1 nodes");
        N *= n[a];
    }
    if (dim == 3 ? false : (n[2] != 1))
        return noalloc_fail(SLR_E_INVALID, "distance_grid_noalloc: n[2] must be 1 in 2-D");
    if (!(h > 0.0)) return noalloc_fail(SLR_E_INVALID, "distance_grid_noalloc: h must be > 0");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the call reads results back to the host and waits on the stream, which
    // a stream capture cannot record
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(SLR_E_CUDA, "distance_grid_noalloc: invalid stream");
    }
    if (cap != cudaStreamCaptureStatusNone)
        return noalloc_fail(SLR_E_INVALID, "distance_grid_noalloc: the call is synchronous and cannot be captured");

    // per-device set-up: the host-side name of the array is not a device
    // address; ask the runtime for this device's address once
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return noalloc_fail(SLR_E_CUDA, "distance_grid_noalloc: no usable current device");
    }
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return noalloc_fail(SLR_E_CUDA, std::string("distance_grid_noalloc: cudaGetSymbolAddress: ") +
                                                    cudaGetErrorString(e));
            }
            g_noalloc_ptr[dev] = p;
        }
        base = (unsigned char*)g_noalloc_ptr[dev];
    }
    IndexScratch S;
    S.bbox = (unsigned long long*)(base + kOffBbox);
    S.flag = (int*)(base + kOffFlag);
    S.codes = (unsigned*)(base + kOffCodes);
    S.counts = (int*)(base + kOffCounts);
    S.tot = (int*)(base + kOffTot);
    S.spt = (float4*)(base + kOffSpt);
    S.blo = (float4*)(base + kOffBoxes);
    S.cyl = (float4*)(base + kOffCyl);

    const long long npts = n_points;
    const int L = dim == 3 ? kNoAllocL3 : kNoAllocL2;
    CloudIndex X;
    long long total_boxes = 0;
    if (!hierarchy_sizes(npts, X.cnt, X.off, &X.nlevels, &total_boxes) || total_boxes > kNoAllocBoxes)
        return noalloc_fail(SLR_E_INVALID, "distance_grid_noalloc: box hierarchy larger than the fixed scratch");
    int num_sms = 0;
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (num_sms <= 0) num_sms = 1;
    double hi[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < dim; ++a) hi[a] = lo[a] + (double)(n[a] - 1) * h;
    long long launches = 0;
    // the array keeps the previous call's contents: build_index resets what
    // must start at zero (bounding box, flag, bin counters)
    e = build_index(pts_dev, npts, dim, L, lo, hi, num_sms, st, S, X, &launches);
    if (e == cudaErrorInvalidValue) {
        cudaGetLastError();
        return noalloc_fail(SLR_E_INVALID, "distance_grid_noalloc: non-finite point coordinates");
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(SLR_E_CUDA, std::string("distance_grid_noalloc: ") + cudaGetErrorString(e));
    }
    SearchArgs A = search_args(dim, n, lo, h, pts_dev, npts, X);
    long long ntiles = (long long)A.tx * A.ty * A.tz;
    unsigned sblocks = (unsigned)((ntiles * 32 + kSearchThreads - 1) / kSearchThreads);
    if (precision == 32) {
        if (dim == 3)
            k_dist_search<float, 3><<<sblocks, kSearchThreads, 0, st>>>(A, (float*)d_dev, argmin_dev);
        else
            k_dist_search<float, 2><<<sblocks, kSearchThreads, 0, st>>>(A, (float*)d_dev, argmin_dev);
    } else {
        if (dim == 3)
            k_dist_search<double, 3><<<sblocks, kSearchThreads, 0, st>>>(A, (double*)d_dev, argmin_dev);
        else
            k_dist_search<double, 2><<<sblocks, kSearchThreads, 0, st>>>(A, (double*)d_dev, argmin_dev);
    }
    int hflag = 0;
    int* flag = S.flag;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return noalloc_fail(SLR_E_CUDA, std::string("distance_grid_noalloc: ") + cudaGetErrorString(e));
    }
    if (hflag & 4) return noalloc_fail(SLR_E_CUDA, "distance_grid_noalloc: traversal stack overflow");
    return SLR_OK;
}

// ---------------------------------------------------------------------------
// Cloud spacing h_S (§4, eq. dxdt): the mean, over a sample of the cloud, of
// the distance from each sampled point to its nearest other point. The
// sampled points are queried in the order of the sorted cloud, so that the
// 32 queries of a warp are neighbours; each lane skips its own point. The
// distances are those of the distance grid (FP32 screen, exact FP64 check of
// (x-qx)^2 + (y-qy)^2 + (z-qz)^2); the mean is summed in sample order.
// ---------------------------------------------------------------------------

namespace slr {

namespace {

struct SampledPred {
    const float4* spt;
    const int* mark;
    __device__ bool operator()(long long t) const { return mark[__float_as_int(spt[t].w)] != 0; }
};

struct SampledEmit {
    const float4* spt;
    const int* mark;
    int* out;
    __device__ void operator()(long long pos, long long t) const { out[pos] = mark[__float_as_int(spt[t].w)] - 1; }
};

__global__ void k_mark_sample(const long long* sample, long long m, int* mark) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < m; s += (long long)gridDim.x * blockDim.x)
        mark[sample[s]] = (int)s + 1;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_point_nn(SearchArgs A, const int* __restrict__ qpos,
                                                  const long long* __restrict__ sample, long long m, double* dist) {
    __shared__ int s_stack[8][kStack];
    __shared__ float4 s_leaf[8][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const long long qb = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (qb * 32 >= m) return;
    int* stack = s_stack[wib];
    const long long qi = qb * 32 + lane;
    const bool valid = qi < m;
    const long long qs = qpos[valid ? qi : m - 1];
    const int self = (int)sample[qs];
    const double* P0 = A.pts + (long long)self * DIM;
    const double x = P0[0], y = P0[1], z = DIM == 3 ? P0[2] : 0.0;
    const float xf = (float)(x - A.lo0), yf = (float)(y - A.lo1), zf = DIM == 3 ? (float)(z - A.lo2) : 0.f;
    const float tlx = warp_minf(xf), tly = warp_minf(yf), tlz = warp_minf(zf);
    const float thx = warp_maxf(xf), thy = warp_maxf(yf), thz = warp_maxf(zf);
    // the FP32 screen's margin, 1.2e-6 (extent + d): the FP32 offsets and
    // squared distances err by ~1e-7 extent, the FP32 square roots of the
    // bounds below by ~1e-7 d; bounds only screen, the decision is FP64
    const float mscale = 1.2e-6f;
    const float extf = (float)A.extent;
    double best = INFINITY;
    float thr = INFINITY, lbound = INFINITY, wb2 = INFINITY;
    float4* leaf = s_leaf[wib];
    int sp = 0;
    {
        const int top = A.nlevels - 1;
        const long long c = lane;
        const bool ex = c < A.cnt[top];
        const float d2 = ex ? box_dist2(tlx, tly, tlz, thx, thy, thz, A.blo[A.off[top] + c], A.bhi[A.off[top] + c])
                            : INFINITY;
        const unsigned msk = __ballot_sync(0xffffffffu, ex);
        const int np = __popc(msk);
        int rank = 0;
        for (int s = 0; s < 32; ++s) {
            const float o = __shfl_sync(0xffffffffu, d2, s);
            if (((msk >> s) & 1u) && (o < d2 || (o == d2 && s < lane))) ++rank;
        }
        if (ex) stack[np - 1 - rank] = (top << 27) | (int)c;
        sp = np;
        __syncwarp();
    }
    while (sp > 0) {
        --sp;
        const int ent = stack[sp];
        __syncwarp();
        const int lvl = ent >> 27;
        const long long id = ent & ((1 << 27) - 1);
        const float bd2 = box_dist2(tlx, tly, tlz, thx, thy, thz, A.blo[A.off[lvl] + id], A.bhi[A.off[lvl] + id]);
        if (bd2 > wb2) continue;
        if (lvl == 0) {
            {
                const float4 blo_ = A.blo[A.off[0] + id], bhi_ = A.bhi[A.off[0] + id];
                const float gx = fmaxf(0.f, fmaxf(blo_.x - xf, xf - bhi_.x));
                const float gy = fmaxf(0.f, fmaxf(blo_.y - yf, yf - bhi_.y));
                const float gz = fmaxf(0.f, fmaxf(blo_.z - zf, zf - bhi_.z));
                const bool need = !(gx * gx + gy * gy + gz * gz > lbound * lbound);
                if (!__any_sync(0xffffffffu, need)) continue;
            }
            const long long base = id * 32;
            const long long rem = A.npts - base;
            const int cnt = rem < 32 ? (int)rem : 32;
            if (lane < cnt) leaf[lane] = A.spt[base + lane];
            __syncwarp();
            if (best == INFINITY) {
                float m2 = INFINITY;
                for (int s = 0; s < cnt; ++s) {
                    const float4 q = leaf[s];
                    if (__float_as_int(q.w) == self) continue;
                    const float dx = xf - q.x, dy = yf - q.y, dz = zf - q.z;
                    m2 = fminf(m2, dx * dx + dy * dy + dz * dz);
                }
                if (m2 < INFINITY) {
                    const float md = sqrtf(m2);
                    const float lim = md + 2.0f * mscale * (extf + md);
                    thr = lim * lim * 1.00001f;
                }
            }
            for (int s = 0; s < cnt; ++s) {
                const float4 q = leaf[s];
                const int pid = __float_as_int(q.w);
                if (pid == self) continue;
                const float dx = xf - q.x, dy = yf - q.y, dz = zf - q.z;
                const float d2f = dx * dx + dy * dy + dz * dz;
                if (d2f <= thr) {
                    const double* Q = A.pts + (long long)pid * DIM;
                    const double ex = __dsub_rn(x, Q[0]);
                    const double ey = __dsub_rn(y, Q[1]);
                    double s2 = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
                    if (DIM == 3) {
                        const double ez = __dsub_rn(z, Q[2]);
                        s2 = __dadd_rn(s2, __dmul_rn(ez, ez));
                    }
                    if (s2 < best) {
                        best = s2;
                        const float bdist = sqrtf((float)s2);
                        const float lim = bdist + mscale * (extf + bdist);
                        thr = lim * lim * 1.00001f;
                        lbound = lim * 1.00001f;
                    }
                }
            }
            __syncwarp();
            const float wb = warp_maxf(lbound);
            wb2 = wb * wb;
        } else {
            const int cl = lvl - 1;
            const long long c = id * 32 + lane;
            const bool ex = c < A.cnt[cl];
            const float d2 = ex ? box_dist2(tlx, tly, tlz, thx, thy, thz, A.blo[A.off[cl] + c], A.bhi[A.off[cl] + c])
                                : INFINITY;
            const bool pass = ex && d2 <= wb2;
            const unsigned msk = __ballot_sync(0xffffffffu, pass);
            const int np = __popc(msk);
            if (sp + np > kStack) {
                if (lane == 0) atomicOr(A.flag, 4);
                break;
            }
            int rank = 0;
            for (int s = 0; s < 32; ++s) {
                const float o = __shfl_sync(0xffffffffu, d2, s);
                if (((msk >> s) & 1u) && (o < d2 || (o == d2 && s < lane))) ++rank;
            }
            if (pass) stack[sp + np - 1 - rank] = (cl << 27) | (int)c;
            sp += np;
            __syncwarp();
        }
    }
    if (valid) dist[qs] = sqrt(best);
}

// mean of dist[0..m) in sample order: thread t sums a contiguous run, the
// runs are added in thread order
__global__ void __launch_bounds__(1024) k_mean_in_order(const double* dist, long long m, double* out) {
    __shared__ double s[1024];
    const long long per = (m + 1023) / 1024;
    const long long beg = threadIdx.x * per, end = beg + per < m ? beg + per : m;
    double a = 0.0;
    for (long long i = beg; i < end; ++i) a += dist[i];
    s[threadIdx.x] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 1024; ++i) t += s[i];
        *out = t / (double)m;
    }
}

}  // namespace

}  // namespace slr

extern "C" slr_status slr_cloud_spacing(slr_ctx* c, const int64_t* sample, int64_t m, double* h_s) {
    using namespace slr;
    if (!c) return SLR_E_INVALID;
    auto bad = [&](slr_status st, const char* msg) {
        c->err = msg;
        return st;
    };
    if (!sample || m < 1 || !h_s) return bad(SLR_E_INVALID, "cloud_spacing: need a sample and an output");
    if (!c->pts || c->npts < 2) return bad(SLR_E_STATE, "cloud_spacing: load a cloud of at least two points first");
    std::vector<int64_t> chk(sample, sample + m);
    std::sort(chk.begin(), chk.end());
    if (chk.front() < 0 || chk.back() >= c->npts) return bad(SLR_E_INVALID, "cloud_spacing: sample index out of range");
    for (int64_t i = 1; i < m; ++i)
        if (chk[i] == chk[i - 1]) return bad(SLR_E_INVALID, "cloud_spacing: sample indices must be distinct");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != c->device) cudaSetDevice(c->device);
    CloudIndex X;
    cudaError_t e = build_cloud_index(c, X);
    int* mark = (int*)dev_alloc(c, sizeof(int) * (size_t)c->npts);
    long long* sdev = (long long*)dev_alloc(c, sizeof(long long) * (size_t)m);
    int* qpos = (int*)dev_alloc(c, sizeof(int) * (size_t)m);
    double* dist = (double*)dev_alloc(c, sizeof(double) * (size_t)(m + 1));
    if (e == cudaSuccess && (!mark || !sdev || !qpos || !dist)) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaMemsetAsync(mark, 0, sizeof(int) * (size_t)c->npts, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sdev, sample, sizeof(long long) * (size_t)m, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        k_mark_sample<<<c->num_sms * 4, 256, 0, c->stream>>>(sdev, m, mark);
        c->launches += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = compact_write(c, SampledPred{X.spt, mark}, SampledEmit{X.spt, mark, qpos}, c->npts);
    if (e == cudaSuccess) {
        SearchArgs A{};
        A.lo0 = c->cfg.lo[0];
        A.lo1 = c->cfg.lo[1];
        A.lo2 = c->cfg.dim == 3 ? c->cfg.lo[2] : 0.0;
        A.spt = X.spt;
        A.pts = c->pts;
        A.npts = c->npts;
        A.blo = X.blo;
        A.bhi = X.bhi;
        A.nlevels = X.nlevels;
        for (int l = 0; l < kMaxLevels; ++l) {
            A.off[l] = l < X.nlevels ? X.off[l] : 0;
            A.cnt[l] = l < X.nlevels ? X.cnt[l] : 0;
        }
        A.extent = X.extent;
        A.flag = X.flag;
        const long long warps = (m + 31) / 32;
        const unsigned blocks = (unsigned)((warps + 7) / 8);
        if (c->cfg.dim == 3)
            k_point_nn<3><<<blocks, 256, 0, c->stream>>>(A, qpos, sdev, m, dist);
        else
            k_point_nn<2><<<blocks, 256, 0, c->stream>>>(A, qpos, sdev, m, dist);
        k_mean_in_order<<<1, 1024, 0, c->stream>>>(dist, m, dist + m);
        c->launches += 2;
        e = cudaGetLastError();
    }
    double hv = 0.0;
    int hflag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hv, dist + m, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, X.flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, X.base);
    dev_free(c, mark);
    dev_free(c, sdev);
    dev_free(c, qpos);
    dev_free(c, dist);
    if (prev >= 0 && prev != c->device) cudaSetDevice(prev);
    if (e == cudaErrorMemoryAllocation) return bad(SLR_E_NOMEM, "cloud_spacing: allocation failed");
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string("cloud_spacing: ") + cudaGetErrorString(e);
        return SLR_E_CUDA;
    }
    if (hflag & 4) return bad(SLR_E_CUDA, "cloud_spacing: traversal stack overflow");
    *h_s = hv;
    return SLR_OK;
}
