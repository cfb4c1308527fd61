// The reinitialisation of Algorithm 1 (§3.7) on Ḡ^n (the band G̃^n of
// the SL step and its face neighbours), then eq. cut.
//
// Besides φ^{n+1} it leaves the next step's scan list (Ḡ^n, ascending node
// indices, in the band-list slot the next step reads) and the energy pass's
// candidate cells (every cell with a corner in Ḡ^n, ascending lower-corner
// index). Every size lives on the device, so the whole stage is part of the
// captured iteration graph.
//
// Sets are row-padded bitmasks (one 32-bit word per 32 nodes of a grid row,
// rows word-aligned): the band bits are set from the sorted band list with
// warp-aggregated atomicOr; the dilation to Ḡ and the candidate cells are
// word-parallel shifts and ORs; ordered lists come from popcount compactions.
//
// Readings (the paper cites Hartmann et al. 2008 and Sussman et al. 1994
// without formulas; these match the oracle):
//  - explicit step on an interface node j (a face neighbour of the other
//    sign class, φ < 0 versus φ >= 0), keeping the interface where φ̃ puts
//    it: (a) the estimate of Russo and Smereka (2000) on every interface node
//    k, D_k = φ̃_k / Δ_k with Δ_k the largest of the gradient norm (centred,
//    one-sided on the domain boundary) and the one-sided differences; then
//    (b) the constraint of the constrained reinitialisation: φ_j = φ̃_j
//    Σ_{k∈S_j} D_k / Σ_{k∈S_j} φ̃_k over the face neighbours S_j of the
//    other sign class, which keeps j's ratio to them as in φ̃;
//  - Jacobi sweeps ψ ← ψ - Δτ sign(φ̃)(|∇ψ|_G - 1) with Godunov's upwind
//    |∇ψ|_G on the other nodes of Ḡ; interface nodes, nodes on the domain
//    boundary and nodes with φ̃ = 0 keep their value;
//  - Δ_φ of the iteration is h^dim Σ_Ḡ |φ^{n+1} - φ^n|.
//
// Buffers: φ̃ is read as the SL step left it (band nodes from the output
// buffer, every other node from the input buffer); the sweeps ping-pong
// between the scratch field W and the output buffer; the last kernel writes
// the cut result into both φ buffers and W, so that the three agree outside
// the next Ḡ, as the sweeps of the next iteration assume.
#include <cstring>

#include "slr_internal.cuh"

namespace slr {

template <typename T>
Params<T> make_params(const slr_ctx* c);
int reinit_grid(const slr_ctx* c);
int reinit_scan_blocks(const slr_ctx* c);

namespace {

constexpr int kRB = 256;            // threads per block
constexpr int kWordsPerThread = 4;  // bitmask words per thread in the compactions
constexpr int kReinitFixedKernels = 10;  // kernels besides the sweeps

struct BitGeom {
    int n0, n1, n2;
    int wpr;          // words per row
    long long words;  // wpr * rows
    int dim;
};

__device__ __forceinline__ int block_reduce_int(int v, int* smem) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) smem[w] = v;
    __syncthreads();
    int r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kRB / 32; ++i) r += smem[i];
    return r;
}

// band bits of G̃^n, the band list the SL step just wrote
__global__ void __launch_bounds__(kRB) k_band_bits(const int* L0, const int* L1, unsigned* bm, BitGeom g,
                                                   DevState* ds) {
    if (ds->stop) return;
    const int n = ds->n;
    const int sel = (n + 1) & 1;
    const int* __restrict__ B = sel ? L1 : L0;
    const int cnt = ds->band_count[sel];
    if (blockIdx.x == 0 && threadIdx.x == 0) ds->band_sl = cnt;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + threadIdx.x - lane; base < cnt; base += stride) {
        const long long p = base + lane;
        long long w = -1;
        unsigned bit = 0u;
        if (p < cnt) {
            const int b = B[p];
            const int r = b / g.n0, x = b - r * g.n0;
            w = (long long)r * g.wpr + (x >> 5);
            bit = 1u << (x & 31);
        }
        const unsigned grp = __match_any_sync(0xffffffffu, w);
        const unsigned orv = __reduce_or_sync(grp, bit);
        if (p < cnt && lane == __ffs(grp) - 1) atomicOr(bm + w, orv);
    }
}

__device__ __forceinline__ unsigned row_tail_mask(const BitGeom& g, int xw, int nvalid) {
    // bits of word xw whose x = 32 xw + b is < nvalid
    const int lo = xw * 32;
    if (nvalid >= lo + 32) return 0xffffffffu;
    if (nvalid <= lo) return 0u;
    return (1u << (nvalid - lo)) - 1u;
}

// Ḡ bits: a node whose own bit or a face neighbour's bit is set
__global__ void __launch_bounds__(kRB) k_dilate_bits(const unsigned* __restrict__ bm, unsigned* __restrict__ gm,
                                                     BitGeom g, DevState* ds) {
    if (ds->stop) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long plane = (long long)g.wpr * g.n1;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < g.words; w += stride) {
        const long long r = w / g.wpr;
        const int xw = (int)(w - r * g.wpr);
        const int y = (int)(r % g.n1), z = (int)(r / g.n1);
        const unsigned m = bm[w];
        const unsigned prev = xw > 0 ? bm[w - 1] : 0u, next = xw < g.wpr - 1 ? bm[w + 1] : 0u;
        unsigned o = m | (m << 1) | (prev >> 31) | (m >> 1) | (next << 31);
        if (y > 0) o |= bm[w - g.wpr];
        if (y < g.n1 - 1) o |= bm[w + g.wpr];
        if (g.dim == 3) {
            if (z > 0) o |= bm[w - plane];
            if (z < g.n2 - 1) o |= bm[w + plane];
        }
        gm[w] = o & row_tail_mask(g, xw, g.n0);
    }
}

// candidate-cell bits: the cell with lower corner (x, y, z) has a corner in Ḡ
__global__ void __launch_bounds__(kRB) k_cell_bits(const unsigned* __restrict__ gm, unsigned* __restrict__ cm,
                                                   BitGeom g, DevState* ds) {
    if (ds->stop) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long plane = (long long)g.wpr * g.n1;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < g.words; w += stride) {
        const long long r = w / g.wpr;
        const int xw = (int)(w - r * g.wpr);
        const int y = (int)(r % g.n1), z = (int)(r / g.n1);
        if (y >= g.n1 - 1 || (g.dim == 3 && z >= g.n2 - 1)) {
            cm[w] = 0u;
            continue;
        }
        unsigned o = 0u;
        for (int dz = 0; dz < (g.dim == 3 ? 2 : 1); ++dz)
            for (int dy = 0; dy < 2; ++dy) {
                const long long ww = w + dy * g.wpr + dz * plane;
                const unsigned m = gm[ww];
                const unsigned nx = xw < g.wpr - 1 ? gm[ww + 1] : 0u;
                o |= m | (m >> 1) | (nx << 31);
            }
        cm[w] = o & row_tail_mask(g, xw, g.n0 - 1);
    }
}

// ordered compaction of a bitmask: per-block counts, one scan, then writes
__global__ void __launch_bounds__(kRB) k_bits_count(const unsigned* __restrict__ m, long long words, int* blk,
                                                    DevState* ds) {
    __shared__ int s[kRB / 32];
    if (ds->stop) return;
    const long long w0 = ((long long)blockIdx.x * kRB + threadIdx.x) * kWordsPerThread;
    int c = 0;
#pragma unroll
    for (int q = 0; q < kWordsPerThread; ++q)
        if (w0 + q < words) c += __popc(m[w0 + q]);
    const int t = block_reduce_int(c, s);
    if (threadIdx.x == 0) blk[blockIdx.x] = t;
}

// exclusive scan of nb block counts (one block); the total goes to the band
// slot the next step reads (kind 0) or to the candidate-cell count (kind 1)
__global__ void __launch_bounds__(1024) k_scan_blocks_dev(int* blk, int nb, int kind, DevState* ds) {
    __shared__ int s[32];
    if (ds->stop) return;
    const int per = (nb + 1023) / 1024;
    const int beg = threadIdx.x * per, end = beg + per < nb ? beg + per : nb;
    int sum = 0;
    for (int i = beg; i < end; ++i) sum += blk[i];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int v = s[lane];
        int iv = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, iv, o);
            if (lane >= o) iv += t;
        }
        s[lane] = iv - v;  // exclusive prefix of the warp totals
        if (lane == 31) {
            if (kind == 0)
                ds->band_count[(ds->n + 1) & 1] = iv;
            else
                ds->n_ecells_dyn = iv;
        }
    }
    __syncthreads();
    int run = s[w] + incl - sum;
    for (int i = beg; i < end; ++i) {
        const int c = blk[i];
        blk[i] = run;
        run += c;
    }
}

// kind 0: Ḡ into the band-list slot the next step reads; kind 1: cells
__global__ void __launch_bounds__(kRB) k_bits_write(const unsigned* __restrict__ m, long long words,
                                                    const int* __restrict__ blk, int kind, int* L0, int* L1,
                                                    int* cells, BitGeom g, DevState* ds) {
    __shared__ int s[kRB / 32 + 1];
    if (ds->stop) return;
    int* __restrict__ out = kind == 0 ? (((ds->n + 1) & 1) ? L1 : L0) : cells;
    const long long w0 = ((long long)blockIdx.x * kRB + threadIdx.x) * kWordsPerThread;
    unsigned wv[kWordsPerThread];
    int c = 0;
#pragma unroll
    for (int q = 0; q < kWordsPerThread; ++q) {
        wv[q] = w0 + q < words ? m[w0 + q] : 0u;
        c += __popc(wv[q]);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s[w] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < kRB / 32; ++i) {
            const int t = s[i];
            s[i] = run;
            run += t;
        }
    }
    __syncthreads();
    int pos = blk[blockIdx.x] + s[w] + incl - c;
#pragma unroll
    for (int q = 0; q < kWordsPerThread; ++q) {
        unsigned v = wv[q];
        if (!v) continue;
        const long long ww = w0 + q;
        const long long r = ww / g.wpr;
        const int xw = (int)(ww - r * g.wpr);
        const int rowbase = (int)(r * g.n0) + xw * 32;
        while (v) {
            const int b = __ffs(v) - 1;
            v &= v - 1u;
            out[pos++] = rowbase + b;
        }
    }
}

// flags per Ḡ position: bit 0 fixed during the sweeps, bits 1-2 sign of φ̃ (1 +, 2 -)
template <typename T, int DIM>
__global__ void __launch_bounds__(kRB) k_reinit_prep(Params<T> P, const T* ub0, const T* ub1, T* __restrict__ W,
                                                     const int* L0, const int* L1, unsigned char* __restrict__ rfl,
                                                     DevState* ds) {
    if (ds->stop) return;
    const int n = ds->n;
    const int sel = (n + 1) & 1;
    const int* __restrict__ G = sel ? L1 : L0;
    const int cnt = ds->band_count[sel];
    const T* __restrict__ uin = (n & 1) ? ub1 : ub0;
    const T* __restrict__ uout = (n & 1) ? ub0 : ub1;
    auto view = [&](int x) -> T {
        // band nodes hold the SL result in the output buffer; both loads are
        // issued at once (every node is in bounds) and one is kept
        const T a = __ldg(uin + x), b = __ldg(uout + x);
        return fabs(a) < P.gamma ? b : a;
    };
    const int nn[3] = {P.n0, P.n1, P.n2};
    const int st[3] = {1, P.is1, P.is2};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < cnt; p += stride) {
        const int j = G[p];
        int c[3];
        c[0] = j % P.n0;
        const int q = j / P.n0;
        c[1] = DIM == 3 ? q % P.n1 : q;
        c[2] = DIM == 3 ? q / P.n1 : 0;
        const T vj = view(j);
        const bool neg = vj < T(0);
        bool edge = false, iface = false;
        T vm[DIM], vp[DIM];
        bool hm[DIM], hp[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            hm[a] = c[a] > 0;
            hp[a] = c[a] < nn[a] - 1;
            edge |= !hm[a] || !hp[a];
            vm[a] = hm[a] ? view(j - st[a]) : T(0);
            vp[a] = hp[a] ? view(j + st[a]) : T(0);
            iface |= (hm[a] && ((vm[a] < T(0)) != neg)) || (hp[a] && ((vp[a] < T(0)) != neg));
        }
        T out = vj;
        if (iface) {
            // (a) the Russo-Smereka estimate of node k at coordinates ck
            auto rs = [&](int k, const int* ck) -> T {
                const T vk = view(k);
                T cn = T(0), mx = T(0);
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    const bool m = ck[a] > 0, pp = ck[a] < nn[a] - 1;
                    const T wm = m ? view(k - st[a]) : T(0), wp = pp ? view(k + st[a]) : T(0);
                    // differences scaled by the reciprocals 1/h, 1/(2h) (the
                    // oracle divides: results agree to rounding)
                    if (m) mx = fmax(mx, fabs(vk - wm) * P.inv_h);
                    if (pp) mx = fmax(mx, fabs(wp - vk) * P.inv_h);
                    T ce = T(0);  // centred; one-sided on the domain boundary
                    if (m && pp)
                        ce = (wp - wm) * P.inv_2h;
                    else if (pp)
                        ce = (wp - vk) * P.inv_h;
                    else if (m)
                        ce = (vk - wm) * P.inv_h;
                    cn = cn + ce * ce;
                }
                const T den = fmax(sqrt(cn), mx);
                return den > T(0) ? vk / den : vk;
            };
            // (b) the constraint over the face neighbours of the other sign class
            T sd = T(0), sp = T(0);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                if (hm[a] && ((vm[a] < T(0)) != neg)) {
                    int ck[3] = {c[0], c[1], c[2]};
                    ck[a] -= 1;
                    sd = sd + rs(j - st[a], ck);
                    sp = sp + vm[a];
                }
                if (hp[a] && ((vp[a] < T(0)) != neg)) {
                    int ck[3] = {c[0], c[1], c[2]};
                    ck[a] += 1;
                    sd = sd + rs(j + st[a], ck);
                    sp = sp + vp[a];
                }
            }
            out = sp != T(0) ? vj * sd / sp : rs(j, c);
        }
        const unsigned sg = vj > T(0) ? 1u : (vj < T(0) ? 2u : 0u);
        const bool fixed = iface || edge || sg == 0u;
        rfl[p] = (unsigned char)((fixed ? 1u : 0u) | (sg << 1));
        W[j] = out;
    }
}

// one forward-Euler sweep of eq. reinit, Y = X - Δτ sign(φ̃)(|∇X|_G - 1), on
// Ḡ; phase 0 reads W and writes the output buffer, phase 1 the reverse (the
// output buffer is the one the SL step wrote, picked by the iteration parity)
// Programmatic dependent launch (pdl_trigger, pdl_wait): a sweep (and the
// final kernel) lets the next kernel of the chain start as soon as every
// block of its own grid has started, and waits for the previous kernel's
// completion only where it reads that kernel's output. The list of Ḡ and its
// flags, written before the first sweep, are read before the wait, so the
// next launch's latency and those loads overlap the end of the previous
// sweep.

template <typename T, int DIM>
__global__ void __launch_bounds__(kRB) k_reinit_sweep(Params<T> P, T* ub0, T* ub1, T* W, int phase, const int* L0,
                                                      const int* L1, const unsigned char* __restrict__ rfl, T dtau,
                                                      DevState* ds) {
    pdl_trigger();
    if (ds->stop) return;
    const int n = ds->n;
    const int sel = (n + 1) & 1;
    const int* __restrict__ G = sel ? L1 : L0;
    const int cnt = ds->band_count[sel];
    T* uout = (n & 1) ? ub0 : ub1;
    const T* __restrict__ X = phase ? uout : W;
    T* __restrict__ Y = phase ? W : uout;
    const int st[3] = {1, P.is1, P.is2};
    // four positions per thread, p, p + S, p + 2S, p + 3S (S = threads of the
    // grid): all their loads are issued before any store
    constexpr int K = 4;
    const long long S = (long long)gridDim.x * blockDim.x;
    bool waited = false;
    for (long long p0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; p0 < cnt; p0 += K * S) {
        int j[K];
        unsigned f[K];
        T x[K], nb[K][2 * DIM];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const long long p = p0 + k * S;
            const bool v = p < cnt;
            j[k] = v ? G[p] : 0;
            f[k] = v ? (unsigned)rfl[p] : 1u;
        }
        if (!waited) {
            pdl_wait();  // X is the previous sweep's output
            waited = true;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            x[k] = X[j[k]];
            if (!(f[k] & 1u)) {
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    nb[k][2 * a] = X[j[k] - st[a]];
                    nb[k][2 * a + 1] = X[j[k] + st[a]];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (p0 + k * S >= cnt) break;
            if (f[k] & 1u) {
                Y[j[k]] = x[k];
                continue;
            }
            const bool pos = (f[k] >> 1) == 1u;
            T s2 = T(0);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const T am = (x[k] - nb[k][2 * a]) * P.inv_h;
                const T bp = (nb[k][2 * a + 1] - x[k]) * P.inv_h;
                T t1, t2;
                if (pos) {
                    t1 = fmax(am, T(0));
                    t2 = fmin(bp, T(0));
                } else {
                    t1 = fmin(am, T(0));
                    t2 = fmax(bp, T(0));
                }
                s2 += fmax(t1 * t1, t2 * t2);
            }
            const T sgn_dt = pos ? dtau : -dtau;
            Y[j[k]] = x[k] - sgn_dt * (sqrt(s2) - T(1));
        }
    }
}

// after M sweeps the result is in the output buffer (M odd) or in W (M even):
// cut it and write it into both φ buffers and W; Δ_φ partial per block
template <typename T>
__global__ void __launch_bounds__(kRB) k_reinit_final(Params<T> P, T* ub0, T* ub1, T* W, int M, const int* L0,
                                                      const int* L1, double* part, DevState* ds) {
    __shared__ double s[kRB / 32];
    pdl_trigger();
    if (ds->stop) return;
    pdl_wait();  // R is the last sweep's output
    const int n = ds->n;
    const int sel = (n + 1) & 1;
    const int* __restrict__ G = sel ? L1 : L0;
    const int cnt = ds->band_count[sel];
    T* uin = (n & 1) ? ub1 : ub0;
    T* uout = (n & 1) ? ub0 : ub1;
    const T* R = (M & 1) ? uout : W;
    T acc = T(0);
    // R is W or the output buffer, both written here: each thread loads its
    // four positions' values before it stores any of them
    constexpr int K = 4;
    const long long S = (long long)gridDim.x * blockDim.x;
    for (long long p0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; p0 < cnt; p0 += K * S) {
        int j[K];
        T r[K], o[K];
#pragma unroll
        for (int k = 0; k < K; ++k) j[k] = p0 + k * S < cnt ? G[p0 + k * S] : -1;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            r[k] = j[k] >= 0 ? R[j[k]] : T(0);
            o[k] = j[k] >= 0 ? uin[j[k]] : T(0);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (j[k] < 0) break;
            const T v = fmin(fmax(r[k], -P.gamma), P.gamma);  // eq. cut
            acc += fabs(v - o[k]);
            uin[j[k]] = v;
            uout[j[k]] = v;
            W[j[k]] = v;
        }
    }
    const double t = (double)warp_sum(acc);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) s[w] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0.0;
        for (int i = 0; i < kRB / 32; ++i) x += s[i];
        part[blockIdx.x] = x;
    }
}

BitGeom geom(const slr_ctx* c) {
    BitGeom g;
    g.dim = c->cfg.dim;
    g.n0 = (int)c->cfg.n[0];
    g.n1 = (int)c->cfg.n[1];
    g.n2 = c->cfg.dim == 3 ? (int)c->cfg.n[2] : 1;
    g.wpr = (g.n0 + 31) / 32;
    g.words = (long long)g.wpr * g.n1 * g.n2;
    return g;
}

template <typename T, int DIM>
cudaError_t reinit_t(slr_ctx* c) {
    Params<T> P = make_params<T>(c);
    const BitGeom g = geom(c);
    const int grid = reinit_grid(c);
    const int cblocks = reinit_scan_blocks(c);
    T* u0 = (T*)c->u[0];
    T* u1 = (T*)c->u[1];
    T* W = (T*)c->rw;
    cudaError_t e = cudaMemsetAsync(c->bits_band, 0, sizeof(unsigned) * (size_t)g.words, c->stream);
    if (e != cudaSuccess) return e;
    k_band_bits<<<grid, kRB, 0, c->stream>>>(c->band[0], c->band[1], c->bits_band, g, c->ds);
    k_dilate_bits<<<grid, kRB, 0, c->stream>>>(c->bits_band, c->bits_gbar, g, c->ds);
    k_cell_bits<<<grid, kRB, 0, c->stream>>>(c->bits_gbar, c->bits_cell, g, c->ds);
    // Ḡ, ascending, into the slot the next step scans
    k_bits_count<<<cblocks, kRB, 0, c->stream>>>(c->bits_gbar, g.words, c->rblk, c->ds);
    k_scan_blocks_dev<<<1, 1024, 0, c->stream>>>(c->rblk, cblocks, 0, c->ds);
    k_bits_write<<<cblocks, kRB, 0, c->stream>>>(c->bits_gbar, g.words, c->rblk, 0, c->band[0], c->band[1], nullptr,
                                                 g, c->ds);
    // candidate cells of the energy pass, ascending
    k_bits_count<<<cblocks, kRB, 0, c->stream>>>(c->bits_cell, g.words, c->rblk + cblocks, c->ds);
    k_scan_blocks_dev<<<1, 1024, 0, c->stream>>>(c->rblk + cblocks, cblocks, 1, c->ds);
    k_bits_write<<<cblocks, kRB, 0, c->stream>>>(c->bits_cell, g.words, c->rblk + cblocks, 1, nullptr, nullptr,
                                                 c->ecells, g, c->ds);
    // explicit step, sweeps, cut
    k_reinit_prep<T, DIM><<<grid, kRB, 0, c->stream>>>(P, u0, u1, W, c->band[0], c->band[1], c->rflags, c->ds);
    const int M = reinit_sweeps(c);
    const T dtau = (T)reinit_dtau(c);
    // sweep m reads X_m and writes Y_m: W -> out, out -> W, ... ; the output
    // buffer is picked on the device by the iteration parity, so both
    // orders are captured and each kernel selects its own
    // the first sweep depends fully on the interface step (it reads the flags
    // that kernel writes); the later sweeps and the final kernel are
    // programmatic dependents of the kernel before them
    cudaLaunchConfig_t lc;
    memset(&lc, 0, sizeof(lc));
    lc.gridDim = dim3((unsigned)grid);
    lc.blockDim = dim3(kRB);
    lc.stream = c->stream;
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    for (int m = 0; m < M && e == cudaSuccess; ++m) {
        lc.attrs = m == 0 ? nullptr : pdl;
        lc.numAttrs = m == 0 ? 0 : 1;
        e = cudaLaunchKernelEx(&lc, k_reinit_sweep<T, DIM>, P, u0, u1, W, m & 1, (const int*)c->band[0],
                               (const int*)c->band[1], (const unsigned char*)c->rflags, dtau, c->ds);
    }
    lc.attrs = M > 0 ? pdl : nullptr;
    lc.numAttrs = M > 0 ? 1 : 0;
    if (e == cudaSuccess)
        e = cudaLaunchKernelEx(&lc, k_reinit_final<T>, P, u0, u1, W, M, (const int*)c->band[0],
                               (const int*)c->band[1], c->part_dphi_r, c->ds);
    c->launches += kReinitFixedKernels + M;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

int reinit_grid(const slr_ctx* c) { return c->num_sms * 8; }

int reinit_sweeps(const slr_ctx* c) {
    if (c->cfg.reinit_sweeps > 0) return c->cfg.reinit_sweeps;
    return 4 * ((int)floor(c->gamma / c->h + 0.5) + 1);
}

double reinit_dtau(const slr_ctx* c) { return c->cfg.reinit_dtau > 0.0 ? c->cfg.reinit_dtau : 0.5 * c->h; }

size_t reinit_bit_words(const slr_ctx* c) { return (size_t)geom(c).words; }

int reinit_scan_blocks(const slr_ctx* c) {
    const long long words = geom(c).words;
    return (int)((words + (long long)kRB * kWordsPerThread - 1) / ((long long)kRB * kWordsPerThread));
}

cudaError_t launch_reinit(slr_ctx* c) {
    const bool f32 = c->cfg.precision == 32;
    if (c->cfg.dim == 2) return f32 ? reinit_t<float, 2>(c) : reinit_t<double, 2>(c);
    return f32 ? reinit_t<float, 3>(c) : reinit_t<double, 3>(c);
}

}  // namespace slr
