// Device code of the fused narrow-band step (arXiv 2410.22205, §3.1 SL
// update, §3.8 eqs. subgrid and cut): one warp's work on one tile of
// kStepTile consecutive entries of the previous band list. Shared by the
// per-job list-step kernel (slr_step.cu) and the batched persistent kernel
// (slr_batch.cuh); both translation units are compiled without implicit FMA
// contraction, so a tile computes the same bits in either.
#pragma once

#include "slr_internal.cuh"

namespace slr {

// node index -> (i, j, k); 32-bit arithmetic (grids hold at most 2^31-1 nodes)
template <typename T>
__device__ __forceinline__ void decode(const Params<T>& P, long long idx, int& i, int& j, int& k) {
    const int id = (int)idx;
    const int q = id / P.n0;
    i = id - q * P.n0;
    k = q / P.n1;
    j = q - k * P.n1;
}

// Tile t of L^{n-1} (cnt_in entries), one warp: ballot of band membership
// |u^n_j| < γ (storage precision), the members written in order into L^n at
// the tile's prepared offset (band_base of its record slice, per = tiles per
// slice, plus tile_off[t]; every write bounds-checked), the SL update and cut
// of the members, u^n copied into u^{n+1} for the others, and the tile's
// FP64 Δ_φ partial.
template <typename T, int DIM, int INTERP>
__device__ __forceinline__ void band_tile(const Params<T>& P, const T* __restrict__ uin, T* __restrict__ uout,
                                          const T* __restrict__ d, const int* Lin, int* Lout, const int* tile_off,
                                          const int* band_base, int band_cap, int cnt_in, int per, int t, T Ep,
                                          double* part_dphi, DevState* ds) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    constexpr int H = kStepTile / 32;
    int idx[H];
    T v[H];
    bool inb[H], valid[H];
    unsigned m[H];
#pragma unroll
    for (int h = 0; h < H; ++h) {
        const int e = t * kStepTile + h * 32 + lane;
        valid[h] = e < cnt_in;
        idx[h] = valid[h] ? ld(Lin + e) : 0;
        v[h] = valid[h] ? ld(uin + idx[h]) : T(0);
        inb[h] = valid[h] && (fabs(v[h]) < P.gamma);
        m[h] = __ballot_sync(0xffffffffu, inb[h]);
    }
    {
        unsigned run = (unsigned)(__ldcg(band_base + t / per) + ld(tile_off + t));
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const unsigned pos = run + __popc(m[h] & lt);
            if (inb[h]) {
                if (pos < (unsigned)band_cap)
                    Lout[pos] = idx[h];
                else
                    atomicOr(&ds->error, kErrBandOffset);  // offsets not prepared for this band
            }
            run += (unsigned)__popc(m[h]);
        }
    }
    T dabs = T(0);
#pragma unroll 1
    for (int h = 0; h < H; ++h) {
        if (!valid[h]) continue;
        T out = v[h];
        if (inb[h]) {
            int i, j, k;
            decode(P, idx[h], i, j, k);
            out = sl_update<T, DIM, INTERP>(P, uin, d, Ep, i, j, k, idx[h], v[h]);
            out = fmin(fmax(out, -P.gamma), P.gamma);  // eq. cut
        }
        uout[idx[h]] = out;
        dabs += fabs(out - v[h]);
    }
    dabs = warp_sum(dabs);
    if (lane == 0) part_dphi[t] = (double)dabs;
}

}  // namespace slr
