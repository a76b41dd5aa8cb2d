// k_tilecore.cuh -- device helpers shared by the count-tile kernels
// (k_build.cu, k_small.cu): the bin rule, a warp scan, the packed pixel
// load and the staged row stores of the slab and record layouts.
#pragma once

#include "ih_internal.cuh"

namespace ih {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Eq. 2.15's Q: the channel-local bin of value v, or -1 for none.
__device__ __forceinline__ int bin_of(int v, int bins, int mode)
{
    if (mode == 0) return (v * bins) >> 8;
    return v < bins ? v : -1;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    return x;
}

// The 4 pixels (r, c..c+3) of a channel as packed bytes (pixel j in byte j);
// bytes at or beyond `cend` are 0 and must be masked by the caller.
__device__ __forceinline__ uint32_t load4(const uint8_t *plane, int64_t pitch, int r, int c, int cend, bool vec_ok)
{
    const uint8_t *row = plane + (int64_t)r * pitch;
    if (vec_ok && c + 3 < cend) return __ldg(reinterpret_cast<const unsigned int *>(row + c));
    uint32_t v = 0;
#pragma unroll
    for (int jj = 0; jj < 4; ++jj)
        if (c + jj < cend) v |= (uint32_t)__ldg(row + c + jj) << (8 * jj);
    return v;
}

__device__ __forceinline__ uint32_t load4(const ChanDev &ch, int r, int c, int cend, bool vec_ok)
{
    return load4(ch.plane, ch.pitch, r, c, cend, vec_ok);
}

// Slab-layout row store through a per-warp shared buffer.  Lane L's 4
// pixel records (NB int4 units) go to units L*S + k, S the smallest odd
// number > NB, so that both the writes and the reads below hit 8 distinct
// 16-byte bank groups per 8 lanes; the warp then stores the row segment
// (32*NB units, contiguous in global memory) with lane L writing units
// 32m + L: every store instruction covers 512 contiguous bytes.
template <int NB>
struct SlabStage {
    static constexpr int S = (NB + 1) | 1;
};

template <int NB>
__device__ __forceinline__ void store_slab_staged(int32_t *seg, int npx, const int (&acc)[NB][4], int4 *stage,
                                                  int lane)
{
    constexpr int S = SlabStage<NB>::S;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        int v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int f = 4 * k + e;  // flat index: pixel f / NB, bin f % NB
            v[e] = acc[f % NB][f / NB];
        }
        stage[lane * S + k] = make_int4(v[0], v[1], v[2], v[3]);
    }
    __syncwarp();
    // units of pixels below npx (the segment's valid pixels, a multiple of 4)
    const int nunits = npx / 4 * NB;
#pragma unroll
    for (int m = 0; m < NB; ++m) {
        const int u = 32 * m + lane;
        if (u < nunits) reinterpret_cast<int4 *>(seg)[u] = stage[(u / NB) * S + (u % NB)];
    }
}

// Record-layout row store through the same per-warp buffer.  Each of the
// segment's npx pixels owns an NB-word chunk (NB = 8: one whole 32-byte
// sector, so no sector is shared with another warp) at a stride of rec_w
// words; unit u = 32m + L of the row is quarter u % (NB/4) of pixel
// u / (NB/4), so consecutive lanes write consecutive 16-byte pieces of
// consecutive chunks.
template <int NB>
__device__ __forceinline__ void store_record_staged(int32_t *row, int rec_w, int npx, const int (&acc)[NB][4],
                                                    int4 *stage, int lane)
{
    static_assert(NB == 4 || NB == 8, "record chunks are 4 or 8 words");
    constexpr int S = SlabStage<NB>::S, Q = NB / 4;
    __syncwarp();
#pragma unroll
    for (int k = 0; k < NB; ++k) {
        int v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int f = 4 * k + e;  // flat index: pixel f / NB, bin f % NB
            v[e] = acc[f % NB][f / NB];
        }
        stage[lane * S + k] = make_int4(v[0], v[1], v[2], v[3]);
    }
    __syncwarp();
    // unit u = 32m + L' is word chunk k = L' % NB (the same for every m) of
    // lane-pixel group u / NB = (32/NB) m + L' / NB: its destination and its
    // stage slot are a per-lane constant plus m times a stride
    const int nunits = npx * Q;
    const int kk = lane % NB;
    const int64_t c0 = (int64_t)(4 * (lane / NB) + kk / Q) * rec_w + 4 * (kk % Q);
    const int64_t dm = (int64_t)(128 / NB) * rec_w;
    const int s0 = (lane / NB) * S + kk;
#pragma unroll
    for (int m = 0; m < NB; ++m) {
        if (32 * m + lane < nunits) *reinterpret_cast<int4 *>(row + c0 + m * dm) = stage[s0 + m * (32 / NB) * S];
    }
}

}  // namespace

}  // namespace ih
