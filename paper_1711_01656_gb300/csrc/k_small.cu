// k_small.cu -- the count integral histogram (Eq. 2.15) of a frame too small
// to keep the GPU busy with the three-kernel build, in ONE cooperative launch.
//
// On a 640 x 480 frame the three-kernel build (tile sums, carry scan,
// tiles) is bound by latency, not bandwidth: each kernel runs about one warp
// per scheduler, and each warp walks a chain of several thousand dependent
// instructions.  Here the frame is cut into bands of R = 8 * RPW rows and
// strips of 128 columns; CTA (bin group g, band i, strip j) has 8 warps and
// warp w owns rows [R0 + w RPW, R0 + (w+1) RPW) of the tile (RPW = 1..8 rows
// per warp), a lane 4 adjacent columns.  The chains are RPW rows long and
// every tile runs at once:
//  1. Before the barrier, from the tile's own pixels: each warp bins its
//     rows once (the pixel words stay in registers) into packed 8-bit
//     one-hot fields: the column counts of its rows, the strip's row counts
//     (warp reductions) and its rows' 2-D sums D_w(c) over columns [C0, c]
//     (16-bit pairs, one in-lane prefix and four warp scans).  The CTA
//     publishes the band's column counts, its row counts and its bin
//     totals, and keeps the exclusive prefix over the warps of D_w.
//  2. Grid barrier.  The launch is cooperative, so every CTA is resident;
//     a CTA arrives once its sums are published and waits for all others
//     (bounded: a wait that gives up sets bit 2 of the error word, and
//     ih_sync reports IH_ETIMEOUT).  The last CTA past the barrier zeroes
//     its counters for the next launch.
//  3. Carries as direct sums of the published tile sums: the column carry G
//     (the bands above), the row carries L (the strips to the left) and the
//     tile corner (the tiles above and to the left); from them the band's
//     top row H(R0-1, c) = corner + row prefix of G, one warp per bin.
//  4. Each warp seeds its columns with H(R0 + rw - 1, c) = H(R0-1, c) +
//     sum_{w' < w} D_w'(c) + the row carries of the band's rows above it,
//     and writes its rows like the count tiles kernel: per row a packed
//     one-hot, one in-lane prefix and two warp scans, each cell stored once.
// Per cell the arithmetic is the split of Eq. 2.15 at the tile's edges:
//   H(r,c) = H(R0-1, C0-1) + sum_{C0<=c'<=c} G(c')
//          + sum_{R0<=r'<=r} ( L(r') + sum_{C0<=c'<=c} Q(r',c') ).
#include <algorithm>
#include <mutex>

#include <stdlib.h>

#include "ih_internal.cuh"
#include "ih_plan.h"
#include "k_tilecore.cuh"

namespace ih {

namespace {

constexpr int kSmWarps = 8;
constexpr int kSmThreads = 32 * kSmWarps;
constexpr int kSmMaxRpw = 8;                    // rows per warp
constexpr int kSmMaxRows = kSmWarps * kSmMaxRpw;  // band rows
constexpr int kSmMaxStrips = 16;
constexpr long kSmSpinLimit = 1L << 22;

struct SmallSmem {
    uint32_t colw[kSmWarps][kSmThreads];  // per warp: packed column counts, word k of lane L at
                                          // [k * 32 + L] (k = 2 q + h: column 4L + q, bins 4h..4h+3)
    uint32_t D[kSmWarps][2 * kSmThreads]; // per warp: its rows' 2-D sums over columns [C0, c] as
                                          // 16-bit pairs, then the exclusive prefix over the warps
    uint32_t G[2][kSmThreads];            // column carry at the band's top: 16-bit fields of
                                          // bytes 0, 2 ([0]) and 1, 3 ([1]) of word [k * 32 + L]
    uint32_t Gp[4][kSmThreads][2];        // its partial sums over four slices of the bands
    int32_t Htop[kGroupBins][kChunk];     // H(R0 - 1, c) of the strip's columns
    uint32_t rowcnt[kSmMaxRows][2];       // row counts over the strip, packed (bins 0-3, 4-7)
    int32_t L[kSmMaxRows][kGroupBins];    // row carries
    int32_t cpart[kSmWarps][kGroupBins];  // partial corners
    int32_t LS[kSmWarps][kGroupBins];     // per warp: the row carries of the band's rows above it
    int ok;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned int *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// One thread of each CTA: publish the CTA's writes (ordered before this
// thread by the caller's __syncthreads) and arrive.
__device__ __forceinline__ void grid_arrive(unsigned int *bar)
{
    __threadfence();
    atomicAdd(bar, 1u);
}

// ... and wait until the counter reaches `target`.  False when the wait gave
// up (or another CTA's did).
__device__ __forceinline__ bool grid_wait(unsigned int *bar, unsigned target, int *err)
{
    long spins = 0;
    while (ld_acquire_u32(bar) < target) {
        if (++spins > kSmSpinLimit || (*(volatile int *)err & 2)) {
            atomicOr(err, 2);
            return false;
        }
        __nanosleep(32);
    }
    return true;
}

// Field e (0..3) of the 16-bit-pair sums (lo: bytes 0, 2; hi: bytes 1, 3).
__device__ __forceinline__ int pair_field(uint32_t lo, uint32_t hi, int e)
{
    const uint32_t w = (e & 1) ? hi : lo;
    return (int)((e & 2) ? (w >> 16) : (w & 0xffffu));
}

template <int LAYOUT, int NB>
__device__ __forceinline__ void small_body(const PlaneSet &ps, SmallSmem &sm, int4 *stage)
{
    const TileGrid &g = ps.g;
    const int rpw = ps.small;
    const int ntiles = g.nb * g.ns;
    const int gi = (int)blockIdx.x / ntiles, tile = (int)blockIdx.x - gi * ntiles;
    const int i = tile / g.ns, j = tile - (tile / g.ns) * g.ns;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const GroupDev gr = ps.grp[gi];
    const ChanDev &ch = ps.chan[gr.chan];
    const int blo = gr.b_lo, nbg = gr.nb;
    const int bins = ch.bins, mode = ps.uni ? 0 : ch.mode;
    const int64_t bg0 = ch.bin_off + gr.b_lo;
    const int R0 = i * g.R, nr = min(g.R, g.H - R0);
    const int C0 = j * kChunk, c = C0 + 4 * lane;
    const int nvalid = max(0, min(4, g.W - c));
    const int rw = w * rpw;                      // the warp's first row inside the band
    const int nrw = max(0, min(rpw, nr - rw));   // its rows
    const bool vec_ok = ((ch.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(ch.plane) & 3) == 0);

    // 1. the warp's rows: pixel words, column counts (bins 0-3 and 4-7 of
    // each of the lane's columns, fields <= RPW) and row counts
    uint32_t px[kSmMaxRpw];
#pragma unroll
    for (int k = 0; k < kSmMaxRpw; ++k) px[k] = k < nrw ? load4(ch.plane, ch.pitch, R0 + rw + k, c, g.W, vec_ok) : 0u;
    uint32_t colw[4][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}};
#pragma unroll
    for (int k = 0; k < kSmMaxRpw; ++k) {
        if (k >= rpw) break;
        uint32_t r0w = 0u, r1w = 0u;
        if (k < nrw) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int b = bin_of((px[k] >> (8 * q)) & 0xff, bins, mode) - blo;
                if (q < nvalid && b >= 0 && b < nbg) {
                    const uint32_t inc = 1u << (8 * (b & 3));
                    if (b < 4) {
                        colw[q][0] += inc;
                        r0w += inc;
                    } else {
                        colw[q][1] += inc;
                        r1w += inc;
                    }
                }
            }
        }
        r0w = __reduce_add_sync(kFull, r0w);
        r1w = __reduce_add_sync(kFull, r1w);
        if (lane < 2) sm.rowcnt[rw + k][lane] = lane ? r1w : r0w;  // rows past the frame's end: 0
    }
    // the warp's 2-D sums D(b, c) = sum over its rows and columns [C0, c] as
    // 16-bit pairs (fields <= RPW * 128): pair word m = 2h + o holds bins
    // 4h + o (low half) and 4h + o + 2 (high half)
    {
        uint32_t pw[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                pw[q][2 * h] = colw[q][h] & 0x00ff00ffu;
                pw[q][2 * h + 1] = (colw[q][h] >> 8) & 0x00ff00ffu;
            }
            sm.colw[w][(2 * q) * 32 + lane] = colw[q][0];
            sm.colw[w][(2 * q + 1) * 32 + lane] = colw[q][1];
        }
#pragma unroll
        for (int q = 1; q < 4; ++q)
#pragma unroll
            for (int m = 0; m < 4; ++m) pw[q][m] += pw[q - 1][m];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const uint32_t ex = warp_incl_scan(pw[3][m], lane) - pw[3][m];
            uint4 v;
            v.x = ex + pw[0][m];
            v.y = ex + pw[1][m];
            v.z = ex + pw[2][m];
            v.w = ex + pw[3][m];
            reinterpret_cast<uint4 *>(sm.D[w])[m * 32 + lane] = v;
        }
    }
    __syncthreads();

    // the tile's sums: exclusive prefix of the column counts over the warps
    // gives the band's column counts (fields <= R <= 64), published; the
    // exclusive prefix over the warps of D (fields <= R * 128); row counts;
    // bin totals
    {
        uint32_t run = 0u;
#pragma unroll
        for (int ww = 0; ww < kSmWarps; ++ww) run += sm.colw[ww][tid];
        ps.sm_col[(int64_t)blockIdx.x * kSmThreads + tid] = run;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t e = 0u;
#pragma unroll
            for (int ww = 0; ww < kSmWarps; ++ww) {
                const uint32_t v = sm.D[ww][h * kSmThreads + tid];
                sm.D[ww][h * kSmThreads + tid] = e;
                e += v;
            }
        }
    }
    if (tid < 2 * nr)
        ps.sm_row[(((int64_t)j * ps.ngroups + gi) * g.H + R0 + (tid >> 1)) * 2 + (tid & 1)] = sm.rowcnt[tid >> 1][tid & 1];
    if (tid < kGroupBins) {
        int t = 0;
        for (int r = 0; r < nr; ++r) t += (int)((sm.rowcnt[r][tid >> 2] >> (8 * (tid & 3))) & 0xff);
        ps.sm_tot[((int64_t)tile * ps.ngroups + gi) * kGroupBins + tid] = t;
    }
    __syncthreads();

    // 2. every CTA's sums are published
    if (tid == 0) {
        grid_arrive(ps.sm_bar);
        sm.ok = grid_wait(ps.sm_bar, gridDim.x, ps.err) ? 1 : 0;
    }
    __syncthreads();
    if (!sm.ok) return;

    // 3. carries: G over the bands above (16-bit pair fields, <= H), the row
    // carries of the band's rows over the strips to the left, the corner.
    // Loads are issued 8 at a time before they are summed (one L2 round
    // trip per 8): thread = (slice tid >> 6 of the bands, 4 words 4s..4s+3).
    {
        const int sl = tid >> 6, s4 = tid & 63;
        const uint4 *src = reinterpret_cast<const uint4 *>(ps.sm_col + ((int64_t)gi * ntiles + j) * kSmThreads) + s4;
        const int64_t stride = (int64_t)g.ns * (kSmThreads / 4);
        const bool pack8 = 8 * g.R <= 255;  // 8 bands add up packed
        uint32_t lo[4] = {0u, 0u, 0u, 0u}, hi[4] = {0u, 0u, 0u, 0u};
        for (int base = 0; base < i; base += 32) {
            uint4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int ib = base + sl + 4 * u;
                v[u] = ib < i ? __ldcg(src + ib * stride) : make_uint4(0u, 0u, 0u, 0u);
            }
            if (pack8) {
#pragma unroll
                for (int u = 1; u < 8; ++u) {
                    v[0].x += v[u].x;
                    v[0].y += v[u].y;
                    v[0].z += v[u].z;
                    v[0].w += v[u].w;
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (pack8 && u > 0) break;
                const uint32_t vw[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    lo[e] += vw[e] & 0x00ff00ffu;
                    hi[e] += (vw[e] >> 8) & 0x00ff00ffu;
                }
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            sm.Gp[sl][4 * s4 + e][0] = lo[e];
            sm.Gp[sl][4 * s4 + e][1] = hi[e];
        }
    }
    if (tid < 2 * nr) {
        const int r = tid >> 1, h = tid & 1;
        uint32_t lo = 0u, hi = 0u;
        const uint32_t *src = ps.sm_row + ((int64_t)gi * g.H + R0 + r) * 2 + h;
        const int64_t stride = (int64_t)ps.ngroups * g.H * 2;
        for (int base = 0; base < j; base += 8) {
            uint32_t v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = base + u < j ? __ldcg(src + (base + u) * stride) : 0u;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                lo += v[u] & 0x00ff00ffu;
                hi += (v[u] >> 8) & 0x00ff00ffu;
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) sm.L[r][4 * h + e] = pair_field(lo, hi, e);
    } else if (tid >= 2 * nr && tid < 2 * kSmMaxRows) {
        const int r = tid >> 1, h = tid & 1;
#pragma unroll
        for (int e = 0; e < 4; ++e) sm.L[r][4 * h + e] = 0;
    }
    {
        // corner: tiles (i', j') with i' < i, j' < j; thread = (bin tid & 7,
        // bands i' = tid >> 3, + 32, ...), then a reduction over the bands
        const int b = tid & 7;
        int t = 0;
        for (int ii = tid >> 3; ii < i; ii += kSmThreads / 8) {
            const int32_t *src = ps.sm_tot + ((int64_t)ii * g.ns * ps.ngroups + gi) * kGroupBins + b;
            for (int base = 0; base < j; base += 8) {
                int v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    v[u] = base + u < j ? __ldcg(src + (int64_t)(base + u) * ps.ngroups * kGroupBins) : 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) t += v[u];
            }
        }
        t += __shfl_xor_sync(kFull, t, 8);
        t += __shfl_xor_sync(kFull, t, 16);
        if (lane < 8) sm.cpart[w][lane] = t;
    }
    __syncthreads();
    sm.G[0][tid] = sm.Gp[0][tid][0] + sm.Gp[1][tid][0] + sm.Gp[2][tid][0] + sm.Gp[3][tid][0];
    sm.G[1][tid] = sm.Gp[0][tid][1] + sm.Gp[1][tid][1] + sm.Gp[2][tid][1] + sm.Gp[3][tid][1];
    __syncthreads();
    if (w < NB) {
        // H(R0 - 1, c) of bin w: the corner plus the row prefix of G
        int corner = 0;
#pragma unroll
        for (int k = 0; k < kSmWarps; ++k) corner += sm.cpart[k][w];
        int p[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = (2 * q + (w >> 2)) * 32 + lane;
            p[q] = pair_field(sm.G[0][k], sm.G[1][k], w & 3);
        }
        p[1] += p[0];
        p[2] += p[1];
        p[3] += p[2];
        const int base = corner + warp_incl_scan(p[3], lane) - p[3];
        *reinterpret_cast<int4 *>(&sm.Htop[w][4 * lane]) = make_int4(base + p[0], base + p[1], base + p[2], base + p[3]);
    }
    if (tid < kSmWarps * kGroupBins) {
        // the row carries of the band's rows above each warp
        const int ww = tid >> 3, b = tid & 7;
        int t = 0;
        for (int r = 0; r < ww * rpw; ++r) t += sm.L[r][b];
        sm.LS[ww][b] = t;
    }
    __syncthreads();

    // 4. the warp's rows, seeded with H(R0 + rw - 1, c) = H(R0 - 1, c) + the
    // 2-D sums of the warps above + the row carries of the rows above
    if (nrw == 0) return;
    int acc[NB][4];
    {
        uint4 dv[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) dv[m] = reinterpret_cast<const uint4 *>(sm.D[w])[m * 32 + lane];
        const int4 s0 = *reinterpret_cast<const int4 *>(&sm.LS[w][0]);
        const int4 s1 = *reinterpret_cast<const int4 *>(&sm.LS[w][4]);
        const int ls[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int4 ht = *reinterpret_cast<const int4 *>(&sm.Htop[b][4 * lane]);
            const uint4 d = dv[2 * (b >> 2) + (b & 1)];
            const int sh = (b & 2) ? 16 : 0;
            acc[b][0] = ht.x + ls[b] + (int)((d.x >> sh) & 0xffffu);
            acc[b][1] = ht.y + ls[b] + (int)((d.y >> sh) & 0xffffu);
            acc[b][2] = ht.z + ls[b] + (int)((d.z >> sh) & 0xffffu);
            acc[b][3] = ht.w + ls[b] + (int)((d.w >> sh) & 0xffffu);
        }
    }
#pragma unroll 1
    for (int k = 0; k < nrw; ++k) {
        const int r = R0 + rw + k;
        const uint32_t pk = px[0];
#pragma unroll
        for (int u = 0; u + 1 < kSmMaxRpw; ++u) px[u] = px[u + 1];  // the next row's word to the front
        uint32_t P0[4], P1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int qb = bin_of((pk >> (8 * q)) & 0xff, bins, mode);
            const unsigned d = (q < nvalid && qb >= 0) ? (unsigned)(qb - blo) : 0xFFFFFFFFu;
            P0[q] = (q ? P0[q - 1] : 0u) + (d < 4u ? (1u << (d << 3)) : 0u);
            P1[q] = (q ? P1[q - 1] : 0u) + ((d - 4u) < 4u ? (1u << ((d - 4u) << 3)) : 0u);
        }
        const uint32_t i0 = warp_incl_scan(P0[3], lane);
        const uint32_t i1 = NB > 4 ? warp_incl_scan(P1[3], lane) : 0u;
        const uint32_t x0 = i0 - P0[3], x1 = i1 - P1[3];
        const int4 l0 = *reinterpret_cast<const int4 *>(&sm.L[rw + k][0]);
        const int4 l1 = *reinterpret_cast<const int4 *>(&sm.L[rw + k][4]);
        const int rl[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t y0 = x0 + P0[q], y1 = x1 + P1[q];
#pragma unroll
            for (int b = 0; b < NB; ++b) acc[b][q] += rl[b] + (int)__byte_perm(b < 4 ? y0 : y1, 0, 0x4440 + (b & 3));
        }
        if constexpr (LAYOUT == LAYOUT_BIN_MAJOR) {
            if (c < g.P) {
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    *reinterpret_cast<int4 *>(ps.out + ((bg0 + b) * g.H + r) * g.P + c) =
                        make_int4(acc[b][0], acc[b][1], acc[b][2], acc[b][3]);
            }
        } else {
            store_slab_staged<NB>(ps.out + ps.slab_off[gr.plane] + ((int64_t)r * g.P + C0) * NB,
                                  (int)(g.P - C0 < kChunk ? g.P - C0 : kChunk), acc, stage, lane);
        }
    }
}

// 5. Rectangle queries of the frame (Eq. 2.16) after a second grid barrier,
// over every CTA, one item per (rectangle, bin): bin-major, item k = bin;
// slab, item k = 8 g + b (bin b < nb_g of group g; consecutive items read
// consecutive words of a corner's record).  The tensor was written by other
// CTAs of this launch, so its corners are read through L2 (ld.global.cg).
// An invalid rectangle writes -1 over its row and sets bit 0 of the error
// word.
template <int LAYOUT>
__device__ __forceinline__ void small_queries(const PlaneSet &ps, const SmallQuery &q)
{
    const TileGrid &g = ps.g;
    const int64_t per = LAYOUT == LAYOUT_BIN_MAJOR ? ps.B : (int64_t)ps.ngroups * kGroupBins;
    const int64_t total = q.n * per, step = (int64_t)gridDim.x * kSmThreads;
    // two items per pass, every load of both issued before any is used
    for (int64_t t0 = (int64_t)blockIdx.x * kSmThreads + threadIdx.x; t0 < total; t0 += 2 * step) {
        int32_t *o[2] = {nullptr, nullptr};
        int32_t v[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
        int rc[2][4];
        bool use[2], ok[2];
        int kk[2];
        const int32_t *pl[2];
        int64_t stride[2], word[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int64_t t = t0 + u * step;
            use[u] = t < total;
            const int64_t qi = use[u] ? t / per : 0;
            const int k = use[u] ? (int)(t - qi * per) : 0;
            kk[u] = k;
            int64_t bin;
            if (LAYOUT == LAYOUT_BIN_MAJOR) {
                bin = k;
                pl[u] = ps.out + (int64_t)k * g.H * g.P;
                stride[u] = 1;
                word[u] = 0;
            } else {
                const GroupDev gr = ps.grp[k >> 3];
                if ((k & 7) >= gr.nb) use[u] = false;
                bin = ps.chan[gr.chan].bin_off + gr.b_lo + (k & 7);
                pl[u] = ps.out + ps.slab_off[gr.plane];
                stride[u] = gr.nb;
                word[u] = k & 7;
            }
            o[u] = q.out + qi * ps.B + bin;
#pragma unroll
            for (int e = 0; e < 4; ++e) rc[u][e] = use[u] ? __ldg(q.rects + 4 * qi + e) : 0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int r0 = rc[u][0], c0 = rc[u][1], r1 = rc[u][2], c1 = rc[u][3];
            ok[u] = use[u] && r0 >= 0 && c0 >= 0 && r0 <= r1 && c0 <= c1 && r1 < g.H && c1 < g.W;
            if (ok[u]) {
                v[u][0] = __ldcg(pl[u] + ((int64_t)r1 * g.P + c1) * stride[u] + word[u]);
                if (r0 > 0) v[u][1] = __ldcg(pl[u] + ((int64_t)(r0 - 1) * g.P + c1) * stride[u] + word[u]);
                if (c0 > 0) v[u][2] = __ldcg(pl[u] + ((int64_t)r1 * g.P + (c0 - 1)) * stride[u] + word[u]);
                if (r0 > 0 && c0 > 0)
                    v[u][3] = __ldcg(pl[u] + ((int64_t)(r0 - 1) * g.P + (c0 - 1)) * stride[u] + word[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (!use[u]) continue;
            if (ok[u]) {
                *o[u] = v[u][0] - v[u][1] - v[u][2] + v[u][3];
            } else {
                *o[u] = -1;
                if (kk[u] == 0) atomicOr(ps.err, 1);
            }
        }
    }
}

template <int LAYOUT>
__global__ void __launch_bounds__(kSmThreads, 2) k_build_small(const __grid_constant__ PlaneSet ps, const SmallQuery q)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    SmallSmem &sm = *reinterpret_cast<SmallSmem *>(dsm);
    int4 *stage = reinterpret_cast<int4 *>(dsm + ((sizeof(SmallSmem) + 15) & ~size_t(15))) +
                  (threadIdx.x >> 5) * (32 * SlabStage<kGroupBins>::S);
    const int ntiles = ps.g.nb * ps.g.ns;
    switch (ps.grp[blockIdx.x / ntiles].nb) {
    case 1: small_body<LAYOUT, 1>(ps, sm, stage); break;
    case 2: small_body<LAYOUT, 2>(ps, sm, stage); break;
    case 3: small_body<LAYOUT, 3>(ps, sm, stage); break;
    case 4: small_body<LAYOUT, 4>(ps, sm, stage); break;
    case 5: small_body<LAYOUT, 5>(ps, sm, stage); break;
    case 6: small_body<LAYOUT, 6>(ps, sm, stage); break;
    case 7: small_body<LAYOUT, 7>(ps, sm, stage); break;
    default: small_body<LAYOUT, 8>(ps, sm, stage); break;
    }
    if (q.n > 0) {
        // a CTA whose first wait gave up still arrives (without waiting), so
        // that no other CTA waits for it
        __syncthreads();
        if (threadIdx.x == 0) {
            grid_arrive(ps.sm_bar);
            sm.ok = (sm.ok && grid_wait(ps.sm_bar, 2 * gridDim.x, ps.err)) ? 1 : 0;
        }
        __syncthreads();
        if (sm.ok) small_queries<LAYOUT>(ps, q);
    }
    // the last CTA past the barriers zeroes their counters for the next launch
    if (threadIdx.x == 0 && atomicAdd(ps.sm_bar + 1, 1u) == gridDim.x - 1) {
        ps.sm_bar[0] = 0u;
        ps.sm_bar[1] = 0u;
    }
}

size_t small_smem(int layout)
{
    size_t b = (sizeof(SmallSmem) + 15) & ~size_t(15);
    if (layout == LAYOUT_SLAB) b += sizeof(int4) * kSmWarps * 32 * SlabStage<kGroupBins>::S;
    return b;
}

size_t r256(size_t x) { return (x + 255) & ~size_t(255); }

// CTAs of k_build_small<layout> that fit the current device at once.
int small_capacity(int layout)
{
    static std::mutex mu;
    static int cap[64][2] = {{0}};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    const int li = layout == LAYOUT_SLAB ? 1 : 0;
    std::lock_guard<std::mutex> lk(mu);
    if (!cap[dev][li]) {
        int coop = 0, nsm = 0, per_sm = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const size_t smem = small_smem(layout);
        cudaError_t e;
        if (li) {
            e = cudaFuncSetAttribute(k_build_small<LAYOUT_SLAB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_small<LAYOUT_SLAB>, kSmThreads, smem);
        } else {
            e = cudaFuncSetAttribute(k_build_small<LAYOUT_BIN_MAJOR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_small<LAYOUT_BIN_MAJOR>, kSmThreads,
                                                                  smem);
        }
        if (e != cudaSuccess) cudaGetLastError();
        cap[dev][li] = (coop && e == cudaSuccess) ? std::max(0, per_sm) * nsm : -1;
    }
    return std::max(0, cap[dev][li]);
}

}  // namespace

bool small_plan(PlaneSet &ps)
{
    static const bool on = [] {
        const char *e = getenv("IH_SMALL");
        return !(e && e[0] == '0');
    }();
    const int H = ps.g.H, W = ps.g.W;
    if (!on || !ps.err || ps.mom || ps.wch >= 0) return false;
    if (ps.layout != LAYOUT_BIN_MAJOR && ps.layout != LAYOUT_SLAB) return false;
    if (H < 1 || W < 1 || H > 8192 || W > kSmMaxStrips * kChunk || (int64_t)ps.B * H * W > ((int64_t)1 << 25))
        return false;
    const int64_t cap = small_capacity(ps.layout);
    const int ns = (W + kChunk - 1) / kChunk;
    for (int rpw = 1; rpw <= kSmMaxRpw; rpw *= 2) {
        const int R = kSmWarps * rpw;
        const int nb = (H + R - 1) / R;
        if ((int64_t)nb * ns * ps.ngroups <= cap) {
            const int64_t P = ps.g.P;
            ps.g = make_grid(H, W, R, kChunk);
            ps.g.P = P;
            ps.small = rpw;
            return true;
        }
    }
    return false;
}

size_t small_bytes(const PlaneSet &ps)
{
    const TileGrid &g = ps.g;
    const size_t tiles = (size_t)g.nb * g.ns * ps.ngroups;
    return r256(4 * tiles * kSmThreads) + r256(8 * (size_t)g.ns * ps.ngroups * g.H) + r256(4 * tiles * kGroupBins) +
           r256(8);
}

void carve_small(PlaneSet &ps, void *base)
{
    const TileGrid &g = ps.g;
    const size_t tiles = (size_t)g.nb * g.ns * ps.ngroups;
    char *s = static_cast<char *>(base);
    ps.sm_col = reinterpret_cast<uint32_t *>(s);
    s += r256(4 * tiles * kSmThreads);
    ps.sm_row = reinterpret_cast<uint32_t *>(s);
    s += r256(8 * (size_t)g.ns * ps.ngroups * g.H);
    ps.sm_tot = reinterpret_cast<int32_t *>(s);
    s += r256(4 * tiles * kGroupBins);
    ps.sm_bar = reinterpret_cast<unsigned int *>(s);
}

int launch_build_small(const PlaneSet &ps, cudaStream_t st, const Prof *prof, const SmallQuery *queries)
{
    const SmallQuery q = queries ? *queries : SmallQuery{nullptr, 0, nullptr};
    // the counters of fresh scratch are zeroed here; a launch leaves them zero
    if (!ps.sm_zeroed && cudaMemsetAsync(ps.sm_bar, 0, 2 * sizeof(unsigned int), st) != cudaSuccess) return -1;
    const unsigned ctas = (unsigned)((int64_t)ps.g.nb * ps.g.ns * ps.ngroups);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(kSmThreads);
    cfg.dynamicSmemBytes = small_smem(ps.layout);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    prof_mark(prof, KID_SMALL, 0, st);
    if (ps.layout == LAYOUT_SLAB)
        cudaLaunchKernelEx(&cfg, k_build_small<LAYOUT_SLAB>, ps, q);
    else
        cudaLaunchKernelEx(&cfg, k_build_small<LAYOUT_BIN_MAJOR>, ps, q);
    prof_mark(prof, KID_SMALL, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace ih
