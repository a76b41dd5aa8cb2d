// k_build.cu -- integral histograms (Eq. 2.15) and moment planes (Eq. 3.4)
// on a grid of tiles, every output cell written once.
//
// Algorithm 5 adds Q(k, I(x,y)) into a recurrence that is serial along rows
// and columns.  The frame is cut into bands of R rows and strips of Wc
// columns and three kernels remove the serial dependence (ih_internal.cuh):
//
// k_tile_sums_all  per (tile, window of <= 16 bins of one channel), the
//   window's column sums down the band, row sums along the strip and tile
//   sum, all windows of a frame in one launch.  A window of an unweighted
//   channel takes 4 warps: each pixel's bin is an 8-bit field of packed
//   words, column counts add up in registers and a row's totals are one
//   warp reduction per word.  A window of the weighted channel takes a
//   256-thread CTA that stages the tile's bins in shared memory as bytes and
//   walks 32-pixel pieces of columns and rows, flushing each run of equal
//   bins with one shared atomic add; it also sums the offsets (r-R0),
//   (r-R0)^2 per column and (c-C0), (c-C0)^2 per row, which are small enough
//   for int32; the carry scan rebuilds the global int64 moment carries from
//   them.
// k_carry_scan  exclusive prefixes over bands (G), strips (L) and both
//   (corners), int32 for counts and int64 for the moments.
// count tiles  one warp per (tile, group of <= 8 bins).  A lane owns 4
//   adjacent columns of a 128-column chunk; per row each pixel's bin becomes
//   a one-hot packed as 8-bit fields (4 bins per 32-bit word), so one
//   in-lane prefix and one warp shuffle scan of two words give the row
//   prefix of all 8 bins (a field never exceeds 128, the chunk width).  Each
//   column's running sum down the band lives in registers; each cell is
//   stored once with 16-byte stores.  Pixel rows are prefetched 4 rows ahead.
// moment tiles  one warp per (tile, bin of the weighted channel); the same
//   walk produces the four moment planes.  With u the column offset inside
//   the chunk, the row prefixes of Q, u Q and u^2 Q are packed into two words
//   (count: 8 bits, sum of u: 24 bits; sum of u^2: 32 bits), scanned once,
//   and expanded to Sum c Q and Sum c^2 Q with the chunk's base column:
//   c = C + u gives Sum c Q = C n + Sum u Q, Sum c^2 Q = C^2 n + 2C Sum u Q +
//   Sum u^2 Q.  The row-weighted planes accumulate r * (row prefix of Q) and
//   r^2 * (row prefix of Q).  All moment arithmetic is exact in int64.
//
// k_tiles runs the count units and then the moment units of a frame in one
// launch (k_tiles_count when the frame has no moment planes); k_tiles_b does
// the same over the frames of a batch.
//
// These kernels wait on no other CTA: the only inter-CTA data flow is through
// the carry arrays between launches on one stream.  Two opt-in kernels at the
// end of this file do wait, with bounded polls: the persistent batched build
// (per-frame phase counters) and the one-pass build of small frames
// (decoupled look-back over bands); the default small-frame build is in
// k_small.cu (one grid barrier in a cooperative launch).
#include <algorithm>
#include <mutex>

#include <stdlib.h>

#include "ih_internal.cuh"
#include "k_tilecore.cuh"

namespace ih {

namespace {

// count tiles: two rows in flight per step (more ILP) or one (fewer
// registers, so that 4 CTAs fit an SM); the record layout's units, whose
// group may draw on two channels, take the second
template <int LAYOUT>
constexpr bool pair_rows() { return LAYOUT != LAYOUT_RECORD; }
// (the batched kernel, which serves every layout with one register budget,
// always takes the first)
constexpr int kQStride = kSumCols + 4;  // padded row of the staged byte tile

// ------------------------------------------------------------- tile sums

constexpr int kSumThreads = 256;
constexpr int kWalk = 32;  // pixels one thread walks per item

// Dynamic shared memory of a run-length tile-sums CTA (tile_sums_body) for
// bands of up to R rows: the staged byte tile, the column counters of one
// pass and the row counters of the strip (and, with WT, the offset sums of
// both).  The engine runs this CTA for windows of the weighted channel; the
// other windows take the packed-field groups of tile_sums_count_body.
__host__ __device__ constexpr size_t sums_q_bytes(int R) { return ((size_t)R * kQStride + 15) & ~size_t(15); }
__host__ __device__ constexpr size_t sums_smem_bytes(int R, bool weighted)
{
    return sums_q_bytes(R) + (weighted ? 3 : 1) * ((size_t)kWindowBins * kSumCols * 4 + (size_t)kWindowBins * R * 4);
}

// Bins of 4 pixels packed in a word, as window-local bytes (0xFF: none).
__device__ __forceinline__ uint32_t window_bins4(uint32_t px, const ChanDev &ch, int b_lo, int nbw, int valid)
{
    uint32_t out = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int v = k < valid ? bin_of((px >> (8 * k)) & 0xff, ch.bins, ch.mode) - b_lo : -1;
        out |= (uint32_t)((v >= 0 && v < nbw) ? v : 0xFF) << (8 * k);
    }
    return out;
}

// Run-length walks over the staged byte tile.  Each item covers kWalk
// pixels of one column (down the band) or of one row (along the pass); a run
// of equal bins is flushed with one shared-memory atomic, so the counters of
// a column or row shared by several items add up exactly.
template <bool WT>
__device__ __forceinline__ void walk_column(const uint8_t *qt, int t, int rlo, int rhi, int32_t *cnt, int32_t *su,
                                            int32_t *suu)
{
    int cur = 0xFF, n = 0, s1 = 0, s2 = 0;
    for (int rr = rlo; rr < rhi; ++rr) {
        const int q = qt[rr * kQStride + t];
        if (q != cur) {
            if (cur != 0xFF) {
                atomicAdd(cnt + cur * kSumCols + t, n);
                if (WT) {
                    atomicAdd(su + cur * kSumCols + t, s1);
                    atomicAdd(suu + cur * kSumCols + t, s2);
                }
            }
            cur = q;
            n = s1 = s2 = 0;
        }
        ++n;
        if (WT) {
            s1 += rr;
            s2 += rr * rr;
        }
    }
    if (cur != 0xFF) {
        atomicAdd(cnt + cur * kSumCols + t, n);
        if (WT) {
            atomicAdd(su + cur * kSumCols + t, s1);
            atomicAdd(suu + cur * kSumCols + t, s2);
        }
    }
}

template <bool WT>
__device__ __forceinline__ void walk_row(const uint8_t *qt, int t, int clo, int chi, int u0, int R, int32_t *cnt,
                                         int32_t *sv, int32_t *svv)
{
    int cur = 0xFF, n = 0, s1 = 0, s2 = 0;
    const uint32_t *rowq = reinterpret_cast<const uint32_t *>(qt + t * kQStride);
    for (int c4 = clo; c4 < chi; c4 += 4) {
        const uint32_t w4 = rowq[c4 >> 2];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int q = (w4 >> (8 * e)) & 0xff;
            if (q != cur) {
                if (cur != 0xFF) {
                    atomicAdd(cnt + cur * R + t, n);
                    if (WT) {
                        atomicAdd(sv + cur * R + t, s1);
                        atomicAdd(svv + cur * R + t, s2);
                    }
                }
                cur = q;
                n = s1 = s2 = 0;
            }
            ++n;
            if (WT) {
                const int u = u0 + c4 + e;
                s1 += u;
                s2 += u * u;
            }
        }
    }
    if (cur != 0xFF) {
        atomicAdd(cnt + cur * R + t, n);
        if (WT) {
            atomicAdd(sv + cur * R + t, s1);
            atomicAdd(svv + cur * R + t, s2);
        }
    }
}

// Tile sums of window widx over tile (band i, strip j) by one 256-thread CTA
// (WT: also the offset sums of the weighted channel).
template <bool WT>
__device__ __forceinline__ void tile_sums_body(const PlaneSet &ps, int j, int i, int widx)
{
    const TileGrid &g = ps.g;
    const GroupDev wd = ps.win[widx];
    const ChanDev &ch = ps.chan[wd.chan];
    const int R = g.R;
    const int R0 = i * R, nr = min(R, g.H - R0);
    const int C0 = j * g.Wc, C1 = min(C0 + g.Wc, g.W);
    const int nbw = wd.nb;
    const int64_t bglob = ch.bin_off + wd.b_lo;
    const int Bw = WT ? ch.bins : 0;
    const int tid = threadIdx.x;
    const bool vec16 = ((ch.pitch & 15) == 0) && ((reinterpret_cast<uintptr_t>(ch.plane) & 15) == 0);

    extern __shared__ __align__(16) unsigned char sm[];
    uint8_t *qt = sm;
    int32_t *col_cnt = reinterpret_cast<int32_t *>(sm + sums_q_bytes(R));  // [16][kSumCols]
    int32_t *row_cnt = col_cnt + kWindowBins * kSumCols;                   // [16][R]
    int32_t *col_su = row_cnt + kWindowBins * R;
    int32_t *col_suu = col_su + kWindowBins * kSumCols;
    int32_t *row_sv = col_suu + kWindowBins * kSumCols;
    int32_t *row_svv = row_sv + kWindowBins * R;

    for (int k = tid; k < kWindowBins * R; k += kSumThreads) {
        row_cnt[k] = 0;
        if (WT) {
            row_sv[k] = 0;
            row_svv[k] = 0;
        }
    }
    const int rsegs = (nr + kWalk - 1) / kWalk;
    for (int cp = C0; cp < C1; cp += kSumCols) {
        const int cw = min(kSumCols, C1 - cp);
        for (int k = tid; k < kWindowBins * kSumCols; k += kSumThreads) {
            col_cnt[k] = 0;
            if (WT) {
                col_su[k] = 0;
                col_suu[k] = 0;
            }
        }
        // stage the window-local bins of the nr x kSumCols pass, 16 pixels per
        // item; all of a thread's loads are issued before any is used
        constexpr int kSeg = kSumCols / 16;
        constexpr int kItems = kMaxBandRows * kSeg / kSumThreads;
        uint4 v[kItems];
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const int idx = tid + k * kSumThreads, rr = idx / kSeg, c16 = (idx % kSeg) * 16;
            v[k] = make_uint4(0, 0, 0, 0);
            if (rr < nr && c16 < cw) {
                const uint8_t *src = ch.plane + (int64_t)(R0 + rr) * ch.pitch + cp + c16;
                if (vec16 && c16 + 16 <= cw) {
                    v[k] = __ldg(reinterpret_cast<const uint4 *>(src));
                } else {
                    uint32_t w[4] = {0, 0, 0, 0};
                    for (int e = 0; e < 16 && c16 + e < cw; ++e) w[e >> 2] |= (uint32_t)__ldg(src + e) << (8 * (e & 3));
                    v[k] = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const int idx = tid + k * kSumThreads, rr = idx / kSeg, c16 = (idx % kSeg) * 16;
            if (rr < nr) {
                const int valid = cw - c16;
                uint32_t *dst = reinterpret_cast<uint32_t *>(qt + rr * kQStride + c16);
                dst[0] = window_bins4(v[k].x, ch, wd.b_lo, nbw, valid);
                dst[1] = window_bins4(v[k].y, ch, wd.b_lo, nbw, valid - 4);
                dst[2] = window_bins4(v[k].z, ch, wd.b_lo, nbw, valid - 8);
                dst[3] = window_bins4(v[k].w, ch, wd.b_lo, nbw, valid - 12);
            }
        }
        __syncthreads();
        // column items: (row segment, column), consecutive threads take
        // consecutive columns; row items: (column segment, row), consecutive
        // threads take consecutive rows (the padded row stride avoids bank
        // conflicts)
        const int csegs = (cw + kWalk - 1) / kWalk;
        const int ncol = rsegs * cw, nrow = csegs * nr;
        for (int it = tid; it < ncol + nrow; it += kSumThreads) {
            if (it < ncol) {
                const int seg = it / cw, t = it - seg * cw;
                walk_column<WT>(qt, t, seg * kWalk, min(nr, seg * kWalk + kWalk), col_cnt, col_su, col_suu);
            } else {
                const int k = it - ncol, seg = k / nr, t = k - seg * nr;
                walk_row<WT>(qt, t, seg * kWalk, min(cw, seg * kWalk + kWalk), cp - C0, R, row_cnt, row_sv, row_svv);
            }
        }
        __syncthreads();
        for (int k = tid; k < nbw * kSumCols; k += kSumThreads) {
            const int b = k / kSumCols, cc = k % kSumCols;
            if (cc < cw) {
                ps.colsum[((int64_t)i * ps.B + bglob + b) * g.W + cp + cc] = col_cnt[b * kSumCols + cc];
                if (WT) {
                    const int64_t o = ((int64_t)i * Bw + wd.b_lo + b) * g.W + cp + cc;
                    ps.col_su[o] = col_su[b * kSumCols + cc];
                    ps.col_suu[o] = col_suu[b * kSumCols + cc];
                }
            }
        }
        __syncthreads();
    }
    for (int b = tid >> 5; b < nbw; b += kSumThreads / 32) {
        for (int rr = tid & 31; rr < nr; rr += 32) {
            ps.rowsum[((int64_t)j * ps.B + bglob + b) * g.H + R0 + rr] = row_cnt[b * R + rr];
            if (WT) {
                const int64_t o = ((int64_t)j * Bw + wd.b_lo + b) * g.H + R0 + rr;
                ps.row_sv[o] = row_sv[b * R + rr];
                ps.row_svv[o] = row_svv[b * R + rr];
            }
        }
    }
    if (tid < nbw) {
        const int b = tid;
        int32_t n = 0;
        long long su = 0, suu = 0, sv = 0, svv = 0;
        for (int rr = 0; rr < nr; ++rr) {
            const int32_t x = row_cnt[b * R + rr];
            n += x;
            if (WT) {
                su += (long long)rr * x;
                suu += (long long)rr * rr * x;
                sv += row_sv[b * R + rr];
                svv += row_svv[b * R + rr];
            }
        }
        ps.tilesum[((int64_t)i * g.ns + j) * ps.B + bglob + b] = n;
        if (WT) {
            int64_t *tw = ps.tile_w + (((int64_t)i * g.ns + j) * Bw + wd.b_lo + b) * 4;
            tw[0] = su;
            tw[1] = suu;
            tw[2] = sv;
            tw[3] = svv;
        }
    }
}

// Tile sums of a window of an unweighted channel, 4 warps per (band, strip,
// window).  Row rr of the band goes to warp rr % 4; a lane holds 4 adjacent
// columns of the 128-column pass.  A pixel's window-local bin is one 4-bit
// field of two words (8 bins per word), so a pixel costs a shift and two
// adds; a lane's per-column fields add up at most 15 rows before they are
// spread into NW byte words (at most 32 rows per field), and a row's fields
// over the warp are spread into bytes and reduced by one redux.sync.add per
// word (at most 128 per field), so no field overflows.
constexpr int kCntThreads = 128;

// The 128 threads of one group (a whole CTA, or half of a 256-thread CTA:
// tid = thread index in the group, bar = the group's named barrier).
__device__ __forceinline__ void group_sync(int bar)
{
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(kCntThreads) : "memory");
}

template <int NW>
__device__ __forceinline__ void tile_sums_count_body(const PlaneSet &ps, int j, int i, int widx,
                                                     uint32_t (*colpk)[16][32], int32_t (*rows)[kMaxBandRows],
                                                     int tid, int bar)
{
    const TileGrid &g = ps.g;
    const GroupDev wd = ps.win[widx];
    const ChanDev &ch = ps.chan[wd.chan];
    const int R0 = i * g.R, nr = min(g.R, g.H - R0);
    const int C0 = j * g.Wc, C1 = min(C0 + g.Wc, g.W);
    const int nbw = wd.nb, blo = wd.b_lo;
    const int64_t bglob = ch.bin_off + wd.b_lo;
    const int lane = tid & 31, wid = tid >> 5;
    const uint8_t *const pl = ch.plane;
    const int64_t pt = ch.pitch;
    const int bins = ch.bins, mode = ch.mode;
    const bool vec_ok = ((pt & 3) == 0) && ((reinterpret_cast<uintptr_t>(pl) & 3) == 0);

    {
        // zero the row counters (no division by nr: all of rows[][], 16-byte stores)
        int4 *r4 = reinterpret_cast<int4 *>(&rows[0][0]);
        for (int k = tid; k < kWindowBins * kMaxBandRows / 4; k += kCntThreads) r4[k] = make_int4(0, 0, 0, 0);
    }
    group_sync(bar);
    for (int cp = C0; cp < C1; cp += kChunk) {
        const int c = cp + lane * 4;
        const int nvalid = max(0, min(4, C1 - c));
        uint32_t col[4][NW];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int k = 0; k < NW; ++k) col[jj][k] = 0u;
        // two rows of this warp in flight.  A pixel's bin d (0..15) is a 4-bit
        // field of two words (lo: d < 8, hi: d >= 8); a column's fields add up
        // at most 15 rows before they are spread into the byte words col[jj]
        // (word 2h + o holds bins 8h + o, 8h + o + 2, 8h + o + 4, 8h + o + 6)
        uint32_t pa = wid < nr ? load4(pl, pt, R0 + wid, c, C1, vec_ok) : 0u;
        uint32_t pb = wid + 4 < nr ? load4(pl, pt, R0 + wid + 4, c, C1, vec_ok) : 0u;
        uint32_t nib[4][2] = {{0u, 0u}, {0u, 0u}, {0u, 0u}, {0u, 0u}};
        int pend = 0;
        for (int rr = wid; rr < nr; rr += 4) {
            const uint32_t px = pa;
            pa = pb;
            if (rr + 8 < nr) pb = load4(pl, pt, R0 + rr + 8, c, C1, vec_ok);
            uint32_t rlo = 0u, rhi = 0u;
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int q = bin_of((px >> (8 * jj)) & 0xff, bins, mode) - blo;
                const unsigned d = (jj < nvalid && q >= 0 && q < nbw) ? (unsigned)q : 16u;
                const uint32_t e = 1u << ((d & 7u) << 2);
                const uint32_t el = d < 8u ? e : 0u;
                rlo += el;
                nib[jj][0] += el;
                if (NW > 2) {
                    const uint32_t eh = (d - 8u) < 8u ? e : 0u;
                    rhi += eh;
                    nib[jj][1] += eh;
                }
            }
            if (++pend == 15) {
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                    for (int h = 0; h < NW / 2; ++h) {
                        col[jj][2 * h] += nib[jj][h] & 0x0F0F0F0Fu;
                        col[jj][2 * h + 1] += (nib[jj][h] >> 4) & 0x0F0F0F0Fu;
                        nib[jj][h] = 0u;
                    }
                pend = 0;
            }
            // the row's counts over the pass: fields <= 4 per lane, spread
            // into bytes and reduced over the warp (<= 128 per field)
            uint32_t rw[NW];
            rw[0] = __reduce_add_sync(kFull, rlo & 0x0F0F0F0Fu);
            rw[1] = __reduce_add_sync(kFull, (rlo >> 4) & 0x0F0F0F0Fu);
            if (NW > 2) {
                rw[2] = __reduce_add_sync(kFull, rhi & 0x0F0F0F0Fu);
                rw[3] = __reduce_add_sync(kFull, (rhi >> 4) & 0x0F0F0F0Fu);
            }
            if (lane < nbw) {
                const int wsel = ((lane >> 3) << 1) | (lane & 1);
                uint32_t w = rw[0];
#pragma unroll
                for (int k = 1; k < NW; ++k)
                    if (wsel == k) w = rw[k];
                rows[lane][rr] += (int32_t)((w >> (((lane & 7) >> 1) << 3)) & 0xFFu);
            }
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int h = 0; h < NW / 2; ++h) {
                col[jj][2 * h] += nib[jj][h] & 0x0F0F0F0Fu;
                col[jj][2 * h + 1] += (nib[jj][h] >> 4) & 0x0F0F0F0Fu;
            }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
            for (int k = 0; k < NW; ++k) colpk[wid][jj * 4 + k][lane] = col[jj][k];
        group_sync(bar);
        {
            // column 4 l + jj of the pass: thread (warp jj, lane l)
            const int l = lane, jj = wid, cc = 4 * l + jj;
            if (cp + cc < C1) {
                uint32_t sw[NW];
#pragma unroll
                for (int k = 0; k < NW; ++k)
                    sw[k] = colpk[0][jj * 4 + k][l] + colpk[1][jj * 4 + k][l] + colpk[2][jj * 4 + k][l] +
                            colpk[3][jj * 4 + k][l];
                int32_t *dst = ps.colsum + ((int64_t)i * ps.B + bglob) * g.W + cp + cc;
#pragma unroll
                for (int b = 0; b < 4 * NW; ++b)
                    if (b < nbw)
                        dst[(int64_t)b * g.W] = (int32_t)((sw[((b >> 3) << 1) | (b & 1)] >> (((b & 7) >> 1) << 3)) & 0xFFu);
            }
        }
        group_sync(bar);
    }
    for (int b = wid; b < nbw; b += 4) {
        int32_t *dst = ps.rowsum + ((int64_t)j * ps.B + bglob + b) * g.H + R0;
        for (int rr = lane; rr < nr; rr += 32) dst[rr] = rows[b][rr];
    }
    for (int b = wid; b < nbw; b += 4) {
        int32_t t = 0;
        for (int rr = lane; rr < nr; rr += 32) t += rows[b][rr];
        t = (int32_t)__reduce_add_sync(kFull, (uint32_t)t);
        if (lane == 0) ps.tilesum[((int64_t)i * g.ns + j) * ps.B + bglob + b] = t;
    }
}

// Shared memory of one count group.
struct CountSumsSmem {
    uint32_t colpk[4][16][32];
    int32_t rows[kWindowBins][kMaxBandRows];
};

__device__ __forceinline__ void tile_sums_count_group(const PlaneSet &ps, int j, int i, int widx, CountSumsSmem &sm,
                                                      int tid, int bar)
{
    if (ps.win[widx].nb <= 8)
        tile_sums_count_body<2>(ps, j, i, widx, sm.colpk, sm.rows, tid, bar);
    else
        tile_sums_count_body<4>(ps, j, i, widx, sm.colpk, sm.rows, tid, bar);
}


// Tile sums of all windows of a frame in one launch of 256-thread CTAs:
// z < nw_w: one window of the weighted channel per CTA (they take longest,
// so they go first); then two windows of the other channels per CTA, one
// per 128-thread half.
__global__ void __launch_bounds__(kSumThreads) k_tile_sums_all(const __grid_constant__ PlaneSet ps, int nw_w)
{
    pdl_wait();
    const int z = blockIdx.z;
    if (z < nw_w) {
        tile_sums_body<true>(ps, blockIdx.x, blockIdx.y, ps.nwin_count + z);
        return;
    }
    extern __shared__ __align__(16) unsigned char dsm[];
    const int half = threadIdx.x >> 7, widx = 2 * (z - nw_w) + half;
    if (widx >= ps.nwin_count) return;  // the odd window's CTA: a whole idle half
    CountSumsSmem &sm = reinterpret_cast<CountSumsSmem *>(dsm)[half];
    tile_sums_count_group(ps, blockIdx.x, blockIdx.y, widx, sm, threadIdx.x & 127, 1 + half);
}

// Largest f in [0, n) with pre[f] <= x (pre is a prefix sum of n counts).
__device__ __forceinline__ int find_frame(const int64_t *pre, int n, int64_t x)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= x)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Batched, all windows of all frames in one launch of 256-thread CTAs: the
// first nw CTAs each take one (frame, weighted-channel window, tile); then
// each CTA takes two (frame, window, tile) units
// of the other windows, one per 128-thread half (the halves may belong to
// different frames).
__global__ void __launch_bounds__(kSumThreads) k_tile_sums_all_b(const BatchDev bd, unsigned nw)
{
    pdl_wait();
    if (blockIdx.x < nw) {
        const int64_t flat = blockIdx.x;
        const int f = find_frame(bd.pre_sums1, bd.n, flat);
        const PlaneSet &ps = bd.sets[f];
        const int64_t local = flat - bd.pre_sums1[f], per = (int64_t)ps.g.ns * ps.g.nb;
        const int z = (int)(local / per), rem = (int)(local % per);
        tile_sums_body<true>(ps, rem % ps.g.ns, rem / ps.g.ns, ps.nwin_count + z);
        return;
    }
    extern __shared__ __align__(16) unsigned char dsm[];
    const int half = threadIdx.x >> 7;
    const int64_t flat = 2 * (int64_t)(blockIdx.x - nw) + half;
    if (flat >= bd.pre_sums0[bd.n]) return;  // an idle half at the end
    const int f = find_frame(bd.pre_sums0, bd.n, flat);
    const PlaneSet &ps = bd.sets[f];
    const int64_t local = flat - bd.pre_sums0[f], per = (int64_t)ps.g.ns * ps.g.nb;
    const int z = (int)(local / per), rem = (int)(local % per);
    CountSumsSmem &sm = reinterpret_cast<CountSumsSmem *>(dsm)[half];
    tile_sums_count_group(ps, rem % ps.g.ns, rem / ps.g.ns, z, sm, threadIdx.x & 127, 1 + half);
}

// ------------------------------------------------------------- carry scan
//
// G and L are exclusive prefixes over bands and strips.  The tile corners
// are split in two: here, per (band i, bin), the exclusive prefix over strips
// of the tile sums ("corner" then holds sum_{j'<j} tilesum(i, j')); the tiles
// kernels add these up over the bands above their own (a warp reduction).

constexpr int kScanBatch = 8;

__device__ __forceinline__ int64_t carry_scan_items(const PlaneSet &ps)
{
    return (int64_t)ps.B * ps.g.W + (int64_t)ps.B * ps.g.H + (int64_t)ps.g.nb * ps.B;
}

__device__ __forceinline__ void carry_scan_item(const PlaneSet &ps, int64_t t)
{
    const TileGrid &g = ps.g;
    const int64_t B = ps.B;
    const int wch = ps.wch;
    const int64_t bin0 = wch >= 0 ? ps.chan[wch].bin_off : 0;
    const int64_t Bw = wch >= 0 ? ps.chan[wch].bins : 0;
    const int64_t nA = B * g.W, nB = B * g.H, nC = (int64_t)g.nb * B;
    // the corner scans (the longest items) take the first indices
    t = t < nC ? t + nA + nB : t - nC;
    {
        if (t < nA) {  // G(i, c, b): exclusive over bands
            const int64_t b = t / g.W, c = t % g.W, wb = b - bin0;
            const bool wt = wb >= 0 && wb < Bw;
            int32_t run = 0;
            long long rr1 = 0, rr2 = 0;
            for (int i0 = 0; i0 < g.nb; i0 += kScanBatch) {
                const int ni = min(kScanBatch, g.nb - i0);
                int32_t v[kScanBatch];
#pragma unroll
                for (int k = 0; k < kScanBatch; ++k)
                    if (k < ni) v[k] = ps.colsum[(int64_t)(i0 + k) * nA + t];
                int32_t su[kScanBatch], suu[kScanBatch];
                if (wt) {
#pragma unroll
                    for (int k = 0; k < kScanBatch; ++k)
                        if (k < ni) {
                            const int64_t o = ((int64_t)(i0 + k) * Bw + wb) * g.W + c;
                            su[k] = ps.col_su[o];
                            suu[k] = ps.col_suu[o];
                        }
                }
#pragma unroll
                for (int k = 0; k < kScanBatch; ++k) {
                    if (k < ni) {
                        const int i = i0 + k;
                        ps.colsum[(int64_t)i * nA + t] = run;
                        if (wt) {
                            const int64_t o = ((int64_t)i * Bw + wb) * g.W + c;
                            const long long R0 = (long long)i * g.R;
                            ps.g_r[o] = rr1;
                            ps.g_rr[o] = rr2;
                            rr1 += R0 * v[k] + su[k];
                            rr2 += R0 * R0 * v[k] + 2 * R0 * su[k] + suu[k];
                        }
                        run += v[k];
                    }
                }
            }
        } else if (t < nA + nB) {  // L(j, r, b): exclusive over strips
            const int64_t u = t - nA;
            const int64_t b = u / g.H, r = u % g.H, wb = b - bin0;
            const bool wt = wb >= 0 && wb < Bw;
            int32_t run = 0;
            long long rc1 = 0, rc2 = 0;
            for (int j0 = 0; j0 < g.ns; j0 += kScanBatch) {
                const int nj = min(kScanBatch, g.ns - j0);
                int32_t v[kScanBatch], sv[kScanBatch], svv[kScanBatch];
#pragma unroll
                for (int k = 0; k < kScanBatch; ++k)
                    if (k < nj) v[k] = ps.rowsum[(int64_t)(j0 + k) * nB + u];
                if (wt) {
#pragma unroll
                    for (int k = 0; k < kScanBatch; ++k)
                        if (k < nj) {
                            const int64_t o = ((int64_t)(j0 + k) * Bw + wb) * g.H + r;
                            sv[k] = ps.row_sv[o];
                            svv[k] = ps.row_svv[o];
                        }
                }
#pragma unroll
                for (int k = 0; k < kScanBatch; ++k) {
                    if (k < nj) {
                        const int jj = j0 + k;
                        ps.rowsum[(int64_t)jj * nB + u] = run;
                        if (wt) {
                            const int64_t o = ((int64_t)jj * Bw + wb) * g.H + r;
                            const long long C0 = (long long)jj * g.Wc;
                            ps.l_c[o] = rc1;
                            ps.l_cc[o] = rc2;
                            rc1 += C0 * v[k] + sv[k];
                            rc2 += C0 * C0 * v[k] + 2 * C0 * sv[k] + svv[k];
                        }
                        run += v[k];
                    }
                }
            }
        } else {  // per band: exclusive prefix over strips of the tile sums
            const int64_t u = t - nA - nB;
            const int i = (int)(u / B);
            const int64_t b = u % B, wb = b - bin0;
            const bool wt = wb >= 0 && wb < Bw;
            const long long R0 = (long long)i * g.R;
            int32_t run = 0;
            long long rw[4] = {0, 0, 0, 0};  // w = c, r, c^2, r^2
            for (int j0 = 0; j0 < g.ns; j0 += kScanBatch) {
                const int nj = min(kScanBatch, g.ns - j0);
                int32_t v[kScanBatch];
#pragma unroll
                for (int k = 0; k < kScanBatch; ++k)
                    if (k < nj) v[k] = ps.tilesum[((int64_t)i * g.ns + j0 + k) * B + b];
#pragma unroll
                for (int k = 0; k < kScanBatch; ++k)
                    if (k < nj) {
                        ps.corner[((int64_t)i * g.ns + j0 + k) * B + b] = run;
                        run += v[k];
                    }
                if (wt) {
                    for (int k = 0; k < nj; ++k) {
                        const int j = j0 + k;
                        const int64_t wi = (((int64_t)i * g.ns + j) * Bw + wb) * 4;
                        const int64_t *tw = ps.tile_w + wi;
                        int64_t *cw = ps.corner_w + wi;
                        cw[0] = rw[0];
                        cw[1] = rw[1];
                        cw[2] = rw[2];
                        cw[3] = rw[3];
                        const long long C0 = (long long)j * g.Wc, n = ps.tilesum[((int64_t)i * g.ns + j) * B + b];
                        rw[0] += C0 * n + tw[2];
                        rw[1] += R0 * n + tw[0];
                        rw[2] += C0 * C0 * n + 2 * C0 * tw[2] + tw[3];
                        rw[3] += R0 * R0 * n + 2 * R0 * tw[0] + tw[1];
                    }
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_carry_scan(const __grid_constant__ PlaneSet ps)
{
    pdl_wait();
    const int64_t total = carry_scan_items(ps);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
        carry_scan_item(ps, t);
}

__global__ void __launch_bounds__(256) k_carry_scan_b(const BatchDev bd)
{
    pdl_wait();
    const int64_t total = bd.pre_scan[bd.n];
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int f = find_frame(bd.pre_scan, bd.n, t);
        carry_scan_item(bd.sets[f], t - bd.pre_scan[f]);
    }
}

// Sum over the bands above band i of a per-band value (the corner's second
// half): lanes take bands i' = lane, lane + 32, ... < i, then a warp reduction.
template <typename T, typename F>
__device__ __forceinline__ T sum_bands_above(int i, int lane, F at)
{
    T s = 0;
    for (int ib = lane; ib < i; ib += 32) s += at(ib);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(kFull, s, d);
    return s;
}

// ------------------------------------------------------------- count tiles

// One warp-unit of the count tiles: tile (i, j), group gi of exactly NB bins.
// LAYOUT_RECORD: NB = 8 is the group's width in the record and its
// nb + nb1 <= NB real bins may come from two channels (SEG2); the padding
// fields are never hit and hold 0.
// tr: when not null, the tile's corner H(R0-1, C0-1) per bin of the group
// (the one-pass build computes it in its CTA) instead of the sum of the
// per-band corners of the bands above.
template <int LAYOUT, int NB, bool SEG2, bool PAIR, bool UNI = false>
__device__ __forceinline__ void tiles_count_unit(const PlaneSet &ps, int i, int j, int gi, int lane,
                                                 int32_t (*RL)[kGroupBins], int4 *stage, const int32_t *tr = nullptr)
{
    const TileGrid &g = ps.g;
    const GroupDev gr = ps.grp[gi];
    const ChanDev &ch = ps.chan[gr.chan];
    const ChanDev &ch1 = ps.chan[SEG2 ? gr.chan1 : gr.chan];
    const int64_t bg0 = ch.bin_off + gr.b_lo;
    const int nbr = gr.nb + (SEG2 ? gr.nb1 : 0);  // real bins
    const int R0 = i * g.R, nr = min(g.R, g.H - R0);
    const int C0 = j * g.Wc, C1 = min(C0 + g.Wc, g.W);

    __syncwarp();
    for (int k = lane; k < nr * kGroupBins; k += 32) {
        const int rr = k / kGroupBins, b = k % kGroupBins;
        RL[rr][b] = (ps.rowsum && b < nbr) ? ps.rowsum[((int64_t)j * ps.B + bg0 + b) * g.H + R0 + rr] : 0;
    }
    int TR[NB];  // H(R0-1, chunk start - 1) per bin: the tile corner to begin with
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if (tr)
            TR[b] = b < nbr ? tr[b] : 0;
        else
            TR[b] = (ps.corner && b < nbr) ? sum_bands_above<int>(i, lane, [&](int ib) {
                return ps.corner[((int64_t)ib * g.ns + j) * ps.B + bg0 + b];
            }) : 0;
    }
    __syncwarp();

    // the channels' descriptors in registers for the row loop
    const uint8_t *const pl0 = ch.plane, *const pl1 = ch1.plane;
    const int64_t pt0 = ch.pitch, pt1 = ch1.pitch;
    const int bins0 = ch.bins, mode0 = UNI ? 0 : ch.mode, bins1 = ch1.bins, mode1 = UNI ? 0 : ch1.mode;
    const int blo0 = gr.b_lo, nb0 = gr.nb, blo1 = gr.b_lo1, nbs1 = gr.nb1;
    const bool vec_ok = ((pt0 & 3) == 0) && ((reinterpret_cast<uintptr_t>(pl0) & 3) == 0);
    const bool vec_ok1 = ((pt1 & 3) == 0) && ((reinterpret_cast<uintptr_t>(pl1) & 3) == 0);
    // the second segment's loads and bin tests only where the group has one
    // (a warp-uniform branch inside the one loop body of the frame)
    const bool two = SEG2 && nbs1 > 0;
    for (int cc = C0; cc < C1; cc += kChunk) {
        const int c = cc + lane * 4;
        const int nvalid = max(0, min(4, C1 - c));
        int acc[NB][4];
        // seed each column with H(R0-1, c): the corner plus the prefix of G
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            int p[4] = {0, 0, 0, 0};
            if (ps.colsum && b < nbr) {
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
                    if (jj < nvalid) p[jj] = ps.colsum[((int64_t)i * ps.B + bg0 + b) * g.W + c + jj];
            }
            p[1] += p[0];
            p[2] += p[1];
            p[3] += p[2];
            const int incl = warp_incl_scan(p[3], lane);
            const int base = TR[b] + (incl - p[3]);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) acc[b][jj] = p[jj] + base;
            TR[b] += __shfl_sync(kFull, incl, 31);
        }
        uint32_t pf[4], pg[4];  // pixel words 4 rows ahead (pg: the second segment's channel)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            pf[k] = (k < nr) ? load4(pl0, pt0, R0 + k, c, C1, vec_ok) : 0u;
            pg[k] = (two && k < nr) ? load4(pl1, pt1, R0 + k, c, C1, vec_ok1) : 0u;
        }
        if constexpr (PAIR) {
        for (int rr0 = 0; rr0 < nr; rr0 += 4) {
            // two rows at a time: their shuffle scans are independent
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ra = rr0 + 2 * h, rb = ra + 1;
                if (ra >= nr) break;  // warp-uniform
                const bool hasb = rb < nr;
                const uint32_t pxa = pf[2 * h], pxb = pf[2 * h + 1];
                const uint32_t pya = pg[2 * h], pyb = pg[2 * h + 1];
                if (ra + 4 < nr) pf[2 * h] = load4(pl0, pt0, R0 + ra + 4, c, C1, vec_ok);
                if (rb + 4 < nr) pf[2 * h + 1] = load4(pl0, pt0, R0 + rb + 4, c, C1, vec_ok);
                if (SEG2 && ra + 4 < nr) pg[2 * h] = load4(pl1, pt1, R0 + ra + 4, c, C1, vec_ok1);
                if (SEG2 && rb + 4 < nr) pg[2 * h + 1] = load4(pl1, pt1, R0 + rb + 4, c, C1, vec_ok1);
                // packed one-hot of each row's 4 pixels and its in-lane prefix
                uint32_t Pa0[4], Pa1[4], Pb0[4], Pb1[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int qa = bin_of((pxa >> (8 * jj)) & 0xff, bins0, mode0);
                    const int qb = bin_of((pxb >> (8 * jj)) & 0xff, bins0, mode0);
                    unsigned da = (jj < nvalid && qa >= 0) ? (unsigned)(qa - blo0) : 0xFFFFFFFFu;
                    unsigned db = (jj < nvalid && qb >= 0 && hasb) ? (unsigned)(qb - blo0) : 0xFFFFFFFFu;
                    uint32_t ea0 = 0u, ea1 = 0u, eb0 = 0u, eb1 = 0u;
                    if (SEG2) {
                        // a bin of the first channel beyond the group is
                        // dropped; the second channel's bins follow at field nb
                        if (da >= (unsigned)nb0) da = 0xFFFFFFFFu;
                        if (db >= (unsigned)nb0) db = 0xFFFFFFFFu;
                        const int ya = bin_of((pya >> (8 * jj)) & 0xff, bins1, mode1);
                        const int yb = bin_of((pyb >> (8 * jj)) & 0xff, bins1, mode1);
                        unsigned fa = (jj < nvalid && ya >= 0) ? (unsigned)(ya - blo1) : 0xFFFFFFFFu;
                        unsigned fb = (jj < nvalid && yb >= 0 && hasb) ? (unsigned)(yb - blo1) : 0xFFFFFFFFu;
                        fa = fa < (unsigned)nbs1 ? fa + nb0 : 0xFFFFFFFFu;
                        fb = fb < (unsigned)nbs1 ? fb + nb0 : 0xFFFFFFFFu;
                        ea0 = fa < 4u ? (1u << (fa << 3)) : 0u;
                        ea1 = (fa - 4u) < 4u ? (1u << ((fa - 4u) << 3)) : 0u;
                        eb0 = fb < 4u ? (1u << (fb << 3)) : 0u;
                        eb1 = (fb - 4u) < 4u ? (1u << ((fb - 4u) << 3)) : 0u;
                    }
                    Pa0[jj] = (jj ? Pa0[jj - 1] : 0u) + (da < 4u ? (1u << (da << 3)) : 0u) + ea0;
                    Pa1[jj] = (jj ? Pa1[jj - 1] : 0u) + ((da - 4u) < 4u ? (1u << ((da - 4u) << 3)) : 0u) + ea1;
                    Pb0[jj] = (jj ? Pb0[jj - 1] : 0u) + (db < 4u ? (1u << (db << 3)) : 0u) + eb0;
                    Pb1[jj] = (jj ? Pb1[jj - 1] : 0u) + ((db - 4u) < 4u ? (1u << ((db - 4u) << 3)) : 0u) + eb1;
                }
                const uint32_t ia0 = warp_incl_scan(Pa0[3], lane);
                const uint32_t ib0 = warp_incl_scan(Pb0[3], lane);
                const uint32_t ia1 = NB > 4 ? warp_incl_scan(Pa1[3], lane) : 0u;
                const uint32_t ib1 = NB > 4 ? warp_incl_scan(Pb1[3], lane) : 0u;
                const uint32_t xa0 = ia0 - Pa0[3], xa1 = ia1 - Pa1[3];
                const uint32_t xb0 = ib0 - Pb0[3], xb1 = ib1 - Pb1[3];
                const int4 la0 = *reinterpret_cast<const int4 *>(&RL[ra][0]);
                const int4 la1 = *reinterpret_cast<const int4 *>(&RL[ra][4]);
                const int4 lb0 = *reinterpret_cast<const int4 *>(&RL[rb][0]);
                const int4 lb1 = *reinterpret_cast<const int4 *>(&RL[rb][4]);
                const int rla[8] = {la0.x, la0.y, la0.z, la0.w, la1.x, la1.y, la1.z, la1.w};
                const int rlb[8] = {lb0.x, lb0.y, lb0.z, lb0.w, lb1.x, lb1.y, lb1.z, lb1.w};
                // row a
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const uint32_t y0 = xa0 + Pa0[jj], y1 = xa1 + Pa1[jj];
#pragma unroll
                    for (int b = 0; b < NB; ++b)
                        acc[b][jj] += rla[b] + (int)__byte_perm(b < 4 ? y0 : y1, 0, 0x4440 + (b & 3));
                }
                if constexpr (LAYOUT == LAYOUT_BIN_MAJOR) {
                    if (c < g.P) {
#pragma unroll
                        for (int b = 0; b < NB; ++b)
                            *reinterpret_cast<int4 *>(ps.out + ((bg0 + b) * g.H + R0 + ra) * g.P + c) =
                                make_int4(acc[b][0], acc[b][1], acc[b][2], acc[b][3]);
                    }
                } else if constexpr (LAYOUT == LAYOUT_SLAB) {
                    store_slab_staged<NB>(ps.out + ps.slab_off[gr.plane] + ((int64_t)(R0 + ra) * g.P + cc) * NB,
                                          (int)(g.P - cc < kChunk ? g.P - cc : kChunk), acc, stage, lane);
                } else {
                    const int rw = ps.rec_w[gr.plane];
                    store_record_staged<NB>(ps.out + ps.slab_off[gr.plane] + ((int64_t)(R0 + ra) * g.P + cc) * rw + gr.off,
                                            rw, (int)(g.P - cc < kChunk ? g.P - cc : kChunk), acc, stage, lane);
                }
                // row b
                if (hasb) {
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const uint32_t y0 = xb0 + Pb0[jj], y1 = xb1 + Pb1[jj];
#pragma unroll
                        for (int b = 0; b < NB; ++b)
                            acc[b][jj] += rlb[b] + (int)__byte_perm(b < 4 ? y0 : y1, 0, 0x4440 + (b & 3));
                    }
                    if constexpr (LAYOUT == LAYOUT_BIN_MAJOR) {
                        if (c < g.P) {
#pragma unroll
                            for (int b = 0; b < NB; ++b)
                                *reinterpret_cast<int4 *>(ps.out + ((bg0 + b) * g.H + R0 + rb) * g.P + c) =
                                    make_int4(acc[b][0], acc[b][1], acc[b][2], acc[b][3]);
                        }
                    } else if constexpr (LAYOUT == LAYOUT_SLAB) {
                        store_slab_staged<NB>(ps.out + ps.slab_off[gr.plane] + ((int64_t)(R0 + rb) * g.P + cc) * NB,
                                              (int)(g.P - cc < kChunk ? g.P - cc : kChunk), acc, stage, lane);
                    } else {
                        const int rw = ps.rec_w[gr.plane];
                        store_record_staged<NB>(ps.out + ps.slab_off[gr.plane] + ((int64_t)(R0 + rb) * g.P + cc) * rw + gr.off,
                                                rw, (int)(g.P - cc < kChunk ? g.P - cc : kChunk), acc, stage, lane);
                    }
                }
                // the last lane's inclusive sums are the chunk's row totals (the
                // next chunk's row carries; none when this chunk ends the strip)
                __syncwarp();
                if (lane == 31 && cc + kChunk < C1) {
                    int4 a, b4;
                    a.x = rla[0] + (int)__byte_perm(ia0, 0, 0x4440);
                    a.y = rla[1] + (int)__byte_perm(ia0, 0, 0x4441);
                    a.z = rla[2] + (int)__byte_perm(ia0, 0, 0x4442);
                    a.w = rla[3] + (int)__byte_perm(ia0, 0, 0x4443);
                    b4.x = rla[4] + (int)__byte_perm(ia1, 0, 0x4440);
                    b4.y = rla[5] + (int)__byte_perm(ia1, 0, 0x4441);
                    b4.z = rla[6] + (int)__byte_perm(ia1, 0, 0x4442);
                    b4.w = rla[7] + (int)__byte_perm(ia1, 0, 0x4443);
                    *reinterpret_cast<int4 *>(&RL[ra][0]) = a;
                    *reinterpret_cast<int4 *>(&RL[ra][4]) = b4;
                    if (hasb) {
                        a.x = rlb[0] + (int)__byte_perm(ib0, 0, 0x4440);
                        a.y = rlb[1] + (int)__byte_perm(ib0, 0, 0x4441);
                        a.z = rlb[2] + (int)__byte_perm(ib0, 0, 0x4442);
                        a.w = rlb[3] + (int)__byte_perm(ib0, 0, 0x4443);
                        b4.x = rlb[4] + (int)__byte_perm(ib1, 0, 0x4440);
                        b4.y = rlb[5] + (int)__byte_perm(ib1, 0, 0x4441);
                        b4.z = rlb[6] + (int)__byte_perm(ib1, 0, 0x4442);
                        b4.w = rlb[7] + (int)__byte_perm(ib1, 0, 0x4443);
                        *reinterpret_cast<int4 *>(&RL[rb][0]) = a;
                        *reinterpret_cast<int4 *>(&RL[rb][4]) = b4;
                    }
                }
            }
        }
        } else {
        // one row per step, pixel words 4 rows ahead in a register ring
#pragma unroll 1
        for (int ra = 0; ra < nr; ++ra) {
            const uint32_t pxa = pf[0], pya = pg[0];
            pf[0] = pf[1];
            pf[1] = pf[2];
            pf[2] = pf[3];
            pf[3] = (ra + 4 < nr) ? load4(pl0, pt0, R0 + ra + 4, c, C1, vec_ok) : 0u;
            if (two) {
                pg[0] = pg[1];
                pg[1] = pg[2];
                pg[2] = pg[3];
                pg[3] = (ra + 4 < nr) ? load4(pl1, pt1, R0 + ra + 4, c, C1, vec_ok1) : 0u;
            }
            uint32_t ea0[4] = {0u, 0u, 0u, 0u}, ea1[4] = {0u, 0u, 0u, 0u};
            if (two) {
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int ya = bin_of((pya >> (8 * jj)) & 0xff, bins1, mode1);
                    unsigned fa = (jj < nvalid && ya >= 0) ? (unsigned)(ya - blo1) : 0xFFFFFFFFu;
                    fa = fa < (unsigned)nbs1 ? fa + nb0 : 0xFFFFFFFFu;
                    ea0[jj] = fa < 4u ? (1u << (fa << 3)) : 0u;
                    ea1[jj] = (fa - 4u) < 4u ? (1u << ((fa - 4u) << 3)) : 0u;
                }
            }
            uint32_t Pa0[4], Pa1[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int qa = bin_of((pxa >> (8 * jj)) & 0xff, bins0, mode0);
                unsigned da = (jj < nvalid && qa >= 0) ? (unsigned)(qa - blo0) : 0xFFFFFFFFu;
                // a bin of the first channel beyond the group is dropped; the
                // second channel's bins follow at field nb
                if (SEG2 && da >= (unsigned)nb0) da = 0xFFFFFFFFu;
                Pa0[jj] = (jj ? Pa0[jj - 1] : 0u) + (da < 4u ? (1u << (da << 3)) : 0u) + ea0[jj];
                Pa1[jj] = (jj ? Pa1[jj - 1] : 0u) + ((da - 4u) < 4u ? (1u << ((da - 4u) << 3)) : 0u) + ea1[jj];
            }
            const uint32_t ia0 = warp_incl_scan(Pa0[3], lane);
            const uint32_t ia1 = NB > 4 ? warp_incl_scan(Pa1[3], lane) : 0u;
            const uint32_t xa0 = ia0 - Pa0[3], xa1 = ia1 - Pa1[3];
            const int4 la0 = *reinterpret_cast<const int4 *>(&RL[ra][0]);
            const int4 la1 = *reinterpret_cast<const int4 *>(&RL[ra][4]);
            const int rla[8] = {la0.x, la0.y, la0.z, la0.w, la1.x, la1.y, la1.z, la1.w};
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const uint32_t y0 = xa0 + Pa0[jj], y1 = xa1 + Pa1[jj];
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    acc[b][jj] += rla[b] + (int)__byte_perm(b < 4 ? y0 : y1, 0, 0x4440 + (b & 3));
            }
            if constexpr (LAYOUT == LAYOUT_BIN_MAJOR) {
                if (c < g.P) {
#pragma unroll
                    for (int b = 0; b < NB; ++b)
                        *reinterpret_cast<int4 *>(ps.out + ((bg0 + b) * g.H + R0 + ra) * g.P + c) =
                            make_int4(acc[b][0], acc[b][1], acc[b][2], acc[b][3]);
                }
            } else if constexpr (LAYOUT == LAYOUT_SLAB) {
                store_slab_staged<NB>(ps.out + ps.slab_off[gr.plane] + ((int64_t)(R0 + ra) * g.P + cc) * NB,
                                      (int)(g.P - cc < kChunk ? g.P - cc : kChunk), acc, stage, lane);
            } else {
                const int rw = ps.rec_w[gr.plane];
                store_record_staged<NB>(ps.out + ps.slab_off[gr.plane] + ((int64_t)(R0 + ra) * g.P + cc) * rw + gr.off,
                                        rw, (int)(g.P - cc < kChunk ? g.P - cc : kChunk), acc, stage, lane);
            }
            __syncwarp();
            if (lane == 31 && cc + kChunk < C1) {  // the next chunk's row carries
                int4 a, b4;
                a.x = rla[0] + (int)__byte_perm(ia0, 0, 0x4440);
                a.y = rla[1] + (int)__byte_perm(ia0, 0, 0x4441);
                a.z = rla[2] + (int)__byte_perm(ia0, 0, 0x4442);
                a.w = rla[3] + (int)__byte_perm(ia0, 0, 0x4443);
                b4.x = rla[4] + (int)__byte_perm(ia1, 0, 0x4440);
                b4.y = rla[5] + (int)__byte_perm(ia1, 0, 0x4441);
                b4.z = rla[6] + (int)__byte_perm(ia1, 0, 0x4442);
                b4.w = rla[7] + (int)__byte_perm(ia1, 0, 0x4443);
                *reinterpret_cast<int4 *>(&RL[ra][0]) = a;
                *reinterpret_cast<int4 *>(&RL[ra][4]) = b4;
            }
        }
        }
        __syncwarp();
    }
}

// LAYOUT_BIN_MAJOR / LAYOUT_SLAB: unit = group * tiles + tile with the
// groups sorted by size, so the CTAs dispatched first carry the largest
// groups and the tail of the grid is made of the cheapest units.
// LAYOUT_RECORD: unit = tile * groups + group, so the groups sharing a
// plane's records write them at about the same time.
// The count unit of tile (i, j), group gi, with the group's template
// arguments chosen at run time (non-record layouts).
template <int LAYOUT, bool PAIR>
__device__ __forceinline__ void tiles_count_at(const PlaneSet &ps, int i, int j, int gi, int lane,
                                               int32_t (*RL)[kGroupBins], int4 *stage, const int32_t *tr)
{
    switch (ps.grp[gi].nb) {
    case 1: tiles_count_unit<LAYOUT, 1, false, PAIR>(ps, i, j, gi, lane, RL, stage, tr); break;
    case 2: tiles_count_unit<LAYOUT, 2, false, PAIR>(ps, i, j, gi, lane, RL, stage, tr); break;
    case 3: tiles_count_unit<LAYOUT, 3, false, PAIR>(ps, i, j, gi, lane, RL, stage, tr); break;
    case 4: tiles_count_unit<LAYOUT, 4, false, PAIR>(ps, i, j, gi, lane, RL, stage, tr); break;
    case 5: tiles_count_unit<LAYOUT, 5, false, PAIR>(ps, i, j, gi, lane, RL, stage, tr); break;
    case 6: tiles_count_unit<LAYOUT, 6, false, PAIR>(ps, i, j, gi, lane, RL, stage, tr); break;
    case 7: tiles_count_unit<LAYOUT, 7, false, PAIR>(ps, i, j, gi, lane, RL, stage, tr); break;
    default: tiles_count_unit<LAYOUT, 8, false, PAIR>(ps, i, j, gi, lane, RL, stage, tr); break;
    }
}

template <int LAYOUT, bool PAIR>
__device__ __forceinline__ void tiles_count_dispatch(const PlaneSet &ps, int64_t unit, int lane,
                                                     int32_t (*RL)[kGroupBins], int4 *stage)
{
    const int64_t ntiles = (int64_t)ps.g.nb * ps.g.ns;
    if constexpr (LAYOUT == LAYOUT_RECORD) {
        const int tile = (int)(unit / ps.ngroups), gi = (int)(unit % ps.ngroups);
        const int i = tile / ps.g.ns, j = tile % ps.g.ns;
        // one code path per frame: when some group draws on two channels,
        // every group runs the two-channel path (an empty second segment
        // never hits), so an SM never interleaves two large loop bodies
        // (likewise one bin rule per frame)
        if (ps.seg2) {
            if (ps.uni)
                tiles_count_unit<LAYOUT_RECORD, kGroupBins, true, PAIR, true>(ps, i, j, gi, lane, RL, stage);
            else
                tiles_count_unit<LAYOUT_RECORD, kGroupBins, true, PAIR>(ps, i, j, gi, lane, RL, stage);
        } else {
            if (ps.uni)
                tiles_count_unit<LAYOUT_RECORD, kGroupBins, false, PAIR, true>(ps, i, j, gi, lane, RL, stage);
            else
                tiles_count_unit<LAYOUT_RECORD, kGroupBins, false, PAIR>(ps, i, j, gi, lane, RL, stage);
        }
    } else {
    const int gi = (int)(unit / ntiles), tile = (int)(unit % ntiles);
    const int i = tile / ps.g.ns, j = tile % ps.g.ns;
    switch (ps.grp[gi].nb) {
    case 1: tiles_count_unit<LAYOUT, 1, false, PAIR>(ps, i, j, gi, lane, RL, stage); break;
    case 2: tiles_count_unit<LAYOUT, 2, false, PAIR>(ps, i, j, gi, lane, RL, stage); break;
    case 3: tiles_count_unit<LAYOUT, 3, false, PAIR>(ps, i, j, gi, lane, RL, stage); break;
    case 4: tiles_count_unit<LAYOUT, 4, false, PAIR>(ps, i, j, gi, lane, RL, stage); break;
    case 5: tiles_count_unit<LAYOUT, 5, false, PAIR>(ps, i, j, gi, lane, RL, stage); break;
    case 6: tiles_count_unit<LAYOUT, 6, false, PAIR>(ps, i, j, gi, lane, RL, stage); break;
    case 7: tiles_count_unit<LAYOUT, 7, false, PAIR>(ps, i, j, gi, lane, RL, stage); break;
    default: tiles_count_unit<LAYOUT, 8, false, PAIR>(ps, i, j, gi, lane, RL, stage); break;
    }
    }
}

template <int LAYOUT>
__global__ void __launch_bounds__(128, LAYOUT == LAYOUT_SLAB ? 3 : 4) k_tiles_count(const __grid_constant__ PlaneSet ps)
{
    pdl_wait();
    __shared__ __align__(16) int32_t RLs[4][kMaxBandRows][kGroupBins];
    __shared__ int4 stages[4][LAYOUT == LAYOUT_BIN_MAJOR ? 1 : 32 * SlabStage<kGroupBins>::S];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t units = (int64_t)ps.g.nb * ps.g.ns * ps.ngroups;
    const int64_t unit = (int64_t)blockIdx.x * 4 + wid;
    if (unit < units) tiles_count_dispatch<LAYOUT, pair_rows<LAYOUT>()>(ps, unit, lane, RLs[wid], stages[wid]);
}

// Batched: warps over the concatenated units of all frames (any layout).
__global__ void __launch_bounds__(128, 3) k_tiles_count_b(const BatchDev bd)
{
    pdl_wait();
    __shared__ __align__(16) int32_t RLs[4][kMaxBandRows][kGroupBins];
    __shared__ int4 stages[4][32 * SlabStage<kGroupBins>::S];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t unit = (int64_t)blockIdx.x * 4 + wid;
    if (unit >= bd.pre_tiles[bd.n]) return;
    const int f = find_frame(bd.pre_tiles, bd.n, unit);
    const PlaneSet &ps = bd.sets[f];
    if (ps.layout == LAYOUT_SLAB)
        tiles_count_dispatch<LAYOUT_SLAB, true>(ps, unit - bd.pre_tiles[f], lane, RLs[wid], stages[wid]);
    else if (ps.layout == LAYOUT_RECORD)
        tiles_count_dispatch<LAYOUT_RECORD, true>(ps, unit - bd.pre_tiles[f], lane, RLs[wid], stages[wid]);
    else
        tiles_count_dispatch<LAYOUT_BIN_MAJOR, true>(ps, unit - bd.pre_tiles[f], lane, RLs[wid], stages[wid]);
}

// ------------------------------------------------------------- moment tiles

template <bool M32, bool UNI = false>
__device__ __forceinline__ void tiles_moments_unit(const PlaneSet &ps, int i, int j, int wb, int lane,
                                                   int32_t *RLn, long long *RLx, long long *RLxx,
                                                   long long *stage)
{
    const TileGrid &g = ps.g;
    const ChanDev &ch = ps.chan[ps.wch];
    const int Bw = ch.bins;
    const int64_t bglob = ch.bin_off + wb;
    const int R0 = i * g.R, nr = min(g.R, g.H - R0);
    const int C0 = j * g.Wc, C1 = min(C0 + g.Wc, g.W);
    const bool carries = ps.colsum != nullptr;

    __syncwarp();
    for (int rr = lane; rr < nr; rr += 32) {
        RLn[rr] = carries ? ps.rowsum[((int64_t)j * ps.B + bglob) * g.H + R0 + rr] : 0;
        RLx[rr] = carries ? ps.l_c[((int64_t)j * Bw + wb) * g.H + R0 + rr] : 0;
        RLxx[rr] = carries ? ps.l_cc[((int64_t)j * Bw + wb) * g.H + R0 + rr] : 0;
    }
    long long TR[4] = {0, 0, 0, 0};  // w = c, r, c^2, r^2: the tile corners to begin with
    if (carries) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            TR[k] = sum_bands_above<long long>(i, lane, [&](int ib) {
                return (long long)ps.corner_w[(((int64_t)ib * g.ns + j) * Bw + wb) * 4 + k];
            });
    }
    __syncwarp();
    // bin wb's quads: [H][P][4] (w = c, r, c^2, r^2 of one pixel together)
    int64_t *mo = ps.mom + (int64_t)wb * g.H * g.P * 4;
    uint32_t *mo32 = reinterpret_cast<uint32_t *>(ps.mom) + (int64_t)wb * g.H * g.P * 4;
    const bool vec_ok = ((ch.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(ch.plane) & 3) == 0);

    for (int cc = C0; cc < C1; cc += kChunk) {
        const int c = cc + lane * 4;
        const int nvalid = max(0, min(4, C1 - c));
        long long acc[4][4];  // [plane][pixel]
        // seeds: H_w(R0-1, c) = corner_w + prefix over the strip of the top carries
        {
            long long p[4][4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                long long g0 = 0, gr = 0, grr = 0;
                if (carries && jj < nvalid) {
                    const int64_t cidx = c + jj;
                    g0 = ps.colsum[((int64_t)i * ps.B + bglob) * g.W + cidx];
                    gr = ps.g_r[((int64_t)i * Bw + wb) * g.W + cidx];
                    grr = ps.g_rr[((int64_t)i * Bw + wb) * g.W + cidx];
                }
                const long long cj = c + jj;
                p[0][jj] = cj * g0;
                p[1][jj] = gr;
                p[2][jj] = cj * cj * g0;
                p[3][jj] = grr;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                p[k][1] += p[k][0];
                p[k][2] += p[k][1];
                p[k][3] += p[k][2];
                const long long incl = warp_incl_scan(p[k][3], lane);
                const long long base = TR[k] + (incl - p[k][3]);
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[k][jj] = base + p[k][jj];
                TR[k] += __shfl_sync(kFull, incl, 31);
            }
        }
        const long long Cb = cc;
        const int Cb32 = cc;
        const long long CbCb = Cb * Cb;
        uint32_t pf[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) pf[k] = (k < nr) ? load4(ch, R0 + k, c, C1, vec_ok) : 0u;
        for (int rr0 = 0; rr0 < nr; rr0 += 4) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int rr = rr0 + k;
                if (rr >= nr) break;  // warp-uniform
                const uint32_t px = pf[k];
                if (rr + 4 < nr) pf[k] = load4(ch, R0 + rr + 4, c, C1, vec_ok);
                int pn[4], pu[4], puu[4];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int q = bin_of((px >> (8 * jj)) & 0xff, ch.bins, UNI ? 0 : ch.mode);
                    const int e = (jj < nvalid && q == wb) ? 1 : 0;
                    const int u = lane * 4 + jj;
                    pn[jj] = (jj ? pn[jj - 1] : 0) + e;
                    pu[jj] = (jj ? pu[jj - 1] : 0) + e * u;
                    puu[jj] = (jj ? puu[jj - 1] : 0) + e * u * u;
                }
                // count <= 128 (8 bits) | sum of u <= 8128 (24 bits); sum of u^2 <= 690880
                const uint32_t w1 = (uint32_t)pn[3] | ((uint32_t)pu[3] << 8);
                const uint32_t w2 = (uint32_t)puu[3];
                const uint32_t i1 = warp_incl_scan(w1, lane), i2 = warp_incl_scan(w2, lane);
                const uint32_t x1 = i1 - w1, x2 = i2 - w2;
                const uint32_t t1 = __shfl_sync(kFull, i1, 31), t2 = __shfl_sync(kFull, i2, 31);
                const int ex_n = (int)(x1 & 0xFF), ex_u = (int)(x1 >> 8), ex_uu = (int)x2;
                const int rn = RLn[rr];
                const long long rx = RLx[rr], rxx = RLxx[rr];
                // 32-bit operands where the values fit (one widening multiply
                // each); the int64 sums are the same values as in full int64
                const int r = R0 + rr;
                const long long r2 = (long long)r * r;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int n = ex_n + pn[jj];          // row prefix of Q inside the chunk (<= 128)
                    const int su = ex_u + pu[jj];         // ... of u Q (<= 8128)
                    const int suu = ex_uu + puu[jj];      // ... of u^2 Q (<= 690880)
                    const unsigned N = (unsigned)rn + (unsigned)n;  // row prefix of Q from column 0 (<= W)
                    acc[0][jj] += rx + (long long)Cb32 * n + su;
                    acc[1][jj] += (long long)r * (long long)N;
                    acc[2][jj] += rxx + CbCb * n + 2 * ((long long)Cb32 * su) + suu;
                    acc[3][jj] += r2 * (long long)N;
                }
                if (c < g.P) {
                    if (M32) {
                        // the quads modulo 2^32 (16 bytes per pixel) through the
                        // warp's stage: unit u = px at position u ^ ((u >> 3) & 7)
                        // (conflict-free writes of 4 units per lane and reads of
                        // 32 consecutive units per store)
                        uint4 *s4 = reinterpret_cast<uint4 *>(stage);
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const int u = 4 * lane + jj;
                            s4[u ^ ((u >> 3) & 7)] = make_uint4((uint32_t)acc[0][jj], (uint32_t)acc[1][jj],
                                                                (uint32_t)acc[2][jj], (uint32_t)acc[3][jj]);
                        }
                    } else {
                        // through the warp's stage: the row's 128 quads are 256
                        // 16-byte units, unit u = 2 px + h holding planes 2h, 2h+1
                        // of pixel px, at position u ^ ((u >> 3) & 7) so that
                        // both the writes (8 units per lane) and the reads (32
                        // consecutive units per store) hit distinct bank groups
                        longlong2 *s2 = reinterpret_cast<longlong2 *>(stage);
#pragma unroll
                        for (int t = 0; t < 8; ++t) {
                            const int u = 8 * lane + t, jj = t >> 1, h = t & 1;
                            s2[u ^ ((u >> 3) & 7)] = make_longlong2(acc[2 * h][jj], acc[2 * h + 1][jj]);
                        }
                    }
                }
                if (M32) {
                    __syncwarp();
                    // each store writes 512 contiguous bytes of the row's 2 KB of quads
                    uint4 *dst = reinterpret_cast<uint4 *>(mo32 + ((int64_t)(R0 + rr) * g.P + cc) * 4);
                    const uint4 *s4 = reinterpret_cast<const uint4 *>(stage);
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        const int u = 32 * m + lane;
                        if (cc + u < g.P) dst[u] = s4[u ^ ((u >> 3) & 7)];
                    }
                } else {
                    __syncwarp();
                    // each store writes 512 contiguous bytes of the row's 4 KB of quads
                    longlong2 *dst = reinterpret_cast<longlong2 *>(mo + ((int64_t)(R0 + rr) * g.P + cc) * 4);
                    const longlong2 *s2 = reinterpret_cast<const longlong2 *>(stage);
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        const int u = 32 * m + lane;
                        if (cc + (u >> 1) < g.P) dst[u] = s2[u ^ ((u >> 3) & 7)];
                    }
                }
                __syncwarp();
                if (lane == 0 && cc + kChunk < C1) {  // the next chunk's row carries
                    const long long tn = t1 & 0xFF, tu = t1 >> 8, tuu = t2;
                    RLn[rr] = rn + (int)tn;
                    RLx[rr] = rx + Cb * tn + tu;
                    RLxx[rr] = rxx + Cb * Cb * tn + 2 * Cb * tu + tuu;
                }
            }
        }
        __syncwarp();
    }
}

// Count and moment tiles of one frame in a single launch: the first
// CTAs take the count units, the rest the moment units, so the two unit
// kinds share one tail instead of two.  Measured on the FMV frame: count
// units first 332 us, moment units first 349 us, the two kinds alternating
// 369 us, and a persistent launch that kept each SM on one kind (work
// counters, SMs split by %smid) 357 us.  The shared memory is the union of
// the two kinds' buffers.
struct CountSmem {
    int32_t RL[4][kMaxBandRows][kGroupBins];
    int4 stage[4][32 * SlabStage<kGroupBins>::S];
};
struct MomentSmem {
    int32_t RLn[4][kMaxBandRows];
    long long RLx[4][kMaxBandRows], RLxx[4][kMaxBandRows];
    long long stage[4][4 * kChunk];
};
constexpr size_t kTilesSmem = sizeof(CountSmem) > sizeof(MomentSmem) ? sizeof(CountSmem) : sizeof(MomentSmem);

// The count units step one row at a time here, so that 4 CTAs fit an SM
// and the moment units keep the occupancy they have on their own.
template <int LAYOUT>
__global__ void __launch_bounds__(128, 4) k_tiles(const __grid_constant__ PlaneSet ps, unsigned mom_blocks)
{
    pdl_wait();
    __shared__ __align__(16) unsigned char smem[kTilesSmem];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const TileGrid &g = ps.g;
    const unsigned cnt_blocks = gridDim.x - mom_blocks;
    if (blockIdx.x >= cnt_blocks) {
        MomentSmem &m = *reinterpret_cast<MomentSmem *>(smem);
        const int Bw = ps.chan[ps.wch].bins;
        const int64_t unit = (int64_t)(blockIdx.x - cnt_blocks) * 4 + wid;
        if (unit >= (int64_t)g.nb * g.ns * Bw) return;
        const int tile = (int)(unit / Bw), wb = (int)(unit % Bw);
        if (ps.mom32)
            tiles_moments_unit<true>(ps, tile / g.ns, tile % g.ns, wb, lane, m.RLn[wid], m.RLx[wid], m.RLxx[wid],
                                     m.stage[wid]);
        else if (ps.uni)
            tiles_moments_unit<false, true>(ps, tile / g.ns, tile % g.ns, wb, lane, m.RLn[wid], m.RLx[wid],
                                            m.RLxx[wid], m.stage[wid]);
        else
            tiles_moments_unit<false>(ps, tile / g.ns, tile % g.ns, wb, lane, m.RLn[wid], m.RLx[wid], m.RLxx[wid],
                                      m.stage[wid]);
    } else {
        CountSmem &cs = *reinterpret_cast<CountSmem *>(smem);
        const int64_t units = (int64_t)g.nb * g.ns * ps.ngroups;
        const int64_t unit = (int64_t)blockIdx.x * 4 + wid;
        if (unit < units) tiles_count_dispatch<LAYOUT, false>(ps, unit, lane, cs.RL[wid], cs.stage[wid]);
    }
}

// Batched: the count units of all frames, then the moment units of all
// frames, in one launch (count units as in k_tiles_count_b).
__global__ void __launch_bounds__(128, 4) k_tiles_b(const BatchDev bd, unsigned mom_blocks)
{
    pdl_wait();
    __shared__ __align__(16) unsigned char smem[kTilesSmem];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned cnt_blocks = gridDim.x - mom_blocks;
    if (blockIdx.x >= cnt_blocks) {
        MomentSmem &m = *reinterpret_cast<MomentSmem *>(smem);
        const int64_t unit = (int64_t)(blockIdx.x - cnt_blocks) * 4 + wid;
        if (unit >= bd.pre_mom[bd.n]) return;
        const int f = find_frame(bd.pre_mom, bd.n, unit);
        const PlaneSet &ps = bd.sets[f];
        const int Bw = ps.chan[ps.wch].bins;
        const int64_t local = unit - bd.pre_mom[f];
        const int tile = (int)(local / Bw), wb = (int)(local % Bw);
        if (ps.mom32)
            tiles_moments_unit<true>(ps, tile / ps.g.ns, tile % ps.g.ns, wb, lane, m.RLn[wid], m.RLx[wid],
                                     m.RLxx[wid], m.stage[wid]);
        else if (ps.uni)
            tiles_moments_unit<false, true>(ps, tile / ps.g.ns, tile % ps.g.ns, wb, lane, m.RLn[wid], m.RLx[wid],
                                            m.RLxx[wid], m.stage[wid]);
        else
            tiles_moments_unit<false>(ps, tile / ps.g.ns, tile % ps.g.ns, wb, lane, m.RLn[wid], m.RLx[wid],
                                      m.RLxx[wid], m.stage[wid]);
    } else {
        CountSmem &cs = *reinterpret_cast<CountSmem *>(smem);
        const int64_t unit = (int64_t)blockIdx.x * 4 + wid;
        if (unit >= bd.pre_tiles[bd.n]) return;
        const int f = find_frame(bd.pre_tiles, bd.n, unit);
        const PlaneSet &ps = bd.sets[f];
        const int64_t local = unit - bd.pre_tiles[f];
        if (ps.layout == LAYOUT_SLAB)
            tiles_count_dispatch<LAYOUT_SLAB, false>(ps, local, lane, cs.RL[wid], cs.stage[wid]);
        else if (ps.layout == LAYOUT_RECORD)
            tiles_count_dispatch<LAYOUT_RECORD, false>(ps, local, lane, cs.RL[wid], cs.stage[wid]);
        else
            tiles_count_dispatch<LAYOUT_BIN_MAJOR, false>(ps, local, lane, cs.RL[wid], cs.stage[wid]);
    }
}

// ------------------------------------------------------------- persistent batched build
//
// One launch builds every frame of a batch: 256-thread CTAs, as many as fit
// the GPU at once, take work items by ticket (an atomic counter) until the
// batch's items run out.  The items are segments of one kind of work of one
// frame -- weighted-channel tile sums (one window per item), count tile sums
// (two windows per item, one per 128-thread half), carry-scan chunks (256
// scan items), count tiles and moment tiles (8 warp units per item) -- in an
// order the host chooses.  A frame's carry scan may start once all its tile
// sums are done, its tiles once its carry scan is done: each finished item
// adds one to its frame's counter for its phase (after a device-wide fence),
// and an item whose phase depends on another reads that counter with acquire
// semantics until it reaches the frame's total.  Every item it waits for has
// a smaller ticket, so it was taken earlier by a CTA that is running it; the
// wait is bounded all the same: a wait that gives up sets bit 2 of the error
// word (ih_sync reports IH_ETIMEOUT) and the item goes on without the data.
// Loads of data written inside the launch (the carries) are plain loads after
// that acquire; pixels and feature planes are written before the launch.
constexpr int kPThreads = 256;
constexpr long kPSpinLimit = 1L << 24;

enum PersistKind { PK_SUMS_W = 0, PK_SUMS_C = 1, PK_SCAN = 2, PK_TILES_C = 3, PK_TILES_M = 4 };

__device__ __forceinline__ int persist_phase(int kind) { return kind <= PK_SUMS_C ? 0 : (kind == PK_SCAN ? 1 : 2); }

__device__ __forceinline__ int ld_acquire_gpu(const int32_t *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// LAYOUT: the count layout of every frame of the batch, or -1 for a batch of
// several layouts (each count-tile item then dispatches on its frame's).
// Waits until *counter >= need, reading it with acquire semantics, for at
// most `limit` polls (a few dozen ns apart); gives up early once bit 2 of
// the error word is set (another wait gave up: the run is void).  On giving
// up it sets bit 2 and returns false.  One thread of a CTA calls it.
__device__ __forceinline__ bool bounded_wait_geq(const int32_t *counter, int need, long limit, int *err)
{
    long spins = 0;
    while (ld_acquire_gpu(counter) < need) {
        if (++spins > limit || (*(volatile int *)err & 2)) {
            atomicOr(err, 2);
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

// Self-test of the bounded wait: one thread waits for a counter that nothing
// raises and gives up after `limit` polls.
__global__ void k_wait_selftest(const int32_t *never, long limit, int *err)
{
    pdl_wait();
    if (threadIdx.x == 0 && blockIdx.x == 0) bounded_wait_geq(never, 1, limit, err);
}

template <int LAYOUT>
__global__ void __launch_bounds__(kPThreads, 2) k_build_persistent(const PersistDev pd)
{
    pdl_wait();
    extern __shared__ __align__(16) unsigned char dsm[];
    __shared__ unsigned int s_t;
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (;;) {
        if (tid == 0) s_t = atomicAdd(pd.ticket, 1u);
        __syncthreads();
        const int64_t t = s_t;
        if (t >= pd.total) return;
        const int sg = find_frame(pd.seg_pre, pd.nsegs, t);
        const PersistSeg seg = pd.segs[sg];
        const int64_t idx = seg.first + (t - pd.seg_pre[sg]);
        const PlaneSet &ps = pd.sets[seg.frame];
        const int phase = persist_phase(seg.kind);
        int32_t *done = pd.done + 3 * (int64_t)seg.frame;
        if (tid == 0)
            s_abort = phase > 0 && !bounded_wait_geq(done + phase - 1, pd.need[3 * (int64_t)seg.frame + phase - 1],
                                                     kPSpinLimit, pd.err);
        __syncthreads();  // also: every thread has read s_t before it is taken again
        if (!s_abort) {
            const TileGrid &g = ps.g;
            const int64_t per = (int64_t)g.ns * g.nb;
            if (seg.kind == PK_SUMS_W) {
                const int z = (int)(idx / per), rem = (int)(idx % per);
                tile_sums_body<true>(ps, rem % g.ns, rem / g.ns, ps.nwin_count + z);
            } else if (seg.kind == PK_SUMS_C) {
                const int half = tid >> 7;
                const int64_t u = 2 * idx + half;
                if (u < per * ps.nwin_count) {
                    const int z = (int)(u / per), rem = (int)(u % per);
                    CountSumsSmem &sm = reinterpret_cast<CountSumsSmem *>(dsm)[half];
                    tile_sums_count_group(ps, rem % g.ns, rem / g.ns, z, sm, tid & 127, 1 + half);
                }
            } else if (seg.kind == PK_SCAN) {
                const int64_t u = idx * kPThreads + tid;
                if (u < carry_scan_items(ps)) carry_scan_item(ps, u);
            } else if (seg.kind == PK_TILES_C) {
                CountSmem *cs = reinterpret_cast<CountSmem *>(dsm);
                const int64_t u = idx * 8 + wid;
                const int h = wid >> 2, w4 = wid & 3;
                if (u < per * ps.ngroups) {
                    if constexpr (LAYOUT >= 0) {
                        tiles_count_dispatch<LAYOUT, false>(ps, u, lane, cs[h].RL[w4], cs[h].stage[w4]);
                    } else {
                        if (ps.layout == LAYOUT_SLAB)
                            tiles_count_dispatch<LAYOUT_SLAB, false>(ps, u, lane, cs[h].RL[w4], cs[h].stage[w4]);
                        else if (ps.layout == LAYOUT_RECORD)
                            tiles_count_dispatch<LAYOUT_RECORD, false>(ps, u, lane, cs[h].RL[w4], cs[h].stage[w4]);
                        else
                            tiles_count_dispatch<LAYOUT_BIN_MAJOR, false>(ps, u, lane, cs[h].RL[w4], cs[h].stage[w4]);
                    }
                }
            } else {
                MomentSmem *m = reinterpret_cast<MomentSmem *>(dsm);
                const int Bw = ps.chan[ps.wch].bins;
                const int64_t u = idx * 8 + wid;
                const int h = wid >> 2, w4 = wid & 3;
                if (u < per * Bw) {
                    const int tile = (int)(u / Bw), wb = (int)(u % Bw);
                    if (ps.mom32)
                        tiles_moments_unit<true>(ps, tile / g.ns, tile % g.ns, wb, lane, m[h].RLn[w4], m[h].RLx[w4],
                                                 m[h].RLxx[w4], m[h].stage[w4]);
                    else if (ps.uni)
                        tiles_moments_unit<false, true>(ps, tile / g.ns, tile % g.ns, wb, lane, m[h].RLn[w4],
                                                        m[h].RLx[w4], m[h].RLxx[w4], m[h].stage[w4]);
                    else
                        tiles_moments_unit<false>(ps, tile / g.ns, tile % g.ns, wb, lane, m[h].RLn[w4], m[h].RLx[w4],
                                                  m[h].RLxx[w4], m[h].stage[w4]);
                }
            }
        }
        // the CTA's writes, ordered before thread 0 by the barrier, are
        // released device-wide by its fence before the counter moves
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(done + phase, 1);
        }
    }
}

// ------------------------------------------------------------- one-pass build of small frames
//
// A frame without moment planes, in the bin-major or slab layout, cut into
// bands of at most 32 rows and strips of 128 columns (at most 16 strips), is
// built in ONE launch: CTA (band i, bin group g), one warp per strip.
//  1. Each warp reads its strip of the band once: the column counts of the
//     group's bins (8-bit fields) and, row by row, the strip's row counts
//     (packed-field warp reductions, into shared memory).  The CTA publishes
//     its column counts (the band's aggregate) and raises its flag to 1.
//  2. Decoupled look-back over the bands above (Merrill & Garland, "Single-
//     pass parallel prefix scan with decoupled look-back", NVIDIA 2016), 32
//     bands at a time: each lane of a warp polls one band's flag; the
//     nearest band whose inclusive column prefix is published (flag 2) ends
//     the walk, and the aggregates (flag 1) of the bands before it are summed
//     with independent loads.  The sum is G: the column counts over all rows
//     above the band.  The CTA publishes G plus its own counts and raises its
//     flag to 2.  Flags are read with acquire semantics and the published sums
//     with L2-only loads; every poll loop is bounded (a wait that gives up
//     sets bit 2 of the error word: ih_sync reports IH_ETIMEOUT).
//  3. In shared memory: each strip's row carries L (prefix over the strips to
//     its left of the row counts, stored where the tiles body reads them)
//     and its corner H(R0-1, C0-1) (prefix over the strips to its left of
//     the totals of G).
//  4. Each warp runs the count-tile body on its tile with those carries.
// CTAs take (band, group) by ticket in band order, so every band a CTA
// looks back at was taken by a CTA that is running or done.
constexpr int kOneMaxStrips = 16;
constexpr int kOneMaxRows = 32;
constexpr long kOneSpinLimit = 1L << 22;

struct OneSmem {
    int32_t rowtot[kOneMaxStrips][kOneMaxRows][kGroupBins];  // row counts per strip
    int32_t gtot[kOneMaxStrips][kGroupBins];                 // totals of G per strip
    int32_t tr[kOneMaxStrips][kGroupBins];                   // corners
    int32_t RL[kOneMaxStrips][kOneMaxRows][kGroupBins];      // the tiles body's row-carry buffers
};

__device__ __forceinline__ int ld_acquire_flag(const int32_t *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_flag(int32_t *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

template <int LAYOUT>
__global__ void __launch_bounds__(kOneMaxStrips * 32) k_build_onepass(const __grid_constant__ PlaneSet ps)
{
    extern __shared__ __align__(16) unsigned char dsm[];
    OneSmem &sm = *reinterpret_cast<OneSmem *>(dsm);
    int4 *stages = reinterpret_cast<int4 *>(dsm + ((sizeof(OneSmem) + 15) & ~size_t(15)));
    __shared__ unsigned int s_t;
    pdl_wait();
    const TileGrid &g = ps.g;
    const int lane = threadIdx.x & 31, j = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_t = atomicAdd(reinterpret_cast<unsigned int *>(ps.flags) + g.nb * ps.ngroups, 1u);
    __syncthreads();
    const int i = (int)(s_t / ps.ngroups), gi = (int)(s_t % ps.ngroups);
    const GroupDev gr = ps.grp[gi];
    const ChanDev &ch = ps.chan[gr.chan];
    const int nbg = gr.nb;
    const int64_t bg0 = ch.bin_off + gr.b_lo;
    const int R0 = i * g.R, nr = min(g.R, g.H - R0);
    const int C0 = j * kChunk, c = C0 + 4 * lane;
    const int nvalid = max(0, min(4, g.W - c));
    const bool vec_ok = ((ch.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(ch.plane) & 3) == 0);
    int32_t *flag = ps.flags + (int64_t)i * ps.ngroups + gi;

    // 1. column counts (bins 0-3 and 4-7 of each column in 8-bit fields) and row counts
    uint32_t colw[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    for (int r8 = 0; r8 < nr; r8 += 8) {
      // the loads of 8 rows in flight at once
      uint32_t pxs[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) pxs[k] = r8 + k < nr ? load4(ch.plane, ch.pitch, R0 + r8 + k, c, g.W, vec_ok) : 0u;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int rr = r8 + k;
        if (rr >= nr) break;
        const uint32_t px = pxs[k];
        uint32_t rw0 = 0, rw1 = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int b = bin_of((px >> (8 * q)) & 0xff, ch.bins, ch.mode) - gr.b_lo;
            if (q < nvalid && b >= 0 && b < nbg) {
                const uint32_t inc = 1u << (8 * (b & 3));
                if (b < 4) {
                    colw[q][0] += inc;
                    rw0 += inc;
                } else {
                    colw[q][1] += inc;
                    rw1 += inc;
                }
            }
        }
        rw0 = __reduce_add_sync(kFull, rw0);
        rw1 = __reduce_add_sync(kFull, rw1);
        if (lane < kGroupBins) sm.rowtot[j][rr][lane] = (int)(((lane < 4 ? rw0 : rw1) >> (8 * (lane & 3))) & 0xff);
      }
    }
    int cnt[kGroupBins][4];
#pragma unroll
    for (int b = 0; b < kGroupBins; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) cnt[b][q] = (int)((colw[q][b >> 2] >> (8 * (b & 3))) & 0xff);
    // published sums: [band][bin][P] int32, 16-byte rows of 4 columns per lane
    auto pub = [&](int32_t *base, int band, int b) {
        return reinterpret_cast<int4 *>(base + ((int64_t)band * ps.B + bg0 + b) * g.P + c);
    };
    const bool inrow = c < g.P;
    if (i + 1 < g.nb && inrow) {  // the last band's aggregate is never read
#pragma unroll
        for (int b = 0; b < kGroupBins; ++b)
            if (b < nbg) *pub(ps.agg, i, b) = make_int4(cnt[b][0], cnt[b][1], cnt[b][2], cnt[b][3]);
    }
    __syncthreads();
    if (threadIdx.x == 0 && i + 1 < g.nb) {
        __threadfence();
        st_release_flag(flag, 1);
    }
    // 2. warp-parallel look-back, 32 bands at a time: lane l polls band
    // k_hi - l; the nearest band with its inclusive prefix published (flag 2)
    // ends the walk, and the aggregates of the bands before it are summed
    int G[kGroupBins][4];
#pragma unroll
    for (int b = 0; b < kGroupBins; ++b)
#pragma unroll
        for (int q = 0; q < 4; ++q) G[b][q] = 0;
    bool ok = true;
    for (int k_hi = i - 1; k_hi >= 0;) {
        const int kb = k_hi - lane;
        int f = 2;  // bands before the first one count as a published zero prefix
        if (kb >= 0) {
            const int32_t *fk = ps.flags + (int64_t)kb * ps.ngroups + gi;
            long spins = 0;
            while ((f = ld_acquire_flag(fk)) == 0) {
                if (++spins > kOneSpinLimit || (*(volatile int *)ps.err & 2)) {
                    atomicOr(ps.err, 2);
                    break;
                }
                __nanosleep(32);
            }
        }
        const unsigned lost = __ballot_sync(kFull, f == 0);
        if (lost) {
            ok = false;
            break;
        }
        const unsigned incl = __ballot_sync(kFull, f == 2);
        const int stop = incl ? __ffs(incl) - 1 : 32;  // bands k_hi .. k_hi - stop + 1: aggregates
        if (inrow) {
            for (int l = 0; l < stop; ++l) {
#pragma unroll
                for (int b = 0; b < kGroupBins; ++b)
                    if (b < nbg) {
                        const int4 v = __ldcg(pub(ps.agg, k_hi - l, b));
                        G[b][0] += v.x;
                        G[b][1] += v.y;
                        G[b][2] += v.z;
                        G[b][3] += v.w;
                    }
            }
            if (stop < 32 && k_hi - stop >= 0) {
#pragma unroll
                for (int b = 0; b < kGroupBins; ++b)
                    if (b < nbg) {
                        const int4 v = __ldcg(pub(ps.incl, k_hi - stop, b));
                        G[b][0] += v.x;
                        G[b][1] += v.y;
                        G[b][2] += v.z;
                        G[b][3] += v.w;
                    }
            }
        }
        if (stop < 32) break;
        k_hi -= 32;
    }
    const int64_t rowstride = (int64_t)g.W;
    auto at = [&](int32_t *base, int band, int b, int q) { return base + ((int64_t)band * ps.B + bg0 + b) * rowstride + c + q; };
    // publish the inclusive prefix; G is the tiles' column carry
#pragma unroll
    for (int b = 0; b < kGroupBins; ++b) {
        if (b < nbg && i + 1 < g.nb && inrow)
            *pub(ps.incl, i, b) = make_int4(G[b][0] + cnt[b][0], G[b][1] + cnt[b][1], G[b][2] + cnt[b][2],
                                            G[b][3] + cnt[b][3]);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (b < nbg && q < nvalid) *at(ps.colsum, i, b, q) = G[b][q];
    }
    // strip totals of G for the corners
#pragma unroll
    for (int b = 0; b < kGroupBins; ++b) {
        const int t = __reduce_add_sync(kFull, G[b][0] + G[b][1] + G[b][2] + G[b][3]);
        if (lane == b) sm.gtot[j][b] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0 && i + 1 < g.nb) {
        __threadfence();
        st_release_flag(flag, 2);
    }
    // 3. corners and row carries of this warp's tile
    if (lane < kGroupBins) {
        int t = 0;
        for (int jj = 0; jj < j; ++jj) t += sm.gtot[jj][lane];
        sm.tr[j][lane] = t;
    }
    for (int k = lane; k < nr * kGroupBins; k += 32) {
        const int rr = k / kGroupBins, b = k % kGroupBins;
        int t = 0;
        for (int jj = 0; jj < j; ++jj) t += sm.rowtot[jj][rr][b];
        if (b < nbg) ps.rowsum[((int64_t)j * ps.B + bg0 + b) * g.H + R0 + rr] = t;
    }
    __syncwarp();
    // 4. the tile (the body reads colsum[i], rowsum[j] of this band: written above by this CTA)
    __syncthreads();
    if (ok && C0 < g.W)
        tiles_count_at<LAYOUT, true>(ps, i, j, gi, lane, sm.RL[j], stages + j * (32 * SlabStage<kGroupBins>::S),
                                     sm.tr[j]);
}

size_t onepass_smem_bytes() { return ((sizeof(OneSmem) + 15) & ~size_t(15)) + sizeof(int4) * kOneMaxStrips * 32 * SlabStage<kGroupBins>::S; }

template <typename F>
void set_max_smem(F *f, size_t bytes)
{
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

size_t r256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

bool pdl_enabled()
{
    static const bool on = [] {
        const char *e = getenv("IH_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

bool onepass_ok(const PlaneSet &ps)
{
    static const bool on = [] {
        const char *e = getenv("IH_ONEPASS");
        return e && e[0] == '1';
    }();
    const TileGrid &g = ps.g;
    return on && ps.err && !ps.mom && ps.wch < 0 && ps.layout != LAYOUT_RECORD && g.Wc == kChunk && g.R <= kOneMaxRows &&
           g.ns <= kOneMaxStrips && (int64_t)g.nb * g.ns > 1 && (int64_t)ps.B * g.H * g.W <= ((int64_t)1 << 26);
}

size_t carry_bytes(const PlaneSet &ps)
{
    const TileGrid &g = ps.g;
    if (ps.small) return small_bytes(ps);
    if ((int64_t)g.nb * g.ns <= 1) return 0;
    const size_t B = ps.B, W = g.W, H = g.H, nb = g.nb, ns = g.ns;
    size_t n = r256(4 * B * W * nb) + r256(4 * B * H * ns) + 2 * r256(4 * nb * ns * B);
    if (onepass_ok(ps)) n += 2 * r256(4 * B * (size_t)g.P * nb) + r256(4 * (nb * (size_t)ps.ngroups + 1));
    if (ps.wch >= 0) {
        const size_t Bw = ps.chan[ps.wch].bins;
        n += 2 * r256(4 * Bw * W * nb) + 2 * r256(4 * Bw * H * ns) + r256(32 * nb * ns * Bw);
        n += 2 * r256(8 * Bw * W * nb) + 2 * r256(8 * Bw * H * ns) + r256(32 * nb * ns * Bw);
    }
    return n;
}

void carve_carries(PlaneSet &ps, void *base)
{
    const TileGrid &g = ps.g;
    ps.colsum = ps.rowsum = ps.tilesum = ps.corner = nullptr;
    ps.agg = ps.incl = ps.flags = nullptr;
    ps.col_su = ps.col_suu = ps.row_sv = ps.row_svv = nullptr;
    ps.tile_w = ps.g_r = ps.g_rr = ps.l_c = ps.l_cc = ps.corner_w = nullptr;
    ps.sm_col = ps.sm_row = nullptr;
    ps.sm_tot = nullptr;
    ps.sm_bar = nullptr;
    if (base && ps.small) {
        carve_small(ps, base);
        return;
    }
    if (!base || (int64_t)g.nb * g.ns <= 1) return;
    char *s = static_cast<char *>(base);
    const size_t B = ps.B, W = g.W, H = g.H, nb = g.nb, ns = g.ns;
    auto take = [&s](size_t bytes) {
        char *p = s;
        s += r256(bytes);
        return p;
    };
    ps.colsum = reinterpret_cast<int32_t *>(take(4 * B * W * nb));
    ps.rowsum = reinterpret_cast<int32_t *>(take(4 * B * H * ns));
    ps.tilesum = reinterpret_cast<int32_t *>(take(4 * nb * ns * B));
    ps.corner = reinterpret_cast<int32_t *>(take(4 * nb * ns * B));
    if (onepass_ok(ps)) {
        ps.agg = reinterpret_cast<int32_t *>(take(4 * B * (size_t)g.P * nb));
        ps.incl = reinterpret_cast<int32_t *>(take(4 * B * (size_t)g.P * nb));
        ps.flags = reinterpret_cast<int32_t *>(take(4 * (nb * (size_t)ps.ngroups + 1)));
    }
    if (ps.wch >= 0) {
        const size_t Bw = ps.chan[ps.wch].bins;
        ps.col_su = reinterpret_cast<int32_t *>(take(4 * Bw * W * nb));
        ps.col_suu = reinterpret_cast<int32_t *>(take(4 * Bw * W * nb));
        ps.row_sv = reinterpret_cast<int32_t *>(take(4 * Bw * H * ns));
        ps.row_svv = reinterpret_cast<int32_t *>(take(4 * Bw * H * ns));
        ps.tile_w = reinterpret_cast<int64_t *>(take(32 * nb * ns * Bw));
        ps.g_r = reinterpret_cast<int64_t *>(take(8 * Bw * W * nb));
        ps.g_rr = reinterpret_cast<int64_t *>(take(8 * Bw * W * nb));
        ps.l_c = reinterpret_cast<int64_t *>(take(8 * Bw * H * ns));
        ps.l_cc = reinterpret_cast<int64_t *>(take(8 * Bw * H * ns));
        ps.corner_w = reinterpret_cast<int64_t *>(take(32 * nb * ns * Bw));
    }
}

size_t persistent_smem_bytes(int max_R);

void prepare_kernels()
{
    prepare_features();
    // Shared-memory limits are function attributes of the current device:
    // set them once per device, under a lock (callers may be on any thread).
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    set_max_smem(k_tile_sums_all, std::max(sums_smem_bytes(kMaxBandRows, true), 2 * sizeof(CountSumsSmem)));
    set_max_smem(k_tile_sums_all_b, std::max(sums_smem_bytes(kMaxBandRows, true), 2 * sizeof(CountSumsSmem)));
    set_max_smem(k_build_onepass<LAYOUT_SLAB>, onepass_smem_bytes());
    set_max_smem(k_build_onepass<LAYOUT_BIN_MAJOR>, onepass_smem_bytes());
    set_max_smem(k_build_persistent<-1>, persistent_smem_bytes(kMaxBandRows));
    set_max_smem(k_build_persistent<LAYOUT_SLAB>, persistent_smem_bytes(kMaxBandRows));
    set_max_smem(k_build_persistent<LAYOUT_RECORD>, persistent_smem_bytes(kMaxBandRows));
    set_max_smem(k_build_persistent<LAYOUT_BIN_MAJOR>, persistent_smem_bytes(kMaxBandRows));
    done[dev] = true;
}

int launch_build_batch(const BatchDev &bd, const int64_t *totals, cudaStream_t st, const Prof *prof)
{
    prepare_kernels();
    int n = 0;
    if (totals[0] || totals[1]) {
        // both window kinds in one launch, the weighted CTAs first
        const size_t smem = std::max(totals[1] ? sums_smem_bytes(bd.max_R, true) : 0, 2 * sizeof(CountSumsSmem));
        prof_mark(prof, KID_SUMS_ALL, 0, st);
        launch_pdl(k_tile_sums_all_b, (unsigned)(totals[1] + (totals[0] + 1) / 2), kSumThreads, smem, st, bd,
                   (unsigned)totals[1]);
        prof_mark(prof, KID_SUMS_ALL, 1, st);
        ++n;
    }
    if (totals[2]) {
        const int64_t blocks = (totals[2] + 255) / 256;
        prof_mark(prof, KID_SCAN, 0, st);
        launch_pdl(k_carry_scan_b, (unsigned)(blocks < 16384 ? blocks : 16384), 256, 0, st, bd);
        prof_mark(prof, KID_SCAN, 1, st);
        ++n;
    }
    if (totals[3] && totals[4]) {
        // count and moment tiles of all frames in one launch
        const unsigned mblocks = (unsigned)((totals[4] + 3) / 4);
        prof_mark(prof, KID_TILES_BOTH, 0, st);
        launch_pdl(k_tiles_b, mblocks + (unsigned)((totals[3] + 3) / 4), 128, 0, st, bd, mblocks);
        prof_mark(prof, KID_TILES_BOTH, 1, st);
        ++n;
    } else if (totals[3]) {
        prof_mark(prof, KID_TILES_COUNT, 0, st);
        launch_pdl(k_tiles_count_b, (unsigned)((totals[3] + 3) / 4), 128, 0, st, bd);
        prof_mark(prof, KID_TILES_COUNT, 1, st);
        ++n;
    }
    return cudaPeekAtLastError() == cudaSuccess ? n : -1;
}

size_t persistent_smem_bytes(int max_R)
{
    size_t b = std::max(sums_smem_bytes(max_R, true), 2 * sizeof(CountSumsSmem));
    b = std::max(b, std::max(2 * sizeof(CountSmem), 2 * sizeof(MomentSmem)));
    return b;
}

void persistent_counts(const PlaneSet &ps, int64_t *c)
{
    const int64_t tiles = (int64_t)ps.g.nb * ps.g.ns;
    const bool carries = ps.colsum != nullptr;
    c[PK_SUMS_W] = carries ? tiles * (ps.nwin - ps.nwin_count) : 0;
    c[PK_SUMS_C] = carries ? (tiles * ps.nwin_count + 1) / 2 : 0;
    c[PK_SCAN] = carries ? ((int64_t)ps.B * ps.g.W + (int64_t)ps.B * ps.g.H + (int64_t)ps.g.nb * ps.B + kPThreads - 1) /
                               kPThreads
                         : 0;
    c[PK_TILES_C] = (tiles * ps.ngroups + 7) / 8;
    c[PK_TILES_M] = ps.mom ? (tiles * ps.chan[ps.wch].bins + 7) / 8 : 0;
}

int persistent_ctas()
{
    prepare_kernels();
    static std::mutex mu;
    static int ctas[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 1;
    std::lock_guard<std::mutex> lk(mu);
    if (!ctas[dev]) {
        int per_sm = 0, nsm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_build_persistent<-1>, kPThreads,
                                                      persistent_smem_bytes(kMaxBandRows));
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        ctas[dev] = std::max(1, per_sm) * std::max(1, nsm);
    }
    return ctas[dev];
}

int launch_wait_selftest(const int32_t *never, long limit, int *err, cudaStream_t st)
{
    launch_pdl(k_wait_selftest, 1, 32, 0, st, never, limit, err);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_build_persistent(const PersistDev &pd, int layout, int max_R, cudaStream_t st, const Prof *prof)
{
    prepare_kernels();
    const int64_t ctas = std::min<int64_t>(pd.total, persistent_ctas());
    if (ctas <= 0) return 0;
    const size_t smem = persistent_smem_bytes(max_R);
    prof_mark(prof, KID_PERSISTENT, 0, st);
    if (layout == LAYOUT_SLAB)
        launch_pdl(k_build_persistent<LAYOUT_SLAB>, (unsigned)ctas, kPThreads, smem, st, pd);
    else if (layout == LAYOUT_RECORD)
        launch_pdl(k_build_persistent<LAYOUT_RECORD>, (unsigned)ctas, kPThreads, smem, st, pd);
    else if (layout == LAYOUT_BIN_MAJOR)
        launch_pdl(k_build_persistent<LAYOUT_BIN_MAJOR>, (unsigned)ctas, kPThreads, smem, st, pd);
    else
        launch_pdl(k_build_persistent<-1>, (unsigned)ctas, kPThreads, smem, st, pd);
    prof_mark(prof, KID_PERSISTENT, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

void batch_counts(const PlaneSet &ps, int64_t *c)
{
    const int64_t tiles = (int64_t)ps.g.nb * ps.g.ns;
    const bool carries = ps.colsum != nullptr;
    c[0] = carries ? tiles * ps.nwin_count : 0;
    c[1] = carries ? tiles * (ps.nwin - ps.nwin_count) : 0;
    c[2] = carries ? (int64_t)ps.B * ps.g.W + (int64_t)ps.B * ps.g.H + (int64_t)ps.g.nb * ps.B : 0;
    c[3] = tiles * ps.ngroups;
    c[4] = ps.mom ? tiles * ps.chan[ps.wch].bins : 0;
}

int launch_carries(const PlaneSet &ps, cudaStream_t st, const Prof *prof)
{
    prepare_kernels();
    const TileGrid &g = ps.g;
    int n = 0;
    if (ps.colsum) {
        const int nw_count = ps.nwin_count, nw_weighted = ps.nwin - ps.nwin_count;
        // both window kinds in one launch: the weighted CTAs overlap the count CTAs
        const size_t smem = std::max(nw_weighted ? sums_smem_bytes(g.R, true) : 0, 2 * sizeof(CountSumsSmem));
        prof_mark(prof, KID_SUMS_ALL, 0, st);
        launch_pdl(k_tile_sums_all, dim3(g.ns, g.nb, nw_weighted + (nw_count + 1) / 2), kSumThreads, smem, st, ps,
                   nw_weighted);
        prof_mark(prof, KID_SUMS_ALL, 1, st);
        ++n;
        const int64_t tot = (int64_t)ps.B * g.W + (int64_t)ps.B * g.H + (int64_t)g.nb * ps.B;
        const int64_t blocks = (tot + 255) / 256;
        prof_mark(prof, KID_SCAN, 0, st);
        launch_pdl(k_carry_scan, (unsigned)(blocks < 8192 ? blocks : 8192), 256, 0, st, ps);
        prof_mark(prof, KID_SCAN, 1, st);
        ++n;
    }
    return cudaPeekAtLastError() == cudaSuccess ? n : -1;
}

int launch_build(const PlaneSet &ps, cudaStream_t st, const Prof *prof)
{
    const TileGrid &g = ps.g;
    if (ps.small && ps.sm_bar) return launch_build_small(ps, st, prof);
    if (ps.flags && onepass_ok(ps)) {
        prepare_kernels();
        // flags and ticket start at zero; then one launch builds the frame
        if (cudaMemsetAsync(ps.flags, 0, 4 * ((size_t)g.nb * ps.ngroups + 1), st) != cudaSuccess) return -1;
        prof_mark(prof, KID_ONEPASS, 0, st);
        if (ps.layout == LAYOUT_SLAB)
            launch_pdl(k_build_onepass<LAYOUT_SLAB>, (unsigned)(g.nb * ps.ngroups), 32 * g.ns, onepass_smem_bytes(),
                       st, ps);
        else
            launch_pdl(k_build_onepass<LAYOUT_BIN_MAJOR>, (unsigned)(g.nb * ps.ngroups), 32 * g.ns,
                       onepass_smem_bytes(), st, ps);
        prof_mark(prof, KID_ONEPASS, 1, st);
        return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
    }
    int n = launch_carries(ps, st, prof);
    if (n < 0) return -1;
    const int64_t units = (int64_t)g.nb * g.ns * ps.ngroups;
    const unsigned blocks = (unsigned)((units + 3) / 4);
    if (ps.mom) {
        // count and moment tiles in one launch
        const int64_t mu = (int64_t)g.nb * g.ns * ps.chan[ps.wch].bins;
        const unsigned mblocks = (unsigned)((mu + 3) / 4);
        prof_mark(prof, KID_TILES_BOTH, 0, st);
        if (ps.layout == LAYOUT_SLAB)
            launch_pdl(k_tiles<LAYOUT_SLAB>, mblocks + blocks, 128, 0, st, ps, mblocks);
        else if (ps.layout == LAYOUT_RECORD)
            launch_pdl(k_tiles<LAYOUT_RECORD>, mblocks + blocks, 128, 0, st, ps, mblocks);
        else
            launch_pdl(k_tiles<LAYOUT_BIN_MAJOR>, mblocks + blocks, 128, 0, st, ps, mblocks);
        prof_mark(prof, KID_TILES_BOTH, 1, st);
        ++n;
        return cudaPeekAtLastError() == cudaSuccess ? n : -1;
    }
    prof_mark(prof, KID_TILES_COUNT, 0, st);
    if (ps.layout == LAYOUT_SLAB)
        launch_pdl(k_tiles_count<LAYOUT_SLAB>, blocks, 128, 0, st, ps);
    else if (ps.layout == LAYOUT_RECORD)
        launch_pdl(k_tiles_count<LAYOUT_RECORD>, blocks, 128, 0, st, ps);
    else
        launch_pdl(k_tiles_count<LAYOUT_BIN_MAJOR>, blocks, 128, 0, st, ps);
    prof_mark(prof, KID_TILES_COUNT, 1, st);
    ++n;
    return cudaPeekAtLastError() == cudaSuccess ? n : -1;
}

}  // namespace ih
