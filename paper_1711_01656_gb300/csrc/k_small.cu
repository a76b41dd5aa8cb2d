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
//  1. Tile sums.  Each warp bins its rows once (the pixel words stay in
//     registers) into packed 8-bit one-hot fields: the column counts of its
//     rows and, row by row, the strip's row counts (warp reductions).  The
//     CTA turns the warps' column counts into an exclusive prefix over the
//     warps (shared memory) and publishes the tile's column counts, its row
//     counts and its bin totals.
//  2. Grid barrier.  The launch is cooperative, so every CTA is resident;
//     a CTA arrives once its sums are published and waits for all others
//     (bounded: a wait that gives up sets bit 2 of the error word, and
//     ih_sync reports IH_ETIMEOUT).
//  3. Carries as direct sums of the published tile sums: the column carry G
//     (the bands above), the row carries L (the strips to the left) and the
//     tile corner (the tiles above and to the left).
//  4. Each warp seeds its columns with H(r-1, c) -- the corner, the row
//     carries of the band's rows above its own, and the row prefix of G plus
//     the column counts of the warps above -- and writes its rows like the
//     count tiles kernel: per row a packed one-hot, one in-lane prefix and
//     two warp scans, each cell stored once.
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
    uint32_t colw[kSmWarps][kSmThreads];  // per warp: word k of lane L at [k * 32 + L]; then the
                                          // exclusive prefix over the warps
    uint32_t G[2][kSmThreads];            // column carry at the band's top: 16-bit fields of
                                          // bytes 0, 2 ([0]) and 1, 3 ([1]) of word [k * 32 + L]
    uint32_t rowcnt[kSmMaxRows][2];       // row counts over the strip, packed (bins 0-3, 4-7)
    int32_t L[kSmMaxRows][kGroupBins];    // row carries
    int32_t cpart[kSmWarps][kGroupBins];  // partial corners
    int ok;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned int *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// One thread of each CTA: publish the CTA's writes (ordered before this
// thread by the caller's __syncthreads), arrive, and wait until `target`
// CTAs have arrived.  False when the wait gave up.
__device__ __forceinline__ bool grid_arrive_wait(unsigned int *bar, unsigned target, int *err)
{
    __threadfence();
    atomicAdd(bar, 1u);
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
    // each of the lane's columns) and row counts
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
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        sm.colw[w][(2 * q) * 32 + lane] = colw[q][0];
        sm.colw[w][(2 * q + 1) * 32 + lane] = colw[q][1];
    }
    __syncthreads();

    // the tile's sums: exclusive prefix of the column counts over the warps
    // (fields <= R <= 64), published with the tile's total; row counts; bin totals
    {
        uint32_t run = 0u;
#pragma unroll
        for (int ww = 0; ww < kSmWarps; ++ww) {
            const uint32_t v = sm.colw[ww][tid];
            sm.colw[ww][tid] = run;
            run += v;
        }
        ps.sm_col[(int64_t)blockIdx.x * kSmThreads + tid] = run;
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
    if (tid == 0) sm.ok = grid_arrive_wait(ps.sm_bar, gridDim.x, ps.err) ? 1 : 0;
    __syncthreads();
    if (!sm.ok) return;

    // 3. carries: G over the bands above (16-bit pair fields, <= H), the row
    // carries of the band's rows over the strips to the left, the corner
    {
        uint32_t lo = 0u, hi = 0u;
        const uint32_t *src = ps.sm_col + ((int64_t)gi * ntiles + j) * kSmThreads + tid;
        int ib = 0;
        for (; ib + 4 <= i; ib += 4) {
            uint32_t v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldcg(src + (int64_t)(ib + u) * g.ns * kSmThreads);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                lo += v[u] & 0x00ff00ffu;
                hi += (v[u] >> 8) & 0x00ff00ffu;
            }
        }
        for (; ib < i; ++ib) {
            const uint32_t v = __ldcg(src + (int64_t)ib * g.ns * kSmThreads);
            lo += v & 0x00ff00ffu;
            hi += (v >> 8) & 0x00ff00ffu;
        }
        sm.G[0][tid] = lo;
        sm.G[1][tid] = hi;
    }
    if (tid < 2 * nr) {
        const int r = tid >> 1, h = tid & 1;
        uint32_t lo = 0u, hi = 0u;
        for (int jj = 0; jj < j; ++jj) {
            const uint32_t v = __ldcg(ps.sm_row + (((int64_t)jj * ps.ngroups + gi) * g.H + R0 + r) * 2 + h);
            lo += v & 0x00ff00ffu;
            hi += (v >> 8) & 0x00ff00ffu;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) sm.L[r][4 * h + e] = pair_field(lo, hi, e);
    } else if (tid >= 2 * nr && tid < 2 * kSmMaxRows) {
        const int r = tid >> 1, h = tid & 1;
#pragma unroll
        for (int e = 0; e < 4; ++e) sm.L[r][4 * h + e] = 0;
    }
    {
        // corner: tiles (i', j') with i' < i, j' < j; thread = (bin tid & 7, slice tid >> 3)
        const int b = tid & 7, s = tid >> 3, n = i * j;
        int t = 0;
        for (int k = s; k < n; k += kSmThreads / 8) {
            const int ii = k / j, jj = k - (k / j) * j;
            t += __ldcg(ps.sm_tot + ((int64_t)(ii * g.ns + jj) * ps.ngroups + gi) * kGroupBins + b);
        }
        t += __shfl_xor_sync(kFull, t, 8);
        t += __shfl_xor_sync(kFull, t, 16);
        if (lane < 8) sm.cpart[w][lane] = t;
    }
    __syncthreads();

    // 4. the warp's rows
    if (nrw == 0) return;
    int TR[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        int t = 0;
#pragma unroll
        for (int ww = 0; ww < kSmWarps; ++ww) t += sm.cpart[ww][b];
        for (int r = 0; r < rw; ++r) t += sm.L[r][b];
        TR[b] = t;  // H(R0 + rw - 1, C0 - 1)
    }
    int acc[NB][4];
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        // column counts over rows [0, R0 + rw) of the lane's 4 columns
        int p[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = (2 * q + (b >> 2)) * 32 + lane;
            p[q] = pair_field(sm.G[0][k], sm.G[1][k], b & 3) + (int)((sm.colw[w][k] >> (8 * (b & 3))) & 0xff);
            if (q >= nvalid) p[q] = 0;
        }
        p[1] += p[0];
        p[2] += p[1];
        p[3] += p[2];
        const int incl = warp_incl_scan(p[3], lane);
        const int base = TR[b] + (incl - p[3]);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[b][q] = p[q] + base;
    }
#pragma unroll
    for (int k = 0; k < kSmMaxRpw; ++k) {
        if (k >= nrw) break;
        const int r = R0 + rw + k;
        uint32_t P0[4], P1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int qb = bin_of((px[k] >> (8 * q)) & 0xff, bins, mode);
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

template <int LAYOUT>
__global__ void __launch_bounds__(kSmThreads, 2) k_build_small(const __grid_constant__ PlaneSet ps)
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

bool small_plan(PlaneSet &ps, int nsm)
{
    static const bool on = [] {
        const char *e = getenv("IH_SMALL");
        return !(e && e[0] == '0');
    }();
    (void)nsm;
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
           r256(4);
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

int launch_build_small(const PlaneSet &ps, cudaStream_t st, const Prof *prof)
{
    if (cudaMemsetAsync(ps.sm_bar, 0, sizeof(unsigned int), st) != cudaSuccess) return -1;
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
        cudaLaunchKernelEx(&cfg, k_build_small<LAYOUT_SLAB>, ps);
    else
        cudaLaunchKernelEx(&cfg, k_build_small<LAYOUT_BIN_MAJOR>, ps);
    prof_mark(prof, KID_SMALL, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace ih
