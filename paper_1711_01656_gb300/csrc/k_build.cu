// k_build.cu -- integral histograms (Eq. 2.15) and weighted integral
// histograms (Eq. 3.4) on a grid of tiles, written once.
//
// Per pixel the thesis's Algorithm 5 adds Q(k, I(x,y)) into a recurrence that
// is serial in both directions.  Here the frame is cut into bands of R rows
// and strips of Wc columns; three kernels remove the serial dependence:
//
//   k_tile_sums   reads the pixels of one tile and a window of bins and
//                 accumulates, in shared memory, the column sums over the
//                 band and the row sums over the strip (bin-independent
//                 cost per pixel: two shared-memory atomics);
//   k_carry_scan  turns them into the exclusive prefixes G (over bands, per
//                 column), L (over strips, per row) and the tile corners;
//   k_ih_tiles    one warp per (tile, bin group): the warp covers 128
//                 columns (4 per lane), walks the band's rows, forms each
//                 row's prefix with an in-lane prefix plus a warp shuffle
//                 scan, adds the row carry and accumulates down the
//                 columns in registers, and stores each output cell once
//                 with 16-byte stores (a warp writes 512 contiguous bytes
//                 per bin and row).
//
// No kernel waits on another CTA; the only inter-CTA data flow is through
// the carry arrays between launches on the same stream.
#include "ih_internal.cuh"

namespace ih {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int K>
struct Wt;
template <>
struct Wt<WK_ONE> {
    typedef int32_t T;
    __device__ __forceinline__ static T w(int, int) { return 1; }
};
template <>
struct Wt<WK_COL> {
    typedef long long T;
    __device__ __forceinline__ static T w(int, int c) { return c; }
};
template <>
struct Wt<WK_ROW> {
    typedef long long T;
    __device__ __forceinline__ static T w(int r, int) { return r; }
};
template <>
struct Wt<WK_COL2> {
    typedef long long T;
    __device__ __forceinline__ static T w(int, int c) { return (long long)c * c; }
};
template <>
struct Wt<WK_ROW2> {
    typedef long long T;
    __device__ __forceinline__ static T w(int r, int) { return (long long)r * r; }
};

// Eq. 2.15's Q: the channel-local bin of value v, or -1 for none.
__device__ __forceinline__ int bin_of(int v, int bins, int mode)
{
    if (mode == 0) return (v * bins) >> 8;
    return v < bins ? v : -1;
}

__device__ __forceinline__ void sm_add(int32_t *p, int32_t v) { atomicAdd(p, v); }
__device__ __forceinline__ void sm_add(long long *p, long long v)
{
    atomicAdd(reinterpret_cast<unsigned long long *>(p), static_cast<unsigned long long>(v));
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

__device__ __forceinline__ void store4(int32_t *p, const int32_t (&a)[4])
{
    *reinterpret_cast<int4 *>(p) = make_int4(a[0], a[1], a[2], a[3]);
}
__device__ __forceinline__ void store4(long long *p, const long long (&a)[4])
{
    reinterpret_cast<longlong2 *>(p)[0] = make_longlong2(a[0], a[1]);
    reinterpret_cast<longlong2 *>(p)[1] = make_longlong2(a[2], a[3]);
}

// Channel-local bins of the 4 pixels (r, c..c+3); -1 outside [0, cend).
__device__ __forceinline__ void load_bins(const ChanDev &ch, int r, int c, int cend, bool vec_ok,
                                          int (&q)[4])
{
    const uint8_t *row = ch.plane + (int64_t)r * ch.pitch;
    if (vec_ok && c + 3 < cend) {
        const uint32_t v = __ldg(reinterpret_cast<const unsigned int *>(row + c));
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) q[jj] = bin_of((v >> (8 * jj)) & 0xff, ch.bins, ch.mode);
    } else {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
            q[jj] = (c + jj < cend) ? bin_of(__ldg(row + c + jj), ch.bins, ch.mode) : -1;
    }
}

constexpr int kSumCols = 256;  // columns per pass of k_tile_sums

template <int K, int BW>
__global__ void __launch_bounds__(256) k_tile_sums(const __grid_constant__ PlaneSet ps)
{
    typedef typename Wt<K>::T T;
    const TileGrid &g = ps.g;
    const int j = blockIdx.x, i = blockIdx.y;
    const GroupDev pg = ps.pgrp[blockIdx.z];
    const ChanDev &ch = ps.chan[pg.chan];
    const int R0 = i * g.R, nr = min(g.R, g.H - R0);
    const int C0 = j * g.Wc, C1 = min(C0 + g.Wc, g.W);
    const int64_t bg0 = ch.bin_off + pg.b_lo;
    extern __shared__ __align__(16) unsigned char smem[];
    T *row_acc = reinterpret_cast<T *>(smem);  // [R][BW]
    T *col_acc = row_acc + g.R * BW;           // [BW][kSumCols]
    const int tid = threadIdx.x;
    T *colsum = static_cast<T *>(ps.colsum);
    T *rowsum = static_cast<T *>(ps.rowsum);
    T *tilesum = static_cast<T *>(ps.tilesum);

    for (int k = tid; k < nr * BW; k += blockDim.x) row_acc[k] = 0;
    for (int cp = C0; cp < C1; cp += kSumCols) {
        const int cw = min(kSumCols, C1 - cp);
        for (int k = tid; k < BW * kSumCols; k += blockDim.x) col_acc[k] = 0;
        __syncthreads();
        for (int idx = tid; idx < nr * kSumCols; idx += blockDim.x) {
            const int rr = idx / kSumCols, cc = idx % kSumCols;
            if (cc < cw) {
                const int r = R0 + rr, c = cp + cc;
                const int q = bin_of(__ldg(ch.plane + (int64_t)r * ch.pitch + c), ch.bins, ch.mode) -
                              pg.b_lo;
                if (q >= 0 && q < pg.nb) {
                    const T w = Wt<K>::w(r, c);
                    sm_add(&col_acc[q * kSumCols + cc], w);
                    sm_add(&row_acc[rr * BW + q], w);
                }
            }
        }
        __syncthreads();
        for (int k = tid; k < pg.nb * kSumCols; k += blockDim.x) {
            const int b = k / kSumCols, cc = k % kSumCols;
            if (cc < cw) colsum[((int64_t)i * ps.B + bg0 + b) * g.W + cp + cc] = col_acc[b * kSumCols + cc];
        }
        __syncthreads();
    }
    for (int k = tid; k < pg.nb * nr; k += blockDim.x) {
        const int b = k / nr, rr = k % nr;
        rowsum[((int64_t)j * ps.B + bg0 + b) * g.H + R0 + rr] = row_acc[rr * BW + b];
    }
    if (tid < pg.nb) {
        T s = 0;
        for (int rr = 0; rr < nr; ++rr) s += row_acc[rr * BW + tid];
        tilesum[((int64_t)i * g.ns + j) * ps.B + bg0 + tid] = s;
    }
}

template <int K>
__global__ void __launch_bounds__(256) k_carry_scan(const __grid_constant__ PlaneSet ps)
{
    typedef typename Wt<K>::T T;
    const TileGrid &g = ps.g;
    const int64_t B = ps.B;
    const int64_t nA = B * g.W, nB = B * g.H, nC = (int64_t)g.ns * B;
    T *colsum = static_cast<T *>(ps.colsum);
    T *rowsum = static_cast<T *>(ps.rowsum);
    const T *tilesum = static_cast<const T *>(ps.tilesum);
    T *corner = static_cast<T *>(ps.corner);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nA + nB + nC;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (t < nA) {  // G(i, c, b): exclusive over bands
            T *p = colsum + t;
            T run = 0;
            for (int i = 0; i < g.nb; ++i) {
                const T v = p[(int64_t)i * nA];
                p[(int64_t)i * nA] = run;
                run += v;
            }
        } else if (t < nA + nB) {  // L(j, r, b): exclusive over strips
            T *p = rowsum + (t - nA);
            T run = 0;
            for (int j = 0; j < g.ns; ++j) {
                const T v = p[(int64_t)j * nB];
                p[(int64_t)j * nB] = run;
                run += v;
            }
        } else {  // corner(i, j, b) = sum over tiles above-left
            const int64_t u = t - nA - nB;
            const int j = (int)(u / B);
            const int64_t b = u % B;
            T run = 0;
            for (int i = 0; i < g.nb; ++i) {
                corner[((int64_t)i * g.ns + j) * B + b] = run;
                T s = 0;
                for (int jj = 0; jj < j; ++jj) s += tilesum[((int64_t)i * g.ns + jj) * B + b];
                run += s;
            }
        }
    }
}

template <int K, int NB>
__global__ void __launch_bounds__(128) k_ih_tiles(const __grid_constant__ PlaneSet ps)
{
    typedef typename Wt<K>::T T;
    __shared__ T RLs[4][kMaxBandRows * NB];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const TileGrid &g = ps.g;
    const int ng = ps.ngroups;
    const int64_t unit = (int64_t)blockIdx.x * 4 + wid;
    if (unit >= (int64_t)g.nb * g.ns * ng) return;  // whole warp
    const int tile = (int)(unit / ng), gi = (int)(unit % ng);
    const int i = tile / g.ns, j = tile % g.ns;
    const GroupDev gr = ps.grp[gi];
    const ChanDev &ch = ps.chan[gr.chan];
    const int64_t bg0 = ch.bin_off + gr.b_lo;
    const int R0 = i * g.R, nr = min(g.R, g.H - R0);
    const int C0 = j * g.Wc, C1 = min(C0 + g.Wc, g.W);
    T *RL = RLs[wid];
    const T *Lc = static_cast<const T *>(ps.rowsum);
    const T *Gc = static_cast<const T *>(ps.colsum);
    const T *Cc = static_cast<const T *>(ps.corner);
    T *out = static_cast<T *>(ps.out);

    // row carries L(j, r, b) of this band, per bin of the group
    for (int k = lane; k < nr * NB; k += 32) {
        const int rr = k / NB, b = k % NB;
        RL[k] = (Lc && b < gr.nb) ? Lc[((int64_t)j * ps.B + bg0 + b) * g.H + R0 + rr] : T(0);
    }
    T TR[NB];  // corner + sum of G over the strip's columns left of the chunk
#pragma unroll
    for (int b = 0; b < NB; ++b)
        TR[b] = (Cc && b < gr.nb) ? Cc[((int64_t)i * g.ns + j) * ps.B + bg0 + b] : T(0);
    __syncwarp();

    const bool vec_ok = ((ch.pitch & 3) == 0) && ((reinterpret_cast<uintptr_t>(ch.plane) & 3) == 0);
    for (int cc = C0; cc < C1; cc += kChunk) {
        const int c = cc + lane * 4;
        T acc[NB][4];
        // seed each column with H(R0-1, c): corner + prefix of G along the strip
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            T p[4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
                p[jj] = (Gc && b < gr.nb && c + jj < C1)
                            ? Gc[((int64_t)i * ps.B + bg0 + b) * g.W + c + jj]
                            : T(0);
            p[1] += p[0];
            p[2] += p[1];
            p[3] += p[2];
            const T incl = warp_incl_scan(p[3], lane);
            const T base = TR[b] + (incl - p[3]);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) acc[b][jj] = base + p[jj];
            TR[b] += __shfl_sync(kFull, incl, 31);
        }
        for (int rr = 0; rr < nr; ++rr) {
            const int r = R0 + rr;
            int q[4];
            load_bins(ch, r, c, C1, vec_ok, q);
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                if (b < gr.nb) {  // warp-uniform
                    const int bin = gr.b_lo + b;
                    T p[4];
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) p[jj] = (q[jj] == bin) ? Wt<K>::w(r, c + jj) : T(0);
                    p[1] += p[0];
                    p[2] += p[1];
                    p[3] += p[2];
                    const T incl = warp_incl_scan(p[3], lane);
                    const T base = RL[rr * NB + b] + (incl - p[3]);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc[b][jj] += base + p[jj];
                    if (c < g.P) store4(out + ((bg0 + b) * g.H + r) * g.P + c, acc[b]);
                    const T tot = __shfl_sync(kFull, incl, 31);
                    __syncwarp();
                    if (lane == 0) RL[rr * NB + b] += tot;
                }
            }
        }
        __syncwarp();
    }
}

template <int K, int BW>
void set_smem_attr(size_t bytes)
{
    cudaFuncSetAttribute(k_tile_sums<K, BW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int K, int NB>
int launch_kind(const PlaneSet &ps, cudaStream_t st, const Prof *prof)
{
    constexpr int BW = (K == WK_ONE) ? 32 : 16;
    int n = 0;
    const TileGrid &g = ps.g;
    if (ps.colsum) {
        const size_t smem = tile_sums_smem_bytes(ps, K);
        if (smem > 48 * 1024) set_smem_attr<K, BW>(smem);
        prof_mark(prof, kid_sums(K), 0, st);
        k_tile_sums<K, BW><<<dim3(g.ns, g.nb, ps.npgroups), 256, smem, st>>>(ps);
        prof_mark(prof, kid_sums(K), 1, st);
        ++n;
        const int64_t tot = (int64_t)ps.B * g.W + (int64_t)ps.B * g.H + (int64_t)g.ns * ps.B;
        const int64_t blocks = (tot + 255) / 256;
        prof_mark(prof, kid_scan(K), 0, st);
        k_carry_scan<K><<<(unsigned)(blocks < 4864 ? blocks : 4864), 256, 0, st>>>(ps);
        prof_mark(prof, kid_scan(K), 1, st);
        ++n;
    }
    const int64_t units = (int64_t)g.nb * g.ns * ps.ngroups;
    prof_mark(prof, kid_tiles(K), 0, st);
    k_ih_tiles<K, NB><<<(unsigned)((units + 3) / 4), 128, 0, st>>>(ps);
    prof_mark(prof, kid_tiles(K), 1, st);
    ++n;
    return cudaPeekAtLastError() == cudaSuccess ? n : -1;
}

}  // namespace

size_t tile_sums_smem_bytes(const PlaneSet &ps, int kind)
{
    const size_t bw = (kind == WK_ONE) ? 32 : 16;
    const size_t el = (kind == WK_ONE) ? 4 : 8;
    return (ps.g.R * bw + bw * kSumCols) * el;
}

int launch_plane_set(const PlaneSet &ps, int kind, cudaStream_t st, const Prof *prof)
{
    switch (kind) {
    case WK_ONE: return launch_kind<WK_ONE, 8>(ps, st, prof);
    case WK_COL: return launch_kind<WK_COL, 4>(ps, st, prof);
    case WK_ROW: return launch_kind<WK_ROW, 4>(ps, st, prof);
    case WK_COL2: return launch_kind<WK_COL2, 4>(ps, st, prof);
    case WK_ROW2: return launch_kind<WK_ROW2, 4>(ps, st, prof);
    }
    return -1;
}

}  // namespace ih
