// k_phog.cu -- spatial pyramids of gradient orientations (Algorithm 2) and
// their pyramid match kernel (Sec. 2.4.4, Eq. 2.23-2.24).
//
// Steps 1-3: per pixel of a grayscale search window, central differences
// (step 1, replicated borders), the gradient magnitude in fixed point with 4
// fractional bits, w = floor(16 sqrt(gx^2 + gy^2)) (exact integer square
// root: a rounded sqrt corrected by integer comparisons), and the 9-bin
// unsigned orientation (ih_orient.cuh); a pixel is an edge pixel when
// w >= 16 tau.  Step 4: the w-weighted integral histogram of the orientation
// bins over edge pixels (Eq. 3.4 with a pixel weight), int64, by a row pass
// (one warp per (bin, row): chunked warp scans) and a column pass (one thread
// per (bin, column), running sums down the rows).  Steps 5-20: the L+1-level
// descriptor of a window is, for level l, its 2^l x 2^l cells of
// floor(h/2^l) x floor(w/2^l) pixels, each cell's 9-bin histogram by four
// corners (Eq. 2.16).  The match kernel of a placement is
//   kappa = (I^0 + sum_{l=1..L} 2^(l-1) I^l) / 2^L,
// the I^l (sums of min over level l's entries) exact in int64 and the
// quotient rounded once to float.
#include <math.h>

#include "ih_internal.cuh"
#include "ih_orient.cuh"

namespace ih {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// floor(sqrt(n)), exact: CUDA's sqrt gives a candidate, integer comparisons
// fix it.
__device__ __forceinline__ int64_t isqrt_exact(int64_t n)
{
    int64_t s = (int64_t)sqrt((double)n);
    while (s * s > n) --s;
    while ((s + 1) * (s + 1) <= n) ++s;
    return s;
}

__global__ void __launch_bounds__(256) k_phog_planes(const uint8_t *__restrict__ gray, int64_t pitch, int H, int W,
                                                     int tau, uint8_t *__restrict__ bins, int32_t *__restrict__ wt)
{
    pdl_wait();
    const int64_t total = (int64_t)H * W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / W), c = (int)(t % W);
        const uint8_t *row = gray + (int64_t)r * pitch;
        const int gx = (int)__ldg(row + min(c + 1, W - 1)) - (int)__ldg(row + max(c - 1, 0));
        const int gy = (int)__ldg(gray + (int64_t)min(r + 1, H - 1) * pitch + c) -
                       (int)__ldg(gray + (int64_t)max(r - 1, 0) * pitch + c);
        const int64_t m = isqrt_exact(256 * ((int64_t)gx * gx + (int64_t)gy * gy));
        const bool edge = m >= 16 * (int64_t)tau;
        bins[t] = edge ? (uint8_t)orientation_bin9(gx, gy) : (uint8_t)255;
        wt[t] = edge ? (int32_t)m : 0;
    }
}

// Row pass: out[b][r][c] = sum_{c' <= c, bin(r, c') = b} w(r, c').  One warp
// per (bin, row); each lane takes 4 adjacent pixels of a 128-column chunk.
__global__ void __launch_bounds__(256) k_phog_rows(const uint8_t *__restrict__ bins, const int32_t *__restrict__ wt,
                                                   int H, int W, int64_t P, int64_t *__restrict__ out)
{
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int64_t unit = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (unit >= (int64_t)kPhogBins * H) return;
    const int b = (int)(unit / H), r = (int)(unit % H);
    int64_t run = 0;
    for (int cc = 0; cc < W; cc += 128) {
        int64_t v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = cc + 4 * lane + j;
            const int64_t i = (int64_t)r * W + c;
            v[j] = (c < W && __ldg(bins + i) == b) ? (int64_t)__ldg(wt + i) : 0;
            if (j) v[j] += v[j - 1];
        }
        int64_t x = v[3];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, x, d);
            if (lane >= d) x += y;
        }
        const int64_t excl = run + x - v[3];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = cc + 4 * lane + j;
            if (c < P) out[((int64_t)b * H + r) * P + c] = excl + v[j];
        }
        run += __shfl_sync(kFull, x, 31);
    }
}

// Column pass, in place: running sums down the rows, one thread per (bin,
// column).
__global__ void __launch_bounds__(256) k_phog_cols(int H, int64_t P, int64_t *__restrict__ out)
{
    pdl_wait();
    const int64_t total = (int64_t)kPhogBins * P;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(t / P);
        const int64_t c = t % P;
        int64_t *col = out + (int64_t)b * H * P + c;
        int64_t run = 0;
        for (int r = 0; r < H; ++r) {
            run += col[(int64_t)r * P];
            col[(int64_t)r * P] = run;
        }
    }
}

// Four-corner weighted count of bin b over rows [r0, r1] x cols [c0, c1].
__device__ __forceinline__ int64_t phog_box(const int64_t *ih, int H, int64_t P, int b, int r0, int c0, int r1,
                                            int c1)
{
    if (r1 < r0 || c1 < c0) return 0;
    const int64_t *p = ih + (int64_t)b * H * P;
    int64_t s = __ldg(p + (int64_t)r1 * P + c1);
    if (r0 > 0) s -= __ldg(p + (int64_t)(r0 - 1) * P + c1);
    if (c0 > 0) s -= __ldg(p + (int64_t)r1 * P + (c0 - 1));
    if (r0 > 0 && c0 > 0) s += __ldg(p + (int64_t)(r0 - 1) * P + (c0 - 1));
    return s;
}

// Entry e of a descriptor: its level, cell and bin.
__device__ __forceinline__ void phog_entry(int64_t e, int &l, int &i, int &j, int &q)
{
    int64_t off = 0;
    l = 0;
    while (e >= off + (int64_t)kPhogBins * (1 << (2 * l))) {
        off += (int64_t)kPhogBins * (1 << (2 * l));
        ++l;
    }
    const int64_t k = e - off;
    const int cell = (int)(k / kPhogBins), s = 1 << l;
    q = (int)(k % kPhogBins);
    i = cell / s;
    j = cell % s;
}

// One thread per (window, descriptor entry).
__global__ void __launch_bounds__(256) k_phog_desc(const int64_t *__restrict__ ih, int H, int W, int64_t P, int L,
                                                   const int32_t *__restrict__ wins, int64_t n, int64_t D,
                                                   int64_t *__restrict__ out, int *err)
{
    pdl_wait();
    const int64_t total = n * D;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t wi = t / D, e = t % D;
        const int r0 = __ldg(wins + 4 * wi), c0 = __ldg(wins + 4 * wi + 1);
        const int r1 = __ldg(wins + 4 * wi + 2), c1 = __ldg(wins + 4 * wi + 3);
        if (r0 < 0 || c0 < 0 || r0 > r1 || c0 > c1 || r1 >= H || c1 >= W) {
            out[t] = -1;
            if (e == 0) atomicOr(err, 1);
            continue;
        }
        const int wh = r1 - r0 + 1, ww = c1 - c0 + 1;
        int l, i, j, q;
        phog_entry(e, l, i, j, q);
        const int ch = wh >> l, cw = ww >> l;
        out[t] = phog_box(ih, H, P, q, r0 + i * ch, c0 + j * cw, r0 + (i + 1) * ch - 1, c0 + (j + 1) * cw - 1);
    }
}

// One thread per placement: the pyramid match kernel against the target
// descriptor (in shared memory).
__global__ void __launch_bounds__(256) k_phog_match(const int64_t *__restrict__ ih, int H, int64_t P, int L,
                                                    const int64_t *__restrict__ target, int64_t D, int wh, int ww,
                                                    int sr0, int sc0, int sr1, int sc1, float *__restrict__ out)
{
    pdl_wait();
    extern __shared__ int64_t s_t[];
    for (int64_t k = threadIdx.x; k < D; k += blockDim.x) s_t[k] = __ldg(target + k);
    __syncthreads();
    const int nc = sc1 - sc0 + 1;
    const int64_t total = (int64_t)(sr1 - sr0 + 1) * nc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r0 = sr0 + (int)(t / nc), c0 = sc0 + (int)(t % nc);
        int64_t num = 0, k = 0;
        for (int l = 0; l <= L; ++l) {
            const int s = 1 << l, ch = wh >> l, cw = ww >> l;
            int64_t il = 0;
            for (int i = 0; i < s; ++i)
                for (int j = 0; j < s; ++j)
                    for (int q = 0; q < kPhogBins; ++q, ++k) {
                        const int64_t x = phog_box(ih, H, P, q, r0 + i * ch, c0 + j * cw, r0 + (i + 1) * ch - 1,
                                                   c0 + (j + 1) * cw - 1);
                        il += x < s_t[k] ? x : s_t[k];
                    }
            num += l == 0 ? il : (il << (l - 1));
        }
        out[t] = (float)num / (float)(1 << L);
    }
}

unsigned grid_for(int64_t total)
{
    const int64_t b = (total + 255) / 256;
    return (unsigned)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

}  // namespace

int launch_phog_build(const uint8_t *gray, int64_t pitch, int H, int W, int tau, uint8_t *bins, int32_t *wt,
                      int64_t P, int64_t *ih, cudaStream_t st, const Prof *prof)
{
    prof_mark(prof, KID_PHOG_BUILD, 0, st);
    launch_pdl(k_phog_planes, grid_for((int64_t)H * W), 256, 0, st, gray, pitch, H, W, tau, bins, wt);
    const int64_t warps = (int64_t)kPhogBins * H;
    launch_pdl(k_phog_rows, (unsigned)((warps + 7) / 8), 256, 0, st, bins, wt, H, W, P, ih);
    launch_pdl(k_phog_cols, grid_for((int64_t)kPhogBins * P), 256, 0, st, H, P, ih);
    prof_mark(prof, KID_PHOG_BUILD, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 3 : -1;
}

int launch_phog_descriptors(const int64_t *ih, int H, int W, int64_t P, int L, const int32_t *wins, int64_t n,
                            int64_t *out, int *err, cudaStream_t st, const Prof *prof)
{
    const int64_t D = phog_descriptor_len(L);
    prof_mark(prof, KID_PHOG_QUERY, 0, st);
    launch_pdl(k_phog_desc, grid_for(n * D), 256, 0, st, ih, H, W, P, L, wins, n, D, out, err);
    prof_mark(prof, KID_PHOG_QUERY, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_phog_match(const int64_t *ih, int H, int64_t P, int L, const int64_t *target, int wh, int ww, int sr0,
                      int sc0, int sr1, int sc1, float *out, cudaStream_t st, const Prof *prof)
{
    const int64_t D = phog_descriptor_len(L);
    const int64_t total = (int64_t)(sr1 - sr0 + 1) * (sc1 - sc0 + 1);
    prof_mark(prof, KID_PHOG_QUERY, 0, st);
    launch_pdl(k_phog_match, grid_for(total), 256, (size_t)D * 8, st, ih, H, P, L, target, D, wh, ww, sr0, sc0, sr1, sc1,
                                                               out);
    prof_mark(prof, KID_PHOG_QUERY, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace ih
