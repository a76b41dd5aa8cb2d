// k_phog.cu -- spatial pyramids of gradient orientations (Algorithm 2) and
// their pyramid match kernel (Sec. 2.4.4, Eq. 2.23-2.24).
//
// Step 1: Canny's edge detector (below, k_canny_*).  Steps 2-3: per edge
// pixel of a grayscale search window, the window's central differences
// (replicated borders), the gradient magnitude in fixed point with 4
// fractional bits, w = floor(16 sqrt(gx^2 + gy^2)) (exact integer square
// root: a rounded sqrt corrected by integer comparisons), and the 9-bin
// unsigned orientation (ih_orient.cuh).  Step 4: the w-weighted integral histogram of the orientation
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

// ---- step 1: Canny's detector (J. Canny 1986), integer-exact ------------
//
// k_canny_nms, one CTA per 32 x 32 tile: the 5 x 5 binomial smoothing
// S = sum b_i b_j I (b = 1 4 6 4 1, replicated borders, unnormalised), the
// central-difference gradient of S (replicated borders), its squared
// magnitude M2 = Gx^2 + Gy^2 (int64), non-maximum suppression in four
// direction sectors decided exactly by (|Gx| + |Gy|)^2 < 2 Gx^2 (within
// 22.5 degrees of the column axis) or < 2 Gy^2 (of the row axis), else the
// diagonal given by the signs: a pixel survives when its M2 is above the
// neighbour's on the lower-column side of the line (upper-row side for the
// vertical sector) and not below the opposite one (neighbours outside the
// window count as 0), then the double threshold: class 2 (strong) when
// M2 >= (256 hi)^2, class 1 (weak) when M2 >= (256 lo)^2.  The tile stages
// I (halo 4), the horizontal sums, S (halo 2) and M2 (halo 1) in shared
// memory; a staged position outside the window holds the value of its
// clamped position, which is what the replicated borders give.
//
// Hysteresis (8-connected survivors joined to a strong one) is a union-find
// over the survivors: k_canny_union links each survivor to its survivor
// neighbours W, NW, N and NE (roots always point to smaller indices;
// atomicMin hooks a root, and a hook that lost a race re-links the tree it
// displaced); k_canny_mark then flattens every survivor's parent to its root
// and marks roots of strong survivors; a survivor is an edge pixel when its
// root is marked.  Every pointer walk is bounded (parents strictly decrease,
// and a walk gives up after kUfMaxSteps steps, setting bit 2 of the error
// word, which ih_sync reports as IH_ETIMEOUT).
constexpr int kCT = 32;           // output tile side
constexpr int kCI = kCT + 8;      // staged input side (halo 4)
constexpr int kCS = kCT + 4;      // staged smoothed side (halo 2)
constexpr int kCM = kCT + 2;      // staged magnitude side (halo 1)
constexpr int kUfMaxSteps = 1 << 26;

struct CannySmem {
    int32_t hs[kCI][kCS];         // horizontal binomial sums, rows R0-4.., columns C0-2..
    int32_t s[kCS][kCS];          // S at rows R0-2.., columns C0-2.. (clamped positions)
    long long m2[kCM][kCM];       // M2 at rows R0-1.., columns C0-1.. (0 outside the window)
    uint8_t in[kCI][kCI];         // I at rows R0-4.., columns C0-4.. (clamped)
};

__device__ __forceinline__ int clampi_d(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__global__ void __launch_bounds__(256) k_canny_nms(const uint8_t *__restrict__ gray, int64_t pitch, int H, int W,
                                                   long long tlo, long long thi, uint8_t *__restrict__ cls,
                                                   int32_t *__restrict__ parent, uint8_t *__restrict__ mark)
{
    __shared__ CannySmem sm;
    pdl_wait();
    const int R0 = blockIdx.y * kCT, C0 = blockIdx.x * kCT, tid = threadIdx.x;
    for (int k = tid; k < kCI * kCI; k += 256) {
        const int y = k / kCI, x = k % kCI;
        sm.in[y][x] = __ldg(gray + (int64_t)clampi_d(R0 - 4 + y, 0, H - 1) * pitch + clampi_d(C0 - 4 + x, 0, W - 1));
    }
    __syncthreads();
    for (int k = tid; k < kCI * kCS; k += 256) {
        const int y = k / kCS, xs = k % kCS;
        const int o = clampi_d(C0 - 2 + xs, 0, W - 1) - C0 + 2;  // in-column of tap j = 0
        sm.hs[y][xs] = sm.in[y][o] + 4 * sm.in[y][o + 1] + 6 * sm.in[y][o + 2] + 4 * sm.in[y][o + 3] +
                       sm.in[y][o + 4];
    }
    __syncthreads();
    for (int k = tid; k < kCS * kCS; k += 256) {
        const int ys = k / kCS, xs = k % kCS;
        const int o = clampi_d(R0 - 2 + ys, 0, H - 1) - R0 + 2;
        sm.s[ys][xs] = sm.hs[o][xs] + 4 * sm.hs[o + 1][xs] + 6 * sm.hs[o + 2][xs] + 4 * sm.hs[o + 3][xs] +
                       sm.hs[o + 4][xs];
    }
    __syncthreads();
    for (int k = tid; k < kCM * kCM; k += 256) {
        const int ym = k / kCM, xm = k % kCM;
        const int y = R0 - 1 + ym, x = C0 - 1 + xm;
        long long v = 0;
        if (y >= 0 && y < H && x >= 0 && x < W) {
            const long long gx = sm.s[ym + 1][xm + 2] - sm.s[ym + 1][xm];
            const long long gy = sm.s[ym + 2][xm + 1] - sm.s[ym][xm + 1];
            v = gx * gx + gy * gy;
        }
        sm.m2[ym][xm] = v;
    }
    __syncthreads();
    for (int k = tid; k < kCT * kCT; k += 256) {
        const int ty = k / kCT, tx = k % kCT;
        const int r = R0 + ty, c = C0 + tx;
        if (r >= H || c >= W) continue;
        const long long gx = sm.s[ty + 2][tx + 3] - sm.s[ty + 2][tx + 1];
        const long long gy = sm.s[ty + 3][tx + 2] - sm.s[ty + 1][tx + 2];
        const long long ax = gx < 0 ? -gx : gx, ay = gy < 0 ? -gy : gy, s2 = (ax + ay) * (ax + ay);
        int dr, dc;  // the neighbour on the "minus" side is (r - dr, c - dc)
        if (s2 < 2 * ax * ax) {
            dr = 0; dc = 1;
        } else if (s2 < 2 * ay * ay) {
            dr = 1; dc = 0;
        } else if ((gx > 0) == (gy > 0)) {
            dr = 1; dc = 1;
        } else {
            dr = -1; dc = 1;
        }
        const long long m = sm.m2[ty + 1][tx + 1];
        const long long mm = sm.m2[ty + 1 - dr][tx + 1 - dc], mp = sm.m2[ty + 1 + dr][tx + 1 + dc];
        uint8_t q = 0;
        if (m > mm && m >= mp) q = m >= thi ? 2 : (m >= tlo ? 1 : 0);
        const int64_t i = (int64_t)r * W + c;
        cls[i] = q;
        parent[i] = q ? (int32_t)i : -1;
        mark[i] = 0;
    }
}

__device__ __forceinline__ int32_t uf_find(const volatile int32_t *parent, int32_t x, int *err)
{
    for (int k = 0; k < kUfMaxSteps; ++k) {
        const int32_t p = parent[x];
        if (p == x) return x;
        x = p;
    }
    atomicOr(err, 2);
    return x;
}

__device__ __forceinline__ void uf_unite(int32_t *parent, int32_t a, int32_t b, int *err)
{
    for (int k = 0; k < kUfMaxSteps; ++k) {
        a = uf_find(parent, a, err);
        b = uf_find(parent, b, err);
        if (a == b) return;
        if (a < b) {
            const int32_t t = a;
            a = b;
            b = t;
        }
        const int32_t old = atomicMin(parent + a, b);
        if (old == a) return;  // a was a root and now hangs under b
        a = old;               // a had been re-parented meanwhile: join its new parent to b
    }
    atomicOr(err, 2);
}

__global__ void __launch_bounds__(256) k_canny_union(int H, int W, const uint8_t *__restrict__ cls,
                                                     int32_t *parent, int *err)
{
    pdl_wait();
    const int64_t total = (int64_t)H * W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (!cls[t]) continue;
        const int r = (int)(t / W), c = (int)(t % W);
        if (c > 0 && cls[t - 1]) uf_unite(parent, (int32_t)t, (int32_t)(t - 1), err);
        if (r > 0) {
            const int64_t u = t - W;
            if (c > 0 && cls[u - 1]) uf_unite(parent, (int32_t)t, (int32_t)(u - 1), err);
            if (cls[u]) uf_unite(parent, (int32_t)t, (int32_t)u, err);
            if (c + 1 < W && cls[u + 1]) uf_unite(parent, (int32_t)t, (int32_t)(u + 1), err);
        }
    }
}

// Flattens each survivor's parent to its root and marks the roots of strong
// survivors (all unions are complete when this kernel starts).
__global__ void __launch_bounds__(256) k_canny_mark(int64_t total, const uint8_t *__restrict__ cls, int32_t *parent,
                                                    uint8_t *mark, int *err)
{
    pdl_wait();
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t q = cls[t];
        if (!q) continue;
        const int32_t root = uf_find(parent, (int32_t)t, err);
        parent[t] = root;
        if (q == 2) mark[root] = 1;
    }
}

// Canny edge pixel: a survivor whose (flattened) root is marked.
__device__ __forceinline__ bool canny_edge(const uint8_t *cls, const int32_t *parent, const uint8_t *mark, int64_t i)
{
    return cls[i] && mark[parent[i]];
}

__global__ void __launch_bounds__(256) k_canny_edges(int H, int W, const uint8_t *__restrict__ cls,
                                                     const int32_t *__restrict__ parent,
                                                     const uint8_t *__restrict__ mark, uint8_t *__restrict__ edges,
                                                     int64_t epitch)
{
    pdl_wait();
    const int64_t total = (int64_t)H * W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / W), c = (int)(t % W);
        edges[(int64_t)r * epitch + c] = canny_edge(cls, parent, mark, t) ? 1 : 0;
    }
}

// ---- steps 2-3: the window's own central-difference gradient at edge pixels
__global__ void __launch_bounds__(256) k_phog_planes(const uint8_t *__restrict__ gray, int64_t pitch, int H, int W,
                                                     const uint8_t *__restrict__ cls, const int32_t *__restrict__ parent,
                                                     const uint8_t *__restrict__ mark, uint8_t *__restrict__ bins,
                                                     int32_t *__restrict__ wt)
{
    pdl_wait();
    const int64_t total = (int64_t)H * W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / W), c = (int)(t % W);
        const bool edge = canny_edge(cls, parent, mark, t);
        const uint8_t *row = gray + (int64_t)r * pitch;
        const int gx = (int)__ldg(row + min(c + 1, W - 1)) - (int)__ldg(row + max(c - 1, 0));
        const int gy = (int)__ldg(gray + (int64_t)min(r + 1, H - 1) * pitch + c) -
                       (int)__ldg(gray + (int64_t)max(r - 1, 0) * pitch + c);
        const int64_t m = isqrt_exact(256 * ((int64_t)gx * gx + (int64_t)gy * gy));
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

// Canny's detector into the scratch of one window (classes, parents, marks);
// 3 launches.
static void launch_canny(const uint8_t *gray, int64_t pitch, int H, int W, int lo, int hi, const CannyScratch &cs,
                         int *err, cudaStream_t st)
{
    const long long tlo = (long long)(256 * lo) * (256 * lo), thi = (long long)(256 * hi) * (256 * hi);
    const dim3 grid((W + kCT - 1) / kCT, (H + kCT - 1) / kCT);
    launch_pdl(k_canny_nms, grid, 256, 0, st, gray, pitch, H, W, tlo, thi, cs.cls, cs.parent, cs.mark);
    launch_pdl(k_canny_union, grid_for((int64_t)H * W), 256, 0, st, H, W, (const uint8_t *)cs.cls, cs.parent, err);
    launch_pdl(k_canny_mark, grid_for((int64_t)H * W), 256, 0, st, (int64_t)H * W, (const uint8_t *)cs.cls,
               cs.parent, cs.mark, err);
}

size_t canny_scratch_bytes(int H, int W) { return (size_t)H * W * 6 + 256; }

CannyScratch carve_canny(void *base, int H, int W)
{
    const size_t px = (size_t)H * W;
    CannyScratch cs;
    cs.parent = static_cast<int32_t *>(base);
    cs.cls = reinterpret_cast<uint8_t *>(cs.parent + px);
    cs.mark = cs.cls + px;
    return cs;
}

int launch_canny_edges(const uint8_t *gray, int64_t pitch, int H, int W, int lo, int hi, const CannyScratch &cs,
                       uint8_t *edges, int64_t epitch, int *err, cudaStream_t st, const Prof *prof)
{
    prof_mark(prof, KID_PHOG_BUILD, 0, st);
    launch_canny(gray, pitch, H, W, lo, hi, cs, err, st);
    launch_pdl(k_canny_edges, grid_for((int64_t)H * W), 256, 0, st, H, W, (const uint8_t *)cs.cls,
               (const int32_t *)cs.parent, (const uint8_t *)cs.mark, edges, epitch);
    prof_mark(prof, KID_PHOG_BUILD, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 4 : -1;
}

int launch_phog_build(const uint8_t *gray, int64_t pitch, int H, int W, int lo, int hi, const CannyScratch &cs,
                      uint8_t *bins, int32_t *wt, int64_t P, int64_t *ih, int *err, cudaStream_t st, const Prof *prof)
{
    prof_mark(prof, KID_PHOG_BUILD, 0, st);
    launch_canny(gray, pitch, H, W, lo, hi, cs, err, st);
    launch_pdl(k_phog_planes, grid_for((int64_t)H * W), 256, 0, st, gray, pitch, H, W, (const uint8_t *)cs.cls,
               (const int32_t *)cs.parent, (const uint8_t *)cs.mark, bins, wt);
    const int64_t warps = (int64_t)kPhogBins * H;
    launch_pdl(k_phog_rows, (unsigned)((warps + 7) / 8), 256, 0, st, bins, wt, H, W, P, ih);
    launch_pdl(k_phog_cols, grid_for((int64_t)kPhogBins * P), 256, 0, st, H, P, ih);
    prof_mark(prof, KID_PHOG_BUILD, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 6 : -1;
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
