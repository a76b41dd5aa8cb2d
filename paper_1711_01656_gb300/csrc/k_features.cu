// k_features.cu -- the tracker's feature channels from planar RGB.
//
// Intensity I = floor((R+G+B)/3) (Eq. 2.33) and, for central-difference
// steps s = 1, 2, 4 with replicated borders, the unsigned gradient
// orientation of I quantised into 9 bins of 20 degrees (the orientation
// channel of Fig. 2.3 / Algorithm 2, at three cell levels).
//
// The orientation bin is decided without trigonometry: after folding the
// gradient into the upper half plane, theta >= 20j degrees iff the cross
// product of the unit vector at 20j degrees with (gx, gy) is >= 0, so the bin
// is the number of the 8 inner boundaries the gradient lies at or beyond.
// Only the four boundaries of the first quadrant are tested: with
// theta' = atan2(gy, |gx|) in [0, 90] and n the number of j = 1..4 with
// theta' >= 20j, the bin is n for gx >= 0 and 8 - n for gx < 0 (theta =
// 180 - theta' lies at or beyond 20j for all j <= 4 and for j = 9 - m,
// m = 1..4, exactly when theta' <= 20m; no integer gradient other than 0
// lies on a boundary, so "<=" and "<" agree).
// The unit vectors are scaled by 2^22 and rounded; for integer gradients in
// [-255,255]^2 the angle to the nearest boundary is > 1e-5 rad, so the sign
// of the cross product is exact: the rounding of the constants moves it by
// at most |gx|/2 + |gy|/2 <= |g|, while its true magnitude exceeds
// 2^22 * 1e-5 * |g| > 41 |g|.  Every term stays below 2^31 (4.2e6 * 255 +
// 4.2e6 * 255 < 2.1e9), so the test runs in int32.  The pre-pass reads n
// for the folded gradient from a table that this same test fills once per
// device (256 x 256 entries, one per (|gx|, gy)).
//
// One CTA computes a 16 x 128 tile, 4 adjacent pixels per thread as one
// 32-bit word of bytes.  It stages I for the tile plus a 4-pixel halo in
// shared memory as words, clamping coordinates when it loads, which gives the
// replicated borders: the staged byte for column x is I at clamp(x), which is
// exactly the neighbour a central difference at the frame edge needs.  The
// neighbours at horizontal distance s = 1, 2 are assembled from two staged
// words with byte permutes; s = 4 is the adjacent word.
#include <mutex>

#include "ih_internal.cuh"
#include "ih_orient.cuh"

namespace ih {

namespace {

constexpr int kTR = 16, kTC = 128, kHalo = 4;
constexpr int kSR = kTR + 2 * kHalo;  // staged rows
constexpr int kSW = kTC / 4 + 2;      // staged words per row (one halo word each side)
constexpr int kThreads = 256;

__device__ __forceinline__ int byte_of(uint32_t w, int j) { return (int)((w >> (8 * j)) & 0xff); }

// The count n of orientation_bin9 for every folded gradient: entry
// ax * 256 + gy (0 <= ax, gy <= 255) holds the number of the four
// first-quadrant boundaries at or below the angle of (ax, gy), computed by
// the same int32 test (0 for the zero gradient).  Filled once per device by
// prepare_features; 64 KB, so it stays in L1 while the pre-pass runs.
__device__ uint8_t g_orient_n[256 * 256];

__global__ void k_orient_table()
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 256 * 256) return;
    const int ax = t >> 8, gy = t & 255;
    g_orient_n[t] = (uint8_t)((ax | gy) ? orientation_bin9(ax, gy) : 0);
}

// orientation_bin9 through the table: fold into the upper half plane, look
// up n for (|gx|, gy), and mirror for gx < 0.
__device__ __forceinline__ int orientation_bin9_table(int gx, int gy)
{
    if (gy < 0 || (gy == 0 && gx < 0)) {
        gx = -gx;
        gy = -gy;
    }
    const int n = __ldg(g_orient_n + ((gx < 0 ? -gx : gx) << 8) + gy);
    return gx < 0 ? 8 - n : n;
}

// floor((R+G+B)/3) of 4 packed pixels.
__device__ __forceinline__ uint32_t intensity4(uint32_t r, uint32_t g, uint32_t b)
{
    uint32_t out = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) out |= (uint32_t)((byte_of(r, j) + byte_of(g, j) + byte_of(b, j)) / 3) << (8 * j);
    return out;
}

// The 4 bytes of row `row` at columns c..c+3, each column clamped to [0, W).
__device__ __forceinline__ uint32_t load4_clamped(const uint8_t *row, int c, int W, bool vec)
{
    if (vec && c >= 0 && c + 3 < W) return __ldg(reinterpret_cast<const unsigned int *>(row + c));
    uint32_t v = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) v |= (uint32_t)__ldg(row + min(max(c + j, 0), W - 1)) << (8 * j);
    return v;
}

__device__ __forceinline__ void store4(uint8_t *dst, uint32_t v, int nv, bool vec)
{
    if (vec && nv == 4) {
        *reinterpret_cast<uint32_t *>(dst) = v;
        return;
    }
    for (int j = 0; j < nv; ++j) dst[j] = (uint8_t)(v >> (8 * j));
}

__device__ __forceinline__ void features_tile(const uint8_t *__restrict__ pr, const uint8_t *__restrict__ pg,
                                              const uint8_t *__restrict__ pb, int64_t pitch, int H, int W,
                                              uint8_t *out_rgb, uint8_t *out_i, uint8_t *out_hog, int64_t opitch,
                                              int tr, int tc)
{
    __shared__ uint32_t sI[kSR][kSW];
    const int r0 = tr * kTR, c0 = tc * kTC;
    const int tid = threadIdx.x;
    const bool vin = ((pitch & 3) == 0) &&
                     (((reinterpret_cast<uintptr_t>(pr) | reinterpret_cast<uintptr_t>(pg) |
                        reinterpret_cast<uintptr_t>(pb)) & 3) == 0);
    for (int k = tid; k < kSR * kSW; k += kThreads) {
        const int sr = k / kSW, sw = k - sr * kSW;
        const int64_t ro = (int64_t)min(max(r0 - kHalo + sr, 0), H - 1) * pitch;
        const int c = c0 - kHalo + 4 * sw;
        sI[sr][sw] = intensity4(load4_clamped(pr + ro, c, W, vin), load4_clamped(pg + ro, c, W, vin),
                                load4_clamped(pb + ro, c, W, vin));
    }
    __syncthreads();
    const int tx = tid & 31, ty = tid >> 5;
    const int c = c0 + 4 * tx;
    if (c >= W) return;
    const int nv = min(4, W - c);
    const bool vout = ((opitch & 3) == 0) &&
                      (((reinterpret_cast<uintptr_t>(out_i) | reinterpret_cast<uintptr_t>(out_hog) |
                         reinterpret_cast<uintptr_t>(out_rgb)) & 3) == 0);
    const int64_t plane = (int64_t)H * opitch;
    for (int rr = ty; rr < kTR; rr += kThreads / 32) {
        const int r = r0 + rr;
        if (r >= H) break;
        const int sr = rr + kHalo;
        const uint32_t L = sI[sr][tx], C = sI[sr][tx + 1], Rt = sI[sr][tx + 2];
        const int64_t o = (int64_t)r * opitch + c;
        store4(out_i + o, C, nv, vout);
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const int s = 1 << l;
            const uint32_t right = s == 1 ? __byte_perm(C, Rt, 0x4321) : s == 2 ? __byte_perm(C, Rt, 0x5432) : Rt;
            const uint32_t left = s == 1 ? __byte_perm(L, C, 0x6543) : s == 2 ? __byte_perm(L, C, 0x5432) : L;
            const uint32_t up = sI[sr - s][tx + 1], down = sI[sr + s][tx + 1];
            uint32_t bins = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int gx = byte_of(right, j) - byte_of(left, j);
                const int gy = byte_of(down, j) - byte_of(up, j);
                bins |= (uint32_t)orientation_bin9_table(gx, gy) << (8 * j);
            }
            store4(out_hog + l * plane + o, bins, nv, vout);
        }
        if (out_rgb) {
            const int64_t oi = (int64_t)r * pitch;
            store4(out_rgb + o, load4_clamped(pr + oi, c, W, vin), nv, vout);
            store4(out_rgb + plane + o, load4_clamped(pg + oi, c, W, vin), nv, vout);
            store4(out_rgb + 2 * plane + o, load4_clamped(pb + oi, c, W, vin), nv, vout);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 8) k_features(const uint8_t *__restrict__ pr, const uint8_t *__restrict__ pg,
                                                       const uint8_t *__restrict__ pb, int64_t pitch, int H, int W,
                                                       uint8_t *out_rgb, uint8_t *out_i, uint8_t *out_hog,
                                                       int64_t opitch)
{
    pdl_wait();
    features_tile(pr, pg, pb, pitch, H, W, out_rgb, out_i, out_hog, opitch, blockIdx.y, blockIdx.x);
}

// Batched: one CTA per (frame, tile), frames concatenated.
__global__ void __launch_bounds__(kThreads) k_features_b(const FeatJob *__restrict__ jobs,
                                                         const int64_t *__restrict__ pre, int n)
{
    pdl_wait();
    const int64_t flat = blockIdx.x;
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= flat)
            lo = mid;
        else
            hi = mid;
    }
    const FeatJob &jb = jobs[lo];
    const int local = (int)(flat - pre[lo]);
    const int tcols = (jb.W + kTC - 1) / kTC;
    features_tile(jb.r, jb.g, jb.b, jb.pitch, jb.H, jb.W, nullptr, jb.out_i, jb.out_hog, jb.opitch, local / tcols,
                  local % tcols);
}

}  // namespace

void prepare_features()
{
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64 || done[dev]) return;
    k_orient_table<<<256, 256>>>();
    if (cudaDeviceSynchronize() == cudaSuccess) done[dev] = true;
}

int launch_features(const uint8_t *r, const uint8_t *g, const uint8_t *b, int64_t pitch, int H,
                    int W, uint8_t *out_rgb, uint8_t *out_i, uint8_t *out_hog, int64_t out_pitch,
                    cudaStream_t st, const Prof *prof)
{
    dim3 grid((W + kTC - 1) / kTC, (H + kTR - 1) / kTR);
    prof_mark(prof, KID_FEATURES, 0, st);
    launch_pdl(k_features, grid, kThreads, 0, st, r, g, b, pitch, H, W, out_rgb, out_i, out_hog, out_pitch);
    prof_mark(prof, KID_FEATURES, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace ih

namespace ih {
int64_t feature_tiles(int H, int W) { return (int64_t)((H + kTR - 1) / kTR) * ((W + kTC - 1) / kTC); }

int launch_features_batch(const FeatJob *jobs, const int64_t *pre, int n, int64_t total, cudaStream_t st,
                          const Prof *prof)
{
    if (!total) return 0;
    prof_mark(prof, KID_FEATURES, 0, st);
    launch_pdl(k_features_b, (unsigned)total, kThreads, 0, st, jobs, pre, n);
    prof_mark(prof, KID_FEATURES, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}
}  // namespace ih
