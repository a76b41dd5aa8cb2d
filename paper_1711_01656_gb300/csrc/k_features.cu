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
// The unit vectors are scaled by 2^22 and rounded; for integer gradients in
// [-255,255]^2 the angle to the nearest boundary is > 1e-5 rad, so the sign
// of the cross product is exact: the rounding of the constants moves it by
// at most |gx|/2 + |gy|/2 <= |g|, while its true magnitude exceeds
// 2^22 * 1e-5 * |g| > 41 |g|.  Every term stays below 2^31 (4.2e6 * 255 +
// 4.2e6 * 255 < 2.1e9), so the test runs in int32.
//
// One CTA computes a 32 x 32 tile; it stages I for the tile plus a 4-pixel
// halo in shared memory, clamping coordinates when it loads, which gives the
// replicated borders.
#include "ih_internal.cuh"

namespace ih {

namespace {

constexpr int kT = 32, kHalo = 4, kS = kT + 2 * kHalo;

// round(2^22 cos(20j deg)), round(2^22 sin(20j deg)), j = 1..8
__constant__ int kUx[8] = {3941357, 3213023, 2097152, 728333, -728333, -2097152, -3213023, -3941357};
__constant__ int kUy[8] = {1434536, 2696047, 3632374, 4130583, 4130583, 3632374, 2696047, 1434536};

__device__ __forceinline__ int orientation_bin9(int gx, int gy)
{
    if (gy < 0 || (gy == 0 && gx < 0)) {
        gx = -gx;
        gy = -gy;
    }
    if ((gx | gy) == 0) return 0;
    int b = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) b += (kUx[k] * gy - kUy[k] * gx >= 0) ? 1 : 0;
    return b;
}

__device__ __forceinline__ void features_tile(const uint8_t *__restrict__ pr, const uint8_t *__restrict__ pg,
                                              const uint8_t *__restrict__ pb, int64_t pitch, int H, int W,
                                              uint8_t *out_rgb, uint8_t *out_i, uint8_t *out_hog, int64_t opitch,
                                              int tr, int tc)
{
    __shared__ uint8_t sI[kS][kS + 4];
    const int r0 = tr * kT, c0 = tc * kT;
    for (int sr = threadIdx.y; sr < kS; sr += blockDim.y) {
        const int64_t ro = (int64_t)min(max(r0 - kHalo + sr, 0), H - 1) * pitch;
        for (int sc = threadIdx.x; sc < kS; sc += blockDim.x) {
            const int64_t o = ro + min(max(c0 - kHalo + sc, 0), W - 1);
            sI[sr][sc] = (uint8_t)(((int)__ldg(pr + o) + (int)__ldg(pg + o) + (int)__ldg(pb + o)) / 3);
        }
    }
    __syncthreads();
    const int64_t plane = (int64_t)H * opitch;
    for (int rr = threadIdx.y; rr < kT; rr += blockDim.y) {
        const int r = r0 + rr, c = c0 + threadIdx.x;
        if (r >= H || c >= W) continue;
        const int sr = rr + kHalo, sc = threadIdx.x + kHalo;
        const int64_t o = (int64_t)r * opitch + c;
        out_i[o] = sI[sr][sc];
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const int s = 1 << l;
            // clamped neighbours: the halo already holds replicated borders,
            // but a neighbour past the frame edge must read the edge pixel
            const int cl = max(c - s, 0) - c0 + kHalo, cr = min(c + s, W - 1) - c0 + kHalo;
            const int ru = max(r - s, 0) - r0 + kHalo, rd = min(r + s, H - 1) - r0 + kHalo;
            const int gx = (int)sI[sr][cr] - (int)sI[sr][cl];
            const int gy = (int)sI[rd][sc] - (int)sI[ru][sc];
            out_hog[l * plane + o] = (uint8_t)orientation_bin9(gx, gy);
        }
        if (out_rgb) {
            const int64_t oi = (int64_t)r * pitch + c;
            out_rgb[o] = __ldg(pr + oi);
            out_rgb[plane + o] = __ldg(pg + oi);
            out_rgb[2 * plane + o] = __ldg(pb + oi);
        }
    }
}

__global__ void __launch_bounds__(256) k_features(const uint8_t *__restrict__ pr, const uint8_t *__restrict__ pg,
                                                  const uint8_t *__restrict__ pb, int64_t pitch, int H, int W,
                                                  uint8_t *out_rgb, uint8_t *out_i, uint8_t *out_hog, int64_t opitch)
{
    features_tile(pr, pg, pb, pitch, H, W, out_rgb, out_i, out_hog, opitch, blockIdx.y, blockIdx.x);
}

// Batched: one CTA per (frame, 32 x 32 tile), frames concatenated.
__global__ void __launch_bounds__(256) k_features_b(const FeatJob *__restrict__ jobs, const int64_t *__restrict__ pre,
                                                    int n)
{
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
    const int tcols = (jb.W + kT - 1) / kT;
    features_tile(jb.r, jb.g, jb.b, jb.pitch, jb.H, jb.W, nullptr, jb.out_i, jb.out_hog, jb.opitch, local / tcols,
                  local % tcols);
}

}  // namespace

int launch_features(const uint8_t *r, const uint8_t *g, const uint8_t *b, int64_t pitch, int H,
                    int W, uint8_t *out_rgb, uint8_t *out_i, uint8_t *out_hog, int64_t out_pitch,
                    cudaStream_t st, const Prof *prof)
{
    dim3 grid((W + kT - 1) / kT, (H + kT - 1) / kT);
    prof_mark(prof, KID_FEATURES, 0, st);
    k_features<<<grid, dim3(kT, 8), 0, st>>>(r, g, b, pitch, H, W, out_rgb, out_i, out_hog, out_pitch);
    prof_mark(prof, KID_FEATURES, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace ih

namespace ih {
int64_t feature_tiles(int H, int W) { return (int64_t)((H + kT - 1) / kT) * ((W + kT - 1) / kT); }

int launch_features_batch(const FeatJob *jobs, const int64_t *pre, int n, int64_t total, cudaStream_t st,
                          const Prof *prof)
{
    if (!total) return 0;
    prof_mark(prof, KID_FEATURES, 0, st);
    k_features_b<<<(unsigned)total, dim3(kT, 8), 0, st>>>(jobs, pre, n);
    prof_mark(prof, KID_FEATURES, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}
}  // namespace ih
