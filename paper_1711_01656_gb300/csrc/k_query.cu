// k_query.cu -- O(1) region queries on a built integral histogram.
//
// Rectangle histograms by the four-corner rule of Eq. 2.16 and spatially
// weighted local histograms (Eq. 3.1) from the moment planes of Eq. 3.4.
// Rectangles: one thread per (rectangle, bin group); weighted windows: one
// thread per (window, bin).
//
// Weighted histogram, Epanechnikov window kernel.  For window
// [r0,r1] x [c0,c1] with w = c1-c0+1, h = r1-r0+1, mc = c0+c1, mr = r0+r1:
//     k(r,c) = 1 - (2c-mc)^2 / (2w^2) - (2r-mr)^2 / (2h^2)
// so for bin b, with N, Sc, Sr, Scc, Srr the four-corner sums of the count
// plane and of the planes weighted by c, r, c^2, r^2:
//     X2 = sum (2c-mc)^2 = 4 Scc - 4 mc Sc + mc^2 N      (exact int64)
//     Y2 = sum (2r-mr)^2 = 4 Srr - 4 mr Sr + mr^2 N
//     S_b = N - X2/(2w^2) - Y2/(2h^2).
// The integer parts of the two quotients are taken exactly; the remaining
// fraction (< 2) is an exact uint64 ratio; S_b is then an integer plus one
// fraction in (0,1] and is rounded to float with at most a few roundings
// (relative error < 4e-7).  No step needs FP64.
// The window's total weight has the closed form
//     K = (4 w^2 h^2 + w^2 + h^2) / (6 w h),
// used by IH_NORMALIZE.
// The moment planes are stored as quads, [Bw][H][P][4]: the four moments
// (w = c, r, c^2, r^2) of a bin at one pixel are 32 contiguous bytes (16 with
// 32-bit moments), so a window corner costs one sector per bin.
#include "ih_internal.cuh"

namespace ih {

namespace {

__device__ __forceinline__ bool box_ok(int r0, int c0, int r1, int c1, int H, int W)
{
    return r0 >= 0 && c0 >= 0 && r0 <= r1 && c0 <= c1 && r1 < H && c1 < W;
}

// Address of H(b, r, c) in either count layout.
__device__ __forceinline__ const int32_t *count_ptr(const CountView &v, int b, int64_t r, int64_t c)
{
    if (v.layout == LAYOUT_BIN_MAJOR) return v.d + ((int64_t)b * v.H + r) * v.P + c;
    const int g = v.bin_group[b];
    return v.d + v.slab_off[g] + (r * v.P + c) * v.group_nb[g] + v.bin_local[b];
}

__device__ __forceinline__ long long four_corner(const int64_t *p, int64_t P, int r0, int c0, int r1, int c1)
{
    const long long a = __ldg(p + (int64_t)r1 * P + c1);
    const long long b = r0 > 0 ? (long long)__ldg(p + (int64_t)(r0 - 1) * P + c1) : 0;
    const long long c = c0 > 0 ? (long long)__ldg(p + (int64_t)r1 * P + (c0 - 1)) : 0;
    const long long d = (r0 > 0 && c0 > 0) ? (long long)__ldg(p + (int64_t)(r0 - 1) * P + (c0 - 1)) : 0;
    return a - b - c + d;
}

__device__ __forceinline__ uint32_t four_corner_u32(const uint32_t *p, int64_t P, int r0, int c0, int r1, int c1)
{
    const uint32_t a = __ldg(p + (int64_t)r1 * P + c1);
    const uint32_t b = r0 > 0 ? __ldg(p + (int64_t)(r0 - 1) * P + c1) : 0u;
    const uint32_t c = c0 > 0 ? __ldg(p + (int64_t)r1 * P + (c0 - 1)) : 0u;
    const uint32_t d = (r0 > 0 && c0 > 0) ? __ldg(p + (int64_t)(r0 - 1) * P + (c0 - 1)) : 0u;
    return a - b - c + d;
}

// LAYOUT_BIN_MAJOR: one thread per (rectangle, bin), item t = rect * B + bin:
// four independent loads, one store.
__device__ __forceinline__ void rect_item_bin(const CountView &v, const int32_t *__restrict__ rects,
                                              int32_t *__restrict__ out, int64_t t, int *err)
{
    const int64_t qi = t / v.B;
    const int b = (int)(t - qi * v.B);
    const int r0 = __ldg(rects + 4 * qi), c0 = __ldg(rects + 4 * qi + 1);
    const int r1 = __ldg(rects + 4 * qi + 2), c1 = __ldg(rects + 4 * qi + 3);
    if (!box_ok(r0, c0, r1, c1, v.H, v.W)) {
        out[t] = -1;
        if (b == 0) atomicOr(err, 1);
        return;
    }
    const int32_t *p = v.d + (int64_t)b * v.H * v.P;
    int32_t s = __ldg(p + (int64_t)r1 * v.P + c1);
    if (r0 > 0) s -= __ldg(p + (int64_t)(r0 - 1) * v.P + c1);
    if (c0 > 0) s -= __ldg(p + (int64_t)r1 * v.P + (c0 - 1));
    if (r0 > 0 && c0 > 0) s += __ldg(p + (int64_t)(r0 - 1) * v.P + (c0 - 1));
    out[t] = s;
}

// One thread per (rectangle, bin group): the group's bins of each corner
// are nb_g contiguous words in the slab layout.
template <typename TN>
__device__ __forceinline__ void rect_item(const CountView &v, const int64_t *g_off, const TN *g_nb, const TN *g_b0,
                                          const int32_t *__restrict__ rects, int32_t *__restrict__ out, int64_t t,
                                          int *err)
{
    const int ng = v.ngroups;
    const int64_t plane = (int64_t)v.H * v.P;
    const int64_t qi = t / ng;
    const int gi = (int)(t - qi * ng);
    const int nb = g_nb[gi], b0 = g_b0[gi];
    int32_t *o = out + qi * v.B + b0;
    const int r0 = __ldg(rects + 4 * qi), c0 = __ldg(rects + 4 * qi + 1);
    const int r1 = __ldg(rects + 4 * qi + 2), c1 = __ldg(rects + 4 * qi + 3);
    if (!box_ok(r0, c0, r1, c1, v.H, v.W)) {
        for (int b = 0; b < nb; ++b) o[b] = -1;
        if (gi == 0) atomicOr(err, 1);
        return;
    }
    // corner offsets (element index of bin 0 of the group) and strides
    const bool slab = v.layout == LAYOUT_SLAB;
    const int64_t base = slab ? g_off[gi] : (int64_t)b0 * plane;
    const int64_t px = slab ? nb : 1, bs = slab ? 1 : plane;
    const int64_t a = base + ((int64_t)r1 * v.P + c1) * px;
    const int64_t bq = base + ((int64_t)(r0 - 1) * v.P + c1) * px;
    const int64_t cq = base + ((int64_t)r1 * v.P + (c0 - 1)) * px;
    const int64_t dq = base + ((int64_t)(r0 - 1) * v.P + (c0 - 1)) * px;
    const bool top = r0 > 0, left = c0 > 0;
    if (slab && (nb & 3) == 0) {
        // nb a multiple of 4: each corner's record is nb/4 aligned int4s;
        // all loads are issued before the sums
        for (int b = 0; b < nb; b += 8) {
            const bool two = b + 4 < nb;
            int4 A0 = __ldg(reinterpret_cast<const int4 *>(v.d + a + b)), A1 = A0;
            int4 B0 = make_int4(0, 0, 0, 0), B1 = B0, C0 = B0, C1 = B0, D0 = B0, D1 = B0;
            if (two) A1 = __ldg(reinterpret_cast<const int4 *>(v.d + a + b + 4));
            if (top) {
                B0 = __ldg(reinterpret_cast<const int4 *>(v.d + bq + b));
                if (two) B1 = __ldg(reinterpret_cast<const int4 *>(v.d + bq + b + 4));
            }
            if (left) {
                C0 = __ldg(reinterpret_cast<const int4 *>(v.d + cq + b));
                if (two) C1 = __ldg(reinterpret_cast<const int4 *>(v.d + cq + b + 4));
            }
            if (top && left) {
                D0 = __ldg(reinterpret_cast<const int4 *>(v.d + dq + b));
                if (two) D1 = __ldg(reinterpret_cast<const int4 *>(v.d + dq + b + 4));
            }
            o[b + 0] = A0.x - B0.x - C0.x + D0.x;
            o[b + 1] = A0.y - B0.y - C0.y + D0.y;
            o[b + 2] = A0.z - B0.z - C0.z + D0.z;
            o[b + 3] = A0.w - B0.w - C0.w + D0.w;
            if (two) {
                o[b + 4] = A1.x - B1.x - C1.x + D1.x;
                o[b + 5] = A1.y - B1.y - C1.y + D1.y;
                o[b + 6] = A1.z - B1.z - C1.z + D1.z;
                o[b + 7] = A1.w - B1.w - C1.w + D1.w;
            }
        }
        return;
    }
#pragma unroll 8
    for (int b = 0; b < nb; ++b) {
        const int64_t ob = b * bs;
        int32_t s = __ldg(v.d + a + ob);
        if (top) s -= __ldg(v.d + bq + ob);
        if (left) s -= __ldg(v.d + cq + ob);
        if (top && left) s += __ldg(v.d + dq + ob);
        o[b] = s;
    }
}

// LAYOUT_RECORD: one thread per (rectangle, 4-word quarter of the pixel
// record).  Quarter k lies in plane qp[k] at word 4k - w0[plane]; the four
// corners are four aligned int4 loads, and consecutive threads read
// consecutive quarters of the same records.  wb[] maps record words to
// output bins (-1: padding).
__device__ __forceinline__ void rect_item_record(const CountView &v, const int64_t *off, const int16_t *rw,
                                                 const int16_t *w0, const int16_t *qp, const int16_t *wb,
                                                 const int32_t *__restrict__ rects, int32_t *__restrict__ out,
                                                 int64_t t, int *err)
{
    const int nq = v.nquarters;
    const int64_t qi = t / nq;
    const int k = (int)(t - qi * nq);
    int32_t *o = out + qi * v.B;
    const int r0 = __ldg(rects + 4 * qi), c0 = __ldg(rects + 4 * qi + 1);
    const int r1 = __ldg(rects + 4 * qi + 2), c1 = __ldg(rects + 4 * qi + 3);
    int sum[4] = {-1, -1, -1, -1};
    if (!box_ok(r0, c0, r1, c1, v.H, v.W)) {
        if (k == 0) atomicOr(err, 1);
    } else {
        const int p = qp[k];
        const int64_t w = rw[p];
        const int32_t *base = v.d + off[p] + (4 * k - w0[p]);
        const bool top = r0 > 0, left = c0 > 0;
        const int4 A = __ldg(reinterpret_cast<const int4 *>(base + ((int64_t)r1 * v.P + c1) * w));
        int4 B = make_int4(0, 0, 0, 0), C = B, D = B;
        if (top) B = __ldg(reinterpret_cast<const int4 *>(base + ((int64_t)(r0 - 1) * v.P + c1) * w));
        if (left) C = __ldg(reinterpret_cast<const int4 *>(base + ((int64_t)r1 * v.P + (c0 - 1)) * w));
        if (top && left) D = __ldg(reinterpret_cast<const int4 *>(base + ((int64_t)(r0 - 1) * v.P + (c0 - 1)) * w));
        sum[0] = A.x - B.x - C.x + D.x;
        sum[1] = A.y - B.y - C.y + D.y;
        sum[2] = A.z - B.z - C.z + D.z;
        sum[3] = A.w - B.w - C.w + D.w;
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int b = wb[4 * k + e];
        if (b >= 0) o[b] = sum[e];
    }
}

// The rectangle items of CTA bx of nbx (a grid-stride loop over the items).
// The group tables are copied to shared memory so that threads of different
// groups do not serialise on the kernel-parameter bank.
__device__ __forceinline__ void query_rects_cta(const CountView &v, const int32_t *__restrict__ rects, int64_t n,
                                                int32_t *__restrict__ out, int *err, unsigned bx, unsigned nbx)
{
    __shared__ int64_t s_off[kMaxGroups];
    __shared__ int s_nb[kMaxGroups], s_b0[kMaxGroups];
    __shared__ int16_t s_rw[kMaxGroups], s_w0[kMaxGroups], s_qp[kMaxBins / 4], s_wb[kMaxBins];
    for (int k = threadIdx.x; k < v.ngroups; k += blockDim.x) {
        s_off[k] = v.slab_off[k];
        s_nb[k] = v.group_nb[k];
        s_b0[k] = v.group_bin0[k];
        s_rw[k] = v.group_nb[k];
        s_w0[k] = v.plane_w0[k];
    }
    if (v.layout == LAYOUT_RECORD) {
        for (int k = threadIdx.x; k < v.nquarters; k += blockDim.x) s_qp[k] = v.quarter_plane[k];
        for (int k = threadIdx.x; k < 4 * v.nquarters; k += blockDim.x) s_wb[k] = v.word_bin[k];
    }
    __syncthreads();
    if (v.layout == LAYOUT_RECORD) {
        const int64_t total = n * v.nquarters;
        for (int64_t t = bx * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)nbx * blockDim.x)
            rect_item_record(v, s_off, s_rw, s_w0, s_qp, s_wb, rects, out, t, err);
        return;
    }
    if (v.layout == LAYOUT_BIN_MAJOR) {
        const int64_t total = n * v.B;
        for (int64_t t = bx * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)nbx * blockDim.x)
            rect_item_bin(v, rects, out, t, err);
        return;
    }
    const int64_t total = n * v.ngroups;
    for (int64_t t = bx * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)nbx * blockDim.x)
        rect_item(v, s_off, s_nb, s_b0, rects, out, t, err);
}

__global__ void __launch_bounds__(256) k_query_rects(const __grid_constant__ CountView v,
                                                     const int32_t *__restrict__ rects, int64_t n,
                                                     int32_t *__restrict__ out, int *err)
{
    pdl_wait();
    query_rects_cta(v, rects, n, out, err, blockIdx.x, gridDim.x);
}

// Largest f in [0, n) with pre[f] <= x.
__device__ __forceinline__ int find_job(const int64_t *pre, int n, int64_t x)
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

// Batched: work items of all frames concatenated; tables read from global.
// CTA bx of nbx runs a grid-stride loop over the items.
__device__ __forceinline__ void query_rects_b_cta(const QueryJob *__restrict__ jobs, const int64_t *__restrict__ pre,
                                                  int n, int *err, unsigned bx, unsigned nbx)
{
    const int64_t total = pre[n];
    for (int64_t t = bx * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)nbx * blockDim.x) {
        const int f = find_job(pre, n, t);
        const QueryJob &jb = jobs[f];
        const CountView &v = *jb.v;
        if (v.layout == LAYOUT_RECORD)
            rect_item_record(v, v.slab_off, v.group_nb, v.plane_w0, v.quarter_plane, v.word_bin, jb.rects,
                             jb.rect_out, t - pre[f], err);
        else if (v.layout == LAYOUT_BIN_MAJOR)
            rect_item_bin(v, jb.rects, jb.rect_out, t - pre[f], err);
        else
            rect_item(v, v.slab_off, v.group_nb, v.group_bin0, jb.rects, jb.rect_out, t - pre[f], err);
    }
}

__global__ void __launch_bounds__(256) k_query_rects_b(const QueryJob *__restrict__ jobs,
                                                       const int64_t *__restrict__ pre, int n, int *err)
{
    pdl_wait();
    query_rects_b_cta(jobs, pre, n, err, blockIdx.x, gridDim.x);
}

// Element offset of bin gb's count at (0, 0) and its per-pixel stride.
__device__ __forceinline__ void count_base(const CountView &v, int gb, int64_t &base, int64_t &px)
{
    if (v.layout != LAYOUT_BIN_MAJOR) {
        const int g = v.bin_group[gb];
        base = v.slab_off[g] + v.bin_local[gb];
        px = v.group_nb[g];
    } else {
        base = (int64_t)gb * v.H * v.P;
        px = 1;
    }
}

// The four moments (w = c, r, c^2, r^2) of one bin at (r, c): one quad, 32
// bytes (int64) or 16 bytes (uint32), so each corner of a window costs one
// sector per bin.
__device__ __forceinline__ void quad_at(const long long *q, int64_t P, int r, int c, long long (&o)[4])
{
    const longlong2 *p = reinterpret_cast<const longlong2 *>(q + ((int64_t)r * P + c) * 4);
    const longlong2 a = __ldg(p), b = __ldg(p + 1);
    o[0] = a.x;
    o[1] = a.y;
    o[2] = b.x;
    o[3] = b.y;
}

__device__ __forceinline__ uint4 quad_at_u32(const uint32_t *q, int64_t P, int r, int c)
{
    return __ldg(reinterpret_cast<const uint4 *>(q + ((int64_t)r * P + c) * 4));
}

// Four-corner differences of the four moments of a bin (Eq. 2.16 on Eq. 3.4's
// planes); q points at the bin's quads.
__device__ __forceinline__ void four_corner_quad(const long long *q, int64_t P, int r0, int c0, int r1, int c1,
                                                 long long (&S)[4])
{
    long long a[4];
    quad_at(q, P, r1, c1, a);
#pragma unroll
    for (int k = 0; k < 4; ++k) S[k] = a[k];
    if (r0 > 0) {
        quad_at(q, P, r0 - 1, c1, a);
#pragma unroll
        for (int k = 0; k < 4; ++k) S[k] -= a[k];
    }
    if (c0 > 0) {
        quad_at(q, P, r1, c0 - 1, a);
#pragma unroll
        for (int k = 0; k < 4; ++k) S[k] -= a[k];
    }
    if (r0 > 0 && c0 > 0) {
        quad_at(q, P, r0 - 1, c0 - 1, a);
#pragma unroll
        for (int k = 0; k < 4; ++k) S[k] += a[k];
    }
}

// The same modulo 2^32.
__device__ __forceinline__ uint4 four_corner_quad_u32(const uint32_t *q, int64_t P, int r0, int c0, int r1, int c1)
{
    uint4 s = quad_at_u32(q, P, r1, c1);
    auto sub = [&](uint4 a) { s.x -= a.x; s.y -= a.y; s.z -= a.z; s.w -= a.w; };
    auto add = [&](uint4 a) { s.x += a.x; s.y += a.y; s.z += a.z; s.w += a.w; };
    if (r0 > 0) sub(quad_at_u32(q, P, r0 - 1, c1));
    if (c0 > 0) sub(quad_at_u32(q, P, r1, c0 - 1));
    if (r0 > 0 && c0 > 0) add(quad_at_u32(q, P, r0 - 1, c0 - 1));
    return s;
}

__device__ __forceinline__ void weighted_item(const CountView &v, const MomentView &m, const int32_t *__restrict__ wins,
                                              int normalize, float *__restrict__ out, int64_t t, int *err)
{
    const int64_t plane = (int64_t)v.H * v.P;
    const int64_t qi = t / m.Bw;
    const int b = (int)(t - qi * m.Bw);
    const int r0 = __ldg(wins + 4 * qi), c0 = __ldg(wins + 4 * qi + 1);
    const int r1 = __ldg(wins + 4 * qi + 2), c1 = __ldg(wins + 4 * qi + 3);
    const int smax = m.m32 ? 256 : 32768;
    if (!box_ok(r0, c0, r1, c1, v.H, v.W) || r1 - r0 >= smax || c1 - c0 >= smax) {
        out[t] = -1.0f;
        if (b == 0) atomicOr(err, 1);
        return;
    }
    int64_t cbase, px;
    count_base(v, m.bin0 + b, cbase, px);
    const int32_t *cp = v.d + cbase;
    const long long N = (long long)__ldg(cp + ((int64_t)r1 * v.P + c1) * px) -
                        (r0 > 0 ? (long long)__ldg(cp + ((int64_t)(r0 - 1) * v.P + c1) * px) : 0) -
                        (c0 > 0 ? (long long)__ldg(cp + ((int64_t)r1 * v.P + (c0 - 1)) * px) : 0) +
                        ((r0 > 0 && c0 > 0) ? (long long)__ldg(cp + ((int64_t)(r0 - 1) * v.P + (c0 - 1)) * px) : 0);
    const int64_t mo = b * plane * 4;  // bin b's quads
    const long long w = c1 - c0 + 1, h = r1 - r0 + 1;
    const long long mc = c0 + c1, mr = r0 + r1;
    long long X2, Y2;
    if (m.m32) {
        // moments modulo 2^32: the centred sums X2, Y2 < 2^32 for sides <= 256,
        // so computing them modulo 2^32 gives them exactly
        const uint4 S = four_corner_quad_u32(reinterpret_cast<const uint32_t *>(m.m) + mo, v.P, r0, c0, r1, c1);
        const uint32_t n32 = (uint32_t)N, mc32 = (uint32_t)mc, mr32 = (uint32_t)mr;
        X2 = (long long)(uint32_t)(4u * S.z - 4u * mc32 * S.x + mc32 * mc32 * n32);
        Y2 = (long long)(uint32_t)(4u * S.w - 4u * mr32 * S.y + mr32 * mr32 * n32);
    } else {
        long long S[4];  // w = c, r, c^2, r^2
        four_corner_quad(reinterpret_cast<const long long *>(m.m) + mo, v.P, r0, c0, r1, c1, S);
        X2 = 4 * S[2] - 4 * mc * S[0] + mc * mc * N;
        Y2 = 4 * S[3] - 4 * mr * S[1] + mr * mr * N;
    }
    const long long A = 2 * w * w, Bh = 2 * h * h;
    const long long qx = X2 / A, rx = X2 - qx * A;
    const long long qy = Y2 / Bh, ry = Y2 - qy * Bh;
    long long I = N - qx - qy;
    unsigned long long F = (unsigned long long)rx * (unsigned long long)Bh +
                           (unsigned long long)ry * (unsigned long long)A;
    const unsigned long long Den = (unsigned long long)A * (unsigned long long)Bh;
    if (F >= Den) {
        I -= 1;
        F -= Den;
    }
    // S = I - F/Den, with S > 0 whenever N > 0, so I >= 1 when F > 0
    float s;
    if (F == 0)
        s = (float)I;
    else
        s = (float)(I - 1) + (float)(Den - F) / (float)Den;
    if (normalize) {
        const float K = (4.0f * (float)(w * w) * (float)(h * h) + (float)(w * w) + (float)(h * h)) /
                        (6.0f * (float)w * (float)h);
        s = s / K;
    }
    out[t] = s;
}

// Sums over a box on the 3 x 3 grid of corner points: P[i][j] holds the
// plane's prefix at (y[i], x[j]) (0 outside the frame), and the box between
// grid lines i..i+1 and j..j+1 is the four-corner difference.
template <typename T>
__device__ __forceinline__ T grid_box(const T (&P)[3][3], int i, int j)
{
    return P[i + 1][j + 1] - P[i][j + 1] - P[i + 1][j] + P[i][j];
}

template <typename T, typename L>
__device__ __forceinline__ void grid_load(T (&P)[3][3], const int (&y)[3], const int (&x)[3], L at)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) P[i][j] = (y[i] >= 0 && x[j] >= 0) ? at(y[i], x[j]) : T(0);
}

// The Manhattan kernel of Sec. 3.1.3 (Eq. 3.3) and the wedding-cake rings of
// Sec. 3.1.2 (Eq. 3.2), one thread per (window, bin).
//
// Manhattan: k(r,c) = (h + w) - |2r - Sr| - |2c - Sc|, Sr = r0 + r1,
// Sc = c0 + c1.  Split at rs = floor(Sr/2), cs = floor(Sc/2) into four
// quadrants (Fig. 3.4); in the quadrant with row sign er and column sign ec
// (-1: top/left, where |2r - Sr| = Sr - 2r) the weight is linear,
//   k = (h + w + er Sr + ec Sc) - 2 er r - 2 ec c,
// so its weighted sum is (h + w + er Sr + ec Sc) N - 2 er Sum r - 2 ec Sum c
// with N, Sum r, Sum c the quadrant's four-corner sums of the count plane and
// the r- and c-weighted moment planes (Eq. 3.4).  The 4 quadrants share a
// 3 x 3 grid of corner points (27 loads).  The sum is an exact integer
// (int64; modulo 2^32 with 32-bit planes, exact as it stays below 2^32 for
// sides <= 256); IH_NORMALIZE divides by
//   K = (h + w) h w - w floor(h^2/2) - h floor(w^2/2).
//
// Wedding cake, L layers: R_j = the window shrunk by floor(j h/(2L)) rows and
// floor(j w/(2L)) columns per side, ring j = R_j minus R_{j+1} weighs
// (h + w)(j + 1)/L, which telescopes to (h + w)/L times the sum of the L
// nested windows' plain counts.  IH_NORMALIZE divides by the same sum over a
// constant image, (h + w)/L times the sum of the windows' areas.
__device__ __forceinline__ void weighted_item_alt(const CountView &v, const MomentView &m,
                                                  const int32_t *__restrict__ wins, int kernel, int layers,
                                                  int normalize, float *__restrict__ out, int64_t t, int *err)
{
    const int64_t plane = (int64_t)v.H * v.P;
    const int64_t qi = t / m.Bw;
    const int b = (int)(t - qi * m.Bw);
    const int r0 = __ldg(wins + 4 * qi), c0 = __ldg(wins + 4 * qi + 1);
    const int r1 = __ldg(wins + 4 * qi + 2), c1 = __ldg(wins + 4 * qi + 3);
    const int smax = (kernel == IH_KERNEL_MANHATTAN && m.m32) ? 256 : 32768;
    if (!box_ok(r0, c0, r1, c1, v.H, v.W) || r1 - r0 >= smax || c1 - c0 >= smax) {
        out[t] = -1.0f;
        if (b == 0) atomicOr(err, 1);
        return;
    }
    int64_t cbase, px;
    count_base(v, m.bin0 + b, cbase, px);
    const int32_t *cp = v.d + cbase;
    const long long w = c1 - c0 + 1, h = r1 - r0 + 1;
    auto count_at = [&](int r, int c) -> long long { return __ldg(cp + ((int64_t)r * v.P + c) * px); };
    if (kernel == IH_KERNEL_MANHATTAN) {
        const long long Sr = r0 + r1, Sc = c0 + c1;
        const int y[3] = {r0 - 1, (r0 + r1) >> 1, r1}, x[3] = {c0 - 1, (c0 + c1) >> 1, c1};
        const int64_t mo = b * plane * 4;  // bin b's quads; w = c and w = r are their first two entries
        long long S;
        if (m.m32) {
            const uint32_t *m32 = reinterpret_cast<const uint32_t *>(m.m) + mo;
            uint32_t N[3][3], C[3][3], R[3][3];
            grid_load(N, y, x, [&](int r, int c) { return (uint32_t)count_at(r, c); });
            grid_load(C, y, x, [&](int r, int c) { return __ldg(m32 + ((int64_t)r * v.P + c) * 4); });
            grid_load(R, y, x, [&](int r, int c) { return __ldg(m32 + ((int64_t)r * v.P + c) * 4 + 1); });
            uint32_t s = 0;
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int er = i ? 1 : -1, ec = j ? 1 : -1;
                    s += (uint32_t)(h + w + er * Sr + ec * Sc) * grid_box(N, i, j) -
                         (uint32_t)(2 * er) * grid_box(R, i, j) - (uint32_t)(2 * ec) * grid_box(C, i, j);
                }
            S = (long long)s;
        } else {
            long long N[3][3], C[3][3], R[3][3];
            grid_load(N, y, x, count_at);
            const long long *mq = reinterpret_cast<const long long *>(m.m) + mo;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    longlong2 a = make_longlong2(0, 0);
                    if (y[i] >= 0 && x[j] >= 0)
                        a = __ldg(reinterpret_cast<const longlong2 *>(mq + ((int64_t)y[i] * v.P + x[j]) * 4));
                    C[i][j] = a.x;
                    R[i][j] = a.y;
                }
            S = 0;
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const long long er = i ? 1 : -1, ec = j ? 1 : -1;
                    S += (h + w + er * Sr + ec * Sc) * grid_box(N, i, j) - 2 * er * grid_box(R, i, j) -
                         2 * ec * grid_box(C, i, j);
                }
        }
        if (normalize) {
            const long long K = (h + w) * h * w - w * (h * h / 2) - h * (w * w / 2);
            out[t] = (float)S / (float)K;
        } else {
            out[t] = (float)S;
        }
        return;
    }
    // wedding cake
    long long S = 0, area = 0;
    for (int j = 0; j < layers; ++j) {
        const int dr = (int)(j * h / (2 * layers)), dc = (int)(j * w / (2 * layers));
        const int a0 = r0 + dr, b0 = c0 + dc, a1 = r1 - dr, b1 = c1 - dc;
        S += count_at(a1, b1) - (a0 > 0 ? count_at(a0 - 1, b1) : 0) - (b0 > 0 ? count_at(a1, b0 - 1) : 0) +
             ((a0 > 0 && b0 > 0) ? count_at(a0 - 1, b0 - 1) : 0);
        area += (long long)(a1 - a0 + 1) * (b1 - b0 + 1);
    }
    out[t] = normalize ? (float)S / (float)area : (float)((h + w) * S) / (float)layers;
}

template <int KERNEL>
__global__ void __launch_bounds__(256) k_query_weighted(const __grid_constant__ CountView v, const MomentView m,
                                                        const int32_t *__restrict__ wins, int64_t n, int layers,
                                                        int normalize, float *__restrict__ out, int *err)
{
    pdl_wait();
    const int64_t total = n * m.Bw;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (KERNEL == IH_KERNEL_EPANECHNIKOV)
            weighted_item(v, m, wins, normalize, out, t, err);
        else
            weighted_item_alt(v, m, wins, KERNEL, layers, normalize, out, t, err);
    }
}

// Both query kinds of one frame in one launch: the first wblocks CTAs run
// the weighted items (few CTAs, each bound by the latency of its scattered
// corner loads), the rest the rectangle items, so that the weighted CTAs
// overlap the rectangles' loads instead of running alone on a mostly idle
// GPU.
template <int KERNEL>
__global__ void __launch_bounds__(256) k_query_both(const __grid_constant__ CountView v, const MomentView m,
                                                    const int32_t *__restrict__ rects, int64_t nr,
                                                    int32_t *__restrict__ rout, const int32_t *__restrict__ wins,
                                                    int64_t nw, int layers, int normalize,
                                                    float *__restrict__ wout, unsigned wblocks, int *err)
{
    pdl_wait();
    if (blockIdx.x < wblocks) {
        const int64_t total = nw * m.Bw;
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
             t += (int64_t)wblocks * blockDim.x) {
            if (KERNEL == IH_KERNEL_EPANECHNIKOV)
                weighted_item(v, m, wins, normalize, wout, t, err);
            else
                weighted_item_alt(v, m, wins, KERNEL, layers, normalize, wout, t, err);
        }
        return;
    }
    query_rects_cta(v, rects, nr, rout, err, blockIdx.x - wblocks, gridDim.x - wblocks);
}

__device__ __forceinline__ void query_weighted_b_cta(const QueryJob *__restrict__ jobs,
                                                     const int64_t *__restrict__ pre, int n, int *err, unsigned bx,
                                                     unsigned nbx)
{
    const int64_t total = pre[n];
    for (int64_t t = bx * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)nbx * blockDim.x) {
        const int f = find_job(pre, n, t);
        const QueryJob &jb = jobs[f];
        if (jb.kernel == IH_KERNEL_EPANECHNIKOV)
            weighted_item(*jb.v, jb.m, jb.wins, jb.normalize, jb.wout, t - pre[f], err);
        else
            weighted_item_alt(*jb.v, jb.m, jb.wins, jb.kernel, jb.layers, jb.normalize, jb.wout, t - pre[f], err);
    }
}

__global__ void __launch_bounds__(256) k_query_weighted_b(const QueryJob *__restrict__ jobs,
                                                          const int64_t *__restrict__ pre, int n, int *err)
{
    pdl_wait();
    query_weighted_b_cta(jobs, pre, n, err, blockIdx.x, gridDim.x);
}

// Batched, both kinds in one launch: the first wblocks CTAs run the weighted
// items (as in k_query_both).
__global__ void __launch_bounds__(256) k_query_both_b(const QueryJob *__restrict__ jobs,
                                                      const int64_t *__restrict__ pre_rects,
                                                      const int64_t *__restrict__ pre_wins, int n, unsigned wblocks,
                                                      int *err)
{
    pdl_wait();
    if (blockIdx.x < wblocks)
        query_weighted_b_cta(jobs, pre_wins, n, err, blockIdx.x, wblocks);
    else
        query_rects_b_cta(jobs, pre_rects, n, err, blockIdx.x - wblocks, gridDim.x - wblocks);
}

// Sliding-window matching (Sec. 2.4.3, Eq. 2.22 with p = 1): one thread per
// placement; consecutive threads take consecutive columns, so each corner
// load of a bin is coalesced across the warp.  The bin tables and the target
// histogram sit in shared memory.
__global__ void __launch_bounds__(256) k_match_window(const __grid_constant__ CountView v, int bin0, int nbins,
                                                      const int32_t *__restrict__ target, int wh, int ww, int sr0,
                                                      int sc0, int sr1, int sc1, int32_t *__restrict__ out)
{
    pdl_wait();
    __shared__ int64_t s_base[kMaxBins];  // element offset of bin (bin0 + i) at pixel (0, 0)
    __shared__ int s_px[kMaxBins], s_t[kMaxBins];
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
        int64_t base, px;
        count_base(v, bin0 + i, base, px);
        s_base[i] = base;
        s_px[i] = (int)px;
        s_t[i] = __ldg(target + i);
    }
    __syncthreads();
    const int nc = sc1 - sc0 + 1;
    const int64_t total = (int64_t)(sr1 - sr0 + 1) * nc;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = sr0 + (int)(t / nc), c = sc0 + (int)(t % nc);
        const int r1 = r + wh - 1, c1 = c + ww - 1;
        const int64_t a = (int64_t)r1 * v.P + c1, bq = (int64_t)(r - 1) * v.P + c1;
        const int64_t cq = (int64_t)r1 * v.P + (c - 1), dq = (int64_t)(r - 1) * v.P + (c - 1);
        const bool top = r > 0, left = c > 0;
        int32_t d = 0;
        for (int i = 0; i < nbins; ++i) {
            const int32_t *p = v.d + s_base[i];
            const int64_t px = s_px[i];
            int32_t n = __ldg(p + a * px);
            if (top) n -= __ldg(p + bq * px);
            if (left) n -= __ldg(p + cq * px);
            if (top && left) n += __ldg(p + dq * px);
            const int32_t e = n - s_t[i];
            d += e < 0 ? -e : e;
        }
        out[t] = d;
    }
}

// Joint integral histogram update (Algorithm 4): dst += add - sub, 16 bytes
// per thread and step (the tensors are 16-byte aligned and a multiple of 4
// words long).
__global__ void __launch_bounds__(256) k_accumulate(int4 *__restrict__ dst, const int4 *__restrict__ add,
                                                    const int4 *__restrict__ sub, int64_t n4)
{
    pdl_wait();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        int4 d = dst[i];
        if (add) {
            const int4 a = __ldg(add + i);
            d.x += a.x, d.y += a.y, d.z += a.z, d.w += a.w;
        }
        if (sub) {
            const int4 b = __ldg(sub + i);
            d.x -= b.x, d.y -= b.y, d.z -= b.z, d.w -= b.w;
        }
        dst[i] = d;
    }
}

// Local median (Algorithm 4): one thread per pixel, consecutive threads on
// consecutive columns (coalesced corner loads).  A first pass over the bins
// gives the box total N, a second accumulates until ceil(N/2).
__global__ void __launch_bounds__(256) k_local_median(const __grid_constant__ CountView v, int bin0, int nbins,
                                                      int m, int n, int32_t *__restrict__ out)
{
    pdl_wait();
    __shared__ int64_t s_base[kMaxBins];
    __shared__ int s_px[kMaxBins];
    for (int i = threadIdx.x; i < nbins; i += blockDim.x) {
        int64_t base, px;
        count_base(v, bin0 + i, base, px);
        s_base[i] = base;
        s_px[i] = (int)px;
    }
    __syncthreads();
    const int64_t total = (int64_t)v.H * v.W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / v.W), c = (int)(t % v.W);
        const int ra = max(r - m / 2, 0), rb = min(r + (m + 1) / 2 - 1, v.H - 1);
        const int ca = max(c - n / 2, 0), cb = min(c + (n + 1) / 2 - 1, v.W - 1);
        const int64_t a = (int64_t)rb * v.P + cb, bq = (int64_t)(ra - 1) * v.P + cb;
        const int64_t cq = (int64_t)rb * v.P + (ca - 1), dq = (int64_t)(ra - 1) * v.P + (ca - 1);
        const bool top = ra > 0, left = ca > 0;
        auto box = [&](int i) -> int32_t {
            const int32_t *p = v.d + s_base[i];
            const int64_t px = s_px[i];
            int32_t x = __ldg(p + a * px);
            if (top) x -= __ldg(p + bq * px);
            if (left) x -= __ldg(p + cq * px);
            if (top && left) x += __ldg(p + dq * px);
            return x;
        };
        int64_t N = 0;
        for (int i = 0; i < nbins; ++i) N += box(i);
        int med = -1;
        if (N > 0) {
            const int64_t half = (N + 1) / 2;
            int64_t run = 0;
            for (int i = 0; i < nbins; ++i) {
                run += box(i);
                if (run >= half) {
                    med = i;
                    break;
                }
            }
        }
        out[t] = med;
    }
}

__global__ void __launch_bounds__(256) k_export(const __grid_constant__ CountView v, int32_t *__restrict__ dst)
{
    pdl_wait();
    const int64_t total = (int64_t)v.B * v.H * v.W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t % v.W, rb = t / v.W;
        const int64_t r = rb % v.H;
        const int b = (int)(rb / v.H);
        dst[t] = __ldg(count_ptr(v, b, r, c));
    }
}

__global__ void __launch_bounds__(256) k_export_moments(const void *__restrict__ m, int m32, int Bw, int H, int W,
                                                        int64_t P, int k, int64_t *__restrict__ dst)
{
    pdl_wait();
    const int64_t total = (int64_t)Bw * H * W;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t % W, rb = t / W;
        const int64_t o = (rb * P + c) * 4 + k;  // entry k of the quad of (bin, row) rb, column c
        dst[t] = m32 ? (int64_t)__ldg(static_cast<const uint32_t *>(m) + o) : __ldg(static_cast<const int64_t *>(m) + o);
    }
}

unsigned grid_for(int64_t total)
{
    const int64_t b = (total + 255) / 256;
    return (unsigned)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

}  // namespace

int launch_query_rects(const CountView &v, const int32_t *rects, int64_t n, int32_t *out, int *err,
                       cudaStream_t st, const Prof *prof)
{
    if (n == 0) return 0;
    prof_mark(prof, KID_QUERY_RECTS, 0, st);
    launch_pdl(k_query_rects, grid_for(n * rect_items(v)), 256, 0, st, v, rects, n, out, err);
    prof_mark(prof, KID_QUERY_RECTS, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_query_weighted(const CountView &v, const MomentView &m, const int32_t *wins, int64_t n, int kernel,
                          int layers, int normalize, float *out, int *err, cudaStream_t st, const Prof *prof)
{
    if (n == 0) return 0;
    prof_mark(prof, KID_QUERY_WEIGHTED, 0, st);
    const unsigned blocks = grid_for(n * m.Bw);
    if (kernel == IH_KERNEL_MANHATTAN)
        launch_pdl(k_query_weighted<IH_KERNEL_MANHATTAN>, blocks, 256, 0, st, v, m, wins, n, layers, normalize, out, err);
    else if (kernel == IH_KERNEL_WEDDING_CAKE)
        launch_pdl(k_query_weighted<IH_KERNEL_WEDDING_CAKE>, blocks, 256, 0, st, v, m, wins, n, layers, normalize, out, err);
    else
        launch_pdl(k_query_weighted<IH_KERNEL_EPANECHNIKOV>, blocks, 256, 0, st, v, m, wins, n, layers, normalize, out, err);
    prof_mark(prof, KID_QUERY_WEIGHTED, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_query_both(const CountView &v, const MomentView &m, const int32_t *rects, int64_t nr, int32_t *rout,
                      const int32_t *wins, int64_t nw, int kernel, int layers, int normalize, float *wout, int *err,
                      cudaStream_t st, const Prof *prof)
{
    if (nw == 0) return launch_query_rects(v, rects, nr, rout, err, st, prof);
    if (nr == 0)
        return launch_query_weighted(v, m, wins, nw, kernel, layers, normalize, wout, err, st, prof);
    const unsigned wb = grid_for(nw * m.Bw), rb = grid_for(nr * rect_items(v));
    prof_mark(prof, KID_QUERY_BOTH, 0, st);
    if (kernel == IH_KERNEL_MANHATTAN)
        launch_pdl(k_query_both<IH_KERNEL_MANHATTAN>, wb + rb, 256, 0, st, v, m, rects, nr, rout, wins, nw, layers,
                   normalize, wout, wb, err);
    else if (kernel == IH_KERNEL_WEDDING_CAKE)
        launch_pdl(k_query_both<IH_KERNEL_WEDDING_CAKE>, wb + rb, 256, 0, st, v, m, rects, nr, rout, wins, nw, layers,
                   normalize, wout, wb, err);
    else
        launch_pdl(k_query_both<IH_KERNEL_EPANECHNIKOV>, wb + rb, 256, 0, st, v, m, rects, nr, rout, wins, nw, layers,
                   normalize, wout, wb, err);
    prof_mark(prof, KID_QUERY_BOTH, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_queries_batch(const QueryJob *jobs, const int64_t *pre_rects, const int64_t *pre_wins, int n,
                         int64_t total_rects, int64_t total_wins, int *err, cudaStream_t st, const Prof *prof)
{
    int k = 0;
    if (total_rects && total_wins) {
        const unsigned wb = grid_for(total_wins);
        prof_mark(prof, KID_QUERY_BOTH, 0, st);
        launch_pdl(k_query_both_b, wb + grid_for(total_rects), 256, 0, st, jobs, pre_rects, pre_wins, n, wb, err);
        prof_mark(prof, KID_QUERY_BOTH, 1, st);
        return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
    }
    if (total_rects) {
        prof_mark(prof, KID_QUERY_RECTS, 0, st);
        launch_pdl(k_query_rects_b, grid_for(total_rects), 256, 0, st, jobs, pre_rects, n, err);
        prof_mark(prof, KID_QUERY_RECTS, 1, st);
        ++k;
    }
    if (total_wins) {
        prof_mark(prof, KID_QUERY_WEIGHTED, 0, st);
        launch_pdl(k_query_weighted_b, grid_for(total_wins), 256, 0, st, jobs, pre_wins, n, err);
        prof_mark(prof, KID_QUERY_WEIGHTED, 1, st);
        ++k;
    }
    return cudaPeekAtLastError() == cudaSuccess ? k : -1;
}

int launch_export_moments(const void *m, int m32, int Bw, int H, int W, int64_t P, int k, int64_t *dst,
                          cudaStream_t st, const Prof *prof)
{
    prof_mark(prof, KID_EXPORT, 0, st);
    launch_pdl(k_export_moments, grid_for((int64_t)Bw * H * W), 256, 0, st, m, m32, Bw, H, W, P, k, dst);
    prof_mark(prof, KID_EXPORT, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_match_window(const CountView &v, int bin0, int nbins, const int32_t *target, int wh, int ww, int sr0,
                        int sc0, int sr1, int sc1, int32_t *out, cudaStream_t st, const Prof *prof)
{
    const int64_t total = (int64_t)(sr1 - sr0 + 1) * (sc1 - sc0 + 1);
    prof_mark(prof, KID_MATCH, 0, st);
    launch_pdl(k_match_window, grid_for(total), 256, 0, st, v, bin0, nbins, target, wh, ww, sr0, sc0, sr1, sc1, out);
    prof_mark(prof, KID_MATCH, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_accumulate(int32_t *dst, const int32_t *add, const int32_t *sub, int64_t n, cudaStream_t st,
                      const Prof *prof)
{
    const int64_t n4 = n / 4;
    prof_mark(prof, KID_ACCUMULATE, 0, st);
    launch_pdl(k_accumulate, grid_for(n4), 256, 0, st, reinterpret_cast<int4 *>(dst), reinterpret_cast<const int4 *>(add),
                                               reinterpret_cast<const int4 *>(sub), n4);
    prof_mark(prof, KID_ACCUMULATE, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_local_median(const CountView &v, int bin0, int nbins, int m, int n, int32_t *out, cudaStream_t st,
                        const Prof *prof)
{
    prof_mark(prof, KID_MEDIAN, 0, st);
    launch_pdl(k_local_median, grid_for((int64_t)v.H * v.W), 256, 0, st, v, bin0, nbins, m, n, out);
    prof_mark(prof, KID_MEDIAN, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

int launch_export(const CountView &v, int32_t *dst, cudaStream_t st, const Prof *prof)
{
    prof_mark(prof, KID_EXPORT, 0, st);
    launch_pdl(k_export, grid_for((int64_t)v.B * v.H * v.W), 256, 0, st, v, dst);
    prof_mark(prof, KID_EXPORT, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace ih
