/*
 * ih_oracle.c -- plain, slow, obviously-correct CPU oracle for the
 * integral-histogram path of Poostchi (2017), arXiv 1711.01656.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the test suite, the smoke check of __graft_entry__ and
 * the cpu_baseline / reference leg of bench.py use it.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Every routine below follows one passage of the thesis, in its order and
 * notation, with no blocking, fusion or reordering:
 *   - binning function Q                         Eq. 2.15 (and Eq. 3.1's Q(f))
 *   - integral histogram by the sequential
 *     recurrence H(k,x,y)=H(k,x-1,y)+H(k,x,y-1)
 *                 -H(k,x-1,y-1)+Q(k,I(x,y))       Algorithm 5, Sec. 5 intro
 *   - weighted integral histogram IH_w            Eq. 3.4 (same recurrence,
 *                                                 the increment times w)
 *   - rectangle histogram by enumeration of the
 *     region's pixels                             Eq. 2.15 + Eq. 2.16 (definition)
 *   - spatially weighted local histogram by
 *     direct summation (the brute force)          Eq. 3.1, Sec. 3.1.1
 *     with the Manhattan kernel                   Eq. 3.3, Sec. 3.1.3
 *     or the wedding-cake rings                   Eq. 3.2, Sec. 3.1.2
 *   - sliding-window histogram matching by the
 *     city-block distance of every placement      Eq. 2.22 (p = 1), Sec. 2.4.3
 *   - spatio-temporal median by sorting the box's
 *     quantised values over the frames             Algorithm 4, Sec. 4.1.1
 *   - Canny edges (smoothing, non-maximum
 *     suppression, hysteresis), magnitude-weighted
 *     orientation planes, their integral histogram,
 *     pyramid descriptors by pixel sums and the
 *     pyramid match kernel                         Algorithm 2, Eq. 2.23-2.24
 *   - feature channels: intensity I=(R+G+B)/3     Eq. 2.33
 *     and gradient orientation tan^-1(Iy/Ix)      Fig. 2.3, Algorithm 2
 *
 * Readings where the thesis is silent:
 *   - uniform binning of 8-bit values into B bins over [0,256):
 *     Q(v) = floor(v*B/256); "index" channels carry the bin itself and a
 *     value >= B belongs to no bin;
 *   - the integral histogram is inclusive (Eq. 2.15, Alg. 5), 0-based,
 *     r = row (the thesis's x), c = column (the thesis's y);
 *   - a rectangle is inclusive [r0,r1] x [c0,c1]; an invalid one (outside
 *     the frame or r0>r1 / c0>c1) yields a row of -1;
 *   - the spatial kernel of Eq. 3.1 is an Epanechnikov profile whose
 *     ellipse passes through the window's outer corners:
 *       k(r,c) = 1 - (2c-(c0+c1))^2/(2w^2) - (2r-(r0+r1))^2/(2h^2),
 *     w = c1-c0+1, h = r1-r0+1 (every pixel centre has k > 0);
 *   - the Manhattan kernel is h + w minus the city-block distance from the
 *     window centre in doubled coordinates (the thesis leaves the scale and
 *     the normalisation open); the wedding-cake windows shrink by
 *     floor(j*h/(2L)), floor(j*w/(2L)) per side and ring j weighs
 *     (h + w)(j + 1)/L (the thesis leaves the ring sizes and weights open);
 *   - the median of Algorithm 4 is the lower median bin of the box's
 *     quantised values, the box clipped at the frame border (the thesis
 *     leaves both open);
 *   - Algorithm 2's Canny step follows Canny (1986) in integers: 5 x 5
 *     binomial smoothing, central-difference gradient, non-maximum
 *     suppression in four exact direction sectors (ties broken towards the
 *     lower column / upper row), double threshold on |G| (lo, hi) and
 *     hysteresis over 8-connected survivors; step 2's gradient is the
 *     window's own (unsmoothed) central difference, its magnitude kept in
 *     fixed point (floor(16 |g|)); the pyramid cells are floor(h/2^l) x
 *     floor(w/2^l) at multiples of that size, and its garbled index
 *     updates are read as visiting the s x s cells once each;
 *   - intensity rounds down; gradient orientation is unsigned, in
 *     [0,180) degrees, 9 bins of 20 degrees, central differences at step
 *     s with replicated borders, (0,0) -> bin 0.
 *
 * Floating point is FP64 throughout; counts are exact integers (int64
 * accumulation, checked to fit int32 where the output is int32).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_BIN_UNIFORM8 0
#define OR_BIN_INDEX 1

/* weight functions w(r,c) of Eq. 3.4 used for moment planes */
#define OR_W_ONE 0
#define OR_W_COL 1    /* w = c   */
#define OR_W_ROW 2    /* w = r   */
#define OR_W_COL2 3   /* w = c^2 */
#define OR_W_ROW2 4   /* w = r^2 */

/* Eq. 2.15: Q(I(r,c), b) is 1 iff the pixel value falls in bin b.  Returns
 * the bin the value falls in, or -1 if it falls in none. */
int oracle_bin_of(int v, int B, int mode)
{
    if (mode == OR_BIN_UNIFORM8) {
        /* B equal-width bins over [0,256): bin b holds [256b/B, 256(b+1)/B) */
        return (v * B) / 256;
    }
    return (v >= 0 && v < B) ? v : -1;
}

static int64_t weight_of(int w, int64_t r, int64_t c)
{
    switch (w) {
    case OR_W_ONE: return 1;
    case OR_W_COL: return c;
    case OR_W_ROW: return r;
    case OR_W_COL2: return c * c;
    case OR_W_ROW2: return r * r;
    }
    return 0;
}

/* Algorithm 5 with the increment Q(k, I(x,y)) replaced by
 * Q(k, I(x,y)) * w(x,y): this is Eq. 3.4's weighted integral histogram, and
 * with w = 1 exactly Algorithm 5.  Output is bin-major b x h x w (Fig. 5.1),
 * packed. H(k,-1,.) = H(k,.,-1) = 0. */
static void alg5_weighted(const uint8_t *img, int64_t pitch, int h, int w,
                          int b, int mode, int wk, int64_t *out, int k_lo,
                          int k_hi)
{
    for (int k = k_lo; k < k_hi; k++) {
        int64_t *Hk = out + (int64_t)k * h * w;
        for (int x = 0; x < h; x++) {
            for (int y = 0; y < w; y++) {
                int64_t up = x > 0 ? Hk[(int64_t)(x - 1) * w + y] : 0;
                int64_t left = y > 0 ? Hk[(int64_t)x * w + (y - 1)] : 0;
                int64_t diag = (x > 0 && y > 0) ? Hk[(int64_t)(x - 1) * w + (y - 1)] : 0;
                int q = oracle_bin_of(img[(int64_t)x * pitch + y], b, mode) == k;
                Hk[(int64_t)x * w + y] = up + left - diag + (q ? weight_of(wk, x, y) : 0);
            }
        }
    }
}

typedef struct {
    const uint8_t *img;
    int64_t pitch;
    int h, w, b, mode, wk;
    int64_t *out;
    int k_lo, k_hi;
} alg5_job;

static void *alg5_thread(void *p)
{
    alg5_job *j = (alg5_job *)p;
    alg5_weighted(j->img, j->pitch, j->h, j->w, j->b, j->mode, j->wk, j->out,
                  j->k_lo, j->k_hi);
    return NULL;
}

/* Algorithm 5 / Eq. 3.4 for bins [0,b), split over `threads` host threads by
 * bin (the bins are independent, Sec. 5.1.2).  out: int64 b x h x w. */
int oracle_weighted_ih(const uint8_t *img, int64_t pitch, int h, int w, int b,
                       int mode, int wk, int64_t *out, int threads)
{
    if (h < 0 || w < 0 || b < 1 || pitch < w) return -1;
    if (threads < 1) threads = 1;
    if (threads > b) threads = b;
    if (threads == 1) {
        alg5_weighted(img, pitch, h, w, b, mode, wk, out, 0, b);
        return 0;
    }
    pthread_t *tid = (pthread_t *)malloc(sizeof(pthread_t) * threads);
    alg5_job *jobs = (alg5_job *)malloc(sizeof(alg5_job) * threads);
    for (int t = 0; t < threads; t++) {
        alg5_job j = {img, pitch, h, w, b, mode, wk, out, b * t / threads,
                      b * (t + 1) / threads};
        jobs[t] = j;
        pthread_create(&tid[t], NULL, alg5_thread, &jobs[t]);
    }
    for (int t = 0; t < threads; t++) pthread_join(tid[t], NULL);
    free(tid);
    free(jobs);
    return 0;
}

/* Algorithm 5 proper: int32 integral histogram b x h x w.  Accumulates in
 * int64 and returns 1 if any cell does not fit int32 (never for h*w < 2^31). */
int oracle_ih(const uint8_t *img, int64_t pitch, int h, int w, int b, int mode,
              int32_t *out, int threads)
{
    int64_t n = (int64_t)b * h * w;
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    if (!tmp) return -2;
    int rc = oracle_weighted_ih(img, pitch, h, w, b, mode, OR_W_ONE, tmp, threads);
    if (rc == 0) {
        for (int64_t i = 0; i < n; i++) {
            if (tmp[i] > INT32_MAX) rc = 1;
            out[i] = (int32_t)tmp[i];
        }
    }
    free(tmp);
    return rc;
}

static int rect_valid(int h, int w, const int32_t *q)
{
    return q[0] >= 0 && q[1] >= 0 && q[0] <= q[2] && q[1] <= q[3] && q[2] < h &&
           q[3] < w;
}

/* Histogram of rectangle R = [r0,r1] x [c0,c1] (inclusive) by enumerating
 * its pixels: the quantity Eq. 2.16 evaluates from four corners, taken here
 * from its definition (Eq. 2.15 summed over R).  rects: n x 4 (r0,c0,r1,c1);
 * out: n x b int32.  Returns the number of invalid rectangles (row of -1). */
int64_t oracle_rect_hist(const uint8_t *img, int64_t pitch, int h, int w, int b,
                         int mode, const int32_t *rects, int64_t n,
                         int32_t *out)
{
    int64_t bad = 0;
    for (int64_t i = 0; i < n; i++) {
        const int32_t *q = rects + 4 * i;
        int32_t *o = out + i * b;
        if (!rect_valid(h, w, q)) {
            for (int k = 0; k < b; k++) o[k] = -1;
            bad++;
            continue;
        }
        for (int k = 0; k < b; k++) o[k] = 0;
        for (int r = q[0]; r <= q[2]; r++)
            for (int c = q[1]; c <= q[3]; c++) {
                int k = oracle_bin_of(img[(int64_t)r * pitch + c], b, mode);
                if (k >= 0) o[k]++;
            }
    }
    return bad;
}

/* Sliding-window histogram matching (Sec. 2.4.3): for every placement of a
 * wh x ww window whose top-left pixel (r, c) lies in [sr0, sr1] x
 * [sc0, sc1], the city-block distance of Eq. 2.22 (p = 1),
 *   sum_i |H_window(i) - target(i)|,
 * with the window histogram counted pixel by pixel.  out: row-major
 * (sr1-sr0+1) x (sc1-sc0+1) int64.  Returns -1 if a placement leaves the
 * image, else 0. */
int64_t oracle_match_window(const uint8_t *img, int64_t pitch, int h, int w, int b, int mode,
                            const int32_t *target, int wh, int ww, int sr0, int sc0, int sr1,
                            int sc1, int64_t *out)
{
    if (sr0 < 0 || sc0 < 0 || sr1 < sr0 || sc1 < sc0 || sr1 + wh > h || sc1 + ww > w || wh < 1 || ww < 1)
        return -1;
    int64_t *hist = (int64_t *)malloc(sizeof(int64_t) * (size_t)b);
    int64_t k = 0;
    for (int r = sr0; r <= sr1; r++)
        for (int c = sc0; c <= sc1; c++) {
            for (int i = 0; i < b; i++) hist[i] = 0;
            for (int y = r; y < r + wh; y++)
                for (int x = c; x < c + ww; x++) {
                    int i = oracle_bin_of(img[(int64_t)y * pitch + x], b, mode);
                    if (i >= 0) hist[i]++;
                }
            int64_t d = 0;
            for (int i = 0; i < b; i++) d += hist[i] > target[i] ? hist[i] - target[i] : target[i] - hist[i];
            out[k++] = d;
        }
    free(hist);
    return 0;
}

static int cmp_int(const void *a, const void *b)
{
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* Spatio-temporal median (Sec. 4.1.1, Algorithm 4): for every pixel (r, c),
 * the quantised values of the nf frames (`frames`: nf planes of h x w) over
 * the m x n box of rows r - floor(m/2) .. r + ceil(m/2) - 1 and columns
 * c - floor(n/2) .. c + ceil(n/2) - 1, clipped to the frame, are sorted and
 * the element of rank ceil(N/2) (the lower median of the N values) is the
 * pixel's median bin; a value that falls in no bin is left out.  out: h x w
 * int32, -1 where the box holds no binned value. */
void oracle_local_median(const uint8_t *frames, int nf, int h, int w, int b, int mode, int m, int n,
                         int32_t *out)
{
    int *vals = (int *)malloc(sizeof(int) * (size_t)nf * m * n);
    for (int r = 0; r < h; r++)
        for (int c = 0; c < w; c++) {
            int cnt = 0;
            for (int f = 0; f < nf; f++)
                for (int y = r - m / 2; y <= r + (m + 1) / 2 - 1; y++)
                    for (int x = c - n / 2; x <= c + (n + 1) / 2 - 1; x++) {
                        if (y < 0 || y >= h || x < 0 || x >= w) continue;
                        int k = oracle_bin_of(frames[((int64_t)f * h + y) * w + x], b, mode);
                        if (k >= 0) vals[cnt++] = k;
                    }
            if (cnt == 0) {
                out[(int64_t)r * w + c] = -1;
                continue;
            }
            qsort(vals, (size_t)cnt, sizeof(int), cmp_int);
            out[(int64_t)r * w + c] = vals[(cnt + 1) / 2 - 1];
        }
    free(vals);
}

/* The spatial kernel of Eq. 3.1 for window [r0,r1] x [c0,c1] (Epanechnikov
 * profile through the window's outer corners), in FP64. */
double oracle_kernel_weight(const int32_t *q, int r, int c)
{
    double wdt = (double)(q[3] - q[1] + 1), hgt = (double)(q[2] - q[0] + 1);
    double dc = 2.0 * c - (double)(q[1] + q[3]);
    double dr = 2.0 * r - (double)(q[0] + q[2]);
    return 1.0 - dc * dc / (2.0 * wdt * wdt) - dr * dr / (2.0 * hgt * hgt);
}

/* The Manhattan (city-block) kernel of Sec. 3.1.3: Eq. 3.3's distance
 * |x_i - x_c| + |y_i - y_c| from the window centre, taken in doubled
 * coordinates so that the centre of an even side is exact, subtracted from
 * h + w (more than the largest doubled distance, h - 1 + w - 1), so weights
 * fall linearly from the centre to the border and stay >= 2. */
double oracle_manhattan_weight(const int32_t *q, int r, int c)
{
    int wdt = q[3] - q[1] + 1, hgt = q[2] - q[0] + 1;
    int dr = 2 * r - (q[0] + q[2]), dc = 2 * c - (q[1] + q[3]);
    return (double)(hgt + wdt - abs(dr) - abs(dc));
}

/* The wedding-cake approximation of Sec. 3.1.2 (Eq. 3.2): `layers` nested
 * windows R_0 = T, R_j = T shrunk by floor(j*h/(2*layers)) rows and
 * floor(j*w/(2*layers)) columns on each side; a pixel of the ring
 * R_j \ R_{j+1} (R_layers empty) gets w_j = (h + w)(j + 1)/layers, a
 * staircase under the Manhattan pyramid above. */
double oracle_wedding_weight(const int32_t *q, int layers, int r, int c)
{
    int wdt = q[3] - q[1] + 1, hgt = q[2] - q[0] + 1;
    int ring = -1;
    for (int j = 0; j < layers; j++) {
        int dr = j * hgt / (2 * layers), dc = j * wdt / (2 * layers);
        if (r >= q[0] + dr && r <= q[2] - dr && c >= q[1] + dc && c <= q[3] - dc) ring = j;
    }
    return ring < 0 ? 0.0 : (double)(hgt + wdt) * (ring + 1) / layers;
}

/* Eq. 3.1 by direct summation (the brute force of Sec. 3.1.1):
 *   H(T, b_i) = sum_{(x,y) in T} delta(Q(f(x,y)) - b_i) * w(x,y)
 * in FP64, with w the Epanechnikov kernel (kernel 0), the Manhattan kernel
 * (1) or the wedding-cake rings (2, `layers` nested windows).  normalize != 0
 * divides every bin by sum_{T} w(x,y), the normalisation step of the SWIH
 * flow (Ch. 3 introduction).  out: n x b double; an invalid window yields a
 * row of -1.  Returns #invalid. */
int64_t oracle_weighted_hist_k(const uint8_t *img, int64_t pitch, int h, int w,
                               int b, int mode, const int32_t *wins, int64_t n,
                               int kernel, int layers, int normalize, double *out)
{
    int64_t bad = 0;
    for (int64_t i = 0; i < n; i++) {
        const int32_t *q = wins + 4 * i;
        double *o = out + i * b;
        if (!rect_valid(h, w, q)) {
            for (int k = 0; k < b; k++) o[k] = -1.0;
            bad++;
            continue;
        }
        double wsum = 0.0;
        for (int k = 0; k < b; k++) o[k] = 0.0;
        for (int r = q[0]; r <= q[2]; r++)
            for (int c = q[1]; c <= q[3]; c++) {
                double wt = kernel == 1 ? oracle_manhattan_weight(q, r, c)
                          : kernel == 2 ? oracle_wedding_weight(q, layers, r, c)
                                        : oracle_kernel_weight(q, r, c);
                int k = oracle_bin_of(img[(int64_t)r * pitch + c], b, mode);
                if (k >= 0) o[k] += wt;
                wsum += wt;
            }
        if (normalize)
            for (int k = 0; k < b; k++) o[k] /= wsum;
    }
    return bad;
}

int64_t oracle_weighted_hist(const uint8_t *img, int64_t pitch, int h, int w,
                             int b, int mode, const int32_t *wins, int64_t n,
                             int normalize, double *out)
{
    return oracle_weighted_hist_k(img, pitch, h, w, b, mode, wins, n, 0, 0, normalize, out);
}

/* Gradient orientation bin (Fig. 2.3, Algorithm 2): unsigned
 * orientation theta = atan2(gy, gx) folded into [0, pi), quantised into nb
 * equal bins; (0,0) -> bin 0.  FP64. */
int oracle_orientation_bin(int gx, int gy, int nb)
{
    if (gy < 0 || (gy == 0 && gx < 0)) {
        gx = -gx;
        gy = -gy;
    }
    if (gx == 0 && gy == 0) return 0;
    double th = atan2((double)gy, (double)gx); /* in [0, pi) after the fold */
    int k = (int)floor(th / (M_PI / nb));
    if (k >= nb) k = nb - 1;
    if (k < 0) k = 0;
    return k;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* The 7 feature channels of the tracker's descriptor set: R, G, B, intensity
 * I = (R+G+B)/3 (Eq. 2.33) and three gradient-orientation index planes of I
 * at central-difference steps s = 1, 2, 4 (9 bins).  rgb: 3 planes of h x w;
 * out: 7 planes of h x w (uint8), packed. */
void oracle_features(const uint8_t *rgb, int h, int w, uint8_t *out)
{
    int64_t n = (int64_t)h * w;
    const uint8_t *R = rgb, *G = rgb + n, *B = rgb + 2 * n;
    uint8_t *I = out + 3 * n;
    memcpy(out, rgb, (size_t)(3 * n));
    for (int64_t i = 0; i < n; i++) I[i] = (uint8_t)(((int)R[i] + G[i] + B[i]) / 3);
    const int steps[3] = {1, 2, 4};
    for (int l = 0; l < 3; l++) {
        int s = steps[l];
        uint8_t *O = out + (4 + l) * n;
        for (int r = 0; r < h; r++)
            for (int c = 0; c < w; c++) {
                int gx = (int)I[(int64_t)r * w + clampi(c + s, 0, w - 1)] -
                         (int)I[(int64_t)r * w + clampi(c - s, 0, w - 1)];
                int gy = (int)I[(int64_t)clampi(r + s, 0, h - 1) * w + c] -
                         (int)I[(int64_t)clampi(r - s, 0, h - 1) * w + c];
                O[(int64_t)r * w + c] = (uint8_t)oracle_orientation_bin(gx, gy, 9);
            }
    }
}

/* ---- spatial pyramid of gradient orientations (Algorithm 2, Sec. 2.4.4) */

/* floor(sqrt(n)) of a non-negative integer by bisection. */
int64_t oracle_isqrt(int64_t n)
{
    int64_t lo = 0, hi = 1;
    while (hi * hi <= n) hi *= 2;
    while (hi - lo > 1) {
        int64_t mid = lo + (hi - lo) / 2;
        if (mid * mid <= n)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

/* Algorithm 2, step 1: Canny's edge detector (J. Canny, "A computational
 * approach to edge detection", IEEE TPAMI 8(6), 1986), in integers:
 *   (a) smoothing by the 5 x 5 binomial kernel (1 4 6 4 1) x (1 4 6 4 1),
 *       replicated borders, left unnormalised: S = 256 x the smoothed image;
 *   (b) the gradient of S by central differences (replicated borders),
 *       Gx = S(r, c+1) - S(r, c-1), Gy = S(r+1, c) - S(r-1, c), and its
 *       squared magnitude M2 = Gx^2 + Gy^2;
 *   (c) non-maximum suppression across the edge: the gradient direction is
 *       put in one of four sectors (horizontal, vertical, and the two
 *       diagonals) by the exact tests |Gy| < tan(22.5 deg) |Gx|, i.e.
 *       (|Gx| + |Gy|)^2 < 2 Gx^2, and its mirror with the axes swapped; the
 *       pixel survives when M2 > M2 of the neighbour on the lower-column
 *       side of the sector's line (the upper-row side for the vertical
 *       sector) and M2 >= M2 of the opposite neighbour (neighbours outside
 *       the window count as 0), so a two-pixel plateau yields one pixel;
 *   (d) double threshold: a survivor is strong when M2 >= (256 hi)^2 and
 *       weak when (256 lo)^2 <= M2 < (256 hi)^2;
 *   (e) hysteresis: a weak survivor is an edge pixel when a chain of
 *       8-connected survivors (weak or strong) joins it to a strong one;
 *       strong survivors are edge pixels.  Breadth-first search from every
 *       strong survivor.
 * lo and hi are in the units of a central difference of the normalised
 * smoothed image (|G| / 256).  edges: h x w uint8 (1 = edge).  Optional
 * outputs (NULL to skip): smooth (S, int32), mag2 (M2, int64), cls (0 none,
 * 1 weak, 2 strong survivor). */
static const int or_binom5[5] = {1, 4, 6, 4, 1};

void oracle_canny(const uint8_t *gray, int h, int w, int lo, int hi, uint8_t *edges, int32_t *smooth,
                  int64_t *mag2, uint8_t *cls)
{
    const int64_t n = (int64_t)h * w;
    int32_t *S = (int32_t *)malloc(sizeof(int32_t) * (n ? n : 1));
    int64_t *M = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
    uint8_t *K = (uint8_t *)malloc(n ? n : 1);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (n ? n : 1));
    /* (a) */
    for (int r = 0; r < h; r++)
        for (int c = 0; c < w; c++) {
            int32_t acc = 0;
            for (int i = 0; i < 5; i++)
                for (int j = 0; j < 5; j++)
                    acc += or_binom5[i] * or_binom5[j] *
                           (int32_t)gray[(int64_t)clampi(r + i - 2, 0, h - 1) * w + clampi(c + j - 2, 0, w - 1)];
            S[(int64_t)r * w + c] = acc;
        }
    /* (b) */
    for (int r = 0; r < h; r++)
        for (int c = 0; c < w; c++) {
            int64_t gx = (int64_t)S[(int64_t)r * w + clampi(c + 1, 0, w - 1)] - S[(int64_t)r * w + clampi(c - 1, 0, w - 1)];
            int64_t gy = (int64_t)S[(int64_t)clampi(r + 1, 0, h - 1) * w + c] - S[(int64_t)clampi(r - 1, 0, h - 1) * w + c];
            M[(int64_t)r * w + c] = gx * gx + gy * gy;
        }
    /* (c) + (d) */
    const int64_t thi = (int64_t)256 * hi * (int64_t)256 * hi, tlo = (int64_t)256 * lo * (int64_t)256 * lo;
    for (int r = 0; r < h; r++)
        for (int c = 0; c < w; c++) {
            int64_t gx = (int64_t)S[(int64_t)r * w + clampi(c + 1, 0, w - 1)] - S[(int64_t)r * w + clampi(c - 1, 0, w - 1)];
            int64_t gy = (int64_t)S[(int64_t)clampi(r + 1, 0, h - 1) * w + c] - S[(int64_t)clampi(r - 1, 0, h - 1) * w + c];
            int64_t ax = gx < 0 ? -gx : gx, ay = gy < 0 ? -gy : gy, s2 = (ax + ay) * (ax + ay);
            int dr, dc; /* the neighbour on the "minus" side is (r - dr, c - dc) */
            if (s2 < 2 * ax * ax) {
                dr = 0; dc = 1;            /* gradient near 0 deg: compare left / right */
            } else if (s2 < 2 * ay * ay) {
                dr = 1; dc = 0;            /* near 90 deg: compare up / down */
            } else if ((gx > 0) == (gy > 0)) {
                dr = 1; dc = 1;            /* near 45 deg (rows grow downwards): (r-1,c-1) / (r+1,c+1) */
            } else {
                dr = -1; dc = 1;           /* near 135 deg: (r+1,c-1) / (r-1,c+1) */
            }
            int64_t m = M[(int64_t)r * w + c];
            int rm = r - dr, cm = c - dc, rp = r + dr, cp = c + dc;
            int64_t mm = (rm >= 0 && rm < h && cm >= 0 && cm < w) ? M[(int64_t)rm * w + cm] : 0;
            int64_t mp = (rp >= 0 && rp < h && cp >= 0 && cp < w) ? M[(int64_t)rp * w + cp] : 0;
            uint8_t k = 0;
            if (m > mm && m >= mp) k = m >= thi ? 2 : (m >= tlo ? 1 : 0);
            K[(int64_t)r * w + c] = k;
        }
    /* (e) */
    int64_t head = 0, tail = 0;
    for (int64_t i = 0; i < n; i++) {
        edges[i] = K[i] == 2;
        if (K[i] == 2) queue[tail++] = i;
    }
    while (head < tail) {
        int64_t i = queue[head++];
        int r = (int)(i / w), c = (int)(i % w);
        for (int a = -1; a <= 1; a++)
            for (int b = -1; b <= 1; b++) {
                int y = r + a, x = c + b;
                if ((a == 0 && b == 0) || y < 0 || y >= h || x < 0 || x >= w) continue;
                int64_t j = (int64_t)y * w + x;
                if (K[j] != 0 && !edges[j]) {
                    edges[j] = 1;
                    queue[tail++] = j;
                }
            }
    }
    if (smooth) memcpy(smooth, S, sizeof(int32_t) * n);
    if (mag2) memcpy(mag2, M, sizeof(int64_t) * n);
    if (cls) memcpy(cls, K, n);
    free(S);
    free(M);
    free(K);
    free(queue);
}

/* Algorithm 2, steps 1-3 on a grayscale search window: the Canny edge
 * pixels of step 1 (oracle_canny, thresholds lo and hi); step 2's gradient
 * of the window by central differences (replicated borders) and its
 * magnitude in fixed point with 4 fractional bits,
 * w = floor(16 sqrt(gx^2 + gy^2)); step 3's 9-bin unsigned orientation of
 * the edge pixels.  bins: h x w uint8 (the bin, 255 off edges); weight:
 * h x w int32 (w on edges, 0 off them). */
void oracle_phog_planes(const uint8_t *gray, int h, int w, int lo, int hi, uint8_t *bins, int32_t *weight)
{
    uint8_t *edge = (uint8_t *)malloc((size_t)h * w ? (size_t)h * w : 1);
    oracle_canny(gray, h, w, lo, hi, edge, NULL, NULL, NULL);
    for (int r = 0; r < h; r++)
        for (int c = 0; c < w; c++) {
            int gx = (int)gray[(int64_t)r * w + clampi(c + 1, 0, w - 1)] -
                     (int)gray[(int64_t)r * w + clampi(c - 1, 0, w - 1)];
            int gy = (int)gray[(int64_t)clampi(r + 1, 0, h - 1) * w + c] -
                     (int)gray[(int64_t)clampi(r - 1, 0, h - 1) * w + c];
            int64_t m = oracle_isqrt(256 * ((int64_t)gx * gx + (int64_t)gy * gy));
            int e = edge[(int64_t)r * w + c];
            bins[(int64_t)r * w + c] = e ? (uint8_t)oracle_orientation_bin(gx, gy, 9) : 255;
            weight[(int64_t)r * w + c] = e ? (int32_t)m : 0;
        }
    free(edge);
}

/* Algorithm 2, step 4: the magnitude-weighted integral histogram of the
 * orientation bins (Eq. 3.4 with w = the magnitude plane), by Algorithm 5's
 * recurrence.  out: b x h x w int64. */
void oracle_phog_ih(const uint8_t *bins, const int32_t *weight, int h, int w, int b, int64_t *out)
{
    for (int k = 0; k < b; k++) {
        int64_t *o = out + (int64_t)k * h * w;
        for (int r = 0; r < h; r++)
            for (int c = 0; c < w; c++) {
                int64_t above = r > 0 ? o[(int64_t)(r - 1) * w + c] : 0;
                int64_t before = c > 0 ? o[(int64_t)r * w + c - 1] : 0;
                int64_t corner = (r > 0 && c > 0) ? o[(int64_t)(r - 1) * w + c - 1] : 0;
                int64_t inc = bins[(int64_t)r * w + c] == k ? weight[(int64_t)r * w + c] : 0;
                o[(int64_t)r * w + c] = above + before - corner + inc;
            }
    }
}

/* Algorithm 2, steps 5-20 for one window [r0, r0+wh) x [c0, c0+ww): level
 * l = 0..L cuts the window into s x s cells (s = 2^l) of floor(wh/s) x
 * floor(ww/s) pixels at offsets (i*floor(wh/s), j*floor(ww/s)); each cell's
 * weighted histogram is summed pixel by pixel.  desc: b * sum_l 4^l int64,
 * level after level, cells row-major, bins innermost. */
void oracle_phog_descriptor(const uint8_t *bins, const int32_t *weight, int h, int w, int b, int L, int r0,
                            int c0, int wh, int ww, int64_t *desc)
{
    int64_t k = 0;
    for (int l = 0; l <= L; l++) {
        int s = 1 << l, ch = wh / s, cw = ww / s;
        for (int i = 0; i < s; i++)
            for (int j = 0; j < s; j++) {
                for (int q = 0; q < b; q++) desc[k + q] = 0;
                for (int y = r0 + i * ch; y < r0 + (i + 1) * ch; y++)
                    for (int x = c0 + j * cw; x < c0 + (j + 1) * cw; x++) {
                        if (y >= h || x >= w) continue;
                        int q = bins[(int64_t)y * w + x];
                        if (q < b) desc[k + q] += weight[(int64_t)y * w + x];
                    }
                k += b;
            }
    }
}

/* The pyramid match kernel of Eq. 2.23-2.24 between two descriptors of L+1
 * levels: I^l = sum of min over level l's entries, and
 *   kappa = I^0 / 2^L + sum_{l=1..L} I^l / 2^(L-l+1). */
double oracle_pyramid_match(const int64_t *x, const int64_t *y, int b, int L)
{
    double kappa = 0.0;
    int64_t k = 0;
    for (int l = 0; l <= L; l++) {
        int64_t n = (int64_t)b << (2 * l);
        double il = 0.0;
        for (int64_t i = 0; i < n; i++) il += (double)(x[k + i] < y[k + i] ? x[k + i] : y[k + i]);
        kappa += l == 0 ? il / (double)(1 << L) : il / (double)(1 << (L - l + 1));
        k += n;
    }
    return kappa;
}

