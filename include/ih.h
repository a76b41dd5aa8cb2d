/*
 * ih.h -- C ABI of the GB300 integral-histogram engine.
 *
 * The engine computes, on one GPU, the data-parallel path of the integral
 * histogram of Poostchi (2017), arXiv 1711.01656:
 *
 *   Q      binning of uint8 feature channels into one-hot bins     Eq. 2.15
 *   H      H(b,r,c) = sum_{r'<=r, c'<=c} Q(I(r',c'), b), inclusive Eq. 2.15,
 *          the tensor of Algorithm 5 (b x h x w, Fig. 5.1)
 *   h(R)   rectangle histogram from four corners of H               Eq. 2.16
 *   IH_w   weighted integral histograms (moment planes w = c, r,
 *          c^2, r^2)                                                 Eq. 3.4
 *   S(T)   spatially weighted local histogram of a window in O(1)   Eq. 3.1,
 *          evaluated from the moment planes (SWIH, Sec. 3.1.3)
 *
 * Conventions used by every call:
 *   - r is the row (the thesis's x), c the column (its y), both 0-based,
 *     origin top-left (Fig. 2.8).
 *   - A rectangle or window is four int32 (r0, c0, r1, c1), inclusive.
 *   - "device" pointers are CUDA device (or managed) addresses on the
 *     context's device; "host" pointers are ordinary CPU memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     Every call that takes a stream only enqueues work on it and returns;
 *     results are ready when the stream reaches that point.
 *   - The caller owns every buffer it passes in (pixels, rectangles,
 *     outputs).  The context owns the integral-histogram tensors it builds
 *     until ih_release() or ih_destroy().
 *   - Argument errors are detected on the host before anything is
 *     enqueued and return IH_EINVAL (or IH_EBUDGET / IH_ENOMEM); nothing is
 *     launched then.  Errors found on the device (an invalid rectangle, a
 *     CUDA launch failure) are recorded in the context and returned by the
 *     next ih_sync().  ih_last_error() gives a one-line message.
 *   - A context may be used from several host threads; calls are
 *     serialised internally.
 */
#ifndef IH_H
#define IH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ih_ctx ih_ctx;

typedef enum {
    IH_OK = 0,
    IH_EINVAL = 1,    /* invalid argument (host check) or invalid query (device) */
    IH_ENOMEM = 2,    /* device allocation failed */
    IH_EBUDGET = 3,   /* the build would exceed the context's HBM budget */
    IH_ECUDA = 4,     /* a CUDA runtime call or launch failed */
    IH_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    IH_ENOTBUILT = 6, /* the handle names no live frame */
    IH_ETOOBIG = 7,   /* ih_build_counts_static: the frame needs more carry
                         scratch than IH_STATIC_SCRATCH_BYTES */
    IH_ECANCELLED = 8 /* a server request was cancelled (ih_server_cancel) */
} ih_status;

/* Binning function Q of one channel (Eq. 2.15). */
typedef enum {
    IH_BIN_UNIFORM8 = 0, /* B equal bins over [0,256): Q(v) = floor(v*B/256) */
    IH_BIN_INDEX = 1     /* v is the bin; a value >= B falls in no bin       */
} ih_binmode;

typedef struct {
    int32_t bins; /* B_c >= 1 (<= 256) */
    int32_t mode; /* ih_binmode */
} ih_channel;

/* What the pixels of an ih_frame are. */
typedef enum {
    /* `channels` uint8 planes, binned as given by chan[] */
    IH_INPUT_PLANES = 0,
    /* 3 uint8 planes R, G, B; the engine derives the tracker's 7 feature
     * channels R, G, B, I = floor((R+G+B)/3) (Eq. 2.33) and the gradient
     * orientation index of I at central-difference steps 1, 2, 4 (9
     * unsigned 20-degree bins, replicated borders; Fig. 2.3) and bins them
     * as given by chan[0..6] (channels must be 7). */
    IH_INPUT_RGB_FEATURES = 1
} ih_input;

/* ih_frame.layout: how the context stores the count tensor (ih_export
 * always returns the packed bin-major tensor of Algorithm 5). */
typedef enum {
    IH_LAYOUT_BIN_MAJOR = 0, /* b x h x pitch, as Fig. 5.1 */
    /* bins innermost: each channel's bins are split in order into
     * ceil(B_c/8) groups of near-equal size (floor/ceil of B_c/groups), and
     * each group g of nb_g bins is stored as h x pitch x nb_g; a rectangle
     * query then reads each corner's bins from a few contiguous words */
    IH_LAYOUT_SLAB = 1,
    /* per-pixel records: the bin order (channel after channel) is cut into
     * groups of up to 8 consecutive bins drawn from at most two channels
     * (a new group starts where a third channel would begin); each group
     * takes 8 words (one 32-byte sector), its padding words holding 0, and
     * pairs of consecutive groups share a plane (the last group may be
     * alone).  Plane p is stored as h x pitch x w_p, w_p = 16 or 8.  A
     * rectangle query reads each corner from one 64-byte record per plane. */
    IH_LAYOUT_RECORD = 2
} ih_layout;

typedef struct {
    int32_t height, width;      /* H, W >= 1 */
    int32_t channels;           /* number of binned channels, 1..16, with
                                   at most 1024 bins in total */
    int32_t input;              /* ih_input */
    const ih_channel *chan;     /* host array [channels] */
    const uint8_t *d_pixels;    /* device; planar: plane p, row r starts at
                                   d_pixels + (p*H + r)*pitch_bytes */
    int64_t pitch_bytes;        /* >= W */
    int32_t weighted_channel;   /* -1: no moment planes; else the channel whose
                                   moment planes (Eq. 3.4) are built for
                                   ih_query_weighted */
    int32_t layout;             /* ih_layout */
    int32_t moment_bits;        /* 0 or 64: exact int64 moment planes;
                                   32: the planes modulo 2^32 (half the bytes),
                                   which still gives exact weighted histograms
                                   for windows of side <= 256 (the centred
                                   sums they need stay below 2^32); larger
                                   windows are refused */
} ih_frame;

typedef struct {
    int32_t device;             /* CUDA device ordinal */
    uint64_t hbm_budget_bytes;  /* cap on the bytes of live frames; 0 = none */
    uint32_t flags;             /* IH_CFG_* */
} ih_config;

/* ih_config.flags: record a CUDA event pair around every kernel launch on
 * the launching stream, read back by ih_profile_read(). */
enum { IH_CFG_PROFILE = 1 };

/* Creates a context on cfg->device.  *out receives the context.
 * Returns IH_EINVAL for a NULL argument or bad device, IH_ECUDA if the device
 * cannot be initialised. */
ih_status ih_create(const ih_config *cfg, ih_ctx **out);

/* Builds the integral histogram (Eq. 2.15; the tensor Algorithm 5 defines)
 * of each of the n >= 1 frames, plus the moment planes of Eq. 3.4 for a frame
 * whose weighted_channel >= 0, and enqueues the work on `stream`.
 * out_handles (host, n entries) receives one handle per frame.  The tensors
 * are owned by the context.  The pixels must stay valid until the stream
 * passes the build.  A frame without moment planes in the bin-major or slab
 * layout, small enough that all its tiles fit the GPU at once (a 640 x 480
 * frame, say), is built by one cooperative launch whose CTAs meet at a
 * bounded grid barrier (IH_SMALL=0 in the environment turns this off); a
 * barrier wait that gives up makes the next ih_sync return IH_ETIMEOUT.
 * Returns IH_EINVAL for an invalid descriptor, IH_EBUDGET if the frames'
 * bytes would exceed the HBM budget (no frame is built then), IH_ENOMEM /
 * IH_ECUDA on allocation or launch failure. */
ih_status ih_build(ih_ctx *ctx, const ih_frame *frames, int32_t n, int32_t *out_handles,
                   void *stream);

/* The count build of ih_build (Eq. 2.15, Algorithm 5's tensor) with the
 * tiles' 2-D prefixes computed on the tensor cores: for a 128 x 128 tile and
 * bin b, H_local = T O_b T^t with O_b the tile's one-hot plane of b and T
 * the lower-triangular ones, as two chained tcgen05 MMAs (kind::f16, bf16
 * 0/1 operands, fp32 accumulators in tensor memory: exact, since a tile's
 * counts stay below 2^24), plus the same tile carries as ih_build.  An
 * alternative kernel of the count path, kept for measurement beside the
 * scan-based tiles: the frame must use IH_INPUT_PLANES, IH_LAYOUT_BIN_MAJOR
 * and no weighted channel (IH_EINVAL otherwise).  The frame it builds is an
 * ordinary frame (*out_handle) for every query, export and release call.
 * A bounded device-side wait that gives up makes the next ih_sync() return
 * IH_ETIMEOUT. */
ih_status ih_build_mma(ih_ctx *ctx, const ih_frame *frame, int32_t *out_handle, void *stream);

/* Rectangle histograms by the four-corner rule of Eq. 2.16:
 *   h(R,b) = H(r1,c1,b) - H(r0-1,c1,b) - H(r1,c0-1,b) + H(r0-1,c0-1,b)
 * with H(-1,.) = H(.,-1) = 0.  d_rects: device, n x 4 int32 (r0,c0,r1,c1);
 * d_out: device, n x B int32 (B = the frame's total bins, channels'
 * bins in channel order).  An invalid rectangle (outside the frame, r0>r1 or
 * c0>c1) gets a row of -1 and makes the next ih_sync() return IH_EINVAL.
 * n may be 0. */
ih_status ih_query_rects(ih_ctx *ctx, int32_t handle, const int32_t *d_rects, int64_t n,
                         int32_t *d_out, void *stream);

/* Spatial kernels for ih_query_weighted (w = c1-c0+1, h = r1-r0+1). */
typedef enum {
    /* Epanechnikov profile whose ellipse passes through the window's outer
     * corners: k(r,c) = 1 - (2c-c0-c1)^2/(2w^2) - (2r-r0-r1)^2/(2h^2)
     * (every pixel of the window has k > 0) */
    IH_K_EPANECHNIKOV = 0,
    /* Manhattan (city-block) kernel, Eq. 3.3: k(r,c) = (h + w) -
     * |2r-r0-r1| - |2c-c0-c1| (>= 2 inside the window), evaluated exactly
     * from four quadrants (Sec. 3.1.3, Fig. 3.4) of the count plane and the
     * c- and r-weighted moment planes */
    IH_K_MANHATTAN = 1,
    /* wedding-cake approximation, Eq. 3.2 (Sec. 3.1.2): L nested windows,
     * window j shrunk by floor(j*h/(2L)) rows and floor(j*w/(2L)) columns
     * per side; the ring between windows j and j+1 weighs (h + w)(j + 1)/L.
     * Only the count plane is read; L = IH_LAYERS field of `flags`. */
    IH_K_WEDDING_CAKE = 2
} ih_kernel;

enum { IH_NORMALIZE = 1 }; /* divide each histogram by sum_T k(r,c) */
/* flags field: wedding-cake layers L (1..64; 0 means 4) */
#define IH_LAYERS(n) ((((uint32_t)(n)) & 0xffu) << 8)

/* Spatially weighted local histograms (Eq. 3.1) of n windows on the frame's
 * weighted channel, in O(1) each from the moment planes (Sec. 3.1.3):
 * every bin's weighted sum is an exact rational number (integer part and
 * remainder computed exactly in int64/uint64) converted to float with a
 * relative error below 4e-7; no step uses FP64.  d_windows: device,
 * n x 4 int32; d_out: device, n x B_w float (B_w = bins of the weighted
 * channel).  Windows must have sides <= 32768 (<= 256 for the Epanechnikov
 * and Manhattan kernels when the frame's moment planes are 32-bit).  Invalid
 * windows give a row of -1 and IH_EINVAL at the next ih_sync().  IH_EINVAL
 * (host) if the frame has no moment planes, for an unknown kernel or flag,
 * or for more than 64 layers. */
ih_status ih_query_weighted(ih_ctx *ctx, int32_t handle, const int32_t *d_windows, int64_t n,
                            uint32_t kernel, uint32_t flags, float *d_out, void *stream);

/* Both query kinds of one frame in one call and one launch: the rectangles
 * of ih_query_rects (Eq. 2.16) and the weighted windows of
 * ih_query_weighted (Sec. 3.1.3), with the same arguments, layouts, results
 * and errors as those two calls; either count may be 0 (then its pointers
 * may be NULL, and a frame without moment planes is accepted when
 * n_windows = 0).  The weighted work runs in its own CTAs beside the
 * rectangle CTAs, so its latency overlaps the rectangles' loads. */
ih_status ih_query(ih_ctx *ctx, int32_t handle, const int32_t *d_rects, int64_t n_rects, int32_t *d_rect_out,
                   const int32_t *d_windows, int64_t n_windows, uint32_t kernel, uint32_t flags,
                   float *d_weighted_out, void *stream);

/* Sliding-window histogram matching (Sec. 2.4.3): for every placement of a
 * win_h x win_w window whose top-left pixel (r, c) lies in the search region
 * search = (sr0, sc0, sr1, sc1) (host, 4 int32, inclusive), the city-block
 * distance of Eq. 2.22 with p = 1 between the window's histogram over the
 * tensor bins bin0 .. bin0 + nbins - 1 (four corners each, Eq. 2.16) and
 * d_target (device, nbins int32):
 *   d_out[(r - sr0) * (sc1 - sc0 + 1) + (c - sc0)] = sum_i |H(i) - target(i)|
 * (device, int32).  IH_EINVAL (host) if a placement leaves the frame or the
 * bin range is empty or leaves the frame's bins. */
ih_status ih_match_window(ih_ctx *ctx, int32_t handle, int32_t bin0, int32_t nbins, const int32_t *d_target,
                          int32_t win_h, int32_t win_w, const int32_t *search, int32_t *d_out,
                          void *stream);

/* Joint integral histogram update of Algorithm 4 (Sec. 4.1.1):
 *   count tensor of dst += count tensor of add - count tensor of sub,
 * element by element, in one stream-ordered pass; add or sub may be -1
 * (none).  The frames must have the same size, channels' bins and layout and
 * no moment planes; the counts must stay within int32 (a joint histogram of
 * F frames holds at most F*H*W per cell).  IH_EINVAL (host) otherwise. */
ih_status ih_accumulate(ih_ctx *ctx, int32_t dst, int32_t add, int32_t sub, void *stream);

/* Local median of Algorithm 4 (ComputeLocalMedian): for every pixel (r, c)
 * the box of rows r - floor(m/2) .. r + ceil(m/2) - 1 and columns
 * c - floor(n/2) .. c + ceil(n/2) - 1, clipped to the frame, gives by four
 * corners (Eq. 2.16) the histogram H over the bins bin0 .. bin0 + nbins - 1;
 * the output is the smallest i with H(bin0) + ... + H(bin0 + i) >= ceil(N/2),
 * N = H's total (the lower median bin), or -1 when N = 0.  On a joint
 * histogram of F frames (ih_accumulate) this is the spatio-temporal median of
 * the m x n x F neighbourhood.  d_out: device, h x w int32, row-major. */
ih_status ih_local_median(ih_ctx *ctx, int32_t handle, int32_t bin0, int32_t nbins, int32_t m, int32_t n,
                          int32_t *d_out, void *stream);

/* Spatial pyramids of gradient orientations (Algorithm 2, Sec. 2.3).
 *
 * ih_canny_edges runs step 1 alone, Canny's edge detector (J. Canny 1986),
 * on a grayscale window d_gray (device, height x width uint8, row pitch
 * pitch_bytes; height * width <= 2^30), in integers: 5 x 5 binomial
 * smoothing (1 4 6 4 1 x 1 4 6 4 1, replicated borders, left unnormalised:
 * S = 256 x the smoothed image); the gradient G of S by central differences
 * (replicated borders); non-maximum suppression across the edge in four
 * direction sectors (a pixel survives when |G|^2 is above its neighbour's on
 * the lower-column side of the sector's line -- the upper-row side for the
 * vertical sector -- and not below the opposite neighbour's; neighbours
 * outside the window count as 0); the double threshold: strong when
 * |G| >= 256 tau_high, weak when |G| >= 256 tau_low (0 <= tau_low <=
 * tau_high <= IH_CANNY_MAX_THRESHOLD, in units of a central difference of
 * the normalised smoothed image); and hysteresis: a weak survivor is an edge
 * pixel when 8-connected survivors join it to a strong one.  d_edges
 * (device, caller-owned, height rows of edges_pitch >= width bytes) receives
 * 1 on edge pixels and 0 elsewhere.  Hysteresis is a union-find whose
 * pointer walks are bounded: one that gives up makes the next ih_sync()
 * return IH_ETIMEOUT.  Scratch of 6 bytes per pixel comes from the
 * context's pool.
 *
 * ih_phog_build runs steps 1-4 on the window: Canny's edge pixels (as
 * above); the window's own gradient by central differences (replicated
 * borders) and its magnitude in fixed point with 4 fractional bits,
 * w = floor(16 sqrt(gx^2 + gy^2)) (exact integer square root); the
 * unsigned orientation of edge pixels in 9 bins of 20 degrees; and the
 * w-weighted integral histogram of those bins (Eq. 3.4 with a pixel
 * weight), int64 9 x height x pitch, owned by the context as frame
 * *out_handle (ih_info reports it with 9 bins and its bytes as
 * moment_bytes; count-tensor calls refuse it).  Errors as for ih_build. */
#define IH_CANNY_MAX_THRESHOLD 1024
ih_status ih_canny_edges(ih_ctx *ctx, const uint8_t *d_gray, int32_t height, int32_t width, int64_t pitch_bytes,
                         int32_t tau_low, int32_t tau_high, uint8_t *d_edges, int64_t edges_pitch, void *stream);
ih_status ih_phog_build(ih_ctx *ctx, const uint8_t *d_gray, int32_t height, int32_t width, int64_t pitch_bytes,
                        int32_t tau_low, int32_t tau_high, int32_t *out_handle, void *stream);

/* Steps 5-20: the descriptor of each of n windows (device n x 4 int32
 * r0, c0, r1, c1): for l = 0 .. levels, the window's 2^l x 2^l cells of
 * floor(h/2^l) x floor(w/2^l) pixels at multiples of that size, each cell's
 * 9 weighted bins; d_out: device n x 9 * sum_l 4^l int64, level after level,
 * cells row-major, bins innermost.  levels 0..4 (IH_EINVAL otherwise).  A
 * window outside the frame gets a row of -1 and makes the next ih_sync()
 * return IH_EINVAL. */
ih_status ih_phog_descriptors(ih_ctx *ctx, int32_t handle, int32_t levels, const int32_t *d_windows, int64_t n,
                              int64_t *d_out, void *stream);

/* Sec. 2.4.4: the pyramid match kernel (Eq. 2.24) of d_target (device, a
 * descriptor from ih_phog_descriptors with the same levels) against the
 * descriptor of every win_h x win_w window whose top-left pixel lies in
 * search = (sr0, sc0, sr1, sc1) (host): kappa = I^0/2^L + sum_{l>=1}
 * I^l/2^(L-l+1), I^l = sum of min over level l's entries; d_out: device,
 * (sr1-sr0+1) x (sc1-sc0+1) float.  IH_EINVAL (host) for a placement outside
 * the frame. */
ih_status ih_phog_match(ih_ctx *ctx, int32_t handle, int32_t levels, const int64_t *d_target, int32_t win_h,
                        int32_t win_w, const int32_t *search, float *d_out, void *stream);

/* Frees every tensor the context owns and the context.  NULL-safe.
 * Synchronises the device first. */
ih_status ih_destroy(ih_ctx *ctx);

/* ---- helpers ---------------------------------------------------------- */

/* Frees the frame's tensors (stream-ordered on `stream`); the handle may be
 * reused by a later build. */
ih_status ih_release(ih_ctx *ctx, int32_t handle, void *stream);

/* Waits for `stream`, then returns the first device-side error recorded since
 * the previous ih_sync (and clears it), else IH_OK. */
ih_status ih_sync(ih_ctx *ctx, void *stream);

typedef struct {
    int32_t height, width, channels, total_bins;
    int32_t weighted_channel, weighted_bins;
    int64_t pitch_elems;        /* row pitch of the count tensor, elements */
    int64_t count_bytes;        /* bytes of the count tensor */
    int64_t moment_bytes;       /* bytes of the moment planes (0 if none) */
    int32_t tile_rows, tile_cols; /* tile grid the build used (band rows,
                                     strip columns) */
} ih_frame_info;

/* Host copy of a live frame's geometry. */
ih_status ih_info(ih_ctx *ctx, int32_t handle, ih_frame_info *out);

/* Copies the count tensor to d_dst (device, B x H x W int32, packed,
 * bin-major as Algorithm 5's output), enqueued on `stream`. */
ih_status ih_export(ih_ctx *ctx, int32_t handle, int32_t *d_dst, void *stream);

/* Copies moment plane `plane` (0: w=c, 1: w=r, 2: w=c^2, 3: w=r^2; Eq. 3.4)
 * to d_dst (device, B_w x H x W int64, packed); for a frame built with
 * moment_bits = 32 each value is the plane modulo 2^32. */
ih_status ih_export_moments(ih_ctx *ctx, int32_t handle, int32_t plane, int64_t *d_dst,
                            void *stream);

/* The feature pre-pass alone: 3 planes R,G,B (device, H rows of pitch_bytes,
 * plane stride H*pitch_bytes) -> 7 planes (device, packed H x W each) as
 * described for IH_INPUT_RGB_FEATURES. */
ih_status ih_features(ih_ctx *ctx, const uint8_t *d_rgb, int32_t height, int32_t width,
                      int64_t pitch_bytes, uint8_t *d_out, void *stream);

/* Per-kernel launch statistics of a context created with IH_CFG_PROFILE. */
typedef struct {
    char name[40];      /* e.g. "tiles/count", "tiles/moment_c2", "query_rects" */
    int64_t launches;   /* launches since the last reset */
    double total_ms;    /* sum of the event-timed durations */
} ih_kernel_stat;

/* Waits for the recorded events, then copies up to `max` statistics (one per
 * kernel that ran) to `out` (host) and their number to *count (host).
 * reset != 0 clears them afterwards.  IH_EINVAL without IH_CFG_PROFILE. */
ih_status ih_profile_read(ih_ctx *ctx, ih_kernel_stat *out, int32_t max, int32_t *count,
                          int32_t reset);

/* Restricts the event pairs of a context created with IH_CFG_PROFILE to the
 * kernels named in `names` (host, n NUL-terminated strings as reported by
 * ih_profile_read, e.g. "tiles/count+moments"); n = 0 restores all kernels.
 * Fewer events perturb the timed work less.  IH_EINVAL without
 * IH_CFG_PROFILE or for an unknown name. */
ih_status ih_profile_select(ih_ctx *ctx, const char *const *names, int32_t n);

/* Kernel launches issued by this context since it was created (all of them
 * are this library's own kernels). */
int64_t ih_launch_count(ih_ctx *ctx);

/* Checks the device-side wait that the persistent batched build and the
 * tensor-core tiles use: one thread waits, on `stream`, for a counter that
 * nothing raises and gives up after `polls` polls (1..2^24, a few dozen ns
 * apart), exactly as a wait whose producer never finishes would.  The next
 * ih_sync() then returns IH_ETIMEOUT and clears the error; the context stays
 * usable.  No GPU fault is involved. */
ih_status ih_wait_selftest(ih_ctx *ctx, int32_t polls, void *stream);

/* Bytes of the frames (count tensors and moment planes) the context owns now,
 * the quantity its HBM budget bounds (0 for a NULL context). */
uint64_t ih_memory_used(ih_ctx *ctx);

/* One-line description of the last error of this context ("" if none). */
const char *ih_last_error(ih_ctx *ctx);

/* ---- batches ---------------------------------------------------------- */

/* A batch builds many frames of uneven size and channel or bin count with ONE
 * launch of each build kernel over all of them (and one launch of each query
 * kernel over all their queries), optionally replayed from a CUDA graph. */
typedef struct ih_batch ih_batch;

typedef struct {
    const int32_t *d_rects;     /* device: every frame's rectangles (x4 int32),
                                   frame 0's first; NULL = no rectangle queries */
    const int64_t *rects;       /* host, n entries: rectangles of frame k */
    int32_t *d_rect_out;        /* device: frame k's rects[k] x B_k int32 block,
                                   blocks in frame order */
    const int32_t *d_windows;   /* device: every frame's weighted windows;
                                   NULL = no weighted queries */
    const int64_t *windows;     /* host, n entries: windows of frame k */
    float *d_weighted_out;      /* device: frame k's windows[k] x B_w,k floats,
                                   blocks in frame order */
    uint32_t kernel, flags;     /* as for ih_query_weighted */
} ih_batch_queries;

enum {
    IH_BATCH_GRAPH = 1,      /* capture the run's launches in a CUDA graph */
    IH_BATCH_AUTOTUNE = 2,   /* ih_autotune every distinct frame shape first */
    IH_BATCH_PERSISTENT = 4  /* build every frame in ONE persistent launch:
                                CTAs take the tile sums, carry scans and tiles
                                of all frames by ticket, each frame's phases
                                ordered by per-frame counters with bounded
                                waits (a wait that gives up makes ih_sync
                                return IH_ETIMEOUT); a run is then the feature
                                pre-pass of the RGB frames, the build and the
                                queries: 3 launches (2 without RGB frames) */
};

/* Plans a batch of n frames: allocates every frame's tensors (the frames are
 * registered in the context; out_handles, host, n entries; release them with
 * ih_release), their feature scratch and tile carries, and uploads the
 * descriptor tables; with IH_BATCH_GRAPH also captures the run in a CUDA
 * graph.  Pixel, rectangle, window and output pointers are baked into the
 * plan: each run reads and writes the same buffers.  Synchronous (allocates
 * and uploads).  Errors as for ih_build. */
ih_status ih_batch_create(ih_ctx *ctx, const ih_frame *frames, int32_t n, const ih_batch_queries *queries,
                          uint32_t flags, ih_batch **out, int32_t *out_handles);

/* Enqueues one run of the batch on `stream`: the feature pre-pass of every
 * RGB frame, the build of every frame and the batch's queries. */
ih_status ih_batch_run(ih_batch *batch, void *stream);

/* Frees the plan (not the frames).  Synchronises the device first. */
ih_status ih_batch_destroy(ih_batch *batch);

/* Times the build of `frame` on each candidate tile grid (band rows 32, 64,
 * 128 x strip columns 128..1024) and makes the context build every later
 * frame of the same shape (size, channels, bins, input kind, weighted
 * channel, layout) with the fastest.  Synchronous. */
ih_status ih_autotune(ih_ctx *ctx, const ih_frame *frame, void *stream);

/* Makes the context build every later frame of `frame`'s shape (as for
 * ih_autotune) on tiles of band_rows (1..128) x strip_cols (a multiple of
 * 128) pixels, e.g. to compare kernels on one tile grid.  Host only. */
ih_status ih_tune_set(ih_ctx *ctx, const ih_frame *frame, int32_t band_rows, int32_t strip_cols);

/* ---- serving ---------------------------------------------------------- */

/* A server runs a request loop for many concurrent tracker streams: each
 * request is a frame plus its rectangle and weighted queries.  A scheduler
 * thread admits pending requests as in-flight slots and HBM (the context's
 * budget) free up, merges the requests admitted together into one batched
 * build and one batched query launch (a "tick"), and runs ticks on several
 * CUDA streams so that they overlap on the device.  Each tracker's latest
 * completed frame stays resident until its next frame completes or memory is
 * needed for a pending request (least recently completed first). */
typedef struct ih_server ih_server;

typedef struct {
    int32_t streams;       /* CUDA streams ticks are spread over (>= 1) */
    int32_t max_inflight;  /* ticks on the device at once (>= 1) */
    int32_t max_batch;     /* requests merged into one tick (>= 1, <= 256) */
    uint32_t flags;        /* reserved, 0 */
} ih_server_config;

typedef struct {
    int32_t tracker;             /* tracker stream id, >= 0 */
    ih_frame frame;              /* chan copied at submit; pixels must stay
                                    valid until the request completes */
    ih_channel chan[16];         /* storage the server copies frame.chan into */
    const int32_t *d_rects;      /* device, n_rects x 4, or NULL */
    int64_t n_rects;
    int32_t *d_rect_out;         /* device, n_rects x B int32 */
    const int32_t *d_windows;    /* device, n_windows x 4, or NULL */
    int64_t n_windows;
    float *d_weighted_out;       /* device, n_windows x B_w float */
    uint32_t weighted_flags;     /* IH_NORMALIZE or 0 */
    uint64_t user;               /* returned in the completion */
} ih_request;

typedef struct {
    uint64_t user;
    int32_t status;       /* ih_status of the request */
    int32_t handle;       /* the frame while it stays resident, or -1 */
    double t_submit;      /* seconds on the server clock (ih_server_clock) */
    double t_admit;       /* the tick holding the request was enqueued */
    double t_done;        /* the device finished the request's tick */
} ih_completion;

/* Starts a server on ctx.  Synchronous. */
ih_status ih_server_create(ih_ctx *ctx, const ih_server_config *cfg, ih_server **out);
/* Queues a request (validated now: IH_EINVAL without queueing). */
ih_status ih_server_submit(ih_server *srv, const ih_request *req);
/* Copies up to max completions (host) to out, waiting up to wait_ms for the
 * first one; returns how many were copied. */
int32_t ih_server_poll(ih_server *srv, ih_completion *out, int32_t max, int32_t wait_ms);
/* Cancels the request submitted with tag `user` (the first such request
 * that has not completed).  A request still waiting for admission leaves
 * the queue at once and completes with IH_ECANCELLED; it never holds budget.
 * A request already on the device cannot be stopped: it completes with
 * IH_ECANCELLED when its tick finishes, and its frame is released then
 * instead of staying resident, which returns its bytes to the budget; its
 * buffers stay in use until that completion.  Returns IH_OK, or IH_EINVAL
 * when no uncompleted request carries the tag. */
ih_status ih_server_cancel(ih_server *srv, uint64_t user);
/* Waits until every submitted request has completed. */
ih_status ih_server_drain(ih_server *srv);
/* Seconds since the server started (host monotonic clock). */
double ih_server_clock(ih_server *srv);
/* Drains, stops the scheduler and releases the resident frames. */
ih_status ih_server_destroy(ih_server *srv);

/* ---- allocation-free variant ------------------------------------------ */

/* The thesis has no counterpart to this call; it exists for callers that
 * cannot allocate device memory while they run (a real-time loop whose
 * device memory is reserved up front by its own arena, where a cudaMalloc
 * would synchronise the device, or an application whose allocator owns all
 * device memory).
 *
 * Builds the count integral histogram of ONE uint8 channel on the
 * CURRENT device, enqueued on `stream`, without allocating anything:
 *   d_pixels  device, H rows of pitch_bytes (>= W) bytes;
 *   bins      1..256, mode an ih_binmode;
 *   d_out     device, caller-owned, bins x H x out_pitch int32, bin-major;
 *             out_pitch >= W and a multiple of 4, d_out 16-byte aligned;
 *             columns W..out_pitch-1 receive unspecified values.
 * Tile carries live in one device array of IH_STATIC_SCRATCH_BYTES that the
 * library holds on every GPU that loads it until the process exits.  The
 * first call made on each device does a one-time set-up: it looks up the
 * array's device address and prepares the build kernels for that device,
 * which SYNCHRONISES THE DEVICE once; make that first call before any stream
 * capture begins and before the loop that must not stall.  Later calls only
 * enqueue kernels: the three-kernel build of ih_build (tile sums, carry scan,
 * count tiles), also for the small frames that ih_build builds in one
 * cooperative launch.  All calls share the
 * array: calls whose work overlaps on the GPU race on it and must be ordered
 * by the caller (one stream, or events).  Returns IH_EINVAL for bad arguments,
 * IH_ETOOBIG when even the largest tiles need more than the array holds
 * (about 4*bins*(W*ceil(H/128) + H*ceil(W/1024)) bytes: a 1920x1080 channel
 * fits up to 107 bins), IH_ECUDA on a CUDA error. */
#define IH_STATIC_SCRATCH_BYTES (8u << 20)
ih_status ih_build_counts_static(const uint8_t *d_pixels, int32_t height, int32_t width,
                                 int64_t pitch_bytes, int32_t bins, int32_t mode, int32_t *d_out,
                                 int64_t out_pitch, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* IH_H */
