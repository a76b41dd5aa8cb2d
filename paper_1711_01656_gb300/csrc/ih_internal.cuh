// ih_internal.cuh -- descriptors shared by the engine's kernels and its C ABI.
//
// A build computes, over a grid of tiles of R rows (a band) by Wc columns (a
// strip), the count integral histogram of every channel (Eq. 2.15, the
// tensor of Algorithm 5) and, for one optional "weighted" channel, the four
// moment planes of Eq. 3.4 with w in {c, r, c^2, r^2}.  Three kernels remove
// Algorithm 5's serial dependence:
//
//   tile sums  : per tile and bin, the column sums over the band and the row
//                sums over the strip (and, for the weighted channel, the same
//                sums weighted by the offset inside the tile and its square);
//   carry scan : exclusive prefixes of those sums over bands (G), over strips
//                (L) and over both (the tile corners), in int32 for counts
//                and int64 for the moments;
//   tiles      : per tile and bin group, the tile's 2-D inclusive prefix
//                seeded with its carries, each output cell written once.
//
// With tile origin (R0, C0) and any weight w:
//   H_w(r,c) = corner_w + sum_{C0<=c'<=c} G_w(c')
//            + sum_{R0<=r'<=r} ( L_w(r') + sum_{C0<=c'<=c} w(r',c') Q(r',c') )
// which is Eq. 3.4 (Eq. 2.15 for w = 1) split at the tile's top and left edges.
// A single count-only frame whose tiles all fit the GPU at once takes the
// same split in one cooperative launch instead (small_plan, k_small.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ih {

constexpr int kMaxChannels = 16;
constexpr int kMaxGroups = 128;
constexpr int kMaxBins = 1024;   // total bins of a frame
constexpr int kChunk = 128;       // columns a warp covers at once (4 per lane)
constexpr int kMaxBandRows = 128;
constexpr int kGroupBins = 8;     // bins per warp in the count tiles kernel
constexpr int kWindowBins = 16;   // bins per CTA in the tile-sums kernel
constexpr int kSumCols = 128;     // columns per pass of the tile-sums kernel

// Count-tensor layouts.
enum Layout {
    LAYOUT_BIN_MAJOR = 0,  // [B][H][P]                (Fig. 5.1)
    LAYOUT_SLAB = 1,       // per bin group g: [H][P][nb_g], bins innermost
    LAYOUT_RECORD = 2      // per plane p: [H][P][rec_w_p]; a plane's record
                           // holds up to two 8-bin spans of the bin order
};

// Spatial kernels of the weighted queries (the values of ih_kernel).
enum WeightKernel { IH_KERNEL_EPANECHNIKOV = 0, IH_KERNEL_MANHATTAN = 1, IH_KERNEL_WEDDING_CAKE = 2 };

// Weight kinds, used by the kernel-id table and the moment planes.
enum WeightKind { WK_ONE = 0, WK_COL = 1, WK_ROW = 2, WK_COL2 = 3, WK_ROW2 = 4 };

// Kernel ids for the optional per-launch event timing (ids 1, 2 and 5 name
// no kernel any more: the tile sums of both window kinds and the moment
// tiles run inside KID_SUMS_ALL and KID_TILES_BOTH; the ids stay fixed).
enum KernelId {
    KID_FEATURES = 0,
    KID_SUMS_COUNT = 1,
    KID_SUMS_WEIGHTED = 2,
    KID_SCAN = 3,
    KID_TILES_COUNT = 4,
    KID_TILES_MOMENTS = 5,
    KID_QUERY_RECTS = 6,
    KID_QUERY_WEIGHTED = 7,
    KID_EXPORT = 8,
    KID_TILES_BOTH = 9,  // count and moment tiles of one frame in one launch
    KID_MATCH = 10,
    KID_ACCUMULATE = 11,
    KID_MEDIAN = 12,
    KID_PHOG_BUILD = 13,
    KID_PHOG_QUERY = 14,
    KID_SUMS_ALL = 15,  // tile sums of all windows of one frame in one launch
    KID_QUERY_BOTH = 16,  // rectangle and weighted queries of one frame in one launch
    KID_TILES_MMA = 17,   // count tiles as tensor-core products (k_mma.cu)
    KID_PERSISTENT = 18,  // tile sums, carry scan and tiles of a batch in one persistent launch
    KID_ONEPASS = 19,     // the one-pass build of a small frame
    KID_SMALL = 20,       // the small-frame build (one cooperative launch)
    KID_COUNT = 21
};

// Optional launch hook: mark(ctx, kid, 0, st) before a kernel is launched on
// st and mark(ctx, kid, 1, st) right after.
struct Prof {
    void *ctx;
    void (*mark)(void *ctx, int kid, int phase, cudaStream_t st);
};
inline void prof_mark(const Prof *p, int kid, int phase, cudaStream_t st)
{
    if (p && p->mark) p->mark(p->ctx, kid, phase, st);
}

// Programmatic dependent launch.  A kernel launched with launch_pdl is set up
// while the previous kernel on its stream drains: its CTAs are dispatched as
// soon as every CTA of the previous grid has exited, overlapping that grid's
// completion and memory flush, and each calls pdl_wait() before it reads or
// writes anything, which returns once the previous grid has completed and its
// writes are visible.  No kernel triggers its dependents early (triggering at
// a CTA's start filled the SMs with waiting CTAs and measured slower than the
// implicit trigger at CTA exit).  Setting the environment variable IH_PDL=0
// launches every kernel with plain stream order instead.
bool pdl_enabled();
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

struct ChanDev {
    const uint8_t *plane;  // row r starts at plane + r * pitch
    int64_t pitch;
    int32_t bins;          // bins of the channel
    int32_t mode;          // 0: uniform over [0,256), 1: value is the bin
    int32_t bin_off;       // first bin of the channel in the count tensor
    int32_t pad;
};

// A bin group: bins [b_lo, b_lo + nb) of channel `chan` (channel-local) and,
// in LAYOUT_RECORD only, the first nb1 bins [b_lo1, b_lo1 + nb1) of the next
// channel chan1.  Either way the group's bins are consecutive in the
// tensor's bin order; bin k of the group (0 <= k < nb + nb1) is field k of
// the packed one-hot words of the count tiles kernel.  plane / off: the
// plane holding the group and the word offset of its bins inside the
// plane's per-pixel record (LAYOUT_SLAB: the group's own plane, offset 0).
struct GroupDev {
    int16_t chan, b_lo, nb, pad;
    int16_t chan1, b_lo1, nb1, pad1;
    int16_t plane, off, pad2, pad3;
};

struct TileGrid {
    int32_t H, W;      // frame
    int32_t R, Wc;     // band rows (<= kMaxBandRows), strip columns (% kChunk == 0)
    int32_t nb, ns;    // number of bands, strips
    int64_t P;         // row pitch of the outputs, elements (multiple of 4)
};

struct PlaneSet {
    TileGrid g;
    int32_t B;            // total bins (all channels)
    int32_t nchan;
    int32_t layout;       // Layout of the count tensor
    int32_t wch;          // weighted channel, or -1
    int32_t mom32;        // moment planes stored as uint32
    int32_t uni;          // every channel bins uniformly (mode 0): the tiles kernels take a
                          // code path with the bin rule folded in
    ChanDev chan[kMaxChannels];
    int32_t ngroups;      // count bin groups (<= kGroupBins bins each)
    int32_t nwin;         // tile-sums windows (<= kWindowBins bins each)
    int32_t nwin_count;   // the first nwin_count windows are not of channel wch
    GroupDev grp[kMaxGroups];
    GroupDev win[kMaxGroups];
    int32_t nplanes;      // LAYOUT_SLAB / LAYOUT_RECORD planes
    int32_t seg2;         // LAYOUT_RECORD: some group draws on two channels
    int16_t rec_w[kMaxGroups];     // words per pixel record of each plane
    int64_t slab_off[kMaxGroups];  // element offset of each plane
    int32_t *out;         // count tensor
    int64_t *mom;         // moment planes as quads [Bw][H][P][4] (w = c, r, c^2, r^2 of
                          // one pixel together), or null; uint32 (values mod 2^32) when mom32
    // carries (null when the frame is a single tile)
    int32_t *colsum;      // [nb][B][W]  column counts -> G0 after the scan
    int32_t *rowsum;      // [ns][B][H]  row counts    -> L0 after the scan
    int32_t *tilesum;     // [nb][ns][B]
    int32_t *corner;      // [nb][ns][B]
    // weighted-channel carries (Bw = bins of channel wch)
    int32_t *col_su;      // [nb][Bw][W] sum of (r-R0), (r-R0)^2 over the band
    int32_t *col_suu;
    int32_t *row_sv;      // [ns][Bw][H] sum of (c-C0), (c-C0)^2 over the strip
    int32_t *row_svv;
    int64_t *tile_w;      // [nb][ns][Bw][4]: sums of (r-R0), (r-R0)^2, (c-C0), (c-C0)^2
    int64_t *g_r;         // [nb][Bw][W] G for w = r and r^2 (int64)
    int64_t *g_rr;
    int64_t *l_c;         // [ns][Bw][H] L for w = c and c^2 (int64)
    int64_t *l_cc;
    int64_t *corner_w;    // [nb][ns][Bw][4] corners for w = c, r, c^2, r^2
    // one-pass build of small frames (onepass_ok): per band and bin the
    // published column counts (agg) and inclusive column prefixes (incl),
    // [nb][B][P]; per band and group a flag, then a ticket counter
    int32_t *agg, *incl, *flags;
    // small-frame build (small_plan): rows per warp (0: not planned), and per
    // tile its packed column counts [ngroups][nb][ns][256], per strip its
    // packed row counts [ns][ngroups][H][2], per tile its bin totals
    // [nb][ns][ngroups][8], and the grid barrier's arrival and exit counters
    // (zero before a launch; every launch leaves them zero).  sm_zeroed: the
    // counters are known to be zero (scratch kept from launch to launch), so
    // the launch needs no memset first.
    int32_t small, sm_zeroed;
    uint32_t *sm_col, *sm_row;
    int32_t *sm_tot;
    unsigned int *sm_bar;
    int *err;             // the context's error word (bounded waits)
};

// True when a frame is built by the one-pass kernel (k_build_onepass): a
// context's frame (an error word for its bounded waits), no moment planes,
// bin-major or slab layout, bands of <= 32 rows, strips of 128 columns, at
// most 16 strips, several tiles, and at most 2^26 count cells, when
// IH_ONEPASS=1 is in the environment (read once): measured slower than the
// three-kernel build on the 640 x 480 frame, so it is off by default.
bool onepass_ok(const PlaneSet &ps);
// Small-frame build (k_small.cu): when a count-only frame in the bin-major
// or slab layout is small enough that every tile of a 128-column grid fits
// the GPU at once, picks the band height (ps.g) and rows per warp
// (ps.small) and returns true; the frame is then built by one cooperative
// launch.  IH_SMALL=0 in the environment (read once) turns it off.
bool small_plan(PlaneSet &ps);
// Scratch bytes of a small-frame build, and its carving.
size_t small_bytes(const PlaneSet &ps);
void carve_small(PlaneSet &ps, void *base);
// Rectangle queries answered by the small-frame build's own launch (after a
// second grid barrier): n x 4 rectangles in, n x B counts out.
struct SmallQuery {
    const int32_t *rects;
    int64_t n;
    int32_t *out;
};
// The small-frame build (a memset of the barrier counters unless
// ps.sm_zeroed, then one launch), with the frame's rectangle queries when
// `queries` is given; returns the number of kernels launched, or -1.
int launch_build_small(const PlaneSet &ps, cudaStream_t st, const Prof *prof, const SmallQuery *queries = nullptr);
// Bytes of carry scratch a plane set needs (0 for a single tile), and the
// carving of one scratch block into the carry arrays.
size_t carry_bytes(const PlaneSet &ps);
void carve_carries(PlaneSet &ps, void *base);

// Launchers (k_build.cu).  Return the number of kernels launched, or -1 with
// the CUDA error left pending.
int launch_build(const PlaneSet &ps, cudaStream_t st, const Prof *prof);
// One-time kernel attributes (shared-memory limits); call before a capture.
void prepare_kernels();
// The tile sums and the carry scan of a build alone (the first two kernels
// of launch_build); returns the number of kernels launched, or -1.
int launch_carries(const PlaneSet &ps, cudaStream_t st, const Prof *prof);
// The count tiles of a bin-major frame on 128 x 128 tiles (ps.g.Wc == 128,
// ps.g.R <= 128, no moment planes) as tcgen05 products (k_mma.cu), after
// launch_carries.  A bounded wait that gives up sets bit 2 of *err.
int launch_tiles_mma(const PlaneSet &ps, int *err, cudaStream_t st, const Prof *prof);

// Batched build: every kernel runs once over the concatenated work of n
// frames.  The prefix arrays (n + 1 entries, device) give each frame's first
// CTA / work item / warp unit of the five kernels.
struct BatchDev {
    const PlaneSet *sets;     // device, n entries
    int32_t n;
    const int64_t *pre_sums0; // tile sums, windows of unweighted channels (CTAs)
    const int64_t *pre_sums1; // tile sums, windows of the weighted channel (CTAs)
    const int64_t *pre_scan;  // carry-scan work items
    const int64_t *pre_tiles; // count-tile warp units
    const int64_t *pre_mom;   // moment-tile warp units
    int32_t max_R = kMaxBandRows;  // the frames' largest band (sizes the tile sums' shared memory)
};
// Work counts of one frame for the five batched kernels (host).
void batch_counts(const PlaneSet &ps, int64_t *counts5);

// Persistent batched build (k_build_persistent): a segment is `count` items
// of one kind of one frame starting at item `first` of that kind; the items
// of a launch are the segments in table order (tickets 0 .. total-1).
// Kinds: 0 weighted-channel tile sums (one window, one tile), 1 count tile
// sums (two (window, tile) units), 2 carry-scan chunks (256 scan items),
// 3 count tiles, 4 moment tiles (8 warp units each).
constexpr int kPersistKinds = 5;
struct PersistSeg {
    int32_t frame, kind;
    int64_t first, count;
};
struct PersistDev {
    const PlaneSet *sets;
    const PersistSeg *segs;
    const int64_t *seg_pre;  // [nsegs + 1] first ticket of each segment
    int32_t nsegs;
    int64_t total;           // items of the launch
    int32_t *done;           // [n][3] finished items per frame and phase (sums, scan, tiles); zero before the launch
    const int32_t *need;     // [n][3] items per frame and phase
    unsigned int *ticket;    // zero before the launch
    int *err;
};
// Items of each kind of one frame (host).
void persistent_counts(const PlaneSet &ps, int64_t *counts5);
// One thread waits (bounded, `limit` polls) for *never >= 1; it gives up and
// sets bit 2 of *err unless something raises the counter.
int launch_wait_selftest(const int32_t *never, long limit, int *err, cudaStream_t st);
// layout: the count layout of every frame, or -1 when the frames differ.
int launch_build_persistent(const PersistDev &pd, int layout, int max_R, cudaStream_t st, const Prof *prof);
// totals: the five totals over all frames (host).
int launch_build_batch(const BatchDev &bd, const int64_t *totals, cudaStream_t st, const Prof *prof);

// Feature pre-pass (k_features.cu): intensity and three orientation planes
// (and optionally a copy of R, G, B) from planar RGB.
int launch_features(const uint8_t *r, const uint8_t *g, const uint8_t *b, int64_t pitch, int H,
                    int W, uint8_t *out_rgb /* nullable: 3 planes */, uint8_t *out_i,
                    uint8_t *out_hog /* 3 planes */, int64_t out_pitch, cudaStream_t st,
                    const Prof *prof);

// The feature pre-pass's orientation table on the current device (once per
// device; synchronises the device, so call it outside stream capture).
void prepare_features();

// One frame of a batched feature pre-pass.
struct FeatJob {
    const uint8_t *r, *g, *b;
    int64_t pitch;
    int32_t H, W;
    uint8_t *out_i, *out_hog;  // intensity plane and 3 orientation planes
    int64_t opitch;
};
int64_t feature_tiles(int H, int W);  // CTAs of one frame
int launch_features_batch(const FeatJob *jobs, const int64_t *pre, int n, int64_t total, cudaStream_t st,
                          const Prof *prof);

// Read access to a count tensor in either layout (k_query.cu).
struct CountView {
    const int32_t *d;
    int32_t B, H, W, layout;
    int64_t P;
    int32_t ngroups;              // planes (LAYOUT_SLAB, LAYOUT_RECORD)
    int16_t bin_group[kMaxBins];  // global bin -> plane
    int16_t bin_local[kMaxBins];  // global bin -> word inside the plane's record
    int16_t group_nb[kMaxGroups]; // words per record of each plane
    int16_t group_bin0[kMaxGroups];  // LAYOUT_SLAB: first global bin of each plane
    int64_t slab_off[kMaxGroups];    // element offset of each plane
    // LAYOUT_RECORD: the concatenated records of all planes as nquarters
    // 4-word quarters; quarter k lies in plane quarter_plane[k] at word
    // 4k - plane_w0[plane]; word w holds global bin word_bin[w] (-1: padding)
    int32_t nquarters;
    int16_t plane_w0[kMaxGroups];
    int16_t quarter_plane[kMaxBins / 4];
    int16_t word_bin[kMaxBins];
};
struct MomentView {
    int32_t bin0;        // first bin of the weighted channel in the count tensor
    const int64_t *m;    // quads [Bw][H][P][4]: w = c, r, c^2, r^2 (uint32 when m32)
    int32_t Bw;
    int32_t m32;
};
int launch_query_rects(const CountView &v, const int32_t *rects, int64_t n, int32_t *out,
                       int *err, cudaStream_t st, const Prof *prof);
// Work items of one rectangle query (threads per rectangle): a 4-word
// quarter of the pixel record (record layout), a bin (bin-major) or a bin
// group (slab).
inline int64_t rect_items(const CountView &v)
{
    return v.layout == LAYOUT_RECORD ? v.nquarters : v.layout == LAYOUT_BIN_MAJOR ? v.B : v.ngroups;
}
// Queries of one frame of a batch (device table).
struct QueryJob {
    const CountView *v;   // device copy of the frame's view
    MomentView m;
    const int32_t *rects;
    int32_t *rect_out;
    const int32_t *wins;
    float *wout;
    int32_t normalize;
    int32_t kernel, layers;  // spatial kernel (WeightKernel) and wedding-cake layers
};
// pre_rects: rect work items (rects x groups), pre_wins: windows x Bw, per frame.
int launch_queries_batch(const QueryJob *jobs, const int64_t *pre_rects, const int64_t *pre_wins, int n,
                         int64_t total_rects, int64_t total_wins, int *err, cudaStream_t st, const Prof *prof);
int launch_query_weighted(const CountView &v, const MomentView &m, const int32_t *wins, int64_t n, int kernel,
                          int layers, int normalize, float *out, int *err, cudaStream_t st, const Prof *prof);
// Rectangle and weighted queries of one frame in one launch (either count may be 0).
int launch_query_both(const CountView &v, const MomentView &m, const int32_t *rects, int64_t nr, int32_t *rout,
                      const int32_t *wins, int64_t nw, int kernel, int layers, int normalize, float *wout, int *err,
                      cudaStream_t st, const Prof *prof);
// Sliding-window city-block distances (Eq. 2.22, p = 1) over bins
// [bin0, bin0 + nbins) for placements [sr0, sr1] x [sc0, sc1] of a wh x ww window.
int launch_match_window(const CountView &v, int bin0, int nbins, const int32_t *target, int wh, int ww, int sr0,
                        int sc0, int sr1, int sc1, int32_t *out, cudaStream_t st, const Prof *prof);
// dst[i] += add[i] - sub[i] over n int32 words (add / sub may be null).
int launch_accumulate(int32_t *dst, const int32_t *add, const int32_t *sub, int64_t n, cudaStream_t st,
                      const Prof *prof);
// Lower-median bin of each pixel's m x n box over bins [bin0, bin0 + nbins).
int launch_local_median(const CountView &v, int bin0, int nbins, int m, int n, int32_t *out, cudaStream_t st,
                        const Prof *prof);
// Spatial pyramids of gradient orientations (k_phog.cu, Algorithm 2).
constexpr int kPhogBins = 9;
constexpr int kPhogMaxLevels = 4;  // descriptors of at most 9 * 341 entries
inline int64_t phog_descriptor_len(int L)
{
    int64_t n = 0;
    for (int l = 0; l <= L; ++l) n += (int64_t)kPhogBins << (2 * l);
    return n;
}
// Scratch of Canny's detector on an H x W window: union-find parents
// (int32), survivor classes and root marks (uint8), H x W each.
struct CannyScratch {
    int32_t *parent;
    uint8_t *cls;
    uint8_t *mark;
};
size_t canny_scratch_bytes(int H, int W);
CannyScratch carve_canny(void *base, int H, int W);
// Algorithm 2 step 1 alone: Canny edge pixels (1) of the window into edges
// (row pitch epitch bytes), thresholds lo <= hi on |G| / 256.  A pointer
// walk that gives up sets bit 2 of *err.  Returns launches or -1.
int launch_canny_edges(const uint8_t *gray, int64_t pitch, int H, int W, int lo, int hi, const CannyScratch &cs,
                       uint8_t *edges, int64_t epitch, int *err, cudaStream_t st, const Prof *prof);
// Steps 1-4: Canny edges, orientation bins and magnitude weights of the edge
// pixels (scratch, h x w each) and the weighted integral histogram ih:
// kPhogBins x H x P int64.  Returns launches or -1.
int launch_phog_build(const uint8_t *gray, int64_t pitch, int H, int W, int lo, int hi, const CannyScratch &cs,
                      uint8_t *bins, int32_t *wt, int64_t P, int64_t *ih, int *err, cudaStream_t st,
                      const Prof *prof);
int launch_phog_descriptors(const int64_t *ih, int H, int W, int64_t P, int L, const int32_t *wins, int64_t n,
                            int64_t *out, int *err, cudaStream_t st, const Prof *prof);
int launch_phog_match(const int64_t *ih, int H, int64_t P, int L, const int64_t *target, int wh, int ww, int sr0,
                      int sc0, int sr1, int sc1, float *out, cudaStream_t st, const Prof *prof);
// Count tensor -> packed bin-major B x H x W int32.
int launch_export(const CountView &v, int32_t *dst, cudaStream_t st, const Prof *prof);
// Moment plane k (entry k of the quads [Bw][H][P][4], int64 or uint32 when
// m32) -> packed Bw x H x W int64.
int launch_export_moments(const void *m, int m32, int Bw, int H, int W, int64_t P, int k, int64_t *dst,
                          cudaStream_t st, const Prof *prof);

}  // namespace ih
