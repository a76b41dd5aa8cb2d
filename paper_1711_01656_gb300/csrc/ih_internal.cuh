// ih_internal.cuh -- descriptors shared by the engine's kernels and its C ABI.
//
// A "plane set" is one weighted integral histogram (Eq. 3.4) over a set of
// channels: the count tensor (w = 1, Eq. 2.15 / Algorithm 5) or one of the
// four moment planes w in {c, r, c^2, r^2} of the weighted channel.  Every
// plane set is built by the same three kernels over a grid of tiles of R
// rows (a band) by Wc columns (a strip):
//
//   tile sums  : per tile and bin, the column sums over the band's rows and
//                the row sums over the strip's columns (reads pixels only);
//   carry scan : exclusive prefixes of those sums over bands (G), over
//                strips (L) and over both (corner);
//   tiles      : per tile and bin group, the 2-D inclusive prefix of the
//                tile, seeded with its carries, written once.
//
// With tile origin (R0, C0):
//   H(r,c) = corner + sum_{C0<=c'<=c} G(c')
//          + sum_{R0<=r'<=r} ( L(r') + sum_{C0<=c'<=c} w(r',c') Q(r',c') )
// which is Eq. 2.15 split at the tile's top and left edges.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ih {

constexpr int kMaxChannels = 16;
constexpr int kMaxGroups = 128;
constexpr int kChunk = 128;      // columns a warp covers at once (4 per lane)
constexpr int kMaxBandRows = 128;

enum WeightKind { WK_ONE = 0, WK_COL = 1, WK_ROW = 2, WK_COL2 = 3, WK_ROW2 = 4 };

// Kernel ids for the optional per-launch event timing.  Plane-set kernels
// of weight kind k have ids kid_sums(k), kid_scan(k), kid_tiles(k).
enum KernelId { KID_FEATURES = 0, KID_QUERY_RECTS = 16, KID_QUERY_WEIGHTED = 17, KID_COUNT = 18 };
inline int kid_sums(int kind) { return 1 + 3 * kind; }
inline int kid_scan(int kind) { return 2 + 3 * kind; }
inline int kid_tiles(int kind) { return 3 + 3 * kind; }

// Optional launch hook: mark(ctx, kid, 0, st) is called before a kernel is
// launched on st and mark(ctx, kid, 1, st) right after.
struct Prof {
    void *ctx;
    void (*mark)(void *ctx, int kid, int phase, cudaStream_t st);
};
inline void prof_mark(const Prof *p, int kid, int phase, cudaStream_t st)
{
    if (p && p->mark) p->mark(p->ctx, kid, phase, st);
}

struct ChanDev {
    const uint8_t *plane;  // row r starts at plane + r * pitch
    int64_t pitch;
    int32_t bins;          // bins of the channel
    int32_t mode;          // 0: uniform over [0,256), 1: value is the bin
    int32_t bin_off;       // first bin of the channel inside the plane set
    int32_t pad;
};

struct GroupDev {  // bins [b_lo, b_lo + nb) of channel `chan` (channel-local)
    int16_t chan, b_lo, nb, pad;
};

struct TileGrid {
    int32_t H, W;      // frame
    int32_t R, Wc;     // band rows, strip columns (Wc % kChunk == 0)
    int32_t nb, ns;    // number of bands, strips
    int64_t P;         // row pitch of the output, elements (multiple of 4)
};

struct PlaneSet {
    TileGrid g;
    int32_t B;          // bins of the plane set
    int32_t nchan;
    ChanDev chan[kMaxChannels];
    int32_t ngroups;    // bin groups of the tiles kernel
    int32_t npgroups;   // bin windows of the tile-sums kernel
    GroupDev grp[kMaxGroups];
    GroupDev pgrp[kMaxGroups];
    void *out;          // T [B][H][P]
    void *colsum;       // T [nb][B][W]   column sums -> G after the scan
    void *rowsum;       // T [ns][B][H]   row sums    -> L after the scan
    void *tilesum;      // T [nb][ns][B]
    void *corner;       // T [nb][ns][B]
};

// Launchers (k_build.cu).  Each returns the number of kernels launched, or
// -1 with the CUDA error left pending.
int launch_plane_set(const PlaneSet &ps, int kind, cudaStream_t st, const Prof *prof);
size_t tile_sums_smem_bytes(const PlaneSet &ps, int kind);

// Feature pre-pass (k_features.cu): intensity and three orientation planes
// (and optionally a copy of R, G, B) from planar RGB.
int launch_features(const uint8_t *r, const uint8_t *g, const uint8_t *b, int64_t pitch, int H,
                    int W, uint8_t *out_rgb /* nullable: 3 planes */, uint8_t *out_i,
                    uint8_t *out_hog /* 3 planes */, int64_t out_pitch, cudaStream_t st,
                    const Prof *prof);

// Queries (k_query.cu).
struct CountView {
    const int32_t *d;  // [B][H][P]
    int32_t B, H, W;
    int64_t P;
};
struct MomentView {
    const int32_t *n;    // count planes of the weighted channel [Bw][H][P]
    const int64_t *m;    // [4][Bw][H][P]: w = c, r, c^2, r^2
    int32_t Bw, H, W;
    int64_t P;
};
int launch_query_rects(const CountView &v, const int32_t *rects, int64_t n, int32_t *out,
                       int *err, cudaStream_t st, const Prof *prof);
int launch_query_weighted(const MomentView &v, const int32_t *wins, int64_t n, int normalize,
                          float *out, int *err, cudaStream_t st, const Prof *prof);

}  // namespace ih
