// ih_ctx.h -- the context behind the C ABI (private to the library).
#pragma once

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ih.h"
#include "ih_internal.cuh"

namespace ih {

struct FrameRec {
    bool live = false;
    int H = 0, W = 0, nchan = 0, B = 0;
    int bins[kMaxChannels] = {0};
    int bin_off[kMaxChannels] = {0};
    int64_t P = 0;
    int32_t *d_ih = nullptr;
    int wch = -1, Bw = 0, mbits = 64;
    int64_t *d_mom = nullptr;  // int64 or uint32 planes (mbits)
    int64_t count_bytes = 0, moment_bytes = 0;
    int R = 0, Wc = 0;  // tile grid used by the build
    bool phog = false;  // d_mom holds Algorithm 2's 9 weighted planes; no count tensor
    CountView view{};
};

struct ProfRec {
    int kid;
    cudaEvent_t a, b;
};

}  // namespace ih

struct ih_ctx {
    std::map<std::string, std::pair<int, int>> tuned;  // shape key -> (band rows, strip columns)
    int device = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<ih::ProfRec> prof_pending;
    int prof_open_kid = -1;
    cudaEvent_t prof_open = nullptr;
    int64_t prof_launches[ih::KID_COUNT] = {0};
    double prof_ms[ih::KID_COUNT] = {0};
    ih::Prof prof;
    uint32_t prof_mask = ~0u;  // kernel ids (bits) that get event pairs
    uint64_t budget = 0;
    uint64_t used = 0;
    cudaMemPool_t pool = nullptr;
    std::vector<ih::FrameRec> frames;
    int *d_err = nullptr;
    std::recursive_mutex mu;
    std::string last_error;
    int64_t launches = 0;
    int nsm = 0;
};


namespace ih {

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <typename T>
cudaError_t pool_alloc(ih_ctx *ctx, T **p, size_t bytes, cudaStream_t st)
{
    void *v = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&v, bytes ? bytes : 16, ctx->pool, st);
    *p = static_cast<T *>(v);
    return e;
}

ih_status fail(ih_ctx *ctx, ih_status s, const char *fmt, ...);
ih_status cuda_fail(ih_ctx *ctx, cudaError_t e, const char *what);
const Prof *prof_of(ih_ctx *ctx);
ih_status validate(ih_ctx *ctx, const ih_frame &f);
// Wedding-cake layers from ih_query_weighted's flags (IH_LAYERS field, 0 -> 4).
inline int weighted_layers(uint32_t flags)
{
    const int l = (int)((flags >> 8) & 0xffu);
    return l ? l : 4;
}
// LAYOUT_RECORD groups and planes of a frame's channels (ih_capi.cu).
int record_plan(const int *bins, int nchan, GroupDev *sp, int max_sp, int16_t *rec_w, int *nplanes, int *words);
// Geometry, byte sizes and bin offsets of a valid frame descriptor.
void frame_record(const ih_frame &f, FrameRec &fr);
// The plane set of one frame: channels, bin groups, tile grid (tuned if the
// context has a tuned grid for this shape), slab offsets, outputs.  Carries
// are left null.  small: a single frame that may take the small-frame build
// (one cooperative launch, small_plan) when it qualifies.
bool make_planeset(ih_ctx *ctx, const ih_frame &f, const FrameRec &fr, const uint8_t *const *planes,
                   const int64_t *cpitch, PlaneSet &ps, bool small = false);
std::string shape_key(const ih_frame &f);
void make_view(const PlaneSet &ps, const int32_t *d, CountView &v);
FrameRec *get_frame(ih_ctx *ctx, int32_t handle);
// A live frame with a count tensor (not a pyramid frame), else null.
FrameRec *count_frame(ih_ctx *ctx, int32_t handle);
int publish_frame(ih_ctx *ctx, FrameRec &fr);  // registers a built frame, returns its handle

}  // namespace ih
