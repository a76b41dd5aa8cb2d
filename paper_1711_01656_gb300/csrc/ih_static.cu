// ih_static.cu -- ih_build_counts_static: the count build of one channel
// without any device allocation.
//
// Who needs it: callers that must not allocate device memory once they are
// running -- a real-time tracking loop whose device memory is reserved up
// front by its own arena (a cudaMalloc there would synchronise the device and
// stall every stream), or a host application whose allocator owns all device
// memory.  ih_build allocates its tensors and its carry scratch from a
// context's memory pool; this entry point writes into the caller's buffer and
// keeps the carries (column, row and corner sums of the tiles) in one
// statically sized device array of this library.
//
// The array lives in every GPU that loads the library until the process
// exits.  The first call made on each device (with that device current) does
// the set-up: it looks up the array's device address with
// cudaGetSymbolAddress and caches it, and it prepares the build kernels once
// for the device (shared-memory limits, and the feature pre-pass's table,
// whose fill synchronises the device).  Make that first call before any
// stream capture begins and outside a loop that must not stall; later calls
// only enqueue kernels.  This call takes the same kernel path as ih_build
// on the same frame (a uniform channel takes the folded bin rule).  Every call
// shares the array: calls whose work overlaps on the GPU (on different
// streams, or on one device from several threads) race on it.  Every carry
// cell a call reads is written earlier by the same call, so nothing needs
// clearing between calls.
#include <mutex>

#include "../../include/ih.h"
#include "ih_internal.cuh"
#include "ih_plan.h"

using namespace ih;

namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // IH_STATIC_SCRATCH_BYTES
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {nullptr};

cudaError_t static_scratch_address(int dev, void **out)
{
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        prepare_kernels();
        const cudaError_t e2 = cudaGetLastError();
        if (e2 != cudaSuccess) return e2;
        g_static_addr[dev] = p;
    }
    *out = g_static_addr[dev];
    return cudaSuccess;
}

int split_groups(int bins, int cap, GroupDev *out)
{
    const int ng = (bins + cap - 1) / cap;
    for (int g = 0; g < ng; ++g) {
        out[g] = GroupDev{};
        out[g].b_lo = (int16_t)(bins * g / ng);
        out[g].nb = (int16_t)(bins * (g + 1) / ng - bins * g / ng);
    }
    return ng;
}

}  // namespace

extern "C" ih_status ih_build_counts_static(const uint8_t *d_pixels, int32_t height, int32_t width,
                                            int64_t pitch_bytes, int32_t bins, int32_t mode,
                                            int32_t *d_out, int64_t out_pitch, void *stream)
{
    if (!d_pixels || !d_out || height < 1 || width < 1 || pitch_bytes < width || bins < 1 || bins > 256 ||
        (mode != IH_BIN_UNIFORM8 && mode != IH_BIN_INDEX) || out_pitch < width || (out_pitch & 3) ||
        (reinterpret_cast<uintptr_t>(d_out) & 15) || (int64_t)height * width > ((int64_t)1 << 31))
        return IH_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IH_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return IH_ECUDA;

    PlaneSet ps{};
    ps.B = bins;
    ps.nchan = 1;
    ps.layout = LAYOUT_BIN_MAJOR;
    ps.wch = -1;
    ps.chan[0].plane = d_pixels;
    ps.chan[0].pitch = pitch_bytes;
    ps.chan[0].bins = bins;
    ps.chan[0].mode = mode;
    ps.chan[0].bin_off = 0;
    ps.uni = (mode == IH_BIN_UNIFORM8) ? 1 : 0;
    // groups by size, largest first (one tiles launch per size)
    GroupDev tmp[kMaxGroups];
    const int ng = split_groups(bins, kGroupBins, tmp);
    ps.ngroups = 0;
    for (int size = kGroupBins; size >= 1; --size)
        for (int k = 0; k < ng; ++k)
            if (tmp[k].nb == size) ps.grp[ps.ngroups++] = tmp[k];
    ps.nwin = split_groups(bins, kWindowBins, ps.win);
    ps.nwin_count = ps.nwin;
    ps.g = choose_grid(height, width, ps.ngroups, nsm);
    if (carry_bytes(ps) > kStaticScratchBytes) ps.g = make_grid(height, width, kMaxBandRows, 1024);
    if (carry_bytes(ps) > kStaticScratchBytes) return IH_ETOOBIG;
    ps.g.P = out_pitch;
    ps.out = d_out;
    void *base = nullptr;
    if (static_scratch_address(dev, &base) != cudaSuccess) return IH_ECUDA;
    if (!carry_bytes(ps)) base = nullptr;
    carve_carries(ps, base);
    if (launch_build(ps, static_cast<cudaStream_t>(stream), nullptr) < 0) return IH_ECUDA;
    return IH_OK;
}
