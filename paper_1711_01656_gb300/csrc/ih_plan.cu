// ih_plan.cu -- see ih_plan.h.
#include "ih_plan.h"

namespace ih {

namespace {
constexpr int kWarpsPerSm = 16;
constexpr int kBatchR = 128, kBatchWc = 512;  // tiles of a batch that fills the GPU

int cdiv(int a, int b) { return (a + b - 1) / b; }
}  // namespace

TileGrid make_grid(int H, int W, int R, int Wc)
{
    TileGrid g{};
    g.H = H;
    g.W = W;
    const int wmax = cdiv(W, kChunk) * kChunk;
    g.R = R < H ? R : H;
    if (g.R > kMaxBandRows) g.R = kMaxBandRows;
    if (g.R < 1) g.R = 1;
    Wc = cdiv(Wc < kChunk ? kChunk : Wc, kChunk) * kChunk;
    g.Wc = Wc < wmax ? Wc : wmax;
    g.nb = cdiv(H, g.R);
    g.ns = cdiv(W, g.Wc);
    return g;
}

TileGrid choose_grid(int H, int W, int groups, int nsm)
{
    // the largest tiles that still give every SM kWarpsPerSm warp units;
    // frames too small for that take the smallest tiles (8 x 128: shorter
    // per-warp row chains, measured 45 -> 43 us for a 640x480 frame)
    static const int kR[] = {128, 64, 32, 16, 8};
    static const int kWc[] = {1024, 512, 256, 128};
    for (int R : kR)
        for (int Wc : kWc) {
            const TileGrid g = make_grid(H, W, R, Wc);
            if ((long long)g.nb * g.ns * groups >= (long long)kWarpsPerSm * nsm) return g;
        }
    return make_grid(H, W, 8, kChunk);
}

void batch_grids(PlaneSet *sets, int n, int nsm)
{
    // a batch whose frames, cut into the largest tiles, still give every SM
    // 4 x kWarpsPerSm warp units runs all of them on those tiles: the frames
    // supply the parallelism, and large tiles carry less (the 64-frame FMV
    // batch: 35.1 ms with per-shape tuned tiles, 32.8 ms with 128 x 512)
    long long units = 0;
    if (n == 1 && sets[0].small) return;  // a single small frame keeps its own grid
    for (int k = 0; k < n; ++k) {
        const TileGrid g = make_grid(sets[k].g.H, sets[k].g.W, kBatchR, kBatchWc);
        units += (long long)g.nb * g.ns * sets[k].ngroups;
    }
    if (units < 4LL * kWarpsPerSm * nsm) return;
    for (int k = 0; k < n; ++k) {
        const int64_t P = sets[k].g.P;
        sets[k].g = make_grid(sets[k].g.H, sets[k].g.W, kBatchR, kBatchWc);
        sets[k].g.P = P;
    }
}

}  // namespace ih
