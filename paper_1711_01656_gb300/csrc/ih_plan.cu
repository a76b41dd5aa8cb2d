// ih_plan.cu -- see ih_plan.h.
#include "ih_plan.h"

namespace ih {

namespace {
constexpr int kWarpsPerSm = 16;

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

}  // namespace ih
