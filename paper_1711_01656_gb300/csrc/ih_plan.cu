// ih_plan.cu -- see ih_plan.h.
#include "ih_plan.h"

namespace ih {

namespace {
constexpr int kWarpsPerSm = 16;

int cdiv(int a, int b) { return (a + b - 1) / b; }
}  // namespace

TileGrid choose_grid(int H, int W, int B, int kind, int nsm)
{
    const int per_group = (kind == WK_ONE) ? 8 : 4;
    const int groups = cdiv(B, per_group);
    static const int kR[] = {128, 64, 32};
    static const int kWc[] = {1024, 512, 256, 128};
    TileGrid g{};
    g.H = H;
    g.W = W;
    int bestR = 32, bestWc = kChunk;
    bool found = false;
    for (int R : kR) {
        for (int Wc : kWc) {
            const int r = R < H ? R : H;
            const int wc = Wc < cdiv(W, kChunk) * kChunk ? Wc : cdiv(W, kChunk) * kChunk;
            const long long units = (long long)cdiv(H, r) * cdiv(W, wc) * groups;
            if (units >= (long long)kWarpsPerSm * nsm) {
                bestR = r;
                bestWc = wc;
                found = true;
                break;
            }
        }
        if (found) break;
    }
    if (!found) {
        bestR = H < 32 ? H : 32;
        bestWc = kChunk;
    }
    g.R = bestR;
    g.Wc = bestWc;
    g.nb = cdiv(H, g.R);
    g.ns = cdiv(W, g.Wc);
    return g;
}

}  // namespace ih
