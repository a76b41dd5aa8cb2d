// ih_orient.cuh -- the unsigned 9-bin gradient orientation of an integer
// gradient (Fig. 2.3, Algorithm 2), decided exactly in int32 (private to the
// library; the derivation of the test is in k_features.cu's header).
#pragma once

namespace ih {

namespace {

// round(2^22 cos(20j deg)), round(2^22 sin(20j deg)), j = 1..4
__constant__ int kUx[4] = {3941357, 3213023, 2097152, 728333};
__constant__ int kUy[4] = {1434536, 2696047, 3632374, 4130583};

__device__ __forceinline__ int orientation_bin9(int gx, int gy)
{
    if (gy < 0 || (gy == 0 && gx < 0)) {
        gx = -gx;
        gy = -gy;
    }
    if ((gx | gy) == 0) return 0;
    const int ax = gx < 0 ? -gx : gx;
    int n = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) n += (kUx[k] * gy - kUy[k] * ax >= 0) ? 1 : 0;
    return gx < 0 ? 8 - n : n;
}

}  // namespace

}  // namespace ih
