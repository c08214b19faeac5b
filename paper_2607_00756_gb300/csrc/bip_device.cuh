// Device helpers shared by several kernels of the map path.
#pragma once

#include <cuda_runtime.h>

// Crop mask of Sec. 2.2.4: a site at pixel position (ty, tx) contributes to
// the scan at (ry, rx) when the minimum-image offset lies in
// [-N/(2f), N/(2f)) on both axes.  FP64 so the decision matches a host
// FP64 evaluation of the same formula.
__device__ __forceinline__ bool in_crop(double ry, double rx, double ty, double tx, int ny, int nx, int fy,
                                        int fx) {
    double d = ry - ty;
    d -= ny * floor((d + 0.5 * ny) / ny);
    const double hy = 0.5 * ny / fy;
    if (!(d >= -hy && d < hy)) return false;
    d = rx - tx;
    d -= nx * floor((d + 0.5 * nx) / nx);
    const double hx = 0.5 * nx / fx;
    return d >= -hx && d < hx;
}

// x mod n in [0, n) for any sign of x (grid lengths need not be powers of
// two: 3 M lengths are allowed).
__device__ __forceinline__ int wrap_n(int x, int n) {
    if ((n & (n - 1)) == 0) return x & (n - 1);   // a power of two: a mask (two's complement)
    const int r = x % n;
    return r < 0 ? r + n : r;
}
