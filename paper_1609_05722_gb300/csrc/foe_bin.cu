// Binning variant of the denoiser (FoEPNRbin, Sec. 4): a 3x3 ones kernel sums the counts of each bin before the
// solve (nine times the peak, on a ninth of the pixels), and bilinear interpolation brings the estimate back to
// full size after it.  Bins are the non-overlapping 3x3 blocks from pixel (0, 0); a bin cut by the image border
// (n < 9 pixels) is scaled by 9 / n.  The estimate at pixel (r, c) interpolates the bin image at
// ((r - 1) / 3, (c - 1) / 3) (bin (I, J) is centred on pixel (3I + 1, 3J + 1)), clamped to the edge bins, and is
// divided by 9.  Both kernels are memory-bound passes over the image (4 B read + 4/9 B written per pixel, and the
// reverse), negligible next to the solve.
#include <algorithm>

#include "foe_common.cuh"
#include "foe_kernels.h"

namespace foe {

namespace {

constexpr int kBinThreads = 128;

// one thread per bin (rows by a grid-stride loop over blockIdx.y)
__global__ void k_bin3(const float *__restrict__ y, int H, int W, int ld, float *__restrict__ yb, int Hb, int Wb,
                       int ldb)
{
    const int J = blockIdx.x * blockDim.x + threadIdx.x;
    if (J >= Wb) return;
    for (int I = blockIdx.y; I < Hb; I += gridDim.y) {
        const int r0 = 3 * I, c0 = 3 * J, nr = min(3, H - r0), nc = min(3, W - c0);
        float s = 0.0f;
        for (int a = 0; a < nr; ++a)
            for (int b = 0; b < nc; ++b) s += y[(size_t)(r0 + a) * ld + c0 + b];
        const int n = nr * nc;
        yb[(size_t)I * ldb + J] = n == 9 ? s : s * 9.0f / (float)n;
    }
}

// one thread per output pixel.  r - 1 = 3q + m (m in 0..2): bins q and q + 1 with weights (3 - m) / 3 and m / 3.
__global__ void k_upscale3(const float *__restrict__ xb, int Hb, int Wb, int ldb, float *__restrict__ x, int H, int W,
                           int ld)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= W) return;
    const int qx = (c + 2) / 3 - 1, mx = c - 1 - 3 * qx;
    const int xa = min(max(qx, 0), Wb - 1), xc = min(max(qx + 1, 0), Wb - 1);
    const float wx = (float)mx * (1.0f / 3.0f);
    for (int r = blockIdx.y; r < H; r += gridDim.y) {
        const int qy = (r + 2) / 3 - 1, my = r - 1 - 3 * qy;
        const int ya = min(max(qy, 0), Hb - 1), yc = min(max(qy + 1, 0), Hb - 1);
        const float wy = (float)my * (1.0f / 3.0f);
        const float *ra = xb + (size_t)ya * ldb, *rc = xb + (size_t)yc * ldb;
        const float top = (1.0f - wx) * ra[xa] + wx * ra[xc];
        const float bot = (1.0f - wx) * rc[xa] + wx * rc[xc];
        x[(size_t)r * ld + c] = ((1.0f - wy) * top + wy * bot) * (1.0f / 9.0f);
    }
}

}  // namespace

cudaError_t launch_bin3(const float *y, int H, int W, int ld, float *yb, int ldb, cudaStream_t s)
{
    const int Hb = (H + 2) / 3, Wb = (W + 2) / 3;
    if (Hb <= 0 || Wb <= 0) return cudaSuccess;
    const dim3 grid((Wb + kBinThreads - 1) / kBinThreads, std::min(Hb, 65535));
    k_bin3<<<grid, kBinThreads, 0, s>>>(y, H, W, ld, yb, Hb, Wb, ldb);
    return cudaGetLastError();
}

cudaError_t launch_upscale3(const float *xb, int ldb, float *x, int H, int W, int ld, cudaStream_t s)
{
    const int Hb = (H + 2) / 3, Wb = (W + 2) / 3;
    if (H <= 0 || W <= 0) return cudaSuccess;
    const dim3 grid((W + kBinThreads - 1) / kBinThreads, std::min(H, 65535));
    k_upscale3<<<grid, kBinThreads, 0, s>>>(xb, Hb, Wb, ldb, x, H, W, ld);
    return cudaGetLastError();
}

}  // namespace foe
