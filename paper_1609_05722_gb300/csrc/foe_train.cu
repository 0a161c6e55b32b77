// Backward pass of the unrolled iPiano solve (training of the FoE prior, Sec. 2.5; loss of Sec. 3.2), FP32.
// With hvp_only set, the same kernel is the Hessian-vector product of the implicit-differentiation gradient:
// tau = -1, gamma = lambda - 1, c1 = 1 and no gbar^{n+2} give gout = lambda w + H(u) w = H_E(u) w.
//
// One launch handles one step n of the reverse sweep for a batch of images.  With w = c1 gbar^{n+1}
// (c1 = 1/(1 + tau lambda), the derivative of the quadratic prox of Eq. subproblemGL2), each CTA computes
// on its 32x32 output tile:
//   r_i = K_i u^n and s_i = K_i w on the tile plus a 3-pixel ring (two forward convolutions),
//   the Hessian-vector product H(u^n) w = sum_i alpha_i K_i^T (rho''(r_i) s_i)  (Sec. 2.5.2),
//   gbar^n = (1 + gamma) w - tau H(u^n) w - gamma c1 gbar^{n+2}                   (unrolled Eq. iPianoupdate),
// and per-tile partial sums of the parameter gradients (before the factor -tau alpha_i):
//   G_i(a, b) = sum_p [ (P w)(p + (a, b)) rho'(r_i(p)) + s_i(p) rho''(r_i(p)) (P u^n)(p + (a, b)) ]
//               (correlation orientation, over the tile's own pixels),
//   A_i       = sum_p s_i(p) rho'(r_i(p)).
// The filter gradient is computed by the warps in parallel, one filter per warp and one column per lane:
// each padded input row's 7-tap windows of w and u are loaded once and serve all 7 tap rows.
#include "foe_common.cuh"
#include "foe_kernels.h"

namespace foe {

namespace {

constexpr int T = 32;
constexpr int UROWS = 44, UCOLS = 48;
constexpr int R0 = 6, C0 = 7;
constexpr int PLANE = UROWS * UCOLS;
constexpr int CH = 8;
constexpr int NTHREADS = 256;
constexpr int RESP_ROWS = T + 6;
constexpr int RESP_STRIPS_X = (T + 8) / 2;

struct BwdSmem {
    float u[PLANE];             // P u^n on tile-relative rows [-6, 38), cols [-7, 41)
    float w[PLANE];             // P w   (w = c1 gbar^{n+1})
    float psi[CH * PLANE];      // rho''(r) s / 2 on the response region, zero elsewhere
    float A[CH][T * T];         // rho'(r) at the tile's own pixels (0 outside the image)
    float B[CH][T * T];         // s rho''(r) at the tile's own pixels
    float wf[6 * kKK * CH];     // forward weights [chunk][tap][8 filters]
    float wa[kNF * kKS * 8];    // adjoint weights 2 alpha_i w_i(a, b)
    float ared[NTHREADS / 32][CH];
};

__device__ float ring_gather_b(const BwdSmem &S, int chunk, int qy, int qx, int ty0, int tx0, int H, int W)
{
    float h = 0.0f;
    for (int c = 0; c < CH; ++c) {
        const int fi = chunk * CH + c;
        for (int a = 0; a < kKS; ++a) {
            const int py = qy - (a - kR);
            const int gy = ty0 + py;
            if (gy < 0 || gy >= H || py < -R0 || py >= UROWS - R0) continue;
            for (int b = 0; b < kKS; ++b) {
                const int px = qx - (b - kR);
                const int gx = tx0 + px;
                if (gx < 0 || gx >= W || px < -C0 || px >= UCOLS - C0) continue;
                h = fmaf(S.wa[(fi * kKS + a) * 8 + b], S.psi[c * PLANE + (py + R0) * UCOLS + (px + C0)], h);
            }
        }
    }
    return h;
}

__global__ void __launch_bounds__(NTHREADS, 1) k_foe_bwd(const __grid_constant__ BwdArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem &S = *reinterpret_cast<BwdSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x;
    int im = 0;
    {
        int lo = 0, hi = A.nimg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (A.tile_prefix[mid] <= tile) lo = mid;
            else hi = mid - 1;
        }
        im = lo;
    }
    const BwdImg &D = A.img[im];
    const int lt = tile - A.tile_prefix[im];
    const int ty0 = (lt / D.tiles_x) * T, tx0 = (lt % D.tiles_x) * T;
    const int H = D.H, W = D.W, ld = D.ld;
    float *part = A.hvp_only ? nullptr : A.partials + (size_t)tile * kBwdPartials;

    for (int j = tid; j < 6 * kKK * CH; j += NTHREADS) {
        const int c = j / (kKK * CH), t = (j / CH) % kKK, f = j % CH;
        S.wf[j] = A.wts[(c * CH + f) * kKK + t];
    }
    for (int j = tid; j < kNF * kKS * 8; j += NTHREADS) {
        const int f = j / (kKS * 8), a = (j / 8) % kKS, b = j % 8;
        S.wa[j] = b < kKS ? 2.0f * A.alpha[f] * A.wts[f * kKK + a * kKS + b] : 0.0f;
    }
    for (int j = tid; j < PLANE; j += NTHREADS) {
        const int r = j / UCOLS, c = j % UCOLS;
        const int sy = pad_index(ty0 + r - R0, H, A.bc), sx = pad_index(tx0 + c - C0, W, A.bc);
        const bool z = sy < 0 || sx < 0;
        const size_t idx = (size_t)sy * ld + sx;
        S.u[j] = z ? 0.0f : D.u[idx];
        S.w[j] = z ? 0.0f : A.c1 * D.gb1[idx];
    }
    for (int j = tid; j < CH * PLANE; j += NTHREADS) S.psi[j] = 0.0f;
    __syncthreads();

    const int oy = tid / 8, ox0 = (tid % 8) * 4;
    const bool ring_tile = (A.bc == kSymmetric) && (ty0 < kR || tx0 < kR || ty0 + T > H - kR || tx0 + T > W - kR);
    float h[4] = {0.f, 0.f, 0.f, 0.f}, hr[4] = {0.f, 0.f, 0.f, 0.f};

    for (int ch = 0; ch < A.nchunks; ++ch) {
        float aacc[CH];
#pragma unroll
        for (int f = 0; f < CH; ++f) aacc[f] = 0.0f;
        // ---- responses of u and w, rho', rho'' ----
        for (int s = tid; s < RESP_ROWS * RESP_STRIPS_X; s += NTHREADS) {
            const int ry = s / RESP_STRIPS_X - kR, rx0 = (s % RESP_STRIPS_X) * 2 - 4;
            float ru0[CH], ru1[CH], rw0[CH], rw1[CH];
#pragma unroll
            for (int f = 0; f < CH; ++f) ru0[f] = ru1[f] = rw0[f] = rw1[f] = 0.0f;
#pragma unroll 1
            for (int a = 0; a < kKS; ++a) {
                const float *urow = &S.u[(ry + a - kR + R0) * UCOLS + (rx0 - kR + C0)];
                const float *wrow = &S.w[(ry + a - kR + R0) * UCOLS + (rx0 - kR + C0)];
                float vu[8], vw[8];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 q = *reinterpret_cast<const float2 *>(urow + 2 * j);
                    const float2 e = *reinterpret_cast<const float2 *>(wrow + 2 * j);
                    vu[2 * j] = q.x;
                    vu[2 * j + 1] = q.y;
                    vw[2 * j] = e.x;
                    vw[2 * j + 1] = e.y;
                }
#pragma unroll
                for (int b = 0; b < kKS; ++b) {
                    const float *wp = &S.wf[(ch * kKK + a * kKS + b) * CH];
                    const float4 w0 = *reinterpret_cast<const float4 *>(wp);
                    const float4 w1 = *reinterpret_cast<const float4 *>(wp + 4);
                    const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                    for (int f = 0; f < CH; ++f) {
                        ru0[f] = fmaf(wv[f], vu[b], ru0[f]);
                        ru1[f] = fmaf(wv[f], vu[b + 1], ru1[f]);
                        rw0[f] = fmaf(wv[f], vw[b], rw0[f]);
                        rw1[f] = fmaf(wv[f], vw[b + 1], rw1[f]);
                    }
                }
            }
            const int gy = ty0 + ry;
#pragma unroll
            for (int px = 0; px < 2; ++px) {
                const int rx = rx0 + px, gx = tx0 + rx;
                const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
                const bool own = ry >= 0 && ry < T && rx >= 0 && rx < T;
#pragma unroll
                for (int f = 0; f < CH; ++f) {
                    const float r = px ? ru1[f] : ru0[f];
                    const float sv = px ? rw1[f] : rw0[f];
                    const float q = fmaf(r, r, 1.0f);
                    const float iq = 1.0f / q;
                    const float rho1 = 2.0f * r * iq;                     // rho'(r)
                    const float rho2 = 2.0f * (1.0f - r * r) * iq * iq;    // rho''(r)
                    S.psi[f * PLANE + (ry + R0) * UCOLS + (rx + C0)] = in ? 0.5f * rho2 * sv : 0.0f;
                    if (own) {
                        S.A[f][ry * T + rx] = in ? rho1 : 0.0f;
                        S.B[f][ry * T + rx] = in ? sv * rho2 : 0.0f;
                        if (in) aacc[f] = fmaf(sv, rho1, aacc[f]);
                    }
                }
            }
        }
        // alpha partials of this chunk
#pragma unroll
        for (int f = 0; f < CH; ++f) {
            float v = aacc[f];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) S.ared[warp][f] = v;
        }
        __syncthreads();
        if (!A.hvp_only && tid < CH) {
            float v = 0.0f;
            for (int w8 = 0; w8 < NTHREADS / 32; ++w8) v += S.ared[w8][tid];
            part[kNF * kKK + ch * CH + tid] = v;
        }

        // ---- Hessian-vector product: h(q) += sum_c sum_{a,b} 2 alpha_c w_c(a, b) psi_c(q - (a, b)) ----
#pragma unroll 1
        for (int c = 0; c < CH; ++c) {
            const int fi = ch * CH + c;
            const float *pp = &S.psi[c * PLANE];
#pragma unroll
            for (int a = 0; a < kKS; ++a) {
                const float *prow = pp + (oy - a + kR + R0) * UCOLS + ox0 + 4;
                const float4 x0 = *reinterpret_cast<const float4 *>(prow);
                const float4 x1 = *reinterpret_cast<const float4 *>(prow + 4);
                const float4 x2 = *reinterpret_cast<const float4 *>(prow + 8);
                const float v[12] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w, x2.x, x2.y, x2.z, x2.w};
                const float *wp = &S.wa[(fi * kKS + a) * 8];
                const float4 w0 = *reinterpret_cast<const float4 *>(wp);
                const float4 w1 = *reinterpret_cast<const float4 *>(wp + 4);
                const float wv[7] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z};
#pragma unroll
                for (int b = 0; b < kKS; ++b)
#pragma unroll
                    for (int p = 0; p < 4; ++p) h[p] = fmaf(wv[b], v[6 + p - b], h[p]);
            }
        }
        if (ring_tile) {
            const int gy = ty0 + oy;
            const int my = gy < kR ? -1 - gy : (gy >= H - kR ? 2 * H - 1 - gy : -1000);
            for (int p = 0; p < 4; ++p) {
                const int gx = tx0 + ox0 + p;
                if (gy >= H || gx >= W) continue;
                const int mx = gx < kR ? -1 - gx : (gx >= W - kR ? 2 * W - 1 - gx : -1000);
                if (my != -1000) hr[p] += ring_gather_b(S, ch, my - ty0, gx - tx0, ty0, tx0, H, W);
                if (mx != -1000) hr[p] += ring_gather_b(S, ch, gy - ty0, mx - tx0, ty0, tx0, H, W);
                if (my != -1000 && mx != -1000) hr[p] += ring_gather_b(S, ch, my - ty0, mx - tx0, ty0, tx0, H, W);
            }
        }

        // ---- filter gradient: warp = filter of the chunk, lane = column ----
        if (!A.hvp_only) {
            const int f = warp;
            float g[kKS][kKS];
#pragma unroll
            for (int a = 0; a < kKS; ++a)
#pragma unroll
                for (int b = 0; b < kKS; ++b) g[a][b] = 0.0f;
            // input row rho = y + a - 3 for own row y and tap row a; rho in [-3, 34]
#pragma unroll 1
            for (int rho = -kR; rho < T + kR; ++rho) {
                const float *wrow = &S.w[(rho + R0) * UCOLS + lane - kR + C0];
                const float *urow = &S.u[(rho + R0) * UCOLS + lane - kR + C0];
                float pw[kKS], pu[kKS];
#pragma unroll
                for (int b = 0; b < kKS; ++b) {
                    pw[b] = wrow[b];
                    pu[b] = urow[b];
                }
#pragma unroll
                for (int a = 0; a < kKS; ++a) {
                    const int y = rho - a + kR;
                    if (y < 0 || y >= T) continue;
                    const float av = S.A[f][y * T + lane], bv = S.B[f][y * T + lane];
#pragma unroll
                    for (int b = 0; b < kKS; ++b) g[a][b] = fmaf(av, pw[b], fmaf(bv, pu[b], g[a][b]));
                }
            }
#pragma unroll
            for (int a = 0; a < kKS; ++a)
#pragma unroll
                for (int b = 0; b < kKS; ++b) {
                    float v = g[a][b];
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane == 0) part[(ch * CH + f) * kKK + a * kKS + b] = v;
                }
        }
        __syncthreads();
    }

    // ---- gbar^n = (1 + gamma) w - tau (H w) - gamma c1 gbar^{n+2} ----
    if (!A.write_g) return;
    const int gy = ty0 + oy;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int gx = tx0 + ox0 + p;
        if (gy >= H || gx >= W) continue;
        const size_t idx = (size_t)gy * ld + gx;
        const float wv = S.w[(oy + R0) * UCOLS + ox0 + p + C0];
        const float g2 = D.gb2 ? D.gb2[idx] : 0.0f;
        D.gout[idx] = (1.0f + A.gamma) * wv - A.tau * (h[p] + hr[p]) - A.gamma * A.c1 * g2;
    }
}

// Loss 1/2 (I_C(max(u, sqrt(3/2))) - g)^2 per pixel (FP64 block partials) and its derivative gbar^T.
__device__ __forceinline__ double ic_d(double z)
{
    const double s = 1.2247448713915890491;
    const double zi = 1.0 / z;
    return 0.25 * z * z + 0.25 * s * zi - 1.375 * zi * zi + 0.625 * s * zi * zi * zi - 0.125;
}

__device__ __forceinline__ double ic_deriv_d(double z)
{
    const double s = 1.2247448713915890491;
    const double zi = 1.0 / z;
    return 0.5 * z - 0.25 * s * zi * zi + 2.75 * zi * zi * zi - 1.875 * s * zi * zi * zi * zi;
}

__global__ void k_train_loss(const float *u_hi, const float *u_lo, const float *clean, int H, int W, int ld,
                             int cld, float *gbar, double *partials)
{
    __shared__ double red[8];
    double acc = 0.0;
    const long n = (long)H * W;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const long y = i / W, x = i % W;
        const double u = (double)u_hi[y * ld + x] + (double)u_lo[y * ld + x];
        const double zmin = 1.2247448713915890491;
        const double e = ic_d(u > zmin ? u : zmin) - (double)clean[y * cld + x];
        acc += 0.5 * e * e;
        gbar[y * ld + x] = u > zmin ? (float)(ic_deriv_d(u) * e) : 0.0f;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        partials[blockIdx.x] = t;
    }
}

// acc[e] += sum over tiles of partials[tile][e] (FP64, fixed order).
__global__ void k_reduce_partials(const float *partials, int tiles, double *acc)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kBwdPartials) return;
    double s = 0.0;
    for (int t = 0; t < tiles; ++t) s += (double)partials[(size_t)t * kBwdPartials + e];
    acc[e] += s;
}

// Final gradients: dL/dk_i in convolution orientation (k_i(a, b) = w_i(-a, -b)) and dL/d log alpha_i,
// both scaled by -tau alpha_i; the loss is the sum of the block partials.
__global__ void k_train_finish(const double *acc, const float *alpha, float tau, int nf, float *dk, float *dla)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < nf * kKK) {
        const int f = e / kKK, t = e % kKK;
        dk[f * kKK + (kKK - 1 - t)] = (float)(-(double)tau * (double)alpha[f] * acc[e]);
    } else if (e < nf * kKK + nf) {
        const int f = e - nf * kKK;
        dla[f] = (float)(-(double)tau * (double)alpha[f] * acc[kNF * kKK + f]);
    }
}

__global__ void k_copy_planes(const float *src, float *dst, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) dst[i] = src[i];
}

}  // namespace

size_t bwd_smem_bytes() { return sizeof(BwdSmem); }

cudaError_t bwd_setup()
{
    return cudaFuncSetAttribute(k_foe_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BwdSmem));
}

cudaError_t bwd_launch(const BwdArgs &a, cudaStream_t s)
{
    const int tiles = a.tile_prefix[a.nimg];
    if (tiles <= 0) return cudaSuccess;
    k_foe_bwd<<<tiles, NTHREADS, sizeof(BwdSmem), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_train_loss(const float *u_hi, const float *u_lo, const float *clean, int H, int W, int ld, int cld,
                              float *gbar, double *partials, int nblocks, cudaStream_t s)
{
    k_train_loss<<<nblocks, 256, 0, s>>>(u_hi, u_lo, clean, H, W, ld, cld, gbar, partials);
    return cudaGetLastError();
}

cudaError_t launch_reduce_partials(const float *partials, int tiles, double *acc, cudaStream_t s)
{
    k_reduce_partials<<<(kBwdPartials + 255) / 256, 256, 0, s>>>(partials, tiles, acc);
    return cudaGetLastError();
}

cudaError_t launch_train_finish(const double *acc, const float *alpha, float tau, int nf, float *dk, float *dla,
                                cudaStream_t s)
{
    k_train_finish<<<(kNF * kKK + kNF + 255) / 256, 256, 0, s>>>(acc, alpha, tau, nf, dk, dla);
    return cudaGetLastError();
}

cudaError_t launch_copy(const float *src, float *dst, long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_copy_planes<<<(unsigned)blocks, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

int bwd_tile() { return T; }

}  // namespace foe
