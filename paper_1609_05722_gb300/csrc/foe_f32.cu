// Plain-FP32 (FFMA) fused FoE tile kernel and the elementwise kernels of the solve.
//
// One CTA owns a 32x32 output tile.  Per chunk of 8 filters it computes the filter responses
// r_i = K_i u on the tile plus a 3-pixel ring (Eq. FOEmodel), psi_i = 2 alpha_i rho'(r_i) / 2
// (Eq. FoEF, rho' of Sec. 2.5.2; the factor 2 alpha_i is folded into the adjoint weights), masked
// to zero outside the image, and accumulates the adjoint K_i^T psi_i on the tile.  Nothing but u
// and the final result touches global memory: the 48 response planes live in shared memory one
// chunk at a time.  The epilogue applies the iPiano step (Eq. iPianoupdate) with the data-term prox
// (Eq. subproblemGIdiv / subproblemGL2), or writes the energy gradient, or the energy partials.
#include "foe_common.cuh"
#include "foe_kernels.h"

namespace foe {

namespace {

constexpr int T = 32;                       // output tile side
constexpr int UROWS = 44, UCOLS = 48;       // shared arrays cover tile-relative rows [-6, 38), cols [-7, 41)
constexpr int R0 = 6, C0 = 7;
constexpr int PLANE = UROWS * UCOLS;
constexpr int CH = 8;                       // filters per chunk
constexpr int NTHREADS = 256;
constexpr int RESP_ROWS = T + 6;            // responses on tile-relative rows [-3, 35)
constexpr int RESP_STRIPS_X = (T + 8) / 2;  // 1x2 strips over cols [-4, 36)
constexpr int NSTRIPS = RESP_ROWS * RESP_STRIPS_X;
constexpr int NSTRIP = (NSTRIPS + NTHREADS - 1) / NTHREADS;  // strips per thread: 3

struct F32Smem {
    float u[PLANE];
    float psi[CH * PLANE];
    float wf[6 * kKK * CH];   // forward weights, [chunk][tap][8 filters]
    float wa[kNF * kKS * 8];  // adjoint weights 2 alpha_i w_i(a, b), [filter][a][b (8, padded)];
                              // the padding slot [f][6][7] holds alpha_f for the energy
    double red[NTHREADS / 32];
};

// h(q') for a reflected position q' (tile-relative), skipping psi positions outside the image.
__device__ float ring_gather(const F32Smem &S, int chunk, int qy, int qx, int ty0, int tx0, int H, int W)
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

template <int MODE>
__global__ void __launch_bounds__(NTHREADS, 2) k_foe_f32(const __grid_constant__ LaunchArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    F32Smem &S = *reinterpret_cast<F32Smem *>(smem_raw);
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int im = tile_image(A, tile);
    const ImgDesc &D = A.img[im];
    if (image_stopped(D)) return;  // CTA-uniform
    const int lt = tile - A.tile_prefix[im];
    const int ty0 = (lt / D.tiles_x) * T, tx0 = (lt % D.tiles_x) * T;
    const int H = D.H, W = D.W, ld = D.ld;
    const float *uin = D.u_hi[A.parity];

    // ---- stage weights, the input region and a zeroed psi buffer ----
    for (int j = tid; j < 6 * kKK * CH; j += NTHREADS) {
        const int c = j / (kKK * CH), t = (j / CH) % kKK, f = j % CH;
        S.wf[j] = A.wts[(c * CH + f) * kKK + t];
    }
    for (int j = tid; j < kNF * kKS * 8; j += NTHREADS) {
        const int f = j / (kKS * 8), a = (j / 8) % kKS, b = j % 8;
        S.wa[j] = b < kKS ? 2.0f * A.alpha[f] * A.wts[f * kKK + a * kKS + b] : (a == kKS - 1 ? A.alpha[f] : 0.0f);
    }
    for (int j = tid; j < PLANE; j += NTHREADS) {
        const int r = j / UCOLS, c = j % UCOLS;
        const int sy = pad_index(ty0 + r - R0, H, A.bc), sx = pad_index(tx0 + c - C0, W, A.bc);
        S.u[j] = (sy < 0 || sx < 0) ? 0.0f : __ldg(uin + (size_t)sy * ld + sx);
    }
    if (MODE != kEnergy)
        for (int j = tid; j < CH * PLANE; j += NTHREADS) S.psi[j] = 0.0f;
    __syncthreads();

    const int oy = tid / 8, ox0 = (tid % 8) * 4;     // this thread's 1x4 output strip
    const bool ring_tile = (A.bc == kSymmetric) &&
                           (ty0 < kR || tx0 < kR || ty0 + T > H - kR || tx0 + T > W - kR);
    float h[4] = {0.f, 0.f, 0.f, 0.f};
    float hr[4] = {0.f, 0.f, 0.f, 0.f};
    double eacc = 0.0;

    for (int ch = 0; ch < A.nchunks; ++ch) {
        // ---- forward responses and expert derivative on the response region ----
        // each thread computes its NSTRIP strips s = tid + k NTHREADS together, so that every weight load serves all
        // of them (a thread without a k-th strip computes a copy of its first one and discards it)
        float acc[NSTRIP][2][CH];
#pragma unroll
        for (int k = 0; k < NSTRIP; ++k)
#pragma unroll
            for (int f = 0; f < CH; ++f) acc[k][0][f] = acc[k][1][f] = 0.0f;
        int sk[NSTRIP];
#pragma unroll
        for (int k = 0; k < NSTRIP; ++k) {
            const int sv = tid + k * NTHREADS;
            sk[k] = sv < NSTRIPS ? sv : tid;
        }
#pragma unroll 1
        for (int a = 0; a < kKS; ++a) {
            float v[NSTRIP][8];
#pragma unroll
            for (int k = 0; k < NSTRIP; ++k) {
                const int ry = sk[k] / RESP_STRIPS_X - kR, rx0 = (sk[k] % RESP_STRIPS_X) * 2 - 4;
                const float *urow = &S.u[(ry + a - kR + R0) * UCOLS + (rx0 - kR + C0)];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float2 q = *reinterpret_cast<const float2 *>(urow + 2 * j);
                    v[k][2 * j] = q.x;
                    v[k][2 * j + 1] = q.y;
                }
            }
#pragma unroll
            for (int b = 0; b < kKS; ++b) {
                const float *wp = &S.wf[(ch * kKK + a * kKS + b) * CH];
                const float4 w0 = *reinterpret_cast<const float4 *>(wp);
                const float4 w1 = *reinterpret_cast<const float4 *>(wp + 4);
                const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                for (int k = 0; k < NSTRIP; ++k)
#pragma unroll
                    for (int f = 0; f < CH; ++f) {
                        acc[k][0][f] = fmaf(wv[f], v[k][b], acc[k][0][f]);
                        acc[k][1][f] = fmaf(wv[f], v[k][b + 1], acc[k][1][f]);
                    }
            }
        }
#pragma unroll
        for (int k = 0; k < NSTRIP; ++k) {
            if (tid + k * NTHREADS >= NSTRIPS) continue;
            const int ry = sk[k] / RESP_STRIPS_X - kR, rx0 = (sk[k] % RESP_STRIPS_X) * 2 - 4;
            const int gy = ty0 + ry;
#pragma unroll
            for (int px = 0; px < 2; ++px) {
                const int rx = rx0 + px, gx = tx0 + rx;
                const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
                if (MODE == kEnergy) {
                    if (in && ry >= 0 && ry < T && rx >= 0 && rx < T) {
                        float es = 0.0f;
#pragma unroll
                        for (int f = 0; f < CH; ++f) {
                            const float r = acc[k][px][f];
                            es = fmaf(S.wa[((ch * CH + f) * kKS + kKS - 1) * 8 + 7], log1pf(r * r), es);
                        }
                        eacc += (double)es;
                    }
                } else {
#pragma unroll
                    for (int f = 0; f < CH; ++f) {
                        const float r = acc[k][px][f];
                        S.psi[f * PLANE + (ry + R0) * UCOLS + (rx + C0)] = in ? __fdividef(r, fmaf(r, r, 1.0f)) : 0.0f;
                    }
                }
            }
        }
        if (MODE == kEnergy) continue;  // the energy needs no adjoint
        __syncthreads();

        // ---- adjoint: h(q) += sum_c sum_{a,b} 2 alpha_c w_c(a, b) psi_c(q - (a, b)) ----
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
        // ---- symmetric padding: fold the adjoint at reflected positions back (P^T) ----
        if (ring_tile) {
            const int gy = ty0 + oy;
            const int my = gy < kR ? -1 - gy : (gy >= H - kR ? 2 * H - 1 - gy : -1000);
            for (int p = 0; p < 4; ++p) {
                const int gx = tx0 + ox0 + p;
                if (gy >= H || gx >= W) continue;
                const int mx = gx < kR ? -1 - gx : (gx >= W - kR ? 2 * W - 1 - gx : -1000);
                if (my != -1000) hr[p] += ring_gather(S, ch, my - ty0, gx - tx0, ty0, tx0, H, W);
                if (mx != -1000) hr[p] += ring_gather(S, ch, gy - ty0, mx - tx0, ty0, tx0, H, W);
                if (my != -1000 && mx != -1000) hr[p] += ring_gather(S, ch, my - ty0, mx - tx0, ty0, tx0, H, W);
            }
        }
        __syncthreads();
    }

    // ---- epilogue ----
    const int gy = ty0 + oy;
    if (MODE == kEnergy) {
        for (int p = 0; p < 4; ++p) {
            const int gx = tx0 + ox0 + p;
            if (gy < H && gx < W) {
                const size_t idx = (size_t)gy * ld + gx;
                if (!A.prior_only)
                    eacc += data_energy(S.u[(oy + R0) * UCOLS + ox0 + p + C0], D.d[idx], D.model, D.sc.lambda);
            }
        }
        for (int o = 16; o > 0; o >>= 1) eacc += __shfl_xor_sync(0xffffffffu, eacc, o);
        if ((tid & 31) == 0) S.red[tid >> 5] = eacc;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NTHREADS / 32; ++w) t += S.red[w];
            A.partials[tile] = t;
        }
        return;
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int gx = tx0 + ox0 + p;
        if (gy >= H || gx >= W) continue;
        const size_t idx = (size_t)gy * ld + gx;
        const float g = h[p] + hr[p];
        const float uh = S.u[(oy + R0) * UCOLS + ox0 + p + C0];
        if (MODE == kGrad) {
            D.out[idx] = A.prior_only ? g : g + data_grad(uh, D.d[idx], D.model, D.sc.lambda);
        } else {
            const float ul = D.u_lo ? D.u_lo[idx] : 0.0f;
            float nh, nl, nd;
            ipiano_update(g, uh, ul, D.delta[idx], D.d[idx], D.model, A.sc_dev ? *A.sc_dev : D.sc, nh, nl, nd);
            D.u_hi[A.parity ^ 1][idx] = nh;
            if (D.u_lo) D.u_lo[idx] = nl;
            D.delta[idx] = nd;
        }
    }
}

// ---- elementwise kernels ----

// Data term and initial iterate u^0 = u^{-1} = d: the Anscombe transform (Eq. Anscombetransform) in
// FP64 for the transform-domain models, the zero-replaced counts (Sec. 3.1.1) for the direct model.
__global__ void k_init(const float *y, int H, int W, int yld, int ld, int model, float zero_c, float *d, float *uh,
                       float *ul, float *delta)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, yrow = blockIdx.y;
    if (x >= W || yrow >= H) return;
    const float yv = y[(size_t)yrow * yld + x];
    const size_t i = (size_t)yrow * ld + x;
    float hi, lo = 0.0f;
    if (model == kDirect) {
        hi = yv == 0.0f ? zero_c : yv;
    } else {
        const double v = 2.0 * sqrt((double)yv + 0.375);
        hi = (float)v;
        lo = (float)(v - (double)hi);
    }
    d[i] = hi;
    uh[i] = hi;
    if (ul) ul[i] = lo;
    delta[i] = 0.0f;
}

__device__ __forceinline__ double inv_anscombe(double z)
{
    const double s = 1.2247448713915890491;  // sqrt(3/2)
    if (z < s) z = s;
    const double zi = 1.0 / z;
    return 0.25 * z * z + 0.25 * s * zi - 1.375 * zi * zi + 0.625 * s * zi * zi * zi - 0.125;
}

// Output map: x = I_C(max(u, sqrt(3/2))) (Eq. invAns) for the Anscombe models, x = u for the direct one.
// Output map; counts the non-finite outputs into *nonfinite when it is given (a NaN / Inf sentinel).
// status (nullable): the context's sticky device status; while it is set the solve's step launches did nothing,
// so the output is NaN rather than a stale iterate (for callers that return without reading the status)
__global__ void k_output(const float *uh, const float *ul, int H, int W, int ld, int xld, int model, float *x,
                         int *nonfinite, const int *status, const float *uh_alt, int budget, const int *stop)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (c >= W || r >= H) return;
    if (status && *(const volatile int *)status != 0) {
        x[(size_t)r * xld + c] = __int_as_float(0x7fc00000);
        return;
    }
    if (stop) {
        const int n = __ldcg(stop);
        if (n != 0 && ((n ^ budget) & 1)) uh = uh_alt;
    }
    const size_t i = (size_t)r * ld + c;
    const double u = (double)uh[i] + (ul ? (double)ul[i] : 0.0);
    const float v = model == kDirect ? (float)u : (float)inv_anscombe(u);
    x[(size_t)r * xld + c] = v;
    if (nonfinite && !isfinite(v)) atomicAdd(nonfinite, 1);
}

__global__ void k_anscombe(const float *y, float *v, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        v[i] = (float)(2.0 * sqrt((double)y[i] + 0.375));
}

__global__ void k_inverse(const float *z, float *x, long n)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        x[i] = (float)inv_anscombe((double)z[i]);
}

// Deterministic FP64 sum of per-tile partials (one block).
__global__ void k_reduce(const double *p, int n, double *out)
{
    __shared__ double s[32];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += p[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += s[w];
        *out = r;
    }
}

}  // namespace

int f32_tile() { return T; }
size_t f32_smem_bytes() { return sizeof(F32Smem); }

cudaError_t f32_setup()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_foe_f32<kStep>, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(F32Smem))))
        return e;
    if ((e = cudaFuncSetAttribute(k_foe_f32<kGrad>, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(F32Smem))))
        return e;
    return cudaFuncSetAttribute(k_foe_f32<kEnergy>, cudaFuncAttributeMaxDynamicSharedMemorySize, sizeof(F32Smem));
}

cudaError_t f32_launch(const LaunchArgs &a, int mode, cudaStream_t s)
{
    const int tiles = a.tile_prefix[a.nimg];
    if (tiles <= 0) return cudaSuccess;
    if (mode == kStep) k_foe_f32<kStep><<<tiles, NTHREADS, sizeof(F32Smem), s>>>(a);
    else if (mode == kGrad) k_foe_f32<kGrad><<<tiles, NTHREADS, sizeof(F32Smem), s>>>(a);
    else k_foe_f32<kEnergy><<<tiles, NTHREADS, sizeof(F32Smem), s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_init(const float *y, int H, int W, int yld, int ld, int model, float zero_c, float *d, float *uh,
                        float *ul, float *delta, cudaStream_t s)
{
    dim3 g((W + 127) / 128, H);
    k_init<<<g, 128, 0, s>>>(y, H, W, yld, ld, model, zero_c, d, uh, ul, delta);
    return cudaGetLastError();
}

cudaError_t launch_output(const float *uh, const float *ul, int H, int W, int ld, int xld, int model, float *x, int *nonfinite,
                          cudaStream_t s, const int *status, const float *uh_alt, int budget, const int *stop)
{
    dim3 g((W + 127) / 128, H);
    k_output<<<g, 128, 0, s>>>(uh, ul, H, W, ld, xld, model, x, nonfinite, status, uh_alt, budget, stop);
    return cudaGetLastError();
}

cudaError_t launch_anscombe(const float *y, float *v, long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_anscombe<<<(unsigned)blocks, 256, 0, s>>>(y, v, n);
    return cudaGetLastError();
}

cudaError_t launch_inverse(const float *z, float *x, long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_inverse<<<(unsigned)blocks, 256, 0, s>>>(z, x, n);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const double *p, int n, double *out, cudaStream_t s)
{
    k_reduce<<<1, 256, 0, s>>>(p, n, out);
    return cudaGetLastError();
}

}  // namespace foe
