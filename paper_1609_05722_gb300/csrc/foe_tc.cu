// Tensor-core fused FoE tile kernel for sm_103a: tcgen05.mma (BF16 operands, kind::f16, or TF32 operands,
// kind::tf32; FP32 accumulators in tensor memory), one iPiano step (Eq. iPianoupdate) per launch.
//
// One CTA owns a 26-wide output tile of 58 or 26 rows (below).  The prior gradient sum_i alpha_i K_i^T rho'(K_i u)
// (Eq. FoEF) needs the responses on the tile plus a 3-pixel ring: a 32-wide response region of 64 (32) rows,
// processed as 16 (8) M-tiles of 128 response pixels (4 rows of 32).
//
//   forward   R[m][i]  = sum_k A[m][k] Wf[i][k]        M=128, N=48 filters, K=64 (8x8 taps, 49 used)
//             A is never materialised as an im2col matrix: E holds, for every input position, the 8
//             horizontally adjacent bf16 values u(y, x..x+7), so the K-slice "tap rows 2s, 2s+1" of
//             the 128 pixels of an M-tile is two shifted, regularly strided views of E that one shared
//             memory descriptor addresses (leading offset = one E row, stride = 8 entries).
//   expert    psi[m][i] = rho'(R) / 2 = R / (1 + R^2), zero outside the image; 2 alpha_i lives in Wa.
//   adjoint   Z[m][n]  = sum_i Psi[m][i] Wa[n][i]      M=128, N=64 taps (8a+b), K=48 filters
//             g(q) = sum_{a,b} Z[q - (a-3, b-3)][8a+b]: the horizontal part of this col2im is done
//             with warp shuffles (a warp holds one response row of 32 pixels), the vertical part
//             through shared memory.
//
// Roles (320 threads): warps 0-7 move data between tensor memory and registers (warps w and w+4 access
// TMEM lanes 32(w%4)..32(w%4)+31, i.e. response row 4t+w%4 of M-tile t): warps 0-3 run the expert step,
// warps 4-7 the col2im.  Warp 8 issues the forward MMAs and warp 9 the adjoint MMAs (one elected lane each), so
// neither kind of MMA waits behind the other's dependencies.
// Tensor memory holds two response stages (columns 0 and 64) and two adjoint stages (columns 128 and 192); M-tile g
// (counted over all tiles of the CTA) uses stage g & 1.  The epilogue writes Psi(g) (packed bf16 pairs, or tf32)
// over the first columns of R(g)'s stage, and the adjoint MMA reads its A operand from there, so Psi never passes
// through shared memory; the stage is free again once that MMA is complete, Z(g) once the col2im has loaded it.  Expert and
// col2im warps run decoupled, so the MMAs of later M-tiles overlap the epilogue of earlier ones.
// CTAs are persistent (tiles c, c + gridDim.x, ...).  While a tile is computed, the next tile's input region is
// copied in (cp.async, double-buffered; its completion arrives on an mbarrier), and once the tile's last forward
// MMA is complete the expert warps build the next tile's E while the last adjoint and col2im finish; then all
// warps run the output pass (vertical col2im, padding fold, iPiano step).  Launches are programmatically
// dependent: a CTA sets up barriers and tensor memory before it waits for the previous step to complete.
// Every mbarrier wait is bounded: on expiry the CTA records FOE_ETIMEOUT in *status, drains its MMAs,
// frees its tensor memory and finishes without further waits.
//
// BF16 range: filters are zero-mean, so K(u - c) = K u for any constant c (the padded image of a
// constant is constant under symmetric padding; under zero padding the padded zeros are shifted by -c
// too).  The mean of 64 samples of the tile's input region is subtracted before rounding u to BF16 / TF32.
#include <algorithm>
#include <cstdint>

#include <cuda_fp16.h>

#include "foe_common.cuh"
#include "foe_kernels.h"
#include "foe_ptx.cuh"

namespace foe {

namespace {

using namespace ptx;

constexpr int TO = 26;                 // output tile width
constexpr int RS = TO + 6;             // response region width = 32 = warp width
constexpr int UC = RS + 8;             // floats per input-region row (RS + 7 used)

// Tile height: 26 (the instance built here; the kernel keeps it a template parameter).  This kernel runs the TF32
// path and BF16 images below the pixel-pair kernel's size (tc_tile_h); larger BF16 images go to that kernel.  An
// image is tiled the same way whatever else shares its launch, so its result does not depend on the batch.  The
// horizontal col2im sums are kept in FP16 on the BF16 path (their magnitude stays far below its range, and its
// 11-bit significand is finer than the BF16 rounding of u and psi); TF32 keeps FP32 sums and its ~4x smaller error.
constexpr int kShortH = 26;
template <bool TF>
struct HsType {
    using T = __half;
};
template <>
struct HsType<true> {
    using T = float;
};
template <int TOH>
constexpr int kRR = TOH + 6;              // response rows of a tile
template <int TOH>
constexpr int kNMT = kRR<TOH> / 4;        // M-tiles per tile
template <int TOH>
constexpr int kUR = kRR<TOH> + 7;         // input rows = E rows (7 tap rows + 1 zero-weight row)
constexpr int NEPI = 8;                // epilogue warps: two per TMEM lane quarter
constexpr int FWD_WARP = NEPI;         // one thread of this warp issues the forward MMAs
constexpr int ADJ_WARP = NEPI + 1;     // one thread of this warp issues the adjoint MMAs
constexpr int NWARP = NEPI + 2;
constexpr int NTHR = 32 * NWARP;
constexpr uint32_t TMEM_COLS = 256;
constexpr uint32_t Z_COL0 = 128;       // R(g) at 64 (g & 1) (48 columns), Z(g) at 128 + 64 (g & 1) (64 columns)

// Operand images in shared memory.  BF16: 16-byte entries of 8 values.  TF32: 16-byte entries of 4 values,
// so every 8-value K-chunk of the BF16 layout becomes two chunks (E is split into E[0] = u(x..x+3) and
// E[1] = u(x+4..x+7); the descriptor's leading offset steps from one half to the other).
template <bool TF>
struct TcOps;
template <>
struct TcOps<false> {
    static constexpr int EB = 1, WF = 8 * 48, WA = 6 * 64;
};
template <>
struct TcOps<true> {
    static constexpr int EB = 2, WF = 8 * 2 * 48, WA = 12 * 64;
};

// mbarriers
constexpr int B_FWD = 0;     // [2] forward MMAs of M-tile g complete (g & 1)             count 1 (commit)
constexpr int B_RFREE = 2;   // [2] adjoint MMAs of M-tile t complete: stage t & 1 free  count 1 (commit)
constexpr int B_PSI = 4;     // [2] Psi(g) written to tensor memory (g & 1)              count 128
constexpr int B_ADJ = 6;     // [2] adjoint MMAs of M-tile g complete (g & 1)             count 1 (commit)
constexpr int B_ZFREE = 8;   // [2] Z(g) loaded by every col2im thread (g & 1)           count 128
constexpr int B_W = 10;      // filter operand images arrived (bulk copy)                count 1 + tx
constexpr int B_DRAIN = 11;  // [2] all MMAs of the forward / adjoint thread complete    count 1 (commit)
constexpr int B_UREADY = 13; // [2] input region of buffer b landed (every thread's copies) count NTHR (cp.async)
constexpr int NBAR = 15;

template <bool TF, int TOH>
struct TcSmem {
    uint4 E[TcOps<TF>::EB][kUR<TOH> * RS];  // forward A operand: entry (row, x) holds u(row, x..x+7)
    uint4 Wf[TcOps<TF>::WF];               // forward B operand [tap row a][(chunk)][filter][tap cols]
    uint4 Wa[TcOps<TF>::WA];               // adjoint B operand [filter chunk][tap 8a+b][filters in chunk]
    typename HsType<TF>::T Hs[7 * kRR<TOH> * RS];  // horizontal col2im partial sums [a][response row][col]
    float U[2][kUR<TOH> * UC];                     // fp32 input region (this tile / the next one, copied in meanwhile)
    float O[2][TO * TOH];                          // output-pass operands delta, d (staged after the previous tile)
    int srow[2][kUR<TOH>], scol[2][RS + 7];        // source row / column of each region row / column (-1: zero)
    int geo[2][5];                                 // image, oy0, ox0, column write range [xs, xe) of the tile in buffer b
    int tprefix[kMaxBatch + 1];                    // the launch's tile prefix, and per image: tiles per row, H, W
    int timg[kMaxBatch][3];
    int live[kMaxBatch];               // 0 once the image's stopping rule has held (its tiles are skipped)
    int tnext[2];                      // the CTA's tile after the tile in buffer b (>= ntiles: none)
    uint64_t bar[NBAR];
    uint32_t tmem_base;
    int abort_flag;
    float mean0;                                   // BF16 / TF32 range offset of the first tile
};
// Two CTAs share an SM: 228 KB of shared memory per SM, 1 KB of it reserved per CTA
static_assert(sizeof(TcSmem<false, kShortH>) + 1024 <= 228 * 1024 / 2, "BF16 tiles: two CTAs per SM");
static_assert(sizeof(TcSmem<true, kShortH>) + 1024 <= 228 * 1024 / 2, "TF32 tiles: two CTAs per SM");
// Wf and Wa are filled by one bulk copy of the packed operand images
using SmemBf16 = TcSmem<false, kShortH>;
using SmemTf32 = TcSmem<true, kShortH>;
static_assert(offsetof(SmemBf16, Wa) == offsetof(SmemBf16, Wf) + sizeof(uint4) * TcOps<false>::WF, "");
static_assert(offsetof(SmemTf32, Wa) == offsetof(SmemTf32, Wf) + sizeof(uint4) * TcOps<true>::WF, "");
static_assert(offsetof(SmemBf16, U) % 8 == 0 && offsetof(SmemTf32, U) % 8 == 0 && UC % 2 == 0 && UC >= 40, "");

// psi = r / (1 + r^2) for a pair of responses with packed f32x2 arithmetic, rounded to a bf16x2 word
__device__ __forceinline__ uint32_t psi_bf16x2(float r0, float r1)
{
    uint64_t a, den, inv, p;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(r0), "f"(r1));
    asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(den) : "l"(a), "l"(0x3f8000003f800000ull));
    float d0, d1;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d0), "=f"(d1) : "l"(den));
    const float i0 = rcp_approx(d0), i1 = rcp_approx(d1);
    asm("mov.b64 %0, {%1, %2};" : "=l"(inv) : "f"(i0), "f"(i1));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(p) : "l"(a), "l"(inv));
    float p0, p1;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(p0), "=f"(p1) : "l"(p));
    return pack_bf16x2(p0, p1);
}

__device__ __forceinline__ float hs_val(float v) { return v; }
__device__ __forceinline__ float hs_val(__half v) { return __half2float(v); }
__device__ __forceinline__ void hs_put(float &d, float v) { d = v; }
__device__ __forceinline__ void hs_put(__half &d, float v) { d = __float2half_rn(v); }

// Sum over the 7 tap rows of the horizontal partials at (qy, qx) of the response region.  Unchecked:
// for an output position (qy in 3..TOH+2, qx in 3..28) every row qy - a + 3 lies in the region.
template <bool TF, int TOH>
__device__ __forceinline__ float hs_sum(const TcSmem<TF, TOH> &S, int qy, int qx)
{
    const auto *p = &S.Hs[(qy + 3) * RS + qx];
    float g = 0.0f;
#pragma unroll
    for (int a = 0; a < 7; ++a) g += hs_val(p[a * (kRR<TOH> * RS - RS)]);
    return g;
}

// The same at an arbitrary region position (padding fold); rows and columns outside the region are
// outside the image whenever they are asked for, so they add 0.
template <bool TF, int TOH>
__device__ __forceinline__ float hs_gather(const TcSmem<TF, TOH> &S, int qy, int qx)
{
    if (qx < 0 || qx >= RS) return 0.0f;
    float g = 0.0f;
#pragma unroll
    for (int a = 0; a < 7; ++a) {
        const int r = qy - a + 3;
        if (r >= 0 && r < kRR<TOH>) g += hs_val(S.Hs[(a * kRR<TOH> + r) * RS + qx]);
    }
    return g;
}

// Image of a tile: a search of the launch's tile table in its copy in shared memory, made at the start of the
// kernel (parameter-space loads here sat on the staging thread's dependent chain).
template <bool TF, int TOH>
__device__ __forceinline__ int tc_image(const LaunchArgs &A, const TcSmem<TF, TOH> &S, int tile)
{
    int lo = 0, hi = A.nimg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.tprefix[mid] <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The CTA's tiles are c, c + gridDim.x, ... without those of stopped images.
template <bool TF, int TOH>
__device__ __noinline__ int tc_next_live(const LaunchArgs &A, const TcSmem<TF, TOH> &S, int ntiles, int tile)
{
    while (tile < ntiles && !S.live[tc_image(A, S, tile)]) tile += gridDim.x;
    return tile;
}

// Image, origin and column write range [xs, xe) of a tile.  The horizontal col2im of a response row is formed
// across the 32 lanes of a warp, so its sums exist only at region columns 0..31.  The padding fold of a pixel
// within 3 columns of the right border needs the sum at its reflection (up to column W + 2), which lies inside the
// region only if the tile reaches that border: the last tile of a row is therefore placed flush right (origin
// W - 26) and the tile before it writes only the columns left of max(W - 26, 3).  The bound 3 keeps the columns
// within 3 of the left border in the first tile (origin 0), whose region holds their reflections, when the flush
// tile starts at column 1 or 2 (W = 27, 28).  Rows need no such rule: the vertical part of the col2im reads
// response rows, and the rows that a reflection asks for that lie in the image are always within 3 rows of the
// output row.
template <bool TF, int TOH>
__device__ __forceinline__ void tile_geometry(const LaunchArgs &A, const TcSmem<TF, TOH> &S, int tile, int &im,
                                              int &oy0, int &ox0, int &xe, int &xs)
{
    im = tc_image(A, S, tile);
    const int tiles_x = S.timg[im][0], W = S.timg[im][2];
    const int lt = tile - S.tprefix[im];
    const int tx = lt % tiles_x;
    oy0 = (lt / tiles_x) * TOH;
    ox0 = tx * TO;
    xe = min(ox0 + TO, W);
    xs = ox0;
    if (W > TO) {
        const int last = W - TO, split = max(last, 3);
        ox0 = min(ox0, last);
        xs = tx + 1 < tiles_x ? ox0 : split;
        xe = tx + 1 < tiles_x ? min(xe, split) : W;
    }
}

// Issue the asynchronous copies of a tile's input region into buffer b and record its geometry there (all
// threads; the caller commits the cp.async group).  Positions outside the padded image are zero-filled by the copy
// engine too, and each thread then arrives on the buffer's mbarrier once its copies have landed.
template <bool TF, int TOH>
__device__ __forceinline__ void stage_input(const LaunchArgs &A, TcSmem<TF, TOH> &S, int tile, int b, int tid, int warp,
                                            int lane)
{
    if (tid == 0) tile_geometry(A, S, tile, S.geo[b][0], S.geo[b][1], S.geo[b][2], S.geo[b][3], S.geo[b][4]);
    __syncthreads();
    const int im = S.geo[b][0], oy0 = S.geo[b][1], ox0 = S.geo[b][2];
    const ImgDesc &D = A.img[im];
    const int H = D.H, W = D.W, ld = D.ld;
    constexpr int UR = kUR<TOH>, UCU = RS + 7;  // input rows, input columns used
    if (tid < UR) S.srow[b][tid] = pad_index(oy0 - 6 + tid, H, A.bc);
    else if (tid < UR + UCU) S.scol[b][tid - UR] = pad_index(ox0 - 6 + tid - UR, W, A.bc);
    __syncthreads();
    const float *uin = D.u_hi[A.parity];
    float *U = S.U[b];
    if (ox0 >= 6 && ((ox0 - 6) & 1) == 0 && ox0 + 34 <= W) {
        // the region's columns ox0 - 6 .. ox0 + 33 lie in the image (no reflection) and start 8-byte aligned (the
        // API takes 16-byte aligned images with a pitch of a multiple of 4 floats): 20 lanes copy 8 bytes of each
        // row, one warp instruction per row instead of two (column 39 is copied but not used)
        if (lane < 20) {
            for (int r = warp; r < UR; r += NWARP) {
                const int sy = S.srow[b][r];
                float *dst = &U[r * UC + 2 * lane];
                if (sy < 0) cp_async_zero(dst, uin, 8);
                else cp_async8(dst, uin + (size_t)sy * ld + ox0 - 6 + 2 * lane);
            }
        }
    } else {
        const int sx0 = S.scol[b][lane], sx1 = lane + 32 < UCU ? S.scol[b][lane + 32] : -1;
        for (int r = warp; r < UR; r += NWARP) {
            const int sy = S.srow[b][r];
            const float *src = uin + (size_t)(sy < 0 ? 0 : sy) * ld;
            float *dst = &U[r * UC];
            if (sy < 0 || sx0 < 0) cp_async_zero(&dst[lane], uin, 4);
            else cp_async4(&dst[lane], src + sx0);
            if (lane + 32 < UCU) {
                if (sy < 0 || sx1 < 0) cp_async_zero(&dst[lane + 32], uin, 4);
                else cp_async4(&dst[lane + 32], src + sx1);
            }
        }
    }
    cp_async_mbar_arrive(&S.bar[B_UREADY + b]);
}

// E rows [r0, r1) of the tile whose input region is Ub, with range offset `mean`: one item = 4 consecutive entries
// of an E row, whose 11 inputs are loaded (three 16-byte loads), shifted and rounded once.  Items idx, idx +
// stride, ... of the range.
template <bool TF, int TOH>
__device__ __forceinline__ void build_e(TcSmem<TF, TOH> &S, const float *Ub, float mean, int r0, int r1, int idx,
                                        int stride)
{
    for (int item = r0 * (RS / 4) + idx; item < r1 * (RS / 4); item += stride) {
        const int i = item / (RS / 4), x0 = 4 * (item % (RS / 4));
        const float4 *src = reinterpret_cast<const float4 *>(&Ub[i * UC + x0]);
        const float4 a0 = src[0], a1 = src[1], a2 = src[2];
        const float v[11] = {a0.x - mean, a0.y - mean, a0.z - mean, a0.w - mean, a1.x - mean, a1.y - mean,
                             a1.z - mean, a1.w - mean, a2.x - mean, a2.y - mean, a2.z - mean};
        uint4 *dst = &S.E[0][i * RS + x0];
        if (TF) {
            uint32_t c[11];
#pragma unroll
            for (int j2 = 0; j2 < 11; ++j2) c[j2] = to_tf32(v[j2]);
            uint4 *dst1 = &S.E[TcOps<TF>::EB - 1][i * RS + x0];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                dst[e] = make_uint4(c[e], c[e + 1], c[e + 2], c[e + 3]);
                dst1[e] = make_uint4(c[e + 4], c[e + 5], c[e + 6], c[e + 7]);
            }
        } else {
            uint32_t pr[10];
#pragma unroll
            for (int j2 = 0; j2 < 10; ++j2) pr[j2] = pack_bf16x2(v[j2], v[j2 + 1]);
#pragma unroll
            for (int e = 0; e < 4; ++e) dst[e] = make_uint4(pr[e], pr[e + 2], pr[e + 4], pr[e + 6]);
        }
    }
}

// Range offset of the tile whose input region is Ub (warp-collective; every lane gets it).  Any constant c gives
// K(u - c) = K u (zero-mean filters); c only sets the BF16 / TF32 rounding, so the mean of 64 samples of the
// region (an 8 x 8 grid) serves.
template <int TOH>
__device__ __forceinline__ float region_mean(const float *Ub, int lane)
{
    float v = 0.0f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int sidx = lane + 32 * h;
        v += Ub[(2 + (kUR<TOH> - 4) / 7 * (sidx >> 3)) * UC + 2 + 5 * (sidx & 7)];
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v * (1.0f / 64.0f);
}

// Issue the asynchronous copies of the output-pass operands (delta, d) of the tile whose geometry is in buffer b
// (all threads; the caller commits).  The operand buffer is single: these are issued once the previous tile's
// output pass is over, and are first needed at the end of the tile's own pipeline.
template <int MODE, bool TF, int TOH>
__device__ __forceinline__ void stage_operands(const LaunchArgs &A, TcSmem<TF, TOH> &S, int b, int warp, int lane)
{
    const int im = S.geo[b][0], oy0 = S.geo[b][1], ox0 = S.geo[b][2];
    const ImgDesc &D = A.img[im];
    const int H = D.H, W = D.W, ld = D.ld;
    if (lane < TO) {
        const int gx = ox0 + lane;
        for (int r = warp; r < TOH; r += NWARP) {
            const int gy = oy0 + r, j = r * TO + lane;
            if (gy >= H || gx >= W) continue;
            const size_t idx = (size_t)gy * ld + gx;
            if (MODE == kStep) cp_async4(&S.O[0][j], D.delta + idx);
            if (MODE == kStep || MODE == kGrad) cp_async4(&S.O[1][j], D.d + idx);
        }
    }
}

// Persistent: CTA c processes tiles c, c + gridDim.x, ...; tensor memory, barriers and the filter operands
// are set up once, and the input region of the next tile is copied in while the current one is computed.
// (kHvp / kHess hold 48 Hessian factors per expert thread: one CTA per SM, which leaves them the registers)
template <int MODE, bool TF, int TOH>
__global__ void __launch_bounds__(NTHR, (MODE == kHvp || MODE == kHess) ? 1 : 2)
    k_foe_tc(const __grid_constant__ LaunchArgs A, int *status)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem<TF, TOH> &S = *reinterpret_cast<TcSmem<TF, TOH> *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = A.tile_prefix[A.nimg];
    if ((int)blockIdx.x >= ntiles) return;
    // the next launch in the stream may be scheduled now; its CTAs take an SM as ours leave it and set up their
    // barriers and tensor memory while the rest of this grid finishes
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    // ---- barriers, tensor memory, filter operands (one bulk copy) ----
    constexpr uint32_t WBYTES = sizeof(uint4) * (TcOps<TF>::WF + TcOps<TF>::WA);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&S.bar[B_FWD + b], 1);
            mbar_init(&S.bar[B_RFREE + b], 1);
            mbar_init(&S.bar[B_PSI + b], 16 * NEPI);
            mbar_init(&S.bar[B_ADJ + b], 1);
            mbar_init(&S.bar[B_ZFREE + b], 16 * NEPI);
            mbar_init(&S.bar[B_DRAIN + b], 1);
        }
        mbar_init(&S.bar[B_W], 1);
        mbar_init(&S.bar[B_UREADY], NTHR);
        mbar_init(&S.bar[B_UREADY + 1], NTHR);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the tile table for tile_geometry (read after the __syncthreads below)
    if (tid <= A.nimg) S.tprefix[tid] = A.tile_prefix[tid];
    if (tid < A.nimg) {
        S.timg[tid][0] = A.img[tid].tiles_x;
        S.timg[tid][1] = A.img[tid].H;
        S.timg[tid][2] = A.img[tid].W;
    }
    if (warp == FWD_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // nothing above read memory that an earlier launch writes: from here on its results (the iterate, the filter
    // operands, *status) are needed, so wait until that grid has completed and its writes are visible (returns at
    // once when this launch has no programmatic dependency)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    // an earlier launch that gave up leaves *status set: then do nothing (CTA-uniform decision)
    // (and the stopping words: tiles of stopped images are skipped)
    if (tid == 0) S.abort_flag = *(volatile int *)status;
    if (tid < A.nimg) S.live[tid] = !image_stopped(A.img[tid]);
    __syncthreads();
    const int tile0 = tc_next_live(A, S, ntiles, blockIdx.x);
    if (tid == 0) S.tnext[0] = tc_next_live(A, S, ntiles, tile0 + (int)gridDim.x);  // read after the barrier below
    if (S.abort_flag || tile0 >= ntiles) {
        if (warp == FWD_WARP) {
            const uint32_t tm = S.tmem_base;
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(TMEM_COLS) : "memory");
        }
        return;
    }
    if (tid == 0) {
        mbar_arrive_expect_tx(&S.bar[B_W], WBYTES);
        bulk_g2s(S.Wf, TF ? A.tcops32 : A.tcops, WBYTES, &S.bar[B_W]);
    }
    stage_input<TF, TOH>(A, S, tile0, 0, tid, warp, lane);
    stage_operands<MODE, TF, TOH>(A, S, 0, warp, lane);
    cp_async_commit();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_base;
    volatile int *abort_flag = &S.abort_flag;

    int k = 0;
    // the CTA's next tile is kept in shared memory (S.tnext[buf], written by thread 0 one tile ahead): a value
    // kept live in registers across the tile made the kernel spill
    for (int tile = tile0; tile < ntiles; tile = S.tnext[k & 1], ++k) {
        const int buf = k & 1;
        const int im = S.geo[buf][0], oy0 = S.geo[buf][1], ox0 = S.geo[buf][2], xe = S.geo[buf][3], xs = S.geo[buf][4];
        const ImgDesc &D = A.img[im];
        const int H = D.H, W = D.W, ld = D.ld;

        // this tile's input region has landed (it was copied in during the previous tile; the newest group, this
        // tile's output-pass operands, may still be in flight); start the next tile's.  Groups are committed even
        // when empty, so their count per tile is fixed.
        if (k > 0) cp_async_wait<1>();
        else cp_async_wait<0>();
        __syncthreads();
        if (tid == 0) {
            const int tn = S.tnext[buf];
            S.tnext[buf ^ 1] = tn < ntiles ? tc_next_live(A, S, ntiles, tn + (int)gridDim.x) : ntiles;
        }
        if (const int tn = S.tnext[buf]; tn < ntiles) stage_input<TF, TOH>(A, S, tn, buf ^ 1, tid, warp, lane);
        cp_async_commit();

        // ---- E: built here for the first tile; the expert warps build it for the later ones at the end of the
        // previous tile ----
        const float *Ub = S.U[buf];
        if (k == 0) {
            if (warp == 0) {
                const float m = region_mean<TOH>(Ub, lane);
                if (lane == 0) S.mean0 = m;
            }
            __syncthreads();
            build_e(S, Ub, S.mean0, 0, kUR<TOH>, tid, NTHR);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
        fence_after();

        if (warp == FWD_WARP || warp == ADJ_WARP) {
            {
                // ---------------- MMA issue (warp-uniform; one elected lane issues) ----------------
                // g counts M-tiles over all tiles of the CTA: M-tile g uses stage g & 1, and a stage barrier's phase
                // for M-tile g has parity (g >> 1) & 1 (a tile may hold an odd number of M-tiles)
                bool ok = k > 0 || mbar_wait_warp(&S.bar[B_W], 0, abort_flag, status);
                if (warp == FWD_WARP) {
                    // R(t) = E-window(t) x Wf^T into stage t & 1, once the adjoint of M-tile t - 2 is complete
                    constexpr uint32_t IDF = TF ? idesc_tf32(128, 48) : idesc_bf16(128, 48);
                    const uint32_t e0 = smem_u32(S.E[0]), e1 = smem_u32(S.E[TcOps<TF>::EB - 1]);
                    const uint64_t dE = sdesc(e0, TF ? e1 - e0 : RS * 16, 128), dW = sdesc(smem_u32(S.Wf), 768, 128);
                    for (int t = 0; ok && t < kNMT<TOH>; ++t) {
                        const int g = kNMT<TOH> * k + t;
                        if (g >= 2 && !mbar_wait_warp(&S.bar[B_RFREE + (g & 1)], ((g - 2) >> 1) & 1, abort_flag, status)) break;
                        fence_after();
                        const uint32_t d = tmem + 64 * (g & 1);
                        if (TF) {
                            // K-step a = one tap row (8 columns: E[0] holds columns 0-3, E[1] columns 4-7); row 7 has
                            // zero weights and is skipped
#pragma unroll
                            for (int kk = 0; kk < 7; ++kk)
                                mma_elect<TF>(d, dE + (uint64_t)((4 * t + kk) * RS), dW + (uint64_t)(kk * 96), IDF, kk > 0);
                        } else {
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                mma_elect<TF>(d, dE + (uint64_t)((4 * t + 2 * kk) * RS), dW + (uint64_t)(kk * 96), IDF, kk > 0);
                        }
                        commit_elect(&S.bar[B_FWD + (g & 1)]);
                    }
                } else {
                    // Z(t) = Psi(t) x Wa^T into Z stage t & 1, once Psi(t) is in tensor memory and Z(t - 2) has
                    // been loaded; A = Psi(t) in the first columns of R(t)'s stage (8 columns per K-step: 16 bf16
                    // or 8 tf32 filters)
                    constexpr uint32_t IDA = TF ? idesc_tf32(128, 64) : idesc_bf16(128, 64);
                    const uint64_t dWa = sdesc(smem_u32(S.Wa), 1024, 128);
                    for (int t = 0; ok && t < kNMT<TOH>; ++t) {
                        const int g = kNMT<TOH> * k + t;
                        if (!mbar_wait_warp(&S.bar[B_PSI + (g & 1)], (g >> 1) & 1, abort_flag, status)) break;
                        if (g >= 2 && !mbar_wait_warp(&S.bar[B_ZFREE + (g & 1)], ((g - 2) >> 1) & 1, abort_flag, status)) break;
                        fence_after();
                        const uint32_t d = tmem + Z_COL0 + 64 * (g & 1), a = tmem + 64 * (g & 1);
#pragma unroll
                        for (int kk = 0; kk < (TF ? 6 : 3); ++kk)
                            mma_ta_elect<TF>(d, a + 8 * kk, dWa + (uint64_t)(kk * 128), IDA, kk > 0);
                        // (a failure-detection test makes CTA 0 withhold this arrival once: the col2im warps' bounded
                        // wait then expires and the launch reports FOE_ETIMEOUT)
                        if (!(A.withhold_arrival && blockIdx.x == 0 && g == 0)) commit_elect(&S.bar[B_ADJ + (g & 1)]);
                        commit_elect(&S.bar[B_RFREE + (g & 1)]);
                    }
                }
            }
            __syncwarp();
        } else {
            // ---------------- epilogue warps ----------------
            // warp w reads and writes TMEM lanes 32q..32q+31, q = w % 4 (response row 4t+q of M-tile t).  Warps 0-3
            // run the expert step of all 48 filters (R(t) -> Psi(t), in place in R(t)'s stage), warps 4-7 the
            // col2im of all 7 tap rows (Z(t) -> horizontal partials in shared memory).
            const int q = warp & 3;
            // interior tile: the whole response region lies in the image, so no response is masked and no
            // lane outside 3..28 is ever read (no padding fold)
            const bool interior = oy0 >= 3 && ox0 >= 3 && oy0 + kRR<TOH> - 3 <= H && ox0 + RS - 3 <= W;
            const uint32_t lane_base = (uint32_t)(32 * q) << 16;
            if (warp < 4) {
                const int gx = ox0 - 3 + lane;
                bool done = false;
                for (int t = 0; t < kNMT<TOH>; ++t) {
                    const int g = kNMT<TOH> * k + t;
                    const int gy = oy0 - 3 + 4 * t + q;
                    const bool in_img = gy >= 0 && gy < H && gx >= 0 && gx < W;
                    const uint32_t keep = (interior || in_img) ? 0xFFFFFFFFu : 0u;
                    // kHvp: the Hessian factors of this lane's response pixel, loaded before the wait so that the
                    // load overlaps it (zero outside the image, where the product is masked anyway)
                    float fh[MODE == kHvp ? 48 : 1];
                    if constexpr (MODE == kHvp) {
                        const float4 *fp = reinterpret_cast<const float4 *>(D.hess + ((size_t)gy * W + gx) * 48);
#pragma unroll
                        for (int j = 0; j < 12; ++j) {
                            const float4 v = in_img ? __ldg(fp + j) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                            fh[4 * j] = v.x;
                            fh[4 * j + 1] = v.y;
                            fh[4 * j + 2] = v.z;
                            fh[4 * j + 3] = v.w;
                        }
                    }
                    // kHess: the factors are stored for the pixels of the tile's own output region (every image pixel
                    // belongs to one tile), so each is written once
                    const bool own = MODE == kHess && gy >= oy0 && gy < oy0 + TOH && gy < H && gx >= xs && gx < xe;
                    if (!mbar_wait(&S.bar[B_FWD + (g & 1)], (g >> 1) & 1, abort_flag, status)) break;
                    fence_after();
                    const uint32_t rc = tmem + lane_base + 64 * (g & 1);
                    if (TF) {
                        // Psi takes R's columns one for one: two halves of 24 filters keep the registers low
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            float r[24];
                            tmem_ld16(rc + 24 * hh, r);
                            tmem_ld8(rc + 24 * hh + 16, r + 16);
                            tmem_wait_ld();
                            uint32_t w[24];
                            if constexpr (MODE == kHvp) {
                                // the Hessian applied to the direction: (rho''(K_i u) / 2) (K_i p) (2 alpha_i in Wa)
#pragma unroll
                                for (int j = 0; j < 24; ++j) w[j] = to_tf32(r[j] * fh[24 * hh + j]) & keep;
                            } else if constexpr (MODE == kHess) {
                                float fac[24];
#pragma unroll
                                for (int j = 0; j < 24; ++j) {
                                    const float r0 = r[j], inv = rcp_approx(fmaf(r0, r0, 1.0f));
                                    fac[j] = fmaf(-r0, r0, 1.0f) * inv * inv;
                                    w[j] = 0u;
                                }
                                if (own) {
                                    float4 *fo = reinterpret_cast<float4 *>(D.hess + ((size_t)gy * W + gx) * 48 + 24 * hh);
#pragma unroll
                                    for (int j = 0; j < 6; ++j)
                                        fo[j] = make_float4(fac[4 * j], fac[4 * j + 1], fac[4 * j + 2], fac[4 * j + 3]);
                                }
                            } else {
#pragma unroll
                                for (int j = 0; j < 24; ++j) {
                                    const float r0 = r[j];
                                    w[j] = to_tf32(r0 * rcp_approx(fmaf(r0, r0, 1.0f))) & keep;
                                }
                            }
                            tmem_st16(rc + 24 * hh, w);
                            tmem_st8(rc + 24 * hh + 16, w + 16);
                        }
                    } else {
                        float r[48];
                        tmem_ld32(rc, r);
                        tmem_ld16(rc + 32, r + 32);
                        tmem_wait_ld();
                        uint32_t w[24];
#pragma unroll
                        for (int j = 0; j < 24; ++j) w[j] = psi_bf16x2(r[2 * j], r[2 * j + 1]);
                        if (!interior) {
#pragma unroll
                            for (int j = 0; j < 24; ++j) w[j] &= keep;
                        }
                        tmem_st16(rc, w);
                        tmem_st8(rc + 16, w + 16);
                    }
                    tmem_wait_st();
                    fence_before();
                    mbar_arrive(&S.bar[B_PSI + (g & 1)]);
                    if (t == kNMT<TOH> - 1) done = true;
                }
                // every forward MMA of this tile is complete (each expert thread saw the last one), so E is free:
                // the next tile's E is built while the last adjoint and col2im finish
                if (done && S.tnext[buf] < ntiles &&
                    mbar_wait(&S.bar[B_UREADY + (buf ^ 1)], ((k + 1) >> 1) & 1, abort_flag, status)) {
                    const float m = region_mean<TOH>(S.U[buf ^ 1], lane);
                    build_e(S, S.U[buf ^ 1], m, 0, kUR<TOH>, tid, 128);
                }
            } else {
                for (int t = 0; t < kNMT<TOH>; ++t) {
                    const int g = kNMT<TOH> * k + t;
                    if (!mbar_wait(&S.bar[B_ADJ + (g & 1)], (g >> 1) & 1, abort_flag, status)) break;
                    fence_after();
                    float z[56];
                    const uint32_t zc = tmem + lane_base + Z_COL0 + 64 * (g & 1);
                    tmem_ld32(zc, z);
                    tmem_ld16(zc + 32, z + 32);
                    tmem_ld8(zc + 48, z + 48);  // tap row 7 has zero weights
                    tmem_wait_ld();
                    fence_before();
                    mbar_arrive(&S.bar[B_ZFREE + (g & 1)]);
                    const int rr = 4 * t + q;
                    if (interior) {
                        // all 42 shuffles first, then the sums: independent work to cover the shuffle latency
                        float sh[7][6];
#pragma unroll
                        for (int a = 0; a < 7; ++a) {
                            sh[a][0] = __shfl_down_sync(0xffffffffu, z[8 * a + 0], 3);
                            sh[a][1] = __shfl_down_sync(0xffffffffu, z[8 * a + 1], 2);
                            sh[a][2] = __shfl_down_sync(0xffffffffu, z[8 * a + 2], 1);
                            sh[a][3] = __shfl_up_sync(0xffffffffu, z[8 * a + 4], 1);
                            sh[a][4] = __shfl_up_sync(0xffffffffu, z[8 * a + 5], 2);
                            sh[a][5] = __shfl_up_sync(0xffffffffu, z[8 * a + 6], 3);
                        }
#pragma unroll
                        for (int a = 0; a < 7; ++a)
                            hs_put(S.Hs[(a * kRR<TOH> + rr) * RS + lane],
                                   ((z[8 * a + 3] + sh[a][0]) + (sh[a][1] + sh[a][2])) + ((sh[a][3] + sh[a][4]) + sh[a][5]));
                    } else {
#pragma unroll
                        for (int a = 0; a < 7; ++a) {
                            const float *za = z + 8 * a;
                            float h;
                            h = za[3];
#pragma unroll
                            for (int bb = 0; bb < 7; ++bb) {
                                if (bb == 3) continue;
                                const int src = lane + 3 - bb;
                                const float v = __shfl_sync(0xffffffffu, za[bb], src & 31);
                                h += (src >= 0 && src < 32) ? v : 0.0f;
                            }
                            hs_put(S.Hs[(a * kRR<TOH> + rr) * RS + lane], h);
                        }
                    }
                }
            }
        }

        // the output-pass operands have landed (only the next tile's input region may still be in flight)
        cp_async_wait<1>();
        fence_before();
        __syncthreads();

        // ---------------- output pass: vertical col2im, padding fold, iPiano step ----------------
        // warp w handles output rows w, w + 9/10, w + 2*(9/10) (lane = column): the rows are unrolled so that their
        // independent update chains interleave
        const bool ring = A.bc == kSymmetric && (oy0 < 3 || ox0 < 3 || oy0 + TOH > H - 3 || ox0 + TO > W - 3);
        constexpr int NR = (TOH + NWARP - 1) / NWARP;
        if (lane < TO) {
            const int xo = 3 + lane, gx = ox0 + lane;
            float g[NR], uh[NR];
            bool ok_r[NR];
#pragma unroll
            for (int k2 = 0; k2 < NR; ++k2) {
                const int r = warp + k2 * NWARP, yo = 3 + r, gy = oy0 + r;
                ok_r[k2] = r < TOH && gy < H && gx < xe && gx >= xs;
                g[k2] = 0.0f;
                uh[k2] = 0.0f;
                if (ok_r[k2]) {
                    g[k2] = hs_sum(S, yo, xo);
                    uh[k2] = Ub[(yo + 3) * UC + xo + 3];
                    if (ring) {
                        const int my = gy < 3 ? -1 - gy : (gy >= H - 3 ? 2 * H - 1 - gy : -1000);
                        const int mx = gx < 3 ? -1 - gx : (gx >= W - 3 ? 2 * W - 1 - gx : -1000);
                        if (my != -1000) g[k2] += hs_gather(S, my - oy0 + 3, xo);
                        if (mx != -1000) g[k2] += hs_gather(S, yo, mx - ox0 + 3);
                        if (my != -1000 && mx != -1000) g[k2] += hs_gather(S, my - oy0 + 3, mx - ox0 + 3);
                    }
                }
            }
#pragma unroll
            for (int k2 = 0; k2 < NR; ++k2) {
                if (!ok_r[k2]) continue;
                const int r = warp + k2 * NWARP, j = r * TO + lane;
                const size_t idx = (size_t)(oy0 + r) * ld + gx;
                if (MODE == kGrad) {
                    D.out[idx] = g[k2] + data_grad(uh[k2], S.O[1][j], D.model, D.sc.lambda);
                } else if (MODE == kHvp) {
                    // H_E p = H_prior p + lambda p (the quadratic data term of the Anscombe-L2 model)
                    D.out[idx] = g[k2] + D.sc.lambda * uh[k2];
                } else if (MODE == kHess) {
                    // factors only
                } else {
                    float nh, nd;
                    ipiano_update_f32(g[k2], uh[k2], S.O[0][j], S.O[1][j], D.model, D.sc, nh, nd);
                    D.u_hi[A.parity ^ 1][idx] = nh;
                    D.delta[idx] = nd;
                }
            }
        }

        // Hs and this tile's buffers are reused by the next tiles
        __syncthreads();
        if (*abort_flag) break;
        if (S.tnext[buf] < ntiles) stage_operands<MODE, TF, TOH>(A, S, buf ^ 1, warp, lane);
        cp_async_commit();
    }

    // every MMA issued by the two MMA threads is complete before tensor memory is released.  If this bounded wait
    // expired the launch has already recorded FOE_ETIMEOUT and its results are discarded; the columns are released
    // all the same: a CTA must free its tensor memory before it exits, and columns left allocated would hold every
    // later CTA of the SM in tcgen05.alloc
    if (warp == FWD_WARP || warp == ADJ_WARP) {
        uint64_t *bar = &S.bar[B_DRAIN + (warp == FWD_WARP ? 0 : 1)];
        commit_elect(bar);
        const long long t0 = clock64();
        while (!mbar_try_wait(bar, 0))
            if (clock64() - t0 > kTimeoutCycles) {
                atomicExch(status, 5);
                break;
            }
    }
    cp_async_wait<0>();
    fence_before();
    __syncthreads();
    if (warp == FWD_WARP) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// Dynamic shared memory per CTA.  At most two CTAs share an SM (2 x 256 TMEM columns); the request is
// raised so that a third CTA, which would wait in tcgen05.alloc, is never made resident.
template <bool TF, int TOH>
constexpr size_t smem_request()
{
    return sizeof(TcSmem<TF, TOH>) > 80 * 1024 ? sizeof(TcSmem<TF, TOH>) : 80 * 1024;
}

template <int MODE, bool TF, int TOH>
cudaError_t tc_launch_one(const LaunchArgs &a, int grid, int *d_status, cudaStream_t s)
{
    // programmatic dependent launch: the kernel waits (griddepcontrol.wait) for the preceding grid before it
    // reads anything that grid may write
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NTHR);
    cfg.dynamicSmemBytes = smem_request<TF, TOH>();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_foe_tc<MODE, TF, TOH>, a, d_status);
}

template <int MODE, bool TF, int TOH>
cudaError_t tc_attr()
{
    return cudaFuncSetAttribute(k_foe_tc<MODE, TF, TOH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_request<TF, TOH>());
}

}  // namespace

// BF16 images of at least pair_min_rows() rows and pair_min_pixels() pixels take the pixel-pair kernel's tiles;
// the rest take 26 x 26 tiles.  The pair kernel runs one CTA per SM and a tile in about 20 us; the 26 x 26 kernel
// runs two CTAs per SM and a tile in about 10 us, so it finishes small images sooner (300 iterations: 256^2 alone
// 3.7 ms against 7.1 ms) while the pair kernel does more per SM once there is enough work (five 512^2 images together:
// 15.8 ms against 19.5 ms).  The threshold of 90000 pixels (300^2) gave the most on 64 uneven images in one batch
// (29.2 k MPix.iter/s, against 26.6 k at 200000 and 28.9 k with pair tiles for all).  The choice depends on the image
// alone, so an image is tiled, and rounded, the same way in any batch.
int tc_tile_h(bool tf32, int H, int W)
{
    return !tf32 && H >= pair_min_rows() && (long)H * W >= pair_min_pixels() ? pair_tile_h() : kShortH;
}
int tc_tile_w(int tile_h) { return tile_h == pair_tile_h() ? pair_tile_w() : TO; }

cudaError_t tc_setup()
{
    cudaError_t e;
    if ((e = tc_attr<kStep, false, kShortH>())) return e;
    if ((e = tc_attr<kGrad, false, kShortH>())) return e;
    if ((e = tc_attr<kStep, true, kShortH>())) return e;
    if ((e = tc_attr<kGrad, true, kShortH>())) return e;
    if ((e = tc_attr<kHvp, true, kShortH>())) return e;
    if ((e = tc_attr<kHess, true, kShortH>())) return e;
    return pair_setup();
}

cudaError_t tc_launch(const LaunchArgs &a, int mode, bool tf32, int *d_status, cudaStream_t s, const SideStream &side)
{
    if (a.nimg <= 0 || a.tile_prefix[a.nimg] <= 0) return cudaSuccess;
    if (mode != kStep && mode != kGrad && !(tf32 && (mode == kHvp || mode == kHess))) return cudaErrorNotSupported;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // images in pixel-pair tiles run in the pixel-pair kernel (foe_pair.cu), the others (26 x 26 tiles, and every TF32
    // image) here; a launch holding both kinds runs one launch of each kernel at the same time: the 26 x 26 kernel
    // on the side stream, forked after the work queued so far and joined back before whatever is queued next, so that
    // each kernel's CTAs take the SMs that the other leaves free (one pair CTA or two 26 x 26 CTAs fit an SM)
    int npair = 0;
    for (int i = 0; i < a.nimg; ++i) npair += a.img[i].tile_h == pair_tile_h();
    const bool both = npair > 0 && npair < a.nimg;
    if (both) {
        if ((e = cudaEventRecord(side.fork, s)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side.stream, side.fork, 0)) != cudaSuccess) return e;
    }
    if (npair > 0 && (e = pair_launch(a, mode, npair == a.nimg, sms, d_status, s)) != cudaSuccess) return e;
    if (npair == a.nimg) return cudaSuccess;
    const cudaStream_t s26 = both ? side.stream : s;
    LaunchArgs b = a;
    b.nimg = 0;
    b.tile_prefix[0] = 0;
    for (int i = 0; i < a.nimg; ++i) {
        if (a.img[i].tile_h == pair_tile_h()) continue;
        b.img[b.nimg] = a.img[i];
        b.tile_prefix[b.nimg + 1] = b.tile_prefix[b.nimg] + (a.tile_prefix[i + 1] - a.tile_prefix[i]);
        b.nimg++;
    }
    const int tiles = b.tile_prefix[b.nimg];
    // persistent CTAs: as many as are resident at once (tensor memory admits two per SM)
    const int grid = std::min(tiles, 2 * sms);
    if (tf32) e = mode == kStep  ? tc_launch_one<kStep, true, kShortH>(b, grid, d_status, s26)
                  : mode == kGrad ? tc_launch_one<kGrad, true, kShortH>(b, grid, d_status, s26)
                  : mode == kHvp  ? tc_launch_one<kHvp, true, kShortH>(b, std::min(tiles, sms), d_status, s26)
                                  : tc_launch_one<kHess, true, kShortH>(b, std::min(tiles, sms), d_status, s26);
    else e = mode == kStep ? tc_launch_one<kStep, false, kShortH>(b, grid, d_status, s26)
                           : tc_launch_one<kGrad, false, kShortH>(b, grid, d_status, s26);
    if (e != cudaSuccess || !both) return e;
    if ((e = cudaEventRecord(side.join, side.stream)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(s, side.join, 0);
}

}  // namespace foe
