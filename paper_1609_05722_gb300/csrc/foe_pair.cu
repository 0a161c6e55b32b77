// Pixel-pair tensor-core FoE step kernel for sm_103a (BF16 operands, kind::f16, FP32 accumulators in tensor
// memory): one iPiano step (Eq. iPianoupdate) per launch over output tiles of 58 columns x 66 rows, one persistent
// CTA per SM.
//
// The prior gradient sum_i alpha_i K_i^T rho'(K_i u) (Eq. FoEF) of a tile needs the responses on the tile plus a
// 3-pixel ring: a response region of 64 columns x 72 rows.  Each tensor-memory lane holds two horizontally adjacent
// response pixels (a pair), so an M-tile of 128 lanes is 4 response rows of 32 pairs and a tile is 18 M-tiles.  The
// width is fixed by the 32 pairs of a lane quarter; the height is a choice: 66 rows against 58 (16 M-tiles) cut the
// ten-image 512^2 benchmark step from 28.6 to 27.1 ms (720 tiles per launch fill 5 waves of 152 CTAs, 810 filled
// 6) and 64 uneven images from 29.1 to 29.7 k MPix.iter/s, while a lone 512^2 image (one wave either way) takes
// 7.9 ms against 7.2 ms and five 512^2 images 17.4 against 15.9 ms.
//
//   forward  R[m][n] = sum_k E-window(m)[k] Wf[n][k]        M = 128 pairs, N = 96 = 2 pixels x 48 filters,
//            K = 64 = 8 tap rows x 8 columns: the 8 columns cover the 7 taps of both pixels of a pair, and the
//            E operand holds for every pair position the 8 bf16 inputs u(y, x-3 .. x+4) in one 16-byte entry,
//            so the K-slice "tap rows 2s, 2s+1" of an M-tile is two row-shifted views of E.
//   expert   psi = rho'(R) / 2 = R / (1 + R^2) (the factor 2 alpha_i lives in Wa), zero outside the image, written
//            as bf16 pairs into a Psi stage of 48 columns (the adjoint's K order: pixel, then filter).  One
//            reciprocal serves two filters, psi_0 = r_0 d_1 / (d_0 d_1) with d = 1 + r^2, which halves the MUFU
//            work (16 reciprocals per clock and SM bound the step otherwise).
//   adjoint  Z2[m][n'] = sum_K Psi[m][K] Wa[n'][K]          K = 96 (both pixels' psi, read from tensor memory),
//            N = 64 = 8 tap rows x 8 column offsets c: Z2_{a,c}(pair j) is the contribution of pair j to the output
//            column 2j + c - 3 of response row y + a - 3.
//   col2im   horizontal: each output pair sums 4 values from pairs j-2 .. j+2 per tap row (6 warp shuffles and
//            3 packed adds for two pixels); vertical: a register carry over the rows of each lane quarter, stored as
//            four FP16 partial rows per output row, summed in FP32 in the output pass.
//
// Roles (20 warps): 0-7 expert (warp w: TMEM lane quarter w % 4, response columns 48 (w / 4) .. + 47, one pixel of
// the pair), 8-11 col2im (lane quarter w % 4), 12 forward MMA issue, 13 adjoint MMA issue, 14-17 output pass,
// 18-19 staging.  (12 expert warps of 32 columns measured 52.8 us per 5 x 512^2 launch, 8 of 48 columns 50.9 us,
// 4 of 96 columns 51.2 us; with the current output pass, 12 expert warps take the ten-image step to 24.1 ms against
// 23.0.)  The staging warps copy in the next tile's input region (one TMA box; for border tiles under symmetric
// padding the reflected ring is then filled in from the box) and build its E operand (double-buffered) while the
// current tile runs; the output warps run the
// output pass (padding fold, iPiano step) of the current tile row by row as the col2im warps finish its M-tiles,
// with their operands loaded into registers two M-tiles ahead.  No role waits for a whole-CTA barrier between
// tiles.  Tensor memory holds three stages of R (96 columns), two of Psi (48) and two of Z2 (64); M-tile g (counted
// over all tiles of the CTA) uses R stage g % 3 and Psi / Z2 stage g % 2.  An R stage is free for the forward MMAs
// of M-tile g + 3 as soon as the expert warps have loaded R(g), so the forward MMAs run ahead of the adjoint.
// Every mbarrier wait is bounded: on expiry the CTA records FOE_ETIMEOUT in *status, the other roles give up at
// their next wait, the MMAs drain, tensor memory is freed.
//
// BF16 range: filters are zero-mean, so K(u - c) = K u; the mean of 64 samples of the tile's input region is
// subtracted before rounding u to BF16 (under zero padding the padded zeros are shifted too).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include "foe_common.cuh"
#include "foe_kernels.h"
#include "foe_ptx.cuh"

namespace foe {

namespace {

using namespace ptx;

constexpr int PTX = 58;              // output tile width (32 pairs of response columns, less the 3-pixel ring)
constexpr int PTY = 66;              // output tile height
constexpr int PRX = PTX + 6;         // response columns: 64
constexpr int PRY = PTY + 6;         // response rows
constexpr int PNMT = PRY / 4;        // M-tiles per tile
constexpr int PER = PRY + 7;         // E rows = input rows: 7 tap rows + the zero-weight eighth
static_assert(PRX == 64 && PRY % 4 == 0, "tile geometry");
constexpr int PUW = 70;              // input columns used: 64 response columns + 6
constexpr int PUC = 76;              // floats per staged input row (the TMA box: 70 + up to 3 of alignment slack)
constexpr int kPairMinRows = PTY + 1; // images of fewer rows keep the 26 x 26 tiles
constexpr int NRST = 3;              // response stages R (96 columns each)
constexpr int NPST = 2;              // Psi stages (48 columns each)
constexpr int NZST = 2;              // Z2 stages (64 columns each)
constexpr uint32_t kRCols = 96, kPsiCols = 48, kZCols = 64;
constexpr uint32_t kPsiCol0 = NRST * kRCols, kZCol0 = kPsiCol0 + NPST * kPsiCols;
static_assert(kZCol0 + NZST * kZCols <= 512, "tensor memory");
constexpr uint32_t kTmemCols = 512;
constexpr int NEXP = 8, FWDW = NEXP + 4, ADJW = FWDW + 1, OUTW0 = ADJW + 1, STGW0 = OUTW0 + 4, NSTGW = 2;
constexpr int kExpCols = 96 / (NEXP / 4);  // response columns (of the 96 of a pair) per expert warp
constexpr int kExpPart = kExpCols > 48 ? 48 : kExpCols;  // columns loaded and converted at a time
static_assert(kExpCols == 32 || kExpCols == 48 || kExpCols == 96, "expert warps");
constexpr int NW = STGW0 + NSTGW, NT = 32 * NW, NPROD = 128;  // 4 output warps
constexpr int NSTG = 32 * NSTGW;     // staging threads
constexpr int WF_ENT = 8 * 96;       // forward B: [tap row a][n = 48 s + e] of 8 tap columns
constexpr int WA_ENT = 12 * 64;      // adjoint B: [K chunk][n' = 8 a + slot] of 8 K values
constexpr uint32_t kOpsBytes = 16u * (WF_ENT + WA_ENT);
constexpr uint32_t kUBoxBytes = 4u * PUC * PER;
constexpr int kEItems = PER * 8;     // E build items (4 entries of one row each)
constexpr int kBarProd = 1;          // named barrier of the staging warps

// mbarriers
constexpr int B_FWD = 0;      // [3] forward MMAs of M-tile g complete: R(g) ready           count 1 (commit)
constexpr int B_RFREE = 3;    // [3] R(g) loaded by every expert thread: the R stage is free  count 32 NEXP
constexpr int B_PSI = 6;      // [NPST] Psi(g) in tensor memory (every expert thread)         count 32 NEXP
constexpr int B_PFREE = 9;    // [NPST] adjoint MMAs of g complete: the Psi stage is free     count 1 (commit)
constexpr int B_ADJ = 12;     // [NZST] adjoint MMAs of g complete: Z2(g) ready                count 1 (commit)
constexpr int B_ZFREE = 15;   // [NZST] Z2(g) loaded by every col2im thread                   count 128
constexpr int B_EREADY = 18;  // [2] E buffer b built                                         count NSTG
constexpr int B_EFREE = 20;   // [2] every forward MMA reading E buffer b complete            count 1 (commit)
constexpr int B_CDONE = 22;   // [2][PNMT] col2im of M-tile t of the tile in buffer b emitted count 128
constexpr int B_GFREE = B_CDONE + 2 * PNMT;  // [2] output pass done with partial-sum buffer b  count 128
constexpr int B_ULAND = B_GFREE + 2;  // input region landed (TMA bytes, or every staging copy) count NSTG
constexpr int B_W = B_ULAND + 1;      // filter operand images landed                         count 1 + tx
constexpr int B_DRAIN = B_W + 1;      // [2] all MMAs of the forward / adjoint issuer complete count 1 (commit)
constexpr int NBAR = B_DRAIN + 2;
static_assert(NRST <= 3 && NPST <= 3 && NZST <= 3, "barrier slots");

struct PairSmem {
    float U[PER * PUC];                  // staged input region (TMA destination: offset 0, 1024-aligned)
    uint4 E[2][PER * 32];                // forward A operand: entry (row i, pair j) = bf16 u(i, 2j .. 2j+7) - mean
    uint4 Wf[WF_ENT];
    uint4 Wa[WA_ENT];
    uint4 G[2][PRY][32];                 // vertical col2im partials: [buffer][output row][pair], the f16x2 words of
                                         // the four lane quarters in one 16-byte entry
    int tprefix[kMaxBatch + 1];
    int timg[kMaxBatch][3];              // tiles per row, H, W
    int live[kMaxBatch];                 // 0 once the image's stopping rule has held (its tiles are skipped)
    uint64_t bar[NBAR];
    uint32_t tmem_base;
    int abort_flag;
};
static_assert(sizeof(PairSmem) + 1024 <= 227 * 1024, "pair kernel shared memory");
static_assert(offsetof(PairSmem, E) % 16 == 0 && offsetof(PairSmem, Wf) % 16 == 0, "operand alignment");
static_assert(offsetof(PairSmem, Wa) == offsetof(PairSmem, Wf) + 16 * WF_ENT, "one bulk copy fills Wf and Wa");
static_assert((PUC * 4) % 16 == 0 && PUC <= 256 && PER <= 256, "TMA box");
static_assert(offsetof(PairSmem, bar) % 8 == 0, "mbarrier alignment");

struct PairArgs {
    CUtensorMap tmap[kMaxBatch][2];      // per image: u_hi[0], u_hi[1] as 2-D FP32 tensors (W x H, row pitch ld)
    int nimg, parity, bc, withhold_arrival;
    const void *ops;                     // Wf then Wa (bf16 operand images), 24 KB
    int tile_prefix[kMaxBatch + 1];
    ImgDesc img[kMaxBatch];
};
static_assert(sizeof(PairArgs) < 32000, "kernel parameter space");

struct Geo {
    int im, oy0, ox0, ys, ye, xs, xe, H, W;
};

// Origin and write range of a tile of P outputs along one axis of length L.  The last tile is placed flush with the
// far border, so that the reflections of the pixels within 3 of that border lie inside its response region; the tile
// before it writes only up to max(L - P, 3), which keeps the pixels within 3 of the near border in the first tile
// (origin 0) when the flush tile starts at 1 or 2 (L = P + 1, P + 2).
template <int P>
__device__ __forceinline__ void pair_axis(int t, int n, int L, int &o, int &s, int &e)
{
    o = t * P;
    s = o;
    e = min(o + P, L);
    if (L > P) {
        const int last = L - P, split = max(last, 3);
        o = min(o, last);
        s = t + 1 < n ? o : split;
        e = t + 1 < n ? min(e, split) : L;
    }
}

__device__ __forceinline__ int pair_image(const PairSmem &S, int nimg, int tile)
{
    int lo = 0, hi = nimg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.tprefix[mid] <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The CTA's tiles are tile0, tile0 + gridDim.x, ... without those of stopped images: every role walks the same list.
__device__ __forceinline__ int pair_next_live(const PairSmem &S, int nimg, int ntiles, int tile)
{
    while (tile < ntiles && !S.live[pair_image(S, nimg, tile)]) tile += gridDim.x;
    return tile;
}

__device__ __forceinline__ Geo pair_geometry(const PairSmem &S, int nimg, int tile)
{
    const int lo = pair_image(S, nimg, tile);
    Geo g;
    g.im = lo;
    const int tiles_x = S.timg[lo][0];
    g.H = S.timg[lo][1];
    g.W = S.timg[lo][2];
    const int tiles_y = (g.H + PTY - 1) / PTY, lt = tile - S.tprefix[lo];
    pair_axis<PTX>(lt % tiles_x, tiles_x, g.W, g.ox0, g.xs, g.xe);
    pair_axis<PTY>(lt / tiles_x, tiles_y, g.H, g.oy0, g.ys, g.ye);
    return g;
}

// psi for filters (f0, f1, f2, f3) of one pixel, given as the tensor-memory column pairs (f0, f2) and (f1, f3):
// d = 1 + r^2, one reciprocal per two filters (1 / (d0 d1), 1 / (d2 d3)), psi_0 = r0 d1 / (d0 d1), ...  The words
// are the bf16 pairs (psi_f0, psi_f2) and (psi_f1, psi_f3), the order of the adjoint's K index.  d0 d1 stays finite
// for |r| < 4e9.
__device__ __forceinline__ void psi_quad(float r0, float r2, float r1, float r3, uint32_t &w02, uint32_t &w13)
{
    const uint64_t a02 = f2_pack(r0, r2), a13 = f2_pack(r1, r3);
    const uint64_t d02 = f2_fma(a02, a02, kF2One), d13 = f2_fma(a13, a13, kF2One);
    float e01, e23;
    f2_unpack(f2_mul(d02, d13), e01, e23);
    const uint64_t inv = f2_pack(rcp_approx(e01), rcp_approx(e23));
    float p0, p2, p1, p3;
    f2_unpack(f2_mul(f2_mul(a02, d13), inv), p0, p2);
    f2_unpack(f2_mul(f2_mul(a13, d02), inv), p1, p3);
    w02 = pack_bf16x2(p0, p2);
    w13 = pack_bf16x2(p1, p3);
}

// The same with one reciprocal for all four filters: 1 / (d0 d1 d2 d3), then 1 / (d0 d1) = (d2 d3) / (d0 d1 d2 d3)
// and 1 / (d2 d3) likewise.  The pair products are clamped at 2^62 so that their product stays finite; a clamped
// pair (|r0 r1| beyond about 2^31) keeps psi within 5e-5 of its value for |r| below 1e5.
__device__ __forceinline__ void psi_quad1(float r0, float r2, float r1, float r3, uint32_t &w02, uint32_t &w13)
{
    const uint64_t a02 = f2_pack(r0, r2), a13 = f2_pack(r1, r3);
    const uint64_t d02 = f2_fma(a02, a02, kF2One), d13 = f2_fma(a13, a13, kF2One);
    float e01, e23;
    f2_unpack(f2_mul(d02, d13), e01, e23);
    e01 = fminf(e01, 4.611686e18f);
    e23 = fminf(e23, 4.611686e18f);
    const float inv = rcp_approx(e01 * e23);
    const uint64_t i2 = f2_pack(inv * e23, inv * e01);
    float p0, p2, p1, p3;
    f2_unpack(f2_mul(f2_mul(a02, d13), i2), p0, p2);
    f2_unpack(f2_mul(f2_mul(a13, d02), i2), p1, p3);
    w02 = pack_bf16x2(p0, p2);
    w13 = pack_bf16x2(p1, p3);
}

constexpr bool kOneRcpPerQuad = false;   // psi_quad1 instead of psi_quad

// ring position of M-tile g: stage g % N, barrier phase parity (g / N) & 1
template <int N>
__device__ __forceinline__ void stage_advance(int &stg, uint32_t &ph)
{
    if (++stg == N) {
        stg = 0;
        ph ^= 1u;
    }
}

// Agreement of the `count` threads of named barrier `id`: true only if every one passes ok (also a barrier).
template <int count>
__device__ __forceinline__ bool group_all(int id, bool ok)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)ok), "r"(id), "n"(count)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ bool prod_all(bool ok) { return group_all<NSTG>(kBarProd, ok); }

// Sum of the four partial rows at region position (Y, X), any position of the response region (padding fold).
__device__ __forceinline__ float g_at(const uint4 (*Gb)[32], int Y, int X)
{
    if (Y < 0 || Y >= PRY || X < 0 || X >= PRX) return 0.0f;
    const uint4 e = Gb[Y][X >> 1];
    const uint32_t w[4] = {e.x, e.y, e.z, e.w};
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        s += __half2float(__ushort_as_half((unsigned short)((X & 1) ? (w[q] >> 16) : (w[q] & 0xFFFFu))));
    return s;
}

// Issue the copy of the tile's input region U(i, c) = u(oy0 - 6 + i, ox0 - 6 + c) into S.U (producer threads; each
// arrives on B_ULAND once).  Returns the column offset of c = 0 in the staged rows.  Images of at least the box size
// take one TMA box at x = floor4(ox0 - 6), positions outside the image zero-filled (zero padding exactly; under
// symmetric padding fill_ring then copies in the reflections).  Smaller images take per-element copies through the
// padding map.
__device__ __forceinline__ int stage_region(const PairArgs &A, PairSmem &S, const Geo &g, int p)
{
    const ImgDesc &D = A.img[g.im];
    if (g.W >= PUC && g.H >= PER) {
        const int x = (g.ox0 - 6) & ~3;
        if (p == 0) {
            fence_async_smem();  // the producers' reads of the previous region precede the copy's writes
            mbar_arrive_expect_tx(&S.bar[B_ULAND], kUBoxBytes);
            tma_load_2d(S.U, &A.tmap[g.im][A.parity], x, g.oy0 - 6, &S.bar[B_ULAND]);
        } else {
            mbar_arrive(&S.bar[B_ULAND]);
        }
        return (g.ox0 - 6) - x;
    }
    const float *uin = D.u_hi[A.parity];
    for (int e = p; e < PER * PUW; e += NSTG) {
        const int i = e / PUW, c = e - i * PUW;
        const int sy = pad_index(g.oy0 - 6 + i, g.H, A.bc), sx = pad_index(g.ox0 - 6 + c, g.W, A.bc);
        float *dst = &S.U[i * PUC + c];
        if (sy < 0 || sx < 0) cp_async_zero(dst, uin, 4);
        else cp_async4(dst, uin + (size_t)sy * D.ld + sx);
    }
    cp_async_mbar_arrive(&S.bar[B_ULAND]);
    return 0;
}

// Symmetric padding of a TMA-staged region: the positions outside the image (zero-filled by the copy) take the value
// of their reflection, which lies inside the image and inside the box.  Rows outside cover all columns; columns
// outside cover the rows inside.  Producer threads; the caller synchronises before and after.
__device__ __forceinline__ void fill_ring(PairSmem &S, const Geo &g, int r, int p)
{
    const int y0 = g.oy0 - 6, x0 = g.ox0 - 6;
    const int rt = max(0, -y0), rb = max(0, y0 + PER - g.H), cl = max(0, -x0), cr = max(0, x0 + PUW - g.W);
    const int nrow = (rt + rb) * PUW, inner = PER - rt - rb, ncol = inner * (cl + cr);
    for (int e = p; e < nrow + ncol; e += NSTG) {
        int i, c;
        if (e < nrow) {
            const int k = e / PUW;
            c = e - k * PUW;
            i = k < rt ? k : PER - rb + (k - rt);
        } else {
            const int f = e - nrow, k = f / (cl + cr), m = f - k * (cl + cr);
            i = rt + k;
            c = m < cl ? m : PUW - cr + (m - cl);
        }
        const int si = pad_index(y0 + i, g.H, kSymmetric) - y0, sc = pad_index(x0 + c, g.W, kSymmetric) - x0;
        S.U[i * PUC + r + c] = S.U[si * PUC + r + sc];
    }
}

__device__ __forceinline__ bool region_outside(const Geo &g)
{
    return g.oy0 < 6 || g.ox0 < 6 || g.oy0 - 6 + PER > g.H || g.ox0 - 6 + PUW > g.W;
}

// Mean of 64 samples of the staged region (warp-collective; every lane gets it).
__device__ __forceinline__ float region_mean(const PairSmem &S, int r, int lane)
{
    float v = 0.0f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int si = lane + 32 * h;
        v += S.U[(2 + 9 * (si >> 3)) * PUC + r + 2 + 9 * (si & 7)];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v * (1.0f / 64.0f);
}

// One E item: 4 consecutive entries of one row (14 inputs, 7 bf16 pairs).
__device__ __forceinline__ void build_e_item(const PairSmem &S, uint4 *E, int r, float mean, int item)
{
    const int i = item >> 3, j0 = 4 * (item & 7);
    const float *src = &S.U[i * PUC + r + 2 * j0];
    uint32_t P[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) P[m] = pack_bf16x2(src[2 * m] - mean, src[2 * m + 1] - mean);
    uint4 *dst = &E[i * 32 + j0];
#pragma unroll
    for (int e = 0; e < 4; ++e) dst[e] = make_uint4(P[e], P[e + 1], P[e + 2], P[e + 3]);
}

// Output pass of a tile, producer thread p < 120: the pair of columns j = 1 + p % 30 of output row 4t - 3 + p / 30
// at step t.  The per-thread column geometry is fixed for the tile (OutCols); the operands (u, delta, d at both
// pixels) are loaded into registers two steps ahead (out_load); the update follows once the partial rows of the step
// are complete (out_finish).
struct OutCols {
    int j, r4, gx0;
    bool c0, c1;                         // columns 2j, 2j + 1 inside the tile's write range
    int mx0, mx1;                        // region columns of their reflections (padding fold), -1 if none
};

__device__ __forceinline__ OutCols out_cols(const Geo &g, int n)
{
    OutCols c;
    const int p = n;
    c.j = 1 + n % 30;
    c.r4 = n / 30;
    c.gx0 = g.ox0 + 2 * c.j - 3;
    const int X0 = 2 * c.j, gx1 = c.gx0 + 1;
    c.c0 = p < 120 && X0 >= 3 && c.gx0 >= g.xs && c.gx0 < g.xe;
    c.c1 = p < 120 && X0 + 1 <= PTX + 2 && gx1 >= g.xs && gx1 < g.xe;
    auto mirror = [&](int gx) {
        const int m = gx < 3 ? -1 - gx : (gx >= g.W - 3 ? 2 * g.W - 1 - gx : -1000);
        return m == -1000 ? -1 : m - g.ox0 + 3;
    };
    c.mx0 = mirror(c.gx0);
    c.mx1 = mirror(gx1);
    return c;
}

// output row of step t for this thread and whether it is written; gy its image row
__device__ __forceinline__ bool out_row(const Geo &g, const OutCols &c, int t, int &Y, int &gy)
{
    Y = 4 * t - 3 + c.r4;
    gy = g.oy0 + Y - 3;
    return Y >= 3 && Y <= PTY + 2 && gy >= g.ys && gy < g.ye;
}

// The image's planes and step constants, read once per tile from the launch parameters (the output pass would
// otherwise re-read them at every step).
struct OutImg {
    const float *u, *d;                  // u^n (this step's plane), data
    float *un, *dl, *out;                // u^{n+1} (the other plane), delta, gradient (kGrad)
    int ld, model;
    StepConsts sc;
};

__device__ __forceinline__ OutImg out_img(const PairArgs &A, int im)
{
    const ImgDesc &D = A.img[im];
    OutImg o;
    o.u = D.u_hi[A.parity];
    o.un = D.u_hi[A.parity ^ 1];
    o.d = D.d;
    o.dl = D.delta;
    o.out = D.out;
    o.ld = D.ld;
    o.model = D.model;
    o.sc = D.sc;
    return o;
}

// u, delta, d of the pair's two pixels at one step
struct OutVals {
    float u[2], dl[2], d[2];
};

// Loads through L2 (ld.global.cg): delta is rewritten in this launch, by the same thread and after this load.
template <int MODE>
__device__ __forceinline__ OutVals out_load(const OutImg &o, const Geo &g, const OutCols &c, int t)
{
    OutVals v = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
    int Y, gy;
    if (t < PNMT && out_row(g, c, t, Y, gy)) {
        const size_t i0 = (size_t)gy * o.ld + c.gx0;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (!(s ? c.c1 : c.c0)) continue;
            v.u[s] = __ldcg(o.u + i0 + s);
            v.d[s] = __ldcg(o.d + i0 + s);
            if (MODE == kStep) v.dl[s] = __ldcg(o.dl + i0 + s);
        }
    }
    return v;
}

// L2: the quadratic prox of the Anscombe L2 model, else the I-divergence prox (direct and Anscombe I-divergence
// models), fixed per tile so that the step carries no model branch.
template <int MODE, bool L2>
__device__ __forceinline__ void out_finish(const OutImg &o, const Geo &g, const OutCols &c, const OutVals &v,
                                           const uint4 (*Gb)[32], bool ring, int t)
{
    int Y, gy;
    if (!out_row(g, c, t, Y, gy) || !(c.c0 || c.c1)) return;
    const uint4 e = Gb[Y][c.j];
    const uint32_t ew[4] = {e.x, e.y, e.z, e.w};
    float gs0 = 0.0f, gs1 = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&ew[q]));
        gs0 += f.x;
        gs1 += f.y;
    }
    if (ring) {
        const int my = gy < 3 ? -1 - gy : (gy >= g.H - 3 ? 2 * g.H - 1 - gy : -1000);
        const int Ym = my == -1000 ? -1 : my - g.oy0 + 3;
        const int X0 = 2 * c.j;
        if (Ym >= 0) {
            gs0 += g_at(Gb, Ym, X0);
            gs1 += g_at(Gb, Ym, X0 + 1);
        }
        if (c.mx0 >= 0) gs0 += g_at(Gb, Y, c.mx0) + (Ym >= 0 ? g_at(Gb, Ym, c.mx0) : 0.0f);
        if (c.mx1 >= 0) gs1 += g_at(Gb, Y, c.mx1) + (Ym >= 0 ? g_at(Gb, Ym, c.mx1) : 0.0f);
    }
    const size_t i0 = (size_t)gy * o.ld + c.gx0;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        if (!(s ? c.c1 : c.c0)) continue;
        const float gv = s ? gs1 : gs0, uh = v.u[s], dd = v.d[s];
        if (MODE == kGrad) {
            o.out[i0 + s] = gv + data_grad(uh, dd, o.model, o.sc.lambda);
        } else {
            float nh, nd;
            ipiano_update_f32(gv, uh, v.dl[s], dd, L2 ? kAnsL2 : kDirect, o.sc, nh, nd);
            o.un[i0 + s] = nh;
            o.dl[i0 + s] = nd;
        }
    }
}

// The output pass of the tile in partial-sum buffer k & 1 by the output warps, item p < 120 of every step: each
// thread's operands are loaded two steps ahead, its row of a step is updated once the col2im of that M-tile is done.
// Returns false if the CTA gave up.
template <int MODE, bool L2>
__device__ __forceinline__ bool output_steps(const OutImg &o, PairSmem &S, const Geo &g, const OutCols &oc, bool ring,
                                             int k, volatile int *abort_flag, int *status)
{
    const int b = k & 1;
    OutVals v0 = out_load<MODE>(o, g, oc, 0), v1 = out_load<MODE>(o, g, oc, 1);
    for (int t = 0; t < PNMT; ++t) {
        const OutVals v2 = out_load<MODE>(o, g, oc, t + 2);
        if (!mbar_wait_warp(&S.bar[B_CDONE + PNMT * b + t], (k >> 1) & 1, abort_flag, status)) return false;
        out_finish<MODE, L2>(o, g, oc, v0, S.G[b], ring, t);
        v0 = v1;
        v1 = v2;
    }
    return true;
}

template <int MODE>
__device__ __forceinline__ bool output_tile(const PairArgs &A, PairSmem &S, int tile, int k, int p,
                                            volatile int *abort_flag, int *status)
{
    const Geo g = pair_geometry(S, A.nimg, tile);
    const bool ring = A.bc == kSymmetric && (g.ys < 3 || g.xs < 3 || g.ye > g.H - 3 || g.xe > g.W - 3);
    OutCols oc = out_cols(g, p < 120 ? p : 0);
    if (p >= 120) oc.c0 = oc.c1 = false;
    const OutImg o = out_img(A, g.im);
    const bool ok = (MODE == kStep && o.model == kAnsL2)
                        ? output_steps<MODE, true>(o, S, g, oc, ring, k, abort_flag, status)
                        : output_steps<MODE, false>(o, S, g, oc, ring, k, abort_flag, status);
    if (ok) mbar_arrive(&S.bar[B_GFREE + (k & 1)]);
    return ok;
}

template <int MODE>
__global__ void __launch_bounds__(NT, 1) k_foe_pair(const __grid_constant__ PairArgs A, int *status)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    PairSmem &S = *reinterpret_cast<PairSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = A.tile_prefix[A.nimg];
    if ((int)blockIdx.x >= ntiles) return;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (tid == 0) {
        for (int b = 0; b < NRST; ++b) {
            mbar_init(&S.bar[B_FWD + b], 1);
            mbar_init(&S.bar[B_RFREE + b], 32 * NEXP);
        }
        for (int b = 0; b < NPST; ++b) {
            mbar_init(&S.bar[B_PSI + b], 32 * NEXP);
            mbar_init(&S.bar[B_PFREE + b], 1);
        }
        for (int b = 0; b < NZST; ++b) {
            mbar_init(&S.bar[B_ADJ + b], 1);
            mbar_init(&S.bar[B_ZFREE + b], 128);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&S.bar[B_EREADY + b], NSTG);
            mbar_init(&S.bar[B_EFREE + b], 1);
            mbar_init(&S.bar[B_GFREE + b], NPROD);
            mbar_init(&S.bar[B_DRAIN + b], 1);
            for (int t = 0; t < PNMT; ++t) mbar_init(&S.bar[B_CDONE + PNMT * b + t], 128);
        }
        mbar_init(&S.bar[B_ULAND], NSTG);
        mbar_init(&S.bar[B_W], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid <= A.nimg) S.tprefix[tid] = A.tile_prefix[tid];
    if (tid < A.nimg) {
        S.timg[tid][0] = A.img[tid].tiles_x;
        S.timg[tid][1] = A.img[tid].H;
        S.timg[tid][2] = A.img[tid].W;
    }
    // from here on the previous step's results (the iterate, *status, the stopping words) are read
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (tid == 0) S.abort_flag = *(volatile int *)status;
    if (tid < A.nimg) S.live[tid] = !image_stopped(A.img[tid]);
    __syncthreads();
    if (S.abort_flag) return;  // an earlier launch gave up: do nothing (CTA-uniform)
    const int tile0 = pair_next_live(S, A.nimg, ntiles, blockIdx.x);
    if (tile0 >= ntiles) return;  // every tile of this CTA belongs to a stopped image (CTA-uniform)
    if (warp == FWDW) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        if (lane == 0) {
            mbar_arrive_expect_tx(&S.bar[B_W], kOpsBytes);
            bulk_g2s(S.Wf, A.ops, kOpsBytes, &S.bar[B_W]);
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_base;
    volatile int *abort_flag = &S.abort_flag;
    const int stride = gridDim.x;
    auto next = [&](int tile) { return pair_next_live(S, A.nimg, ntiles, tile); };

    if (warp < NEXP) {
        // ---------------- expert: R(g) -> Psi(g) ----------------
        // warp w: lanes of quarter q = w % 4, response columns kExpCols c .. + kExpCols - 1 (c = w / 4; columns 0-47 are
        // pixel 0 of the pair, 48-95 pixel 1, filters in the tensor-memory order), Psi words kExpCols / 2 c ..
        const int q = warp & 3, c = warp >> 2;
        const uint32_t lane_off = (uint32_t)(32 * q) << 16;
        int rs = 0, ps = 0;              // R stage g % NRST, Psi stage g % NPST
        uint32_t rph = 0, pph = 0;
        long long gm = 0;
        bool ok = true;
        for (int tile = tile0; ok && tile < ntiles; tile = next(tile + stride)) {
            const Geo g = pair_geometry(S, A.nimg, tile);
            const bool interior = g.oy0 >= 3 && g.ox0 >= 3 && g.oy0 + PTY + 3 <= g.H && g.ox0 + PTX + 3 <= g.W;
            const int gx0 = g.ox0 - 3 + 2 * lane;
            for (int t = 0; t < PNMT; ++t, ++gm) {
                if (!mbar_wait_warp(&S.bar[B_FWD + rs], rph, abort_flag, status)) {
                    ok = false;
                    break;
                }
                fence_after();
                // R columns kExpCols c .. in parts of kExpPart (two for a warp that converts all 96)
                uint32_t w[kExpCols / 2];
#pragma unroll
                for (int h = 0; h < kExpCols / kExpPart; ++h) {
                    const int col0 = kExpCols * c + kExpPart * h;
                    float r[kExpPart];
                    const uint32_t ra = tmem + lane_off + rs * kRCols + col0;
                    tmem_ld32(ra, r);
                    if constexpr (kExpPart == 48) tmem_ld16(ra + 32, r + 32);
                    tmem_wait_ld();
                    if (h == kExpCols / kExpPart - 1) {
                        // the R stage may take the forward MMAs of M-tile g + NRST now
                        fence_before();
                        mbar_arrive(&S.bar[B_RFREE + rs]);
                    }
#pragma unroll
                    for (int m = 0; m < kExpPart / 4; ++m) {
                        uint32_t &wa = w[kExpPart / 2 * h + 2 * m], &wb = w[kExpPart / 2 * h + 2 * m + 1];
                        if (kOneRcpPerQuad) psi_quad1(r[4 * m], r[4 * m + 1], r[4 * m + 2], r[4 * m + 3], wa, wb);
                        else psi_quad(r[4 * m], r[4 * m + 1], r[4 * m + 2], r[4 * m + 3], wa, wb);
                    }
                }
                if (!interior) {
                    const int gy = g.oy0 - 3 + 4 * t + q;
                    const bool row_in = gy >= 0 && gy < g.H;
                    const uint32_t k0 = (row_in && gx0 >= 0 && gx0 < g.W) ? 0xFFFFFFFFu : 0u;
                    const uint32_t k1 = (row_in && gx0 + 1 >= 0 && gx0 + 1 < g.W) ? 0xFFFFFFFFu : 0u;
                    // (most M-tiles of a border tile lie inside the image: then there is nothing to clear)
                    if (!__all_sync(0xffffffffu, (k0 & k1) != 0u))
#pragma unroll
                        for (int m = 0; m < kExpCols / 2; ++m) w[m] &= (kExpCols * c + 2 * m < 48) ? k0 : k1;
                }
                // the Psi stage is free once the adjoint MMAs of M-tile g - NPST (its previous reader) are complete
                if (gm >= NPST && !mbar_wait_warp(&S.bar[B_PFREE + ps], pph ^ 1u, abort_flag, status)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t pa = tmem + lane_off + kPsiCol0 + ps * kPsiCols + (kExpCols / 2) * c;
                if constexpr (kExpCols == 96) {
                    tmem_st32(pa, w);
                    tmem_st16(pa + 32, w + 32);
                } else {
                    tmem_st16(pa, w);
                    if constexpr (kExpCols == 48) tmem_st8(pa + 16, w + 16);
                }
                tmem_wait_st();
                fence_before();
                mbar_arrive(&S.bar[B_PSI + ps]);
                stage_advance<NRST>(rs, rph);
                stage_advance<NPST>(ps, pph);
            }
        }
    } else if (warp < FWDW) {
        // ---------------- col2im: Z2(g) -> partial rows of the tile's buffer, lanes of quarter q ----------------
        const int q = warp & 3;
        const uint32_t lane_off = (uint32_t)(32 * q) << 16;
        int stg = 0;                     // Z2 stage g % NZST
        uint32_t ph = 0;
        bool ok = true;
        int k = 0;
        for (int tile = tile0; ok && tile < ntiles; tile = next(tile + stride), ++k) {
            const Geo g = pair_geometry(S, A.nimg, tile);
            // the lanes at the warp's edges get no shuffled values from outside the region; their sums are used only
            // by the padding fold of a tile at the left or right image border, where the missing terms are zero
            const bool edge = A.bc == kSymmetric && (g.xs < 3 || g.xe > g.W - 3);
            const int b = k & 1;
            if (k >= 2 && !mbar_wait_warp(&S.bar[B_GFREE + b], ((k - 2) >> 1) & 1, abort_flag, status)) break;
            uint32_t *Gq = reinterpret_cast<uint32_t *>(&S.G[b][0][0]) + q;  // word q of entry (Y, pair)
            uint64_t c0 = 0, c1 = 0, c2 = 0;  // carried partial sums of output rows y + 1 .. y + 3 (f32 pairs)
            auto emit = [&](int Y, uint64_t v) {
                if (Y >= 0 && Y < PRY) {
                    float lo, hi;
                    f2_unpack(v, lo, hi);
                    Gq[4 * (Y * 32 + lane)] = pack_f16x2(lo, hi);
                }
            };
            // slots of tap row a: (c3, c4) own, (c1, c2) from pair j + 1, (c5, c6) from j - 1, c7 from j - 2, c0 from
            // j + 2: even output 2j = c3 + c1' + c5'' + c7''', odd 2j + 1 = c4 + c2' + c6'' + c0'''
            auto hrow = [&](const float *z8) {
                float d1a = __shfl_down_sync(0xffffffffu, z8[2], 1), d1b = __shfl_down_sync(0xffffffffu, z8[3], 1);
                float u1a = __shfl_up_sync(0xffffffffu, z8[4], 1), u1b = __shfl_up_sync(0xffffffffu, z8[5], 1);
                float u2 = __shfl_up_sync(0xffffffffu, z8[6], 2), d2 = __shfl_down_sync(0xffffffffu, z8[7], 2);
                if (edge) {
                    if (lane == 31) d1a = d1b = 0.0f;
                    if (lane == 0) u1a = u1b = 0.0f;
                    if (lane < 2) u2 = 0.0f;
                    if (lane > 29) d2 = 0.0f;
                }
                return f2_add(f2_add(f2_pack(z8[0], z8[1]), f2_pack(d1a, d1b)), f2_add(f2_pack(u1a, u1b), f2_pack(u2, d2)));
            };
            for (int t = 0; t < PNMT; ++t) {
                if (!mbar_wait_warp(&S.bar[B_ADJ + stg], ph, abort_flag, status)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t za = tmem + lane_off + kZCol0 + stg * kZCols;
                const int y = 4 * t + q;
                {
                    // tap rows 0-3: the output rows y - 3 .. y are final for this quarter
                    float z[32];
                    tmem_ld32(za, z);
                    tmem_wait_ld();
                    emit(y - 3, f2_add(c0, hrow(z)));
                    emit(y - 2, f2_add(c1, hrow(z + 8)));
                    emit(y - 1, f2_add(c2, hrow(z + 16)));
                    emit(y, hrow(z + 24));
                }
                {
                    // tap rows 4-6: carried to the quarter's next row, y + 4
                    float z[24];
                    tmem_ld16(za + 32, z);
                    tmem_ld8(za + 48, z + 16);
                    tmem_wait_ld();
                    fence_before();
                    mbar_arrive(&S.bar[B_ZFREE + stg]);
                    c0 = hrow(z);
                    c1 = hrow(z + 8);
                    c2 = hrow(z + 16);
                }
                if (t == PNMT - 1) {
                    emit(y + 1, c0);
                    emit(y + 2, c1);
                    emit(y + 3, c2);
                }
                mbar_arrive(&S.bar[B_CDONE + PNMT * b + t]);
                stage_advance<NZST>(stg, ph);
            }
        }
    } else if (warp == FWDW) {
        // ---------------- forward MMA issue (warp-uniform; one elected lane) ----------------
        constexpr uint32_t IDF = idesc_bf16(128, 96);
        const uint64_t dW = sdesc(smem_u32(S.Wf), 16 * 96, 128);
        bool ok = mbar_wait_warp(&S.bar[B_W], 0, abort_flag, status);
        int stg = 0;
        uint32_t ph = 0;
        int k = 0;
        long long g = 0;
        for (int tile = tile0; ok && tile < ntiles; tile = next(tile + stride), ++k) {
            const int b = k & 1;
            if (!mbar_wait_warp(&S.bar[B_EREADY + b], (k >> 1) & 1, abort_flag, status)) break;
            fence_after();
            const uint64_t dE = sdesc(smem_u32(S.E[b]), 32 * 16, 128);
            for (int t = 0; t < PNMT; ++t, ++g) {
                // R stage stg is free once every expert thread has loaded R(g - 3)
                if (g >= NRST && !mbar_wait_warp(&S.bar[B_RFREE + stg], ph ^ 1u, abort_flag, status)) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + stg * kRCols;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    mma_elect<false>(d, dE + (uint64_t)((4 * t + 2 * kk) * 32), dW + (uint64_t)(kk * 2 * 96), IDF, kk > 0);
                commit_elect(&S.bar[B_FWD + stg]);
                stage_advance<NRST>(stg, ph);
            }
            if (!ok) break;
            commit_elect(&S.bar[B_EFREE + b]);
        }
        if (!ok) mbar_wait_drain(&S.bar[B_W], 0, status);  // the operand copy lands before the CTA leaves
    } else if (warp == ADJW) {
        // ---------------- adjoint MMA issue ----------------
        constexpr uint32_t IDA = idesc_bf16(128, 64);
        const uint64_t dWa = sdesc(smem_u32(S.Wa), 16 * 64, 128);
        bool ok = mbar_wait_warp(&S.bar[B_W], 0, abort_flag, status);
        int ps = 0, zs = 0;
        uint32_t pph = 0, zph = 0;
        long long g = 0;
        for (int tile = tile0; ok && tile < ntiles; tile = next(tile + stride)) {
            for (int t = 0; t < PNMT; ++t, ++g) {
                if (!mbar_wait_warp(&S.bar[B_PSI + ps], pph, abort_flag, status) ||
                    (g >= NZST && !mbar_wait_warp(&S.bar[B_ZFREE + zs], zph ^ 1u, abort_flag, status))) {
                    ok = false;
                    break;
                }
                fence_after();
                const uint32_t d = tmem + kZCol0 + zs * kZCols, a0 = tmem + kPsiCol0 + ps * kPsiCols;
                // K-step kk: Psi words 8 kk .. 8 kk + 7 (pixel kk / 3, filters 16 (kk % 3) .. + 15)
#pragma unroll
                for (int kk = 0; kk < 6; ++kk)
                    mma_ta_elect<false>(d, a0 + 8 * kk, dWa + (uint64_t)(kk * 2 * 64), IDA, kk > 0);
                commit_elect(&S.bar[B_PFREE + ps]);
                // (a failure-detection test makes CTA 0 withhold this arrival once: the col2im warps' bounded wait
                // then expires and the launch reports FOE_ETIMEOUT)
                if (!(A.withhold_arrival && blockIdx.x == 0 && g == 0)) commit_elect(&S.bar[B_ADJ + zs]);
                stage_advance<NPST>(ps, pph);
                stage_advance<NZST>(zs, zph);
            }
        }
    } else if (warp < STGW0) {
        // ---------------- output pass of each tile ----------------
        bool ok = true;
        int k = 0;
        for (int tile = tile0; ok && tile < ntiles; tile = next(tile + stride), ++k)
            ok = output_tile<MODE>(A, S, tile, k, tid - 32 * OUTW0, abort_flag, status);
    } else {
        // ---------------- staging: input regions and E operands, one tile ahead ----------------
        const int p = tid - 32 * STGW0;
        int ucount = 0;                  // input regions staged so far (B_ULAND phases)
        bool ok = true, pending = false;
        int r_next = 0;                  // column offset of the staged region
        auto land = [&](const Geo &gr) {
            // wait for the staged region, then fill its reflected ring (symmetric padding, TMA-staged)
            bool w = mbar_wait(&S.bar[B_ULAND], ucount & 1, abort_flag, status);
            if (w) {
                ++ucount;
                pending = false;         // otherwise the copy may still be in flight: drained before the CTA leaves
            }
            if (!prod_all(w)) return false;
            if (A.bc == kSymmetric && gr.W >= PUC && gr.H >= PER && region_outside(gr)) {
                fill_ring(S, gr, r_next, p);
                prod_all(true);
            }
            return true;
        };
        // E of tile k into buffer k & 1, once its region has landed and the forward MMAs of tile k - 2 (the previous
        // user of the buffer) are complete; then the region of tile k + 1 is copied in
        auto build = [&](int tile, int k) {
            const int b = k & 1;
            if (!land(pair_geometry(S, A.nimg, tile))) return false;
            if (k >= 2 && !prod_all(mbar_wait(&S.bar[B_EFREE + b], ((k - 2) >> 1) & 1, abort_flag, status))) return false;
            const float mean = region_mean(S, r_next, lane);
            for (int item = p; item < kEItems; item += NSTG) build_e_item(S, S.E[b], r_next, mean, item);
            fence_async_smem();
            mbar_arrive(&S.bar[B_EREADY + b]);
            if (!prod_all(true)) return false;  // the region is consumed
            const int tn = next(tile + stride);
            if (tn < ntiles) {
                r_next = stage_region(A, S, pair_geometry(S, A.nimg, tn), p);
                pending = true;
            }
            return true;
        };
        r_next = stage_region(A, S, pair_geometry(S, A.nimg, tile0), p);
        pending = true;
        ok = build(tile0, 0);
        int k = 1;
        for (int tile = next(tile0 + stride); ok && tile < ntiles; tile = next(tile + stride), ++k) ok = build(tile, k);
        // a region copy still in flight (after a give-up) lands before the CTA exits
        if (pending) mbar_wait_drain(&S.bar[B_ULAND], ucount & 1, status);
        cp_async_wait<0>();
    }

    // every MMA issued by the two MMA warps is complete before tensor memory is released.  If this bounded wait
    // expired the launch has already recorded FOE_ETIMEOUT and its results are discarded; the columns are released
    // all the same: a CTA must free its tensor memory before it exits, and columns left allocated would hold every
    // later CTA of the SM in tcgen05.alloc
    if (warp == FWDW || warp == ADJW) {
        uint64_t *bar = &S.bar[B_DRAIN + (warp == FWDW ? 0 : 1)];
        commit_elect(bar);
        mbar_wait_drain(bar, 0, status);
    }
    fence_before();
    __syncthreads();
    if (warp == FWDW) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

constexpr size_t kPairSmem = sizeof(PairSmem);

// ---------------- host side ----------------

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

// Tensor maps of the image planes, cached by (address, H, W, ld): the planes of a solve are the same in all of its
// launches.
struct MapEntry {
    const void *p;
    int H, W, ld;
    CUtensorMap map;
};
thread_local std::vector<MapEntry> t_maps;

cudaError_t encode_map(const float *plane, int H, int W, int ld, CUtensorMap *out)
{
    // images smaller than the box always take the per-element copies (their map is never used)
    if (!plane || W < PUC || H < PER) {
        std::memset(out, 0, sizeof(*out));
        return cudaSuccess;
    }
    for (const MapEntry &e : t_maps)
        if (e.p == plane && e.H == H && e.W == W && e.ld == ld) {
            *out = e.map;
            return cudaSuccess;
        }
    if (!g_encode) return cudaErrorInitializationError;
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)PUC, (cuuint32_t)PER};
    const cuuint32_t estr[2] = {1, 1};
    MapEntry e{plane, H, W, ld, {}};
    const CUresult r = g_encode(&e.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(plane), dims, strides, box,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    if (t_maps.size() >= 512) t_maps.erase(t_maps.begin(), t_maps.begin() + 256);
    t_maps.push_back(e);
    *out = e.map;
    return cudaSuccess;
}

template <int MODE>
cudaError_t pair_launch_one(const PairArgs &a, int grid, int *d_status, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = kPairSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_foe_pair<MODE>, a, d_status);
}

thread_local PairArgs t_args;

}  // namespace

int pair_tile_w() { return PTX; }
int pair_tile_h() { return PTY; }
int pair_min_rows() { return kPairMinRows; }
long pair_min_pixels() { return 90000; }

cudaError_t pair_setup()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_foe_pair<kStep>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPairSmem)))
        return e;
    if ((e = cudaFuncSetAttribute(k_foe_pair<kGrad>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPairSmem)))
        return e;
    std::lock_guard<std::mutex> lock(g_encode_mu);
    if (!g_encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if ((e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q)))
            return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    return cudaSuccess;
}

cudaError_t pair_launch(const LaunchArgs &a, int mode, bool all, int sms, int *d_status, cudaStream_t s)
{
    PairArgs &p = t_args;
    p.nimg = 0;
    p.parity = a.parity;
    p.bc = a.bc;
    p.withhold_arrival = a.withhold_arrival;
    p.ops = a.pairops;
    p.tile_prefix[0] = 0;
    cudaError_t e;
    for (int i = 0; i < a.nimg; ++i) {
        const ImgDesc &d = a.img[i];
        if (!all && d.tile_h != PTY) continue;
        p.img[p.nimg] = d;
        p.tile_prefix[p.nimg + 1] = p.tile_prefix[p.nimg] + (a.tile_prefix[i + 1] - a.tile_prefix[i]);
        for (int par = 0; par < 2; ++par)
            if ((e = encode_map(d.u_hi[par], d.H, d.W, d.ld, &p.tmap[p.nimg][par])) != cudaSuccess) return e;
        p.nimg++;
    }
    const int tiles = p.tile_prefix[p.nimg];
    if (tiles <= 0) return cudaSuccess;
    const int grid = std::min(tiles, sms);
    return mode == kStep ? pair_launch_one<kStep>(p, grid, d_status, s) : pair_launch_one<kGrad>(p, grid, d_status, s);
}

}  // namespace foe
