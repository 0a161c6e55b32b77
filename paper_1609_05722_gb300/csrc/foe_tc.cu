// Tensor-core fused FoE tile kernel for sm_103a: tcgen05.mma (BF16 operands, kind::f16, or TF32 operands,
// kind::tf32; FP32 accumulators in tensor memory), one iPiano step (Eq. iPianoupdate) per launch.
//
// One CTA owns a 26x26 output tile.  The prior gradient sum_i alpha_i K_i^T rho'(K_i u) (Eq. FoEF)
// needs the responses on the tile plus a 3-pixel ring: a 32x32 response region, processed as 8
// M-tiles of 128 response pixels (4 rows of 32).
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
// Roles: warps 0-3 move data between tensor memory and registers (warp w reads TMEM lanes 32w..32w+31,
// i.e. response row 4t+w of M-tile t) and do the pointwise work; one thread of warp 4 issues the MMAs.
// R and Z are double-buffered in tensor memory and Psi in shared memory, so the forward MMA of M-tile
// t+1 and the adjoint MMA of tile t overlap the epilogue of tile t.  Every mbarrier wait is bounded:
// on expiry the CTA records FOE_ETIMEOUT in *status, drains its MMAs, frees its tensor memory and
// finishes without further waits.
//
// BF16 range: filters are zero-mean, so K(u - c) = K u for any constant c (the padded image of a
// constant is constant under symmetric padding; under zero padding the padded zeros are shifted by -c
// too).  The tile mean is subtracted before rounding u to BF16.
#include <cstdint>

#include "foe_common.cuh"
#include "foe_kernels.h"

namespace foe {

namespace {

constexpr int TO = 26;                 // output tile side
constexpr int RS = TO + 6;             // response region side = 32 = warp width
constexpr int NMT = RS / 4;            // M-tiles per CTA
constexpr int EROWS = RS + 7;          // input rows (7 tap rows + 1 zero-weight row)
constexpr int UR = RS + 7, UC = RS + 8;
constexpr int NEPI = 8;                // epilogue warps: two per TMEM lane quarter
constexpr int MMA_WARP = NEPI;         // one thread of this warp issues the MMAs
constexpr int NTHR = 32 * (NEPI + 1);
constexpr uint32_t TMEM_COLS = 256;
constexpr int NSTAGE = 4;              // TMEM stages of 64 columns: R (48 columns), then Z over it
constexpr int NPSI = 3;                // Psi buffers in shared memory
constexpr int LAG = 2;                 // the adjoint of M-tile g is issued, and its col2im done, 2 M-tiles later
constexpr long long kTimeoutCycles = 4000000000ll;  // about 2 s at 2 GHz
constexpr uint32_t kSuspendHintNs = 100000;           // a waiting thread may sleep up to 0.1 ms per try

// Operand images in shared memory.  BF16: 16-byte entries of 8 values.  TF32: 16-byte entries of 4 values,
// so every 8-value K-chunk of the BF16 layout becomes two chunks (E is split into E[0] = u(x..x+3) and
// E[1] = u(x+4..x+7); the descriptor's leading offset steps from one half to the other).
template <bool TF>
struct TcOps;
template <>
struct TcOps<false> {
    static constexpr int EB = 1, WF = 8 * 48, WA = 6 * 64, PSI = 6 * 128;
};
template <>
struct TcOps<true> {
    static constexpr int EB = 2, WF = 8 * 2 * 48, WA = 12 * 64, PSI = 12 * 128;
};

template <bool TF>
struct TcSmem {
    uint4 E[TcOps<TF>::EB][EROWS * RS];   // forward A operand: entry (row, x) holds u(row, x..x+7)
    uint4 Wf[TcOps<TF>::WF];               // forward B operand [tap row a][(chunk)][filter][tap cols]
    uint4 Wa[TcOps<TF>::WA];               // adjoint B operand [filter chunk][tap 8a+b][filters in chunk]
    uint4 Psi[NPSI][TcOps<TF>::PSI];       // adjoint A operand [buffer][filter chunk][pixel][filters in chunk]
    float Hs[7 * RS * RS];      // horizontal col2im partial sums [a][response row][col]
    float U[UR * UC];           // fp32 input region
    float O[3][TO * TO];        // output-pass operands, prefetched: u_lo, delta, d
    int srow[UR], scol[UR];     // source row / column of each input-region row / column (-1: zero)
    uint64_t bar[4 * NSTAGE + 1];
    uint32_t tmem_base;
    int abort_flag;
    float red[NTHR / 32];
};

constexpr int B_FWD = 0, B_PSI = NSTAGE, B_ADJ = 2 * NSTAGE, B_ZEMPTY = 3 * NSTAGE, B_DRAIN = 4 * NSTAGE;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendHintNs)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false if the CTA gave up.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, int *status)
{
    const long long t0 = clock64();
    for (uint32_t i = 0;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 31u) == 31u) {
            if (*abort_flag) return false;
            if (clock64() - t0 > kTimeoutCycles) {
                *abort_flag = 1;
                atomicExch(status, (int)5 /* FOE_ETIMEOUT */);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    // K-major, no swizzle: core matrices of 8 rows x 16 B; lbo = next core matrix along K,
    // sbo = next group of 8 rows; bits 46-47 = descriptor version 1.
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t M, uint32_t N)
{
    // D FP32 (bit 4), A BF16 (bits 7-9 = 1), B BF16 (bits 10-12 = 1), both K-major,
    // N >> 3 at bits 17-22, M >> 4 at bits 24-28.
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

__host__ __device__ constexpr uint32_t idesc_tf32(uint32_t M, uint32_t N)
{
    // D FP32 (bit 4), A TF32 (bits 7-9 = 2), B TF32 (bits 10-12 = 2), both K-major.
    return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t d;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(d) : "f"(x));
    return d;
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Sum of the horizontal partials at (qy, qx) of the response region over the 7 tap rows; rows and
// columns outside the region are outside the image whenever they are asked for, so they add 0.
template <bool TF>
__device__ __forceinline__ float hs_gather(const TcSmem<TF> &S, int qy, int qx)
{
    if (qx < 0 || qx >= RS) return 0.0f;
    float g = 0.0f;
#pragma unroll
    for (int a = 0; a < 7; ++a) {
        const int r = qy - a + 3;
        if (r >= 0 && r < RS) g += S.Hs[(a * RS + r) * RS + qx];
    }
    return g;
}

template <int MODE, bool TF>
__global__ void __launch_bounds__(NTHR, TF ? 1 : 2) k_foe_tc(const __grid_constant__ LaunchArgs A, int *status)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem<TF> &S = *reinterpret_cast<TcSmem<TF> *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x;
    const int im = tile_image(A, tile);
    const ImgDesc &D = A.img[im];
    const int lt = tile - A.tile_prefix[im];
    const int oy0 = (lt / D.tiles_x) * TO, ox0 = (lt % D.tiles_x) * TO;
    const int H = D.H, W = D.W, ld = D.ld;
    const float *uin = D.u_hi[A.parity];

    // an earlier launch that gave up leaves *status set: then do nothing (CTA-uniform decision)
    if (tid == 0) S.abort_flag = *(volatile int *)status;
    __syncthreads();
    if (S.abort_flag) return;
    __syncthreads();

    // ---- asynchronous staging: group 0 = input region + filter images, group 1 = output-pass operands ----
    constexpr int NWF = TcOps<TF>::WF, NWA = TcOps<TF>::WA;
    const uint4 *ops = reinterpret_cast<const uint4 *>(TF ? A.tcops32 : A.tcops);
    for (int j = tid; j < NWF + NWA; j += NTHR) cp_async16(j < NWF ? &S.Wf[j] : &S.Wa[j - NWF], ops + j);
    if (tid < UR) S.srow[tid] = pad_index(oy0 - 6 + tid, H, A.bc);
    else if (tid < 2 * UR) S.scol[tid - UR] = pad_index(ox0 - 6 + tid - UR, W, A.bc);
    __syncthreads();
    for (int j = tid; j < UR * UR; j += NTHR) {
        const int r = j / UR, c = j % UR;
        const int sy = S.srow[r], sx = S.scol[c];
        if (sy < 0 || sx < 0) S.U[r * UC + c] = 0.0f;
        else cp_async4(&S.U[r * UC + c], uin + (size_t)sy * ld + sx);
    }
    cp_async_commit();
    if (MODE == kStep) {
        for (int j = tid; j < TO * TO; j += NTHR) {
            const int gy = oy0 + j / TO, gx = ox0 + j % TO;
            if (gy >= H || gx >= W) continue;
            const size_t idx = (size_t)gy * ld + gx;
            if (D.u_lo) cp_async4(&S.O[0][j], D.u_lo + idx);
            else S.O[0][j] = 0.0f;
            cp_async4(&S.O[1][j], D.delta + idx);
            cp_async4(&S.O[2][j], D.d + idx);
        }
    } else {
        for (int j = tid; j < TO * TO; j += NTHR) {
            const int gy = oy0 + j / TO, gx = ox0 + j % TO;
            if (gy < H && gx < W) cp_async4(&S.O[2][j], D.d + (size_t)gy * ld + gx);
        }
    }
    cp_async_commit();

    if (tid == 0) {
        for (int b = 0; b < NSTAGE; ++b) {
            mbar_init(&S.bar[B_FWD + b], 1);
            mbar_init(&S.bar[B_PSI + b], 32 * NEPI);
            mbar_init(&S.bar[B_ADJ + b], 1);
            mbar_init(&S.bar[B_ZEMPTY + b], 32 * NEPI);
        }
        mbar_init(&S.bar[B_DRAIN], 1);
        S.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }

    // ---- tile mean (BF16 range), then E ----
    cp_async_wait<1>();
    __syncthreads();
    float lsum = 0.0f;
    for (int j = tid; j < UR * UR; j += NTHR) lsum += S.U[(j / UR) * UC + j % UR];
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) S.red[warp] = lsum;
    __syncthreads();
    float mean = 0.0f;
#pragma unroll
    for (int w = 0; w < NTHR / 32; ++w) mean += S.red[w];
    mean *= 1.0f / (float)(UR * UR);
    for (int j = tid; j < EROWS * RS; j += NTHR) {
        const int i = j / RS, x = j % RS;
        const float *src = &S.U[i * UC + x];
        if (TF) {
            S.E[0][j] = make_uint4(to_tf32(src[0] - mean), to_tf32(src[1] - mean), to_tf32(src[2] - mean),
                                   to_tf32(src[3] - mean));
            S.E[TcOps<TF>::EB - 1][j] = make_uint4(to_tf32(src[4] - mean), to_tf32(src[5] - mean),
                                                   to_tf32(src[6] - mean), to_tf32(src[7] - mean));
        } else {
            uint4 e;
            e.x = pack_bf16x2(src[0] - mean, src[1] - mean);
            e.y = pack_bf16x2(src[2] - mean, src[3] - mean);
            e.z = pack_bf16x2(src[4] - mean, src[5] - mean);
            e.w = pack_bf16x2(src[6] - mean, src[7] - mean);
            S.E[0][j] = e;
        }
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = S.tmem_base;
    volatile int *abort_flag = &S.abort_flag;

    if (warp == MMA_WARP) {
        if (lane == 0) {
            // ---------------- MMA issue ----------------
            constexpr uint32_t IDF = TF ? idesc_tf32(128, 48) : idesc_bf16(128, 48);
            constexpr uint32_t IDA = TF ? idesc_tf32(128, 64) : idesc_bf16(128, 64);
            const uint32_t e0 = smem_u32(S.E[0]), e1 = smem_u32(S.E[TcOps<TF>::EB - 1]);
            const uint32_t wf0 = smem_u32(S.Wf), wa0 = smem_u32(S.Wa);
            bool ok = true;
            // stage s = t % NSTAGE holds R(t) (columns 64 s .. 64 s + 47) until the epilogue has read it, then
            // the adjoint writes Z(t) over it (64 columns); the stage is free again once Z(t) has been read.
            auto adjoint = [&](int t) {
                const int s = t % NSTAGE, k = t / NSTAGE;
                if (!mbar_wait(&S.bar[B_PSI + s], k & 1, abort_flag, status)) return false;
                fence_after();
                const uint32_t ps = smem_u32(S.Psi[t % NPSI]);
                if (TF) {
                    // K = 48 filters in 6 steps of 8 (two 4-filter chunks each)
#pragma unroll
                    for (int kk = 0; kk < 6; ++kk)
                        mma_tf32(tmem + 64 * s, sdesc(ps + kk * 2 * 2048, 2048, 128),
                                 sdesc(wa0 + kk * 2 * 1024, 1024, 128), IDA, kk > 0);
                } else {
#pragma unroll
                    for (int kk = 0; kk < 3; ++kk)
                        mma_bf16(tmem + 64 * s, sdesc(ps + kk * 2 * 2048, 2048, 128),
                                 sdesc(wa0 + kk * 2 * 1024, 1024, 128), IDA, kk > 0);
                }
                mma_commit(&S.bar[B_ADJ + s]);
                return true;
            };
            for (int t = 0; t < NMT && ok; ++t) {
                const int s = t % NSTAGE, k = t / NSTAGE;
                if (t >= NSTAGE && !mbar_wait(&S.bar[B_ZEMPTY + s], (k - 1) & 1, abort_flag, status)) { ok = false; break; }
                fence_after();
                if (TF) {
                    // K-step a = one tap row (8 columns: E[0] holds columns 0-3, E[1] columns 4-7); row 7 has zero
                    // weights and is skipped
#pragma unroll
                    for (int kk = 0; kk < 7; ++kk)
                        mma_tf32(tmem + 64 * s, sdesc(e0 + (4 * t + kk) * RS * 16, e1 - e0, 128),
                                 sdesc(wf0 + kk * 2 * 768, 768, 128), IDF, kk > 0);
                } else {
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_bf16(tmem + 64 * s, sdesc(e0 + (4 * t + 2 * kk) * RS * 16, RS * 16, 128),
                                 sdesc(wf0 + kk * 2 * 768, 768, 128), IDF, kk > 0);
                }
                mma_commit(&S.bar[B_FWD + s]);
                if (t >= LAG && !adjoint(t - LAG)) ok = false;
            }
            for (int t = NMT - LAG; ok && t < NMT; ++t)
                if (!adjoint(t)) ok = false;
            // all MMAs issued by this thread are complete once the drain barrier flips
            mma_commit(&S.bar[B_DRAIN]);
            const long long t0 = clock64();
            while (!mbar_try_wait(&S.bar[B_DRAIN], 0))
                if (clock64() - t0 > kTimeoutCycles) {
                    atomicExch(status, 5);
                    break;
                }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue warps ----------------
        // warp q = warp % 4 reads TMEM lanes 32q..32q+31 (response row 4t+q of M-tile t); the two warps of a
        // lane quarter split the filters (half = 0: filters 0-23, 1: 24-47) and the tap rows (0: a 0-3, 1: a 4-6).
        const int q = warp & 3, half = warp >> 2;
        // interior tile: the whole response region lies in the image, so no response is masked and no
        // lane outside 3..28 is ever read (no padding fold)
        const bool interior = oy0 >= 3 && ox0 >= 3 && oy0 + RS - 3 <= H && ox0 + RS - 3 <= W;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        const int m = 32 * q + lane;
        auto col2im = [&](int t) {
            const int b = t % NSTAGE, k = t / NSTAGE;
            if (!mbar_wait(&S.bar[B_ADJ + b], k & 1, abort_flag, status)) return false;
            fence_after();
            float z[32];
            const uint32_t zc = tmem + lane_base + 64 * b + 32 * half;
            tmem_ld16(zc, z);
            tmem_ld16(zc + 16, z + 16);
            tmem_wait_ld();
            fence_before();
            mbar_arrive(&S.bar[B_ZEMPTY + b]);
            const int rr = 4 * t + q;
#pragma unroll
            for (int aa = 0; aa < 4; ++aa) {
                const int a = 4 * half + aa;
                if (a > 6) break;
                float h = z[8 * aa + 3];
                if (interior) {
#pragma unroll
                    for (int bb = 0; bb < 3; ++bb) h += __shfl_down_sync(0xffffffffu, z[8 * aa + bb], 3 - bb);
#pragma unroll
                    for (int bb = 4; bb < 7; ++bb) h += __shfl_up_sync(0xffffffffu, z[8 * aa + bb], bb - 3);
                } else {
#pragma unroll
                    for (int bb = 0; bb < 7; ++bb) {
                        if (bb == 3) continue;
                        const int src = lane + 3 - bb;
                        const float v = __shfl_sync(0xffffffffu, z[8 * aa + bb], src & 31);
                        h += (src >= 0 && src < 32) ? v : 0.0f;
                    }
                }
                S.Hs[(a * RS + rr) * RS + lane] = h;
            }
            return true;
        };
        bool ok = true;
        for (int t = 0; t < NMT; ++t) {
            const int b = t % NSTAGE, k = t / NSTAGE;
            if (!mbar_wait(&S.bar[B_FWD + b], k & 1, abort_flag, status)) { ok = false; break; }
            fence_after();
            float r[32];
            const uint32_t rc = tmem + lane_base + 64 * b + 24 * half;
            tmem_ld16(rc, r);
            tmem_ld16(rc + 16, r + 16);  // columns 16-31 of this half; only 16-23 are used
            tmem_wait_ld();
            fence_before();
            const int gy = oy0 - 3 + 4 * t + q, gx = ox0 - 3 + lane;
            const bool in = interior || (gy >= 0 && gy < H && gx >= 0 && gx < W);
            if (TF) {
                uint32_t w[24];
#pragma unroll
                for (int j = 0; j < 24; ++j) {
                    const float r0 = r[j];
                    w[j] = in ? to_tf32(r0 * rcp_approx(fmaf(r0, r0, 1.0f))) : 0u;
                }
                uint4 *dst = &S.Psi[t % NPSI][(6 * half) * 128 + m];
#pragma unroll
                for (int kc = 0; kc < 6; ++kc)
                    dst[kc * 128] = make_uint4(w[4 * kc], w[4 * kc + 1], w[4 * kc + 2], w[4 * kc + 3]);
            } else {
                uint32_t w[12];
#pragma unroll
                for (int j = 0; j < 12; ++j) {
                    const float r0 = r[2 * j], r1 = r[2 * j + 1];
                    const float p0 = r0 * rcp_approx(fmaf(r0, r0, 1.0f));
                    const float p1 = r1 * rcp_approx(fmaf(r1, r1, 1.0f));
                    w[j] = in ? pack_bf16x2(p0, p1) : 0u;
                }
                uint4 *dst = &S.Psi[t % NPSI][(3 * half) * 128 + m];
#pragma unroll
                for (int kc = 0; kc < 3; ++kc)
                    dst[kc * 128] = make_uint4(w[4 * kc], w[4 * kc + 1], w[4 * kc + 2], w[4 * kc + 3]);
            }
            fence_async_smem();
            mbar_arrive(&S.bar[B_PSI + b]);  // R(t) has been read and Psi(t) written: the adjoint may overwrite the stage
            if (t >= LAG && !col2im(t - LAG)) { ok = false; break; }
        }
        for (int t = NMT - LAG; ok && t < NMT; ++t)
            if (!col2im(t)) ok = false;
    }

    cp_async_wait<0>();
    fence_before();
    __syncthreads();

    // ---------------- output pass: vertical col2im, padding fold, iPiano step ----------------
    const bool ring = A.bc == kSymmetric && (oy0 < 3 || ox0 < 3 || oy0 + TO > H - 3 || ox0 + TO > W - 3);
    for (int j = tid; j < TO * TO; j += NTHR) {
        const int yo = 3 + j / TO, xo = 3 + j % TO;
        const int gy = oy0 + yo - 3, gx = ox0 + xo - 3;
        if (gy >= H || gx >= W) continue;
        float g = hs_gather(S, yo, xo);
        if (ring) {
            const int my = gy < 3 ? -1 - gy : (gy >= H - 3 ? 2 * H - 1 - gy : -1000);
            const int mx = gx < 3 ? -1 - gx : (gx >= W - 3 ? 2 * W - 1 - gx : -1000);
            if (my != -1000) g += hs_gather(S, my - oy0 + 3, xo);
            if (mx != -1000) g += hs_gather(S, yo, mx - ox0 + 3);
            if (my != -1000 && mx != -1000) g += hs_gather(S, my - oy0 + 3, mx - ox0 + 3);
        }
        const size_t idx = (size_t)gy * ld + gx;
        const float uh = S.U[(yo + 3) * UC + xo + 3];
        if (MODE == kGrad) {
            D.out[idx] = g + data_grad(uh, S.O[2][j], D.model, D.sc.lambda);
        } else {
            float nh, nl, nd;
            ipiano_update(g, uh, S.O[0][j], S.O[1][j], S.O[2][j], D.model, D.sc, nh, nl, nd);
            D.u_hi[A.parity ^ 1][idx] = nh;
            if (D.u_lo) D.u_lo[idx] = nl;
            D.delta[idx] = nd;
        }
    }

    if (warp == MMA_WARP) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

}  // namespace

int tc_tile_h() { return TO; }
int tc_tile_w() { return TO; }
size_t tc_smem_bytes() { return sizeof(TcSmem<false>); }

cudaError_t tc_setup()
{
    cudaError_t e;
    const int b16 = (int)sizeof(TcSmem<false>), t32 = (int)sizeof(TcSmem<true>);
    if ((e = cudaFuncSetAttribute(k_foe_tc<kStep, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b16))) return e;
    if ((e = cudaFuncSetAttribute(k_foe_tc<kGrad, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b16))) return e;
    if ((e = cudaFuncSetAttribute(k_foe_tc<kStep, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, t32))) return e;
    return cudaFuncSetAttribute(k_foe_tc<kGrad, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, t32);
}

cudaError_t tc_launch(const LaunchArgs &a, int mode, bool tf32, int *d_status, cudaStream_t s)
{
    const int tiles = a.tile_prefix[a.nimg];
    if (tiles <= 0) return cudaSuccess;
    if (mode != kStep && mode != kGrad) return cudaErrorNotSupported;
    if (tf32) {
        if (mode == kStep) k_foe_tc<kStep, true><<<tiles, NTHR, sizeof(TcSmem<true>), s>>>(a, d_status);
        else k_foe_tc<kGrad, true><<<tiles, NTHR, sizeof(TcSmem<true>), s>>>(a, d_status);
    } else {
        if (mode == kStep) k_foe_tc<kStep, false><<<tiles, NTHR, sizeof(TcSmem<false>), s>>>(a, d_status);
        else k_foe_tc<kGrad, false><<<tiles, NTHR, sizeof(TcSmem<false>), s>>>(a, d_status);
    }
    return cudaGetLastError();
}

}  // namespace foe
