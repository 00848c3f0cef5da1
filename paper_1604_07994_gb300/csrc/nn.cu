// Learned initial guess: a small 3D U-Net of 3x3x3 convolutions whose convolutions run as
// BF16 implicit GEMMs on the 5th-generation tensor cores.  One CTA of 128 threads owns 128
// output cells; for each of the 27 taps it gathers the shifted input rows (zero outside the
// grid) and the tap's weights into shared memory in the canonical K-major layout (8 x 16-byte
// core matrices, no swizzle), one elected thread issues tcgen05.mma (M = 128, N = C_out,
// K = 16 per instruction) into an FP32 accumulator in tensor memory, and tcgen05.commit
// signals an mbarrier; two shared-memory stages let the gather of tap t+1 overlap the MMAs of
// tap t.  The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes
// 32w..32w+31) and fuses bias, skip connection, ReLU and the BF16/FP32 store.  The weight
// gradient is a second tcgen05 GEMM, D[(tap, c_out)][c_in] = sum over cells of
// dz[cell - tap][c_out] x[cell][c_in], split over cells and reduced with FP32 atomics.  The
// input gradient is the forward kernel run on tap-flipped, channel-transposed weights.
//
// Layer structure, loss and optimiser are the ones of the network description in the
// header (include/sdx.h); the paper has no counterpart (the learned guess is an addition).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "sdx_internal.h"
#include "bodies.cuh"

namespace sdx {
namespace nn {

typedef __nv_bfloat16 bf16;

constexpr int CONV_M = 128;          // cells per CTA (MMA M)
constexpr int WG_K = 32;             // cells per K chunk of the weight-gradient GEMM
constexpr long long WAIT_LIMIT = 4000000000LL;  // clock cycles before an mbarrier wait gives up

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(dst_smem), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// Wait for the phase of the given parity to complete, at most WAIT_LIMIT cycles; on time-out
// record it in *err and return false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (clock64() - t0 > WAIT_LIMIT) {
            if (err) atomicExch(err, 1);
            return false;
        }
    }
    return true;
}
// After a wait gave up: wait once more, again bounded, for the last of the `issued` commits
// (alternating between the two barriers) so that no MMA issued by this block is still writing
// tensor memory when the block frees it.  Each buffer's previous commit had completed before the
// next one was issued, so the last commit's phase is the only one outstanding on its barrier,
// and it covers every earlier MMA.  The error flag was set by the wait that gave up.
__device__ __forceinline__ void drain_commits(uint64_t* bars, int issued) {
    if (issued > 0) {
        const int last = issued - 1;
        mbar_wait(smem_u32(&bars[last & 1]), (last >> 1) & 1, nullptr);
    }
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        :: "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(bar) : "memory");
}
// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, canonical K-major layout without swizzle: core matrices
// of 8 rows x 16 bytes stored as 128 contiguous bytes; lbo = byte distance between core
// matrices adjacent along K, sbo = between core matrices adjacent along M/N.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: BF16 A and B (both K-major), FP32 D, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Byte offset of element (row r, k) in a K-major no-swizzle tile whose rows hold K elements.
__host__ __device__ constexpr uint32_t kmajor_off(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
__host__ __device__ constexpr int tmem_cols(int n) { return n <= 32 ? 32 : (n <= 64 ? 64 : (n <= 128 ? 128 : 256)); }

__device__ __forceinline__ void tap_offset(int t, int& dx, int& dy, int& dz) {
    dx = t % 3 - 1;
    dy = (t / 3) % 3 - 1;
    dz = t / 9 - 1;
}

// ---------------------------------------------------------------- forward convolution
// y[v][co] = epilogue( sum_t sum_ci W[t][co][ci] x[v + off_t][ci] ): + bias[co], + skip[v][co],
// ReLU; written as BF16 (ybf) or FP32 (yf).
struct ConvArgs {
    int n;                 // cells per side
    const bf16* x;         // [n^3][CIN]
    const bf16* w;         // [27][COUT][CIN]
    const float* bias;     // [COUT] or nullptr
    const bf16* skip;      // [n^3][COUT] or nullptr
    int relu;
    bf16* ybf;             // [n^3][COUT] or nullptr
    float* yf;             // [n^3][COUT] or nullptr
    int* err;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(128) k_conv_fwd(ConvArgs a) {
    constexpr int A_BYTES = CONV_M * CIN * 2;
    constexpr int B_BYTES = COUT * CIN * 2;
    constexpr int KCH = CIN / 8;                 // 16-byte chunks per row
    constexpr int NCOL = tmem_cols(COUT);
    constexpr uint32_t IDESC = idesc_bf16(CONV_M, COUT);
    __shared__ __align__(1024) uint8_t sA[2][A_BYTES];
    __shared__ __align__(1024) uint8_t sB[2][B_BYTES];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int n = a.n;
    const long long V = (long long)n * n * n;
    const long long v0 = (long long)blockIdx.x * CONV_M;
    if (warp == 0) tmem_alloc(smem_u32(&tslot), NCOL);
    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        mbar_init_fence();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    bool ok = true;
    int issued = 0;  // commits issued (block-uniform)
    for (int t = 0; t < 27; ++t) {
        const int buf = t & 1;
        if (t >= 2) ok = mbar_wait(smem_u32(&bars[buf]), ((t >> 1) - 1) & 1, a.err);
        int dx, dy, dz;
        tap_offset(t, dx, dy, dz);
        // A: the 128 output cells' neighbours at this tap
        for (int idx = tid; idx < CONV_M * KCH; idx += 128) {
            const int r = idx % CONV_M, q = idx / CONV_M;
            const long long v = v0 + r;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (v < V) {
                const int i = (int)(v % n), j = (int)((v / n) % n), k = (int)(v / ((long long)n * n));
                const int ii = i + dx, jj = j + dy, kk = k + dz;
                if (ii >= 0 && jj >= 0 && kk >= 0 && ii < n && jj < n && kk < n) {
                    const long long nb = ii + (long long)n * (jj + (long long)n * kk);
                    val = *reinterpret_cast<const uint4*>(a.x + nb * CIN + q * 8);
                }
            }
            *reinterpret_cast<uint4*>(sA[buf] + kmajor_off(r, q * 8, CIN)) = val;
        }
        // B: this tap's weights, rows = output channels
        for (int idx = tid; idx < COUT * KCH; idx += 128) {
            const int r = idx % COUT, q = idx / COUT;
            const uint4 val = *reinterpret_cast<const uint4*>(a.w + ((long long)t * COUT + r) * CIN + q * 8);
            *reinterpret_cast<uint4*>(sB[buf] + kmajor_off(r, q * 8, CIN)) = val;
        }
        fence_async_smem();
        ok = __syncthreads_and(ok);  // a wait that gave up anywhere stops the whole block
        if (!ok) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA[buf]), b0 = smem_u32(sB[buf]);
#pragma unroll
            for (int s = 0; s < CIN / 16; ++s)
                mma_bf16(tmem, sdesc(a0 + s * 256, 128, CIN * 16), sdesc(b0 + s * 256, 128, CIN * 16), IDESC,
                         (t | s) != 0);
            mma_commit(smem_u32(&bars[buf]));
        }
        ++issued;
    }
    // the last commit (tap 26, buffer 0, its 14th use) covers every MMA issued before it
    if (ok) ok = mbar_wait(smem_u32(&bars[0]), 13 & 1, a.err);
    ok = __syncthreads_and(ok);
    if (!ok) drain_commits(bars, issued);
    tc_fence_after();
    if (ok) {
        const int r = warp * 32 + (tid & 31);
        const long long v = v0 + r;
#pragma unroll
        for (int g = 0; g < COUT / 16; ++g) {
            float acc[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + g * 16, acc);
            if (v < V) {
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    float val = acc[c];
                    if (a.bias) val += a.bias[g * 16 + c];
                    if (a.skip) val += __bfloat162float(a.skip[v * COUT + g * 16 + c]);
                    if (a.relu) val = fmaxf(val, 0.0f);
                    acc[c] = val;
                }
                if (a.yf) {
                    float4* dst = reinterpret_cast<float4*>(a.yf + v * COUT + g * 16);
#pragma unroll
                    for (int c = 0; c < 4; ++c) dst[c] = make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
                } else {
                    __align__(16) bf16 o[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16(acc[c]);
                    uint4* dst = reinterpret_cast<uint4*>(a.ybf + v * COUT + g * 16);
                    dst[0] = reinterpret_cast<const uint4*>(o)[0];
                    dst[1] = reinterpret_cast<const uint4*>(o)[1];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NCOL);
}

// ---------------------------------------------------------------- forward convolution, bricks
// The same convolution with the input staged once per CTA.  A CTA owns an output brick of
// BX x BY x ZB cells (x fastest).  Its input with a one-cell halo, (BX+2) x (BY+2) x (ZB+2) cells
// (zero outside the grid), is stored in shared memory as CIN/8 planes of 16-byte cell rows in
// x-fastest order, and all 27 taps' weights in the canonical K-major layout.  For output z-plane
// zz the MMA's A operand (M = 128 = BX x BY cells, K = 16 channels) is then a view of the brick:
// core matrix (group of 8 rows = one x-line of 8 cells, 16 bytes = 8 channels) at
// start + y * (BX+2) * 16 (SBO) and + plane (LBO), and a tap (dx, dy, dz) only moves the start
// address.  One elected thread issues 27 x ZB x CIN/16 MMAs into ZB accumulators in tensor
// memory and one commit; there is no gather and no barrier per tap.
constexpr int BR_X = 8, BR_Y = 16;

template <int CIN, int COUT, int ZB>
struct BrickShape {
    static constexpr int HX = BR_X + 2, HY = BR_Y + 2, HZ = ZB + 2;
    static constexpr int NQ = CIN / 8;
    static constexpr int PLANE = HZ * HY * HX * 16;   // bytes of one 8-channel plane
    static constexpr int BRICK = NQ * PLANE;
    static constexpr int WTAP = COUT * CIN * 2;       // bytes of one tap's weights
    static constexpr int SMEM = BRICK + 27 * WTAP;
    static constexpr int NCOL = tmem_cols(ZB * COUT);
};

template <int CIN, int COUT, int ZB>
__global__ void __launch_bounds__(128) k_conv_brick(ConvArgs a) {
    using S = BrickShape<CIN, COUT, ZB>;
    constexpr uint32_t IDESC = idesc_bf16(128, COUT);
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sBrick = smem;
    uint8_t* sW = smem + S::BRICK;
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int n = a.n;
    const int x0 = blockIdx.x * BR_X, y0 = blockIdx.y * BR_Y, z0 = blockIdx.z * ZB;
    if (warp == 0) tmem_alloc(smem_u32(&tslot), S::NCOL);
    if (tid == 0) {
        mbar_init(smem_u32(&bar), 1);
        mbar_init_fence();
    }
    // the brick with its halo: 16-byte chunk q fastest, then x, y, z (coalesced reads)
    for (int idx = tid; idx < S::NQ * S::HX * S::HY * S::HZ; idx += 128) {
        const int q = idx % S::NQ;
        int r = idx / S::NQ;
        const int hx = r % S::HX;
        r /= S::HX;
        const int hy = r % S::HY, hz = r / S::HY;
        const int i = x0 + hx - 1, j = y0 + hy - 1, k = z0 + hz - 1;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (i >= 0 && j >= 0 && k >= 0 && i < n && j < n && k < n)
            val = *reinterpret_cast<const uint4*>(a.x + (i + (long long)n * (j + (long long)n * k)) * CIN + q * 8);
        *reinterpret_cast<uint4*>(sBrick + q * S::PLANE + ((hz * S::HY + hy) * S::HX + hx) * 16) = val;
    }
    for (int idx = tid; idx < 27 * COUT * S::NQ; idx += 128) {
        const int q = idx % S::NQ;
        const int r = idx / S::NQ;
        const int co = r % COUT, t = r / COUT;
        const uint4 val = *reinterpret_cast<const uint4*>(a.w + ((long long)t * COUT + co) * CIN + q * 8);
        *reinterpret_cast<uint4*>(sW + t * S::WTAP + kmajor_off(co, q * 8, CIN)) = val;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    if (tid == 0) {
        const uint32_t b0 = smem_u32(sBrick), w0 = smem_u32(sW);
        for (int zz = 0; zz < ZB; ++zz) {
            for (int t = 0; t < 27; ++t) {
                int dx, dy, dz;
                tap_offset(t, dx, dy, dz);
                const uint32_t line = (uint32_t)(((zz + dz + 1) * S::HY + (dy + 1)) * S::HX + (dx + 1)) * 16;
#pragma unroll
                for (int s = 0; s < CIN / 16; ++s)
                    mma_bf16(tmem + zz * COUT, sdesc(b0 + 2 * s * S::PLANE + line, S::PLANE, S::HX * 16),
                             sdesc(w0 + t * S::WTAP + s * 256, 128, CIN * 16), IDESC, (t | s) != 0);
            }
        }
        mma_commit(smem_u32(&bar));
    }
    bool ok = mbar_wait(smem_u32(&bar), 0, a.err);
    ok = __syncthreads_and(ok);
    if (!ok) mbar_wait(smem_u32(&bar), 0, nullptr);  // bounded: the one commit before freeing TMEM
    tc_fence_after();
    if (ok) {
        const int m = warp * 32 + (tid & 31);
        const int i = x0 + (m & 7), j = y0 + (m >> 3);
        for (int zz = 0; zz < ZB; ++zz) {
            const int k = z0 + zz;
            const bool in = i < n && j < n && k < n;
            const long long v = i + (long long)n * (j + (long long)n * k);
#pragma unroll
            for (int g = 0; g < COUT / 16; ++g) {
                float acc[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + zz * COUT + g * 16, acc);
                if (!in) continue;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    float val = acc[c];
                    if (a.bias) val += a.bias[g * 16 + c];
                    if (a.skip) val += __bfloat162float(a.skip[v * COUT + g * 16 + c]);
                    if (a.relu) val = fmaxf(val, 0.0f);
                    acc[c] = val;
                }
                if (a.yf) {
                    float4* dst = reinterpret_cast<float4*>(a.yf + v * COUT + g * 16);
#pragma unroll
                    for (int c = 0; c < 4; ++c) dst[c] = make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
                } else {
                    __align__(16) bf16 o[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16(acc[c]);
                    uint4* dst = reinterpret_cast<uint4*>(a.ybf + v * COUT + g * 16);
                    dst[0] = reinterpret_cast<const uint4*>(o)[0];
                    dst[1] = reinterpret_cast<const uint4*>(o)[1];
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, S::NCOL);
}

// ---------------------------------------------------------------- weight gradient
// dW[t][co][ci] += sum_{cells w in this CTA's range} dz[w - off_t][co] x[w][ci]  (FP32 atomics).
// GEMM rows r = t * COUT + co (27 COUT rows, tile of 128 per blockIdx.x), N = CIN, K = cells.
struct WgradArgs {
    int n;
    const bf16* x;     // [n^3][CIN]  layer input
    const bf16* dz;    // [n^3][COUT] gradient at the layer's pre-activation
    float* dw;         // [27][COUT][CIN]
    long long cells_per_cta;
    int* err;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(128) k_conv_wgrad(WgradArgs a) {
    constexpr int A_BYTES = CONV_M * WG_K * 2;
    constexpr int B_BYTES = CIN * WG_K * 2;
    constexpr int NCOL = tmem_cols(CIN);
    constexpr uint32_t IDESC = idesc_bf16(CONV_M, CIN);
    constexpr int TAPS_PER_TILE = (CONV_M + COUT - 1) / COUT;
    __shared__ __align__(1024) uint8_t sA[2][A_BYTES];
    __shared__ __align__(1024) uint8_t sB[2][B_BYTES];
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int n = a.n;
    const long long V = (long long)n * n * n;
    const int row0 = blockIdx.x * CONV_M;          // first GEMM row of this tile
    const int t0 = row0 / COUT;                    // first tap of the tile
    const long long c_begin = (long long)blockIdx.y * a.cells_per_cta;
    const long long c_end = c_begin + a.cells_per_cta < V ? c_begin + a.cells_per_cta : V;
    if (c_begin >= V) return;
    const int nchunks = (int)((c_end - c_begin + WG_K - 1) / WG_K);
    if (warp == 0) tmem_alloc(smem_u32(&tslot), NCOL);
    if (tid == 0) {
        mbar_init(smem_u32(&bars[0]), 1);
        mbar_init(smem_u32(&bars[1]), 1);
        mbar_init_fence();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    bool ok = true;
    int issued = 0;  // commits issued (block-uniform)
    for (int ch = 0; ch < nchunks; ++ch) {
        const int buf = ch & 1;
        if (ch >= 2) ok = mbar_wait(smem_u32(&bars[buf]), ((ch >> 1) - 1) & 1, a.err);
        const long long w0 = c_begin + (long long)ch * WG_K;
        // A[r][k] = dz[w0 + k - off_t][co], r = (t - t0) * COUT + co; zero outside the grid,
        // past the range, or for rows beyond 27 * COUT
        for (int idx = tid; idx < TAPS_PER_TILE * WG_K * (COUT / 8); idx += 128) {
            const int kk = idx % WG_K;
            const int rest = idx / WG_K;
            const int q = rest % (COUT / 8);
            const int tl = rest / (COUT / 8);
            const int t = t0 + tl;
            const int rbase = tl * COUT + q * 8;
            if (rbase >= CONV_M) continue;
            const long long w = w0 + kk;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (t < 27 && w < c_end) {
                int dx, dy, dz;
                tap_offset(t, dx, dy, dz);
                const int i = (int)(w % n), j = (int)((w / n) % n), k = (int)(w / ((long long)n * n));
                const int ii = i - dx, jj = j - dy, kz = k - dz;
                if (ii >= 0 && jj >= 0 && kz >= 0 && ii < n && jj < n && kz < n) {
                    const long long src = ii + (long long)n * (jj + (long long)n * kz);
                    val = *reinterpret_cast<const uint4*>(a.dz + src * COUT + q * 8);
                }
            }
            const bf16* e = reinterpret_cast<const bf16*>(&val);
#pragma unroll
            for (int m = 0; m < 8; ++m)
                *reinterpret_cast<bf16*>(sA[buf] + kmajor_off(rbase + m, kk, WG_K)) = e[m];
        }
        // B[ci][k] = x[w0 + k][ci]
        for (int idx = tid; idx < WG_K * (CIN / 8); idx += 128) {
            const int kk = idx % WG_K, q = idx / WG_K;
            const long long w = w0 + kk;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (w < c_end) val = *reinterpret_cast<const uint4*>(a.x + w * CIN + q * 8);
            const bf16* e = reinterpret_cast<const bf16*>(&val);
#pragma unroll
            for (int m = 0; m < 8; ++m)
                *reinterpret_cast<bf16*>(sB[buf] + kmajor_off(q * 8 + m, kk, WG_K)) = e[m];
        }
        fence_async_smem();
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA[buf]), b0 = smem_u32(sB[buf]);
#pragma unroll
            for (int s = 0; s < WG_K / 16; ++s)
                mma_bf16(tmem, sdesc(a0 + s * 256, 128, WG_K * 16), sdesc(b0 + s * 256, 128, WG_K * 16), IDESC,
                         (ch | s) != 0);
            mma_commit(smem_u32(&bars[buf]));
        }
        ++issued;
    }
    if (ok) {
        const int last = nchunks - 1;
        ok = mbar_wait(smem_u32(&bars[last & 1]), (last >> 1) & 1, a.err);
    }
    ok = __syncthreads_and(ok);
    if (!ok) drain_commits(bars, issued);
    tc_fence_after();
    if (ok) {
        const int r = warp * 32 + (tid & 31);
        const int grow = row0 + r;
        const bool valid = grow < 27 * COUT && r < TAPS_PER_TILE * COUT;
#pragma unroll
        for (int g = 0; g < CIN / 16; ++g) {
            float acc[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + g * 16, acc);
            if (valid) {
#pragma unroll
                for (int c = 0; c < 16; ++c) atomicAdd(a.dw + (long long)grow * CIN + g * 16 + c, acc[c]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NCOL);
}

// ---------------------------------------------------------------- elementwise kernels
constexpr int ETPB = 256;
inline unsigned eblocks(long long count) { return (unsigned)((count + ETPB - 1) / ETPB); }

// mean over 2x2x2 blocks: [n^3][C] -> [(n/2)^3][C]
__global__ void k_pool(int n, int C, const bf16* __restrict__ x, bf16* __restrict__ y) {
    const int m = n / 2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)m * m * m * C) return;
    const int c = (int)(t % C);
    const long long v = t / C;
    const int i = (int)(v % m), j = (int)((v / m) % m), k = (int)(v / ((long long)m * m));
    float s = 0;
    for (int q = 0; q < 8; ++q) {
        const long long src = (2 * i + (q & 1)) + (long long)n * ((2 * j + ((q >> 1) & 1)) + (long long)n * (2 * k + (q >> 2)));
        s += __bfloat162float(x[src * C + c]);
    }
    y[t] = __float2bfloat16(s * 0.125f);
}

// nearest-neighbour upsampling: [m^3][C] -> [(2m)^3][C]
__global__ void k_up(int m, int C, const bf16* __restrict__ x, bf16* __restrict__ y) {
    const int n = 2 * m;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * n * n * C) return;
    const int c = (int)(t % C);
    const long long v = t / C;
    const int i = (int)(v % n), j = (int)((v / n) % n), k = (int)(v / ((long long)n * n));
    y[t] = x[((i >> 1) + (long long)m * ((j >> 1) + (long long)m * (k >> 1))) * C + c];
}

// dz = da * (a > 0) (relu = 0: dz = da); BF16 copy for the tensor cores, optional FP32 copy,
// bias gradient db[c] += sum_v dz[v][c].
__global__ void k_relu_back(long long V, int C, const float* __restrict__ da, const bf16* __restrict__ act,
                            int relu, bf16* __restrict__ dzb, float* __restrict__ dzf, float* __restrict__ db) {
    __shared__ float red[ETPB];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float g = 0;
    if (t < V * C) {
        g = da[t];
        if (relu && !(__bfloat162float(act[t]) > 0.0f)) g = 0.0f;
        dzb[t] = __float2bfloat16(g);
        if (dzf) dzf[t] = g;
    }
    // blocks of ETPB threads cover ETPB / C whole cells (C divides ETPB): sum per channel
    red[threadIdx.x] = g;
    __syncthreads();
    if (threadIdx.x < C) {
        float s = 0;
        for (int q = threadIdx.x; q < ETPB; q += C) s += red[q];
        atomicAdd(db + threadIdx.x, s);
    }
}

// da[v] = (sum of dp over the coarse parent, / 8) + skip[v]: adjoint of the pooling, plus the
// gradient arriving through a skip connection.  dp: [(n/2)^3][C], da/skip: [n^3][C].
__global__ void k_pool_back(int n, int C, const float* __restrict__ dp, const float* __restrict__ skip,
                            float* __restrict__ da) {
    const int m = n / 2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * n * n * C) return;
    const int c = (int)(t % C);
    const long long v = t / C;
    const int i = (int)(v % n), j = (int)((v / n) % n), k = (int)(v / ((long long)n * n));
    float g = 0.125f * dp[((i >> 1) + (long long)m * ((j >> 1) + (long long)m * (k >> 1))) * C + c];
    if (skip) g += skip[t];
    da[t] = g;
}

// adjoint of nearest upsampling: da[v] = sum over the 8 children of du.  du: [(2m)^3][C].
__global__ void k_up_back(int m, int C, const float* __restrict__ du, float* __restrict__ da) {
    const int n = 2 * m;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)m * m * m * C) return;
    const int c = (int)(t % C);
    const long long v = t / C;
    const int i = (int)(v % m), j = (int)((v / m) % m), k = (int)(v / ((long long)m * m));
    float s = 0;
    for (int q = 0; q < 8; ++q) {
        const long long src = (2 * i + (q & 1)) + (long long)n * ((2 * j + ((q >> 1) & 1)) + (long long)n * (2 * k + (q >> 2)));
        s += du[src * C + c];
    }
    da[t] = s;
}

// loss = sum_{v, c<4} (y - t)^2 / (4V) (accumulated into *loss), dy = 2 (y - t) / (4V), 0 for c >= 4
__global__ void k_loss(long long V, const float* __restrict__ y, const float* __restrict__ tgt,
                       float* __restrict__ dy, double* __restrict__ loss) {
    __shared__ double red[ETPB];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0;
    if (t < V * 16) {
        const int c = (int)(t % 16);
        float g = 0;
        if (c < 4) {
            const float d = y[t] - tgt[t];
            l = (double)d * d;
            g = 2.0f * d / (4.0f * (float)V);
        }
        dy[t] = g;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int s = ETPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / (4.0 * (double)V));
}

// Adam with bias correction; writes the FP32 master weights and their BF16 copy.
__global__ void k_adam(long long count, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                       float gscale) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const float gr = g[t] * gscale;
    const float mm = b1 * m[t] + (1.0f - b1) * gr;
    const float vv = b2 * v[t] + (1.0f - b2) * gr * gr;
    m[t] = mm;
    v[t] = vv;
    w[t] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// W'[t'][ci][co] = W[26 - t'][co][ci] (BF16): the input gradient of a convolution is the
// convolution of the output gradient with these weights.
__global__ void k_flip_weights(int cin, int cout, const float* __restrict__ w, bf16* __restrict__ wf) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 27LL * cin * cout) return;
    const int co = (int)(t % cout);
    const long long r = t / cout;
    const int ci = (int)(r % cin);
    const int tp = (int)(r / cin);
    wf[t] = __float2bfloat16(w[((long long)(26 - tp) * cout + co) * cin + ci]);
}

__global__ void k_to_bf16(long long count, const float* __restrict__ x, bf16* __restrict__ y) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) y[t] = __float2bfloat16(x[t]);
}

// ---------------------------------------------------------------- solver grid <-> network grid
// Network input from a level (padded cell ids, viscosity table) and the nodal forcing:
// [log10 mu, cell mean of f / fscale (3), 1, 0...] per cell.
__global__ void k_features(LevelView<double> L, const double* __restrict__ f, const double* __restrict__ fscale,
                           bf16* __restrict__ x) {
    const int n = L.n;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (long long)n * n * n) return;
    const int i = (int)(v % n), j = (int)((v / n) % n), k = (int)(v / ((long long)n * n));
    const double mu = L.mu[L.cid[(i + 1) + (long long)L.P * ((j + 1) + (long long)L.P * (k + 1))]];
    float o[16];
    o[0] = (float)log10(mu);
    const double inv = 1.0 / *fscale;
    for (int c = 0; c < 3; ++c) {
        double s = 0;
        for (int q = 0; q < 8; ++q)
            s += f[c * L.nn + (i + (q & 1)) + L.s1 * (j + ((q >> 1) & 1)) + L.s2 * (k + (q >> 2))];
        o[1 + c] = (float)(s * 0.125 * inv);
    }
    o[4] = 1.0f;
    for (int c = 5; c < 16; ++c) o[c] = 0.0f;
    for (int c = 0; c < 16; ++c) x[v * 16 + c] = __float2bfloat16(o[c]);
}

// Output channel c of the network is VEL_SCALE u_c / fscale (c < 3) or (p - mean p) / fscale
// (c = 3): velocities of the blob-forced problems are about 1/100 of the pressures, and the
// pressure without a traction face is defined up to a constant.
constexpr double VEL_SCALE = 100.0;

// Training target: cell means of the nodal solution, scaled as above, in channels 0..3.
__global__ void k_target(LevelView<double> L, const double* __restrict__ xs, double fscale,
                         const double* __restrict__ pmean, float* __restrict__ t) {
    const int n = L.n;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= (long long)n * n * n) return;
    const int i = (int)(v % n), j = (int)((v / n) % n), k = (int)(v / ((long long)n * n));
    for (int c = 0; c < 4; ++c) {
        double s = 0;
        for (int q = 0; q < 8; ++q)
            s += xs[c * L.nn + (i + (q & 1)) + L.s1 * (j + ((q >> 1) & 1)) + L.s2 * (k + (q >> 2))];
        s *= 0.125;
        t[v * 16 + c] = (float)(c < 3 ? VEL_SCALE * s / fscale : (s - *pmean) / fscale);
    }
    for (int c = 4; c < 16; ++c) t[v * 16 + c] = 0.0f;
}

// mean of count values -> *out (one block)
__global__ void k_mean(const double* __restrict__ x, long long count, double* __restrict__ out) {
    __shared__ double red[1024];
    double s = 0;
    for (long long t = threadIdx.x; t < count; t += blockDim.x) s += x[t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / (double)count;
}

// Initial guess on the nodes: mean of the prediction over the cells around the node, unscaled
// (velocity / VEL_SCALE, times fscale); constrained velocity components zero.
__global__ void k_to_nodes(LevelView<double> L, const float* __restrict__ y, const double* __restrict__ fscale,
                           double* __restrict__ x0) {
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (node >= L.nn) return;
    const int n = L.n;
    int i, j, k;
    node_ijk(node, L.n1, i, j, k);
    double acc[4] = {0, 0, 0, 0};
    int cnt = 0;
    for (int q = 0; q < 8; ++q) {
        const int ci = i - (q & 1), cj = j - ((q >> 1) & 1), ck = k - (q >> 2);
        if (ci < 0 || cj < 0 || ck < 0 || ci >= n || cj >= n || ck >= n) continue;
        const long long v = ci + (long long)n * (cj + (long long)n * ck);
        for (int c = 0; c < 4; ++c) acc[c] += y[v * 16 + c];
        ++cnt;
    }
    const uint16_t inf = L.info[node];
    for (int c = 0; c < 4; ++c) {
        double val = acc[c] / cnt * (*fscale) / (c < 3 ? VEL_SCALE : 1.0);
        if (c < 3 && (inf & (1u << c))) val = 0.0;
        x0[c * L.nn + node] = val;
    }
}

__global__ void k_negate(double* a) { *a = -*a; }

// alpha = <y, b> / <y, y> with y = b - r = K x (the residual-minimising multiple of x)
__global__ void k_line_alpha(const double* __restrict__ d, double* __restrict__ alpha) {
    *alpha = d[1] > 0 ? d[0] / d[1] : 0.0;
}

// max |f| over the three nodal forcing components (1 if zero) -> *out
__global__ void k_absmax(const double* __restrict__ f, long long count, double* __restrict__ out) {
    __shared__ double red[1024];
    double m = 0;
    for (long long t = threadIdx.x; t < count; t += blockDim.x) m = fmax(m, fabs(f[t]));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] > 0 ? red[0] : 1.0;
}

// ---------------------------------------------------------------- launchers
// Brick convolution of one shape: z-planes per brick chosen so that the brick, its halo and all
// 27 taps' weights fit in shared memory (at most 203 KB, for 64 -> 32).
template <int CIN, int COUT, int ZB>
static void launch_brick(const ConvArgs& a, cudaStream_t s) {
    using S = BrickShape<CIN, COUT, ZB>;
    static bool attr = false;
    if (!attr) {
        CK(cudaFuncSetAttribute(k_conv_brick<CIN, COUT, ZB>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM));
        attr = true;
    }
    const dim3 grid((a.n + BR_X - 1) / BR_X, (a.n + BR_Y - 1) / BR_Y, (a.n + ZB - 1) / ZB);
    k_conv_brick<CIN, COUT, ZB><<<grid, 128, S::SMEM, s>>>(a);
}

// SDX_CONV_GATHER=1 selects the per-tap gather kernel (k_conv_fwd) instead of the brick kernel
// (read at every launch, for comparisons).
static bool use_gather_conv() {
    const char* e = std::getenv("SDX_CONV_GATHER");
    return e && e[0] == '1';
}

static void launch_conv(int cin, int cout, const ConvArgs& a, cudaStream_t s) {
    const long long V = (long long)a.n * a.n * a.n;
    const unsigned grid = (unsigned)((V + CONV_M - 1) / CONV_M);
    count_launches(1);
    if (!use_gather_conv()) {
        if (cin == 16 && cout == 16) { launch_brick<16, 16, 4>(a, s); return; }
        if (cin == 16 && cout == 32) { launch_brick<16, 32, 4>(a, s); return; }
        if (cin == 32 && cout == 16) { launch_brick<32, 16, 4>(a, s); return; }
        if (cin == 32 && cout == 32) { launch_brick<32, 32, 4>(a, s); return; }
        if (cin == 32 && cout == 64) { launch_brick<32, 64, 2>(a, s); return; }
        if (cin == 64 && cout == 32) { launch_brick<64, 32, 2>(a, s); return; }
    }
#define SDX_CONV_CASE(I, O) \
    if (cin == I && cout == O) { k_conv_fwd<I, O><<<grid, 128, 0, s>>>(a); return; }
    SDX_CONV_CASE(16, 16) SDX_CONV_CASE(16, 32) SDX_CONV_CASE(32, 16) SDX_CONV_CASE(32, 32)
    SDX_CONV_CASE(32, 64) SDX_CONV_CASE(64, 32)
#undef SDX_CONV_CASE
    count_launches(-1);
    set_error("unsupported convolution shape " + std::to_string(cin) + " -> " + std::to_string(cout));
    throw Fail{SDX_EINVAL};
}

static int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    return sms;
}

static void launch_wgrad(int cin, int cout, int n, const bf16* x, const bf16* dz, float* dw, int* err, cudaStream_t s) {
    const long long V = (long long)n * n * n;
    const int mt = (27 * cout + CONV_M - 1) / CONV_M;
    // enough cell splits to fill the device about twice, at least 8 K chunks per CTA
    long long splits = std::max<long long>(1, (2LL * sm_count() + mt - 1) / mt);
    long long per = (V + splits - 1) / splits;
    per = std::max<long long>(per, 8LL * WG_K);
    per = (per + WG_K - 1) / WG_K * WG_K;
    splits = (V + per - 1) / per;
    WgradArgs a{n, x, dz, dw, per, err};
    dim3 grid(mt, (unsigned)splits);
    count_launches(1);
#define SDX_WG_CASE(I, O) \
    if (cin == I && cout == O) { k_conv_wgrad<I, O><<<grid, 128, 0, s>>>(a); return; }
    SDX_WG_CASE(16, 16) SDX_WG_CASE(16, 32) SDX_WG_CASE(32, 16) SDX_WG_CASE(32, 32)
    SDX_WG_CASE(32, 64) SDX_WG_CASE(64, 32)
#undef SDX_WG_CASE
    count_launches(-1);
    set_error("unsupported convolution shape");
    throw Fail{SDX_EINVAL};
}

// ---------------------------------------------------------------- the network
struct LayerDef {
    int cin, cout, level;
};
static const LayerDef LAYERS[10] = {{16, 16, 0}, {16, 16, 0}, {16, 32, 1}, {32, 32, 1}, {32, 64, 2},
                                    {64, 32, 1}, {32, 32, 1}, {32, 16, 0}, {16, 16, 0}, {16, 16, 0}};

static long long layer_w(int l) { return 27LL * LAYERS[l].cin * LAYERS[l].cout; }
static long long param_count() {
    long long s = 0;
    for (int l = 0; l < 10; ++l) s += layer_w(l) + LAYERS[l].cout;
    return s;
}

struct Net {
    long long np = 0;
    float* w = nullptr;        // FP32 master parameters (layer by layer: W then b)
    float* g = nullptr;        // gradients
    float* m = nullptr;        // Adam moments
    float* v = nullptr;
    bf16* wb = nullptr;        // BF16 weights (forward layout)
    bf16* wf = nullptr;        // BF16 flipped weights (input-gradient layout)
    std::vector<long long> off;   // parameter offset of each layer
    std::vector<long long> offb;  // offset in wb / wf
    long long step = 0;
    int* err = nullptr;
    double* lossd = nullptr;
    // activations for one grid size
    int n = 0;
    bf16 *a[10] = {}, *p1 = nullptr, *p2 = nullptr, *u1 = nullptr, *u2 = nullptr;
    float* y = nullptr;
    float *gy = nullptr, *gA = nullptr, *gB = nullptr, *gC = nullptr, *skip4 = nullptr, *skip2 = nullptr;
    bf16* dzb = nullptr;
    // solver <-> network scratch
    bf16* feat = nullptr;
    double* fscale = nullptr;
};

static void free_acts(Net& N) {
    void* p[] = {N.p1, N.p2, N.u1, N.u2, N.y, N.gy, N.gA, N.gB, N.gC, N.skip4, N.skip2, N.dzb, N.feat};
    for (void* q : p)
        if (q) cudaFree(q);
    for (bf16*& q : N.a) {
        if (q) cudaFree(q);
        q = nullptr;
    }
    N.p1 = N.p2 = N.u1 = N.u2 = N.dzb = N.feat = nullptr;
    N.y = N.gy = N.gA = N.gB = N.gC = N.skip4 = N.skip2 = nullptr;
    N.n = 0;
}

static void ensure_acts(Net& N, int n) {
    if (N.n == n) return;
    if (n < 4 || n % 4 != 0 || n > 1024) {
        set_error("the network needs a grid of n cells per side with n a multiple of 4 (4..1024)");
        throw Fail{SDX_EINVAL};
    }
    cudaDeviceSynchronize();
    free_acts(N);
    const long long V0 = (long long)n * n * n, V1 = V0 / 8, V2 = V1 / 8;
    const long long Vl[3] = {V0, V1, V2};
    for (int l = 0; l < 10; ++l) N.a[l] = dalloc<bf16>(Vl[LAYERS[l].level] * LAYERS[l].cout);
    N.p1 = dalloc<bf16>(V1 * 16);
    N.p2 = dalloc<bf16>(V2 * 32);
    N.u1 = dalloc<bf16>(V1 * 64);
    N.u2 = dalloc<bf16>(V0 * 32);
    N.y = dalloc<float>(V0 * 16);
    N.gy = dalloc<float>(V0 * 16);
    N.gA = dalloc<float>(V0 * 64);
    N.gB = dalloc<float>(V0 * 64);
    N.gC = dalloc<float>(V0 * 64);
    N.skip4 = dalloc<float>(V1 * 32);
    N.skip2 = dalloc<float>(V0 * 16);
    N.dzb = dalloc<bf16>(V0 * 64);
    N.feat = dalloc<bf16>(V0 * 16);
    N.n = n;
}

static void refresh_bf16(Net& N, cudaStream_t s) {
    for (int l = 0; l < 10; ++l) {
        const long long nw = layer_w(l);
        count_launches(2);
        k_to_bf16<<<eblocks(nw), ETPB, 0, s>>>(nw, N.w + N.off[l], N.wb + N.offb[l]);
        k_flip_weights<<<eblocks(nw), ETPB, 0, s>>>(LAYERS[l].cin, LAYERS[l].cout, N.w + N.off[l], N.wf + N.offb[l]);
    }
}

static Net* net_create(unsigned long long seed) {
    Net* N = new (std::nothrow) Net();
    if (!N) { set_error("host allocation failed"); throw Fail{SDX_ENOMEM}; }
    try {
        N->np = param_count();
        long long o = 0, ob = 0;
        for (int l = 0; l < 10; ++l) {
            N->off.push_back(o);
            N->offb.push_back(ob);
            o += layer_w(l) + LAYERS[l].cout;
            ob += layer_w(l);
        }
        N->w = dalloc<float>(N->np);
        N->g = dalloc<float>(N->np);
        N->m = dalloc<float>(N->np);
        N->v = dalloc<float>(N->np);
        N->wb = dalloc<bf16>(ob);
        N->wf = dalloc<bf16>(ob);
        N->err = dalloc<int>(1);
        N->lossd = dalloc<double>(1);
        N->fscale = dalloc<double>(1);
        CK(cudaMemset(N->err, 0, sizeof(int)));
        // He-normal initial weights, zero biases
        std::vector<float> h(N->np, 0.0f);
        std::mt19937_64 gen(seed);
        std::normal_distribution<double> nd(0.0, 1.0);
        for (int l = 0; l < 10; ++l) {
            const double sd = std::sqrt(2.0 / (27.0 * LAYERS[l].cin));
            for (long long q = 0; q < layer_w(l); ++q) h[N->off[l] + q] = (float)(nd(gen) * sd);
        }
        CK(cudaMemcpy(N->w, h.data(), sizeof(float) * N->np, cudaMemcpyHostToDevice));
        CK(cudaMemset(N->m, 0, sizeof(float) * N->np));
        CK(cudaMemset(N->v, 0, sizeof(float) * N->np));
        refresh_bf16(*N, 0);
        CK(cudaDeviceSynchronize());
    } catch (...) {
        free_acts(*N);
        void* p[] = {N->w, N->g, N->m, N->v, N->wb, N->wf, N->err, N->lossd, N->fscale};
        for (void* q : p)
            if (q) cudaFree(q);
        delete N;
        throw;
    }
    return N;
}

static void net_free(Net* N) {
    if (!N) return;
    cudaDeviceSynchronize();
    free_acts(*N);
    void* p[] = {N->w, N->g, N->m, N->v, N->wb, N->wf, N->err, N->lossd, N->fscale};
    for (void* q : p)
        if (q) cudaFree(q);
    delete N;
}

static void conv_layer(Net& N, int l, int n, const bf16* x, const bf16* skip, bool relu, bf16* ybf, float* yf,
                       cudaStream_t s) {
    ConvArgs a{n, x, N.wb + N.offb[l], N.w + N.off[l] + layer_w(l), skip, relu ? 1 : 0, ybf, yf, N.err};
    launch_conv(LAYERS[l].cin, LAYERS[l].cout, a, s);
}

// forward pass for input x [n^3][16] -> N.y [n^3][16] (FP32); activations kept for backward
static void forward(Net& N, int n, const bf16* x, cudaStream_t s) {
    const int n1 = n / 2, n2 = n / 4;
    const long long V1 = (long long)n1 * n1 * n1, V0 = (long long)n * n * n;
    conv_layer(N, 0, n, x, nullptr, true, N.a[0], nullptr, s);
    conv_layer(N, 1, n, N.a[0], nullptr, true, N.a[1], nullptr, s);
    count_launches(1);
    k_pool<<<eblocks(V1 * 16), ETPB, 0, s>>>(n, 16, N.a[1], N.p1);
    conv_layer(N, 2, n1, N.p1, nullptr, true, N.a[2], nullptr, s);
    conv_layer(N, 3, n1, N.a[2], nullptr, true, N.a[3], nullptr, s);
    count_launches(1);
    k_pool<<<eblocks((long long)n2 * n2 * n2 * 32), ETPB, 0, s>>>(n1, 32, N.a[3], N.p2);
    conv_layer(N, 4, n2, N.p2, nullptr, true, N.a[4], nullptr, s);
    count_launches(1);
    k_up<<<eblocks(V1 * 64), ETPB, 0, s>>>(n2, 64, N.a[4], N.u1);
    conv_layer(N, 5, n1, N.u1, N.a[3], true, N.a[5], nullptr, s);
    conv_layer(N, 6, n1, N.a[5], nullptr, true, N.a[6], nullptr, s);
    count_launches(1);
    k_up<<<eblocks(V0 * 32), ETPB, 0, s>>>(n1, 32, N.a[6], N.u2);
    conv_layer(N, 7, n, N.u2, N.a[1], true, N.a[7], nullptr, s);
    conv_layer(N, 8, n, N.a[7], nullptr, true, N.a[8], nullptr, s);
    conv_layer(N, 9, n, N.a[8], nullptr, false, nullptr, N.y, s);
}

// Backward of one layer: dz = da * relu'(act) (into N.dzb, optionally FP32 copy dzf), bias
// and weight gradients, and (if dx) the input gradient dx = conv(dz, flipped W).
static void backward_layer(Net& N, int l, int n, const float* da, const bf16* act, bool relu, const bf16* inp,
                           float* dzf, float* dx, cudaStream_t s) {
    const long long V = (long long)n * n * n;
    const int cin = LAYERS[l].cin, cout = LAYERS[l].cout;
    count_launches(1);
    k_relu_back<<<eblocks(V * cout), ETPB, 0, s>>>(V, cout, da, act, relu ? 1 : 0, N.dzb, dzf,
                                                  N.g + N.off[l] + layer_w(l));
    launch_wgrad(cin, cout, n, inp, N.dzb, N.g + N.off[l], N.err, s);
    if (dx) {
        ConvArgs a{n, N.dzb, N.wf + N.offb[l], nullptr, nullptr, 0, nullptr, dx, N.err};
        launch_conv(cout, cin, a, s);
    }
}

// gradients of the loss into N.g (zeroed first); forward must have run on x
static void backward(Net& N, int n, const bf16* x, cudaStream_t s) {
    const int n1 = n / 2, n2 = n / 4;
    const long long V0 = (long long)n * n * n, V1 = V0 / 8, V2 = V1 / 8;
    // L10 (linear head): dy in N.gy
    backward_layer(N, 9, n, N.gy, nullptr, false, N.a[8], nullptr, N.gA, s);                 // gA = da9
    backward_layer(N, 8, n, N.gA, N.a[8], true, N.a[7], nullptr, N.gB, s);                    // gB = da8
    backward_layer(N, 7, n, N.gB, N.a[7], true, N.u2, N.skip2, N.gA, s);                      // gA = du2, skip2 = dz8
    count_launches(1);
    k_up_back<<<eblocks(V1 * 32), ETPB, 0, s>>>(n1, 32, N.gA, N.gB);                           // gB = da7
    backward_layer(N, 6, n1, N.gB, N.a[6], true, N.a[5], nullptr, N.gA, s);                   // gA = da6
    backward_layer(N, 5, n1, N.gA, N.a[5], true, N.u1, N.skip4, N.gB, s);                     // gB = du1, skip4 = dz6
    count_launches(1);
    k_up_back<<<eblocks(V2 * 64), ETPB, 0, s>>>(n2, 64, N.gB, N.gA);                           // gA = da5
    backward_layer(N, 4, n2, N.gA, N.a[4], true, N.p2, nullptr, N.gB, s);                     // gB = dp2
    count_launches(1);
    k_pool_back<<<eblocks(V1 * 32), ETPB, 0, s>>>(n1, 32, N.gB, N.skip4, N.gA);                // gA = da4
    backward_layer(N, 3, n1, N.gA, N.a[3], true, N.a[2], nullptr, N.gB, s);                   // gB = da3
    backward_layer(N, 2, n1, N.gB, N.a[2], true, N.p1, nullptr, N.gA, s);                     // gA = dp1
    count_launches(1);
    k_pool_back<<<eblocks(V0 * 16), ETPB, 0, s>>>(n, 16, N.gA, N.skip2, N.gB);                 // gB = da2
    backward_layer(N, 1, n, N.gB, N.a[1], true, N.a[0], nullptr, N.gA, s);                    // gA = da1
    backward_layer(N, 0, n, N.gA, N.a[0], true, x, nullptr, nullptr, s);
}

// forward + backward of one sample; the loss is added to *N.lossd (reset by the caller)
static void loss_grad(Net& N, int n, const bf16* x, const float* tgt, cudaStream_t s) {
    ensure_acts(N, n);
    const long long V = (long long)n * n * n;
    forward(N, n, x, s);
    count_launches(1);
    k_loss<<<eblocks(V * 16), ETPB, 0, s>>>(V, N.y, tgt, N.gy, N.lossd);
    backward(N, n, x, s);
}

static void check_err(Net& N, cudaStream_t s) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, N.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (e) {
        CK(cudaMemsetAsync(N.err, 0, sizeof(int), s));
        set_error("a tensor-core wait timed out in a network kernel");
        throw Fail{SDX_ETIMEOUT};
    }
}

}  // namespace nn
}  // namespace sdx

// ===================================================================== C ABI
using namespace sdx;
using namespace sdx::nn;

static Net* as_net(sdx_net_t p) { return reinterpret_cast<Net*>(p); }

extern "C" {

int64_t sdx_net_param_count(void) { return param_count(); }

int sdx_net_create(uint64_t seed, sdx_net_t* out) {
    if (!out) { set_error("null output pointer"); return SDX_EINVAL; }
    *out = nullptr;
    API_BEGIN
    *out = reinterpret_cast<sdx_net_t>(net_create(seed));
    return SDX_OK;
    API_END
}

int sdx_net_destroy(sdx_net_t net) {
    net_free(as_net(net));
    return SDX_OK;
}

int sdx_net_get_params(sdx_net_t net, float* host) {
    Net* N = as_net(net);
    if (!N || !host) { set_error("null argument"); return SDX_EINVAL; }
    API_BEGIN
    CK(cudaMemcpy(host, N->w, sizeof(float) * N->np, cudaMemcpyDeviceToHost));
    return SDX_OK;
    API_END
}

int sdx_net_set_params(sdx_net_t net, const float* host) {
    Net* N = as_net(net);
    if (!N || !host) { set_error("null argument"); return SDX_EINVAL; }
    API_BEGIN
    CK(cudaMemcpy(N->w, host, sizeof(float) * N->np, cudaMemcpyHostToDevice));
    CK(cudaMemset(N->m, 0, sizeof(float) * N->np));
    CK(cudaMemset(N->v, 0, sizeof(float) * N->np));
    N->step = 0;
    refresh_bf16(*N, 0);
    CK(cudaDeviceSynchronize());
    return launched("sdx_net_set_params");
    API_END
}

int sdx_net_forward(sdx_net_t net, int n, const uint16_t* x, float* y, void* stream) {
    Net* N = as_net(net);
    if (!N || !x || !y) { set_error("null argument"); return SDX_EINVAL; }
    API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    ensure_acts(*N, n);
    forward(*N, n, reinterpret_cast<const bf16*>(x), s);
    CK(cudaMemcpyAsync(y, N->y, sizeof(float) * 16 * (size_t)n * n * n, cudaMemcpyDeviceToDevice, s));
    check_err(*N, s);
    return launched("sdx_net_forward");
    API_END
}

int sdx_net_loss_grad(sdx_net_t net, int n, const uint16_t* x, const float* target, double* loss, float* grads,
                      void* stream) {
    Net* N = as_net(net);
    if (!N || !x || !target) { set_error("null argument"); return SDX_EINVAL; }
    API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemsetAsync(N->g, 0, sizeof(float) * N->np, s));
    CK(cudaMemsetAsync(N->lossd, 0, sizeof(double), s));
    loss_grad(*N, n, reinterpret_cast<const bf16*>(x), target, s);
    if (loss) CK(cudaMemcpyAsync(loss, N->lossd, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (grads) CK(cudaMemcpyAsync(grads, N->g, sizeof(float) * N->np, cudaMemcpyDeviceToHost, s));
    check_err(*N, s);
    return launched("sdx_net_loss_grad");
    API_END
}

int sdx_net_train(sdx_net_t net, int n, int count, const uint16_t* x, const float* target, int epochs, int batch,
                  float lr, uint64_t seed, double* loss_history, void* stream) {
    Net* N = as_net(net);
    if (!N || !x || !target || count < 1 || epochs < 1 || batch < 1 || !(lr > 0)) {
        set_error("invalid training arguments");
        return SDX_EINVAL;
    }
    API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    ensure_acts(*N, n);
    const long long V = (long long)n * n * n;
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::mt19937_64 gen(seed);
    std::vector<double> hist;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(order.begin(), order.end(), gen);
        CK(cudaMemsetAsync(N->lossd, 0, sizeof(double), s));
        for (int b0 = 0; b0 < count; b0 += batch) {
            const int nb = std::min(batch, count - b0);
            CK(cudaMemsetAsync(N->g, 0, sizeof(float) * N->np, s));
            for (int q = 0; q < nb; ++q) {
                const int smp = order[b0 + q];
                loss_grad(*N, n, reinterpret_cast<const bf16*>(x) + (long long)smp * V * 16, target + (long long)smp * V * 16, s);
            }
            N->step++;
            const float c1 = 1.0f - std::pow(0.9f, (float)N->step), c2 = 1.0f - std::pow(0.999f, (float)N->step);
            count_launches(1);
            k_adam<<<eblocks(N->np), ETPB, 0, s>>>(N->np, N->w, N->g, N->m, N->v, lr, 0.9f, 0.999f, 1e-8f, c1, c2,
                                                  1.0f / nb);
            refresh_bf16(*N, s);
        }
        double ep_loss = 0;
        CK(cudaMemcpyAsync(&ep_loss, N->lossd, sizeof(double), cudaMemcpyDeviceToHost, s));
        check_err(*N, s);  // synchronises the stream
        hist.push_back(ep_loss / count);
    }
    if (loss_history)
        for (int ep = 0; ep < epochs; ++ep) loss_history[ep] = hist[ep];
    return launched("sdx_net_train");
    API_END
}

int sdx_conv3(int n, int cin, int cout, const uint16_t* x, const uint16_t* w, const float* bias, int relu, float* y,
              void* stream) {
    if (n < 1 || !x || !w || !y) { set_error("invalid convolution arguments"); return SDX_EINVAL; }
    API_BEGIN
    DevTmp<int> err(1);
    CK(cudaMemset(err.p, 0, sizeof(int)));
    ConvArgs a{n, reinterpret_cast<const bf16*>(x), reinterpret_cast<const bf16*>(w), bias, nullptr, relu, nullptr, y, err.p};
    launch_conv(cin, cout, a, (cudaStream_t)stream);
    int e = 0;
    CK(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    err.reset();
    if (e) { set_error("tensor-core wait timed out"); return SDX_ETIMEOUT; }
    return launched("sdx_conv3");
    API_END
}

int sdx_conv3_dgrad(int n, int cin, int cout, const uint16_t* dz, const float* w, float* dx, void* stream) {
    if (n < 1 || !dz || !w || !dx) { set_error("invalid convolution arguments"); return SDX_EINVAL; }
    API_BEGIN
    const long long nw = 27LL * cin * cout;
    DevTmp<int> err(1);
    DevTmp<bf16> wf(nw);
    CK(cudaMemsetAsync(err.p, 0, sizeof(int), (cudaStream_t)stream));
    // the network's backward path: weights flipped in the taps and transposed in the channels,
    // then the forward kernel from the output-gradient channels to the input ones
    count_launches(1);
    k_flip_weights<<<eblocks(nw), ETPB, 0, (cudaStream_t)stream>>>(cin, cout, w, wf.p);
    ConvArgs a{n, reinterpret_cast<const bf16*>(dz), wf.p, nullptr, nullptr, 0, nullptr, dx, err.p};
    launch_conv(cout, cin, a, (cudaStream_t)stream);
    int e = 0;
    CK(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    err.reset();
    wf.reset();
    if (e) { set_error("tensor-core wait timed out"); return SDX_ETIMEOUT; }
    return launched("sdx_conv3_dgrad");
    API_END
}

int sdx_conv3_wgrad(int n, int cin, int cout, const uint16_t* x, const uint16_t* dz, float* dw, void* stream) {
    if (n < 1 || !x || !dz || !dw) { set_error("invalid convolution arguments"); return SDX_EINVAL; }
    API_BEGIN
    DevTmp<int> err(1);
    CK(cudaMemset(err.p, 0, sizeof(int)));
    launch_wgrad(cin, cout, n, reinterpret_cast<const bf16*>(x), reinterpret_cast<const bf16*>(dz), dw, err.p,
                 (cudaStream_t)stream);
    int e = 0;
    CK(cudaMemcpyAsync(&e, err.p, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    err.reset();
    if (e) { set_error("tensor-core wait timed out"); return SDX_ETIMEOUT; }
    return launched("sdx_conv3_wgrad");
    API_END
}

int sdx_guess_features(sdx_hier_t h, const double* f, uint16_t* x, double* fscale, void* stream) {
    Hier* H = reinterpret_cast<Hier*>(h);
    if (!H || !f || !x) { set_error("null argument"); return SDX_EINVAL; }
    API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    const LevelView<double> L = view<double>(*H, 0);
    DevTmp<double> sc(1);
    count_launches(2);
    k_absmax<<<1, 1024, 0, s>>>(f, 3 * L.nn, sc.p);
    k_features<<<eblocks((long long)L.n * L.n * L.n), ETPB, 0, s>>>(L, f, sc.p, reinterpret_cast<bf16*>(x));
    double hs = 1.0;
    CK(cudaMemcpyAsync(&hs, sc.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    sc.reset();
    if (fscale) *fscale = hs;
    return launched("sdx_guess_features");
    API_END
}

int sdx_guess_target(sdx_hier_t h, const double* xs, double fscale, float* t, void* stream) {
    Hier* H = reinterpret_cast<Hier*>(h);
    if (!H || !xs || !t || !(fscale > 0)) { set_error("invalid argument"); return SDX_EINVAL; }
    API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    const LevelView<double> L = view<double>(*H, 0);
    DevTmp<double> pm(1);
    count_launches(2);
    k_mean<<<1, 1024, 0, s>>>(xs + 3 * L.nn, L.nn, pm.p);
    k_target<<<eblocks((long long)L.n * L.n * L.n), ETPB, 0, s>>>(L, xs, fscale, pm.p, t);
    const int rc = launched("sdx_guess_target");
    CK(cudaStreamSynchronize(s));
    pm.reset();
    return rc;
    API_END
}

int sdx_guess_predict(sdx_hier_t h, sdx_net_t net, const double* f, double* x0, void* stream) {
    Hier* H = reinterpret_cast<Hier*>(h);
    Net* N = as_net(net);
    if (!H || !N || !f || !x0) { set_error("null argument"); return SDX_EINVAL; }
    API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    const LevelView<double> L = view<double>(*H, 0);
    ensure_acts(*N, L.n);
    count_launches(2);
    k_absmax<<<1, 1024, 0, s>>>(f, 3 * L.nn, N->fscale);
    k_features<<<eblocks((long long)L.n * L.n * L.n), ETPB, 0, s>>>(L, f, N->fscale, N->feat);
    forward(*N, L.n, N->feat, s);
    count_launches(1);
    k_to_nodes<<<eblocks(L.nn), ETPB, 0, s>>>(L, N->y, N->fscale, x0);
    return launched("sdx_guess_predict");
    API_END
}

int sdx_guess_refine(sdx_hier_t h, const double* b, double* x, int steps, void* stream) {
    Hier* H = reinterpret_cast<Hier*>(h);
    if (!H || !b || !x || steps < 0) { set_error("invalid argument"); return SDX_EINVAL; }
    if (H->released) { set_error("this hierarchy belongs to a batch: use the sdx_batch_* calls"); return SDX_EINVAL; }
    API_BEGIN
    cudaStream_t s = (cudaStream_t)stream;
    const long long v4 = 4 * H->lv[0].nn;
    for (int k = 0; k < steps; ++k) launch_uzawa<double>(*H, 0, x, b, s);
    // y = K x = b - r;  alpha = <y, b> / <y, y>;  x *= alpha
    launch_apply<double>(*H, 0, x, H->r0, b, s);
    vec_axpy(H->r0, b, -1.0, v4, s);  // r0 = r - b = -y
    vec_dot(*H, H->r0, b, v4, H->scal + 250, s);
    vec_dot(*H, H->r0, H->r0, v4, H->scal + 251, s);
    count_launches(2);
    k_line_alpha<<<1, 1, 0, s>>>(H->scal + 250, H->scal + 252);
    k_negate<<<1, 1, 0, s>>>(H->scal + 252);
    vec_scale_dev(x, x, H->scal + 252, false, v4, s);
    return launched("sdx_guess_refine");
    API_END
}

}  // extern "C"
