// Learned birth proposal: a small 1-D convolutional network that maps a tile
// of station windows to a density over the tile's pixels and the event time,
// trained on windows simulated from the model's own generative story, and
// turned into a birth table for cmh_set_birth_table.
//
// Network (one example = 8 x 8 stations of a tile x 256 samples):
//   input  X0[t][s] = log1p(s_t^2) of station s (64 channels) at sample t
//   4 x conv1d (64 -> 64 channels, kernel 5, stride 2, padding 2) + ReLU:
//          256 -> 128 -> 64 -> 32 -> 16 samples
//   FC 1024 -> 512 + ReLU, FC 512 -> 4101 outputs:
//          4096 pixel logits (64 x 64 pixels of the tile), 1 "no event" logit,
//          mean and log sd of the event time (relative to the window start)
//          and of the magnitude.
// Loss: cross-entropy over the 4097 classes, Gaussian negative log-likelihood
// of time and magnitude for windows that hold an event; AdamW.
//
// Every matrix product runs on the fifth-generation tensor cores (tcgen05.mma,
// BF16 operands staged in shared memory, FP32 accumulators in tensor memory;
// a convolution is a product with the im2col matrix of its input, read in
// place by the tile loader);
// activations and gradients are kept in FP32, their BF16 copies feed the
// products, and the parameters have FP32 masters with BF16 copies.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "chromh.h"
#include "cmh_common.cuh"

namespace cmh {

namespace {

constexpr int kNS = 64;        // stations per tile (8 x 8), the first layer's channels
constexpr int kNL = 256;       // samples per window
constexpr int kC = 64;         // channels of every convolution
constexpr int kKW = 5;         // kernel width
constexpr int kKC = kC * kKW;  // 320: im2col width
constexpr int kNPix = 4096;    // 64 x 64 pixels of a tile
constexpr int kNOut = kNPix + 1 + 4;
constexpr int kNOutP = (kNOut + 7) & ~7;   // 4104: the BF16 output gradient's rows, zero-padded to whole 16-byte vectors
constexpr int kF1In = 16 * kC; // 1024
constexpr int kF1Out = 512;
constexpr double kTile = 800.0;   // km, side of a tile (8 stations at 100 km)
constexpr double kPix = kTile / 64.0;
// origin times of simulated events, seconds from the window start: from
// kTMin to the window's end (kTMax at 10 Hz, the prior the output is
// initialised at)
constexpr double kTMin = -15.0, kTMax = 25.6;

// parameter layout (floats): conv l (W [64][320], b [64]) x 4, F1 [512][1024], fb1, F2 [4101][512], fb2
constexpr long long kConvW = (long long)kC * kKC, kConvP = kConvW + kC;
constexpr long long kOffF1 = 4 * kConvP, kOffFb1 = kOffF1 + (long long)kF1Out * kF1In;
constexpr long long kOffF2 = kOffFb1 + kF1Out, kOffFb2 = kOffF2 + (long long)kNOut * kF1Out;
constexpr long long kNParam = kOffFb2 + kNOut;

// ---------------------------------------------------------------------------
// C[M,N] = op(A)[M,K] op(B)[K,N] (+ C) (+ bias[n]) (ReLU), BF16 in, FP32 out.
// A(m,k) = TA ? A[k*lda+m] : A[m*lda+k];  B(k,n) = TB ? B[n*ldb+k] : B[k*ldb+n].
// Split K (gridDim.z > 1): split z covers K range [z kc, (z + 1) kc) and
// writes its partial product to C + z M ldc (no bias, ReLU or accumulate);
// sum_splits adds the partials in split order.
// a_lin > 0: A (not transposed) is the im2col matrix of the activation A
// [B][a_lin][64] for a_lout output samples, read in place (row b a_lout + t,
// column k 64 + c is x[b][2t - 2 + k][c], 0 outside); b_lin likewise for B
// (not transposed; its rows are the im2col rows).
// ---------------------------------------------------------------------------
// The product on the fifth-generation tensor cores (tcgen05).  A CTA of
// 128 threads computes a 128 x 64 tile of C: per K tile of 64, op(A)
// [128 x 64] and op(B)^T [64 x 64] are staged in shared memory in a K-major
// canonical layout without swizzle (8 x 8 core matrices of 128 contiguous
// bytes): by the tensor memory accelerator for an operand that is
// K-contiguous and read as it stands (TMA_A / TMA_B: one 3-D box per tile,
// chunk-major, row r and column k at (k / 8) * rows * 16 + r * 16 +
// (k % 8) * 2), else by the threads (row-group-major, at
// (r / 8) * 1024 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2); then one
// thread issues four tcgen05.mma (M = 128, N = 64, K = 16; BF16 operands,
// FP32 accumulator in tensor memory: row m in TMEM lane m, column n in
// column n of a 64-column allocation) and commits them to the stage's
// mbarrier.  Three stages, staged two tiles ahead: a tile's copies are in
// flight while the tensor cores multiply the tiles before it.  The epilogue reads the
// accumulator with tcgen05.ld (warp w: lanes 32w..32w+31) and applies
// accumulate / bias / ReLU / BF16 copy.  Every mbarrier wait is bounded (50
// ms of wall time); on a timeout the CTA records it in *err.
// VEC: 16-byte operand loads along each operand's contiguous dimension (its
// extent and leading dimension multiples of 8, base 16-byte aligned; 8
// consecutive im2col columns are 8 consecutive channels of one input
// sample); otherwise element-wise loads.
// ---------------------------------------------------------------------------
constexpr int TM = 128, TN = 64, TK = 64;
constexpr int kStages = 3;                            // shared stages of a product's K tiles
constexpr int kStageBytes = (TM + TN) * TK * 2;       // 24 KB: the A and B tiles of one stage
constexpr unsigned long long kTcWaitNs = 50000000ull;   // 50 ms: a product's tile waits take microseconds

__device__ __forceinline__ unsigned tc_smem(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle; lbo = bytes between
// core matrices adjacent along K, sbo = bytes between 8-row groups
__device__ __forceinline__ unsigned long long tc_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D F32, A and B BF16, both K-major
constexpr unsigned tc_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) | ((unsigned)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned d, unsigned long long a, unsigned long long b, unsigned idesc,
                                       int accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_smem(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_bar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(bar)) : "memory");
}

__device__ __forceinline__ unsigned long long tc_now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the phase of parity `ph` of *bar to complete, for at most
// kTcWaitNs nanoseconds of wall time
__device__ __forceinline__ bool tc_bar_wait(unsigned long long* bar, unsigned ph) {
    const unsigned long long t0 = tc_now_ns();
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(tc_smem(bar)), "r"(ph)
            : "memory");
        if (done) return true;
        if (tc_now_ns() - t0 > kTcWaitNs) return false;
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 16 bytes global -> shared without registers (zeros when !valid; src must
// still point into the operand)
__device__ __forceinline__ void tc_cp16(void* dst, const void* src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc_smem(dst)), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void tc_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void tc_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 16 consecutive accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld16(unsigned taddr, float* v) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// arm *bar for `bytes` of asynchronous copies (one arrival)
__device__ __forceinline__ void tc_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(bar)), "r"(bytes)
                 : "memory");
}

// one tile of a K-contiguous operand by the tensor memory accelerator: the
// map views the operand as (8 elements, rows, K / 8 chunks); the box
// (8, rows of the tile, 8 chunks) lands as [chunk][row][8 elements], the
// chunk-major canonical layout (LBO = rows x 16 bytes, SBO = 128 bytes);
// rows and chunks outside the operand are filled with zeros
__device__ __forceinline__ void tc_tma_tile(void* dst, const CUtensorMap* map, int row0, int chunk0,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(tc_smem(dst)), "l"(map), "r"(0), "r"(row0), "r"(chunk0), "r"(tc_smem(bar))
        : "memory");
}

template <bool TA, bool TB, bool VEC, bool TMA_A, bool TMA_B>
__global__ void __launch_bounds__(128) gemm_tc(int M, int N, int K, const __nv_bfloat16* A, int lda,
                                               const __nv_bfloat16* B, int ldb, float* C, int ldc,
                                               const float* bias, int relu, int accumulate, __nv_bfloat16* Cb,
                                               int kc, int a_lin, int a_lout, int b_lin, int b_lout, int* err,
                                               const __grid_constant__ CUtensorMap map_a,
                                               const __grid_constant__ CUtensorMap map_b) {
    static_assert(!TMA_A || (!TA && VEC), "the tensor map views a K-contiguous A");
    static_assert(!TMA_B || (TB && VEC), "the tensor map views a K-contiguous B");
    extern __shared__ __align__(1024) unsigned char tsm[];   // [kStages] x (A 16 KB, B 8 KB)
    __shared__ __align__(8) unsigned long long bar[kStages];    // a stage's products have read it
    __shared__ __align__(8) unsigned long long full[kStages];   // a stage's tensor-map copies have landed
    __shared__ unsigned s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    if (gridDim.z > 1) C += (long long)blockIdx.z * M * ldc;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&s_tmem)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int q = 0; q < kStages; ++q) {
            tc_bar_init(&bar[q]);
            tc_bar_init(&full[q]);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = s_tmem;
    const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    // element (r, k) of a staged K-major tile
    auto at = [](unsigned char* base, int r, int k) {
        return reinterpret_cast<__nv_bfloat16*>(base + (r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
    };
    auto fill = [&](int st, int k0) {
        unsigned char* As = tsm + st * kStageBytes;
        unsigned char* Bs = As + 16384;
        if (VEC) {
#pragma unroll
            for (int i = 0; i < 8 && !TMA_A; ++i) {
                const int v = tid + i * 128;
                // a quarter warp (8 lanes) takes 8 consecutive rows of one
                // 16-byte chunk column: one core-matrix row block of 128
                // contiguous bytes in shared memory (no bank conflict), 64
                // contiguous bytes per row across the warp in global memory
                const int lw = v & 31, vw = v >> 5;
                if (!TA) {   // 128 rows x 8 vectors along k, asynchronous copies
                    const int r = (vw >> 1) * 8 + (lw & 7), c8 = ((vw & 1) * 4 + (lw >> 3)) * 8, gm = m0 + r,
                              gk = k0 + c8;
                    const __nv_bfloat16* src = A;
                    bool ok = gm < M && gk < ke;
                    if (ok) {
                        if (a_lin > 0) {
                            const int bb = gm / a_lout, t = gm - bb * a_lout, sx = 2 * t - 2 + (gk >> 6);
                            ok = sx >= 0 && sx < a_lin;
                            if (ok) src = A + ((long long)bb * a_lin + sx) * kC + (gk & 63);
                        } else {
                            src = A + (long long)gm * lda + gk;
                        }
                    }
                    tc_cp16(at(As, r, c8), src, ok);
                } else {     // 64 k x 16 vectors along m; a quarter warp: 8 consecutive k
                    const int k = (lw & 7) + 8 * (vw & 7), r8 = ((lw >> 3) + 4 * (vw >> 3)) * 8, gm = m0 + r8,
                              gk = k0 + k;
                    uint4 x = (gm < M && gk < ke) ? __ldg(reinterpret_cast<const uint4*>(A + (long long)gk * lda + gm))
                                                  : zero4;
                    const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&x);
#pragma unroll
                    for (int j = 0; j < 8; ++j) *at(As, r8 + j, k) = e[j];
                }
            }
#pragma unroll
            for (int i = 0; i < 4 && !TMA_B; ++i) {
                const int v = tid + i * 128;
                const int lw = v & 31, vw = v >> 5;
                if (TB) {    // 64 rows (n) x 8 vectors along k, asynchronous copies
                    const int r = (vw >> 1) * 8 + (lw & 7), c8 = ((vw & 1) * 4 + (lw >> 3)) * 8, gn = n0 + r,
                              gk = k0 + c8;
                    const bool ok = gn < N && gk < ke;
                    tc_cp16(at(Bs, r, c8), ok ? B + (long long)gn * ldb + gk : B, ok);
                } else {     // 64 k x 8 vectors along n; a quarter warp: 8 consecutive k
                    const int k = (lw & 7) + 8 * (vw & 7), r8 = ((lw >> 3) + 4 * (vw >> 3)) * 8, gn = n0 + r8,
                              gk = k0 + k;
                    uint4 x = zero4;
                    if (gn < N && gk < ke) {
                        if (b_lin > 0) {
                            const int bb = gk / b_lout, t = gk - bb * b_lout, sx = 2 * t - 2 + (gn >> 6);
                            if (sx >= 0 && sx < b_lin)
                                x = __ldg(reinterpret_cast<const uint4*>(B + ((long long)bb * b_lin + sx) * kC + (gn & 63)));
                        } else {
                            x = __ldg(reinterpret_cast<const uint4*>(B + (long long)gk * ldb + gn));
                        }
                    }
                    const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&x);
#pragma unroll
                    for (int j = 0; j < 8; ++j) *at(Bs, r8 + j, k) = e[j];
                }
            }
        } else {
            for (int e = tid; e < TM * TK; e += 128) {
                const int r = TA ? (e & (TM - 1)) : (e >> 6), k = TA ? (e >> 7) : (e & (TK - 1));
                const int gm = m0 + r, gk = k0 + k;
                *at(As, r, k) = (gm < M && gk < ke) ? (TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk])
                                                    : zero;
            }
            for (int e = tid; e < TN * TK; e += 128) {
                const int r = TB ? (e >> 6) : (e & (TN - 1)), k = TB ? (e & (TK - 1)) : (e >> 6);
                const int gn = n0 + r, gk = k0 + k;
                *at(Bs, r, k) = (gn < N && gk < ke) ? (TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn])
                                                    : zero;
            }
        }
    };
    const int nk = ke > kb ? (ke - kb + TK - 1) / TK : 0;
    constexpr unsigned idesc = tc_idesc(TM, TN);
    // byte offsets between core matrices along K (LBO) and between 8-row
    // groups (SBO): the threads' layout, or the tensor map's chunk-major one
    constexpr unsigned lbo_a = TMA_A ? TM * 16 : 128, sbo_a = TMA_A ? 128 : 1024;
    constexpr unsigned lbo_b = TMA_B ? TN * 16 : 128, sbo_b = TMA_B ? 128 : 1024;
    constexpr unsigned tma_bytes = (TMA_A ? TM * TK * 2 : 0) + (TMA_B ? TN * TK * 2 : 0);
    bool ok = true;
    // staging of tile t into stage t % kStages: the tensor-map copies (one
    // thread), the asynchronous copies and the register-staged operands (all
    // threads), closed by one asynchronous-copy group per thread and tile
    auto issue = [&](int t) {
        const int st = t % kStages, k0 = kb + t * TK;
        if ((TMA_A || TMA_B) && tid == 0) {
            tc_expect_tx(&full[st], tma_bytes);
            if (TMA_A) tc_tma_tile(tsm + st * kStageBytes, &map_a, m0, k0 >> 3, &full[st]);
            if (TMA_B) tc_tma_tile(tsm + st * kStageBytes + 16384, &map_b, n0, k0 >> 3, &full[st]);
        }
        if (!(TMA_A && TMA_B)) fill(st, k0);
        tc_cp_commit();
    };
    // tile u of a stage is its (u / kStages)-th use: its mbarrier phases have parity (u / kStages) & 1
    for (int t = 0; t < kStages - 1; ++t) {
        if (t < nk) issue(t);
        else tc_cp_commit();
    }
    for (int t = 0; t < nk; ++t) {
        const int st = t % kStages, tn = t + kStages - 1;
        if (tn < nk) {
            if (tn >= kStages &&   // the products of tile tn - kStages have read that stage
                !tc_bar_wait(&bar[tn % kStages], (unsigned)((tn / kStages - 1) & 1)))
                ok = false;
            issue(tn);
        } else {
            tc_cp_commit();
        }
        tc_cp_wait<kStages - 1>();   // this thread's copies of tile t have landed
        tc_proxy_fence();            // and, with the threads' stores, are visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
            if ((TMA_A || TMA_B) && !tc_bar_wait(&full[st], (unsigned)((t / kStages) & 1)))   // the tensor-map copies
                ok = false;
            tc_fence_after();
            const unsigned a0 = tc_smem(tsm + st * kStageBytes), b0 = a0 + 16384;
#pragma unroll
            for (int j = 0; j < TK / 16; ++j)
                tc_mma(tmem, tc_desc(a0 + j * 2 * lbo_a, lbo_a, sbo_a), tc_desc(b0 + j * 2 * lbo_b, lbo_b, sbo_b),
                       idesc, (t > 0 || j > 0) ? 1 : 0);
            tc_commit(&bar[st]);
        }
    }
    // the last group: every product is done
    if (nk > 0 && !tc_bar_wait(&bar[(nk - 1) % kStages], (unsigned)(((nk - 1) / kStages) & 1))) ok = false;
    tc_fence_after();
    // the accumulator tile through shared memory (the stages are free: every
    // product has completed), so that C is written in whole rows by
    // consecutive threads: row r of the tile at cs[r * (TN + 1)]
    float* cs = reinterpret_cast<float*>(tsm);
#pragma unroll 1
    for (int c0 = 0; c0 < TN; c0 += 16) {
        float v[16];
        if (nk > 0) {
            tc_ld16(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0, v);
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) cs[(warp * 32 + lane) * (TN + 1) + c0 + i] = v[i];
    }
    __syncthreads();
    for (int e = tid; e < TM * TN; e += 128) {
        const int r = e / TN, c = e - r * TN, m = m0 + r, n = n0 + c;
        if (m >= M || n >= N) continue;
        float x = cs[r * (TN + 1) + c];
        const long long o = (long long)m * ldc + n;
        if (accumulate) x += C[o];
        if (bias) x += bias[n];
        if (relu) x = x > 0.f ? x : 0.f;
        C[o] = x;
        if (Cb) Cb[o] = __float2bfloat16(x);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN) : "memory");
    if (!ok && tid == 0) atomicExch(err, 1);
}

// the adjoint of im2col, dX[b][s][c] = sum over (t, k) with 2t - 2 + k = s
// of dA[(b,t)][k*64+c], then through the ReLU of the previous layer (output
// Y): dZ = dX where Y > 0, else 0, and its BF16 copy
__global__ void col2im_relu(const float* dA, int Bn, int Lin, int Lout, const float* Y, float* dZ, __nv_bfloat16* dZb) {
    const long long n = (long long)Bn * Lin * kC;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % kC);
        const int s = (int)((i / kC) % Lin), b = (int)(i / ((long long)kC * Lin));
        float v = 0.f;
        for (int k = 0; k < kKW; ++k) {
            const int t2 = s + 2 - k;   // = 2t
            if (t2 < 0 || (t2 & 1)) continue;
            const int t = t2 >> 1;
            if (t >= Lout) continue;
            v += dA[((long long)b * Lout + t) * kKC + k * kC + c];
        }
        v = Y[i] > 0.f ? v : 0.f;
        dZ[i] = v;
        dZb[i] = __float2bfloat16(v);
    }
}

// dZ = dY (where the ReLU output is positive), and its BF16 copy
__global__ void relu_back(const float* dY, const float* Y, long long n, float* dZ, __nv_bfloat16* dZb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = Y[i] > 0.f ? dY[i] : 0.f;
        dZ[i] = v;
        dZb[i] = __float2bfloat16(v);
    }
}

__global__ void to_bf16(const float* x, long long n, __nv_bfloat16* y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

// the same for the first `cols` columns of `rows` rows (strides ldx, ldy):
// the columns of y beyond `cols` are left as they are
__global__ void to_bf16_rows(const float* x, int rows, int cols, int ldx, __nv_bfloat16* y, int ldy) {
    const long long n = (long long)rows * cols;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / cols, c = i - r * cols;
        y[r * ldy + c] = __float2bfloat16(x[r * ldx + c]);
    }
}

// partial column sums of a [M][N] matrix (bias gradients): block (32, 8)
// sums columns bx*32 + tx over rows [by*rc, (by + 1)*rc) into part[by][n]
__global__ void col_sums(const float* D, int M, int N, int rc, float* part) {
    __shared__ float red[8][33];
    const int n = blockIdx.x * 32 + threadIdx.x, r0 = blockIdx.y * rc, r1 = min(M, r0 + rc);
    float s = 0.f;
    if (n < N)
        for (int m = r0 + threadIdx.y; m < r1; m += 8) s += D[(long long)m * N + n];
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && n < N) {
        float t = 0.f;
        for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
        part[(long long)blockIdx.y * N + n] = t;
    }
}

// out[i] = sum over z < splits of part[z][i], in split order (deterministic)
__global__ void sum_splits(const float* part, long long n, int splits, float* out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += part[(long long)z * n + i];
        out[i] = s;
    }
}

__device__ __forceinline__ float block_sum(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

__device__ __forceinline__ float block_max(float v, float* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = -INFINITY;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    return t;
}

// one block per example: cross-entropy over the 4097 classes and the
// Gaussian NLL of time and magnitude (events only); gradients of the mean
// loss into dO, the example's loss into loss[b]
__global__ void __launch_bounds__(256) loss_grad(const float* O, const int* label, const float* tl, const float* ml,
                                                 int Bn, float* dO, float* loss) {
    __shared__ float red[32];
    const int b = blockIdx.x;
    const float* o = O + (long long)b * kNOut;
    float* g = dO + (long long)b * kNOut;
    const int lab = label[b];
    float mx = -INFINITY;
    for (int i = threadIdx.x; i <= kNPix; i += blockDim.x) mx = fmaxf(mx, o[i]);
    mx = block_max(mx, red);
    float se = 0.f;
    for (int i = threadIdx.x; i <= kNPix; i += blockDim.x) se += expf(o[i] - mx);
    se = block_sum(se, red);
    const float lse = mx + logf(se), inv = 1.f / (float)Bn;
    for (int i = threadIdx.x; i <= kNPix; i += blockDim.x) g[i] = (expf(o[i] - mx) / se - (i == lab ? 1.f : 0.f)) * inv;
    if (threadIdx.x == 0) {
        float l = lse - o[lab];
        float gt[4] = {0.f, 0.f, 0.f, 0.f};
        if (lab < kNPix) {
            // NLL of y under N(mu, e^{2 ls}): ls + (y - mu)^2 / (2 e^{2 ls}), ls clamped
            const float y2[2] = {tl[b], ml[b]};
            for (int q = 0; q < 2; ++q) {
                const float mu = o[kNPix + 1 + 2 * q], ls = fminf(fmaxf(o[kNPix + 2 + 2 * q], -4.f), 6.f);
                const float iv = expf(-2.f * ls), r = y2[q] - mu;
                l += ls + 0.5f * r * r * iv;
                gt[2 * q] = -r * iv * inv;
                const bool in = o[kNPix + 2 + 2 * q] > -4.f && o[kNPix + 2 + 2 * q] < 6.f;
                gt[2 * q + 1] = in ? (1.f - r * r * iv) * inv : 0.f;
            }
        }
        for (int q = 0; q < 4; ++q) g[kNPix + 1 + q] = gt[q];
        loss[b] = l;
    }
}

__global__ void adamw(float* p, const float* g, float* m1, float* m2, long long n, float lr, float b1, float b2,
                      float c1, float c2, float eps, float wd, __nv_bfloat16* pb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.f - b1) * gi, v = b2 * m2[i] + (1.f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        const float q = p[i] - lr * ((a / c1) / (sqrtf(v / c2) + eps) + wd * p[i]);
        p[i] = q;
        pb[i] = __float2bfloat16(q);
    }
}

// ---- simulated training windows (the model's generative story) -------------
// Example b of batch `step`: 8 x 8 stations jittered around the centres of
// 100 km cells of an 800 km tile; with probability 1/2 one event, uniform in
// the tile, magnitude 2 + Exp(1), origin time uniform in [-15, 25.6) s of the
// window; 256 samples at f per station: s = sqrt(noise + arrival variance)
// * N(0, 1) (float32); features log1p(s^2).  Labels: the event's pixel (or
// 4096 for none), its time relative to the window start, its magnitude.
__global__ void __launch_bounds__(256) gen_windows(Geo g, unsigned long long seed, unsigned long long step, int Bn,
                                                   __nv_bfloat16* X, int* label, float* tl, float* ml) {
    const int b = blockIdx.x;
    __shared__ float sx[kNS], sy[kNS];
    __shared__ double ev[4];
    __shared__ int has;
    unsigned long long c[4];
    if (threadIdx.x < kNS) {
        c[0] = step; c[1] = (unsigned long long)b; c[2] = (unsigned long long)threadIdx.x; c[3] = 7ULL;
        philox4x64(c, seed, 3ULL);
        const int r = threadIdx.x / 8, q = threadIdx.x % 8;
        sx[threadIdx.x] = (float)((q + 0.5) * 100.0 + (u01(c[0]) * 2.0 - 1.0) * 25.0);
        sy[threadIdx.x] = (float)((r + 0.5) * 100.0 + (u01(c[1]) * 2.0 - 1.0) * 25.0);
    }
    if (threadIdx.x == 0) {
        c[0] = step; c[1] = (unsigned long long)b; c[2] = 1000ULL; c[3] = 8ULL;
        philox4x64(c, seed, 3ULL);
        has = u01(c[0]) < 0.5;
        ev[0] = u01(c[1]) * kTile;
        ev[1] = u01(c[2]) * kTile;
        ev[2] = kTMin + u01(c[3]) * (kNL / g.f_hz - kTMin);
        c[0] = step; c[1] = (unsigned long long)b; c[2] = 1001ULL; c[3] = 8ULL;
        philox4x64(c, seed, 3ULL);
        ev[3] = 2.0 - log(u01o(c[0]));
        if (has) {
            const int px = min(63, (int)(ev[0] / kPix)), py = min(63, (int)(ev[1] / kPix));
            label[b] = py * 64 + px;
            tl[b] = (float)ev[2];
            ml[b] = (float)ev[3];
        } else {
            label[b] = kNPix;
            tl[b] = 0.f;
            ml[b] = 0.f;
        }
    }
    __syncthreads();
    // per station: reached?, arrival time, amplitude at the arrival
    __shared__ float arr[kNS], amp[kNS];
    __shared__ int reach[kNS];
    if (threadIdx.x < kNS) {
        const int s = threadIdx.x;
        const double dx = ev[0] - sx[s], dy = ev[1] - sy[s], dist = sqrt(dx * dx + dy * dy);
        reach[s] = has && dist < g.R_max;
        arr[s] = (float)(ev[2] + dist / g.v);
        amp[s] = (float)exp(g.alpha * ev[3] - g.beta_att * dist);
    }
    __syncthreads();
    // four samples of one station per Philox block: s = sqrt(noise + c^2) z
    // (variance reading) or c + sqrt(noise) z (additive reading), c = A g(u),
    // z from Box-Muller on both halves of two uniform pairs
    const float fs = (float)g.f_hz, ts = (float)((double)g.n_w / g.f_hz), itau = (float)(1.0 / g.tau);
    const float nv = (float)g.noise_var;
    for (int q = threadIdx.x; q < kNS * kNL / 4; q += blockDim.x) {
        const int s = q % kNS, t0 = (q / kNS) * 4;
        unsigned long long w[4] = {step, (unsigned long long)b, (unsigned long long)q, 9ULL};
        philox4x64(w, seed, 3ULL);
        float z[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float u1 = ((float)(w[2 * h] >> 40) + 0.5f) * (1.0f / 16777216.0f);
            const float u2 = (float)(w[2 * h + 1] >> 40) * (1.0f / 16777216.0f);
            const float r = sqrtf(-2.f * logf(u1));
            float sn, cs;
            sincospif(2.f * u2, &sn, &cs);
            z[2 * h] = r * cs;
            z[2 * h + 1] = r * sn;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int t = t0 + k;
            const float u = (float)t / fs - arr[s];
            const float c = (reach[s] && u >= 0.f && u < ts) ? amp[s] * expf(-u * itau) : 0.f;
            const float x = g.mean_mode ? c + sqrtf(nv) * z[k] : sqrtf(nv + c * c) * z[k];
            X[((long long)b * kNL + t) * kNS + s] = __float2bfloat16(log1pf(x * x));
        }
    }
}

// features of the windows of a tile from a model's signals (float32 rows):
// example b starts at sample k0 + b * hop; station s of the tile is row st[s]
__global__ void gather_windows(const float* sig, long long pitch, long long n_samp, const int* st, long long k0,
                               int hop, int Bn, __nv_bfloat16* X) {
    const long long n = (long long)Bn * kNL * kNS;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(i % kNS), t = (int)((i / kNS) % kNL), b = (int)(i / ((long long)kNS * kNL));
        const long long k = k0 + (long long)b * hop + t;
        float v = 0.f;
        if (k < n_samp) {
            const float x = sig[(long long)st[s] * pitch + k];
            v = log1pf(x * x);
        }
        X[i] = __float2bfloat16(v);
    }
}

// add the network's density of the windows of a tile to a birth table
// (pixels of the world grid, nt bins over [0, T)): pixel mass (softmax
// without the "no event" class) times the time Gaussian's mass in each bin;
// with msum, the same weights times the window's predicted magnitude
__global__ void __launch_bounds__(256) accumulate_table(const float* O, int Bn, double t0, double hop_s, int ox,
                                                        int oy, int nx, int ny, int nt, double dt, float* tab,
                                                        float* msum) {
    __shared__ float red[32];
    const int b = blockIdx.x;
    const float* o = O + (long long)b * kNOut;
    float mx = -INFINITY;
    for (int i = threadIdx.x; i <= kNPix; i += blockDim.x) mx = fmaxf(mx, o[i]);
    mx = block_max(mx, red);
    float se = 0.f;
    for (int i = threadIdx.x; i <= kNPix; i += blockDim.x) se += expf(o[i] - mx);
    se = block_sum(se, red);
    const double mu = t0 + b * hop_s + o[kNPix + 1];
    const double sd = exp(fminf(fmaxf(o[kNPix + 2], -4.f), 6.f)) + 1.0;
    const float mu_m = o[kNPix + 3];
    const int b0 = max(0, (int)floor((mu - 4.0 * sd) / dt)), b1 = min(nt - 1, (int)floor((mu + 4.0 * sd) / dt));
    for (int i = threadIdx.x; i < kNPix; i += blockDim.x) {
        const float p = expf(o[i] - mx) / se;
        if (p < 1e-5f) continue;
        const int gx = ox + (i % 64), gy = oy + (i / 64);
        if (gx < 0 || gy < 0 || gx >= nx || gy >= ny) continue;
        float* row = tab + ((long long)gy * nx + gx) * nt;
        for (int q = b0; q <= b1; ++q) {
            const double a = (q * dt - mu) / (sd * 1.4142135623730951), z = ((q + 1) * dt - mu) / (sd * 1.4142135623730951);
            const float wq = p * (float)(0.5 * (erf(z) - erf(a)));
            atomicAdd(row + q, wq);
            if (msum) atomicAdd(msum + (row - tab) + q, wq * mu_m);
        }
    }
}

inline int blocks_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

}  // namespace
}  // namespace cmh

using namespace cmh;

struct cmh_net {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int bmax = 0;
    unsigned long long seed = 0, steps = 0;
    float *p = nullptr, *gr = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16* pb = nullptr;
    // activations (FP32 and BF16 copies) and gradients
    __nv_bfloat16* x0 = nullptr;
    float *y[4] = {nullptr}, *h = nullptr, *o = nullptr, *dO = nullptr, *dh = nullptr, *dcol = nullptr;
    __nv_bfloat16 *yb[4] = {nullptr}, *hb = nullptr, *dOb = nullptr, *dhb = nullptr, *dyb = nullptr;
    float *dy = nullptr, *dx = nullptr, *loss = nullptr, *tl = nullptr, *ml = nullptr;
    float* ws = nullptr;   // split partials of products and column sums
    int* label = nullptr;
    std::vector<void*> allocs;

    template <typename T>
    bool alloc(T** q, size_t n) {
        if (cudaMalloc((void**)q, sizeof(T) * std::max<size_t>(n, 1)) != cudaSuccess) return false;
        allocs.push_back((void*)*q);
        return true;
    }
    ~cmh_net() {
        if (stream) cudaStreamSynchronize(stream);
        for (void* q : allocs) cudaFree(q);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

constexpr int kMaxSplits = 64;
constexpr long long kWsFloats = (long long)kMaxSplits * kC * kKC;   // split partials of the largest split product

// set by a product whose bounded mbarrier wait ran out (checked by the host
// after each network call; sticky for the process)
__device__ int g_tc_err = 0;

// K is split when the M x N tiles alone would leave most SMs idle and the
// epilogue is a plain store into a dense C (the weight gradients of the
// convolutions: 64 x 320 outputs over up to 32768 rows)
// device address of g_tc_err per device: looked up when a network is
// created on the device (a network's kernels run only while it exists, and a
// device reset that would move the address destroys the networks with it)
std::mutex g_err_mu;
int* g_err_addr[64] = {nullptr};

cudaError_t tc_err_lookup() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_tc_err);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_err_mu);
    g_err_addr[dev] = p;
    return cudaSuccess;
}

cudaError_t tc_err_address(int** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> lock(g_err_mu);
        if (g_err_addr[dev]) {
            *out = g_err_addr[dev];
            return cudaSuccess;
        }
    }
    if ((e = tc_err_lookup()) != cudaSuccess) return e;
    return tc_err_address(out);
}

// cuTensorMapEncodeTiled, reached through the runtime (no link against
// libcuda); null if the driver does not offer it
typedef CUresult (*encode_tiled_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

encode_tiled_fn tensor_map_encoder() {
    static encode_tiled_fn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (encode_tiled_fn)f;
        (void)cudaGetLastError();
    }
    return fn;
}

// tensor map of a K-contiguous BF16 operand [rows][ld] (K columns used, K a
// multiple of 8, base 16-byte aligned, ld a multiple of 8) viewed as
// (8 elements, rows, K / 8 chunks) with a box of (8, box_rows, 8).  The
// network's operands repeat every step, so encoded maps are kept (a small
// cache keyed by every argument; a map describes addresses, not contents).
bool k_tensor_map_encode(CUtensorMap* map, const __nv_bfloat16* base, int rows, int K, int ld, int box_rows);

bool k_tensor_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int K, int ld, int box_rows) {
    struct Entry {
        const void* base;
        int rows, K, ld, box, ok;
        CUtensorMap map;
    };
    static std::mutex mu;
    static std::vector<Entry> cache;
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& e : cache)
        if (e.base == base && e.rows == rows && e.K == K && e.ld == ld && e.box == box_rows) {
            *map = e.map;
            return e.ok;
        }
    Entry e;
    e.base = base;
    e.rows = rows;
    e.K = K;
    e.ld = ld;
    e.box = box_rows;
    std::memset(&e.map, 0, sizeof(e.map));
    e.ok = k_tensor_map_encode(&e.map, base, rows, K, ld, box_rows);
    if (cache.size() >= 256) cache.erase(cache.begin());
    cache.push_back(e);
    *map = e.map;
    return e.ok;
}

bool k_tensor_map_encode(CUtensorMap* map, const __nv_bfloat16* base, int rows, int K, int ld, int box_rows) {
    encode_tiled_fn enc = tensor_map_encoder();
    if (!enc || rows < 1 || K < 8 || K % 8 || ld % 8 || ((unsigned long long)base & 15ULL)) return false;
    const cuuint64_t dims[3] = {8, (cuuint64_t)rows, (cuuint64_t)(K / 8)};
    const cuuint64_t strides[2] = {(cuuint64_t)ld * 2, 16};
    const cuuint32_t box[3] = {8, (cuuint32_t)box_rows, 8};
    const cuuint32_t es[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <bool TA, bool TB, bool VEC, bool TMA_A, bool TMA_B>
cudaError_t launch_tc(dim3 grid, cudaStream_t s, int M, int N, int K, const __nv_bfloat16* A, int lda,
                      const __nv_bfloat16* B, int ldb, float* C, int ldc, const float* bias, int relu, int acc,
                      __nv_bfloat16* Cb, int kc, int a_lin, int a_lout, int b_lin, int b_lout, const CUtensorMap& ma,
                      const CUtensorMap& mb) {
    static bool attr = false;
    constexpr int smem = kStages * kStageBytes;   // the stages of A and B tiles: 72 KB
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(gemm_tc<TA, TB, VEC, TMA_A, TMA_B>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int* err = nullptr;
    cudaError_t e = tc_err_address(&err);
    if (e != cudaSuccess) return e;
    gemm_tc<TA, TB, VEC, TMA_A, TMA_B><<<grid, 128, smem, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, relu, acc,
                                                               Cb, kc, a_lin, a_lout, b_lin, b_lout, err, ma, mb);
    return cudaGetLastError();
}

// the variant for the operands at hand: tensor-map loads for a K-contiguous
// operand read as it stands (not an im2col view), 16-byte or element-wise
// loads by the threads otherwise
template <bool TA, bool TB>
cudaError_t launch_product(dim3 grid, cudaStream_t s, bool vec, int M, int N, int K, const __nv_bfloat16* A,
                           int lda, const __nv_bfloat16* B, int ldb, float* C, int ldc, const float* bias, int relu,
                           int acc, __nv_bfloat16* Cb, int kc, int a_pad, int a_lin, int a_lout, int b_lin, int b_lout) {
    CUtensorMap ma, mb;
    std::memset(&ma, 0, sizeof(ma));
    std::memset(&mb, 0, sizeof(mb));
    if (!vec)
        return launch_tc<TA, TB, false, false, false>(grid, s, M, N, K, A, lda, B, ldb, C, ldc, bias, relu, acc, Cb,
                                                      kc, 0, 0, 0, 0, ma, mb);
    // a zero-padded A is mapped over its padded extent
    const bool ta = !TA && a_lin == 0 && k_tensor_map(&ma, A, M, a_pad ? (K + 7) & ~7 : K, lda, TM);
    const bool tb = TB && b_lin == 0 && k_tensor_map(&mb, B, N, K, ldb, TN);
    if constexpr (!TA && TB) {
        if (ta && tb)
            return launch_tc<TA, TB, true, true, true>(grid, s, M, N, K, A, lda, B, ldb, C, ldc, bias, relu, acc, Cb,
                                                       kc, a_lin, a_lout, b_lin, b_lout, ma, mb);
    }
    if constexpr (!TA) {
        if (ta)
            return launch_tc<TA, TB, true, !TA, false>(grid, s, M, N, K, A, lda, B, ldb, C, ldc, bias, relu, acc,
                                                       Cb, kc, a_lin, a_lout, b_lin, b_lout, ma, mb);
    }
    if constexpr (TB) {
        if (tb)
            return launch_tc<TA, TB, true, false, TB>(grid, s, M, N, K, A, lda, B, ldb, C, ldc, bias, relu, acc, Cb,
                                                      kc, a_lin, a_lout, b_lin, b_lout, ma, mb);
    }
    return launch_tc<TA, TB, true, false, false>(grid, s, M, N, K, A, lda, B, ldb, C, ldc, bias, relu, acc, Cb, kc,
                                                 a_lin, a_lout, b_lin, b_lout, ma, mb);
}

template <bool TA, bool TB>
// a_pad: every row of A (along its contiguous dimension: M when TA, else K)
// is zero-padded in memory to a multiple of 8 elements, so 16-byte loads may
// read past the extent
cudaError_t gemm(cudaStream_t s, float* ws, int M, int N, int K, const __nv_bfloat16* A, int lda,
                 const __nv_bfloat16* B, int ldb, float* C, int ldc, const float* bias, int relu, int acc,
                 __nv_bfloat16* Cb, int a_lin = 0, int a_lout = 0, int b_lin = 0, int b_lout = 0, int a_pad = 0) {
    const int gx = (N + TN - 1) / TN, gy = (M + TM - 1) / TM, tiles = gx * gy;
    int splits = 1, kc = K;
    if (ws && !bias && !relu && !acc && !Cb && ldc == N && tiles < 152) {
        splits = std::min(kMaxSplits, std::min((304 + tiles - 1) / tiles, (K + 255) / 256));
        while (splits > 1 && (long long)splits * M * N > kWsFloats) --splits;
        if (splits > 1) {
            kc = ((K + splits - 1) / splits + TK - 1) / TK * TK;
            splits = (K + kc - 1) / kc;
        }
    }
    // 16-byte operand loads when both operands' contiguous dimensions come in
    // whole aligned vectors
    auto al16 = [](const void* p) { return ((unsigned long long)p & 15ULL) == 0; };
    const bool vec = al16(A) && al16(B) && lda % 8 == 0 && ldb % 8 == 0 &&
                     ((TA ? M % 8 == 0 : K % 8 == 0) || a_pad) && (TB ? K % 8 == 0 : N % 8 == 0);
    const dim3 grid(gx, gy, splits);
    float* out = splits > 1 ? ws : C;
    const float* bs = splits > 1 ? nullptr : bias;
    const int rl = splits > 1 ? 0 : relu, ac = splits > 1 ? 0 : acc;
    __nv_bfloat16* cb = splits > 1 ? nullptr : Cb;
    if ((a_lin > 0 || b_lin > 0) && !vec) return cudaErrorInvalidValue;   // im2col operands need the vector loader
    cudaError_t e = launch_product<TA, TB>(grid, s, vec, M, N, K, A, lda, B, ldb, out, ldc, bs, rl, ac, cb, kc, a_pad,
                                           a_lin, a_lout, b_lin, b_lout);
    if (e != cudaSuccess) return e;
    if (splits > 1) sum_splits<<<blocks_for((long long)M * N), 256, 0, s>>>(ws, (long long)M * N, splits, C);
    return cudaGetLastError();
}

// column sums of a [M][N] matrix over row chunks, added in chunk order
void colsum(cudaStream_t s, float* ws, const float* D, int M, int N, float* out) {
    const int sp = std::max(1, std::min(kMaxSplits, (M + 255) / 256)), rc = (M + sp - 1) / sp;
    col_sums<<<dim3((N + 31) / 32, sp), dim3(32, 8), 0, s>>>(D, M, N, rc, ws);
    sum_splits<<<blocks_for(N), 256, 0, s>>>(ws, N, sp, out);
}

const int kLin[5] = {256, 128, 64, 32, 16};

// forward of a batch whose features are in n->x0; outputs in n->o
cudaError_t forward(cmh_net* n, int Bn) {
    cudaStream_t s = n->stream;
    cudaError_t e = cudaSuccess;
    const __nv_bfloat16* in = n->x0;
    for (int l = 0; l < 4 && e == cudaSuccess; ++l) {
        const int Lin = kLin[l], Lout = kLin[l + 1];
        const long long rows = (long long)Bn * Lout;
        // the im2col matrix of `in` is read in place by the product
        e = gemm<false, true>(s, n->ws, (int)rows, kC, kKC, in, 0, n->pb + l * kConvP, kKC, n->y[l], kC,
                              n->p + l * kConvP + kConvW, 1, 0, n->yb[l], Lin, Lout);
        in = n->yb[l];
    }
    if (e) return e;
    // FC1: [B][1024] x F1^T -> [B][512]
    if ((e = gemm<false, true>(s, n->ws, Bn, kF1Out, kF1In, n->yb[3], kF1In, n->pb + kOffF1, kF1In, n->h, kF1Out,
                               n->p + kOffFb1, 1, 0, n->hb)))
        return e;
    return gemm<false, true>(s, n->ws, Bn, kNOut, kF1Out, n->hb, kF1Out, n->pb + kOffF2, kF1Out, n->o, kNOut,
                             n->p + kOffFb2, 0, 0, nullptr);
}

// loss and gradients of a batch (labels in n->label / tl / ml) into n->gr
cudaError_t backward(cmh_net* n, int Bn) {
    cudaStream_t s = n->stream;
    cudaError_t e;
    loss_grad<<<Bn, 256, 0, s>>>(n->o, n->label, n->tl, n->ml, Bn, n->dO, n->loss);
    // the BF16 output gradient in rows of kNOutP (the padding stays zero)
    to_bf16_rows<<<blocks_for((long long)Bn * kNOut), 256, 0, s>>>(n->dO, Bn, kNOut, kNOut, n->dOb, kNOutP);
    // FC2: dF2 = dO^T h, dfb2 = colsum dO, dh = dO F2
    if ((e = gemm<true, false>(s, n->ws, kNOut, kF1Out, Bn, n->dOb, kNOutP, n->hb, kF1Out, n->gr + kOffF2, kF1Out,
                               nullptr, 0, 0, nullptr, 0, 0, 0, 0, 1)))
        return e;
    colsum(s, n->ws, n->dO, Bn, kNOut, n->gr + kOffFb2);
    if ((e = gemm<false, false>(s, n->ws, Bn, kF1Out, kNOut, n->dOb, kNOutP, n->pb + kOffF2, kF1Out, n->dh, kF1Out,
                                nullptr, 0, 0, nullptr, 0, 0, 0, 0, 1)))
        return e;
    relu_back<<<blocks_for((long long)Bn * kF1Out), 256, 0, s>>>(n->dh, n->h, (long long)Bn * kF1Out, n->dh, n->dhb);
    // FC1: dF1 = dh^T x4, dfb1, dx4 = dh F1 (into dy as [B*16][64])
    if ((e = gemm<true, false>(s, n->ws, kF1Out, kF1In, Bn, n->dhb, kF1Out, n->yb[3], kF1In, n->gr + kOffF1, kF1In, nullptr,
                               0, 0, nullptr)))
        return e;
    colsum(s, n->ws, n->dh, Bn, kF1Out, n->gr + kOffFb1);
    if ((e = gemm<false, false>(s, n->ws, Bn, kF1In, kF1Out, n->dhb, kF1Out, n->pb + kOffF1, kF1In, n->dy, kF1In, nullptr, 0,
                                0, nullptr)))
        return e;
    for (int l = 3; l >= 0; --l) {
        const int Lin = kLin[l], Lout = kLin[l + 1];
        const long long rows = (long long)Bn * Lout;
        // through the ReLU of layer l (below the top layer, col2im_relu did it)
        if (l == 3) relu_back<<<blocks_for(rows * kC), 256, 0, s>>>(n->dy, n->y[l], rows * kC, n->dy, n->dyb);
        // dW = dy^T col (the layer input's im2col matrix read in place), db = colsum dy
        const __nv_bfloat16* in = l == 0 ? n->x0 : n->yb[l - 1];
        if ((e = gemm<true, false>(s, n->ws, kC, kKC, (int)rows, n->dyb, kC, in, 0, n->gr + l * kConvP, kKC, nullptr, 0,
                                   0, nullptr, 0, 0, Lin, Lout)))
            return e;
        colsum(s, n->ws, n->dy, (int)rows, kC, n->gr + l * kConvP + kConvW);
        if (l == 0) break;
        // dcol = dy W, dx = col2im(dcol) (the previous layer's output
        // gradient), through that layer's ReLU
        if ((e = gemm<false, false>(s, n->ws, (int)rows, kKC, kC, n->dyb, kC, n->pb + l * kConvP, kKC, n->dcol, kKC, nullptr,
                                    0, 0, nullptr)))
            return e;
        col2im_relu<<<blocks_for((long long)Bn * Lin * kC), 256, 0, s>>>(n->dcol, Bn, Lin, Lout, n->y[l - 1], n->dy,
                                                                          n->dyb);
    }
    return cudaGetLastError();
}

int net_err(cudaError_t e) {
    if (e == cudaSuccess) {
        // a product whose bounded wait ran out (sticky)
        int f = 0;
        if (cudaMemcpyFromSymbol(&f, g_tc_err, sizeof(int)) != cudaSuccess) return CMH_ERR_CUDA;
        return f ? CMH_ERR_TIMEOUT : CMH_OK;
    }
    if (e == cudaErrorMemoryAllocation) return CMH_ERR_OOM;
    return CMH_ERR_CUDA;
}

}  // namespace

extern "C" int64_t cmh_net_param_count(void) { return kNParam; }

extern "C" int cmh_net_create(int32_t max_batch, uint64_t seed, void* cuda_stream, cmh_net** out) {
    if (!out || max_batch < 1 || max_batch > 4096) return CMH_ERR_ARG;
    *out = nullptr;
    (void)cudaGetLastError();
    cmh_net* n = new (std::nothrow) cmh_net;
    if (!n) return CMH_ERR_OOM;
    n->bmax = max_batch;
    n->seed = seed;
    n->stream = (cudaStream_t)cuda_stream;
    if (!n->stream) {
        if (cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete n;
            return CMH_ERR_CUDA;
        }
        n->own_stream = true;
    }
    if (tc_err_lookup() != cudaSuccess) {
        delete n;
        return CMH_ERR_CUDA;
    }
    const long long B = max_batch;
    bool ok = n->alloc(&n->p, kNParam) && n->alloc(&n->gr, kNParam) && n->alloc(&n->m1, kNParam) &&
              n->alloc(&n->m2, kNParam) && n->alloc(&n->pb, kNParam) && n->alloc(&n->x0, B * kNL * kNS) &&
              n->alloc(&n->h, B * kF1Out) && n->alloc(&n->hb, B * kF1Out) &&
              n->alloc(&n->o, B * kNOut) && n->alloc(&n->dO, B * kNOut) && n->alloc(&n->dOb, B * kNOutP) &&
              n->alloc(&n->dh, B * kF1Out) && n->alloc(&n->dhb, B * kF1Out) && n->alloc(&n->dcol, B * 128 * kKC) &&
              n->alloc(&n->dy, B * 128 * kC) && n->alloc(&n->dyb, B * 128 * kC) && n->alloc(&n->dx, B * 256 * kC) &&
              n->alloc(&n->loss, B) && n->alloc(&n->tl, B) && n->alloc(&n->ml, B) && n->alloc(&n->label, B) && n->alloc(&n->ws, kWsFloats);
    for (int l = 0; l < 4 && ok; ++l) ok = n->alloc(&n->y[l], B * kLin[l + 1] * kC) && n->alloc(&n->yb[l], B * kLin[l + 1] * kC);
    if (!ok || cudaMemset(n->dOb, 0, sizeof(__nv_bfloat16) * B * kNOutP) != cudaSuccess) {
        delete n;
        return CMH_ERR_OOM;
    }
    // He-style initialisation on the host (seeded), biases 0
    std::vector<float> hp(kNParam, 0.f);
    unsigned long long st = seed * 0x9E3779B97F4A7C15ULL + 1;
    auto unif = [&]() {   // splitmix64
        st += 0x9E3779B97F4A7C15ULL;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](long long off, long long cnt, int fan_in) {
        const double a = std::sqrt(6.0 / fan_in);
        for (long long i = 0; i < cnt; ++i) hp[off + i] = (float)((2.0 * unif() - 1.0) * a);
    };
    for (int l = 0; l < 4; ++l) fill(l * kConvP, kConvW, kKC);
    fill(kOffF1, (long long)kF1Out * kF1In, kF1In);
    fill(kOffF2, (long long)kNOut * kF1Out, kF1Out);
    // output layer: small weights and biases at the training prior, so the
    // first steps start from the uninformed loss (even odds of "no event"
    // against a uniform pixel; time and magnitude at their prior mean and
    // spread) instead of from an NLL of thousands that kills the ReLUs
    for (long long i = 0; i < (long long)kNOut * kF1Out; ++i) hp[kOffF2 + i] *= 0.05f;
    hp[kOffFb2 + kNPix] = (float)std::log((double)kNPix);
    hp[kOffFb2 + kNPix + 1] = (float)(0.5 * (kTMin + kTMax));
    hp[kOffFb2 + kNPix + 2] = (float)std::log((kTMax - kTMin) / std::sqrt(12.0));
    hp[kOffFb2 + kNPix + 3] = 3.f;
    hp[kOffFb2 + kNPix + 4] = 0.f;
    cudaError_t e = cudaMemcpy(n->p, hp.data(), sizeof(float) * kNParam, cudaMemcpyHostToDevice);
    if (!e) e = cudaMemset(n->m1, 0, sizeof(float) * kNParam);
    if (!e) e = cudaMemset(n->m2, 0, sizeof(float) * kNParam);
    if (!e) {
        to_bf16<<<blocks_for(kNParam), 256, 0, n->stream>>>(n->p, kNParam, n->pb);
        e = cudaStreamSynchronize(n->stream);
    }
    if (e) {
        delete n;
        return net_err(e);
    }
    *out = n;
    return CMH_OK;
}

extern "C" void cmh_net_destroy(cmh_net* n) { delete n; }

extern "C" int cmh_net_get_params(cmh_net* n, float* out) {
    if (!n || !out) return CMH_ERR_ARG;
    return net_err(cudaMemcpy(out, n->p, sizeof(float) * kNParam, cudaMemcpyDeviceToHost));
}

extern "C" int cmh_net_set_params(cmh_net* n, const float* in) {
    if (!n || !in) return CMH_ERR_ARG;
    cudaError_t e = cudaMemcpy(n->p, in, sizeof(float) * kNParam, cudaMemcpyHostToDevice);
    if (e) return net_err(e);
    to_bf16<<<blocks_for(kNParam), 256, 0, n->stream>>>(n->p, kNParam, n->pb);
    return net_err(cudaStreamSynchronize(n->stream));
}

extern "C" int cmh_net_forward(cmh_net* n, const float* features, int32_t batch, float* out) {
    if (!n || !features || !out || batch < 1 || batch > n->bmax) return CMH_ERR_ARG;
    (void)cudaGetLastError();
    const long long nf = (long long)batch * kNL * kNS;
    std::vector<__nv_bfloat16> hb(nf);
    for (long long i = 0; i < nf; ++i) hb[i] = __float2bfloat16(features[i]);
    cudaError_t e = cudaMemcpyAsync(n->x0, hb.data(), sizeof(__nv_bfloat16) * nf, cudaMemcpyHostToDevice, n->stream);
    if (!e) e = forward(n, batch);
    if (!e) e = cudaMemcpyAsync(out, n->o, sizeof(float) * batch * kNOut, cudaMemcpyDeviceToHost, n->stream);
    if (!e) e = cudaStreamSynchronize(n->stream);
    return net_err(e);
}

extern "C" int cmh_net_gradients(cmh_net* n, const float* features, const int32_t* label, const float* t_label,
                                 const float* m_label, int32_t batch, float* grads, double* loss) {
    if (!n || !features || !label || !t_label || !m_label || !grads || batch < 1 || batch > n->bmax)
        return CMH_ERR_ARG;
    for (int b = 0; b < batch; ++b)
        if (label[b] < 0 || label[b] > kNPix) return CMH_ERR_ARG;
    (void)cudaGetLastError();
    const long long nf = (long long)batch * kNL * kNS;
    std::vector<__nv_bfloat16> hb(nf);
    for (long long i = 0; i < nf; ++i) hb[i] = __float2bfloat16(features[i]);
    cudaStream_t s = n->stream;
    cudaError_t e = cudaMemcpyAsync(n->x0, hb.data(), sizeof(__nv_bfloat16) * nf, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(n->label, label, sizeof(int) * batch, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(n->tl, t_label, sizeof(float) * batch, cudaMemcpyHostToDevice, s);
    if (!e) e = cudaMemcpyAsync(n->ml, m_label, sizeof(float) * batch, cudaMemcpyHostToDevice, s);
    if (!e) e = forward(n, batch);
    if (!e) e = backward(n, batch);
    std::vector<float> lv(batch);
    if (!e) e = cudaMemcpyAsync(grads, n->gr, sizeof(float) * kNParam, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaMemcpyAsync(lv.data(), n->loss, sizeof(float) * batch, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return net_err(e);
    if (loss) {
        double t = 0.0;
        for (float v : lv) t += v;
        *loss = t / batch;
    }
    return CMH_OK;
}

extern "C" int cmh_net_train(cmh_net* n, const cmh_model* geometry, int32_t steps, int32_t batch, double lr,
                             double* loss_out) {
    if (!n || !geometry || steps < 0 || batch < 1 || batch > n->bmax || !(lr > 0.0)) return CMH_ERR_ARG;
    (void)cudaGetLastError();
    const Geo g = cmh_model_geo(geometry);
    cudaStream_t s = n->stream;
    const float b1 = 0.9f, b2 = 0.999f;
    double last = 0.0;
    for (int it = 0; it < steps; ++it) {
        const unsigned long long step = ++n->steps;
        gen_windows<<<batch, 256, 0, s>>>(g, n->seed, step, batch, n->x0, n->label, n->tl, n->ml);
        cudaError_t e = forward(n, batch);
        if (!e) e = backward(n, batch);
        if (e) return net_err(e);
        const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
        adamw<<<blocks_for(kNParam), 256, 0, s>>>(n->p, n->gr, n->m1, n->m2, kNParam, (float)lr, b1, b2, c1, c2,
                                                  1e-8f, 1e-4f, n->pb);
        if (it == steps - 1 && loss_out) {
            std::vector<float> lv(batch);
            e = cudaMemcpyAsync(lv.data(), n->loss, sizeof(float) * batch, cudaMemcpyDeviceToHost, s);
            if (!e) e = cudaStreamSynchronize(s);
            if (e) return net_err(e);
            double t = 0.0;
            for (float v : lv) t += v;
            last = t / batch;
        }
    }
    if (loss_out) *loss_out = last;
    return net_err(cudaStreamSynchronize(s));
}

extern "C" int cmh_net_birth_table(cmh_net* n, cmh_model* m, const int32_t* tiles, const double* tile_origin,
                                   int32_t n_tiles, int32_t nx, int32_t ny, int32_t nt, double hop_s, float* table,
                                   float* magnitude) {
    if (!n || !m || !tiles || !tile_origin || n_tiles < 1 || nx < 1 || ny < 1 || nt < 1 || !table || !(hop_s > 0.0))
        return CMH_ERR_ARG;
    (void)cudaGetLastError();
    const Geo g = cmh_model_geo(m);
    const Dev d = cmh_model_dev(m);
    if (!g.f32) return CMH_ERR_ARG;
    for (int i = 0; i < n_tiles * kNS; ++i)
        if (tiles[i] < 0 || tiles[i] >= g.n_st) return CMH_ERR_ARG;
    cudaStream_t s = n->stream;
    const int hop = std::max(1, (int)std::lround(hop_s * g.f_hz));
    const long long n_win = std::max<long long>(1, (g.n_samp + hop - 1) / hop);
    const size_t ne = (size_t)nx * ny * nt;
    int* dst = nullptr;
    float *dtab = nullptr, *dmag = nullptr;
    cudaError_t e = cudaMalloc(&dst, sizeof(int) * kNS);
    if (!e) e = cudaMalloc(&dtab, sizeof(float) * ne);
    if (!e) e = cudaMemsetAsync(dtab, 0, sizeof(float) * ne, s);
    if (!e && magnitude) e = cudaMalloc(&dmag, sizeof(float) * ne);
    if (!e && magnitude) e = cudaMemsetAsync(dmag, 0, sizeof(float) * ne, s);
    const double dt = g.T / nt;
    for (int ti = 0; ti < n_tiles && !e; ++ti) {
        e = cudaMemcpyAsync(dst, tiles + ti * kNS, sizeof(int) * kNS, cudaMemcpyHostToDevice, s);
        const int ox = (int)std::lround(tile_origin[2 * ti] / (g.W / nx));
        const int oy = (int)std::lround(tile_origin[2 * ti + 1] / (g.W / ny));
        for (long long w0 = 0; w0 < n_win && !e; w0 += n->bmax) {
            const int Bn = (int)std::min<long long>(n->bmax, n_win - w0);
            gather_windows<<<blocks_for((long long)Bn * kNL * kNS), 256, 0, s>>>((const float*)d.sig, g.pitch, g.n_samp,
                                                                                dst, w0 * hop, hop, Bn, n->x0);
            e = forward(n, Bn);
            if (!e) {
                accumulate_table<<<Bn, 256, 0, s>>>(n->o, Bn, (double)(w0 * hop) / g.f_hz, hop / g.f_hz, ox, oy, nx, ny,
                                                    nt, dt, dtab, dmag);
                e = cudaGetLastError();
            }
        }
    }
    if (!e) e = cudaMemcpyAsync(table, dtab, sizeof(float) * ne, cudaMemcpyDeviceToHost, s);
    if (!e && magnitude) e = cudaMemcpyAsync(magnitude, dmag, sizeof(float) * ne, cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (!e && magnitude)   // weighted mean of the predicted magnitudes; the prior mean where nothing was added
        for (size_t i = 0; i < ne; ++i) magnitude[i] = table[i] > 0.f ? magnitude[i] / table[i] : 3.f;
    if (dst) cudaFree(dst);
    if (dtab) cudaFree(dtab);
    if (dmag) cudaFree(dmag);
    return net_err(e);
}
