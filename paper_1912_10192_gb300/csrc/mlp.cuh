// mlp.cuh -- the learned starting point of the inversion (device side).
//
// A 10 -> 64 -> 64 -> 64 -> 2 tanh network maps the normal-frame scalars of
// a conserved state (Sec. 2.6) and four metric invariants to a guess of
// (W, v^2); Newton (c2p.cuh) always refines it, and the start from the
// previous primitives is the fallback. The paper has no such guess.
//
// Inputs (the ten features), from the FP64 scalars D, Q.n, Qt^2, B^2, Q.B:
//   f0 ln D; f1 ln((-Q.n - D)/D); f2 ln(Qt^2/D^2 + 1e-30);
//   f3 (Q.B)^2/(Qt^2 B^2) (0 if either is 0); f4 ln(U_kappa/U_rho) + (gam-1) ln D;
//   f5 ln(B^2/D + 1e-30); f6 alpha; f7 ln(beta_i beta^i + 1e-30), beta^i = alpha^2 g^{ti};
//   f8 ln(sqrt(-g)/alpha); f9 x1.
// Targets: y0 = ln(W/D), y1 = ln Gamma^2; the guess is W = D e^y0, v^2 = 1 - e^-y1.
//
// Inference runs on the 5th-generation tensor cores, one 128-row tile per
// CTA of 128 threads (one row per thread): the standardised inputs and the
// hidden activations are bfloat16 rows of a K-major operand in shared
// memory, the weights a bfloat16 image brought in by one bulk TMA copy, and
// each layer is tcgen05.mma (M = 128, N = 64, K = 16 per instruction) into
// 64 TMEM columns, read back with tcgen05.ld (each warp its 32 lanes); bias
// and tanh in FP32. The 64 -> 2 output layer is a per-thread FP32 dot product.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include "c2p.cuh"

namespace hamr {

constexpr int MLP_NIN = 10;
constexpr int MLP_H = 64;
constexpr int MLP_NOUT = 2;
constexpr int MLP_ROWS = 128;  // rows of one tile = threads of the CTA
// flat FP32 parameter vector: W1 (64 x 10, row = output unit), b1, W2 (64 x 64), b2, W3, b3, W4 (2 x 64), b4
constexpr int P_W1 = 0, P_B1 = 640, P_W2 = 704, P_B2 = 4800, P_W3 = 4864, P_B3 = 8960, P_W4 = 9024, P_B4 = 9152;
constexpr int MLP_NPARAM = 9154;
constexpr int MLP_NNORM = 24;  // fmean[10], fstd[10], ymean[2], ystd[2]

// Inference image (global memory, copied whole into shared memory):
// bfloat16 weight operands in the no-swizzle K-major core-matrix layout
// (a core matrix = 8 rows x 16 bytes stored contiguously; the 8-row groups
// of an operand with K columns are (K / 8) * 128 bytes apart, the K-groups
// of a row group 128 bytes apart), then FP32 values.
constexpr int IMG_W1 = 0;      // 64 x 16 (inputs padded 10 -> 16): 2048 B
constexpr int IMG_W2 = 2048;   // 64 x 64: 8192 B
constexpr int IMG_W3 = 10240;  // 64 x 64: 8192 B
constexpr int IMG_F = 18432;   // floats below
constexpr int IMGF_B1 = 0, IMGF_B2 = 64, IMGF_B3 = 128, IMGF_W4 = 192, IMGF_B4 = 320, IMGF_FM = 324,
              IMGF_FI = 334, IMGF_YM = 344, IMGF_YS = 346, IMGF_N = 348;
constexpr int MLP_IMG_BYTES = IMG_F + IMGF_N * 4;  // 19824, a multiple of 16
// shared memory of one CTA
constexpr int SM_A = 0;                       // activation operand, 128 x 64 bf16 (16 KB)
constexpr int SM_IMG = 16384;                 // the image
constexpr int SM_BAR = SM_IMG + 19840;        // two mbarriers + the TMEM address slot
constexpr int MLP_SMEM_BYTES = SM_BAR + 64;   // 36288
constexpr uint32_t MLP_TMEM_COLS = 64;

__host__ __device__ constexpr int core_off(int row, int k, int K) {  // byte offset of bf16 element (row, k)
    return (row >> 3) * (K / 8) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// waits for the phase of the given parity; gives up after ~1 s (returns false)
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
    if (mbar_try_wait(a, parity)) return true;
    const uint64_t t0 = gtimer_ns();
    while (!mbar_try_wait(a, parity))
        if (gtimer_ns() - t0 > 1000000000ull) return false;
    return true;
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
// bulk (non-tensor) TMA copy global -> shared, completion counted on the mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D[tmem] (+)= A[smem] . B[smem]^T, bf16 operands, FP32 accumulators
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; q++) v[q] = __uint_as_float(r[q]);
}

// shared-memory matrix descriptor: no swizzle, K-major core matrices; lbo = byte
// stride between K-adjacent core matrices, sbo = between 8-row groups
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;  // descriptor version (fixed 0b001 at bits 46..48)
    return d;                 // base offset 0, absolute LBO mode, layout type 0 (no swizzle)
}
// instruction descriptor of kind::f16: D FP32, A and B bf16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ------------------------------------------------------------ features
__device__ __forceinline__ void mlp_features(const C2PScalars& S, double Urho, double Uent, const Metric<double>& m,
                                             double x1, double gam, float f[MLP_NIN]) {
    // exact power-of-two scaling by 1/2^e (e the binary exponent of D) keeps
    // the FP32 copies of the density-scaled scalars in range
    const int hi = __double2hiint(S.D);
    const int e = ((hi >> 20) & 0x7FF) - 1023;
    const double s = __hiloint2double((1023 - e) << 20, 0);
    const float Dn = (float)(S.D * s);
    const float En = (float)((-S.Qdotn - S.D) * s);
    const float Qn = (float)(S.Qtsq * s * s);
    const float Bn = (float)(S.Bsq * s);
    const float QBn = (float)(S.QB2 * (s * s) * s);
    const float lnD = logf(Dn) + (float)e * 0.69314718056f;
    f[0] = lnD;
    f[1] = logf(fmaxf(En, 1e-30f * Dn) / Dn);
    f[2] = logf(Qn / (Dn * Dn) + 1e-30f);
    const float den = Qn * Bn;
    f[3] = (den > 0.0f) ? fminf(QBn / den, 1.0f) : 0.0f;
    f[4] = logf((float)Uent / (float)Urho) + (float)(gam - 1.0) * lnD;
    f[5] = logf(Bn / Dn + 1e-30f);
    const float al = (float)m.alpha;
    const float b1 = al * al * (float)m.c01;
    f[6] = al;
    f[7] = logf((float)m.g11 * b1 * b1 + 1e-30f);
    f[8] = logf((float)m.gdet / al);
    f[9] = (float)x1;
}

// ------------------------------------------------------------ one CTA's network
struct MlpCta {
    uint8_t* sm;     // dynamic shared memory (MLP_SMEM_BYTES)
    uint32_t tmem;   // TMEM base of the CTA's 64 columns
    uint32_t phase;  // parity of the next MMA-barrier phase
    bool ok;         // false once a wait gave up (the guesses are then not used)
    bool loaded;
};

// All 128 threads. Allocates TMEM, starts the image copy.
__device__ __forceinline__ void mlp_begin(MlpCta& C, uint8_t* sm, const uint8_t* img) {
    C.sm = sm;
    C.phase = 0;
    C.ok = true;
    C.loaded = false;
    const uint32_t bar_load = smem_u32(sm + SM_BAR), bar_mma = bar_load + 8, slot = bar_load + 16;
    if (threadIdx.x == 0) {
        mbar_init(bar_load, 1);
        mbar_init(bar_mma, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        tmem_alloc(slot, MLP_TMEM_COLS);
        tmem_relinquish();
    }
    if (threadIdx.x == 0) {
        mbar_expect_tx(bar_load, (uint32_t)MLP_IMG_BYTES);
        bulk_g2s(smem_u32(sm + SM_IMG), img, (uint32_t)MLP_IMG_BYTES, bar_load);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    C.tmem = *(volatile uint32_t*)(sm + SM_BAR + 16);
}

// All 128 threads; frees the TMEM columns.
__device__ __forceinline__ void mlp_end(MlpCta& C) {
    const uint32_t bar_load = smem_u32(C.sm + SM_BAR);
    if (!C.loaded) {  // the image copy must have landed before the CTA exits
        if (!mbar_wait(bar_load, 0)) C.ok = false;
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) {
        tc_fence_after();
        tmem_dealloc(C.tmem, MLP_TMEM_COLS);
    }
}

// issues the MMAs of one layer (thread 0) and waits for them (all threads)
__device__ __forceinline__ void mlp_layer(MlpCta& C, int w_off, int K) {
    const uint32_t bar_mma = smem_u32(C.sm + SM_BAR) + 8;
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && C.ok) {
        tc_fence_after();
        const uint32_t a0 = smem_u32(C.sm + SM_A), b0 = smem_u32(C.sm + SM_IMG + w_off);
        const uint32_t sbo = (uint32_t)(K / 8) * 128u;
        for (int ks = 0; ks < K / 16; ks++)
            mma_bf16(C.tmem, smem_desc(a0 + ks * 256, 128, sbo), smem_desc(b0 + ks * 256, 128, sbo),
                     idesc_bf16(MLP_ROWS, MLP_H), ks > 0 ? 1u : 0u);
        mma_commit(bar_mma);
    }
    bool ok = C.ok && mbar_wait(bar_mma, C.phase);
    C.phase ^= 1u;
    C.ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
}

// writes 16 activations (columns c0..c0+15 of this thread's row) as bf16 into the K = 64 operand
__device__ __forceinline__ void put_row16(uint8_t* A, int row, int c0, const float h[16]) {
#pragma unroll
    for (int half = 0; half < 2; half++) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const __nv_bfloat162 b = __floats2bfloat162_rn(h[half * 8 + 2 * q], h[half * 8 + 2 * q + 1]);
            w[q] = *reinterpret_cast<const uint32_t*>(&b);
        }
        *reinterpret_cast<uint4*>(A + core_off(row, c0 + half * 8, 64)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// All 128 threads. f: this thread's raw features (ignored if !active).
// Returns true with out = (W/D ratio's log, ln Gamma^2) when the network ran.
__device__ __forceinline__ bool mlp_infer(MlpCta& C, const float f[MLP_NIN], bool active, float out[MLP_NOUT]) {
    uint8_t* A = C.sm + SM_A;
    const float* F = reinterpret_cast<const float*>(C.sm + SM_IMG + IMG_F);
    const int row = threadIdx.x;
    if (!C.loaded) {
        C.ok = __syncthreads_and(C.ok && mbar_wait(smem_u32(C.sm + SM_BAR), 0)) != 0;
        C.loaded = true;
    }
    // layer 1 operand: standardised inputs, K padded to 16
    {
        float x[16];
#pragma unroll
        for (int q = 0; q < 16; q++) x[q] = 0.0f;
        if (active && C.ok) {
#pragma unroll
            for (int q = 0; q < MLP_NIN; q++) x[q] = (f[q] - F[IMGF_FM + q]) * F[IMGF_FI + q];
        }
#pragma unroll
        for (int half = 0; half < 2; half++) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const __nv_bfloat162 b = __floats2bfloat162_rn(x[half * 8 + 2 * q], x[half * 8 + 2 * q + 1]);
                w[q] = *reinterpret_cast<const uint32_t*>(&b);
            }
            *reinterpret_cast<uint4*>(A + core_off(row, half * 8, 16)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    mlp_layer(C, IMG_W1, 16);
    const uint32_t lane_addr = C.tmem + ((uint32_t)(threadIdx.x & ~31u) << 16);
    // hidden layers 1 and 2 -> operand of the next layer
#pragma unroll 1
    for (int layer = 0; layer < 2; layer++) {
        const int boff = layer == 0 ? IMGF_B1 : IMGF_B2;
        if (C.ok) {
#pragma unroll
            for (int c = 0; c < 4; c++) {
                float h[16];
                tmem_ld16(lane_addr + 16 * c, h);
#pragma unroll
                for (int q = 0; q < 16; q++) h[q] = tanhf(h[q] + F[boff + 16 * c + q]);
                put_row16(A, row, 16 * c, h);
            }
        }
        mlp_layer(C, layer == 0 ? IMG_W2 : IMG_W3, 64);
    }
    // hidden layer 3 and the output layer
    float y0 = F[IMGF_B4], y1 = F[IMGF_B4 + 1];
    if (C.ok) {
#pragma unroll
        for (int c = 0; c < 4; c++) {
            float h[16];
            tmem_ld16(lane_addr + 16 * c, h);
#pragma unroll
            for (int q = 0; q < 16; q++) {
                const float t = tanhf(h[q] + F[IMGF_B3 + 16 * c + q]);
                y0 = fmaf(F[IMGF_W4 + 16 * c + q], t, y0);
                y1 = fmaf(F[IMGF_W4 + 64 + 16 * c + q], t, y1);
            }
        }
    }
    out[0] = y0 * F[IMGF_YS] + F[IMGF_YM];
    out[1] = y1 * F[IMGF_YS + 1] + F[IMGF_YM + 1];
    return C.ok;
}

// (W, v^2) start from the network's outputs
__device__ __forceinline__ void mlp_guess(double D, const float y[MLP_NOUT], double g[2]) {
    g[0] = D * (double)__expf(fminf(y[0], 60.0f));
    g[1] = 1.0 - (double)__expf(-fmaxf(y[1], 0.0f));
}

}  // namespace hamr
