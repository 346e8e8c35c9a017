// mlp.cu -- the learned starting point of the inversion: model state,
// primitive -> conserved for training pairs, the ten inputs and two
// targets, standardisation, training (forward and backward on the CUDA cores
// in FP32, Adam), the bf16 inference image and the standalone inference.
// The paper has no counterpart (its Newton starts from the previous
// primitives, Sec. 2.6); the network only moves Newton's starting point.
#include <cmath>
#include <cstring>
#include <vector>

#include "hamr_internal.h"
#include "metric.cuh"
#include "mlp.cuh"

namespace hamr {
namespace {

constexpr int TB = 128;  // samples (= threads) per CTA of the training kernels
constexpr int HS = 65;   // row stride of the per-sample activation arrays (bank-conflict free)
constexpr int XS = 11;   // row stride of the input array
// shared memory of k_mlp_fb: parameters, inputs, three hidden layers, output errors
constexpr int FB_SMEM = (MLP_NPARAM + 2 + TB * XS + 3 * TB * HS + TB * 2) * 4;

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {  // Steele, Lea & Flood (2014)
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ void metric_sparse(const hamr_c2p_desc& d, double x1, double x2, Metric<double>& m) {
    FullMetric M;
    metric_at(d.metric, d.a, x1, x2, M);
    to_sparse(M, m);
}

// ---------------------------------------------------------------- data
__global__ void k_prim2cons(hamr_c2p_desc d, int64_t n, const double* __restrict__ prim,
                            const double* __restrict__ x1, const double* __restrict__ x2, double* __restrict__ U) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    Metric<double> m;
    metric_sparse(d, x1[s], x2[s], m);
    double pr[NPRIM];
#pragma unroll
    for (int q = 0; q < NPRIM; q++) pr[q] = prim[q * n + s];
    Fluid<double> st;
    fluid_state(pr, m, st);
    double row[NFLUX];
    flux_row(pr, st, 0, 1, d.gam, entropy_kappa(pr, d.gam), row);
#pragma unroll
    for (int q = 0; q < NCONS; q++) U[q * n + s] = row[q] * m.gdet;
}

__global__ void k_features(hamr_c2p_desc d, int64_t n, const double* __restrict__ U, const double* __restrict__ B,
                           const double* __restrict__ x1, const double* __restrict__ x2,
                           const double* __restrict__ prim, float* __restrict__ feat, float* __restrict__ targ) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    Metric<double> m;
    metric_sparse(d, x1[s], x2[s], m);
    double u[NCONS], bc[3];
#pragma unroll
    for (int q = 0; q < NCONS; q++) u[q] = U[q * n + s];
#pragma unroll
    for (int q = 0; q < 3; q++) bc[q] = B[q * n + s];
    C2PScalars S;
    c2p_scalars(u, bc, m, S);
    float f[MLP_NIN];
    mlp_features(S, u[C_RHO], u[C_ENT], m, x1[s], d.gam, f);
#pragma unroll
    for (int q = 0; q < MLP_NIN; q++) feat[q * n + s] = f[q];
    if (prim && targ) {
        const double q1 = prim[U1 * n + s], q2 = prim[U2 * n + s], q3 = prim[U3 * n + s];
        const double qsq = m.g11 * q1 * q1 + m.g22 * q2 * q2 + m.g33 * q3 * q3 + 2.0 * m.g13 * q1 * q3;
        const double h = 1.0 + d.gam * prim[UU * n + s] / prim[RHO * n + s];
        targ[s] = (float)log(h * sqrt(1.0 + qsq));
        targ[n + s] = (float)log1p(qsq);
    }
}

// sums and sums of squares of the 12 columns (inputs, targets), FP64
__global__ void k_norm_sums(int64_t n, const float* __restrict__ feat, const float* __restrict__ targ,
                            double* __restrict__ sums) {
    __shared__ double red[24][4];
    double acc[24];
#pragma unroll
    for (int q = 0; q < 24; q++) acc[q] = 0.0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < 12; q++) {
            const double v = (q < MLP_NIN) ? feat[q * n + s] : targ[(q - MLP_NIN) * n + s];
            acc[q] += v;
            acc[12 + q] += v * v;
        }
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 24; q++) {
        double v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[q][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 24) {
        double v = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) v += red[threadIdx.x][k];
        atomicAdd(&sums[threadIdx.x], v);
    }
}

// ---------------------------------------------------------------- inference image
__global__ void k_pack(const float* __restrict__ P, const float* __restrict__ norm, uint8_t* __restrict__ img) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    // bf16 operands: W1 padded to 64 x 16, W2 and W3 64 x 64 (row = output unit n, column = input k)
    if (t < 64 * 16) {
        const int r = t / 16, k = t % 16;
        const float w = (k < MLP_NIN) ? P[P_W1 + r * MLP_NIN + k] : 0.0f;
        *reinterpret_cast<__nv_bfloat16*>(img + IMG_W1 + core_off(r, k, 16)) = __float2bfloat16_rn(w);
    } else if (t < 64 * 16 + 2 * 4096) {
        const int u = t - 64 * 16;
        const int which = u / 4096, e = u % 4096, r = e / 64, k = e % 64;
        const float w = P[(which ? P_W3 : P_W2) + r * 64 + k];
        *reinterpret_cast<__nv_bfloat16*>(img + (which ? IMG_W3 : IMG_W2) + core_off(r, k, 64)) =
            __float2bfloat16_rn(w);
    } else if (t < 64 * 16 + 2 * 4096 + IMGF_N) {
        const int q = t - 64 * 16 - 2 * 4096;
        float v = 0.0f;
        if (q < IMGF_W4) v = P[(q < 64 ? P_B1 : (q < 128 ? P_B2 : P_B3)) + (q & 63)];
        else if (q < IMGF_B4) v = __bfloat162float(__float2bfloat16_rn(P[P_W4 + q - IMGF_W4]));
        else if (q < IMGF_B4 + 2) v = P[P_B4 + q - IMGF_B4];
        else if (q < IMGF_FM) v = 0.0f;
        else if (q < IMGF_FI) v = norm[q - IMGF_FM];
        else if (q < IMGF_YM) v = 1.0f / norm[10 + q - IMGF_FI];
        else if (q < IMGF_YS) v = norm[20 + q - IMGF_YM];
        else v = norm[22 + q - IMGF_YS];
        reinterpret_cast<float*>(img + IMG_F)[q] = v;
    }
}
constexpr int PACK_THREADS = 64 * 16 + 2 * 4096 + IMGF_N;

// ---------------------------------------------------------------- training (FP32)
// One CTA: TB samples, forward and backward; the parameter gradient of
// loss = sum over samples and outputs of r^2 / (2 count), r = yn - tn, is
// accumulated into grad; sum r^2 into loss[0].
// mode 0: samples off + 0.., mode 1: sample ids splitmix64(seed ^ (step * batch + b)) mod n.
__global__ void __launch_bounds__(TB) k_mlp_fb(const float* __restrict__ Pg, const float* __restrict__ norm,
                                               const float* __restrict__ feat, const float* __restrict__ targ,
                                               int64_t n, int mode, int64_t off, int64_t count, uint64_t seed,
                                               int64_t step, float* __restrict__ grad, float* __restrict__ loss) {
    extern __shared__ __align__(16) float fsm[];
    float* P = fsm;                       // MLP_NPARAM (+2 pad)
    float* X = P + MLP_NPARAM + 2;        // TB x XS
    float* H1 = X + TB * XS;              // TB x HS, later dz1
    float* H2 = H1 + TB * HS;             // later dz2
    float* H3 = H2 + TB * HS;             // later dz3
    float* DY = H3 + TB * HS;             // TB x 2
    const int t = threadIdx.x;
    for (int q = t; q < MLP_NPARAM; q += TB) P[q] = Pg[q];
    const int64_t b = (int64_t)blockIdx.x * TB + t;
    int64_t g = 0;
    bool active;
    if (mode == 0) {
        g = off + b;
        active = (b < count) && (g < n);
    } else {
        active = b < count;
        g = (int64_t)(splitmix64(seed ^ (uint64_t)(step * count + b)) % (uint64_t)n);
    }
    const float* W1 = P + P_W1;
    const float* W2 = P + P_W2;
    const float* W3 = P + P_W3;
    const float* W4 = P + P_W4;
    __syncthreads();
    // forward
    float x[MLP_NIN];
#pragma unroll
    for (int i = 0; i < MLP_NIN; i++) {
        x[i] = active ? (feat[i * n + g] - norm[i]) / norm[10 + i] : 0.0f;
        X[t * XS + i] = x[i];
    }
    for (int o = 0; o < 64; o++) {
        float z = P[P_B1 + o];
#pragma unroll
        for (int i = 0; i < MLP_NIN; i++) z = fmaf(W1[o * MLP_NIN + i], x[i], z);
        H1[t * HS + o] = tanhf(z);
    }
    for (int o = 0; o < 64; o++) {
        float z = P[P_B2 + o];
        for (int i = 0; i < 64; i++) z = fmaf(W2[o * 64 + i], H1[t * HS + i], z);
        H2[t * HS + o] = tanhf(z);
    }
    for (int o = 0; o < 64; o++) {
        float z = P[P_B3 + o];
        for (int i = 0; i < 64; i++) z = fmaf(W3[o * 64 + i], H2[t * HS + i], z);
        H3[t * HS + o] = tanhf(z);
    }
    float r2 = 0.0f;
    const float inv_count = 1.0f / (float)count;
#pragma unroll
    for (int j = 0; j < 2; j++) {
        float y = P[P_B4 + j];
        for (int o = 0; o < 64; o++) y = fmaf(W4[j * 64 + o], H3[t * HS + o], y);
        const float tn = active ? (targ[j * n + g] - norm[20 + j]) / norm[22 + j] : 0.0f;
        const float r = active ? y - tn : 0.0f;
        r2 += r * r;
        DY[t * 2 + j] = r * inv_count;
    }
    __syncthreads();
    // output layer gradients
    {
        const int j = t >> 6, o = t & 63;
        float a = 0.0f;
        for (int s = 0; s < TB; s++) a = fmaf(DY[s * 2 + j], H3[s * HS + o], a);
        atomicAdd(&grad[P_W4 + j * 64 + o], a);
        if (t < 2) {
            float bsum = 0.0f;
            for (int s = 0; s < TB; s++) bsum += DY[s * 2 + t];
            atomicAdd(&grad[P_B4 + t], bsum);
        }
    }
    __syncthreads();
    // dz3 = (W4^T dy) (1 - h3^2), own row
    for (int o = 0; o < 64; o++) {
        const float h = H3[t * HS + o];
        H3[t * HS + o] = (W4[o] * DY[t * 2] + W4[64 + o] * DY[t * 2 + 1]) * (1.0f - h * h);
    }
    __syncthreads();
    // hidden layers 3 and 2: dW = dz^T h_prev, db = sum dz; then dz_prev = (W^T dz) (1 - h_prev^2)
#pragma unroll 1
    for (int layer = 3; layer >= 2; layer--) {
        float* Z = (layer == 3) ? H3 : H2;
        float* Hp = (layer == 3) ? H2 : H1;
        const float* Wl = (layer == 3) ? W3 : W2;
        const int pw = (layer == 3) ? P_W3 : P_W2, pb = (layer == 3) ? P_B3 : P_B2;
        {
            const int o = t >> 1, i0 = (t & 1) * 32;
            float acc[32];
#pragma unroll
            for (int q = 0; q < 32; q++) acc[q] = 0.0f;
            float bs = 0.0f;
            for (int s = 0; s < TB; s++) {
                const float z = Z[s * HS + o];
                bs += z;
#pragma unroll
                for (int q = 0; q < 32; q++) acc[q] = fmaf(z, Hp[s * HS + i0 + q], acc[q]);
            }
#pragma unroll
            for (int q = 0; q < 32; q++) atomicAdd(&grad[pw + o * 64 + i0 + q], acc[q]);
            if ((t & 1) == 0) atomicAdd(&grad[pb + o], bs);
        }
        __syncthreads();
        {
            float dz[64];
            for (int i = 0; i < 64; i++) {
                float a = 0.0f;
                for (int o = 0; o < 64; o++) a = fmaf(Wl[o * 64 + i], Z[t * HS + o], a);
                const float h = Hp[t * HS + i];
                dz[i] = a * (1.0f - h * h);
            }
            for (int i = 0; i < 64; i++) Hp[t * HS + i] = dz[i];
        }
        __syncthreads();
    }
    // first layer: dW1 = dz1^T x, db1
    {
        const int o = t >> 1, i0 = (t & 1) * 5;
        float acc[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        float bs = 0.0f;
        for (int s = 0; s < TB; s++) {
            const float z = H1[s * HS + o];
            bs += z;
#pragma unroll
            for (int q = 0; q < 5; q++) acc[q] = fmaf(z, X[s * XS + i0 + q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 5; q++) atomicAdd(&grad[P_W1 + o * MLP_NIN + i0 + q], acc[q]);
        if ((t & 1) == 0) atomicAdd(&grad[P_B1 + o], bs);
    }
    // loss
    float v = r2;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) atomicAdd(loss, v);
}

__global__ void k_adam(float* __restrict__ P, float* __restrict__ grad, float* __restrict__ m1,
                       float* __restrict__ m2, float lr, float c1, float c2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= MLP_NPARAM) return;
    const float g = grad[q];
    const float a = 0.9f * m1[q] + 0.1f * g;
    const float b = 0.999f * m2[q] + 0.001f * g * g;
    m1[q] = a;
    m2[q] = b;
    P[q] -= lr * (a * c1) / (sqrtf(b * c2) + 1e-8f);
    grad[q] = 0.0f;
}

// FP32 forward of the training path, one thread per sample
__global__ void k_fwd32(const float* __restrict__ Pg, const float* __restrict__ norm, const float* __restrict__ feat,
                        int64_t n, float* __restrict__ out) {
    extern __shared__ __align__(16) float P[];
    for (int q = threadIdx.x; q < MLP_NPARAM; q += blockDim.x) P[q] = Pg[q];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[MLP_NIN], h[64], h2[64];
#pragma unroll
    for (int i = 0; i < MLP_NIN; i++) x[i] = (feat[i * n + s] - norm[i]) / norm[10 + i];
    for (int o = 0; o < 64; o++) {
        float z = P[P_B1 + o];
#pragma unroll
        for (int i = 0; i < MLP_NIN; i++) z = fmaf(P[P_W1 + o * MLP_NIN + i], x[i], z);
        h[o] = tanhf(z);
    }
    for (int o = 0; o < 64; o++) {
        float z = P[P_B2 + o];
        for (int i = 0; i < 64; i++) z = fmaf(P[P_W2 + o * 64 + i], h[i], z);
        h2[o] = tanhf(z);
    }
    for (int o = 0; o < 64; o++) {
        float z = P[P_B3 + o];
        for (int i = 0; i < 64; i++) z = fmaf(P[P_W3 + o * 64 + i], h2[i], z);
        h[o] = tanhf(z);
    }
    for (int j = 0; j < 2; j++) {
        float y = P[P_B4 + j];
        for (int o = 0; o < 64; o++) y = fmaf(P[P_W4 + j * 64 + o], h[o], y);
        out[j * n + s] = y * norm[22 + j] + norm[20 + j];
    }
}

// bf16 tensor-core inference of given inputs, 128 samples per CTA
__global__ void __launch_bounds__(MLP_ROWS) k_fwd16(const uint8_t* __restrict__ img, const float* __restrict__ feat,
                                                   int64_t n, float* __restrict__ out, int* err) {
    extern __shared__ __align__(16) uint8_t sm[];
    const int64_t s = (int64_t)blockIdx.x * MLP_ROWS + threadIdx.x;
    const bool active = s < n;
    MlpCta C;
    mlp_begin(C, sm, img);
    float f[MLP_NIN], y[MLP_NOUT];
#pragma unroll
    for (int q = 0; q < MLP_NIN; q++) f[q] = active ? feat[q * n + s] : 0.0f;
    const bool ran = mlp_infer(C, f, active, y);
    mlp_end(C);
    if (!C.ok && threadIdx.x == 0) atomicExch(err, 1);
    if (active) {
        out[s] = ran ? y[0] : __int_as_float(0x7fc00000);
        out[n + s] = ran ? y[1] : __int_as_float(0x7fc00000);
    }
}

int check_model(const hamr_mlp* m) {
    if (!m) return set_error(HAMR_EINVAL, "model is NULL");
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != m->device) return set_error(HAMR_EINVAL, "the model lives on device %d, device %d is current", m->device,
                                           dev);
    return HAMR_OK;
}

#define MLP_CUDA(x)                                                                       \
    do {                                                                                  \
        cudaError_t e_ = (x);                                                             \
        if (e_ != cudaSuccess) return set_error(HAMR_ECUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
    } while (0)

int repack(hamr_mlp* m, cudaStream_t s) {
    k_pack<<<(PACK_THREADS + 255) / 256, 256, 0, s>>>(m->params, m->norm, m->img);
    MLP_CUDA(cudaGetLastError());
    return HAMR_OK;
}

}  // namespace

// inference launch of the standalone inversion (c2p.cu) and the grid
const uint8_t* mlp_image(const hamr_mlp* m) { return m ? m->img : nullptr; }
int* mlp_error_ptr(const hamr_mlp* m) { return m ? m->err : nullptr; }

}  // namespace hamr

using namespace hamr;

extern "C" {

int hamr_prim2cons(const hamr_c2p_desc* d, int64_t n, const double* prim, const double* x1, const double* x2,
                   double* U, void* stream) {
    if (!d || n < 0) return set_error(HAMR_EINVAL, "descriptor NULL or n < 0");
    if (n == 0) return HAMR_OK;
    if (!prim || !x1 || !x2 || !U) return set_error(HAMR_EINVAL, "NULL array");
    k_prim2cons<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(*d, n, prim, x1, x2, U);
    MLP_CUDA(cudaGetLastError());
    return HAMR_OK;
}

int hamr_mlp_create(hamr_mlp** out, uint64_t seed) {
    if (!out) return set_error(HAMR_EINVAL, "out is NULL");
    *out = nullptr;
    hamr_mlp* m = new hamr_mlp;
    cudaGetDevice(&m->device);
    auto fail_free = [&](cudaError_t e) {
        hamr_mlp_destroy(m);
        return set_error(HAMR_ECUDA, "model allocation failed: %s", cudaGetErrorString(e));
    };
    cudaError_t e;
    if ((e = cudaMalloc(&m->params, 4 * MLP_NPARAM * sizeof(float))) != cudaSuccess) return fail_free(e);
    m->grad = m->params + MLP_NPARAM;
    m->m1 = m->grad + MLP_NPARAM;
    m->m2 = m->m1 + MLP_NPARAM;
    if ((e = cudaMalloc(&m->norm, MLP_NNORM * sizeof(float))) != cudaSuccess) return fail_free(e);
    if ((e = cudaMalloc(&m->img, MLP_IMG_BYTES)) != cudaSuccess) return fail_free(e);
    if ((e = cudaMalloc(&m->sums, 24 * sizeof(double))) != cudaSuccess) return fail_free(e);
    if ((e = cudaMalloc(&m->err, sizeof(int))) != cudaSuccess) return fail_free(e);
    // Glorot-uniform weights (bound sqrt(6 / (fan_in + fan_out))), zero biases; uniform
    // numbers from SplitMix64 of seed ^ parameter index
    std::vector<float> P(MLP_NPARAM, 0.0f);
    auto sm64 = [](uint64_t x) {
        x += 0x9E3779B97F4A7C15ull;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        return x ^ (x >> 31);
    };
    const int offs[4] = {P_W1, P_W2, P_W3, P_W4}, fin[4] = {MLP_NIN, 64, 64, 64}, fout[4] = {64, 64, 64, 2};
    for (int l = 0; l < 4; l++) {
        const double bound = std::sqrt(6.0 / (fin[l] + fout[l]));
        for (int q = 0; q < fin[l] * fout[l]; q++) {
            const uint64_t z = sm64(seed ^ (uint64_t)(offs[l] + q));
            const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
            P[offs[l] + q] = (float)((2.0 * u - 1.0) * bound);
        }
    }
    std::vector<float> norm(MLP_NNORM, 0.0f);
    for (int q = 0; q < 10; q++) norm[10 + q] = 1.0f;
    norm[22] = norm[23] = 1.0f;
    if ((e = cudaMemcpy(m->params, P.data(), MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail_free(e);
    if ((e = cudaMemset(m->grad, 0, 3 * MLP_NPARAM * sizeof(float))) != cudaSuccess) return fail_free(e);
    if ((e = cudaMemcpy(m->norm, norm.data(), MLP_NNORM * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail_free(e);
    if ((e = cudaMemset(m->err, 0, sizeof(int))) != cudaSuccess) return fail_free(e);
    int rc = repack(m, 0);
    if (rc) {
        hamr_mlp_destroy(m);
        return rc;
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail_free(e);
    *out = m;
    return HAMR_OK;
}

int hamr_mlp_destroy(hamr_mlp* m) {
    if (!m) return HAMR_OK;
    cudaFree(m->params);
    cudaFree(m->norm);
    cudaFree(m->img);
    cudaFree(m->sums);
    cudaFree(m->loss);
    cudaFree(m->err);
    delete m;
    return HAMR_OK;
}

int hamr_mlp_get_params(const hamr_mlp* m, float* params, float* norm) {
    if (int rc = check_model(m)) return rc;
    MLP_CUDA(cudaDeviceSynchronize());
    if (params) MLP_CUDA(cudaMemcpy(params, m->params, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
    if (norm) MLP_CUDA(cudaMemcpy(norm, m->norm, MLP_NNORM * sizeof(float), cudaMemcpyDeviceToHost));
    return HAMR_OK;
}

int hamr_mlp_set_params(hamr_mlp* m, const float* params, const float* norm) {
    if (int rc = check_model(m)) return rc;
    if (norm)
        for (int q = 0; q < MLP_NNORM; q++)
            if (!std::isfinite(norm[q]) || (((q >= 10 && q < 20) || q >= 22) && !(norm[q] > 0.0f)))
                return set_error(HAMR_EINVAL, "norm[%d] must be finite (standard deviations > 0)", q);
    MLP_CUDA(cudaDeviceSynchronize());
    if (params) MLP_CUDA(cudaMemcpy(m->params, params, MLP_NPARAM * sizeof(float), cudaMemcpyHostToDevice));
    if (norm) MLP_CUDA(cudaMemcpy(m->norm, norm, MLP_NNORM * sizeof(float), cudaMemcpyHostToDevice));
    if (int rc = repack(m, 0)) return rc;
    MLP_CUDA(cudaDeviceSynchronize());
    return HAMR_OK;
}

int hamr_mlp_features(const hamr_c2p_desc* d, int64_t n, const double* U, const double* B, const double* x1,
                      const double* x2, const double* prim, float* feat, float* targ, void* stream) {
    if (!d || n < 0) return set_error(HAMR_EINVAL, "descriptor NULL or n < 0");
    if (n == 0) return HAMR_OK;
    if (!U || !B || !x1 || !x2 || !feat) return set_error(HAMR_EINVAL, "NULL array");
    if ((prim == nullptr) != (targ == nullptr)) return set_error(HAMR_EINVAL, "prim and targ go together");
    k_features<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(*d, n, U, B, x1, x2, prim, feat, targ);
    MLP_CUDA(cudaGetLastError());
    return HAMR_OK;
}

int hamr_mlp_fit_norm(hamr_mlp* m, int64_t n, const float* feat, const float* targ, void* stream) {
    if (int rc = check_model(m)) return rc;
    if (n < 2 || !feat || !targ) return set_error(HAMR_EINVAL, "need n >= 2 samples with targets");
    cudaStream_t s = (cudaStream_t)stream;
    MLP_CUDA(cudaMemsetAsync(m->sums, 0, 24 * sizeof(double), s));
    k_norm_sums<<<1216, 128, 0, s>>>(n, feat, targ, m->sums);
    MLP_CUDA(cudaGetLastError());
    double h[24];
    MLP_CUDA(cudaMemcpyAsync(h, m->sums, sizeof(h), cudaMemcpyDeviceToHost, s));
    MLP_CUDA(cudaStreamSynchronize(s));
    float norm[MLP_NNORM];
    for (int q = 0; q < 12; q++) {
        const double mean = h[q] / (double)n;
        const double var = std::max(h[12 + q] / (double)n - mean * mean, 0.0);
        const double sd = std::max(std::sqrt(var), 1e-6 * std::max(1.0, std::fabs(mean)));
        if (q < MLP_NIN) {
            norm[q] = (float)mean;
            norm[10 + q] = (float)sd;
        } else {
            norm[20 + q - MLP_NIN] = (float)mean;
            norm[22 + q - MLP_NIN] = (float)sd;
        }
    }
    return hamr_mlp_set_params(m, nullptr, norm);
}

int hamr_mlp_train(hamr_mlp* m, int64_t n, const float* feat, const float* targ, const hamr_mlp_train_args* a,
                   float* loss, void* stream) {
    if (int rc = check_model(m)) return rc;
    if (!a || n < 1 || !feat || !targ) return set_error(HAMR_EINVAL, "need arguments, n >= 1 and data");
    if (a->steps < 1 || a->batch < TB || a->batch % TB) return set_error(HAMR_EINVAL, "steps >= 1, batch a multiple of 128");
    if (!(a->lr > 0.0f) || !(a->lr_final >= 0.0f)) return set_error(HAMR_EINVAL, "lr > 0, lr_final >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (m->loss_cap < a->steps) {
        cudaFree(m->loss);
        m->loss = nullptr;
        MLP_CUDA(cudaMalloc(&m->loss, (size_t)a->steps * sizeof(float)));
        m->loss_cap = a->steps;
    }
    MLP_CUDA(cudaFuncSetAttribute(k_mlp_fb, cudaFuncAttributeMaxDynamicSharedMemorySize, FB_SMEM));
    MLP_CUDA(cudaMemsetAsync(m->loss, 0, (size_t)a->steps * sizeof(float), s));
    MLP_CUDA(cudaMemsetAsync(m->grad, 0, MLP_NPARAM * sizeof(float), s));
    const unsigned nb = (unsigned)(a->batch / TB);
    for (int64_t k = 0; k < a->steps; k++) {
        k_mlp_fb<<<nb, TB, FB_SMEM, s>>>(m->params, m->norm, feat, targ, n, 1, 0, a->batch, a->seed, k, m->grad,
                                         m->loss + k);
        m->adam_t++;
        const double tt = (double)m->adam_t;
        const double frac = (a->steps > 1) ? (double)k / (double)(a->steps - 1) : 1.0;
        const double lr = a->lr_final + 0.5 * (a->lr - a->lr_final) * (1.0 + std::cos(3.14159265358979323846 * frac));
        const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, tt)));
        const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, tt)));
        k_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, s>>>(m->params, m->grad, m->m1, m->m2, (float)lr, c1, c2);
    }
    MLP_CUDA(cudaGetLastError());
    if (int rc = repack(m, s)) return rc;
    if (loss) {
        MLP_CUDA(cudaMemcpyAsync(loss, m->loss, (size_t)a->steps * sizeof(float), cudaMemcpyDeviceToHost, s));
        MLP_CUDA(cudaStreamSynchronize(s));
        for (int64_t k = 0; k < a->steps; k++) loss[k] /= (float)(2 * a->batch);
    }
    MLP_CUDA(cudaStreamSynchronize(s));
    return HAMR_OK;
}

int hamr_mlp_loss_grad(hamr_mlp* m, int64_t n, const float* feat, const float* targ, float* grad, float* loss,
                       void* stream) {
    if (int rc = check_model(m)) return rc;
    if (n < 1 || !feat || !targ || !grad || !loss) return set_error(HAMR_EINVAL, "need n >= 1, data and outputs");
    cudaStream_t s = (cudaStream_t)stream;
    if (m->loss_cap < 1) {
        MLP_CUDA(cudaMalloc(&m->loss, sizeof(float)));
        m->loss_cap = 1;
    }
    MLP_CUDA(cudaFuncSetAttribute(k_mlp_fb, cudaFuncAttributeMaxDynamicSharedMemorySize, FB_SMEM));
    MLP_CUDA(cudaMemsetAsync(m->loss, 0, sizeof(float), s));
    MLP_CUDA(cudaMemsetAsync(m->grad, 0, MLP_NPARAM * sizeof(float), s));
    const unsigned nb = (unsigned)((n + TB - 1) / TB);
    k_mlp_fb<<<nb, TB, FB_SMEM, s>>>(m->params, m->norm, feat, targ, n, 0, 0, n, 0, 0, m->grad, m->loss);
    MLP_CUDA(cudaGetLastError());
    MLP_CUDA(cudaMemcpyAsync(grad, m->grad, MLP_NPARAM * sizeof(float), cudaMemcpyDeviceToHost, s));
    MLP_CUDA(cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
    MLP_CUDA(cudaMemsetAsync(m->grad, 0, MLP_NPARAM * sizeof(float), s));
    MLP_CUDA(cudaStreamSynchronize(s));
    loss[0] /= (float)(2 * n);
    return HAMR_OK;
}

int hamr_mlp_forward(const hamr_mlp* m, int64_t n, const float* feat, float* out, int tensor_cores, void* stream) {
    if (int rc = check_model(m)) return rc;
    if (n < 0 || (n > 0 && (!feat || !out))) return set_error(HAMR_EINVAL, "n >= 0 with arrays");
    if (n == 0) return HAMR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (tensor_cores) {
        MLP_CUDA(cudaFuncSetAttribute(k_fwd16, cudaFuncAttributeMaxDynamicSharedMemorySize, MLP_SMEM_BYTES));
        k_fwd16<<<(unsigned)((n + MLP_ROWS - 1) / MLP_ROWS), MLP_ROWS, MLP_SMEM_BYTES, s>>>(m->img, feat, n, out,
                                                                                         m->err);
    } else {
        MLP_CUDA(cudaFuncSetAttribute(k_fwd32, cudaFuncAttributeMaxDynamicSharedMemorySize, MLP_NPARAM * 4));
        k_fwd32<<<(unsigned)((n + 127) / 128), 128, MLP_NPARAM * 4, s>>>(m->params, m->norm, feat, n, out);
    }
    MLP_CUDA(cudaGetLastError());
    return HAMR_OK;
}

int hamr_mlp_error_flag(hamr_mlp* m, int* flag) {
    if (int rc = check_model(m)) return rc;
    if (!flag) return set_error(HAMR_EINVAL, "flag is NULL");
    MLP_CUDA(cudaDeviceSynchronize());
    MLP_CUDA(cudaMemcpy(flag, m->err, sizeof(int), cudaMemcpyDeviceToHost));
    MLP_CUDA(cudaMemset(m->err, 0, sizeof(int)));
    return HAMR_OK;
}

}  // extern "C"
