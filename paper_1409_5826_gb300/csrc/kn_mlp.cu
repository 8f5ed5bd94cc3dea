// kn_mlp.cu -- the learned timestep proposal's network: 64 -> 128 -> 128 -> 1
// (ReLU), BF16 weights and activations, FP32 accumulation, FP32 master weights
// trained with Adam (Kingma & Ba).  The paper has no learned component; this
// is the library's addition on top of the Sec. 4 timestep controller.
//
// Training GEMMs run on the tensor cores with mma.sync.m16n8k16 (BF16 inputs,
// FP32 accumulate).  The batch GEMMs here are tiny (a few hundred MFLOP per
// training step), so one warp per 16x8 output tile with strided fragment
// loads is enough; every fragment load is bounds-checked, so any M, N, K work.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/kn.h"
#include "kn_internal.h"

namespace kn {
kn_status noalloc_fail(kn_status s, const char* msg);  // sets kn_last_error (kn_api.cu)
}
using namespace kn;

typedef __nv_bfloat16 bf16;

struct kn_mlp {
    // FP32 master parameters: W1 [64][128] (in, out), b1 [128], W2 [128][128], b2 [128], w3 [128], b3 [1]
    float* P = nullptr;   // all parameters, contiguous (kMlpParams floats)
    float* G = nullptr;   // gradients, same layout
    float* Am = nullptr;  // Adam first moments
    float* Av = nullptr;  // Adam second moments
    bf16* Wb = nullptr;   // BF16 copies of W1 then W2 (same layouts as the master)
    float* norm = nullptr;  // mu [64], inv_sigma [64]
    // activations for a batch of up to cap rows
    int cap = 0;
    bf16 *X = nullptr, *H1 = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
    float *out = nullptr, *dout = nullptr;
    long long step = 0;
};

namespace {

constexpr int NF = kMlpFeatures, NH = kMlpHidden;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NF * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH;
static_assert(OFF_B3 + 1 == kMlpParams, "parameter layout");

__device__ __forceinline__ uint32_t pack_bf16(bf16 lo, bf16 hi) {
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

enum { EPI_F32 = 0, EPI_RELU_BF16 = 1, EPI_MASK_BF16 = 2 };

// C[m][n] = sum_k A(m,k) B(k,n) (+ bias[n]); A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn].  One warp per 16x8 tile of C.
template <int EPI>
__global__ void gemm_bf16(int M, int N, int K, const bf16* __restrict__ A, long sam, long sak,
                          const bf16* __restrict__ B, long sbk, long sbn, const float* __restrict__ bias,
                          void* C, long ldc, const bf16* __restrict__ mask, long ldm) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int tiles_n = (N + 7) >> 3;
    const int tm = warp / tiles_n, tn = warp - tm * tiles_n;
    if (tm * 16 >= M) return;  // uniform across the warp
    const int m0 = tm * 16, n0 = tn * 8, g = lane >> 2, t = lane & 3;
    const bf16 z = __float2bfloat16(0.f);
    auto lda = [&](int m, int k) { return (m < M && k < K) ? A[m * sam + k * sak] : z; };
    auto ldb = [&](int k, int n) { return (k < K && n < N) ? B[k * sbk + n * sbn] : z; };
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4], b[2];
        a[0] = pack_bf16(lda(m0 + g, k0 + 2 * t), lda(m0 + g, k0 + 2 * t + 1));
        a[1] = pack_bf16(lda(m0 + g + 8, k0 + 2 * t), lda(m0 + g + 8, k0 + 2 * t + 1));
        a[2] = pack_bf16(lda(m0 + g, k0 + 2 * t + 8), lda(m0 + g, k0 + 2 * t + 9));
        a[3] = pack_bf16(lda(m0 + g + 8, k0 + 2 * t + 8), lda(m0 + g + 8, k0 + 2 * t + 9));
        b[0] = pack_bf16(ldb(k0 + 2 * t, n0 + g), ldb(k0 + 2 * t + 1, n0 + g));
        b[1] = pack_bf16(ldb(k0 + 2 * t + 8, n0 + g), ldb(k0 + 2 * t + 9, n0 + g));
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + g + (i >> 1) * 8, n = n0 + 2 * t + (i & 1);
        if (m >= M || n >= N) continue;
        float v = c[i] + (bias ? bias[n] : 0.f);
        if (EPI == EPI_F32) {
            ((float*)C)[m * ldc + n] = v;
        } else if (EPI == EPI_RELU_BF16) {
            ((bf16*)C)[m * ldc + n] = __float2bfloat16(v > 0.f ? v : 0.f);
        } else {
            const float keep = __bfloat162float(mask[m * ldm + n]) > 0.f ? 1.f : 0.f;
            ((bf16*)C)[m * ldc + n] = __float2bfloat16(v * keep);
        }
    }
}

__global__ void prep_x(const float* __restrict__ f, int B, const float* __restrict__ norm, bf16* __restrict__ X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B * NF) {
        const int k = i % NF;
        X[i] = __float2bfloat16((f[i] - norm[k]) * norm[NF + k]);
    }
}

// out[b] = H2[b] . w3 + b3 (one warp per row, FP32)
__global__ void head_fwd(const bf16* __restrict__ H2, int B, const float* __restrict__ P, float* __restrict__ out) {
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= B) return;
    float s = 0.f;
    for (int n = lane; n < NH; n += 32) s += __bfloat162float(H2[row * NH + n]) * P[OFF_W3 + n];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[row] = s + P[OFF_B3];
}

// dout = 2 (out - y) / B; dZ2 = dout w3 (ReLU mask of H2)
__global__ void head_bwd(const float* __restrict__ out, const float* __restrict__ y, int B,
                         const bf16* __restrict__ H2, const float* __restrict__ P, float* __restrict__ dout,
                         bf16* __restrict__ dZ2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B * NH) {
        const int b = i / NH, n = i - b * NH;
        const float d = 2.f * (out[b] - y[b]) / (float)B;
        if (n == 0) dout[b] = d;
        const float keep = __bfloat162float(H2[i]) > 0.f ? 1.f : 0.f;
        dZ2[i] = __float2bfloat16(d * P[OFF_W3 + n] * keep);
    }
}

// column sums in fixed order: db[n] = sum_b D[b][n]; gw3[n] = sum_b H2[b][n] dout[b]; gb3 = sum dout
__global__ void col_sums(const bf16* __restrict__ dZ1, const bf16* __restrict__ dZ2, const bf16* __restrict__ H2,
                         const float* __restrict__ dout, int B, float* __restrict__ G) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < NH) {
        float s1 = 0.f, s2 = 0.f, s3 = 0.f;
        for (int b = 0; b < B; ++b) {
            s1 += __bfloat162float(dZ1[b * NH + n]);
            s2 += __bfloat162float(dZ2[b * NH + n]);
            s3 += __bfloat162float(H2[b * NH + n]) * dout[b];
        }
        G[OFF_B1 + n] = s1;
        G[OFF_B2 + n] = s2;
        G[OFF_W3 + n] = s3;
    } else if (n == NH) {
        float s = 0.f;
        for (int b = 0; b < B; ++b) s += dout[b];
        G[OFF_B3] = s;
    }
}

__global__ void mse(const float* __restrict__ out, const float* __restrict__ y, int B, float* loss) {
    __shared__ float part[256];
    float s = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        const float d = out[b] - y[b];
        s += d * d;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = part[0] / (float)B;
}

__global__ void adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m, float* __restrict__ v,
                     bf16* __restrict__ Wb, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kMlpParams) {
        const float g = G[i];
        const float mi = b1 * m[i] + (1.f - b1) * g;
        const float vi = b2 * v[i] + (1.f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        const float p = P[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        P[i] = p;
        if (i < OFF_B1) Wb[i] = __float2bfloat16(p);
        else if (i >= OFF_W2 && i < OFF_B2) Wb[NF * NH + (i - OFF_W2)] = __float2bfloat16(p);
    }
}

__global__ void to_bf16(const float* __restrict__ P, bf16* __restrict__ Wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NF * NH) Wb[i] = __float2bfloat16(P[OFF_W1 + i]);
    else if (i < NF * NH + NH * NH) Wb[i] = __float2bfloat16(P[OFF_W2 + (i - NF * NH)]);
}

static kn_status cuda_fail(cudaError_t e) { return noalloc_fail(KN_ERR_CUDA, cudaGetErrorString(e)); }
#define MC(x)                                  \
    do {                                       \
        cudaError_t e_ = (x);                  \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

static kn_status ensure_cap(kn_mlp* m, int B) {
    if (B <= m->cap) return KN_OK;
    cudaFree(m->X);
    cudaFree(m->H1);
    cudaFree(m->H2);
    cudaFree(m->dZ2);
    cudaFree(m->dZ1);
    cudaFree(m->out);
    cudaFree(m->dout);
    m->X = m->H1 = m->H2 = m->dZ2 = m->dZ1 = nullptr;
    m->out = m->dout = nullptr;
    m->cap = 0;
    MC(cudaMalloc(&m->X, sizeof(bf16) * (size_t)B * NF));
    MC(cudaMalloc(&m->H1, sizeof(bf16) * (size_t)B * NH));
    MC(cudaMalloc(&m->H2, sizeof(bf16) * (size_t)B * NH));
    MC(cudaMalloc(&m->dZ2, sizeof(bf16) * (size_t)B * NH));
    MC(cudaMalloc(&m->dZ1, sizeof(bf16) * (size_t)B * NH));
    MC(cudaMalloc(&m->out, sizeof(float) * (size_t)B));
    MC(cudaMalloc(&m->dout, sizeof(float) * (size_t)B));
    m->cap = B;
    return KN_OK;
}

static int gemm_grid(int M, int N) {
    const long warps = (long)((M + 15) / 16) * ((N + 7) / 8);
    return (int)((warps * 32 + 127) / 128);
}

static kn_status forward(kn_mlp* m, const float* feat, int B, cudaStream_t st) {
    kn_status s = ensure_cap(m, B);
    if (s != KN_OK) return s;
    prep_x<<<(B * NF + 255) / 256, 256, 0, st>>>(feat, B, m->norm, m->X);
    const bf16* W1 = m->Wb;
    const bf16* W2 = m->Wb + NF * NH;
    gemm_bf16<EPI_RELU_BF16><<<gemm_grid(B, NH), 128, 0, st>>>(B, NH, NF, m->X, NF, 1, W1, NH, 1, m->P + OFF_B1,
                                                               m->H1, NH, nullptr, 0);
    gemm_bf16<EPI_RELU_BF16><<<gemm_grid(B, NH), 128, 0, st>>>(B, NH, NH, m->H1, NH, 1, W2, NH, 1, m->P + OFF_B2,
                                                               m->H2, NH, nullptr, 0);
    head_fwd<<<(B * 32 + 127) / 128, 128, 0, st>>>(m->H2, B, m->P, m->out);
    MC(cudaGetLastError());
    return KN_OK;
}

}  // namespace

extern "C" {

kn_status kn_mlp_create(kn_mlp** out) {
    if (!out) return noalloc_fail(KN_ERR_INVALID_ARG, "kn_mlp_create: NULL argument");
    kn_mlp* m = new kn_mlp();
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&m->P, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->G, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->Am, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->Av, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->Wb, sizeof(bf16) * (NF * NH + NH * NH));
    if (e == cudaSuccess) e = cudaMalloc(&m->norm, sizeof(float) * 2 * NF);
    if (e == cudaSuccess) e = cudaMemset(m->P, 0, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMemset(m->G, 0, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMemset(m->Am, 0, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMemset(m->Av, 0, sizeof(float) * kMlpParams);
    if (e == cudaSuccess) e = cudaMemset(m->Wb, 0, sizeof(bf16) * (NF * NH + NH * NH));
    if (e == cudaSuccess) {
        std::vector<float> nm(2 * NF, 0.f);
        for (int k = 0; k < NF; ++k) nm[NF + k] = 1.f;
        e = cudaMemcpy(m->norm, nm.data(), sizeof(float) * 2 * NF, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        kn_mlp_destroy(m);
        return cuda_fail(e);
    }
    *out = m;
    return KN_OK;
}

kn_status kn_mlp_destroy(kn_mlp* m) {
    if (!m) return KN_OK;
    cudaDeviceSynchronize();
    for (void* p : {(void*)m->P, (void*)m->G, (void*)m->Am, (void*)m->Av, (void*)m->Wb, (void*)m->norm,
                    (void*)m->X, (void*)m->H1, (void*)m->H2, (void*)m->dZ2, (void*)m->dZ1, (void*)m->out,
                    (void*)m->dout})
        if (p) cudaFree(p);
    delete m;
    return KN_OK;
}

kn_status kn_mlp_set_params(kn_mlp* m, const float* params, const float* mu, const float* sigma) {
    if (!m || !params || !mu || !sigma) return noalloc_fail(KN_ERR_INVALID_ARG, "kn_mlp_set_params: NULL argument");
    std::vector<float> nm(2 * NF);
    for (int k = 0; k < NF; ++k) {
        if (!(std::isfinite(sigma[k]) && sigma[k] > 0 && std::isfinite(mu[k])))
            return noalloc_fail(KN_ERR_INVALID_ARG, "kn_mlp_set_params: need finite mu and sigma > 0");
        nm[k] = mu[k];
        nm[NF + k] = 1.f / sigma[k];
    }
    for (int i = 0; i < kMlpParams; ++i)
        if (!std::isfinite(params[i])) return noalloc_fail(KN_ERR_INVALID_ARG, "kn_mlp_set_params: non-finite parameter");
    MC(cudaMemcpy(m->P, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice));
    MC(cudaMemcpy(m->norm, nm.data(), sizeof(float) * 2 * NF, cudaMemcpyHostToDevice));
    MC(cudaMemset(m->Am, 0, sizeof(float) * kMlpParams));
    MC(cudaMemset(m->Av, 0, sizeof(float) * kMlpParams));
    to_bf16<<<(NF * NH + NH * NH + 255) / 256, 256>>>(m->P, m->Wb);
    MC(cudaGetLastError());
    MC(cudaDeviceSynchronize());
    m->step = 0;
    return KN_OK;
}

kn_status kn_mlp_get_params(const kn_mlp* m, float* params, float* grads) {
    if (!m) return noalloc_fail(KN_ERR_INVALID_ARG, "kn_mlp_get_params: NULL handle");
    MC(cudaDeviceSynchronize());
    if (params) MC(cudaMemcpy(params, m->P, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
    if (grads) MC(cudaMemcpy(grads, m->G, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
    return KN_OK;
}

kn_status kn_mlp_forward(kn_mlp* m, const float* feat, int32_t B, float* out, void* stream) {
    if (!m || !feat || !out || B < 1) return noalloc_fail(KN_ERR_INVALID_ARG, "kn_mlp_forward: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    kn_status s = forward(m, feat, B, st);
    if (s != KN_OK) return s;
    MC(cudaMemcpyAsync(out, m->out, sizeof(float) * B, cudaMemcpyDeviceToDevice, st));
    return KN_OK;
}

kn_status kn_mlp_backward(kn_mlp* m, const float* feat, const float* y, int32_t B, float* loss, void* stream) {
    if (!m || !feat || !y || B < 1) return noalloc_fail(KN_ERR_INVALID_ARG, "kn_mlp_backward: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    kn_status s = forward(m, feat, B, st);
    if (s != KN_OK) return s;
    if (loss) mse<<<1, 256, 0, st>>>(m->out, y, B, loss);
    head_bwd<<<(B * NH + 255) / 256, 256, 0, st>>>(m->out, y, B, m->H2, m->P, m->dout, m->dZ2);
    const bf16* W2 = m->Wb + NF * NH;
    // dW2 = H1^T dZ2
    gemm_bf16<EPI_F32><<<gemm_grid(NH, NH), 128, 0, st>>>(NH, NH, B, m->H1, 1, NH, m->dZ2, NH, 1, nullptr,
                                                          m->G + OFF_W2, NH, nullptr, 0);
    // dZ1 = (dZ2 W2^T) * [H1 > 0]
    gemm_bf16<EPI_MASK_BF16><<<gemm_grid(B, NH), 128, 0, st>>>(B, NH, NH, m->dZ2, NH, 1, W2, 1, NH, nullptr, m->dZ1,
                                                               NH, m->H1, NH);
    // dW1 = X^T dZ1
    gemm_bf16<EPI_F32><<<gemm_grid(NF, NH), 128, 0, st>>>(NF, NH, B, m->X, 1, NF, m->dZ1, NH, 1, nullptr,
                                                          m->G + OFF_W1, NH, nullptr, 0);
    col_sums<<<1, 160, 0, st>>>(m->dZ1, m->dZ2, m->H2, m->dout, B, m->G);
    MC(cudaGetLastError());
    return KN_OK;
}

kn_status kn_mlp_adam(kn_mlp* m, float lr, float beta1, float beta2, float eps, void* stream) {
    if (!m || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps >= 0))
        return noalloc_fail(KN_ERR_INVALID_ARG, "kn_mlp_adam: bad arguments");
    m->step += 1;
    const float c1 = 1.f - powf(beta1, (float)m->step), c2 = 1.f - powf(beta2, (float)m->step);
    adam<<<(kMlpParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(m->P, m->G, m->Am, m->Av, m->Wb, lr, beta1,
                                                                      beta2, eps, c1, c2);
    MC(cudaGetLastError());
    return KN_OK;
}

}  // extern "C"

namespace kn {
// device pointers the integrator reads when it stages the network for inference
void mlp_device_view(const void* h, const float** P, const void** Wb, const float** norm) {
    const kn_mlp* m = (const kn_mlp*)h;
    *P = m->P;
    *Wb = m->Wb;
    *norm = m->norm;
}
}  // namespace kn
