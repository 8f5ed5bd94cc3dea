// kn_mlp.cu -- the learned timestep proposal's network: 64 -> 128 -> 128 -> 1
// (ReLU), BF16 weights and activations, FP32 accumulation, FP32 master weights
// trained with Adam (Kingma & Ba).  The paper has no learned component; this
// is the library's addition on top of the Sec. 4 timestep controller.
//
// Training: one kernel per batch does the forward and backward pass of a
// 64-row tile per CTA entirely in shared memory -- weights, inputs, hidden
// activations and their gradients staged in 16-byte padded rows, every GEMM
// on the tensor cores with ldmatrix and mma.sync.m16n8k16 (BF16 operands,
// FP32 accumulation) -- and writes the tile's partial weight gradients; a
// second kernel adds the tiles in a fixed order, then Adam updates the FP32
// master weights.  Per batch of 4096 rows the three GEMM layers hold about
// 0.6 GFLOP spread over 64 CTAs, so the tiles are latency-bound; the fusion
// removes the activations' round trips through global memory and all but
// three launches per step.
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
    // per-tile partial gradients [tiles][kPartStride] and squared errors [tiles], for up to cap_tiles tiles
    int cap_tiles = 0;
    float* part = nullptr;
    float* loss_part = nullptr;
    long long step = 0;
};

namespace {

constexpr int NF = kMlpFeatures, NH = kMlpHidden;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NF * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH;
static_assert(OFF_B3 + 1 == kMlpParams, "parameter layout");

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// ldmatrix: four 8x8 BF16 matrices; lane l gives the row address of matrix l / 8.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], uint32_t addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
// D += A (16x16, row) B (16x8, col), BF16 inputs, FP32 accumulation
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Warp tile of C (16 rows from m0, 8*NT columns from n0) += A B over K, all
// operands BF16 in shared memory with 16-byte padded rows (conflict-free
// ldmatrix).  Operand storage:
//   A_ROW: A is [M][K] (row m holds K values);  else A is stored [K][M].
//   B_ROW: B is [K][N] (row k holds N values);  else B is stored [N][K].
// Lane l addresses row (l & 7) of matrix l >> 3 of each ldmatrix.x4.
template <int NT, bool A_ROW, bool B_ROW>
__device__ __forceinline__ void warp_mma(float (&c)[NT][4], const bf16* A, int lda, int m0, const bf16* B, int ldb,
                                         int n0, int K, int lane) {
    const int r = lane & 7, q = lane >> 3;
    const int lo8 = (q & 1) << 3, hi8 = (q & 2) << 2;  // matrix q: +8 on its first / second index
#pragma unroll 2
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4];
        if (A_ROW)  // matrices (m, k): (0,0) (8,0) (0,8) (8,8)
            ldsm_x4(a, smem_addr(A + (m0 + r + lo8) * lda + k0 + hi8));
        else        // stored [k][m], transposed: (k, m) = (0,0) (0,8) (8,0) (8,8)
            ldsm_x4_t(a, smem_addr(A + (k0 + r + hi8) * lda + m0 + lo8));
#pragma unroll
        for (int j = 0; j < NT; j += 2) {
            uint32_t b[4];
            if (B_ROW)  // stored [k][n], transposed: (k, n) = (0,0) (8,0) (0,8) (8,8)
                ldsm_x4_t(b, smem_addr(B + (k0 + r + lo8) * ldb + n0 + 8 * j + hi8));
            else        // stored [n][k]: (n, k) = (0,0) (0,8) (8,0) (8,8)
                ldsm_x4(b, smem_addr(B + (n0 + 8 * j + r + hi8) * ldb + k0 + lo8));
            mma_bf16(c[j], a, b[0], b[1]);
            mma_bf16(c[j + 1], a, b[2], b[3]);
        }
    }
}

// One CTA per tile of kTileRows rows of the batch: the whole forward pass and,
// with BWD, the backward pass of the mean squared error, every GEMM on the
// tensor cores from shared memory.  Row-tile partial gradients (in the
// parameter layout) and the tile's sum of squared errors go to global memory;
// reduce_partials adds the tiles in a fixed order.
constexpr int kTileRows = 64;
// row stride of the per-tile partial gradients: the parameter count padded to
// 16 bytes, so every tile's row keeps the float2 stores 8-byte aligned
constexpr int kPartStride = (kMlpParams + 3) & ~3;
constexpr int kTileThreads = 256;  // 8 warps
constexpr int LDF = NF + 8, LDN = NH + 8;  // padded row strides (BF16 elements)
constexpr int kTileSmem = (NF * LDN + NH * LDN + kTileRows * LDF + 4 * kTileRows * LDN) * 2 +
                          (3 * NH + 2 * kTileRows + 8 + 2 * kTileThreads / 32) * 4;

template <bool BWD>
__global__ void __launch_bounds__(kTileThreads, 1)
mlp_tile(const float* __restrict__ feat, const float* __restrict__ y, int B, const float* __restrict__ norm,
         const float* __restrict__ P, const bf16* __restrict__ Wb, float* __restrict__ out,
         float* __restrict__ part, float* __restrict__ loss_part) {
    extern __shared__ __align__(128) unsigned char sm[];
    bf16* W1s = (bf16*)sm;                 // [NF][LDN]
    bf16* W2s = W1s + NF * LDN;            // [NH][LDN]
    bf16* Xs = W2s + NH * LDN;             // [rows][LDF]
    bf16* H1s = Xs + kTileRows * LDF;      // [rows][LDN]
    bf16* H2s = H1s + kTileRows * LDN;
    bf16* dZ2s = H2s + kTileRows * LDN;
    bf16* dZ1s = dZ2s + kTileRows * LDN;
    float* b1s = (float*)(dZ1s + kTileRows * LDN);
    float* b2s = b1s + NH;
    float* w3s = b2s + NH;
    float* outs = w3s + NH;                // [rows]
    float* douts = outs + kTileRows;       // [rows]
    float* red = douts + kTileRows;        // [8] + per-warp sums
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int r0 = blockIdx.x * kTileRows;
    const int rows = min(kTileRows, B - r0);

    // stage the BF16 weights, the FP32 biases and the normalised inputs
    for (int i = tid; i < NF * (NH / 8); i += kTileThreads) {
        const int k = i / (NH / 8), c = i - k * (NH / 8);
        *(int4*)(W1s + k * LDN + 8 * c) = *(const int4*)(Wb + k * NH + 8 * c);
    }
    for (int i = tid; i < NH * (NH / 8); i += kTileThreads) {
        const int k = i / (NH / 8), c = i - k * (NH / 8);
        *(int4*)(W2s + k * LDN + 8 * c) = *(const int4*)(Wb + NF * NH + k * NH + 8 * c);
    }
    for (int i = tid; i < NH; i += kTileThreads) {
        b1s[i] = P[OFF_B1 + i];
        b2s[i] = P[OFF_B2 + i];
        w3s[i] = P[OFF_W3 + i];
    }
    for (int i = tid; i < kTileRows * (NF / 4); i += kTileThreads) {
        const int m = i / (NF / 4), c = i - m * (NF / 4);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m < rows) {
            v = *(const float4*)(feat + (size_t)(r0 + m) * NF + 4 * c);
            v.x = (v.x - norm[4 * c]) * norm[NF + 4 * c];
            v.y = (v.y - norm[4 * c + 1]) * norm[NF + 4 * c + 1];
            v.z = (v.z - norm[4 * c + 2]) * norm[NF + 4 * c + 2];
            v.w = (v.w - norm[4 * c + 3]) * norm[NF + 4 * c + 3];
        }
        __nv_bfloat162* d = (__nv_bfloat162*)(Xs + m * LDF + 4 * c);
        d[0] = __floats2bfloat162_rn(v.x, v.y);
        d[1] = __floats2bfloat162_rn(v.z, v.w);
    }
    __syncthreads();

    const int g = lane >> 2, t = lane & 3;
    const int wm = (w & 3) * 16, wn = (w >> 2) * 64;  // 64 x 128 outputs: 4 x 2 warp tiles
    // H = ReLU(A W + b), BF16, for the 64 x 128 warp-tiled outputs
    auto dense_relu = [&](const bf16* A, int lda, const bf16* W, int K, const float* bias, bf16* H) {
        float c[8][4] = {};
        warp_mma<8, true, true>(c, A, lda, wm, W, LDN, wn, K, lane);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = wn + 8 * j + 2 * t;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float v0 = c[j][2 * h] + bias[n], v1 = c[j][2 * h + 1] + bias[n + 1];
                *(__nv_bfloat162*)(H + (wm + g + 8 * h) * LDN + n) =
                    __floats2bfloat162_rn(v0 > 0.f ? v0 : 0.f, v1 > 0.f ? v1 : 0.f);
            }
        }
    };
    dense_relu(Xs, LDF, W1s, NF, b1s, H1s);
    __syncthreads();
    dense_relu(H1s, LDN, W2s, NH, b2s, H2s);
    __syncthreads();
    // out = H2 w3 + b3 (FP32), 8 rows per warp
    const float b3 = P[OFF_B3];
    float se = 0.f;
    for (int m = w * (kTileRows / 8); m < (w + 1) * (kTileRows / 8); ++m) {
        float s = 0.f;
        for (int n = lane; n < NH; n += 32) s = fmaf(__bfloat162float(H2s[m * LDN + n]), w3s[n], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float o_m = s + b3;
        if (lane == 0) {
            if (!BWD) {
                if (m < rows) out[r0 + m] = o_m;
            } else {
                const float e = m < rows ? o_m - y[r0 + m] : 0.f;
                outs[m] = o_m;
                douts[m] = 2.f * e / (float)B;
                se = fmaf(e, e, se);
            }
        }
    }
    if (!BWD) return;
    if (lane == 0) red[w] = se;
    __syncthreads();
    if (tid == 0) {
        float l = 0.f;
        for (int i = 0; i < kTileThreads / 32; ++i) l += red[i];
        loss_part[blockIdx.x] = l;
    }
    // dZ2 = dout w3 [H2 > 0]  (BF16)
    for (int i = tid; i < kTileRows * NH; i += kTileThreads) {
        const int m = i / NH, n = i - m * NH;
        const float keep = __bfloat162float(H2s[m * LDN + n]) > 0.f ? 1.f : 0.f;
        dZ2s[m * LDN + n] = __float2bfloat16(douts[m] * w3s[n] * keep);
    }
    __syncthreads();
    // dZ1 = (dZ2 W2^T) [H1 > 0]  (W2 stored [k][n] is W2^T stored [n][k])
    {
        float c[8][4] = {};
        warp_mma<8, true, false>(c, dZ2s, LDN, wm, W2s, LDN, wn, NH, lane);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = wn + 8 * j + 2 * t;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = wm + g + 8 * h;
                const float k0 = __bfloat162float(H1s[m * LDN + n]) > 0.f ? 1.f : 0.f;
                const float k1 = __bfloat162float(H1s[m * LDN + n + 1]) > 0.f ? 1.f : 0.f;
                *(__nv_bfloat162*)(dZ1s + m * LDN + n) = __floats2bfloat162_rn(c[j][2 * h] * k0, c[j][2 * h + 1] * k1);
            }
        }
    }
    __syncthreads();
    float* G = part + (size_t)blockIdx.x * kPartStride;
    // dW1 = X^T dZ1 (64 x 128, K = tile rows): 4 x 2 warp tiles
    {
        float c[8][4] = {};
        warp_mma<8, false, true>(c, Xs, LDF, wm, dZ1s, LDN, wn, kTileRows, lane);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int n = wn + 8 * j + 2 * t;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                *(float2*)(G + OFF_W1 + (wm + g + 8 * h) * NH + n) = make_float2(c[j][2 * h], c[j][2 * h + 1]);
        }
    }
    // dW2 = H1^T dZ2 (128 x 128, K = tile rows): warp w takes rows 16 w
    {
        float c[16][4] = {};
        warp_mma<16, false, true>(c, H1s, LDN, 16 * w, dZ2s, LDN, 0, kTileRows, lane);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int n = 8 * j + 2 * t;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                *(float2*)(G + OFF_W2 + (16 * w + g + 8 * h) * NH + n) = make_float2(c[j][2 * h], c[j][2 * h + 1]);
        }
    }
    // column sums: b1 = sum dZ1, b2 = sum dZ2, w3 = sum H2 dout, b3 = sum dout
    if (tid < NH) {
        float s1 = 0.f, s3 = 0.f;
        for (int m = 0; m < rows; ++m) {
            s1 += __bfloat162float(dZ1s[m * LDN + tid]);
            s3 = fmaf(__bfloat162float(H2s[m * LDN + tid]), douts[m], s3);
        }
        G[OFF_B1 + tid] = s1;
        G[OFF_W3 + tid] = s3;
    } else {
        const int n = tid - NH;
        float s2 = 0.f, s4 = 0.f;
        for (int m = 0; m < rows; ++m) {
            s2 += __bfloat162float(dZ2s[m * LDN + n]);
            s4 += douts[m];
        }
        G[OFF_B2 + n] = s2;
        if (n == 0) G[OFF_B3] = s4;
    }
}

// Gradients = the tiles' partials added in tile order; loss = their squared errors / B.
__global__ void reduce_partials(const float* __restrict__ part, int T, float* __restrict__ G,
                                const float* __restrict__ loss_part, float* __restrict__ loss, float inv_B) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kMlpParams) {
        float s = 0.f;
        for (int i = 0; i < T; ++i) s += part[(size_t)i * kPartStride + p];
        G[p] = s;
    }
    if (loss && p == 0) {
        float l = 0.f;
        for (int i = 0; i < T; ++i) l += loss_part[i];
        *loss = l * inv_B;
    }
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
    const int T = (B + kTileRows - 1) / kTileRows;
    if (T <= m->cap_tiles) return KN_OK;
    cudaFree(m->part);
    cudaFree(m->loss_part);
    m->part = m->loss_part = nullptr;
    m->cap_tiles = 0;
    MC(cudaMalloc(&m->part, sizeof(float) * (size_t)T * kPartStride));
    MC(cudaMalloc(&m->loss_part, sizeof(float) * (size_t)T));
    m->cap_tiles = T;
    return KN_OK;
}

static kn_status tile_smem_limit() {
    static bool done = false;
    if (!done) {
        MC(cudaFuncSetAttribute(mlp_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmem));
        MC(cudaFuncSetAttribute(mlp_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmem));
        done = true;
    }
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
                    (void*)m->part, (void*)m->loss_part})
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
    if ((uintptr_t)feat & 15) return noalloc_fail(KN_ERR_INVALID_ARG, "kn_mlp_forward: features must be 16-byte aligned");
    kn_status s = tile_smem_limit();
    if (s != KN_OK) return s;
    const int T = (B + kTileRows - 1) / kTileRows;
    mlp_tile<false><<<T, kTileThreads, kTileSmem, (cudaStream_t)stream>>>(feat, nullptr, B, m->norm, m->P, m->Wb,
                                                                         out, nullptr, nullptr);
    MC(cudaGetLastError());
    return KN_OK;
}

kn_status kn_mlp_backward(kn_mlp* m, const float* feat, const float* y, int32_t B, float* loss, void* stream) {
    if (!m || !feat || !y || B < 1) return noalloc_fail(KN_ERR_INVALID_ARG, "kn_mlp_backward: bad arguments");
    if ((uintptr_t)feat & 15) return noalloc_fail(KN_ERR_INVALID_ARG, "kn_mlp_backward: features must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    kn_status s = tile_smem_limit();
    if (s != KN_OK) return s;
    if ((s = ensure_cap(m, B)) != KN_OK) return s;
    const int T = (B + kTileRows - 1) / kTileRows;
    mlp_tile<true><<<T, kTileThreads, kTileSmem, st>>>(feat, y, B, m->norm, m->P, m->Wb, nullptr, m->part,
                                                       m->loss_part);
    reduce_partials<<<(kMlpParams + 255) / 256, 256, 0, st>>>(m->part, T, m->G, m->loss_part, loss, 1.f / (float)B);
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
