// MLP surrogate for dynamic-aperture triage: 8 -> 4 x [Linear 256 + GELU] -> 1.
// BF16 weights and activations into tensor-core products (mma.sync m16n8k16,
// FP32 accumulation), FP32 master weights, biases and gradients, Adam.
//
// Rounding points (kept identical to the oracle's):
//   h0 = bf16(x); z_l = h_{l-1} W_l^T + b_l (FP32); h_l = bf16(gelu(z_l))
//   logit = h4 . w5 + b5;  dlogit = (sigmoid(logit) - y)/M
//   dz_4 = (dlogit w5) * gelu'(z_4); dzb = bf16(dz)
//   dW_l = dzb_l^T h_{l-1}; db_l = sum_m dz_l; dz_{l-1} = (dzb_l W_l) * gelu'(z_{l-1})
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "trk_internal.cuh"

namespace trk {
namespace {

constexpr int kIn = 8, kInPad = 64, kW = 256, kHidden = 4;  // inputs padded to one 64-wide tile
constexpr int BM = 64, BN = 64, BK = 32, SK = BK + 8;  // smem row stride (bf16), padded against bank conflicts

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

enum { EPI_F32 = 0, EPI_GELU = 1, EPI_GELU_STOREZ = 2, EPI_DGELU = 3 };

// C[M x N] = A[M x K] * B[K x N].
//   A_T = false: A[m][k] = A[m * lda + k];  A_T = true: A[m][k] = A[k * lda + m]
//   B_NK = true: B[k][n] = B[n * ldb + k];  B_NK = false: B[k][n] = B[k * ldb + n]
// Epilogues: EPI_F32 stores acc (FP32, ldc); EPI_GELU stores bf16(gelu(acc + bias));
// EPI_GELU_STOREZ also stores z = acc + bias (FP32); EPI_DGELU multiplies acc by
// gelu'(aux[m][n]) and stores the product (FP32 and BF16).
// Split-K: block z sums k in [z * k_split, min(K, (z + 1) * k_split)) and stores
// its FP32 partial at Cf + z * c_split (EPI_F32 only; the caller reduces).
// M, N multiples of 64, K and k_split multiples of 32, lda, ldb multiples of 8
// and A, B 16-byte aligned (the caller pads): tiles move as 16-byte vectors.
template <bool A_T, bool B_NK, int EPI>
__global__ void __launch_bounds__(128) k_gemm(const __nv_bfloat16 *__restrict__ A, int lda,
                                              const __nv_bfloat16 *__restrict__ B, int ldb, int K,
                                              float *__restrict__ Cf, int ldc, __nv_bfloat16 *__restrict__ Cb,
                                              const float *__restrict__ bias, const float *__restrict__ aux,
                                              int k_split, size_t c_split) {
    // two shared-memory stages: the next tile's global loads are in flight in
    // registers while the current tile's MMAs run, then land in the other stage
    __shared__ __align__(16) __nv_bfloat16 sA[2][BM * SK];
    __shared__ __align__(16) __nv_bfloat16 sB[2][BN * SK];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, tg = lane & 3;
    const int kbeg = blockIdx.z * k_split, kend = kbeg + k_split < K ? kbeg + k_split : K;
    if (EPI == EPI_F32) Cf += blockIdx.z * c_split;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;

    // A tile BM x BK and B tile (stored n-major, sB[n][k]) BN x BK: 256 16-byte
    // vectors each, two per thread.
    uint4 ra[2], rb[2];
    const auto load = [&](int k0) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = tid + q * 128;
            if (!A_T) {
                const int m = e >> 2, k = (e & 3) * 8;
                ra[q] = *reinterpret_cast<const uint4 *>(&A[(size_t)(m0 + m) * lda + (k0 + k)]);
            } else {
                const int k = e >> 3, m = (e & 7) * 8;
                ra[q] = *reinterpret_cast<const uint4 *>(&A[(size_t)(k0 + k) * lda + (m0 + m)]);
            }
            if (B_NK) {
                const int n = e >> 2, k = (e & 3) * 8;
                rb[q] = *reinterpret_cast<const uint4 *>(&B[(size_t)(n0 + n) * ldb + (k0 + k)]);
            } else {
                const int k = e >> 3, n = (e & 7) * 8;
                rb[q] = *reinterpret_cast<const uint4 *>(&B[(size_t)(k0 + k) * ldb + (n0 + n)]);
            }
        }
    };
    const auto store = [&](int st) {
        __nv_bfloat16 *a = sA[st], *b = sB[st];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = tid + q * 128;
            if (!A_T) {
                const int m = e >> 2, k = (e & 3) * 8;
                *reinterpret_cast<uint4 *>(&a[m * SK + k]) = ra[q];
            } else {
                const int k = e >> 3, m = (e & 7) * 8;
                const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&ra[q]);
#pragma unroll
                for (int i = 0; i < 8; ++i) a[(m + i) * SK + k] = h[i];
            }
            if (B_NK) {
                const int n = e >> 2, k = (e & 3) * 8;
                *reinterpret_cast<uint4 *>(&b[n * SK + k]) = rb[q];
            } else {
                const int k = e >> 3, n = (e & 7) * 8;
                const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&rb[q]);
#pragma unroll
                for (int i = 0; i < 8; ++i) b[(n + i) * SK + k] = h[i];
            }
        }
    };
    int st = 0;
    if (kbeg < kend) {
        load(kbeg);
        store(0);
    }
    __syncthreads();
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        const bool more = k0 + BK < kend;
        if (more) load(k0 + BK);
        const __nv_bfloat16 *a = sA[st], *b = sB[st];
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + g, c = kk + tg * 2;
                af[i][0] = *reinterpret_cast<const uint32_t *>(&a[r * SK + c]);
                af[i][1] = *reinterpret_cast<const uint32_t *>(&a[(r + 8) * SK + c]);
                af[i][2] = *reinterpret_cast<const uint32_t *>(&a[r * SK + c + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t *>(&a[(r + 8) * SK + c + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = wn + j * 8 + g, c = kk + tg * 2;
                bf[j][0] = *reinterpret_cast<const uint32_t *>(&b[n * SK + c]);
                bf[j][1] = *reinterpret_cast<const uint32_t *>(&b[n * SK + c + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                        : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bf[j][0]),
                          "r"(bf[j][1]));
        }
        // the other stage was last read before the previous barrier
        if (more) store(st ^ 1);
        __syncthreads();
        st ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int row = m0 + wm + i * 16 + g + (r >= 2 ? 8 : 0);
                const int col = n0 + wn + j * 8 + tg * 2 + (r & 1);
                const size_t o = (size_t)row * ldc + col;
                float v = acc[i][j][r];
                if (EPI == EPI_F32) {
                    Cf[o] = v;
                } else if (EPI == EPI_GELU || EPI == EPI_GELU_STOREZ) {
                    v += bias[col];
                    if (EPI == EPI_GELU_STOREZ) Cf[o] = v;
                    Cb[o] = __float2bfloat16_rn(gelu_f(v));
                } else {  // EPI_DGELU
                    v *= gelu_grad_f(aux[o]);
                    Cf[o] = v;
                    Cb[o] = __float2bfloat16_rn(v);
                }
            }
}

// x [M x 8] FP32 -> h0 [M x 64] BF16 (zero padded)
__global__ void k_input(const float *__restrict__ X, int64_t M, int64_t m_pad, __nv_bfloat16 *__restrict__ H0) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad * kInPad;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i / kInPad;
        const int k = (int)(i % kInPad);
        const float v = (m < M && k < kIn) ? X[m * kIn + k] : 0.0f;
        H0[i] = __float2bfloat16_rn(v);
    }
}

// logit[m] = h4[m] . w5 + b5 (warp per row)
__global__ void k_head(const __nv_bfloat16 *__restrict__ H4, const __nv_bfloat16 *__restrict__ w5, const float *b5,
                       int64_t M, float *__restrict__ logit) {
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= M) return;
    float s = 0.0f;
#pragma unroll
    for (int k = lane; k < kW; k += 32) s += __bfloat162float(H4[row * kW + k]) * __bfloat162float(w5[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) logit[row] = s + b5[0];
}

// dlogit = (sigmoid - y)/M, loss terms; dz4 = (dlogit w5) * gelu'(z4) for valid rows
__global__ void k_head_back(const float *__restrict__ logit, const float *__restrict__ y, int64_t M, int64_t m_pad,
                            const __nv_bfloat16 *__restrict__ w5, const float *__restrict__ Z4, float *__restrict__ dl,
                            float *__restrict__ dz, __nv_bfloat16 *__restrict__ dzb, float *__restrict__ loss_terms) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad * kW;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i / kW;
        const int k = (int)(i % kW);
        float d = 0.0f;
        if (m < M) {
            const float l = logit[m];
            d = (1.0f / (1.0f + expf(-l)) - y[m]) / (float)M;
            if (k == 0) {
                dl[m] = d;
                loss_terms[m] = fmaxf(l, 0.0f) + log1pf(expf(-fabsf(l))) - y[m] * l;
            }
        }
        const float v = d * __bfloat162float(w5[k]) * gelu_grad_f(Z4[i]);
        dz[i] = m < M ? v : 0.0f;
        dzb[i] = __float2bfloat16_rn(m < M ? v : 0.0f);
    }
}

// out[n] = sum_m A[m][n] (* w[m] if w): column sums over N = 256 columns in a
// fixed order, FP32, in one launch: each of kColSlices blocks writes the partial
// sums of its row slice; the last block to finish (a ticket counter, reset for
// the next call) adds the partials in slice order, so the result does not
// depend on which block came last.
constexpr int kColSlices = 64;
__global__ void k_colsum(const float *__restrict__ A, const __nv_bfloat16 *__restrict__ Ab,
                         const float *__restrict__ w, int64_t M, float *part, unsigned *ticket,
                         float *__restrict__ out) {
    __shared__ bool last;
    const int n = threadIdx.x;  // blockDim.x == kW
    const int64_t per = (M + kColSlices - 1) / kColSlices;
    const int64_t m0 = blockIdx.x * per, m1 = m0 + per < M ? m0 + per : M;
    float s = 0.0f;
    for (int64_t m = m0; m < m1; ++m) {
        const float a = A ? A[m * kW + n] : __bfloat162float(Ab[m * kW + n]);
        s += w ? a * w[m] : a;
    }
    part[blockIdx.x * kW + n] = s;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    float t = 0.0f;
    for (int j = 0; j < kColSlices; ++j) t += __ldcg(part + j * kW + n);
    out[n] = t;
    if (threadIdx.x == 0) *ticket = 0u;
}

// out[b] = scale[b] * sum_i a_b[i] for the two arrays b = blockIdx.x (one block each).
__global__ void k_sum2(const float *__restrict__ a0, const float *__restrict__ a1, int64_t n, float scale0,
                       float scale1, float *__restrict__ out0, float *__restrict__ out1) {
    __shared__ float sh[256];
    const float *a = blockIdx.x ? a1 : a0;
    float s = 0.0f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += a[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *(blockIdx.x ? out1 : out0) = sh[0] * (blockIdx.x ? scale1 : scale0);
}

// out[i] = sum over slices s = 0, 1, ... of part[s * n + i], in slice order.
constexpr int kSplits = 16;
__global__ void k_reduce_splits(const float *__restrict__ part, int splits, int64_t n, float *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float a = part[i];
        for (int z = 1; z < splits; ++z) a += part[z * n + i];
        out[i] = a;
    }
}

// Adam on FP32 master weights; writes the BF16 copy.  The bias corrections
// c1 = 1 - beta1^t, c2 = 1 - beta2^t come as values, or (c12 != NULL) from the
// table c12[2 * step], c12[2 * step + 1] at the device step counter.
__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v, const float *__restrict__ g,
                       __nv_bfloat16 *__restrict__ pb, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2, const float *__restrict__ c12, const int64_t *__restrict__ step) {
    if (c12) {
        c1 = c12[2 * *step];
        c2 = c12[2 * *step + 1];
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = w;
        if (pb) pb[i] = __float2bfloat16_rn(w);
    }
}

__global__ void k_to_bf16(const float *__restrict__ a, __nv_bfloat16 *__restrict__ b, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace
}  // namespace trk

using namespace trk;

namespace {
thread_local std::string g_mlp_err;
}

// Parameter blocks: layer l has W [out x in_pad] and b [out]; in_pad = 64 for the
// first layer (inputs padded with zeros), 256 otherwise; the head is [1 x 256].
struct trk_mlp {
    int in_pad[5], out[5];
    size_t w_off[5], b_off[5], n_par;  // offsets into the flat FP32 parameter arrays
    float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;  // master, Adam, gradients
    __nv_bfloat16 *pb = nullptr;                                   // BF16 copy of p
    int64_t cap = 0;                                               // rows of the activation buffers
    __nv_bfloat16 *H[kHidden + 1] = {};                            // h0 .. h4
    float *Z[kHidden] = {};                                        // z1 .. z4
    float *dz = nullptr;                                           // FP32 dz of the current layer
    __nv_bfloat16 *dzb = nullptr, *dzb2 = nullptr;
    float *logit = nullptr, *dl = nullptr, *loss_terms = nullptr, *loss = nullptr;
    float *part = nullptr;                                         // column-sum partials, then the ticket
    float *splitk = nullptr;                                       // split-K partials of dW [kSplits][256][256]
    uint16_t *wt = nullptr;                                        // BF16 weights of layers 0..3, tcgen05 tiled layout
    size_t wt_off[kHidden] = {};
    uint16_t *act[2] = {nullptr, nullptr};                         // tiled activations for inference (ping-pong)
    int64_t act_rows = 0;
    int *d_err = nullptr;                                          // device error flag of the tcgen05 layers
    int64_t t = 0;                                                 // Adam step
};

static trk_status mlp_fail(trk_status s, const std::string &m) { return set_error(s, m); }

// The column sums' ticket counter, kept after the partials (zero between calls).
static unsigned *col_ticket(trk_mlp *N) { return reinterpret_cast<unsigned *>(N->part + kColSlices * kW); }

static void mlp_free_acts(trk_mlp *N) {
    for (auto &h : N->H) {
        cudaFree(h);
        h = nullptr;
    }
    for (auto &z : N->Z) {
        cudaFree(z);
        z = nullptr;
    }
    cudaFree(N->dz);
    cudaFree(N->dzb);
    cudaFree(N->dzb2);
    cudaFree(N->logit);
    cudaFree(N->dl);
    cudaFree(N->loss_terms);
    N->dz = nullptr;
    N->dzb = N->dzb2 = nullptr;
    N->logit = N->dl = N->loss_terms = nullptr;
    N->cap = 0;
}

static trk_status mlp_ensure(trk_mlp *N, int64_t rows, bool training) {
    if (rows <= N->cap && (!training || N->Z[0])) return TRK_OK;
    mlp_free_acts(N);
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&N->H[0], rows * kInPad * sizeof(__nv_bfloat16));
    for (int l = 1; l <= kHidden && e == cudaSuccess; ++l) e = cudaMalloc(&N->H[l], rows * kW * sizeof(__nv_bfloat16));
    if (training)
        for (int l = 0; l < kHidden && e == cudaSuccess; ++l) e = cudaMalloc(&N->Z[l], rows * kW * sizeof(float));
    if (e == cudaSuccess && training) e = cudaMalloc(&N->dz, rows * kW * sizeof(float));
    if (e == cudaSuccess && training) e = cudaMalloc(&N->dzb, rows * kW * sizeof(__nv_bfloat16));
    if (e == cudaSuccess && training) e = cudaMalloc(&N->dzb2, rows * kW * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&N->logit, rows * sizeof(float));
    if (e == cudaSuccess && training) e = cudaMalloc(&N->dl, rows * sizeof(float));
    if (e == cudaSuccess && training) e = cudaMalloc(&N->loss_terms, rows * sizeof(float));
    if (e != cudaSuccess) {
        mlp_free_acts(N);
        return mlp_fail(TRK_ENOMEM, "trk_mlp: activation allocation failed");
    }
    N->cap = rows;
    return TRK_OK;
}

extern "C" trk_status trk_mlp_create(const float *const *host_W, const float *const *host_b, trk_mlp **out) {
    if (!out || !host_W || !host_b) return mlp_fail(TRK_EINVAL, "trk_mlp_create: NULL argument");
    *out = nullptr;
    auto *N = new trk_mlp();
    const int in_true[5] = {kIn, kW, kW, kW, kW};
    size_t off = 0;
    for (int l = 0; l < 5; ++l) {
        N->in_pad[l] = l == 0 ? kInPad : kW;
        N->out[l] = l == 4 ? 1 : kW;
        N->w_off[l] = off;
        off += (size_t)N->out[l] * N->in_pad[l];
        N->b_off[l] = off;
        off += N->out[l];
        if (!host_W[l] || !host_b[l]) {
            delete N;
            return mlp_fail(TRK_EINVAL, "trk_mlp_create: NULL weight array");
        }
    }
    N->n_par = off;
    std::vector<float> h(off, 0.0f);
    for (int l = 0; l < 5; ++l) {
        for (int o = 0; o < N->out[l]; ++o)
            for (int i = 0; i < in_true[l]; ++i) h[N->w_off[l] + (size_t)o * N->in_pad[l] + i] = host_W[l][o * in_true[l] + i];
        for (int o = 0; o < N->out[l]; ++o) h[N->b_off[l] + o] = host_b[l][o];
    }
    cudaError_t e = cudaMalloc(&N->p, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N->m, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N->v, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N->g, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N->pb, off * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&N->loss, sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N->part, (kColSlices * kW + 4) * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(N->part + kColSlices * kW, 0, 4 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N->splitk, (size_t)kSplits * kW * kW * sizeof(float));
    {
        size_t o = 0;
        for (int l = 0; l < kHidden; ++l) {
            N->wt_off[l] = o;
            o += (size_t)kW * N->in_pad[l];
        }
        if (e == cudaSuccess) e = cudaMalloc(&N->wt, o * sizeof(uint16_t));
    }
    if (e == cudaSuccess) e = cudaMalloc(&N->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(N->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(N->p, h.data(), off * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(N->m, 0, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(N->v, 0, off * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(N->g, 0, off * sizeof(float));
    if (e == cudaSuccess) {
        k_to_bf16<<<grid_for(off), 256>>>(N->p, N->pb, off);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        cudaFree(N->p);
        cudaFree(N->m);
        cudaFree(N->v);
        cudaFree(N->g);
        cudaFree(N->pb);
        cudaFree(N->loss);
        cudaFree(N->part);
        cudaFree(N->splitk);
        cudaFree(N->wt);
        cudaFree(N->d_err);
        delete N;
        return mlp_fail(TRK_ENOMEM, std::string("trk_mlp_create: ") + cudaGetErrorString(e));
    }
    *out = N;
    return TRK_OK;
}

extern "C" trk_status trk_mlp_destroy(trk_mlp *N) {
    if (!N) return TRK_OK;
    cudaDeviceSynchronize();
    mlp_free_acts(N);
    cudaFree(N->p);
    cudaFree(N->m);
    cudaFree(N->v);
    cudaFree(N->g);
    cudaFree(N->pb);
    cudaFree(N->loss);
    cudaFree(N->part);
    cudaFree(N->splitk);
    cudaFree(N->wt);
    cudaFree(N->d_err);
    cudaFree(N->act[0]);
    cudaFree(N->act[1]);
    delete N;
    return TRK_OK;
}

// Forward over rows [0, m_pad) of the buffers (m_pad a multiple of 64).
static cudaError_t mlp_forward_rows(trk_mlp *N, const float *X, int64_t M, int64_t m_pad, bool training,
                                    cudaStream_t s) {
    k_input<<<grid_for(m_pad * kInPad), 256, 0, s>>>(X, M, m_pad, N->H[0]);
    for (int l = 0; l < kHidden; ++l) {
        const int K = N->in_pad[l];
        const dim3 grid(kW / BN, (unsigned)(m_pad / BM));
        const __nv_bfloat16 *W = N->pb + N->w_off[l];
        const float *b = N->p + N->b_off[l];
        if (training)
            k_gemm<false, true, EPI_GELU_STOREZ><<<grid, 128, 0, s>>>(N->H[l], K, W, K, K, N->Z[l], kW, N->H[l + 1],
                                                                      b, nullptr, K, 0);
        else
            k_gemm<false, true, EPI_GELU><<<grid, 128, 0, s>>>(N->H[l], K, W, K, K, nullptr, kW, N->H[l + 1], b,
                                                               nullptr, K, 0);
    }
    const int rows_per_block = 8;
    k_head<<<(unsigned)((M + rows_per_block - 1) / rows_per_block), 32 * rows_per_block, 0, s>>>(
        N->H[kHidden], N->pb + N->w_off[4], N->p + N->b_off[4], M, N->logit);
    return cudaGetLastError();
}

// Inference on the tcgen05 layers: inputs and activations in the tiled layout
// of trk_mlp_umma.cu, 2^18-row chunks (a multiple of the 128-row tile).  With
// d_hidden, each hidden layer's BF16 output of rows [r0, r0 + m) is also copied
// out row-major to d_hidden + (l * M + r0) * 256.
extern "C" trk_status trk_mlp_forward_hidden(trk_mlp *N, const float *d_X, int64_t M, float *d_logits,
                                             uint16_t *d_hidden, void *stream) {
    if (!N || M < 0 || (M > 0 && (!d_X || !d_logits))) return mlp_fail(TRK_EINVAL, "trk_mlp_forward: bad argument");
    if (M == 0) return TRK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t chunk = 1 << 18;
    const int64_t rows = M < chunk ? (M + 127) / 128 * 128 : chunk;
    cudaError_t e = cudaSuccess;
    if (rows > N->act_rows) {
        cudaFree(N->act[0]);
        cudaFree(N->act[1]);
        N->act[0] = N->act[1] = nullptr;
        N->act_rows = 0;
        e = cudaMalloc(&N->act[0], (size_t)rows * kW * sizeof(uint16_t));
        if (e == cudaSuccess) e = cudaMalloc(&N->act[1], (size_t)rows * kW * sizeof(uint16_t));
        if (e != cudaSuccess) return mlp_fail(TRK_ENOMEM, "trk_mlp_forward: activation allocation failed");
        N->act_rows = rows;
    }
    const uint16_t *pb = reinterpret_cast<const uint16_t *>(N->pb);
    for (int l = 0; l < kHidden && e == cudaSuccess; ++l)
        e = launch_to_tiled(pb + N->w_off[l], kW, N->in_pad[l], kW, N->wt + N->wt_off[l], s);
    for (int64_t r0 = 0; r0 < M && e == cudaSuccess; r0 += chunk) {
        const int64_t m = M - r0 < chunk ? M - r0 : chunk;
        const int64_t m_pad = (m + 127) / 128 * 128;
        e = launch_input_tiled(d_X + r0 * kIn, m, m_pad, N->act[0], s);
        int cur = 0;
        for (int l = 0; l < kHidden && e == cudaSuccess; ++l, cur ^= 1) {
            e = launch_umma_layer(N->act[cur], N->wt + N->wt_off[l], N->p + N->b_off[l], N->in_pad[l], m_pad / 128,
                                  N->act[cur ^ 1], N->d_err, s);
            if (e == cudaSuccess && d_hidden)
                e = launch_from_tiled(N->act[cur ^ 1], m, d_hidden + ((size_t)l * M + r0) * kW, s);
        }
        if (e == cudaSuccess) e = launch_head_tiled(N->act[cur], pb + N->w_off[4], N->p + N->b_off[4], m, d_logits + r0, s);
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, N->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return mlp_fail(TRK_ECUDA, std::string("trk_mlp_forward: ") + cudaGetErrorString(e));
    if (herr) {
        cudaMemsetAsync(N->d_err, 0, sizeof(int), s);
        return mlp_fail(TRK_ETIMEOUT, "trk_mlp_forward: a tensor-core layer gave up waiting on a barrier");
    }
    return TRK_OK;
}

extern "C" trk_status trk_mlp_forward(trk_mlp *N, const float *d_X, int64_t M, float *d_logits, void *stream) {
    return trk_mlp_forward_hidden(N, d_X, M, d_logits, nullptr, stream);
}

// Gradients of the mean BCE over M rows into N->g; loss into N->loss.
static cudaError_t mlp_grad_rows(trk_mlp *N, const float *X, const float *y, int64_t M, cudaStream_t s) {
    const int64_t m_pad = (M + BM - 1) / BM * BM;
    cudaError_t e = mlp_forward_rows(N, X, M, m_pad, true, s);
    if (e != cudaSuccess) return e;
    // head backward: dlogit, dz4 (rows beyond M are zero)
    k_head_back<<<grid_for(m_pad * kW), 256, 0, s>>>(N->logit, y, M, m_pad, N->pb + N->w_off[4], N->Z[kHidden - 1],
                                                    N->dl, N->dz, N->dzb, N->loss_terms);
    k_colsum<<<kColSlices, kW, 0, s>>>(nullptr, N->H[kHidden], N->dl, M, N->part, col_ticket(N),
                                       N->g + N->w_off[4]);
    k_sum2<<<2, 256, 0, s>>>(N->dl, N->loss_terms, M, 1.0f, 1.0f / (float)M, N->g + N->b_off[4], N->loss);
    // dW reduces over the rows: split them into at most kSplits slices of
    // k_split rows, one block column each, then sum the partials in slice order.
    int splits = (int)(m_pad / 256) < kSplits ? (int)(m_pad / 256) : kSplits;
    if (splits < 1) splits = 1;
    const int k_split = (int)(((m_pad + splits - 1) / splits + BK - 1) / BK * BK);
    splits = (int)((m_pad + k_split - 1) / k_split);
    __nv_bfloat16 *dzb = N->dzb, *dzb_next = N->dzb2;
    for (int l = kHidden - 1; l >= 0; --l) {
        const int K = N->in_pad[l];
        // dW_l [256 x K] = dzb^T [256 x m_pad] * h_{l} [m_pad x K]   (A transposed, B k-major rows)
        k_gemm<true, false, EPI_F32><<<dim3((K + BN - 1) / BN, kW / BM, splits), 128, 0, s>>>(
            dzb, kW, N->H[l], K, (int)m_pad, N->splitk, K, nullptr, nullptr, nullptr, k_split, (size_t)kW * K);
        k_reduce_splits<<<grid_for((int64_t)kW * K), 256, 0, s>>>(N->splitk, splits, (int64_t)kW * K,
                                                                  N->g + N->w_off[l]);
        // db_l = sum_m dz (FP32)
        k_colsum<<<kColSlices, kW, 0, s>>>(N->dz, nullptr, nullptr, M, N->part, col_ticket(N), N->g + N->b_off[l]);
        if (l > 0) {
            // dz_{l-1} = (dzb W_l) * gelu'(z_{l-1}), W_l [256 x 256] as B[k = out][n = in]
            k_gemm<false, false, EPI_DGELU><<<dim3(kW / BN, (unsigned)(m_pad / BM)), 128, 0, s>>>(
                dzb, kW, N->pb + N->w_off[l], kW, kW, N->dz, kW, dzb_next, nullptr, N->Z[l - 1], kW, 0);
            __nv_bfloat16 *t = dzb;
            dzb = dzb_next;
            dzb_next = t;
        }
    }
    return cudaGetLastError();
}

extern "C" trk_status trk_mlp_grad(trk_mlp *N, const float *d_X, const float *d_y, int32_t M, float *d_loss,
                                   void *stream) {
    if (!N || M < 1 || !d_X || !d_y) return mlp_fail(TRK_EINVAL, "trk_mlp_grad: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t m_pad = ((int64_t)M + BM - 1) / BM * BM;
    trk_status st = mlp_ensure(N, m_pad, true);
    if (st != TRK_OK) return st;
    cudaError_t e = mlp_grad_rows(N, d_X, d_y, M, s);
    if (e == cudaSuccess && d_loss) e = cudaMemcpyAsync(d_loss, N->loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return mlp_fail(TRK_ECUDA, std::string("trk_mlp_grad: ") + cudaGetErrorString(e));
    return TRK_OK;
}

extern "C" trk_status trk_mlp_adam(trk_mlp *N, float lr, float beta1, float beta2, float eps, void *stream) {
    if (!N) return mlp_fail(TRK_EINVAL, "trk_mlp_adam: NULL network");
    N->t += 1;
    const float c1 = 1.0f - powf(beta1, (float)N->t), c2 = 1.0f - powf(beta2, (float)N->t);
    k_adam<<<grid_for(N->n_par), 256, 0, (cudaStream_t)stream>>>(N->p, N->m, N->v, N->g, N->pb, N->n_par, lr, beta1,
                                                                 beta2, eps, c1, c2, nullptr, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mlp_fail(TRK_ECUDA, std::string("trk_mlp_adam: ") + cudaGetErrorString(e));
    return TRK_OK;
}

namespace trk {
namespace {
// Rows of training step *step: epoch e = step / spe, rows [r0, r0 + m) of the
// epoch's order with r0 = (step % spe) * batch; the order is perm[e * n + r]
// (identity without perm).
__global__ void k_gather_rows(const float *__restrict__ X, const float *__restrict__ y, const int32_t *__restrict__ perm,
                              int64_t n, int64_t batch, int64_t spe, const int64_t *__restrict__ step, int64_t m,
                              float *__restrict__ Xo, float *__restrict__ yo) {
    const int64_t st = *step, ep = st / spe, r0 = (st % spe) * batch;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = perm ? (int64_t)perm[ep * n + r0 + i] : r0 + i;
        for (int k = 0; k < kIn; ++k) Xo[i * kIn + k] = X[r * kIn + k];
        yo[i] = y[r];
    }
}

// End of a training step: record the loss, advance the step counter.
__global__ void k_step_end(const float *__restrict__ loss, float *__restrict__ hist, int64_t *__restrict__ step) {
    if (hist) hist[*step] = *loss;
    *step += 1;
}

// One training step on m rows, enqueued on s (captured into a graph).
cudaError_t train_step(trk_mlp *N, const float *d_X, const float *d_y, const int32_t *d_perm, int64_t n,
                       int64_t batch, int64_t spe, int64_t m, float lr, const float *c12, int64_t *dstep, float *Xb,
                       float *yb, float *d_loss_hist, cudaStream_t s) {
    k_gather_rows<<<grid_for(m), 256, 0, s>>>(d_X, d_y, d_perm, n, batch, spe, dstep, m, Xb, yb);
    cudaError_t e = mlp_grad_rows(N, Xb, yb, m, s);
    if (e != cudaSuccess) return e;
    k_adam<<<grid_for(N->n_par), 256, 0, s>>>(N->p, N->m, N->v, N->g, N->pb, N->n_par, lr, 0.9f, 0.999f, 1e-8f, 0.0f,
                                              0.0f, c12, dstep);
    k_step_end<<<1, 1, 0, s>>>(N->loss, d_loss_hist, dstep);
    return cudaGetLastError();
}

struct TrainRes {
    float *Xb = nullptr, *yb = nullptr, *c12 = nullptr;
    int64_t *dstep = nullptr;
    cudaStream_t ps = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraph_t g[2] = {};
    cudaGraphExec_t x[2] = {};
    ~TrainRes() {
        for (int i = 0; i < 2; ++i) {
            if (x[i]) cudaGraphExecDestroy(x[i]);
            if (g[i]) cudaGraphDestroy(g[i]);
        }
        if (ps) cudaStreamSynchronize(ps);
        cudaFree(Xb);
        cudaFree(yb);
        cudaFree(c12);
        cudaFree(dstep);
        if (ev) cudaEventDestroy(ev);
        if (ps) cudaStreamDestroy(ps);
    }
};
}  // namespace
}  // namespace trk

// epochs x ceil(n / batch) Adam steps; step k of an epoch takes rows
// [k batch, min(n, (k + 1) batch)) of the epoch's order.  Each step (the full
// one and, when batch does not divide n, the short last one) is captured once
// as a CUDA graph on a private stream; a device step counter selects the rows
// and the Adam bias corrections, so the same graph replays every step.
extern "C" trk_status trk_mlp_train(trk_mlp *N, const float *d_X, const float *d_y, int64_t n, int32_t batch,
                                    int32_t epochs, const int32_t *d_perm, float lr, float *d_loss_hist,
                                    void *stream) {
    if (!N || n < 1 || batch < 1 || epochs < 1 || !d_X || !d_y)
        return mlp_fail(TRK_EINVAL, "trk_mlp_train: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t b = batch < n ? batch : n;
    const int64_t spe = (n + b - 1) / b, total = spe * epochs, tail = n - (spe - 1) * b;
    const int64_t m_pad = (b + BM - 1) / BM * BM;
    trk_status st = mlp_ensure(N, m_pad, true);
    if (st != TRK_OK) return st;
    TrainRes R;
    std::vector<float> c12(2 * total);
    for (int64_t k = 0; k < total; ++k) {
        const float t = (float)(N->t + k + 1);
        c12[2 * k] = 1.0f - powf(0.9f, t);
        c12[2 * k + 1] = 1.0f - powf(0.999f, t);
    }
    cudaError_t e = cudaMalloc(&R.Xb, (size_t)b * kIn * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&R.yb, (size_t)b * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&R.c12, c12.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&R.dstep, sizeof(int64_t));
    if (e != cudaSuccess) return mlp_fail(TRK_ENOMEM, "trk_mlp_train: allocation failed");
    e = cudaStreamCreateWithFlags(&R.ps, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R.ev, cudaEventDisableTiming);
    // order the private stream after the caller's work
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.c12, c12.data(), c12.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(R.dstep, 0, sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaEventRecord(R.ev, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(R.ps, R.ev, 0);
    const int n_graphs = tail == b ? 1 : 2;
    for (int k = 0; k < n_graphs && e == cudaSuccess; ++k) {
        e = cudaStreamBeginCapture(R.ps, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        cudaError_t ec = train_step(N, d_X, d_y, d_perm, n, b, spe, k == 0 ? b : tail, lr, R.c12, R.dstep, R.Xb,
                                    R.yb, d_loss_hist, R.ps);
        e = cudaStreamEndCapture(R.ps, &R.g[k]);
        if (ec != cudaSuccess) e = ec;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&R.x[k], R.g[k], 0);
    }
    for (int64_t k = 0; k < total && e == cudaSuccess; ++k)
        e = cudaGraphLaunch(R.x[(n_graphs == 2 && k % spe == spe - 1) ? 1 : 0], R.ps);
    if (e == cudaSuccess) e = cudaEventRecord(R.ev, R.ps);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, R.ev, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return mlp_fail(TRK_ECUDA, std::string("trk_mlp_train: ") + cudaGetErrorString(e));
    N->t += total;
    return TRK_OK;
}

// Host copies of the FP32 master weights / biases and of the last gradients,
// in the unpadded [out][in] layout.  Any pointer may be NULL.  Synchronises.
extern "C" trk_status trk_mlp_get(trk_mlp *N, float *const *W, float *const *b, float *const *gW, float *const *gb) {
    if (!N) return mlp_fail(TRK_EINVAL, "trk_mlp_get: NULL network");
    if (cudaDeviceSynchronize() != cudaSuccess) return mlp_fail(TRK_ECUDA, "trk_mlp_get: device error");
    std::vector<float> p(N->n_par), g(N->n_par);
    if (cudaMemcpy(p.data(), N->p, N->n_par * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(g.data(), N->g, N->n_par * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return mlp_fail(TRK_ECUDA, "trk_mlp_get: copy failed");
    const int in_true[5] = {kIn, kW, kW, kW, kW};
    for (int l = 0; l < 5; ++l) {
        for (int o = 0; o < N->out[l]; ++o) {
            for (int i = 0; i < in_true[l]; ++i) {
                const size_t src = N->w_off[l] + (size_t)o * N->in_pad[l] + i;
                if (W && W[l]) W[l][o * in_true[l] + i] = p[src];
                if (gW && gW[l]) gW[l][o * in_true[l] + i] = g[src];
            }
            if (b && b[l]) b[l][o] = p[N->b_off[l] + o];
            if (gb && gb[l]) gb[l][o] = g[N->b_off[l] + o];
        }
    }
    return TRK_OK;
}
