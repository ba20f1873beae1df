// MLP surrogate for dynamic-aperture triage: 8 -> 4 x [Linear 256 + GELU] -> 1.
// BF16 weights and activations into tcgen05 tensor-core products (FP32
// accumulation in tensor memory, trk_mlp_umma.cu), FP32 master weights, biases
// and gradients, Adam.  This file holds the network's parameters and buffers,
// the small reductions and the Adam update, and drives the products.
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
// the backward pass's concurrent branches: the head's sums and each layer's
// bias sums (kColSlots column sums in flight), each layer's weight gradient
constexpr int kColSlots = kHidden + 1, kSide = 3, kEvents = 2 * kHidden + 4;

// out[n] = sum_m A[m][n] (* w[m] if w): column sums over N = 256 columns in a
// fixed order, FP32, in one launch: each of kColSlices blocks writes the partial
// sums of its row slice; the last block to finish (a ticket counter, reset for
// the next call) adds the partials in slice order, so the result does not
// depend on which block came last.
constexpr int kColSlices = 64;
constexpr size_t kColSlot = kColSlices * kW + 4;   // partials and the ticket of one column sum
__global__ void k_colsum(const float *__restrict__ A, const __nv_bfloat16 *__restrict__ Ab,
                         const float *__restrict__ w, int64_t M, float *part, unsigned *ticket,
                         float *__restrict__ out) {
    __shared__ bool last;
    pdl_wait();
    pdl_trigger();
    const int n = threadIdx.x;  // blockDim.x == kW
    const int64_t per = (M + kColSlices - 1) / kColSlices;
    const int64_t m0 = blockIdx.x * per, m1 = m0 + per < M ? m0 + per : M;
    // the rows are added one after another in row order; the loads of 16 rows
    // are issued before their adds so that they are in flight together
    float s = 0.0f;
    int64_t m = m0;
    if (A) {
        for (; m + 16 <= m1; m += 16) {
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = A[(m + q) * kW + n];
#pragma unroll
            for (int q = 0; q < 16; ++q) s += v[q];
        }
        for (; m < m1; ++m) s += A[m * kW + n];
    } else {
        for (; m + 16 <= m1; m += 16) {
            float v[16], ww[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                v[q] = __bfloat162float(Ab[(m + q) * kW + n]);
                ww[q] = w ? w[m + q] : 1.0f;
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) s += w ? v[q] * ww[q] : v[q];
        }
        for (; m < m1; ++m) {
            const float a = __bfloat162float(Ab[m * kW + n]);
            s += w ? a * w[m] : a;
        }
    }
    part[blockIdx.x * kW + n] = s;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    float t = 0.0f;
    for (int j = 0; j < kColSlices; j += 16) {
        float pv[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) pv[q] = __ldcg(part + (j + q) * kW + n);
#pragma unroll
        for (int q = 0; q < 16; ++q) t += pv[q];
    }
    out[n] = t;
    if (threadIdx.x == 0) *ticket = 0u;
}

// out[b] = scale[b] * sum_i a_b[i] for the two arrays b = blockIdx.x (one block each).
__global__ void k_sum2(const float *__restrict__ a0, const float *__restrict__ a1, int64_t n, float scale0,
                       float scale1, float *__restrict__ out0, float *__restrict__ out1) {
    __shared__ float sh[256];
    pdl_wait();
    pdl_trigger();
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
__global__ void k_reduce_splits(const float *__restrict__ part, int splits, int64_t n, float *__restrict__ out) {
    pdl_wait();
    pdl_trigger();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        // up to 16 slices' loads in flight, added in slice order
        float a = 0.0f;
        for (int z0 = 0; z0 < splits; z0 += 16) {
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = z0 + q < splits ? part[(int64_t)(z0 + q) * n + i] : 0.0f;
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (z0 + q < splits) a = (z0 + q == 0) ? v[q] : a + v[q];
        }
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
    float *loss = nullptr;                                         // mean loss of the last gradient
    float *part = nullptr;                                         // column-sum partials, then the ticket
    uint16_t *wt = nullptr;                                        // BF16 weights of layers 0..3, tcgen05 tiled layout
    size_t wt_off[kHidden] = {};
    uint16_t *act[2] = {nullptr, nullptr};                         // tiled activations for inference (ping-pong)
    int64_t act_rows = 0;
    int *d_err = nullptr;                                          // device error flag of the tcgen05 layers
    int64_t t = 0;                                                 // Adam step
    // training on tcgen05: activations tiled (A of the products) and
    // transposed-tiled (B of the weight gradients), pre-activations, the
    // gradient chain, the transposed weight tiles and the split partials
    int64_t tc_cap = 0;
    uint16_t *Ht[kHidden + 1] = {}, *HT[kHidden + 1] = {}, *H4rm = nullptr;
    // the gradient chain keeps one set per layer (dz FP32, its BF16 copy tiled
    // and transposed-tiled, the weight-gradient split partials), so that each
    // layer's weight and bias gradients run beside the next input gradient
    float *Zt[kHidden] = {}, *tlogit = nullptr, *tdl = nullptr, *tloss_terms = nullptr;
    float *tdz[kHidden] = {}, *tpart[kHidden] = {};
    uint16_t *dzbt[kHidden] = {}, *dzbT[kHidden] = {};
    cudaStream_t side[kSide] = {};  // the branches' streams (joined back before the step ends)
    cudaEvent_t ev[kEvents] = {};
    unsigned *tickets = nullptr;   // [9]: the Adam step's block counter (zero between launches)
    uint16_t *wtT = nullptr;
    size_t wtT_off[kHidden] = {};
};

static trk_status mlp_fail(trk_status s, const std::string &m) { return set_error(s, m); }

// The column sums' ticket counter, kept after the partials (zero between calls).
// Column sums run concurrently, each with its own slot of partials and ticket.
static float *col_part(trk_mlp *N, int slot) { return N->part + (size_t)slot * kColSlot; }
static unsigned *col_ticket(trk_mlp *N, int slot) {
    return reinterpret_cast<unsigned *>(col_part(N, slot) + kColSlices * kW);
}

static void mlp_free_tc(trk_mlp *N) {
    for (int l = 0; l <= kHidden; ++l) {
        cudaFree(N->Ht[l]);
        cudaFree(N->HT[l]);
        N->Ht[l] = N->HT[l] = nullptr;
    }
    for (int l = 0; l < kHidden; ++l) {
        cudaFree(N->Zt[l]);
        N->Zt[l] = nullptr;
    }
    for (int l = 0; l < kHidden; ++l) {
        cudaFree(N->tdz[l]);
        cudaFree(N->tpart[l]);
        cudaFree(N->dzbt[l]);
        cudaFree(N->dzbT[l]);
        N->tdz[l] = N->tpart[l] = nullptr;
        N->dzbt[l] = N->dzbT[l] = nullptr;
    }
    cudaFree(N->H4rm);
    cudaFree(N->tlogit);
    cudaFree(N->tdl);
    cudaFree(N->tloss_terms);
    cudaFree(N->tickets);
    N->H4rm = nullptr;
    N->tlogit = N->tdl = N->tloss_terms = nullptr;
    N->tickets = nullptr;
    N->tc_cap = 0;
}

// Buffers of the tcgen05 training step for up to `rows` rows (a multiple of 128).
static trk_status mlp_ensure_tc(trk_mlp *N, int64_t rows) {
    if (rows <= N->tc_cap) return TRK_OK;
    mlp_free_tc(N);
    cudaError_t e = cudaSuccess;
    const size_t r = (size_t)rows;
    for (int l = 0; l <= kHidden && e == cudaSuccess; ++l) {
        const size_t k = l == 0 ? kInPad : kW;
        e = cudaMalloc(&N->Ht[l], r * k * sizeof(uint16_t));
        if (e == cudaSuccess) e = cudaMalloc(&N->HT[l], r * k * sizeof(uint16_t));
    }
    for (int l = 0; l < kHidden && e == cudaSuccess; ++l) e = cudaMalloc(&N->Zt[l], r * kW * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N->H4rm, r * kW * sizeof(uint16_t));
    for (int l = 0; l < kHidden && e == cudaSuccess; ++l) {
        e = cudaMalloc(&N->tdz[l], r * kW * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&N->dzbt[l], r * kW * sizeof(uint16_t));
        if (e == cudaSuccess) e = cudaMalloc(&N->dzbT[l], r * kW * sizeof(uint16_t));
        if (e == cudaSuccess)
            e = cudaMalloc(&N->tpart[l], (size_t)train_dw_splits(rows) * kW * N->in_pad[l] * sizeof(float));
    }
    if (e == cudaSuccess) e = cudaMalloc(&N->tlogit, r * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N->tdl, r * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N->tloss_terms, r * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&N->tickets, 16 * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(N->tickets, 0, 16 * sizeof(unsigned));
    if (e != cudaSuccess) {
        mlp_free_tc(N);
        return mlp_fail(TRK_ENOMEM, "trk_mlp: training buffer allocation failed");
    }
    N->tc_cap = rows;
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
    if (e == cudaSuccess) e = cudaMalloc(&N->part, kColSlots * kColSlot * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(N->part, 0, kColSlots * kColSlot * sizeof(float));
    for (int k = 0; k < kSide && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&N->side[k], cudaStreamNonBlocking);
    for (int k = 0; k < kEvents && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&N->ev[k], cudaEventDisableTiming);
    {
        size_t o = 0;
        for (int l = 0; l < kHidden; ++l) {
            N->wt_off[l] = o;
            o += (size_t)kW * N->in_pad[l];
        }
        if (e == cudaSuccess) e = cudaMalloc(&N->wt, o * sizeof(uint16_t));
        size_t ot = 0;
        for (int l = 1; l < kHidden; ++l) {
            N->wtT_off[l] = ot;
            ot += (size_t)kW * kW;
        }
        if (e == cudaSuccess) e = cudaMalloc(&N->wtT, ot * sizeof(uint16_t));
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
        cudaFree(N->wt);
        cudaFree(N->wtT);
        cudaFree(N->d_err);
        for (int k = 0; k < kSide; ++k)
            if (N->side[k]) cudaStreamDestroy(N->side[k]);
        for (int k = 0; k < kEvents; ++k)
            if (N->ev[k]) cudaEventDestroy(N->ev[k]);
        delete N;
        return mlp_fail(TRK_ENOMEM, std::string("trk_mlp_create: ") + cudaGetErrorString(e));
    }
    *out = N;
    return TRK_OK;
}

extern "C" trk_status trk_mlp_destroy(trk_mlp *N) {
    if (!N) return TRK_OK;
    cudaDeviceSynchronize();
    cudaFree(N->p);
    cudaFree(N->m);
    cudaFree(N->v);
    cudaFree(N->g);
    cudaFree(N->pb);
    cudaFree(N->loss);
    cudaFree(N->part);
    cudaFree(N->wt);
    cudaFree(N->wtT);
    cudaFree(N->d_err);
    cudaFree(N->act[0]);
    cudaFree(N->act[1]);
    mlp_free_tc(N);
    for (int k = 0; k < kSide; ++k)
        if (N->side[k]) cudaStreamDestroy(N->side[k]);
    for (int k = 0; k < kEvents; ++k)
        if (N->ev[k]) cudaEventDestroy(N->ev[k]);
    delete N;
    return TRK_OK;
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

// The tiled weight copies (wt for the forward products, wtT = W^T for the
// input gradients) from the BF16 weights.
static cudaError_t mlp_retile(trk_mlp *N, cudaStream_t s) {
    const uint16_t *pb = reinterpret_cast<const uint16_t *>(N->pb);
    const int in_pad[kHidden] = {N->in_pad[0], N->in_pad[1], N->in_pad[2], N->in_pad[3]};
    return launch_retile_weights(pb, N->w_off, N->wt_off, N->wtT_off, in_pad, N->wt, N->wtT, s);
}

// Gradients of the mean BCE over M rows into N->g and the loss into N->loss,
// every product on tcgen05 (the tiled weights must be current: mlp_retile).
// Rounding points (the file header's): h0 = bf16(x), z FP32, h = bf16(gelu(z)),
// dz FP32, dzb = bf16(dz), dW = dzb^T h and dh = dzb W in FP32, db = sum dz.
struct GatherRows {
    const int32_t *perm = nullptr;
    int64_t n = 0, batch = 0, spe = 1;
    const int64_t *step = nullptr;   // NULL: rows [0, M) of X and y as given
    const float *y_all = nullptr;
};

// With sums_in_adam the first layer's weight gradient stays as split partials
// (N->tpart[0]) for the Adam step to sum: its product is the last of the
// backward pass, so its sum would otherwise be one more launch before Adam.
static cudaError_t mlp_grad_tc(trk_mlp *N, const float *X, const float *y, int64_t M, cudaStream_t s,
                               const GatherRows &gr = GatherRows(), bool sums_in_adam = false) {
    const int64_t m_pad = (M + 127) / 128 * 128;
    const uint16_t *pb = reinterpret_cast<const uint16_t *>(N->pb);
    // with a gather, y is the batch's label buffer that the input kernel fills
    cudaError_t e = launch_train_input(X, M, m_pad, N->Ht[0], N->HT[0], gr.perm, gr.n, gr.batch, gr.spe, gr.step,
                                       gr.y_all, const_cast<float *>(y), s);
    for (int l = 0; l < kHidden && e == cudaSuccess; ++l)
        e = launch_train_fwd(N->Ht[l], N->in_pad[l], N->wt + N->wt_off[l], N->p + N->b_off[l], m_pad, N->Zt[l],
                             N->Ht[l + 1], N->HT[l + 1], l == kHidden - 1 ? N->H4rm : nullptr, N->d_err, s);
    if (e == cudaSuccess)
        e = launch_train_head(N->Ht[kHidden], pb + N->w_off[4], N->p + N->b_off[4], y, M, m_pad, N->Zt[kHidden - 1],
                              N->tlogit, N->tdl, N->tdz[kHidden - 1], N->dzbt[kHidden - 1], N->dzbT[kHidden - 1],
                              N->tloss_terms, s);
    // The backward pass as a fork-join: the main stream runs the input
    // gradients dx_3, dx_2, dx_1 (each writing its own layer's buffers); as soon
    // as layer l's dz exists, side streams take its weight gradient (split
    // products, then their sum in split order) and its bias column sums.  Each
    // result has one writer and a fixed summation order, so the gradients are
    // the same as in one stream.  Everything joins the main stream at the end.
    int ev = 0;
    auto fork = [&](cudaStream_t to) {
        if (e == cudaSuccess) e = cudaEventRecord(N->ev[ev], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(to, N->ev[ev], 0);
        ++ev;
    };
    cudaStream_t cs = N->side[0];   // column sums (head, then every layer's bias)
    fork(cs);
    if (e == cudaSuccess) {
        e = pdl_launch(k_colsum, dim3(kColSlices), dim3(kW), 0, cs, (const float *)nullptr,
                       reinterpret_cast<const __nv_bfloat16 *>(N->H4rm), (const float *)N->tdl, M,
                       col_part(N, kHidden), col_ticket(N, kHidden), N->g + N->w_off[4]);
        if (e == cudaSuccess)
            e = pdl_launch(k_sum2, dim3(2), dim3(256), 0, cs, (const float *)N->tdl, (const float *)N->tloss_terms, M,
                           1.0f, 1.0f / (float)M, N->g + N->b_off[4], N->loss);
    }
    for (int l = kHidden - 1; l >= 0 && e == cudaSuccess; --l) {
        const int K = N->in_pad[l];
        // layer l's weight gradient on a side stream (layer 0's on the main
        // stream, which has nothing else left); the fork's event marks dz_l as
        // written, and the column-sum stream waits for it as well
        cudaStream_t ws = l > 0 ? N->side[1 + (l & 1)] : s;
        fork(l > 0 ? ws : cs);
        if (l > 0 && e == cudaSuccess) e = cudaStreamWaitEvent(cs, N->ev[ev - 1], 0);
        if (e != cudaSuccess) break;
        e = launch_train_dw(N->dzbT[l], N->HT[l], K, m_pad, N->tpart[l], N->d_err, ws);
        if (e != cudaSuccess) break;
        if (!(sums_in_adam && l == 0))
            e = pdl_launch(k_reduce_splits, dim3(grid_for((int64_t)kW * K)), dim3(256), 0, ws,
                           (const float *)N->tpart[l], train_dw_splits(m_pad), (int64_t)kW * K, N->g + N->w_off[l]);
        if (e == cudaSuccess)
            e = pdl_launch(k_colsum, dim3(kColSlices), dim3(kW), 0, cs, (const float *)N->tdz[l],
                           (const __nv_bfloat16 *)nullptr, (const float *)nullptr, M, col_part(N, l),
                           col_ticket(N, l), N->g + N->b_off[l]);
        if (e != cudaSuccess) break;
        if (l > 0)
            e = launch_train_dx(N->dzbt[l], N->wtT + N->wtT_off[l], N->Zt[l - 1], m_pad, N->tdz[l - 1],
                                N->dzbt[l - 1], N->dzbT[l - 1], N->d_err, s);
    }
    // join: the main stream waits for every side stream
    for (int k = 0; k < kSide; ++k) {
        if (e == cudaSuccess) e = cudaEventRecord(N->ev[ev], N->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, N->ev[ev], 0);
        ++ev;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

extern "C" trk_status trk_mlp_grad(trk_mlp *N, const float *d_X, const float *d_y, int32_t M, float *d_loss,
                                   void *stream) {
    if (!N || M < 1 || !d_X || !d_y) return mlp_fail(TRK_EINVAL, "trk_mlp_grad: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t m_pad = ((int64_t)M + 127) / 128 * 128;
    trk_status st = mlp_ensure_tc(N, m_pad);
    if (st != TRK_OK) return st;
    cudaError_t e = mlp_retile(N, s);
    if (e == cudaSuccess) e = mlp_grad_tc(N, d_X, d_y, M, s);
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
// One training step on m rows, enqueued on s (captured into a graph).
cudaError_t train_step(trk_mlp *N, const float *d_X, const float *d_y, const int32_t *d_perm, int64_t n,
                       int64_t batch, int64_t spe, int64_t m, float lr, const float *c12, int64_t *dstep,
                       float *yb, float *d_loss_hist, cudaStream_t s) {
    GatherRows gr;
    gr.perm = d_perm;
    gr.n = n;
    gr.batch = batch;
    gr.spe = spe;
    gr.step = dstep;
    gr.y_all = d_y;
    cudaError_t e = mlp_grad_tc(N, d_X, yb, m, s, gr, true);
    if (e != cudaSuccess) return e;
    // Adam, the tiled weight copies for the next step and the step counter in one launch
    size_t w_end[kHidden];
    for (int l = 0; l < kHidden; ++l) w_end[l] = N->b_off[l];
    const int in_pad[kHidden] = {N->in_pad[0], N->in_pad[1], N->in_pad[2], N->in_pad[3]};
    const float *first_part[kHidden] = {N->tpart[0], nullptr, nullptr, nullptr};
    e = launch_adam_step(N->p, N->m, N->v, N->g, reinterpret_cast<uint16_t *>(N->pb), (int64_t)N->n_par, lr, c12, dstep,
                         N->loss, d_loss_hist, N->tickets + 9, N->w_off, w_end, N->wt_off, N->wtT_off, in_pad, N->wt,
                         N->wtT, first_part, train_dw_splits((m + 127) / 128 * 128), s);
    return e;
}

struct TrainRes {
    float *yb = nullptr, *c12 = nullptr;
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
    const int64_t m_pad = (b + 127) / 128 * 128;
    trk_status st = mlp_ensure_tc(N, m_pad);
    if (st != TRK_OK) return st;
    TrainRes R;
    std::vector<float> c12(2 * total);
    for (int64_t k = 0; k < total; ++k) {
        const float t = (float)(N->t + k + 1);
        c12[2 * k] = 1.0f - powf(0.9f, t);
        c12[2 * k + 1] = 1.0f - powf(0.999f, t);
    }
    cudaError_t e = cudaMalloc(&R.yb, (size_t)b * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&R.c12, c12.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&R.dstep, sizeof(int64_t));
    if (e != cudaSuccess) return mlp_fail(TRK_ENOMEM, "trk_mlp_train: allocation failed");
    e = cudaStreamCreateWithFlags(&R.ps, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R.ev, cudaEventDisableTiming);
    // order the private stream after the caller's work
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.c12, c12.data(), c12.size() * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(R.dstep, 0, sizeof(int64_t), s);
    if (e == cudaSuccess) e = mlp_retile(N, s);   // the first step's products read the current weights
    if (e == cudaSuccess) e = cudaEventRecord(R.ev, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(R.ps, R.ev, 0);
    const int n_graphs = tail == b ? 1 : 2;
    for (int k = 0; k < n_graphs && e == cudaSuccess; ++k) {
        e = cudaStreamBeginCapture(R.ps, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        cudaError_t ec = train_step(N, d_X, d_y, d_perm, n, b, spe, k == 0 ? b : tail, lr, R.c12, R.dstep,
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
    int herr = 0;
    if (cudaMemcpy(&herr, N->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return mlp_fail(TRK_ECUDA, "trk_mlp_train: error flag read failed");
    if (herr) {
        cudaMemset(N->d_err, 0, sizeof(int));
        return mlp_fail(TRK_ETIMEOUT, "trk_mlp_train: a tensor-core product gave up waiting on a barrier");
    }
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
