// Surrogate inference layers on the 5th-generation tensor cores (tcgen05).
//
// One hidden layer is Out[M x 256] = bf16(gelu(A[M x K] W^T + b)) with BF16
// A and W, FP32 accumulation in tensor memory (TMEM) and FP32 bias / GELU in
// the epilogue: the same rounding points as the mma.sync layers, a different
// FP32 summation order inside the products.
//
// Layout.  Activations and weights live in global memory in the layout the
// MMA reads from shared memory (K-major, no swizzle): a matrix with R rows is
// cut into 128-row tiles (256 for the weights) and 64-column chunks; a (tile,
// chunk) block is contiguous and holds 8 x 8 "core matrices" of 128 bytes,
// core (row group g, column group c) at (g * 8 + c) * 128 bytes, element
// (r, e) of a core at (r * 8 + e) * 2 bytes.  So one bulk copy moves a block
// into shared memory, and the smem matrix descriptor uses a leading (K) byte
// offset of 128 and a stride (row group) byte offset of 1024.
//
// Kernel.  Persistent, one CTA per SM, warp-specialised:
//   warp 0     bulk-copy producer: the layer's weights once, then the A blocks
//              of the CTA's tiles through a 4-stage ring (mbarrier full/empty);
//   warp 1     allocates 512 TMEM columns (two 128 x 256 FP32 accumulators)
//              and one thread issues tcgen05.mma (M 128, N 256, K 16), commits
//              to free each A stage and to publish each finished accumulator;
//   warps 2-17 epilogue: tcgen05.ld of their TMEM lane quadrant and column quarter,
//              bias + GELU + BF16, 16-byte stores in the tiled layout; the
//              accumulator is released to the MMA thread for the tile after next.
// Every mbarrier wait is bounded; on expiry the kernel records an error,
// stops issuing work, drains what it started and frees TMEM.
#include <cuda_bf16.h>

#include <cstdint>

#include "trk_internal.cuh"

namespace trk {
namespace {

constexpr int UM = 128, UN = 256, KCH = 64;
constexpr int kStages = 4;
constexpr int kEpiWarps = 16;                       // 4 per TMEM lane quadrant
constexpr int kUmmaThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kABlockBytes = UM * KCH * 2;  // 16 KB
constexpr uint32_t kWBlockBytes = UN * KCH * 2;  // 32 KB
constexpr uint32_t kSpin = 1u << 20;               // try_wait polls before a wait is abandoned

struct UmmaShared {
    uint64_t w_full, full[kStages], empty[kStages], acc_full[2], acc_empty[2], drain;
    uint32_t tmem_base;
    int abort;
    float bias[UN];
};

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, volatile int *abort) {
    for (uint32_t it = 0; it < kSpin; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(su32(b)), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 1023u) == 1023u && *abort) return false;
    }
    *abort = 1;
    return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

// Shared-memory matrix descriptor: K-major, no swizzle, leading byte offset 128
// (next 8-column group), stride byte offset 1024 (next 8-row group).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(1024u >> 4) << 32) |
           (1ull << 46);
}
// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, N 256, M 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(UN >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ float gelu_u(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__global__ void __launch_bounds__(kUmmaThreads, 1)
    k_umma_layer(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ W,
                 const float *__restrict__ bias, int K, int64_t n_tiles, __nv_bfloat16 *__restrict__ Out,
                 int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned carve-up: weights, then the A ring, then the control block
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int kc = K / KCH;
    unsigned char *sW = base;
    unsigned char *sA = sW + (size_t)kc * kWBlockBytes;
    UmmaShared &S = *reinterpret_cast<UmmaShared *>(sA + kStages * kABlockBytes);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        mbar_init(&S.w_full, 1);
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&S.acc_full[b], 1);
            mbar_init(&S.acc_empty[b], kEpiWarps);
        }
        mbar_init(&S.drain, 1);
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < UN; i += blockDim.x) S.bias[i] = bias[i];
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(&S.tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = S.tmem_base;
    volatile int *abort = &S.abort;

    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(&S.w_full, (uint32_t)kc * kWBlockBytes);
            for (int c = 0; c < kc; ++c)
                bulk_g2s(sW + (size_t)c * kWBlockBytes, W + (size_t)c * (kWBlockBytes / 2), kWBlockBytes, &S.w_full);
            uint32_t it = 0;
            for (int64_t t = blockIdx.x; t < n_tiles && !*abort; t += gridDim.x) {
                for (int c = 0; c < kc; ++c, ++it) {
                    const uint32_t s = it % kStages, ph = (it / kStages) & 1u;
                    if (!mbar_wait(&S.empty[s], ph ^ 1u, abort)) break;
                    mbar_expect_tx(&S.full[s], kABlockBytes);
                    bulk_g2s(sA + (size_t)s * kABlockBytes, A + ((size_t)t * kc + c) * (kABlockBytes / 2), kABlockBytes,
                             &S.full[s]);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t it = 0, j = 0;
            bool ok = mbar_wait(&S.w_full, 0, abort);
            for (int64_t t = blockIdx.x; ok && t < n_tiles; t += gridDim.x, ++j) {
                const uint32_t b = j & 1u, aph = (j >> 1) & 1u;
                if (!(ok = mbar_wait(&S.acc_empty[b], aph ^ 1u, abort))) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + b * UN;
                for (int c = 0; c < kc; ++c, ++it) {
                    const uint32_t s = it % kStages, ph = (it / kStages) & 1u;
                    if (!(ok = mbar_wait(&S.full[s], ph, abort))) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = su32(sA + (size_t)s * kABlockBytes), w0 = su32(sW + (size_t)c * kWBlockBytes);
#pragma unroll
                    for (int kk = 0; kk < KCH / 16; ++kk)
                        umma(d, sdesc(a0 + kk * 256), sdesc(w0 + kk * 256), (c | kk) != 0);
                    umma_commit(&S.empty[s]);   // frees the stage once these MMAs have read it
                }
                if (!ok) break;
                umma_commit(&S.acc_full[b]);    // accumulator b complete
            }
            // drain: a last commit arrives once every MMA issued above is done
            umma_commit(&S.drain);
            mbar_wait(&S.drain, 0, abort);
        }
    } else {
        constexpr int kCols = UN / (kEpiWarps / 4);   // columns per epilogue warp
        const int q = warp & 3, part = (warp - 2) >> 2;
        const int row = q * 32 + lane;   // TMEM lane = row of the tile
        uint32_t j = 0;
        for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++j) {
            const uint32_t b = j & 1u, ph = (j >> 1) & 1u;
            if (!mbar_wait(&S.acc_full[b], ph, abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            __nv_bfloat16 *orow = Out + ((size_t)t * 4 * 16 * 8 * 64) + (size_t)(row >> 3) * 8 * 64 + (row & 7) * 8;
#pragma unroll 1
            for (int c0 = part * kCols; c0 < part * kCols + kCols; c0 += 32) {
                uint32_t r[32];
                const uint32_t ta = tmem + b * UN + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                      "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                      "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    const int n0 = c0 + g * 8;   // 8 output columns = one 16-byte piece
                    uint4 v;
                    uint32_t *pv = reinterpret_cast<uint32_t *>(&v);
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        pv[e] = pack_bf16(gelu_u(__uint_as_float(r[g * 8 + 2 * e]) + S.bias[n0 + 2 * e]),
                                          gelu_u(__uint_as_float(r[g * 8 + 2 * e + 1]) + S.bias[n0 + 2 * e + 1]));
                    // output column n0 lies in chunk n0 / 64, column group (n0 % 64) / 8
                    *reinterpret_cast<uint4 *>(orow + (size_t)(n0 >> 6) * 16 * 8 * 64 + ((n0 & 63) >> 3) * 64) = v;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&S.acc_empty[b]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
    }
    if (threadIdx.x == 0 && S.abort) atomicExch(err, 1);
}

// Row-major [rows][K] (K a multiple of 64) -> tiled blocks of `tile_rows` rows.
__global__ void k_to_tiled(const __nv_bfloat16 *__restrict__ src, int64_t rows, int K, int tile_rows,
                           __nv_bfloat16 *__restrict__ dst) {
    const int kc = K / KCH;
    const int64_t pieces = rows * (K / 8);   // 16-byte pieces
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pieces; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = p / (K / 8);
        const int cg = (int)(p % (K / 8));   // 8-column group over the whole row
        const int64_t t = r / tile_rows;
        const int rr = (int)(r % tile_rows), c = cg >> 3, kg = cg & 7;
        const size_t off = (((size_t)t * kc + c) * (tile_rows / 8) + (rr >> 3)) * 8 * 64 + (size_t)kg * 64 + (rr & 7) * 8;
        *reinterpret_cast<uint4 *>(dst + off) = *reinterpret_cast<const uint4 *>(src + r * K + cg * 8);
    }
}

// Tiled activations (K = 256, 128-row tiles) -> row-major [rows][256]: the
// inverse of k_to_tiled for rows [0, rows) of an activation buffer.
__global__ void k_from_tiled(const __nv_bfloat16 *__restrict__ src, int64_t rows, __nv_bfloat16 *__restrict__ dst) {
    constexpr int K = UN, kc = K / KCH;
    const int64_t pieces = rows * (K / 8);
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pieces; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = p / (K / 8);
        const int cg = (int)(p % (K / 8));
        const int64_t t = r / UM;
        const int rr = (int)(r % UM), c = cg >> 3, kg = cg & 7;
        const size_t off = (((size_t)t * kc + c) * (UM / 8) + (rr >> 3)) * 8 * 64 + (size_t)kg * 64 + (rr & 7) * 8;
        *reinterpret_cast<uint4 *>(dst + r * K + cg * 8) = *reinterpret_cast<const uint4 *>(src + off);
    }
}

// x [M x 8] FP32 -> h0 tiled (K = 64: one chunk; columns 8..63 zero; rows >= M zero).
__global__ void k_input_tiled(const float *__restrict__ X, int64_t M, int64_t m_pad, __nv_bfloat16 *__restrict__ H0) {
    const int64_t pieces = m_pad * 8;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < pieces; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = p >> 3;
        const int kg = (int)(p & 7);
        uint4 v = make_uint4(0, 0, 0, 0);
        if (kg == 0 && r < M) {
            uint32_t *pv = reinterpret_cast<uint32_t *>(&v);
#pragma unroll
            for (int e = 0; e < 4; ++e) pv[e] = pack_bf16(X[r * 8 + 2 * e], X[r * 8 + 2 * e + 1]);
        }
        const int64_t t = r / UM;
        const int rr = (int)(r % UM);
        *reinterpret_cast<uint4 *>(H0 + ((size_t)t * 16 + (rr >> 3)) * 8 * 64 + (size_t)kg * 64 + (rr & 7) * 8) = v;
    }
}

// logit[m] = h4[m] . w5 + b5 from tiled h4 (K = 256): warp per row, lane l
// takes chunk l / 8, column group l % 8 (8 columns).
__global__ void k_head_tiled(const __nv_bfloat16 *__restrict__ H4, const __nv_bfloat16 *__restrict__ w5,
                             const float *__restrict__ b5, int64_t M, float *__restrict__ logit) {
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= M) return;
    const int c = lane >> 3, kg = lane & 7;
    const int64_t t = r / UM;
    const int rr = (int)(r % UM);
    const uint4 hv = *reinterpret_cast<const uint4 *>(H4 + (((size_t)t * 4 + c) * 16 + (rr >> 3)) * 8 * 64 +
                                                      (size_t)kg * 64 + (rr & 7) * 8);
    const uint4 wv = *reinterpret_cast<const uint4 *>(w5 + lane * 8);
    const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&hv);
    const __nv_bfloat16 *w = reinterpret_cast<const __nv_bfloat16 *>(&wv);
    float s = 0.0f;
#pragma unroll
    for (int e = 0; e < 8; ++e) s += __bfloat162float(h[e]) * __bfloat162float(w[e]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) logit[r] = s + b5[0];
}

int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

size_t umma_layer_smem(int K) {
    return 1024 + (size_t)(K / KCH) * kWBlockBytes + kStages * kABlockBytes + sizeof(UmmaShared);
}

cudaError_t launch_umma_layer(const uint16_t *A_tiled, const uint16_t *W_tiled, const float *bias, int K,
                              int64_t n_tiles, uint16_t *out_tiled, int *d_err, cudaStream_t s) {
    if (K % KCH || K < KCH || K > 256 || n_tiles < 1) return cudaErrorInvalidValue;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = umma_layer_smem(K);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_umma_layer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)(n_tiles < nsm ? n_tiles : nsm);
    k_umma_layer<<<grid, kUmmaThreads, smem, s>>>(reinterpret_cast<const __nv_bfloat16 *>(A_tiled),
                                                  reinterpret_cast<const __nv_bfloat16 *>(W_tiled), bias, K, n_tiles,
                                                  reinterpret_cast<__nv_bfloat16 *>(out_tiled), d_err);
    return cudaGetLastError();
}

cudaError_t launch_to_tiled(const uint16_t *src, int64_t rows, int K, int tile_rows, uint16_t *dst, cudaStream_t s) {
    k_to_tiled<<<grid_for(rows * (K / 8)), 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(src), rows, K,
                                                       tile_rows, reinterpret_cast<__nv_bfloat16 *>(dst));
    return cudaGetLastError();
}

cudaError_t launch_from_tiled(const uint16_t *src, int64_t rows, uint16_t *dst, cudaStream_t s) {
    k_from_tiled<<<grid_for(rows * (UN / 8)), 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(src), rows,
                                                         reinterpret_cast<__nv_bfloat16 *>(dst));
    return cudaGetLastError();
}

cudaError_t launch_input_tiled(const float *X, int64_t M, int64_t m_pad, uint16_t *H0, cudaStream_t s) {
    k_input_tiled<<<grid_for(m_pad * 8), 256, 0, s>>>(X, M, m_pad, reinterpret_cast<__nv_bfloat16 *>(H0));
    return cudaGetLastError();
}

cudaError_t launch_head_tiled(const uint16_t *H4, const uint16_t *w5, const float *b5, int64_t M, float *logit,
                              cudaStream_t s) {
    const int rows_per_block = 8;
    k_head_tiled<<<(unsigned)((M + rows_per_block - 1) / rows_per_block), 32 * rows_per_block, 0, s>>>(
        reinterpret_cast<const __nv_bfloat16 *>(H4), reinterpret_cast<const __nv_bfloat16 *>(w5), b5, M, logit);
    return cudaGetLastError();
}

}  // namespace trk
