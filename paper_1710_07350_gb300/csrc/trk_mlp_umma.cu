// Surrogate inference layers on the 5th-generation tensor cores (tcgen05).
//
// One hidden layer is Out[M x 256] = bf16(gelu(A[M x K] W^T + b)) with BF16
// A and W, FP32 accumulation in tensor memory (TMEM) and FP32 bias / GELU in
// the epilogue: the rounding points of the oracle, with the tensor core's own
// FP32 summation order inside the products.  The training products (forward,
// input and weight gradients) are below, after the inference layer.
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

// ------------------------------------------------------------ training ----
// One 128 x TN output tile per CTA of D = A B^T, A [128 rows x K] and B [TN
// rows x K] both K-major in the tiled layout above: chunk c of A's tile t is
// the 16 KB block ((t * a_kc + c) * 128 * 64) elements in, and the TN-row slice
// j of B's chunk c the contiguous TN * 128 bytes at ((c * b_rows + TN j) * 64)
// (a slice of a block covers TN / 8 whole row groups).  The chunks [k0, k1) are copied
// to shared memory in groups of up to kGroupChunks (one mbarrier each group),
// one thread issues the MMAs (M 128, N TN, K 16) into a TN-column TMEM
// accumulator, and after the last commit eight warps (two per TMEM lane
// quadrant, TN / 2 columns each) read the accumulator and apply the epilogue:
//   kTrainFwd  z = acc + bias -> Z [M][256] FP32; h = bf16(gelu(z)) tiled (next
//              layer's A, 128-row tiles, K 256), transposed-tiled (rows = the
//              256 outputs, K = the batch: the weight gradient's B) and, when
//              Hrm is given, row-major [M][256]
//   kTrainDx   v = acc * gelu'(Zin[m][n]) -> dz FP32 [M][256], bf16(v) tiled and
//              transposed-tiled with 128-row tiles (the next weight gradient's A)
//   kTrainDw   acc -> part [z][256][b_n] FP32 (split z = blockIdx.z of the
//              contraction over the batch; the caller sums the splits in order)
// The forward and input-gradient products use 32-column tiles (256 CTAs for a
// 4096-row batch), the weight gradients 64-column tiles over 8 batch splits.
// Rows m >= M of the batch keep the zeros of padded inputs.
enum { kTrainFwd = 0, kTrainDx = 1, kTrainDw = 2 };
constexpr int kGroupChunks = 8;
// instruction descriptor, kind::f16: D FP32, A and B BF16 K-major, N = n, M 128
__host__ __device__ constexpr uint32_t idesc_n(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(UM >> 4) << 24);
}

struct TrainTileArgs {
    const __nv_bfloat16 *A;
    int64_t a_kc;            // chunks per A tile
    const __nv_bfloat16 *B;
    int b_rows;              // rows of B's tile (256 or 64)
    int kc;                  // chunks of the contraction; a CTA takes [z * cps, min(kc, (z + 1) * cps))
    int cps;
    const float *bias;       // fwd
    const float *Zin;        // dx: pre-activations of the layer below, [M][256]
    float *Zout;             // fwd: [M][256]; dx: dz [M][256]
    __nv_bfloat16 *Ht;       // fwd / dx: tiled output (128-row tiles, K 256)
    __nv_bfloat16 *HtT;      // fwd / dx: transposed-tiled output
    __nv_bfloat16 *Hrm;      // fwd: optional row-major output
    int tt_rows;             // rows of HtT's tiles (256 fwd, 128 dx)
    int64_t m_kc;            // batch chunks (m_pad / 64) of the transposed layouts
    float *part;             // dw: split partials [z][256][b_n], summed in split order by the caller
    int *err;
    int group;               // chunks per shared-memory group: min(cps, kGroupChunks)
};

__device__ __forceinline__ float gelu_grad_u(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Element (r, k) of a matrix in the tiled layout with tr-row tiles and kcn chunks per tile.
__device__ __forceinline__ size_t tiled_at(int64_t r, int64_t k, int tr, int64_t kcn) {
    return ((size_t)((r / tr) * kcn + (k >> 6)) * (tr >> 3) + (size_t)((r % tr) >> 3)) * 512 + (size_t)((k & 63) >> 3) * 64 +
           (size_t)(r & 7) * 8 + (size_t)(k & 7);
}
// The same for tiles of 2^tr_log2 rows given at run time (no integer division).
__device__ __forceinline__ size_t tiled_at_pow2(int64_t r, int64_t k, int tr_log2, int64_t kcn) {
    const int64_t tr = (int64_t)1 << tr_log2;
    return ((size_t)((r >> tr_log2) * kcn + (k >> 6)) * (size_t)(tr >> 3) + (size_t)((r & (tr - 1)) >> 3)) * 512 +
           (size_t)((k & 63) >> 3) * 64 + (size_t)(r & 7) * 8 + (size_t)(k & 7);
}

constexpr int kTrainThreads = 256;   // 8 warps: two per TMEM lane quadrant, 32 output columns each

template <int MODE, int TN>
__global__ void __launch_bounds__(kTrainThreads) k_train_tile(TrainTileArgs a) {
    constexpr uint32_t kBSliceBytes = TN * KCH * 2;
    constexpr int kCols = TN / 2;   // columns per warp (two warps per lane quadrant)
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sA = base;
    unsigned char *sB = sA + (size_t)a.group * kABlockBytes;
    __shared__ uint64_t full, done;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = blockIdx.x;              // A tile (batch rows, or output rows for dw)
    const int j = blockIdx.y;                  // 64-column slice of the output
    const int z = blockIdx.z;
    const int c_beg = z * a.cps, c_end = (z + 1) * a.cps < a.kc ? (z + 1) * a.cps : a.kc;
    if (threadIdx.x == 0) {
        mbar_init(&full, 1);
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_base)),
                     "n"(TN < 32 ? 32 : TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the set-up above overlaps the previous kernel of the stream; its outputs
    // are read from here on
    pdl_wait();
    pdl_trigger();
    const uint32_t tmem = tmem_base;
    volatile int *abort = &abort_flag;
    bool ok = true;
    uint32_t phase = 0;
    for (int g0 = c_beg; g0 < c_end && ok; g0 += a.group, phase ^= 1u) {
        const int g1 = g0 + a.group < c_end ? g0 + a.group : c_end;
        if (threadIdx.x == 0) {
            mbar_expect_tx(&full, (uint32_t)(g1 - g0) * (kABlockBytes + kBSliceBytes));
            for (int c = g0; c < g1; ++c) {
                bulk_g2s(sA + (size_t)(c - g0) * kABlockBytes, a.A + ((size_t)t * a.a_kc + c) * (kABlockBytes / 2),
                         kABlockBytes, &full);
                bulk_g2s(sB + (size_t)(c - g0) * kBSliceBytes,
                         a.B + ((size_t)c * a.b_rows + (size_t)j * TN) * KCH, kBSliceBytes, &full);
            }
            ok = mbar_wait(&full, phase, abort);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (ok) {
                for (int c = g0; c < g1; ++c) {
                    const uint32_t a0 = su32(sA + (size_t)(c - g0) * kABlockBytes);
                    const uint32_t b0 = su32(sB + (size_t)(c - g0) * kBSliceBytes);
#pragma unroll
                    for (int kk = 0; kk < KCH / 16; ++kk) {
                        const uint32_t acc = (c != c_beg || kk != 0) ? 1u : 0u;
                        asm volatile(
                            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                            "l"(sdesc(a0 + kk * 256)), "l"(sdesc(b0 + kk * 256)), "r"(idesc_n(TN)), "r"(acc)
                            : "memory");
                    }
                }
            }
            // the next group overwrites the stages: wait until these MMAs have read them
            umma_commit(&done);
            ok = mbar_wait(&done, phase, abort) && ok;
        }
        __syncthreads();
        ok = !*abort;
    }
    // a group that gave up waiting may still have copies in flight: one more
    // bounded wait for them before the CTA leaves
    if (!ok && threadIdx.x == 0) {
        volatile int never = 0;
        mbar_wait(&full, phase ^ 1u, &never);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (MODE == kTrainDw && !(c_beg < c_end)) {
        // an empty split contributes zeros
        const size_t ncol = (size_t)gridDim.y * TN;
        for (int e = threadIdx.x; e < UM * TN; e += blockDim.x)
            a.part[((size_t)z * 256 + (size_t)t * UM + e / TN) * ncol + (size_t)j * TN + e % TN] = 0.0f;
    }
    if (ok && c_beg < c_end) {
        const int quad = warp & 3;          // TMEM lane quadrant of this warp
        const int row = quad * 32 + lane;   // TMEM lane = row of the tile
        const int c0 = (warp >> 2) * kCols;   // this warp's kCols of the TN columns
        uint32_t r[kCols];
        const uint32_t ta = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0;
        if constexpr (kCols == 32) {
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                  "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                  "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                  "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                  "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(ta));
        } else {
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                  "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                  "=r"(r[14]), "=r"(r[15])
                : "r"(ta));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int n0 = j * TN + c0;     // first output column of this warp's columns
        if (MODE == kTrainDw) {
            // part [z][out row][in column], in columns = b_n = gridDim.y * TN
            const size_t ncol = (size_t)gridDim.y * TN;
            float4 *dst = reinterpret_cast<float4 *>(a.part + ((size_t)z * 256 + (size_t)t * UM + row) * ncol + n0);
#pragma unroll
            for (int q = 0; q < kCols / 4; ++q)
                dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                     __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
        } else {
            const int64_t m = t * UM + row;   // batch row
            float v[kCols];
            if (MODE == kTrainFwd) {
                const float4 *bb = reinterpret_cast<const float4 *>(a.bias + n0);
#pragma unroll
                for (int q = 0; q < kCols / 4; ++q) {
                    const float4 b4 = __ldg(bb + q);
                    v[4 * q] = __uint_as_float(r[4 * q]) + b4.x;
                    v[4 * q + 1] = __uint_as_float(r[4 * q + 1]) + b4.y;
                    v[4 * q + 2] = __uint_as_float(r[4 * q + 2]) + b4.z;
                    v[4 * q + 3] = __uint_as_float(r[4 * q + 3]) + b4.w;
                }
            } else {
                const float4 *zin = reinterpret_cast<const float4 *>(a.Zin + (size_t)m * 256 + n0);
#pragma unroll
                for (int q = 0; q < kCols / 4; ++q) {
                    const float4 zz = zin[q];
                    v[4 * q] = __uint_as_float(r[4 * q]) * gelu_grad_u(zz.x);
                    v[4 * q + 1] = __uint_as_float(r[4 * q + 1]) * gelu_grad_u(zz.y);
                    v[4 * q + 2] = __uint_as_float(r[4 * q + 2]) * gelu_grad_u(zz.z);
                    v[4 * q + 3] = __uint_as_float(r[4 * q + 3]) * gelu_grad_u(zz.w);
                }
            }
            float4 *zo = reinterpret_cast<float4 *>(a.Zout + (size_t)m * 256 + n0);
#pragma unroll
            for (int q = 0; q < kCols / 4; ++q) zo[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            // the BF16 values: bf16(gelu(z)) forward, bf16(dz) backward
            uint32_t hv[kCols / 2];
#pragma unroll
            for (int e = 0; e < kCols / 2; ++e)
                hv[e] = MODE == kTrainFwd ? pack_bf16(gelu_u(v[2 * e]), gelu_u(v[2 * e + 1]))
                                          : pack_bf16(v[2 * e], v[2 * e + 1]);
            // tiled (128-row tiles, K 256): 16-byte pieces of 8 columns
#pragma unroll
            for (int g = 0; g < kCols / 8; ++g)
                *reinterpret_cast<uint4 *>(a.Ht + tiled_at(m, n0 + 8 * g, UM, 4)) =
                    make_uint4(hv[4 * g], hv[4 * g + 1], hv[4 * g + 2], hv[4 * g + 3]);
            if (MODE == kTrainFwd && a.Hrm) {
                uint4 *hr = reinterpret_cast<uint4 *>(a.Hrm + (size_t)m * 256 + n0);
#pragma unroll
                for (int g = 0; g < kCols / 8; ++g) hr[g] = make_uint4(hv[4 * g], hv[4 * g + 1], hv[4 * g + 2], hv[4 * g + 3]);
            }
            // transposed-tiled: element (n, m)
            const uint16_t *h16 = reinterpret_cast<const uint16_t *>(hv);
            uint16_t *tt = reinterpret_cast<uint16_t *>(a.HtT);
            const int trl = a.tt_rows == 256 ? 8 : 7;
#pragma unroll
            for (int e = 0; e < kCols; ++e) tt[tiled_at_pow2(n0 + e, m, trl, a.m_kc)] = h16[e];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TN < 32 ? 32 : TN));
    }
    if (threadIdx.x == 0 && abort_flag) atomicExch(a.err, 1);
}

// Training inputs: x [M][8] FP32 -> h0 tiled (128-row tiles, K 64) and
// transposed-tiled (one 64-row tile: the 64 padded features, K = the batch);
// features 8..63 and rows >= M are zero.
// With `step`, batch row m is row perm[e n + r0 + m] of X (identity without
// perm), e = step / spe, r0 = (step % spe) batch, and its label goes to yb.
struct TrainGather {
    const int32_t *perm;
    int64_t n, batch, spe;
    const int64_t *step;
    const float *y;
    float *yb;
};
__global__ void k_train_input(const float *__restrict__ X, int64_t M, int64_t m_pad, __nv_bfloat16 *__restrict__ H0,
                              __nv_bfloat16 *__restrict__ H0T, TrainGather gth) {
    pdl_wait();
    pdl_trigger();
    const int64_t n = m_pad * 64;
    uint16_t *t = reinterpret_cast<uint16_t *>(H0T);
    uint16_t *h = reinterpret_cast<uint16_t *>(H0);
    int64_t ep = 0, r0 = 0;
    if (gth.step) {
        const int64_t st = *gth.step;
        ep = st / gth.spe;
        r0 = (st % gth.spe) * gth.batch;
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = i >> 6;
        const int f = (int)(i & 63);
        int64_t row = m;
        if (gth.step && m < M) {
            row = gth.perm ? (int64_t)gth.perm[ep * gth.n + r0 + m] : r0 + m;
            if (f == 0) gth.yb[m] = gth.y[row];
        }
        const float v = (m < M && f < 8) ? X[row * 8 + f] : 0.0f;
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        const uint16_t u = *reinterpret_cast<const uint16_t *>(&b);
        h[tiled_at(m, f, UM, 1)] = u;
        t[tiled_at(f, m, 64, m_pad / 64)] = u;
    }
}

// The head and its backward step, 16 rows per block (8 warps, 2 rows each):
// for row m, lane l holds the 8 columns k = 64 (l / 8) + 8 (l % 8) + e of the
// tiled h4 row; the logit h4 . w5 + b5 is lane 0's sum after the xor butterfly
// (as k_head_tiled), broadcast to the warp; dlogit = (sigmoid(logit) - y) / M;
// dz = dlogit w5[k] gelu'(z4) goes out as FP32 and BF16 tiled, and the BF16
// values through shared memory to the transposed-tiled copy as 16-byte
// pieces of 8 rows of one column (8 consecutive threads write 128 B).
// Rows m >= M take dz = 0.
constexpr int kHeadRows = 16;
constexpr int kHeadLd = 264;   // shared row length in BF16 (528 B: 8 rows of one column fall in distinct banks)
__global__ void __launch_bounds__(256) k_train_head(const __nv_bfloat16 *__restrict__ H4,
                                                    const __nv_bfloat16 *__restrict__ w5,
                                                    const float *__restrict__ b5, const float *__restrict__ y,
                                                    int64_t M, int64_t m_pad, const float *__restrict__ Z4,
                                                    float *__restrict__ logit, float *__restrict__ dl,
                                                    float *__restrict__ dz, __nv_bfloat16 *__restrict__ dzb,
                                                    __nv_bfloat16 *__restrict__ dzbT, float *__restrict__ loss_terms) {
    __shared__ __align__(16) uint16_t S[kHeadRows * kHeadLd];
    pdl_wait();
    pdl_trigger();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.x * kHeadRows;
    const int c = lane >> 3, kg = lane & 7;
    const int k0 = c * 64 + kg * 8;
    const uint4 wv = *reinterpret_cast<const uint4 *>(w5 + k0);
    const __nv_bfloat16 *w = reinterpret_cast<const __nv_bfloat16 *>(&wv);
    const float bias = b5[0];
    constexpr int R = kHeadRows / 8;   // rows per warp
    float d[R], z[R][8];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int64_t m = m0 + warp * R + i;
        const float4 z0 = *reinterpret_cast<const float4 *>(Z4 + m * 256 + k0);
        const float4 z1 = *reinterpret_cast<const float4 *>(Z4 + m * 256 + k0 + 4);
        z[i][0] = z0.x; z[i][1] = z0.y; z[i][2] = z0.z; z[i][3] = z0.w;
        z[i][4] = z1.x; z[i][5] = z1.y; z[i][6] = z1.z; z[i][7] = z1.w;
        d[i] = 0.0f;
        if (m < M) {
            const int64_t t = m / UM;
            const int rr = (int)(m % UM);
            const uint4 hv = *reinterpret_cast<const uint4 *>(H4 + (((size_t)t * 4 + c) * 16 + (rr >> 3)) * 8 * 64 +
                                                              (size_t)kg * 64 + (rr & 7) * 8);
            const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&hv);
            float s = 0.0f;
#pragma unroll
            for (int e = 0; e < 8; ++e) s += __bfloat162float(h[e]) * __bfloat162float(w[e]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            const float l = __shfl_sync(0xffffffffu, s, 0) + bias;
            const float ym = y[m];
            d[i] = (1.0f / (1.0f + expf(-l)) - ym) / (float)M;
            if (lane == 0) {
                logit[m] = l;
                dl[m] = d[i];
                loss_terms[m] = fmaxf(l, 0.0f) + log1pf(expf(-fabsf(l))) - ym * l;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int rl = warp * R + i;   // row within the block
        const int64_t m = m0 + rl;
        float v[8];
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = m < M ? d[i] * __bfloat162float(w[e]) * gelu_grad_u(z[i][e]) : 0.0f;
#pragma unroll
        for (int e = 0; e < 4; ++e) pk[e] = pack_bf16(v[2 * e], v[2 * e + 1]);
        *reinterpret_cast<float4 *>(dz + m * 256 + k0) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4 *>(dz + m * 256 + k0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
        const uint4 p4 = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        *reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(dzb) + tiled_at(m, k0, UM, 4)) = p4;
        *reinterpret_cast<uint4 *>(S + rl * kHeadLd + k0) = p4;
    }
    __syncthreads();
    // transposed-tiled: element (k, m) of the 256 x m_pad matrix in 128-row
    // tiles over k; piece q holds rows m0 + 8 g .. + 7 of column k
    uint16_t *bT = reinterpret_cast<uint16_t *>(dzbT);
    const int64_t kcn = m_pad / 64;
    constexpr int G = kHeadRows / 8;   // pieces per column
    for (int q = threadIdx.x; q < 256 * G; q += blockDim.x) {
        const int k = ((q / (8 * G)) << 3) | (q & 7);
        const int g = (q >> 3) % G;
        uint16_t u[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) u[r] = S[(g * 8 + r) * kHeadLd + k];
        const size_t at = (((size_t)(k >> 7) * kcn + (size_t)(m0 >> 6)) * 16 + (size_t)((k & 127) >> 3)) * 512 +
                          (size_t)(((m0 & 63) >> 3) + g) * 64 + (size_t)(k & 7) * 8;
        *reinterpret_cast<uint4 *>(bT + at) =
            make_uint4((uint32_t)u[0] | ((uint32_t)u[1] << 16), (uint32_t)u[2] | ((uint32_t)u[3] << 16),
                       (uint32_t)u[4] | ((uint32_t)u[5] << 16), (uint32_t)u[6] | ((uint32_t)u[7] << 16));
    }
}

// BF16 weights [out][in_pad] of the four hidden layers (at w_off[l] in pb) ->
// the tiled copies the products read: wt[l] (256-row tile over the outputs,
// K = in_pad) and, for l >= 1, wtT[l] = W_l^T (256-row tile over the inputs, K 256).
struct RetileArgs {
    const __nv_bfloat16 *pb;
    size_t w_off[4], wt_off[4], wtT_off[4];
    int in_pad[4];
    __nv_bfloat16 *wt, *wtT;
};
__global__ void k_retile_weights(RetileArgs r) {
    const int64_t per1 = 256 * 64, per = 256 * 256;
    const int64_t n = per1 + 3 * per;
    const uint16_t *src = reinterpret_cast<const uint16_t *>(r.pb);
    uint16_t *wt = reinterpret_cast<uint16_t *>(r.wt), *wtT = reinterpret_cast<uint16_t *>(r.wtT);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int l;
        int64_t e;
        if (i < per1) {
            l = 0;
            e = i;
        } else {
            l = 1 + (int)((i - per1) / per);
            e = (i - per1) % per;
        }
        const int K = r.in_pad[l];
        const int64_t o = e / K, k = e % K;
        const uint16_t v = src[r.w_off[l] + e];
        wt[r.wt_off[l] + tiled_at(o, k, 256, K / 64)] = v;
        if (l >= 1) wtT[r.wtT_off[l] + tiled_at(k, o, 256, 4)] = v;
    }
}

// One Adam step of the training graph on FP32 master weights (Kingma & Ba; the
// bias corrections c1 = 1 - beta1^t, c2 = 1 - beta2^t from the table c12 at
// the device step counter), writing the BF16 copy and, for the hidden layers'
// weights, their tiled copies (wt, and wtT = W^T for l >= 1); the last block
// records the step's loss and advances the step counter.
struct AdamStepArgs {
    float *p, *m, *v;
    float *g;
    __nv_bfloat16 *pb;
    int64_t n;
    float lr, b1, b2, eps;
    const float *c12;
    int64_t *step;
    const float *loss;
    float *loss_hist;
    unsigned *ticket;
    RetileArgs r;
    size_t w_end[4];   // the weights of layer l are [w_off[l], w_end[l]) of the parameter array
    // with wpart[l], layer l's weight gradient is the sum of its `splits`
    // batch-split partials (each [256][in_pad], in split order), also stored to g
    const float *wpart[4];
    int splits;
};
__global__ void k_adam_step(AdamStepArgs a) {
    __shared__ bool last;
    pdl_wait();
    pdl_trigger();
    const int64_t st = *a.step;
    const float c1 = a.c12[2 * st], c2 = a.c12[2 * st + 1];
    uint16_t *wt = reinterpret_cast<uint16_t *>(a.r.wt), *wtT = reinterpret_cast<uint16_t *>(a.r.wtT);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        int l = -1;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if ((size_t)i >= a.r.w_off[q] && (size_t)i < a.w_end[q]) l = q;
        const int64_t e = l >= 0 ? (int64_t)((size_t)i - a.r.w_off[l]) : 0;
        float gi;
        if (l >= 0 && a.wpart[l]) {
            const float *wp = a.wpart[l];
            const int64_t len = (int64_t)(a.w_end[l] - a.r.w_off[l]);
            gi = wp[e];
            for (int z = 1; z < a.splits; ++z) gi = gi + wp[(int64_t)z * len + e];
            a.g[i] = gi;
        } else {
            gi = a.g[i];
        }
        const float mi = a.b1 * a.m[i] + (1.0f - a.b1) * gi;
        const float vi = a.b2 * a.v[i] + (1.0f - a.b2) * gi * gi;
        a.m[i] = mi;
        a.v[i] = vi;
        const float w = a.p[i] - a.lr * (mi / c1) / (sqrtf(vi / c2) + a.eps);
        a.p[i] = w;
        const __nv_bfloat16 wb = __float2bfloat16_rn(w);
        a.pb[i] = wb;
        if (l >= 0) {
            const int K = a.r.in_pad[l];
            const int64_t o = e / K, k = e % K;
            const uint16_t u = *reinterpret_cast<const uint16_t *>(&wb);
            wt[a.r.wt_off[l] + tiled_at(o, k, 256, K / 64)] = u;
            if (l >= 1) wtT[a.r.wtT_off[l] + tiled_at(k, o, 256, 4)] = u;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last && threadIdx.x == 0) {
        if (a.loss_hist) a.loss_hist[st] = *a.loss;
        *a.step = st + 1;
        *a.ticket = 0u;
    }
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

constexpr int kTnAct = 32;   // output columns per CTA of the forward and input-gradient products
constexpr int kTnDw = 64;    // the same of the weight gradients

int train_group(int chunks_per_cta) { return chunks_per_cta < kGroupChunks ? chunks_per_cta : kGroupChunks; }

size_t train_tile_smem(int chunks_per_cta, int tn) {
    const int g = train_group(chunks_per_cta);
    return 1024 + (size_t)g * (kABlockBytes + (size_t)tn * KCH * 2);
}

cudaError_t launch_train_fwd(const uint16_t *H_tiled, int K, const uint16_t *W_tiled, const float *bias,
                             int64_t m_pad, float *Z, uint16_t *Hout_tiled, uint16_t *Hout_T, uint16_t *Hout_rm,
                             int *d_err, cudaStream_t s) {
    if (K % KCH || K < KCH || K > 256 || m_pad % UM) return cudaErrorInvalidValue;
    TrainTileArgs a{};
    a.A = reinterpret_cast<const __nv_bfloat16 *>(H_tiled);
    a.a_kc = K / KCH;
    a.B = reinterpret_cast<const __nv_bfloat16 *>(W_tiled);
    a.b_rows = 256;
    a.kc = K / KCH;
    a.cps = a.kc;
    a.bias = bias;
    a.Zout = Z;
    a.Ht = reinterpret_cast<__nv_bfloat16 *>(Hout_tiled);
    a.HtT = reinterpret_cast<__nv_bfloat16 *>(Hout_T);
    a.Hrm = reinterpret_cast<__nv_bfloat16 *>(Hout_rm);
    a.tt_rows = 256;
    a.m_kc = m_pad / KCH;
    a.err = d_err;
    a.group = train_group(a.cps);
    const size_t smem = train_tile_smem(a.cps, kTnAct);
    cudaError_t e = cudaFuncSetAttribute(k_train_tile<kTrainFwd, kTnAct>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return pdl_launch(k_train_tile<kTrainFwd, kTnAct>, dim3((unsigned)(m_pad / UM), 256 / kTnAct, 1),
                      dim3(kTrainThreads), smem, s, a);
}

cudaError_t launch_train_dx(const uint16_t *dzb_tiled, const uint16_t *WT_tiled, const float *Zin, int64_t m_pad,
                            float *dz, uint16_t *dzb_out_tiled, uint16_t *dzb_out_T, int *d_err, cudaStream_t s) {
    if (m_pad % UM) return cudaErrorInvalidValue;
    TrainTileArgs a{};
    a.A = reinterpret_cast<const __nv_bfloat16 *>(dzb_tiled);
    a.a_kc = 4;
    a.B = reinterpret_cast<const __nv_bfloat16 *>(WT_tiled);
    a.b_rows = 256;
    a.kc = 4;
    a.cps = 4;
    a.Zin = Zin;
    a.Zout = dz;
    a.Ht = reinterpret_cast<__nv_bfloat16 *>(dzb_out_tiled);
    a.HtT = reinterpret_cast<__nv_bfloat16 *>(dzb_out_T);
    a.tt_rows = UM;
    a.m_kc = m_pad / KCH;
    a.err = d_err;
    a.group = train_group(a.cps);
    const size_t smem = train_tile_smem(a.cps, kTnAct);
    cudaError_t e = cudaFuncSetAttribute(k_train_tile<kTrainDx, kTnAct>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return pdl_launch(k_train_tile<kTrainDx, kTnAct>, dim3((unsigned)(m_pad / UM), 256 / kTnAct, 1),
                      dim3(kTrainThreads), smem, s, a);
}

int train_dw_splits(int64_t m_pad) {
    const int kc = (int)(m_pad / KCH);
    int S = (kc + kGroupChunks - 1) / kGroupChunks;   // one group of chunks per CTA
    return S < 1 ? 1 : S;
}

cudaError_t launch_train_dw(const uint16_t *dzb_T, const uint16_t *H_T, int n_in, int64_t m_pad, float *part,
                            int *d_err, cudaStream_t s) {
    if (m_pad % UM || n_in % kTnDw || n_in < kTnDw || n_in > 256) return cudaErrorInvalidValue;
    TrainTileArgs a{};
    a.A = reinterpret_cast<const __nv_bfloat16 *>(dzb_T);
    a.a_kc = m_pad / KCH;
    a.B = reinterpret_cast<const __nv_bfloat16 *>(H_T);
    a.b_rows = n_in;
    a.kc = (int)(m_pad / KCH);
    const int S = train_dw_splits(m_pad);
    a.cps = (a.kc + S - 1) / S;
    a.part = part;
    a.err = d_err;
    a.group = train_group(a.cps);
    const size_t smem = train_tile_smem(a.cps, kTnDw);
    cudaError_t e = cudaFuncSetAttribute(k_train_tile<kTrainDw, kTnDw>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return pdl_launch(k_train_tile<kTrainDw, kTnDw>, dim3(256 / UM, (unsigned)(n_in / kTnDw), (unsigned)S),
                      dim3(kTrainThreads), smem, s, a);
}

cudaError_t launch_train_input(const float *X, int64_t M, int64_t m_pad, uint16_t *H0, uint16_t *H0T,
                               const int32_t *perm, int64_t n, int64_t batch, int64_t spe, const int64_t *step,
                               const float *y, float *yb, cudaStream_t s) {
    TrainGather g{perm, n, batch, spe, step, y, yb};
    return pdl_launch(k_train_input, dim3(grid_for(m_pad * 64)), dim3(256), 0, s, X, M, m_pad,
                      reinterpret_cast<__nv_bfloat16 *>(H0), reinterpret_cast<__nv_bfloat16 *>(H0T), g);
}

cudaError_t launch_train_head(const uint16_t *H4_tiled, const uint16_t *w5, const float *b5, const float *y,
                              int64_t M, int64_t m_pad, const float *Z4, float *logit, float *dl, float *dz,
                              uint16_t *dzb, uint16_t *dzbT, float *loss_terms, cudaStream_t s) {
    if (m_pad % kHeadRows) return cudaErrorInvalidValue;
    return pdl_launch(k_train_head, dim3((unsigned)(m_pad / kHeadRows)), dim3(256), 0, s, reinterpret_cast<const __nv_bfloat16 *>(H4_tiled),
                      reinterpret_cast<const __nv_bfloat16 *>(w5), b5, y, M, m_pad, Z4, logit, dl, dz,
                      reinterpret_cast<__nv_bfloat16 *>(dzb), reinterpret_cast<__nv_bfloat16 *>(dzbT), loss_terms);
}

cudaError_t launch_retile_weights(const uint16_t *pb, const size_t *w_off, const size_t *wt_off, const size_t *wtT_off,
                                  const int *in_pad, uint16_t *wt, uint16_t *wtT, cudaStream_t s) {
    RetileArgs r;
    r.pb = reinterpret_cast<const __nv_bfloat16 *>(pb);
    for (int l = 0; l < 4; ++l) {
        r.w_off[l] = w_off[l];
        r.wt_off[l] = wt_off[l];
        r.wtT_off[l] = wtT_off[l];
        r.in_pad[l] = in_pad[l];
    }
    r.wt = reinterpret_cast<__nv_bfloat16 *>(wt);
    r.wtT = reinterpret_cast<__nv_bfloat16 *>(wtT);
    k_retile_weights<<<grid_for(256 * 64 + 3 * 256 * 256), 256, 0, s>>>(r);
    return cudaGetLastError();
}

cudaError_t launch_adam_step(float *p, float *m, float *v, float *g, uint16_t *pb, int64_t n, float lr,
                             const float *c12, int64_t *step, const float *loss, float *loss_hist, unsigned *ticket,
                             const size_t *w_off, const size_t *w_end, const size_t *wt_off, const size_t *wtT_off,
                             const int *in_pad, uint16_t *wt, uint16_t *wtT, const float *const *wpart, int splits,
                             cudaStream_t s) {
    AdamStepArgs a;
    a.p = p;
    a.m = m;
    a.v = v;
    a.g = g;
    a.pb = reinterpret_cast<__nv_bfloat16 *>(pb);
    a.n = n;
    a.lr = lr;
    a.b1 = 0.9f;
    a.b2 = 0.999f;
    a.eps = 1e-8f;
    a.c12 = c12;
    a.step = step;
    a.loss = loss;
    a.loss_hist = loss_hist;
    a.ticket = ticket;
    a.r.pb = a.pb;
    for (int l = 0; l < 4; ++l) {
        a.r.w_off[l] = w_off[l];
        a.w_end[l] = w_end[l];
        a.r.wt_off[l] = wt_off[l];
        a.r.wtT_off[l] = wtT_off[l];
        a.r.in_pad[l] = in_pad[l];
        a.wpart[l] = wpart ? wpart[l] : nullptr;
    }
    a.splits = splits;
    a.r.wt = reinterpret_cast<__nv_bfloat16 *>(wt);
    a.r.wtT = reinterpret_cast<__nv_bfloat16 *>(wtT);
    return pdl_launch(k_adam_step, dim3(grid_for(n)), dim3(256), 0, s, a);
}

cudaError_t launch_head_tiled(const uint16_t *H4, const uint16_t *w5, const float *b5, int64_t M, float *logit,
                              cudaStream_t s) {
    const int rows_per_block = 8;
    k_head_tiled<<<(unsigned)((M + rows_per_block - 1) / rows_per_block), 32 * rows_per_block, 0, s>>>(
        reinterpret_cast<const __nv_bfloat16 *>(H4), reinterpret_cast<const __nv_bfloat16 *>(w5), b5, M, logit);
    return cudaGetLastError();
}

}  // namespace trk
