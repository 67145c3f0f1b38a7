// Fused forward pass of the learned sampling proposal on the 5th-generation
// tensor cores (tcgen05): the three layers of the network of mlp_kernels.cuh,
//   a1 = W1g grid + W1n z + b1,  h1 = relu(a1)
//   a2 = W2 h1 + b2,             h2 = relu(a2)
//   y  = sigmoid(W3 h2 + b3)
// for 128 sample rows per tile, with the activations kept on chip: every
// contraction is a tcgen05.mma chain (BF16 operands in shared memory, FP32
// accumulator in tensor memory), every elementwise step runs on the CTA's
// 256 threads between them, and only the noise in and the two outputs per
// row touch HBM (40 bytes per row).  Warp w reads TMEM lanes 32 (w mod 4) ..
// + 31 (rows) and columns 128 (w / 4) .. + 127: two column halves per row.
//
//   layer 1: D[128 x 256] = Z[128 x 16] * W1n'[256 x 16]^T   (K padded 8 -> 16)
//            h1 = relu(D + (W1g grid + b1)[scene])  -> H (shared, BF16)
//   layer 2: D[128 x 256] = H[128 x 256] * W2[256 x 256]^T
//            h2 = relu(D + b2)                       -> H (overwrites h1)
//   layer 3: D[128 x 16]  = H[128 x 256] * W3'[16 x 256]^T  (N padded 2 -> 16)
//            y = sigmoid(D[:, 0:2] + b3)
//
// The grid part of layer 1 (one 4096 x 256 product per scene) is computed
// once per call outside this kernel; W1g grid + b1 arrives per scene.  The
// rounding points are those of the unfused path: BF16 weights, BF16 noise,
// BF16 h1 and h2, FP32 accumulation, FP32 bias additions and sigmoid.
//
// Persistent: one CTA of 256 threads per SM (about 214 KB of shared memory:
// W2 stays resident across tiles), tiles strided over the grid.  One thread
// issues the MMAs.  Layers 1 and 2 are issued as two N = 128 halves, each
// committed to its own mbarrier, so the first half's epilogue runs while the
// tensor core computes the second (layer 2's h2 is stored only after both
// halves are done, since both read h1 from the same buffer).  Every wait is
// bounded; a thread whose wait expires reports it at the next CTA barrier
// (__syncthreads_or), the CTA stops, waits a bounded time more for its MMAs in
// flight, frees its tensor memory and returns with an error bit set.
//
// Operand layouts in shared memory (K-major, i.e. each row's K elements
// contiguous, as tcgen05 descriptors describe them):
//   * 128-byte swizzle for H, W2 and W3': 8-row groups of 8 x 128 bytes, the
//     16-byte chunk c of row r stored at chunk c ^ (r mod 8); K in blocks of
//     64 elements, one such block of all rows after another;
//   * no swizzle for the K = 16 operands Z and W1n': 8 x 16-byte core
//     matrices, the two K halves 128 bytes apart, 8-row groups 256 bytes
//     apart.
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

#include "mlp_kernels.cuh"

namespace pirrt {
namespace mlp {
namespace tc {

constexpr int kRowsPerTile = 128;
constexpr int kThreads = 256;
constexpr uint32_t kTmemCols = 256;
constexpr int kN3 = 16;   // layer-3 N padded to the smallest M = 128 shape
constexpr int kK1 = 16;   // layer-1 K padded to one MMA step

// shared-memory map, offsets from a 1024-byte-aligned base
constexpr int kW2Bytes = kHidden * kHidden * 2;     // 131072
constexpr int kHBytes = kRowsPerTile * kHidden * 2;  // 65536
constexpr int kW3Bytes = kN3 * kHidden * 2;          // 8192
constexpr int kZBytes = kRowsPerTile * kK1 * 2;      // 4096
constexpr int kW1Bytes = kHidden * kK1 * 2;          // 8192
constexpr int oW2 = 0;
constexpr int oH = oW2 + kW2Bytes;
constexpr int oW3 = oH + kHBytes;
constexpr int oZ = oW3 + kW3Bytes;
constexpr int oW1 = oZ + kZBytes;
constexpr int oB2 = oW1 + kW1Bytes;         // 256 FP32
constexpr int oBar = oB2 + kHidden * 4;     // two mbarriers (column halves), 8 bytes each
constexpr int oTmem = oBar + 16;            // TMEM base address written by tcgen05.alloc
constexpr int kSmemUsed = oTmem + 4;
constexpr int kSmemBytes = kSmemUsed + 1024;  // + alignment slack

constexpr unsigned long long kMmaWaitNs = 1000000000ull;  // 1 s per wait

// Error bits the kernel leaves in *status (0 = success).
constexpr int kErrTimeout = 1;
constexpr int kErrScene = 2;

__device__ __forceinline__ uint32_t saddr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// byte offset of the 16-byte chunk holding elements k .. k+7 of row r in a
// 128-byte-swizzled K-major operand of `rows` rows
__device__ __forceinline__ uint32_t sw128(int r, int k, int rows) {
    const int kb = k >> 6, c = (k >> 3) & 7;
    return (uint32_t)(kb * rows * 128 + (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}

// byte offset of the 16-byte core-matrix row holding elements 8*kc .. 8*kc+7
// of row r in an unswizzled K-major operand with K = 16
__device__ __forceinline__ uint32_t plain16(int r, int kc) {
    return (uint32_t)((r >> 3) * 256 + kc * 128 + (r & 7) * 16);
}

// shared-memory matrix descriptor: start address, leading-dimension byte
// offset (LBO), stride-dimension byte offset (SBO), descriptor version 1,
// swizzle mode (0 none, 2 = 128-byte)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo,
                                              uint32_t swizzle) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)swizzle << 61);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// generic-proxy shared-memory writes made visible to the tensor core's reads
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity, unsigned long long ns) {
    const uint32_t a = saddr(bar);
    const unsigned long long t0 = now_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (now_ns() - t0 > ns) return false;
    }
}

// 32 consecutive FP32 columns of this thread's TMEM lane; the wait that
// completes the load is tied to the registers so no use is scheduled before it
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                   "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 consecutive FP32 columns of this thread's TMEM lane (two 32-column
// loads completed by one wait)
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
    uint32_t r[64];
#define PIRRT_TC_LD32(base, dst)                                                                 \
    asm volatile(                                                                                \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "                                                \
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"                                \
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"               \
        : "=r"(dst[0]), "=r"(dst[1]), "=r"(dst[2]), "=r"(dst[3]), "=r"(dst[4]), "=r"(dst[5]),    \
          "=r"(dst[6]), "=r"(dst[7]), "=r"(dst[8]), "=r"(dst[9]), "=r"(dst[10]), "=r"(dst[11]),  \
          "=r"(dst[12]), "=r"(dst[13]), "=r"(dst[14]), "=r"(dst[15]), "=r"(dst[16]),             \
          "=r"(dst[17]), "=r"(dst[18]), "=r"(dst[19]), "=r"(dst[20]), "=r"(dst[21]),             \
          "=r"(dst[22]), "=r"(dst[23]), "=r"(dst[24]), "=r"(dst[25]), "=r"(dst[26]),             \
          "=r"(dst[27]), "=r"(dst[28]), "=r"(dst[29]), "=r"(dst[30]), "=r"(dst[31])              \
        : "r"(base))
    PIRRT_TC_LD32(taddr, r);
    PIRRT_TC_LD32(taddr + 32, (r + 32));
#undef PIRRT_TC_LD32
#define PIRRT_TC_TIE8(o)                                                                          \
    "+r"(r[o]), "+r"(r[o + 1]), "+r"(r[o + 2]), "+r"(r[o + 3]), "+r"(r[o + 4]), "+r"(r[o + 5]),   \
        "+r"(r[o + 6]), "+r"(r[o + 7])
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : PIRRT_TC_TIE8(0), PIRRT_TC_TIE8(8), PIRRT_TC_TIE8(16), PIRRT_TC_TIE8(24)
                 :
                 : "memory");
    asm volatile("" : PIRRT_TC_TIE8(32), PIRRT_TC_TIE8(40), PIRRT_TC_TIE8(48), PIRRT_TC_TIE8(56)
                 :
                 : "memory");
#undef PIRRT_TC_TIE8
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float &a, float &b) {
    uint32_t r0, r1;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
                 : "=r"(r0), "=r"(r1)
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r0), "+r"(r1) : : "memory");
    a = __uint_as_float(r0);
    b = __uint_as_float(r1);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}


struct FwdArgs {
    int rows, n_scenes;
    const float *hgb;              // [n_scenes x 256] W1g grid + b1 per scene
    const int32_t *scene;          // [rows]
    const float *z;                // [rows x 8]
    const float *W1n;              // [256 x 8] FP32 master weights (rounded here)
    const __nv_bfloat16 *W2b;      // [256 x 256], row = output unit
    const float *b2;               // [256]
    const __nv_bfloat16 *W3b;      // [2 x 256]
    const float *b3;               // [2]
    float *y;                      // [rows x 2] or null
    const float *uniform_xy;       // mixture: out[r] = coin[r] < frac ? y[r] : uniform_xy[r]
    const float *coin;
    float frac;
    float *out;                    // [rows x 2] or null
    __nv_bfloat16 *cap_h1, *cap_h2;  // optional copies of h1 / h2 [rows x 256]
    int *status;                   // error bits (kErr*)
};

// h = relu(v + bias) for 64 columns, packed to BF16 pairs
__device__ __forceinline__ void bias_relu_pack(const float (&v)[64], const float *bias,
                                               uint32_t *p) {
#pragma unroll
    for (int i = 0; i < 64; i += 4) {
        const float4 b = *reinterpret_cast<const float4 *>(bias + i);
        const float a0 = b.x + v[i], a1 = b.y + v[i + 1], a2 = b.z + v[i + 2], a3 = b.w + v[i + 3];
        p[i / 2] = pack_bf16(a0 > 0.f ? a0 : 0.f, a1 > 0.f ? a1 : 0.f);
        p[i / 2 + 1] = pack_bf16(a2 > 0.f ? a2 : 0.f, a3 > 0.f ? a3 : 0.f);
    }
}

// 64 packed columns (32 words) of row r from column c0 into the swizzled H
// (and the optional HBM copy)
__device__ __forceinline__ void store_h(uint8_t *sm, int row, int c0, const uint32_t *p,
                                        __nv_bfloat16 *cap, bool valid, int r) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint4 w = make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
        *reinterpret_cast<uint4 *>(sm + oH + sw128(row, c0 + q * 8, kRowsPerTile)) = w;
        if (cap && valid) *reinterpret_cast<uint4 *>(cap + (size_t)r * kHidden + c0 + q * 8) = w;
    }
}

__global__ void __launch_bounds__(kThreads, 1) mlp_forward_tc(const FwdArgs A) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = saddr(smem_raw);
    uint8_t *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t sb = saddr(sm);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + oBar);  // [0]: columns 0..127, [1]: 128..255
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(sm + oTmem);
    float *s_b2 = reinterpret_cast<float *>(sm + oB2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;  // TMEM lane quadrant, column half
    const int row = quad * 32 + lane;              // row of the tile (TMEM lane)
    const int col0 = half * 128;                   // first column of this thread

    // resident operands: W2, W3' (rows 2..15 zero), W1n' (K 8..15 zero), the
    // zero K half of Z, b2
    for (int i = tid; i < kHidden * (kHidden / 8); i += kThreads) {
        const int n = i >> 5, c = i & 31;
        const uint4 v = *reinterpret_cast<const uint4 *>(A.W2b + (size_t)n * kHidden + c * 8);
        *reinterpret_cast<uint4 *>(sm + oW2 + sw128(n, c * 8, kHidden)) = v;
    }
    for (int i = tid; i < kN3 * (kHidden / 8); i += kThreads) {
        const int n = i >> 5, c = i & 31;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (n < kOut) v = *reinterpret_cast<const uint4 *>(A.W3b + (size_t)n * kHidden + c * 8);
        *reinterpret_cast<uint4 *>(sm + oW3 + sw128(n, c * 8, kN3)) = v;
    }
    for (int n = tid; n < kHidden; n += kThreads) {
        const float *w = A.W1n + n * kNoise;
        *reinterpret_cast<uint4 *>(sm + oW1 + plain16(n, 0)) =
            make_uint4(pack_bf16(w[0], w[1]), pack_bf16(w[2], w[3]), pack_bf16(w[4], w[5]),
                       pack_bf16(w[6], w[7]));
        *reinterpret_cast<uint4 *>(sm + oW1 + plain16(n, 1)) = make_uint4(0u, 0u, 0u, 0u);
        s_b2[n] = A.b2[n];
    }
    if (tid < kRowsPerTile)
        *reinterpret_cast<uint4 *>(sm + oZ + plain16(tid, 1)) = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar)) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar + 1)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(saddr(s_tmem)), "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *s_tmem;
    const uint32_t my_tmem = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)col0;
    const float b30 = A.b3[0], b31 = A.b3[1];
    const uint32_t id128 = idesc_bf16(kRowsPerTile, 128), id16 = idesc_bf16(kRowsPerTile, kN3);
    const int ntiles = (A.rows + kRowsPerTile - 1) / kRowsPerTile;
    uint32_t cA = 0, cB = 0;  // completions of bar[0] / bar[1] before this tile
    uint32_t nA = 0, nB = 0;  // commits issued to bar[0] / bar[1] (thread 0)
    bool bad = false;         // a wait of this thread expired

    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int r = tile * kRowsPerTile + row;
        const bool valid = r < A.rows;
        int s = 0;
        if (valid) {
            s = A.scene[r];
            if (s < 0 || s >= A.n_scenes) {
                if (half == 0) atomicOr(A.status, kErrScene);
                s = 0;
            }
            if (half == 0) {
                const float4 z0 = *reinterpret_cast<const float4 *>(A.z + (size_t)r * kNoise);
                const float4 z1 = *reinterpret_cast<const float4 *>(A.z + (size_t)r * kNoise + 4);
                *reinterpret_cast<uint4 *>(sm + oZ + plain16(row, 0)) =
                    make_uint4(pack_bf16(z0.x, z0.y), pack_bf16(z0.z, z0.w),
                               pack_bf16(z1.x, z1.y), pack_bf16(z1.z, z1.w));
            }
        } else if (half == 0) {
            *reinterpret_cast<uint4 *>(sm + oZ + plain16(row, 0)) = make_uint4(0u, 0u, 0u, 0u);
        }
        fence_async_smem();
        fence_before();
        if (__syncthreads_or(bad)) break;
        // layer 1, two column halves: D[:, h*128 ..] = Z W1n'[h*128 ..]^T
        if (tid == 0) {
            fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                mma(tmem + h * 128, smem_desc(sb + oZ, 128, 256, 0),
                    smem_desc(sb + oW1 + plain16(h * 128, 0), 128, 256, 0), id128, 0u);
                commit(bar + h);
            }
            ++nA;
            ++nB;
        }
        if (!bar_wait(bar + half, (half ? cB : cA) & 1u, kMmaWaitNs)) bad = true;
        fence_after();
        {
            const float *hrow = A.hgb + (size_t)s * kHidden + col0;
#pragma unroll 1
            for (int c = 0; c < 128; c += 64) {
                float v[64];
                tmem_ld64(my_tmem + c, v);
                uint32_t p[32];
#pragma unroll
                for (int i = 0; i < 64; i += 4) {
                    const float4 hb = __ldg(reinterpret_cast<const float4 *>(hrow + c + i));
                    const float a0 = hb.x + v[i], a1 = hb.y + v[i + 1];
                    const float a2 = hb.z + v[i + 2], a3 = hb.w + v[i + 3];
                    p[i / 2] = pack_bf16(a0 > 0.f ? a0 : 0.f, a1 > 0.f ? a1 : 0.f);
                    p[i / 2 + 1] = pack_bf16(a2 > 0.f ? a2 : 0.f, a3 > 0.f ? a3 : 0.f);
                }
                store_h(sm, row, col0 + c, p, A.cap_h1, valid, r);
            }
        }
        fence_async_smem();
        fence_before();
        if (__syncthreads_or(bad)) break;
        // layer 2, two column halves: D[:, h*128 ..] = H W2[h*128 ..]^T, K = 256
        if (tid == 0) {
            fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll 1
                for (int kk = 0; kk < kHidden / 16; ++kk) {
                    const uint32_t kb = kk >> 2, sub = (kk & 3) * 32;
                    mma(tmem + h * 128,
                        smem_desc(sb + oH + kb * (kRowsPerTile * 128) + sub, 16, 1024, 2),
                        smem_desc(sb + oW2 + kb * (kHidden * 128) + h * 16384 + sub, 16, 1024, 2),
                        id128, kk > 0 ? 1u : 0u);
                }
                commit(bar + h);
            }
            ++nA;
            ++nB;
        }
        if (!bar_wait(bar + half, ((half ? cB : cA) + 1) & 1u, kMmaWaitNs)) bad = true;
        fence_after();
        {
            uint32_t p[64];
#pragma unroll
            for (int c = 0; c < 128; c += 64) {
                float v[64];
                tmem_ld64(my_tmem + c, v);
                bias_relu_pack(v, s_b2 + col0 + c, p + c / 2);
            }
            // both halves of layer 2 read h1 from H: store h2 once both are done
            if (half == 0 && !bar_wait(bar + 1, (cB + 1) & 1u, kMmaWaitNs)) bad = true;
            store_h(sm, row, col0, p, A.cap_h2, valid, r);
            store_h(sm, row, col0 + 64, p + 32, A.cap_h2, valid, r);
        }
        fence_async_smem();
        fence_before();
        if (__syncthreads_or(bad)) break;
        // layer 3: D[:, 0:16] = H W3'^T
        if (tid == 0) {
            fence_after();
#pragma unroll 1
            for (int kk = 0; kk < kHidden / 16; ++kk) {
                const uint32_t kb = kk >> 2, sub = (kk & 3) * 32;
                mma(tmem, smem_desc(sb + oH + kb * (kRowsPerTile * 128) + sub, 16, 1024, 2),
                    smem_desc(sb + oW3 + kb * (kN3 * 128) + sub, 16, 1024, 2), id16,
                    kk > 0 ? 1u : 0u);
            }
            commit(bar);
            ++nA;
        }
        if (half == 0) {
            if (!bar_wait(bar, (cA + 2) & 1u, kMmaWaitNs)) bad = true;
            fence_after();
            float d0, d1;
            tmem_ld2(tmem + ((uint32_t)(quad * 32) << 16), d0, d1);
            if (valid) {
                const float y0 = 1.f / (1.f + __expf(-(d0 + b30)));
                const float y1 = 1.f / (1.f + __expf(-(d1 + b31)));
                if (A.y) *reinterpret_cast<float2 *>(A.y + 2 * (size_t)r) = make_float2(y0, y1);
                if (A.out) {
                    const bool learned = A.coin[r] < A.frac;
                    const float2 u = *reinterpret_cast<const float2 *>(A.uniform_xy + 2 * (size_t)r);
                    *reinterpret_cast<float2 *>(A.out + 2 * (size_t)r) =
                        learned ? make_float2(y0, y1) : u;
                }
            }
        }
        cA += 3;
        cB += 2;
        // this tile's TMEM reads and shared-memory use end before the next MMAs
        fence_before();
        if (__syncthreads_or(bad)) break;
    }
    // a wait expired somewhere: record it and give the MMAs in flight (the
    // last commit to each barrier) a bounded time more before the tensor
    // memory is released
    const int any_bad = __syncthreads_or(bad);
    if (any_bad && tid == 0) {
        atomicOr(A.status, kErrTimeout);
        if (nA > 0) bar_wait(bar, (nA - 1) & 1u, kMmaWaitNs);
        if (nB > 0) bar_wait(bar + 1, (nB - 1) & 1u, kMmaWaitNs);
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}

}  // namespace tc
}  // namespace mlp
}  // namespace pirrt
