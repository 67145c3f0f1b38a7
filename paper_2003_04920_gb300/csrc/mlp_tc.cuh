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
//            h2 = relu(D + b2), rounded to BF16, kept in registers
//   layer 3: y = sigmoid(W3 h2 + b3): two FP32 dot products per row on the
//            CUDA cores (N = 2 is too narrow for an MMA round trip), each
//            thread over its 128 columns, the two halves added in shared
//            memory
//
// The grid part of layer 1 (one 4096 x 256 product per scene) is computed
// once per call outside this kernel; W1g grid + b1 arrives per scene.  The
// rounding points are those of the unfused path: BF16 weights, BF16 noise,
// BF16 h1 and h2, FP32 accumulation, FP32 bias additions and sigmoid.
//
// Persistent: one CTA of 256 threads per SM (about 205 KB of shared memory:
// W2 stays resident across tiles), tiles strided over the grid.  One thread
// issues the MMAs.  Layer 2 is issued as two N = 128 halves, each committed to
// its own mbarrier, so the first half's epilogue runs while the tensor core
// computes the second; right behind them the same thread issues the next
// tile's layer 1 into the other half of a 512-column TMEM allocation (its
// noise was prefetched into registers and staged while this tile's layer-1
// epilogue ran), so a tile starts with its layer-1 result already waiting.
// Every wait is bounded; a thread whose wait expires reports it at the next
// CTA barrier (__syncthreads_or), the CTA stops, waits a bounded time more
// for its MMAs in flight, frees its tensor memory and returns with an error
// bit set.
//
// Operand layouts in shared memory (K-major, i.e. each row's K elements
// contiguous, as tcgen05 descriptors describe them):
//   * 128-byte swizzle for H and W2: 8-row groups of 8 x 128 bytes, the
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
constexpr uint32_t kTmemCols = 512;  // two 256-column accumulators (alternate tiles)
constexpr int kK1 = 16;   // layer-1 K padded to one MMA step

// shared-memory map, offsets from a 1024-byte-aligned base
constexpr int kW2Bytes = kHidden * kHidden * 2;     // 131072
constexpr int kHBytes = kRowsPerTile * kHidden * 2;  // 65536
constexpr int kZBytes = kRowsPerTile * kK1 * 2;      // 4096
constexpr int kW1Bytes = kHidden * kK1 * 2;          // 8192
constexpr int oW2 = 0;
constexpr int oH = oW2 + kW2Bytes;
constexpr int oZ = oH + kHBytes;
constexpr int oW1 = oZ + kZBytes;
constexpr int oB2 = oW1 + kW1Bytes;          // b2: 256 FP32
constexpr int oW3 = oB2 + kHidden * 4;       // BF16 W3 as FP32, column-interleaved [256][2]
constexpr int oY = oW3 + kHidden * 2 * 4;    // partial layer-3 sums [2 halves][128 rows][2]
constexpr int oBar = oY + 2 * kRowsPerTile * 2 * 4;  // mbarriers: layer-2 halves, layer 1
constexpr int oTmem = oBar + 24;             // TMEM base address written by tcgen05.alloc
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

// 64 consecutive FP32 columns of this thread's TMEM lane: two 32-column
// loads completed by one wait, which is tied to the registers so that no use
// is scheduled before it
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

// 64 packed columns (32 words) of row `row` from column c0 into the swizzled
// H, and the optional HBM copy of row r
__device__ __forceinline__ void store_h(uint8_t *sm, int row, int c0, const uint32_t *p,
                                        __nv_bfloat16 *cap, bool valid, int r) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const uint4 w = make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
        *reinterpret_cast<uint4 *>(sm + oH + sw128(row, c0 + q * 8, kRowsPerTile)) = w;
        if (cap && valid) *reinterpret_cast<uint4 *>(cap + (size_t)r * kHidden + c0 + q * 8) = w;
    }
}

// 64 packed columns (32 words) into the HBM copy of row r only
__device__ __forceinline__ void store_cap(const uint32_t *p, __nv_bfloat16 *cap, int r, int c0) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
        *reinterpret_cast<uint4 *>(cap + (size_t)r * kHidden + c0 + q * 8) =
            make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
}

// noise of row r as BF16 pairs (zeros past the last row)
__device__ __forceinline__ uint4 load_z(const float *z, int r, bool valid) {
    if (!valid) return make_uint4(0u, 0u, 0u, 0u);
    const float4 z0 = *reinterpret_cast<const float4 *>(z + (size_t)r * kNoise);
    const float4 z1 = *reinterpret_cast<const float4 *>(z + (size_t)r * kNoise + 4);
    return make_uint4(pack_bf16(z0.x, z0.y), pack_bf16(z0.z, z0.w), pack_bf16(z1.x, z1.y),
                      pack_bf16(z1.z, z1.w));
}

__global__ void __launch_bounds__(kThreads, 1) mlp_forward_tc(const FwdArgs A) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = saddr(smem_raw);
    uint8_t *sm = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t sb = saddr(sm);
    // bar[0], bar[1]: layer-2 column halves; bar[2]: layer 1
    uint64_t *bar = reinterpret_cast<uint64_t *>(sm + oBar);
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(sm + oTmem);
    float *s_b2 = reinterpret_cast<float *>(sm + oB2);
    float2 *s_w3 = reinterpret_cast<float2 *>(sm + oW3);  // (W3[0][j], W3[1][j])
    float2 *s_y = reinterpret_cast<float2 *>(sm + oY);    // [half][row]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;  // TMEM lane quadrant, column half
    const int row = quad * 32 + lane;              // row of the tile (TMEM lane)
    const int col0 = half * 128;                   // first column of this thread

    // resident operands: W2 (swizzled), W1n' (K 8..15 zero), the zero K half
    // of Z, b2, W3 (BF16 values as FP32)
    for (int i = tid; i < kHidden * (kHidden / 8); i += kThreads) {
        const int n = i >> 5, c = i & 31;
        const uint4 v = *reinterpret_cast<const uint4 *>(A.W2b + (size_t)n * kHidden + c * 8);
        *reinterpret_cast<uint4 *>(sm + oW2 + sw128(n, c * 8, kHidden)) = v;
    }
    for (int n = tid; n < kHidden; n += kThreads) {
        const float *w = A.W1n + n * kNoise;
        *reinterpret_cast<uint4 *>(sm + oW1 + plain16(n, 0)) =
            make_uint4(pack_bf16(w[0], w[1]), pack_bf16(w[2], w[3]), pack_bf16(w[4], w[5]),
                       pack_bf16(w[6], w[7]));
        *reinterpret_cast<uint4 *>(sm + oW1 + plain16(n, 1)) = make_uint4(0u, 0u, 0u, 0u);
        s_b2[n] = A.b2[n];
        s_w3[n] = make_float2(__bfloat162float(A.W3b[n]), __bfloat162float(A.W3b[kHidden + n]));
    }
    const int ntiles = (A.rows + kRowsPerTile - 1) / kRowsPerTile;
    int tile = blockIdx.x;
    if (half == 0) {
        *reinterpret_cast<uint4 *>(sm + oZ + plain16(row, 1)) = make_uint4(0u, 0u, 0u, 0u);
        const int r = tile * kRowsPerTile + row;
        *reinterpret_cast<uint4 *>(sm + oZ + plain16(row, 0)) = load_z(A.z, r, r < A.rows);
    }
    if (tid == 0) {
        for (int b = 0; b < 3; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar + b)) : "memory");
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
    const uint32_t lane_off = (uint32_t)(quad * 32) << 16;
    const float b30 = A.b3[0], b31 = A.b3[1];
    const uint32_t id128 = idesc_bf16(kRowsPerTile, 128);
    uint32_t nA = 0, nB = 0, nC = 0;  // commits issued per barrier (thread 0)
    bool bad = false;                 // a wait of this thread expired

    // layer 1 of tile `t` into accumulator `acc` (two N = 128 halves, one commit)
    auto issue_layer1 = [&](uint32_t acc) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
            mma(acc + h * 128, smem_desc(sb + oZ, 128, 256, 0),
                smem_desc(sb + oW1 + plain16(h * 128, 0), 128, 256, 0), id128, 0u);
        commit(bar + 2);
        ++nC;
    };
    if (tid == 0) issue_layer1(tmem);

    for (uint32_t it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        const uint32_t acc = tmem + (it & 1u) * 256u;  // this tile's accumulator
        const int r = tile * kRowsPerTile + row;
        const bool valid = r < A.rows;
        const int next = tile + (int)gridDim.x;
        const int rn = next * kRowsPerTile + row;
        int s = 0;
        if (valid) {
            s = A.scene[r];
            if (s < 0 || s >= A.n_scenes) {
                if (half == 0) atomicOr(A.status, kErrScene);
                s = 0;
            }
        }
        // the next tile's noise, in flight while this tile's layer 1 finishes
        uint4 zn = make_uint4(0u, 0u, 0u, 0u);
        if (half == 0 && next < ntiles) zn = load_z(A.z, rn, rn < A.rows);
        if (!bar_wait(bar + 2, it & 1u, kMmaWaitNs)) bad = true;
        fence_after();
        {
            const float *hrow = A.hgb + (size_t)s * kHidden + col0;
#pragma unroll 1
            for (int c = 0; c < 128; c += 64) {
                float v[64];
                tmem_ld64(acc + lane_off + col0 + c, v);
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
        // layer 1 of this tile is complete (waited above): stage the next noise
        if (half == 0 && next < ntiles)
            *reinterpret_cast<uint4 *>(sm + oZ + plain16(row, 0)) = zn;
        fence_async_smem();
        fence_before();
        if (__syncthreads_or(bad)) break;
        // layer 2, two column halves into this tile's accumulator; then the
        // next tile's layer 1 into the other one
        if (tid == 0) {
            fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
#pragma unroll 1
                for (int kk = 0; kk < kHidden / 16; ++kk) {
                    const uint32_t kb = kk >> 2, sub = (kk & 3) * 32;
                    mma(acc + h * 128,
                        smem_desc(sb + oH + kb * (kRowsPerTile * 128) + sub, 16, 1024, 2),
                        smem_desc(sb + oW2 + kb * (kHidden * 128) + h * 16384 + sub, 16, 1024, 2),
                        id128, kk > 0 ? 1u : 0u);
                }
                commit(bar + h);
            }
            ++nA;
            ++nB;
            if (next < ntiles) issue_layer1(tmem + ((it + 1) & 1u) * 256u);
        }
        if (!bar_wait(bar + half, it & 1u, kMmaWaitNs)) bad = true;
        fence_after();
        {
            float y0 = 0.f, y1 = 0.f;
#pragma unroll 1
            for (int c = 0; c < 128; c += 64) {
                float v[64];
                tmem_ld64(acc + lane_off + col0 + c, v);
                uint32_t p[32];
#pragma unroll
                for (int i = 0; i < 64; i += 4) {
                    const float4 b = *reinterpret_cast<const float4 *>(s_b2 + col0 + c + i);
                    const float a0 = v[i] + b.x, a1 = v[i + 1] + b.y;
                    const float a2 = v[i + 2] + b.z, a3 = v[i + 3] + b.w;
                    const uint32_t q0 = pack_bf16(a0 > 0.f ? a0 : 0.f, a1 > 0.f ? a1 : 0.f);
                    const uint32_t q1 = pack_bf16(a2 > 0.f ? a2 : 0.f, a3 > 0.f ? a3 : 0.f);
                    p[i / 2] = q0;
                    p[i / 2 + 1] = q1;
                    // layer 3 on the BF16 h2 values
                    const float h[4] = {__uint_as_float(q0 << 16), __uint_as_float(q0 & 0xFFFF0000u),
                                        __uint_as_float(q1 << 16), __uint_as_float(q1 & 0xFFFF0000u)};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float2 w = s_w3[col0 + c + i + e];
                        y0 += h[e] * w.x;
                        y1 += h[e] * w.y;
                    }
                }
                // (h2 stays in registers: the other half's layer-2 MMA may
                // still be reading h1 from H)
                if (A.cap_h2 && valid) store_cap(p, A.cap_h2, r, col0 + c);
            }
            s_y[half * kRowsPerTile + row] = make_float2(y0, y1);
        }
        // both halves' partial sums (and, before H is rewritten by the next
        // tile, both layer-2 halves) are complete past this barrier
        fence_before();
        if (__syncthreads_or(bad)) break;
        if (half == 0 && valid) {
            const float2 pa = s_y[row], pb = s_y[kRowsPerTile + row];
            const float y0 = 1.f / (1.f + __expf(-(pa.x + pb.x + b30)));
            const float y1 = 1.f / (1.f + __expf(-(pa.y + pb.y + b31)));
            if (A.y) *reinterpret_cast<float2 *>(A.y + 2 * (size_t)r) = make_float2(y0, y1);
            if (A.out) {
                const bool learned = A.coin[r] < A.frac;
                const float2 u = *reinterpret_cast<const float2 *>(A.uniform_xy + 2 * (size_t)r);
                *reinterpret_cast<float2 *>(A.out + 2 * (size_t)r) =
                    learned ? make_float2(y0, y1) : u;
            }
        }
    }
    // a wait expired somewhere: record it and give the MMAs in flight (the
    // last commit to each barrier) a bounded time more before the tensor
    // memory is released
    const int any_bad = __syncthreads_or(bad);
    if (tid == 0) {
        if (any_bad) atomicOr(A.status, kErrTimeout);
        // a layer 1 issued for a tile this CTA did not reach (never, unless
        // the loop stopped early) is waited for as well
        if (nA > 0) bar_wait(bar, (nA - 1) & 1u, kMmaWaitNs);
        if (nB > 0) bar_wait(bar + 1, (nB - 1) & 1u, kMmaWaitNs);
        if (nC > 0) bar_wait(bar + 2, (nC - 1) & 1u, kMmaWaitNs);
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
