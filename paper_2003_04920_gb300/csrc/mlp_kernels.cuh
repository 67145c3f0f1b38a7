// Kernels of the learned sampling proposal: a 3-layer MLP mapping a scene's
// 64x64 occupancy grid plus 8-D Gaussian noise to a sample position,
//   a1 = W1g grid + W1n z + b1,  h1 = relu(a1)
//   a2 = W2 h1 + b2,             h2 = relu(a2)
//   y  = sigmoid(W3 h2 + b3)     in [0, 1]^2
// BF16 weights and layer inputs on the tensor cores (mma m16n8k16, FP32
// accumulate), FP32 master weights updated by Adam.  Trained by implicit
// maximum-likelihood estimation: for each target sample, K noise draws are
// pushed through the network and only the output nearest the target is
// pulled towards it (squared error).
#pragma once

#include <cuda_bf16.h>
#include <cstdint>

namespace pirrt {
namespace mlp {

constexpr int kGrid = 4096;   // 64 x 64 occupancy
constexpr int kNoise = 8;
constexpr int kHidden = 256;
constexpr int kOut = 2;

// ---------------------------------------------------------------------------
// C[M x N] (FP32, row-major, leading dim ldc) = A[M x K] * B[N x K]^T, A and
// B BF16 row-major with K contiguous ("NT").  M and N multiples of 64, K a
// multiple of 32, all leading dimensions multiples of 8 elements.  A 64 x 64
// CTA tile (M tiles along grid x, N tiles along grid y), four warps of
// 32 x 32, K in steps of 32 staged in shared memory; fragments are read with
// 32-bit shared loads in the m16n8k16 register layout.  beta = 0 overwrites
// C, 1 accumulates into it.
// ---------------------------------------------------------------------------
constexpr int kGT = 64, kGK = 32;

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128)
gemm_nt_bf16(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int lda,
             const __nv_bfloat16 *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
             int beta) {
    __shared__ __align__(16) __nv_bfloat16 sA[kGT][kGK + 8];  // +8: fewer bank conflicts
    __shared__ __align__(16) __nv_bfloat16 sB[kGT][kGK + 8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m0 = blockIdx.x * kGT, n0 = blockIdx.y * kGT;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int gid = lane >> 2, tig = lane & 3;
    float acc[2][4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kGK) {
        // 64 x 32 BF16 per operand = 256 16-byte vectors; 2 per thread each
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int idx = tid + r * 128;
            const int row = idx >> 2, col = (idx & 3) * 8;
            *reinterpret_cast<uint4 *>(&sA[row][col]) =
                *reinterpret_cast<const uint4 *>(&A[(size_t)(m0 + row) * lda + k0 + col]);
            *reinterpret_cast<uint4 *>(&sB[row][col]) =
                *reinterpret_cast<const uint4 *>(&B[(size_t)(n0 + row) * ldb + k0 + col]);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + gid;
                af[i][0] = *reinterpret_cast<const uint32_t *>(&sA[r][kk + tig * 2]);
                af[i][1] = *reinterpret_cast<const uint32_t *>(&sA[r + 8][kk + tig * 2]);
                af[i][2] = *reinterpret_cast<const uint32_t *>(&sA[r][kk + tig * 2 + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t *>(&sA[r + 8][kk + tig * 2 + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + gid;
                bf[j][0] = *reinterpret_cast<const uint32_t *>(&sB[c][kk + tig * 2]);
                bf[j][1] = *reinterpret_cast<const uint32_t *>(&sB[c][kk + tig * 2 + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = m0 + wm + i * 16 + gid, c = n0 + wn + j * 8 + tig * 2;
            float *c0 = &C[(size_t)r * ldc + c];
            float *c1 = &C[(size_t)(r + 8) * ldc + c];
            if (beta) {
                c0[0] += acc[i][j][0];
                c0[1] += acc[i][j][1];
                c1[0] += acc[i][j][2];
                c1[1] += acc[i][j][3];
            } else {
                c0[0] = acc[i][j][0];
                c0[1] = acc[i][j][1];
                c1[0] = acc[i][j][2];
                c1[1] = acc[i][j][3];
            }
        }
}

// ---------------------------------------------------------------------------
// Elementwise and small kernels.  Rows are padded to multiples of 64; padded
// rows carry zeros and are excluded by `rows` where it matters.
// ---------------------------------------------------------------------------

// FP32 -> BF16 (round to nearest even), out[r][c] for r < rows, c < cols, with
// an optional transposed copy outT[c][r] (leading dim ldt).
__global__ void to_bf16(int rows, int cols, const float *__restrict__ in, int ldi,
                        __nv_bfloat16 *__restrict__ out, int ldo, __nv_bfloat16 *__restrict__ outT,
                        int ldt) {
    const int64_t total = (int64_t)rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / cols), c = (int)(i % cols);
        const __nv_bfloat16 v = __float2bfloat16_rn(in[(size_t)r * ldi + c]);
        if (out) out[(size_t)r * ldo + c] = v;
        if (outT) outT[(size_t)c * ldt + r] = v;
    }
}

// Layer 1 for sample rows: a1[r][j] = hg[scene[r]][j] + sum_k W1n[j][k] z[r][k]
// + b1[j] (FP32; z and W1n used in their BF16-rounded values), h1 = relu(a1)
// as BF16 (row-major and transposed).
__global__ void layer1_rows(int rows, int rows_pad, const float *__restrict__ hg,
                            const int32_t *__restrict__ scene, const float *__restrict__ z,
                            const float *__restrict__ W1n, const float *__restrict__ b1,
                            float *__restrict__ a1, __nv_bfloat16 *__restrict__ h1,
                            __nv_bfloat16 *__restrict__ h1T) {
    const int64_t total = (int64_t)rows_pad * kHidden;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / kHidden), j = (int)(i % kHidden);
        float a = 0.f;
        if (r < rows) {
            a = hg[(size_t)scene[r] * kHidden + j] + b1[j];
#pragma unroll
            for (int k = 0; k < kNoise; ++k)
                a += __bfloat162float(__float2bfloat16_rn(W1n[j * kNoise + k])) *
                     __bfloat162float(__float2bfloat16_rn(z[r * kNoise + k]));
        }
        a1[i] = a;
        const __nv_bfloat16 h = __float2bfloat16_rn(r < rows && a > 0.f ? a : 0.f);
        h1[i] = h;
        if (h1T) h1T[(size_t)j * rows_pad + r] = h;
    }
}

// a2 += b2 (rows), h2 = relu(a2) as BF16.
__global__ void bias_relu(int rows, int rows_pad, float *__restrict__ a, const float *__restrict__ b,
                          __nv_bfloat16 *__restrict__ h, __nv_bfloat16 *__restrict__ hT) {
    const int64_t total = (int64_t)rows_pad * kHidden;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / kHidden), j = (int)(i % kHidden);
        const float v = r < rows ? a[i] + b[j] : 0.f;
        a[i] = v;
        const __nv_bfloat16 q = __float2bfloat16_rn(v > 0.f ? v : 0.f);
        h[i] = q;
        if (hT) hT[(size_t)j * rows_pad + r] = q;
    }
}

// Output layer (N = 2, plain dot products): y = sigmoid(W3 h2 + b3), one warp
// per row.
__global__ void layer3_rows(int rows, const __nv_bfloat16 *__restrict__ h2,
                            const __nv_bfloat16 *__restrict__ W3b, const float *__restrict__ b3,
                            float *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows;
         r += gridDim.x * (blockDim.x >> 5)) {
        float s0 = 0.f, s1 = 0.f;
        for (int j = lane; j < kHidden; j += 32) {
            const float h = __bfloat162float(h2[(size_t)r * kHidden + j]);
            s0 += h * __bfloat162float(W3b[j]);
            s1 += h * __bfloat162float(W3b[kHidden + j]);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, off);
            s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        }
        if (lane == 0) {
            y[2 * r] = 1.f / (1.f + __expf(-(s0 + b3[0])));
            y[2 * r + 1] = 1.f / (1.f + __expf(-(s1 + b3[1])));
        }
    }
}

// IMLE selection: for target t (rows t*K .. t*K+K-1 of y) the draw whose
// output is nearest the target (lowest index on ties).
__global__ void imle_select(int n_targets, int K, const float *__restrict__ y,
                            const float *__restrict__ target, int32_t *__restrict__ pick) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_targets; t += gridDim.x * blockDim.x) {
        float best = 3.4e38f;
        int bi = 0;
        for (int k = 0; k < K; ++k) {
            const float dx = y[2 * (t * K + k)] - target[2 * t];
            const float dy = y[2 * (t * K + k) + 1] - target[2 * t + 1];
            const float d = dx * dx + dy * dy;
            if (d < best) {
                best = d;
                bi = k;
            }
        }
        pick[t] = bi;
    }
}

// 50/50 (or any fraction) mixture with uniform samples: row r keeps the
// network's output when coin[r] < learned_fraction, else the caller's uniform
// sample.  The random numbers are inputs, so the mixture is reproducible.
__global__ void mix_samples(int rows, const float *__restrict__ y, const float *__restrict__ uni,
                            const float *__restrict__ coin, float learned_fraction,
                            float *__restrict__ out) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        const bool learned = coin[r] < learned_fraction;
        out[2 * r] = learned ? y[2 * r] : uni[2 * r];
        out[2 * r + 1] = learned ? y[2 * r + 1] : uni[2 * r + 1];
    }
}

// draw_scene[t*K + k] = target_scene[t]
__global__ void repeat_scene(int n_targets, int K, const int32_t *__restrict__ scene,
                             int32_t *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_targets * K; i += gridDim.x * blockDim.x)
        out[i] = scene[i / K];
}

// Gather the picked noise vectors: z_sel[t] = z_all[t*K + pick[t]].
__global__ void gather_noise(int n_targets, int K, const float *__restrict__ z_all,
                             const int32_t *__restrict__ pick, float *__restrict__ z_sel) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_targets * kNoise;
         i += gridDim.x * blockDim.x) {
        const int t = i / kNoise, k = i % kNoise;
        z_sel[i] = z_all[(size_t)(t * K + pick[t]) * kNoise + k];
    }
}

// Loss L = (1/T) sum_t |y_t - target_t|^2 and the output-layer backward:
// da3 = dL/da3 = (2/T)(y - target) y (1 - y); dW3 += da3^T h2 (FP32, exact
// sums over rows in a fixed order per output unit); db3 += sum da3;
// dh2 = da3 W3 (BF16 W3) masked by relu -> da2 (FP32 and BF16, both layouts).
// One block per hidden unit j handles dW3[:, j]; the loss is accumulated by
// block 0.
__global__ void output_backward(int rows, int rows_pad, const float *__restrict__ y,
                                const float *__restrict__ target,
                                const __nv_bfloat16 *__restrict__ h2,
                                const __nv_bfloat16 *__restrict__ W3b, const float *__restrict__ a2,
                                float *__restrict__ dW3, float *__restrict__ db3,
                                __nv_bfloat16 *__restrict__ da2b, __nv_bfloat16 *__restrict__ da2T,
                                float *__restrict__ da2f, float *__restrict__ loss) {
    const float scale = 2.f / (float)rows;
    const int j = blockIdx.x;  // hidden unit
    float s0 = 0.f, s1 = 0.f;
    for (int r = threadIdx.x; r < rows_pad; r += blockDim.x) {
        float d0 = 0.f, d1 = 0.f;
        if (r < rows) {
            const float y0 = y[2 * r], y1 = y[2 * r + 1];
            d0 = scale * (y0 - target[2 * r]) * y0 * (1.f - y0);
            d1 = scale * (y1 - target[2 * r + 1]) * y1 * (1.f - y1);
        }
        const float h = __bfloat162float(h2[(size_t)r * kHidden + j]);
        s0 += d0 * h;
        s1 += d1 * h;
        const float dh = d0 * __bfloat162float(W3b[j]) + d1 * __bfloat162float(W3b[kHidden + j]);
        const float da = (r < rows && a2[(size_t)r * kHidden + j] > 0.f) ? dh : 0.f;
        da2f[(size_t)r * kHidden + j] = da;
        const __nv_bfloat16 q = __float2bfloat16_rn(da);
        da2b[(size_t)r * kHidden + j] = q;
        da2T[(size_t)j * rows_pad + r] = q;
    }
    __shared__ float red[2][32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s0;
        red[1][threadIdx.x >> 5] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float t0 = 0.f, t1 = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t0 += red[0][w];
            t1 += red[1][w];
        }
        dW3[j] += t0;
        dW3[kHidden + j] += t1;
    }
    if (j == 0 && threadIdx.x == 0) {
        float l = 0.f, g0 = 0.f, g1 = 0.f;
        for (int r = 0; r < rows; ++r) {
            const float y0 = y[2 * r], y1 = y[2 * r + 1];
            const float e0 = y0 - target[2 * r], e1 = y1 - target[2 * r + 1];
            l += e0 * e0 + e1 * e1;
            g0 += scale * e0 * y0 * (1.f - y0);
            g1 += scale * e1 * y1 * (1.f - y1);
        }
        loss[0] = l / (float)rows;
        db3[0] += g0;
        db3[1] += g1;
    }
}

// Column sums: out[j] += sum_r in[r][j] (FP32), one thread per column.
__global__ void col_sum(int rows, int cols, const float *__restrict__ in, float *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += in[(size_t)r * cols + j];
    out[j] += s;
}

// dh1 (FP32, from the dh1 = da2 W2 GEMM) masked by relu(a1) -> da1 (FP32);
// scene sums D[s][j] += da1 for the W1 grid gradient (BF16 transposed copy
// written afterwards), dW1n += da1^T z (FP32), db1 += sum da1.  One thread
// per hidden unit j, rows in order.
__global__ void layer1_backward(int rows, const float *__restrict__ dh1, const float *__restrict__ a1,
                                const int32_t *__restrict__ scene, const float *__restrict__ z,
                                float *__restrict__ D, float *__restrict__ dW1n,
                                float *__restrict__ db1) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= kHidden) return;
    float gw[kNoise] = {};
    float gb = 0.f;
    for (int r = 0; r < rows; ++r) {
        const float d = a1[(size_t)r * kHidden + j] > 0.f ? dh1[(size_t)r * kHidden + j] : 0.f;
        D[(size_t)scene[r] * kHidden + j] += d;
        gb += d;
#pragma unroll
        for (int k = 0; k < kNoise; ++k)
            gw[k] += d * __bfloat162float(__float2bfloat16_rn(z[r * kNoise + k]));
    }
    db1[j] += gb;
#pragma unroll
    for (int k = 0; k < kNoise; ++k) dW1n[j * kNoise + k] += gw[k];
}

// Adam on FP32 master weights, then the BF16 working copy (and optionally a
// transposed BF16 copy for the backward GEMMs).  rows x cols row-major.
__global__ void adam_step(int rows, int cols, float *__restrict__ w, float *__restrict__ m,
                          float *__restrict__ v, float *__restrict__ grad, float lr, float beta1,
                          float beta2, float eps, float bc1, float bc2,
                          __nv_bfloat16 *__restrict__ wb, __nv_bfloat16 *__restrict__ wbT,
                          int ldT) {
    const int64_t total = (int64_t)rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gr = grad[i];
        const float mi = beta1 * m[i] + (1.f - beta1) * gr;
        const float vi = beta2 * v[i] + (1.f - beta2) * gr * gr;
        m[i] = mi;
        v[i] = vi;
        const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        w[i] = wi;
        grad[i] = 0.f;
        const __nv_bfloat16 q = __float2bfloat16_rn(wi);
        if (wb) wb[i] = q;
        if (wbT) {
            const int r = (int)(i / cols), c = (int)(i % cols);
            wbT[(size_t)c * ldT + r] = q;
        }
    }
}

}  // namespace mlp
}  // namespace pirrt
