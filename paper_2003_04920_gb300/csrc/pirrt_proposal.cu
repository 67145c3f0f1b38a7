// Host runtime and C ABI of the learned sampling proposal (see
// mlp_kernels.cuh for the network and its training rule).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "mlp_kernels.cuh"
#include "mlp_tc.cuh"
#include "pirrt.h"

using namespace pirrt::mlp;

namespace {

// Packed parameter layout (FP32): W1g [256 x 4096], W1n [256 x 8], b1 [256],
// W2 [256 x 256], b2 [256], W3 [2 x 256], b3 [2].
constexpr int64_t oW1g = 0, nW1g = (int64_t)kHidden * kGrid;
constexpr int64_t oW1n = oW1g + nW1g, nW1n = (int64_t)kHidden * kNoise;
constexpr int64_t ob1 = oW1n + nW1n, nb1 = kHidden;
constexpr int64_t oW2 = ob1 + nb1, nW2 = (int64_t)kHidden * kHidden;
constexpr int64_t ob2 = oW2 + nW2, nb2 = kHidden;
constexpr int64_t oW3 = ob2 + nb2, nW3 = (int64_t)kOut * kHidden;
constexpr int64_t ob3 = oW3 + nW3, nb3 = kOut;
constexpr int64_t kParams = ob3 + nb3;  // 1,117,186

int pad64(int x) { return (x + 63) / 64 * 64; }

}  // namespace

struct pirrt_proposal {
    int device = 0;
    cudaStream_t stream = nullptr;
    int max_scenes = 0, max_rows = 0, S = 0, R = 0;  // padded capacities
    float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    __nv_bfloat16 *W1gb = nullptr, *W2b = nullptr, *W2Tb = nullptr, *W3b = nullptr;
    __nv_bfloat16 *gridb = nullptr, *gridT = nullptr;  // [S x 4096], [4096 x S]
    float *hg = nullptr;                                // [S x 256]
    float *a1 = nullptr, *a2 = nullptr, *dh1 = nullptr, *da2f = nullptr;  // [R x 256]
    __nv_bfloat16 *h1 = nullptr, *h1T = nullptr, *h2 = nullptr, *da2b = nullptr, *da2T = nullptr;
    float *y = nullptr;                                 // [R x 2]
    float *D = nullptr;                                 // [S x 256]
    __nv_bfloat16 *DT = nullptr;                        // [256 x S]
    float *loss = nullptr;
    int32_t *draw_scene = nullptr, *pick = nullptr;  // [R], [R]
    float *zsel = nullptr;                           // [R x 8]
    float *hgb = nullptr;                            // [S x 256]: W1g grid + b1
    int *status = nullptr;                           // fused kernel's error bits
    int64_t adam_t = 0;
    int num_sms = 0;
    int forward_kernel = PIRRT_MLP_FORWARD_TCGEN05;
    int keep_activations = 0;
    int last_rows = 0;       // rows of the last forward pass
    int last_has_acts = 0;   // whether that pass left h1 / h2 in HBM
    cudaEvent_t kev[2] = {nullptr, nullptr};  // around the last fused kernel
    int kev_recorded = 0;
};

namespace {

#define PCK(call)                                    \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) {                     \
            cudaGetLastError();                      \
            return e_ == cudaErrorMemoryAllocation ? PIRRT_ERR_OOM : PIRRT_ERR_CUDA; \
        }                                            \
    } while (0)

int blocks_for(int64_t n) {
    int64_t b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

pirrt_status gemm(pirrt_proposal *P, int M, int N, int K, const __nv_bfloat16 *A, int lda,
                  const __nv_bfloat16 *B, int ldb, float *C, int ldc, int beta) {
    dim3 grid(M / kGT, N / kGT);
    gemm_nt_bf16<<<grid, 128, 0, P->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, beta);
    PCK(cudaGetLastError());
    return PIRRT_OK;
}

// Refresh the BF16 working copies from the FP32 master weights.
pirrt_status refresh_bf16(pirrt_proposal *P) {
    to_bf16<<<blocks_for(nW1g), 256, 0, P->stream>>>(kHidden, kGrid, P->w + oW1g, kGrid, P->W1gb,
                                                     kGrid, nullptr, 0);
    to_bf16<<<blocks_for(nW2), 256, 0, P->stream>>>(kHidden, kHidden, P->w + oW2, kHidden, P->W2b,
                                                    kHidden, P->W2Tb, kHidden);
    to_bf16<<<blocks_for(nW3), 256, 0, P->stream>>>(kOut, kHidden, P->w + oW3, kHidden, P->W3b,
                                                    kHidden, nullptr, 0);
    PCK(cudaGetLastError());
    return PIRRT_OK;
}

// Grid part of layer 1 for the scenes: hg = grid W1g^T (BF16 in, FP32 out).
pirrt_status scene_features(pirrt_proposal *P, int n_scenes, const float *grids) {
    if (n_scenes < 1 || n_scenes > P->max_scenes) return PIRRT_ERR_CAPACITY;
    const int Sp = pad64(n_scenes);
    PCK(cudaMemsetAsync(P->gridb, 0, sizeof(__nv_bfloat16) * (size_t)Sp * kGrid, P->stream));
    PCK(cudaMemsetAsync(P->gridT, 0, sizeof(__nv_bfloat16) * (size_t)kGrid * Sp, P->stream));
    to_bf16<<<blocks_for((int64_t)n_scenes * kGrid), 256, 0, P->stream>>>(
        n_scenes, kGrid, grids, kGrid, P->gridb, kGrid, P->gridT, Sp);
    PCK(cudaGetLastError());
    return gemm(P, Sp, kHidden, kGrid, P->gridb, kGrid, P->W1gb, kGrid, P->hg, kHidden, 0);
}

// Rows through the network (after scene_features): y for `rows` samples.
pirrt_status forward_rows(pirrt_proposal *P, int rows, const int32_t *scene, const float *z) {
    if (rows < 1 || rows > P->max_rows) return PIRRT_ERR_CAPACITY;
    const int Rp = pad64(rows);
    layer1_rows<<<blocks_for((int64_t)Rp * kHidden), 256, 0, P->stream>>>(
        rows, Rp, P->hg, scene, z, P->w + oW1n, P->w + ob1, P->a1, P->h1, P->h1T);
    PCK(cudaGetLastError());
    pirrt_status rc = gemm(P, Rp, kHidden, kHidden, P->h1, kHidden, P->W2b, kHidden, P->a2, kHidden, 0);
    if (rc) return rc;
    bias_relu<<<blocks_for((int64_t)Rp * kHidden), 256, 0, P->stream>>>(rows, Rp, P->a2, P->w + ob2,
                                                                         P->h2, nullptr);
    layer3_rows<<<blocks_for((int64_t)rows * 32), 256, 0, P->stream>>>(rows, P->h2, P->W3b,
                                                                        P->w + ob3, P->y);
    PCK(cudaGetLastError());
    return PIRRT_OK;
}

// hgb[s][j] = hg[s][j] + b1[j]: the per-scene part of layer 1 (the first
// addition of the layered path's layer-1 sum, in the same order)
__global__ void scene_bias(int n_scenes, const float *__restrict__ hg, const float *__restrict__ b1,
                           float *__restrict__ hgb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_scenes * kHidden;
         i += gridDim.x * blockDim.x)
        hgb[i] = hg[i] + b1[i % kHidden];
}

// The fused tcgen05 forward pass over `rows` rows (after scene_features):
// y and / or the mixture `out` (see tc::FwdArgs).  The error bits are read
// after the caller's stream synchronisation (read_status).
pirrt_status forward_fused(pirrt_proposal *P, int n_scenes, int rows, const int32_t *scene,
                           const float *z, float *y, const float *uniform_xy, const float *coin,
                           float frac, float *out) {
    if (rows < 1 || rows > P->max_rows) return PIRRT_ERR_CAPACITY;
    if (reinterpret_cast<uintptr_t>(z) % 16 || reinterpret_cast<uintptr_t>(y) % 8 ||
        reinterpret_cast<uintptr_t>(out) % 8 || reinterpret_cast<uintptr_t>(uniform_xy) % 8)
        return PIRRT_ERR_INVALID_ARG;
    PCK(cudaMemsetAsync(P->status, 0, sizeof(int), P->stream));
    scene_bias<<<blocks_for((int64_t)n_scenes * kHidden), 256, 0, P->stream>>>(n_scenes, P->hg,
                                                                              P->w + ob1, P->hgb);
    PCK(cudaGetLastError());
    tc::FwdArgs a{};
    a.rows = rows;
    a.n_scenes = n_scenes;
    a.hgb = P->hgb;
    a.scene = scene;
    a.z = z;
    a.W1n = P->w + oW1n;
    a.W2b = P->W2b;
    a.b2 = P->w + ob2;
    a.W3b = P->W3b;
    a.b3 = P->w + ob3;
    a.y = y;
    a.uniform_xy = uniform_xy;
    a.coin = coin;
    a.frac = frac;
    a.out = out;
    a.cap_h1 = P->keep_activations ? P->h1 : nullptr;
    a.cap_h2 = P->keep_activations ? P->h2 : nullptr;
    a.status = P->status;
    const int tiles = (rows + tc::kRowsPerTile - 1) / tc::kRowsPerTile;
    const int grid = tiles < P->num_sms ? tiles : P->num_sms;
    PCK(cudaEventRecord(P->kev[0], P->stream));
    tc::mlp_forward_tc<<<grid, tc::kThreads, tc::kSmemBytes, P->stream>>>(a);
    PCK(cudaGetLastError());
    PCK(cudaEventRecord(P->kev[1], P->stream));
    P->kev_recorded = 1;
    P->last_rows = rows;
    P->last_has_acts = P->keep_activations;
    return PIRRT_OK;
}

// Error bits of the last fused pass (call after a stream synchronisation).
pirrt_status read_status(pirrt_proposal *P) {
    int st = 0;
    PCK(cudaMemcpy(&st, P->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st & tc::kErrTimeout) return PIRRT_ERR_DEVICE_TIMEOUT;
    if (st & tc::kErrScene) return PIRRT_ERR_BAD_INPUT;
    return PIRRT_OK;
}

// The forward pass of `rows` rows by the selected kernel into y (P->y if
// null); a mixture into `out` when given.
pirrt_status forward_any(pirrt_proposal *P, int n_scenes, int rows, const int32_t *scene,
                         const float *z, float *y, const float *uniform_xy, const float *coin,
                         float frac, float *out) {
    if (P->forward_kernel == PIRRT_MLP_FORWARD_TCGEN05)
        return forward_fused(P, n_scenes, rows, scene, z, y ? y : P->y, uniform_xy, coin, frac,
                             out);
    pirrt_status rc = forward_rows(P, rows, scene, z);
    if (rc) return rc;
    PCK(cudaMemsetAsync(P->status, 0, sizeof(int), P->stream));
    P->last_rows = rows;
    P->last_has_acts = 1;
    if (y && y != P->y)
        PCK(cudaMemcpyAsync(y, P->y, sizeof(float) * kOut * (size_t)rows, cudaMemcpyDeviceToDevice,
                            P->stream));
    if (out) {
        mix_samples<<<blocks_for(rows), 256, 0, P->stream>>>(rows, P->y, uniform_xy, coin, frac, out);
        PCK(cudaGetLastError());
    }
    return PIRRT_OK;
}

void free_all(pirrt_proposal *P) {
    void *bufs[] = {P->w, P->m, P->v, P->grad, P->W1gb, P->W2b, P->W2Tb, P->W3b, P->gridb,
                    P->gridT, P->hg, P->a1, P->a2, P->dh1, P->da2f, P->h1, P->h1T, P->h2,
                    P->da2b, P->da2T, P->y, P->D, P->DT, P->loss, P->draw_scene, P->pick, P->zsel,
                    P->hgb, P->status};
    for (void *b : bufs)
        if (b) cudaFree(b);
    for (cudaEvent_t &e : P->kev)
        if (e) cudaEventDestroy(e);
}

// splitmix64: a counter-based generator for the initial weights
uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int64_t pirrt_proposal_num_params(void) { return kParams; }

pirrt_status pirrt_proposal_create(int32_t max_scenes, int32_t max_rows, uint64_t seed,
                                   int32_t device, void *stream, pirrt_proposal **out) {
    if (!out) return PIRRT_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_scenes < 1 || max_rows < 1) return PIRRT_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return PIRRT_ERR_CUDA;
    pirrt_proposal *P = new (std::nothrow) pirrt_proposal();
    if (!P) return PIRRT_ERR_OOM;
    P->device = device;
    P->stream = static_cast<cudaStream_t>(stream);
    P->max_scenes = max_scenes;
    P->max_rows = max_rows;
    const size_t S = (size_t)pad64(max_scenes), R = (size_t)pad64(max_rows);
    P->S = (int)S;
    P->R = (int)R;
    auto bail = [&](pirrt_status s) {
        free_all(P);
        delete P;
        return s;
    };
#define PA(ptr, bytes)                                                      \
    do {                                                                    \
        if (cudaMalloc((void **)&(ptr), (bytes)) != cudaSuccess) {          \
            cudaGetLastError();                                             \
            return bail(PIRRT_ERR_OOM);                                     \
        }                                                                   \
        if (cudaMemset((ptr), 0, (bytes)) != cudaSuccess) return bail(PIRRT_ERR_CUDA); \
    } while (0)
    const size_t bf = sizeof(__nv_bfloat16), f = sizeof(float);
    PA(P->w, f * kParams);
    PA(P->m, f * kParams);
    PA(P->v, f * kParams);
    PA(P->grad, f * kParams);
    PA(P->W1gb, bf * nW1g);
    PA(P->W2b, bf * nW2);
    PA(P->W2Tb, bf * nW2);
    PA(P->W3b, bf * nW3);
    PA(P->gridb, bf * S * kGrid);
    PA(P->gridT, bf * S * kGrid);
    PA(P->hg, f * S * kHidden);
    PA(P->a1, f * R * kHidden);
    PA(P->a2, f * R * kHidden);
    PA(P->dh1, f * R * kHidden);
    PA(P->da2f, f * R * kHidden);
    PA(P->h1, bf * R * kHidden);
    PA(P->h1T, bf * R * kHidden);
    PA(P->h2, bf * R * kHidden);
    PA(P->da2b, bf * R * kHidden);
    PA(P->da2T, bf * R * kHidden);
    PA(P->y, f * R * kOut);
    PA(P->D, f * S * kHidden);
    PA(P->DT, bf * S * kHidden);
    PA(P->loss, f * 4);
    PA(P->draw_scene, sizeof(int32_t) * R);
    PA(P->pick, sizeof(int32_t) * R);
    PA(P->zsel, f * R * kNoise);
    PA(P->hgb, f * S * kHidden);
    PA(P->status, sizeof(int));
#undef PA
    if (cudaEventCreate(&P->kev[0]) != cudaSuccess || cudaEventCreate(&P->kev[1]) != cudaSuccess ||
        cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        cudaFuncSetAttribute(tc::mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             tc::kSmemBytes) != cudaSuccess) {
        cudaGetLastError();
        return bail(PIRRT_ERR_CUDA);
    }
    // He-uniform initial weights (fan-in of each layer), zero biases
    std::vector<float> h(kParams, 0.f);
    uint64_t st = seed;
    auto uni = [&](float lim) {
        const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
        return (float)((2.0 * u - 1.0) * lim);
    };
    const float l1 = std::sqrt(6.f / (kGrid + kNoise)), l2 = std::sqrt(6.f / kHidden);
    for (int64_t i = 0; i < nW1g; ++i) h[oW1g + i] = uni(l1);
    for (int64_t i = 0; i < nW1n; ++i) h[oW1n + i] = uni(l1);
    for (int64_t i = 0; i < nW2; ++i) h[oW2 + i] = uni(l2);
    for (int64_t i = 0; i < nW3; ++i) h[oW3 + i] = uni(l2);
    if (cudaMemcpy(P->w, h.data(), f * kParams, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    if (refresh_bf16(P) != PIRRT_OK || cudaStreamSynchronize(P->stream) != cudaSuccess)
        return bail(PIRRT_ERR_CUDA);
    *out = P;
    return PIRRT_OK;
}

void pirrt_proposal_destroy(pirrt_proposal *P) {
    if (!P) return;
    cudaSetDevice(P->device);
    cudaStreamSynchronize(P->stream);
    free_all(P);
    delete P;
}

pirrt_status pirrt_proposal_set_weights(pirrt_proposal *P, const float *w, int64_t n) {
    if (!P || !w || n != kParams) return PIRRT_ERR_INVALID_ARG;
    PCK(cudaMemcpyAsync(P->w, w, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, P->stream));
    PCK(cudaMemsetAsync(P->m, 0, sizeof(float) * kParams, P->stream));
    PCK(cudaMemsetAsync(P->v, 0, sizeof(float) * kParams, P->stream));
    PCK(cudaMemsetAsync(P->grad, 0, sizeof(float) * kParams, P->stream));
    P->adam_t = 0;
    pirrt_status rc = refresh_bf16(P);
    if (rc) return rc;
    PCK(cudaStreamSynchronize(P->stream));
    return PIRRT_OK;
}

pirrt_status pirrt_proposal_get_weights(const pirrt_proposal *P, float *w, int64_t n) {
    if (!P || !w || n != kParams) return PIRRT_ERR_INVALID_ARG;
    PCK(cudaMemcpyAsync(w, P->w, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, P->stream));
    PCK(cudaStreamSynchronize(P->stream));
    return PIRRT_OK;
}

pirrt_status pirrt_proposal_get_grads(const pirrt_proposal *P, float *g, int64_t n) {
    if (!P || !g || n != kParams) return PIRRT_ERR_INVALID_ARG;
    PCK(cudaMemcpyAsync(g, P->grad, sizeof(float) * kParams, cudaMemcpyDeviceToDevice, P->stream));
    PCK(cudaStreamSynchronize(P->stream));
    return PIRRT_OK;
}

pirrt_status pirrt_proposal_forward(pirrt_proposal *P, int32_t n_scenes, const float *grids,
                                    int32_t rows, const int32_t *scene, const float *noise,
                                    float *out_xy) {
    if (!P || !grids || !scene || !noise || !out_xy) return PIRRT_ERR_INVALID_ARG;
    PCK(cudaSetDevice(P->device));
    pirrt_status rc = scene_features(P, n_scenes, grids);
    if (rc) return rc;
    if ((rc = forward_any(P, n_scenes, rows, scene, noise, out_xy, nullptr, nullptr, 0.f,
                          nullptr)))
        return rc;
    PCK(cudaStreamSynchronize(P->stream));
    return read_status(P);
}

pirrt_status pirrt_proposal_sample(pirrt_proposal *P, int32_t n_scenes, const float *grids,
                                   int32_t rows, const int32_t *scene, const float *noise,
                                   const float *uniform_xy, const float *coin,
                                   float learned_fraction, float *out_xy) {
    if (!P || !grids || !scene || !noise || !uniform_xy || !coin || !out_xy ||
        !(learned_fraction >= 0.f && learned_fraction <= 1.f))
        return PIRRT_ERR_INVALID_ARG;
    PCK(cudaSetDevice(P->device));
    pirrt_status rc = scene_features(P, n_scenes, grids);
    if (rc) return rc;
    if ((rc = forward_any(P, n_scenes, rows, scene, noise, nullptr, uniform_xy, coin,
                          learned_fraction, out_xy)))
        return rc;
    PCK(cudaStreamSynchronize(P->stream));
    return read_status(P);
}

pirrt_status pirrt_proposal_imle_select(pirrt_proposal *P, int32_t n_scenes, const float *grids,
                                        int32_t n_targets, const int32_t *draw_scene,
                                        const float *targets, int32_t K, const float *noise,
                                        int32_t *pick) {
    if (!P || !grids || !draw_scene || !targets || !noise || !pick || K < 1 || n_targets < 1)
        return PIRRT_ERR_INVALID_ARG;
    PCK(cudaSetDevice(P->device));
    if ((int64_t)n_targets * K > P->max_rows) return PIRRT_ERR_CAPACITY;
    pirrt_status rc = scene_features(P, n_scenes, grids);
    if (rc) return rc;
    if ((rc = forward_any(P, n_scenes, n_targets * K, draw_scene, noise, nullptr, nullptr, nullptr,
                          0.f, nullptr)))
        return rc;
    imle_select<<<blocks_for(n_targets), 256, 0, P->stream>>>(n_targets, K, P->y, targets, pick);
    PCK(cudaGetLastError());
    PCK(cudaStreamSynchronize(P->stream));
    return read_status(P);
}

pirrt_status pirrt_proposal_backward(pirrt_proposal *P, int32_t n_scenes, const float *grids,
                                     int32_t rows, const int32_t *scene, const float *noise,
                                     const float *targets, float *loss_out) {
    if (!P || !grids || !scene || !noise || !targets) return PIRRT_ERR_INVALID_ARG;
    PCK(cudaSetDevice(P->device));
    pirrt_status rc = scene_features(P, n_scenes, grids);
    if (rc) return rc;
    if ((rc = forward_rows(P, rows, scene, noise))) return rc;
    P->last_rows = rows;
    P->last_has_acts = 1;
    const int Rp = pad64(rows), Sp = pad64(n_scenes);
    output_backward<<<kHidden, 256, 0, P->stream>>>(rows, Rp, P->y, targets, P->h2, P->W3b, P->a2,
                                                   P->grad + oW3, P->grad + ob3, P->da2b, P->da2T,
                                                   P->da2f, P->loss);
    PCK(cudaGetLastError());
    // dW2 += da2^T h1 ; db2 += sum da2 ; dh1 = da2 W2
    if ((rc = gemm(P, kHidden, kHidden, Rp, P->da2T, Rp, P->h1T, Rp, P->grad + oW2, kHidden, 1)))
        return rc;
    col_sum<<<1, kHidden, 0, P->stream>>>(rows, kHidden, P->da2f, P->grad + ob2);
    if ((rc = gemm(P, Rp, kHidden, kHidden, P->da2b, kHidden, P->W2Tb, kHidden, P->dh1, kHidden, 0)))
        return rc;
    // da1 = dh1 masked by relu(a1): per-scene sums D, dW1n, db1
    PCK(cudaMemsetAsync(P->D, 0, sizeof(float) * (size_t)Sp * kHidden, P->stream));
    layer1_backward<<<1, kHidden, 0, P->stream>>>(rows, P->dh1, P->a1, scene, noise, P->D,
                                                  P->grad + oW1n, P->grad + ob1);
    PCK(cudaGetLastError());
    // dW1g += D^T grid (BF16 D, transposed)
    PCK(cudaMemsetAsync(P->DT, 0, sizeof(__nv_bfloat16) * (size_t)Sp * kHidden, P->stream));
    to_bf16<<<blocks_for((int64_t)n_scenes * kHidden), 256, 0, P->stream>>>(
        n_scenes, kHidden, P->D, kHidden, nullptr, 0, P->DT, Sp);
    PCK(cudaGetLastError());
    if ((rc = gemm(P, kHidden, kGrid, Sp, P->DT, Sp, P->gridT, Sp, P->grad + oW1g, kGrid, 1)))
        return rc;
    if (loss_out) PCK(cudaMemcpyAsync(loss_out, P->loss, sizeof(float), cudaMemcpyDeviceToHost,
                                      P->stream));
    PCK(cudaStreamSynchronize(P->stream));
    return PIRRT_OK;
}

pirrt_status pirrt_proposal_adam(pirrt_proposal *P, float lr, float beta1, float beta2, float eps) {
    if (!P || !(lr > 0.f)) return PIRRT_ERR_INVALID_ARG;
    PCK(cudaSetDevice(P->device));
    P->adam_t += 1;
    const float bc1 = 1.f - std::pow(beta1, (float)P->adam_t);
    const float bc2 = 1.f - std::pow(beta2, (float)P->adam_t);
    struct Seg { int64_t off; int rows, cols; __nv_bfloat16 *b, *bT; int ldT; };
    const Seg segs[] = {{oW1g, kHidden, kGrid, P->W1gb, nullptr, 0},
                        {oW1n, kHidden, kNoise, nullptr, nullptr, 0},
                        {ob1, 1, kHidden, nullptr, nullptr, 0},
                        {oW2, kHidden, kHidden, P->W2b, P->W2Tb, kHidden},
                        {ob2, 1, kHidden, nullptr, nullptr, 0},
                        {oW3, kOut, kHidden, P->W3b, nullptr, 0},
                        {ob3, 1, kOut, nullptr, nullptr, 0}};
    for (const Seg &g : segs) {
        adam_step<<<blocks_for((int64_t)g.rows * g.cols), 256, 0, P->stream>>>(
            g.rows, g.cols, P->w + g.off, P->m + g.off, P->v + g.off, P->grad + g.off, lr, beta1,
            beta2, eps, bc1, bc2, g.b, g.bT, g.ldT);
    }
    PCK(cudaGetLastError());
    PCK(cudaStreamSynchronize(P->stream));
    return PIRRT_OK;
}

pirrt_status pirrt_proposal_train_step(pirrt_proposal *P, int32_t n_scenes, const float *grids,
                                       int32_t n_targets, const int32_t *target_scene,
                                       const float *targets, int32_t K, const float *noise,
                                       float lr, float *loss_out) {
    if (!P || !grids || !target_scene || !targets || !noise || K < 1 || n_targets < 1)
        return PIRRT_ERR_INVALID_ARG;
    if ((int64_t)n_targets * K > P->max_rows) return PIRRT_ERR_CAPACITY;
    PCK(cudaSetDevice(P->device));
    repeat_scene<<<blocks_for((int64_t)n_targets * K), 256, 0, P->stream>>>(n_targets, K,
                                                                           target_scene,
                                                                           P->draw_scene);
    PCK(cudaGetLastError());
    pirrt_status rc = scene_features(P, n_scenes, grids);
    if (rc) return rc;
    if ((rc = forward_any(P, n_scenes, n_targets * K, P->draw_scene, noise, nullptr, nullptr,
                          nullptr, 0.f, nullptr)))
        return rc;
    imle_select<<<blocks_for(n_targets), 256, 0, P->stream>>>(n_targets, K, P->y, targets, P->pick);
    gather_noise<<<blocks_for((int64_t)n_targets * kNoise), 256, 0, P->stream>>>(n_targets, K, noise,
                                                                                P->pick, P->zsel);
    PCK(cudaGetLastError());
    if ((rc = pirrt_proposal_backward(P, n_scenes, grids, n_targets, target_scene, P->zsel, targets,
                                      loss_out)))
        return rc;
    // the selection pass's error bits (the backward pass synchronised)
    if ((rc = read_status(P))) return rc;
    return pirrt_proposal_adam(P, lr, 0.9f, 0.999f, 1e-8f);
}

pirrt_status pirrt_proposal_set_options(pirrt_proposal *P, int32_t forward_kernel,
                                        int32_t keep_activations) {
    if (!P || (forward_kernel != PIRRT_MLP_FORWARD_TCGEN05 &&
               forward_kernel != PIRRT_MLP_FORWARD_LAYERED))
        return PIRRT_ERR_INVALID_ARG;
    P->forward_kernel = forward_kernel;
    P->keep_activations = keep_activations ? 1 : 0;
    return PIRRT_OK;
}

pirrt_status pirrt_proposal_kernel_ms(const pirrt_proposal *P, float *ms) {
    if (!P || !ms || !P->kev_recorded) return PIRRT_ERR_INVALID_ARG;
    PCK(cudaEventSynchronize(P->kev[1]));
    PCK(cudaEventElapsedTime(ms, P->kev[0], P->kev[1]));
    return PIRRT_OK;
}

pirrt_status pirrt_proposal_get_activations(const pirrt_proposal *P, int32_t rows,
                                            uint16_t *h1_out, uint16_t *h2_out) {
    if (!P || rows < 1 || rows > P->last_rows || !P->last_has_acts) return PIRRT_ERR_INVALID_ARG;
    const size_t bytes = sizeof(__nv_bfloat16) * kHidden * (size_t)rows;
    if (h1_out) PCK(cudaMemcpyAsync(h1_out, P->h1, bytes, cudaMemcpyDeviceToDevice, P->stream));
    if (h2_out) PCK(cudaMemcpyAsync(h2_out, P->h2, bytes, cudaMemcpyDeviceToDevice, P->stream));
    PCK(cudaStreamSynchronize(P->stream));
    return PIRRT_OK;
}

pirrt_status pirrt_proposal_zero_grads(pirrt_proposal *P) {
    if (!P) return PIRRT_ERR_INVALID_ARG;
    PCK(cudaMemsetAsync(P->grad, 0, sizeof(float) * kParams, P->stream));
    PCK(cudaStreamSynchronize(P->stream));
    return PIRRT_OK;
}

}  // extern "C"
