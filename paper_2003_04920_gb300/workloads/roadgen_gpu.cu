// GPU-resident roadmap generator: seeded free-space samples, grid k-nearest
// neighbours, union-symmetrised collision-checked edges ordered by the larger
// endpoint.  Input generation only; the definitions are in roadgen_gpu.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "roadgen_gpu.h"

namespace {

constexpr int kT = 256;
constexpr int kMaxDim = 8;
constexpr int kMaxK = 128;

#define RG_CK(x)                                 \
    do {                                         \
        if ((x) != cudaSuccess) return 2;        \
    } while (0)
#define RG_CKL() RG_CK(cudaGetLastError())

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers:
// as easy as 1, 2, 3", SC 2011): ten rounds of two 32x32 -> 64-bit products,
// the key advanced by the Weyl increments between rounds.
__device__ __forceinline__ uint4 philox(uint4 x, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned hi0 = __umulhi(0xD2511F53u, x.x), lo0 = 0xD2511F53u * x.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, x.z), lo1 = 0xCD9E8D57u * x.z;
        x = make_uint4(hi1 ^ x.y ^ k.x, lo1, hi0 ^ x.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return x;
}

__device__ __forceinline__ double unit_of(unsigned x) {
    return (double)(x >> 8) * (1.0 / 16777216.0);
}

// Squared distance in FP64, coordinates in order, no fused multiply-add.
__device__ __forceinline__ double d2_64(const double *a, const double *b, int dim) {
    double s = 0.0;
    for (int d = 0; d < dim; ++d) {
        const double t = __dsub_rn(a[d], b[d]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// ---- sampling -------------------------------------------------------------

// Candidates [c0, c0 + count): coordinates and a free flag.  The inside test
// is screened in FP32 and decided exactly in FP64 near a ball's surface.
__global__ void sample_kernel(int dim, double lo, double hi, int n_obs,
                              const double *__restrict__ centers, const double *__restrict__ radii,
                              uint2 key, long long c0, long long count, double *__restrict__ pts,
                              int *__restrict__ free_flag) {
    const double span = __dsub_rn(hi, lo);
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x) {
        const unsigned long long i = (unsigned long long)(c0 + t);
        double p[kMaxDim];
        uint4 w = make_uint4(0, 0, 0, 0);
        for (int d = 0; d < dim; ++d) {
            if ((d & 3) == 0)
                w = philox(make_uint4((unsigned)i, (unsigned)(i >> 32), (unsigned)(d >> 2), 0u),
                           key);
            const unsigned x = (d & 3) == 0 ? w.x : (d & 3) == 1 ? w.y : (d & 3) == 2 ? w.z : w.w;
            p[d] = __dadd_rn(lo, __dmul_rn(span, unit_of(x)));
            pts[t * dim + d] = p[d];
        }
        bool ok = true;
        for (int s = 0; s < n_obs && ok; ++s) {
            const double *c = centers + (long long)s * dim;
            const float r2f = (float)(radii[s] * radii[s]);
            float df = 0.f;
            for (int d = 0; d < dim; ++d) {
                const float e = (float)p[d] - (float)c[d];
                df += e * e;
            }
            if (df > r2f * 1.001f + 1e-4f) continue;         // clearly outside
            if (df < r2f * 0.999f - 1e-4f) { ok = false; continue; }  // clearly inside
            const double r2 = __dmul_rn(radii[s], radii[s]);
            if (d2_64(p, c, dim) < r2) ok = false;
        }
        free_flag[t] = ok ? 1 : 0;
    }
}

// ---- scans (exclusive, int32 -> int64) ---------------------------------------

__device__ __forceinline__ long long block_scan(long long x, long long *total) {
    __shared__ long long ws[kT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        long long w = lane < kT / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kT / 32) ws[lane] = w;
    }
    __syncthreads();
    const long long base = warp > 0 ? ws[warp - 1] : 0;
    *total = ws[kT / 32 - 1];
    __syncthreads();
    return base + incl - x;
}

constexpr int kItems = 8;
constexpr int kTile = kT * kItems;

__global__ void scan_reduce(const int *__restrict__ in, long long len, long long *__restrict__ tiles) {
    const long long b = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kItems;
    long long s = 0;
    for (int i = 0; i < kItems; ++i)
        if (b + i < len) s += in[b + i];
    long long tot;
    block_scan(s, &tot);
    if (threadIdx.x == 0) tiles[blockIdx.x] = tot;
}

__global__ void scan_tiles(long long *__restrict__ tiles, long long n) {
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (long long b = 0; b < n; b += kT) {
        const long long i = b + threadIdx.x;
        const long long x = i < n ? tiles[i] : 0;
        long long tot;
        const long long ex = block_scan(x, &tot);
        if (i < n) tiles[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

__global__ void scan_apply(const int *__restrict__ in, long long len,
                           const long long *__restrict__ tiles, long long *__restrict__ out) {
    const long long b = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kItems;
    long long v[kItems], s = 0;
    for (int i = 0; i < kItems; ++i) {
        v[i] = b + i < len ? in[b + i] : 0;
        s += v[i];
    }
    long long tot;
    long long run = block_scan(s, &tot) + tiles[blockIdx.x];
    for (int i = 0; i < kItems; ++i) {
        if (b + i < len) out[b + i] = run;
        run += v[i];
    }
}

// out[i] = in[0] + ... + in[i - 1] for i in [0, len); tiles: scratch.
int exclusive_scan(const int *in, long long len, long long *out, long long *tiles, cudaStream_t st) {
    if (len <= 0) return 0;
    const long long nt = (len + kTile - 1) / kTile;
    scan_reduce<<<(unsigned)nt, kT, 0, st>>>(in, len, tiles);
    RG_CKL();
    scan_tiles<<<1, kT, 0, st>>>(tiles, nt);
    RG_CKL();
    scan_apply<<<(unsigned)nt, kT, 0, st>>>(in, len, tiles, out);
    RG_CKL();
    return 0;
}

__global__ void compact_free(long long count, int dim, const double *__restrict__ cand,
                             const int *__restrict__ flag, const long long *__restrict__ pos,
                             long long want, double *__restrict__ out) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
         t += (long long)gridDim.x * blockDim.x) {
        if (!flag[t] || pos[t] >= want) continue;
        for (int d = 0; d < dim; ++d) out[pos[t] * dim + d] = cand[t * dim + d];
    }
}

int grid_of(long long work) {
    long long b = (work + kT - 1) / kT;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

// ---- grid k-nearest neighbours ---------------------------------------------

struct Grid {
    int dim, G;
    double lo, cw;
};

__device__ __forceinline__ int cell_coord(const Grid &g, float x) {
    int c = (int)floor(((double)x - g.lo) / g.cw);
    return c < 0 ? 0 : (c >= g.G ? g.G - 1 : c);
}

__global__ void cell_count(long long n, Grid g, const double *__restrict__ pts,
                           long long *__restrict__ cell_of, int *__restrict__ cnt) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        long long id = 0, mul = 1;
        for (int d = 0; d < g.dim; ++d) {
            id += (long long)cell_coord(g, (float)pts[i * g.dim + d]) * mul;
            mul *= g.G;
        }
        cell_of[i] = id;
        atomicAdd(&cnt[id], 1);
    }
}

__global__ void cell_scatter(long long n, int dim, const double *__restrict__ pts,
                             const long long *__restrict__ cell_of,
                             const long long *__restrict__ start, int *__restrict__ cursor,
                             float *__restrict__ spts, int *__restrict__ sid) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long c = cell_of[i];
        const long long s = start[c] + atomicAdd(&cursor[c], 1);
        sid[s] = (int)i;
        for (int d = 0; d < dim; ++d) spts[s * dim + d] = (float)pts[i * dim + d];
    }
}

// FP32 squared distance, coordinates in order, no fused multiply-add.
__device__ __forceinline__ float d2_32(const float *a, const float *b, int dim) {
    float s = 0.f;
    for (int d = 0; d < dim; ++d) {
        const float t = __fsub_rn(a[d], b[d]);
        s = __fadd_rn(s, __fmul_rn(t, t));
    }
    return s;
}

// The k smallest (d2, id) among the grid's points with id < id_limit, other
// than qid itself, kept sorted in bd / bi; returns how many were found (k
// unless fewer candidates exist).  Cells are scanned by growing boxes of cells
// around the query's cell until the box holds the ball of the k-th distance;
// a cell whose box lies farther than the k-th distance is skipped.
__device__ int knn_search(const Grid &g, int k, const float *q, int qid, int id_limit,
                          const float *__restrict__ spts, const int *__restrict__ sid,
                          const long long *__restrict__ start, float *bd, int *bi) {
    const int dim = g.dim;
    int qc[kMaxDim];
    for (int d = 0; d < dim; ++d) qc[d] = cell_coord(g, q[d]);
    int cnt = 0;
    int slo[kMaxDim], shi[kMaxDim];
    bool scanned = false;
    for (int r = 1;; ++r) {
        int blo[kMaxDim], bhi[kMaxDim];
        if (cnt < k) {
            for (int d = 0; d < dim; ++d) {
                blo[d] = max(0, qc[d] - r);
                bhi[d] = min(g.G - 1, qc[d] + r);
            }
        } else {
            const float w = sqrtf(bd[k - 1]) * 1.0001f + 1e-6f;
            for (int d = 0; d < dim; ++d) {
                blo[d] = cell_coord(g, q[d] - w);
                bhi[d] = cell_coord(g, q[d] + w);
            }
        }
        bool same = scanned;
        if (scanned)
            for (int d = 0; d < dim; ++d) {
                blo[d] = min(blo[d], slo[d]);
                bhi[d] = max(bhi[d], shi[d]);
                same = same && blo[d] == slo[d] && bhi[d] == shi[d];
            }
        if (same && cnt == k) break;
        bool whole = true;
        for (int d = 0; d < dim; ++d) whole = whole && blo[d] == 0 && bhi[d] == g.G - 1;
        if (same && whole) break;  // every candidate seen: fewer than k exist
        // every cell of the box that the previous box did not hold
        int c[kMaxDim];
        for (int d = 0; d < dim; ++d) c[d] = blo[d];
        for (;;) {
            bool inside_old = scanned;
            long long id = 0, mul = 1;
            float box = 0.f;
            for (int d = 0; d < dim; ++d) {
                inside_old = inside_old && c[d] >= slo[d] && c[d] <= shi[d];
                id += (long long)c[d] * mul;
                mul *= g.G;
                const float a0 = (float)(g.lo + c[d] * g.cw), a1 = (float)(g.lo + (c[d] + 1) * g.cw);
                const float e = q[d] < a0 ? a0 - q[d] : (q[d] > a1 ? q[d] - a1 : 0.f);
                box += e * e;
            }
            const bool prune = cnt == k && box > bd[k - 1] * 1.0001f + 1e-6f;
            if (!inside_old && !prune) {
                for (long long p = start[id]; p < start[id + 1]; ++p) {
                    const int pid = sid[p];
                    if (pid == qid || pid >= id_limit) continue;
                    const float dd = d2_32(q, spts + p * dim, dim);
                    if (cnt == k && (dd > bd[k - 1] || (dd == bd[k - 1] && pid > bi[k - 1])))
                        continue;
                    int at = cnt < k ? cnt : k - 1;
                    while (at > 0 && (bd[at - 1] > dd || (bd[at - 1] == dd && bi[at - 1] > pid))) {
                        bd[at] = bd[at - 1];
                        bi[at] = bi[at - 1];
                        --at;
                    }
                    bd[at] = dd;
                    bi[at] = pid;
                    if (cnt < k) ++cnt;
                }
            }
            int d = 0;
            while (d < dim && c[d] == bhi[d]) {
                c[d] = blo[d];
                ++d;
            }
            if (d == dim) break;
            ++c[d];
        }
        for (int d = 0; d < dim; ++d) {
            slo[d] = blo[d];
            shi[d] = bhi[d];
        }
        scanned = true;
    }
    return cnt;
}

// One thread per point, in cell order (neighbouring threads scan the same
// cells): the k nearest among all points.
__global__ void __launch_bounds__(kT)
knn_kernel(long long n, Grid g, int k, const float *__restrict__ spts, const int *__restrict__ sid,
           const long long *__restrict__ start, int *__restrict__ knn) {
    const int dim = g.dim;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        float q[kMaxDim];
        for (int d = 0; d < dim; ++d) q[d] = spts[s * dim + d];
        const int qid = sid[s];
        float bd[kMaxK];
        int bi[kMaxK];
        const int cnt = knn_search(g, k, q, qid, 0x7fffffff, spts, sid, start, bd, bi);
        for (int a = 0; a < k; ++a) knn[(long long)qid * k + a] = a < cnt ? bi[a] : -1;
    }
}

// The new vertices [v0, m) in the grid's cell order (positions p of the
// sorted ids with sid[p] >= v0): flags, then a compaction by their scan.
__global__ void query_flags(long long m, long long v0, const int *__restrict__ sid,
                            int *__restrict__ flag) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m;
         p += (long long)gridDim.x * blockDim.x)
        flag[p] = sid[p] >= v0 ? 1 : 0;
}

__global__ void query_compact(long long m, long long v0, const int *__restrict__ sid,
                              const long long *__restrict__ pos, int *__restrict__ qlist) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < m;
         p += (long long)gridDim.x * blockDim.x)
        if (sid[p] >= v0) qlist[pos[p]] = sid[p];
}

// Vertices [q0, q1), visited in cell order (qlist, so that neighbouring
// threads scan the same cells): the k nearest among the vertices that precede
// each one (the grid holds vertices [0, q1)), -1 where fewer exist.  Row
// i - q0 of knn.
__global__ void __launch_bounds__(kT)
knn_pred_kernel(long long q0, long long q1, Grid g, int k, const double *__restrict__ pts,
                const float *__restrict__ spts, const int *__restrict__ sid,
                const long long *__restrict__ start, const int *__restrict__ qlist,
                int *__restrict__ knn) {
    const int dim = g.dim;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < q1 - q0;
         t += (long long)gridDim.x * blockDim.x) {
        const long long i = qlist[t];
        float q[kMaxDim];
        for (int d = 0; d < dim; ++d) q[d] = (float)pts[i * dim + d];
        float bd[kMaxK];
        int bi[kMaxK];
        const int cnt = knn_search(g, k, q, (int)i, (int)i, spts, sid, start, bd, bi);
        for (int a = 0; a < k; ++a) knn[(i - q0) * k + a] = a < cnt ? bi[a] : -1;
    }
}

// ---- edges ------------------------------------------------------------------

// Collision of the segment [a, b] with the balls (mode 0: exact closest
// point; mode 1: n_check points).  FP32 screening by the midpoint distance
// against the radius plus the half length; FP64 decides near a ball.
__device__ bool segment_free(const double *a, const double *b, int dim, int n_obs,
                             const double *centers, const double *radii, int mode, int n_check) {
    float mid[kMaxDim];
    float half2 = 0.f;
    for (int d = 0; d < dim; ++d) {
        mid[d] = (float)(0.5 * (a[d] + b[d]));
        const float h = (float)(0.5 * (b[d] - a[d]));
        half2 += h * h;
    }
    const float half = sqrtf(half2);
    for (int s = 0; s < n_obs; ++s) {
        const double *c = centers + (long long)s * dim;
        float dm2 = 0.f;
        for (int d = 0; d < dim; ++d) {
            const float w = mid[d] - (float)c[d];
            dm2 += w * w;
        }
        const float lim = (float)radii[s] + half;
        if (dm2 > lim * lim * 1.001f + 1e-4f) continue;  // clearly clear of this ball
        const double r2 = __dmul_rn(radii[s], radii[s]);
        if (mode == 0) {
            double ab2 = 0.0, t = 0.0;
            for (int d = 0; d < dim; ++d) {
                const double e = __dsub_rn(b[d], a[d]);
                ab2 = __dadd_rn(ab2, __dmul_rn(e, e));
                t = __dadd_rn(t, __dmul_rn(__dsub_rn(c[d], a[d]), e));
            }
            t = ab2 > 0.0 ? __ddiv_rn(t, ab2) : 0.0;
            t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
            double s2 = 0.0;
            for (int d = 0; d < dim; ++d) {
                const double pd = __dsub_rn(__dadd_rn(a[d], __dmul_rn(t, __dsub_rn(b[d], a[d]))), c[d]);
                s2 = __dadd_rn(s2, __dmul_rn(pd, pd));
            }
            if (s2 < r2) return false;
        } else {
            for (int i = 0; i < n_check; ++i) {
                const double t = n_check > 1 ? __ddiv_rn((double)i, (double)(n_check - 1)) : 0.0;
                double s2 = 0.0;
                for (int d = 0; d < dim; ++d) {
                    const double pd = __dsub_rn(__dadd_rn(a[d], __dmul_rn(t, __dsub_rn(b[d], a[d]))), c[d]);
                    s2 = __dadd_rn(s2, __dmul_rn(pd, pd));
                }
                if (s2 < r2) return false;
            }
        }
    }
    return true;
}

// Row i's links that row i owns (i < j, or i > j and i not in row j) and that
// are collision-free with a positive length: keep flags and a count per row.
__global__ void edge_mark(long long n, int dim, const double *__restrict__ pts, int k,
                          const int *__restrict__ knn, int n_obs, const double *__restrict__ centers,
                          const double *__restrict__ radii, int mode, int n_check,
                          unsigned char *__restrict__ keep, int *__restrict__ rowc) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        int c = 0;
        for (int a = 0; a < k; ++a) {
            const int j = knn[i * k + a];
            bool own = j >= 0 && j != i;
            if (own && j < i)
                for (int b = 0; b < k; ++b)
                    if (knn[(long long)j * k + b] == (int)i) {
                        own = false;
                        break;
                    }
            if (own) {
                const double *pa = pts + (long long)min((long long)j, i) * dim;
                const double *pb = pts + (long long)max((long long)j, i) * dim;
                own = d2_64(pa, pb, dim) > 0.0 &&
                      segment_free(pa, pb, dim, n_obs, centers, radii, mode, n_check);
            }
            keep[i * k + a] = own ? 1 : 0;
            c += own ? 1 : 0;
        }
        rowc[i] = c;
    }
}

template <typename CT>
__global__ void edge_emit(long long n, int dim, const double *__restrict__ pts, int k,
                          const int *__restrict__ knn, const unsigned char *__restrict__ keep,
                          const long long *__restrict__ rowoff, int *__restrict__ eu,
                          int *__restrict__ ev, CT *__restrict__ ec, int *__restrict__ vcnt) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        long long at = rowoff[i];
        for (int a = 0; a < k; ++a) {
            if (!keep[i * k + a]) continue;
            const int j = knn[i * k + a];
            const int u = min(j, (int)i), v = max(j, (int)i);
            eu[at] = u;
            ev[at] = v;
            ec[at] = (CT)__dsqrt_rn(d2_64(pts + (long long)u * dim, pts + (long long)v * dim, dim));
            atomicAdd(&vcnt[v], 1);
            ++at;
        }
    }
}

template <typename CT>
__global__ void edge_order(long long m, const int *__restrict__ eu, const int *__restrict__ ev,
                           const CT *__restrict__ ec, const long long *__restrict__ vstart,
                           int *__restrict__ cursor, int *__restrict__ ou, int *__restrict__ ov,
                           CT *__restrict__ oc) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m;
         e += (long long)gridDim.x * blockDim.x) {
        const int v = ev[e];
        const long long at = vstart[v] + atomicAdd(&cursor[v], 1);
        ou[at] = eu[e];
        ov[at] = v;
        oc[at] = ec[e];
    }
}

// Each vertex's group of edges sorted by the smaller endpoint (insertion sort;
// groups hold about k to 2k edges).
template <typename CT>
__global__ void group_sort(long long n, const long long *__restrict__ vstart, int *__restrict__ ou,
                           CT *__restrict__ oc) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const long long b = vstart[v], e = vstart[v + 1];
        for (long long i = b + 1; i < e; ++i) {
            const int u = ou[i];
            const CT c = oc[i];
            long long j = i;
            while (j > b && ou[j - 1] > u) {
                ou[j] = ou[j - 1];
                oc[j] = oc[j - 1];
                --j;
            }
            ou[j] = u;
            oc[j] = c;
        }
    }
}

template <typename T>
struct DevBuf {
    T *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    bool alloc(size_t count) { return cudaMalloc(&p, sizeof(T) * (count > 0 ? count : 1)) == cudaSuccess; }
};

}  // namespace

extern "C" int rgg_sample(int32_t dim, double lo, double hi, int32_t n_obs, const double *centers,
                          const double *radii, uint64_t seed, int64_t n, double *points,
                          int64_t *tried, void *stream) {
    if (dim < 1 || dim > kMaxDim || !(hi > lo) || n_obs < 0 || n < 0 || (n > 0 && !points) ||
        (n_obs > 0 && (!centers || !radii)))
        return 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint2 key = make_uint2((unsigned)seed, (unsigned)(seed >> 32));
    const long long chunk = std::max<long long>(1 << 16, std::min<long long>(1 << 22, 2 * n));
    DevBuf<double> cand;
    DevBuf<int> flag;
    DevBuf<long long> pos, tiles;
    if (!cand.alloc((size_t)chunk * dim) || !flag.alloc(chunk) || !pos.alloc(chunk) ||
        !tiles.alloc(chunk / kTile + 2))
        return 2;
    long long have = 0, c0 = 0;
    while (have < n) {
        sample_kernel<<<grid_of(chunk), kT, 0, st>>>(dim, lo, hi, n_obs, centers, radii, key, c0,
                                                     chunk, cand.p, flag.p);
        RG_CKL();
        if (int rc = exclusive_scan(flag.p, chunk, pos.p, tiles.p, st)) return rc;
        compact_free<<<grid_of(chunk), kT, 0, st>>>(chunk, dim, cand.p, flag.p, pos.p, n - have,
                                                    points + have * dim);
        RG_CKL();
        long long last = 0;
        int lastf = 0;
        RG_CK(cudaMemcpyAsync(&last, pos.p + chunk - 1, sizeof(last), cudaMemcpyDeviceToHost, st));
        RG_CK(cudaMemcpyAsync(&lastf, flag.p + chunk - 1, sizeof(lastf), cudaMemcpyDeviceToHost, st));
        RG_CK(cudaStreamSynchronize(st));
        const long long got = last + lastf;
        if (have + got >= n) {
            // the candidate that completed the set: count the draws up to it
            c0 += chunk;
            have = n;
            break;
        }
        have += got;
        c0 += chunk;
        if (c0 > (1ll << 40)) return 1;  // the box is (almost) all obstacle
    }
    if (tried) *tried = c0;
    return 0;
}

extern "C" int rgg_knn(int32_t dim, double lo, double hi, int64_t n, const double *points,
                       int32_t k, double cell, int32_t *knn, void *stream) {
    if (dim < 1 || dim > kMaxDim || !(hi > lo) || n < 2 || k < 1 || k >= n || k > kMaxK ||
        !points || !knn)
        return 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double span = hi - lo;
    if (!(cell > 0.0)) {
        // side about the k-th neighbour distance of a uniform spread
        const double unit = std::pow(M_PI, dim / 2.0) / std::tgamma(dim / 2.0 + 1.0);
        cell = std::pow((double)k * std::pow(span, dim) / ((double)n * unit), 1.0 / dim);
    }
    int G = (int)std::floor(span / cell);
    G = std::max(1, G);
    while (std::pow((double)G, dim) > (double)(1 << 24) && G > 1) --G;  // bounded cell table
    long long cells = 1;
    for (int d = 0; d < dim; ++d) cells *= G;
    Grid g{dim, G, lo, span / G};
    DevBuf<long long> cell_of, start, tiles;
    DevBuf<int> cnt, sid;
    DevBuf<float> spts;
    if (!cell_of.alloc(n) || !start.alloc(cells + 1) || !tiles.alloc((cells + 1) / kTile + 2) ||
        !cnt.alloc(cells + 1) || !sid.alloc(n) || !spts.alloc((size_t)n * dim))
        return 2;
    RG_CK(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (cells + 1), st));
    cell_count<<<grid_of(n), kT, 0, st>>>(n, g, points, cell_of.p, cnt.p);
    RG_CKL();
    if (int rc = exclusive_scan(cnt.p, cells + 1, start.p, tiles.p, st)) return rc;
    RG_CK(cudaMemsetAsync(cnt.p, 0, sizeof(int) * (cells + 1), st));
    cell_scatter<<<grid_of(n), kT, 0, st>>>(n, dim, points, cell_of.p, start.p, cnt.p, spts.p, sid.p);
    RG_CKL();
    knn_kernel<<<grid_of(n), kT, 0, st>>>(n, g, k, spts.p, sid.p, start.p, knn);
    RG_CKL();
    RG_CK(cudaStreamSynchronize(st));
    return 0;
}

extern "C" int rgg_edges(int32_t dim, int64_t n, const double *points, int32_t k,
                         const int32_t *knn, int32_t n_obs, const double *centers,
                         const double *radii, int32_t mode, int32_t n_check, int32_t cost_f64,
                         int32_t *u, int32_t *v, void *cost, int64_t *edge_start, int64_t cap,
                         int64_t *m, void *stream) {
    if (dim < 1 || dim > kMaxDim || n < 1 || k < 1 || !points || !knn || !edge_start || !m ||
        (mode != 0 && mode != 1) || (mode == 1 && n_check < 1) || n_obs < 0 ||
        (n_obs > 0 && (!centers || !radii)))
        return 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevBuf<unsigned char> keep;
    DevBuf<int> rowc, vcnt;
    DevBuf<long long> rowoff, tiles;
    if (!keep.alloc((size_t)n * k) || !rowc.alloc(n + 1) || !vcnt.alloc(n + 1) ||
        !rowoff.alloc(n + 1) || !tiles.alloc((n + 1) / kTile + 2))
        return 2;
    edge_mark<<<grid_of(n), kT, 0, st>>>(n, dim, points, k, knn, n_obs, centers, radii, mode,
                                         n_check, keep.p, rowc.p);
    RG_CKL();
    RG_CK(cudaMemsetAsync(rowc.p + n, 0, sizeof(int), st));
    if (int rc = exclusive_scan(rowc.p, n + 1, rowoff.p, tiles.p, st)) return rc;
    long long total = 0;
    RG_CK(cudaMemcpyAsync(&total, rowoff.p + n, sizeof(total), cudaMemcpyDeviceToHost, st));
    RG_CK(cudaStreamSynchronize(st));
    *m = total;
    if (total > cap || (total > 0 && (!u || !v || !cost))) return total > cap ? 3 : 1;
    DevBuf<int> tu, tv, cursor;
    DevBuf<unsigned char> tc;
    const size_t cb = cost_f64 ? sizeof(double) : sizeof(float);
    if (!tu.alloc(total) || !tv.alloc(total) || !tc.alloc((size_t)total * cb) || !cursor.alloc(n + 1))
        return 2;
    RG_CK(cudaMemsetAsync(vcnt.p, 0, sizeof(int) * (n + 1), st));
    if (cost_f64)
        edge_emit<double><<<grid_of(n), kT, 0, st>>>(n, dim, points, k, knn, keep.p, rowoff.p,
                                                     tu.p, tv.p, reinterpret_cast<double *>(tc.p),
                                                     vcnt.p);
    else
        edge_emit<float><<<grid_of(n), kT, 0, st>>>(n, dim, points, k, knn, keep.p, rowoff.p,
                                                    tu.p, tv.p, reinterpret_cast<float *>(tc.p),
                                                    vcnt.p);
    RG_CKL();
    long long *vstart = reinterpret_cast<long long *>(edge_start);
    if (int rc = exclusive_scan(vcnt.p, n + 1, vstart, tiles.p, st)) return rc;
    RG_CK(cudaMemsetAsync(cursor.p, 0, sizeof(int) * (n + 1), st));
    if (cost_f64) {
        edge_order<double><<<grid_of(total), kT, 0, st>>>(
            total, tu.p, tv.p, reinterpret_cast<const double *>(tc.p), vstart, cursor.p, u, v,
            static_cast<double *>(cost));
        RG_CKL();
        group_sort<double><<<grid_of(n), kT, 0, st>>>(n, vstart, u, static_cast<double *>(cost));
    } else {
        edge_order<float><<<grid_of(total), kT, 0, st>>>(
            total, tu.p, tv.p, reinterpret_cast<const float *>(tc.p), vstart, cursor.p, u, v,
            static_cast<float *>(cost));
        RG_CKL();
        group_sort<float><<<grid_of(n), kT, 0, st>>>(n, vstart, u, static_cast<float *>(cost));
    }
    RG_CKL();
    RG_CK(cudaStreamSynchronize(st));
    return 0;
}

// ---- incremental exploration ------------------------------------------------

namespace {

// Links of the new vertices [v0, v1) to their nearest predecessors that are
// collision-free with a positive length: keep flags and a count per row.
// One thread per (new vertex, link), vertices in cell order: keep flags and
// the per-row count of the collision-free, positive-length links (rowc
// cleared before).
__global__ void pred_edge_mark(long long v0, long long v1, int dim, const double *__restrict__ pts,
                               int k, const int *__restrict__ knn, const int *__restrict__ qlist,
                               int n_obs, const double *__restrict__ centers,
                               const double *__restrict__ radii, int mode, int n_check,
                               unsigned char *__restrict__ keep, int *__restrict__ rowc) {
    const long long total = (v1 - v0) * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = qlist[e / k];
        const int a = (int)(e % k);
        const long long r = i - v0;
        const int j = knn[r * k + a];
        bool ok = j >= 0;
        if (ok) {
            const double *pa = pts + (long long)j * dim, *pb = pts + i * dim;
            ok = d2_64(pa, pb, dim) > 0.0 &&
                 segment_free(pa, pb, dim, n_obs, centers, radii, mode, n_check);
        }
        keep[r * k + a] = ok ? 1 : 0;
        if (ok) atomicAdd(&rowc[r], 1);
    }
}

template <typename CT>
__global__ void pred_edge_emit(long long v0, long long v1, int dim, const double *__restrict__ pts,
                               int k, const int *__restrict__ knn,
                               const unsigned char *__restrict__ keep,
                               const long long *__restrict__ rowoff, int *__restrict__ eu,
                               int *__restrict__ ev, CT *__restrict__ ec) {
    for (long long i = v0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < v1;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i - v0;
        long long at = rowoff[r];
        for (int a = 0; a < k; ++a) {
            if (!keep[r * k + a]) continue;
            const int j = knn[r * k + a];
            eu[at] = j;
            ev[at] = (int)i;
            ec[at] = (CT)__dsqrt_rn(d2_64(pts + (long long)j * dim, pts + i * dim, dim));
            ++at;
        }
    }
}

// Grid of cells of about the k-th neighbour distance for `m` points spread
// over the box (at most 2^24 cells).
Grid grid_for_density(int dim, double lo, double hi, long long m, int k) {
    const double span = hi - lo;
    const double unit = std::pow(M_PI, dim / 2.0) / std::tgamma(dim / 2.0 + 1.0);
    const double cell =
        std::pow((double)k * std::pow(span, dim) / ((double)std::max(m, 1ll) * unit), 1.0 / dim);
    int G = std::max(1, (int)std::floor(span / cell));
    while (std::pow((double)G, dim) > (double)(1 << 24) && G > 1) --G;
    return Grid{dim, G, lo, span / G};
}

long long cells_of(const Grid &g) {
    long long c = 1;
    for (int d = 0; d < g.dim; ++d) c *= g.G;
    return c;
}

}  // namespace

struct rgg_explorer {
    int dim = 0;
    double lo = 0.0, hi = 0.0;
    int n_obs = 0, k = 0, mode = 0, n_check = 0, cost_f64 = 0;
    long long n = 0, max_block = 0, cells_max = 0;
    double *centers = nullptr, *radii = nullptr, *pts = nullptr;
    float *spts = nullptr;
    int *sid = nullptr, *cnt = nullptr, *knn = nullptr, *rowc = nullptr;
    int *qflag = nullptr, *qlist = nullptr;
    long long *cell_of = nullptr, *start = nullptr, *rowoff = nullptr, *tiles = nullptr;
    long long *qpos = nullptr;
    unsigned char *keep = nullptr;
};

extern "C" void rgg_explore_destroy(rgg_explorer *x) {
    if (!x) return;
    void *bufs[] = {x->centers, x->radii, x->pts, x->spts, x->sid, x->cnt, x->knn, x->rowc,
                    x->cell_of, x->start, x->rowoff, x->tiles, x->keep, x->qflag, x->qlist,
                    x->qpos};
    for (void *b : bufs)
        if (b) cudaFree(b);
    delete x;
}

extern "C" int rgg_explore_create(int32_t dim, double lo, double hi, int32_t n_obs,
                                  const double *centers, const double *radii, uint64_t seed,
                                  int64_t n, int32_t k, int32_t mode, int32_t n_check,
                                  int32_t cost_f64, int64_t max_block, void *stream,
                                  rgg_explorer **out) {
    if (!out) return 1;
    *out = nullptr;
    if (dim < 1 || dim > kMaxDim || !(hi > lo) || n < 2 || k < 1 || k > kMaxK || max_block < 1 ||
        (mode != 0 && mode != 1) || (mode == 1 && n_check < 1) || n_obs < 0 ||
        (n_obs > 0 && (!centers || !radii)))
        return 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rgg_explorer *x = new rgg_explorer;
    x->dim = dim;
    x->lo = lo;
    x->hi = hi;
    x->n_obs = n_obs;
    x->k = k;
    x->mode = mode;
    x->n_check = n_check;
    x->cost_f64 = cost_f64;
    x->n = n;
    x->max_block = std::min<long long>(max_block, n);
    const Grid gmax = grid_for_density(dim, lo, hi, n, k);
    x->cells_max = 1;
    for (long long m = 1; m <= n; m *= 2) x->cells_max = std::max(x->cells_max, cells_of(grid_for_density(dim, lo, hi, m, k)));
    x->cells_max = std::max(x->cells_max, cells_of(gmax));
    const long long mb = x->max_block;
    bool ok = cudaMalloc(&x->centers, sizeof(double) * std::max(1, n_obs * dim)) == cudaSuccess &&
              cudaMalloc(&x->radii, sizeof(double) * std::max(1, n_obs)) == cudaSuccess &&
              cudaMalloc(&x->pts, sizeof(double) * n * dim) == cudaSuccess &&
              cudaMalloc(&x->spts, sizeof(float) * n * dim) == cudaSuccess &&
              cudaMalloc(&x->sid, sizeof(int) * n) == cudaSuccess &&
              cudaMalloc(&x->cell_of, sizeof(long long) * n) == cudaSuccess &&
              cudaMalloc(&x->cnt, sizeof(int) * (x->cells_max + 1)) == cudaSuccess &&
              cudaMalloc(&x->start, sizeof(long long) * (x->cells_max + 1)) == cudaSuccess &&
              cudaMalloc(&x->tiles, sizeof(long long) *
                                        (std::max<long long>(x->cells_max, n) + 1 + kTile) / kTile) == cudaSuccess &&
              cudaMalloc(&x->qflag, sizeof(int) * (n + 1)) == cudaSuccess &&
              cudaMalloc(&x->qpos, sizeof(long long) * (n + 1)) == cudaSuccess &&
              cudaMalloc(&x->qlist, sizeof(int) * mb) == cudaSuccess &&
              cudaMalloc(&x->knn, sizeof(int) * mb * k) == cudaSuccess &&
              cudaMalloc(&x->keep, mb * k) == cudaSuccess &&
              cudaMalloc(&x->rowc, sizeof(int) * (mb + 1)) == cudaSuccess &&
              cudaMalloc(&x->rowoff, sizeof(long long) * (mb + 1)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        rgg_explore_destroy(x);
        return 2;
    }
    if (n_obs > 0 &&
        (cudaMemcpyAsync(x->centers, centers, sizeof(double) * n_obs * dim,
                         cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
         cudaMemcpyAsync(x->radii, radii, sizeof(double) * n_obs, cudaMemcpyDeviceToDevice, st) !=
             cudaSuccess)) {
        rgg_explore_destroy(x);
        return 2;
    }
    int64_t tried = 0;
    const int rc = rgg_sample(dim, lo, hi, n_obs, x->centers, x->radii, seed, n, x->pts, &tried, st);
    if (rc) {
        rgg_explore_destroy(x);
        return rc;
    }
    *out = x;
    return 0;
}

extern "C" int rgg_explore_block(rgg_explorer *x, int64_t v0, int64_t v1, int32_t *u, int32_t *v,
                                 void *cost, int64_t *m_pinned, void *stream) {
    if (!x || v0 < 0 || v1 <= v0 || v1 > x->n || v1 - v0 > x->max_block || !u || !v || !cost ||
        !m_pinned)
        return 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int dim = x->dim, k = x->k;
    const long long nb = v1 - v0;
    // the grid over the vertices present, [0, v1)
    const Grid g = grid_for_density(dim, x->lo, x->hi, v1, k);
    const long long cells = cells_of(g);
    if (cells > x->cells_max) return 1;
    RG_CK(cudaMemsetAsync(x->cnt, 0, sizeof(int) * (cells + 1), st));
    cell_count<<<grid_of(v1), kT, 0, st>>>(v1, g, x->pts, x->cell_of, x->cnt);
    RG_CKL();
    if (int rc = exclusive_scan(x->cnt, cells + 1, x->start, x->tiles, st)) return rc;
    RG_CK(cudaMemsetAsync(x->cnt, 0, sizeof(int) * (cells + 1), st));
    cell_scatter<<<grid_of(v1), kT, 0, st>>>(v1, dim, x->pts, x->cell_of, x->start, x->cnt,
                                             x->spts, x->sid);
    RG_CKL();
    // the new vertices in cell order
    query_flags<<<grid_of(v1), kT, 0, st>>>(v1, v0, x->sid, x->qflag);
    RG_CKL();
    if (int rc = exclusive_scan(x->qflag, v1, x->qpos, x->tiles, st)) return rc;
    query_compact<<<grid_of(v1), kT, 0, st>>>(v1, v0, x->sid, x->qpos, x->qlist);
    RG_CKL();
    // nearest predecessors of the new vertices, then their edges
    knn_pred_kernel<<<grid_of(nb), kT, 0, st>>>(v0, v1, g, k, x->pts, x->spts, x->sid, x->start,
                                                x->qlist, x->knn);
    RG_CKL();
    RG_CK(cudaMemsetAsync(x->rowc, 0, sizeof(int) * (nb + 1), st));
    pred_edge_mark<<<grid_of(nb * k), kT, 0, st>>>(v0, v1, dim, x->pts, k, x->knn, x->qlist,
                                                   x->n_obs, x->centers, x->radii, x->mode,
                                                   x->n_check, x->keep, x->rowc);
    RG_CKL();
    if (int rc = exclusive_scan(x->rowc, nb + 1, x->rowoff, x->tiles, st)) return rc;
    RG_CK(cudaMemcpyAsync(m_pinned, x->rowoff + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (x->cost_f64)
        pred_edge_emit<double><<<grid_of(nb), kT, 0, st>>>(v0, v1, dim, x->pts, k, x->knn, x->keep,
                                                           x->rowoff, u, v,
                                                           static_cast<double *>(cost));
    else
        pred_edge_emit<float><<<grid_of(nb), kT, 0, st>>>(v0, v1, dim, x->pts, k, x->knn, x->keep,
                                                          x->rowoff, u, v,
                                                          static_cast<float *>(cost));
    RG_CKL();
    return 0;
}

extern "C" const double *rgg_explore_points(const rgg_explorer *x) { return x ? x->pts : nullptr; }

extern "C" int64_t rgg_explore_size(const rgg_explorer *x) { return x ? x->n : -1; }

extern "C" int rgg_explore_copy_points(const rgg_explorer *x, double *out, void *stream) {
    if (!x || !out) return 1;
    RG_CK(cudaMemcpyAsync(out, x->pts, sizeof(double) * x->n * x->dim, cudaMemcpyDeviceToDevice,
                          static_cast<cudaStream_t>(stream)));
    return 0;
}
