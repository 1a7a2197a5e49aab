// k_entry.cu -- where a search enters the graph (a project addition: the paper draws
// the seed set B of Alg. 2 at random, and the library's attribute-entry rule takes
// evenly spaced members of the query's tuple, which for a frequent tuple lie all over
// the vector space).
//
// Coarse cells.  E centroids are the objects floor(j N / E); every object belongs to
// the cell of its nearest centroid by (delta, j) (the brute-force top-1 over the E
// centroid rows, plain L2).  The objects are also sorted by (attribute word, cell) with
// ascending ids inside, so the members of a tuple within one cell form one run.
//
// Entry rule for a query whose tuple has members P (closed queries): S = min(ef, 32, |P|);
// B = the first S members of P in the query's chosen cells (best cell first, ascending
// ids within a cell), then, while fewer than S, the evenly spaced P[floor(j |P| / S2)],
// j < S2 = S - |B|; |P| = 0 takes the random stream of NHQ_SEED_RANDOM.  The chosen
// cells are the T nearest centroids (NHQ_SEED_CELL_NEAREST) or the T best-scored cells
// of the entry model (NHQ_SEED_CELL_LEARNED).
//
// Entry model: a 2-layer perceptron, q (d values) -> x = s q -> 64 ReLU units -> E cell
// logits, fp16 weights and f32 accumulation at inference, f32 master weights for
// training (softmax cross-entropy against the cell of each training query's answer,
// Adam).  Parameters, one flat f32 vector: s | W1 [d][64] | b1 [64] | W2 [64][E] | b2 [E].
//
// Both cell rules score every cell of every query of the batch with one register-tiled
// dense kernel (64 x 64 output tiles, k ascending per output in one fma chain, so the
// seed pass and nhq_entry_forward produce the same bits): the learned rule runs the two
// layers, the nearest rule scores q.c - |c|^2 / 2 against the transposed centroids (the
// largest score is the nearest centroid; every product and sum is exact for integer
// components, where the order equals the (delta, cell) order).  A warp per query then
// takes the T best scores (ties to the smaller cell) and assembles the seeds.
#include <cub/cub.cuh>

#include "nhq_internal.cuh"

namespace nhq {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int EH = NHQ_ENTRY_HIDDEN;

struct EntryLayout {
    int64_t oW1, oB1, oW2, oB2, total;
};
__host__ __device__ inline EntryLayout entry_layout(int d, int E) {
    EntryLayout L;
    L.oW1 = 1;
    L.oB1 = L.oW1 + (int64_t)d * EH;
    L.oW2 = L.oB1 + EH;
    L.oB2 = L.oW2 + (int64_t)EH * E;
    L.total = L.oB2 + E;
    return L;
}

__global__ void gather_centroids_kernel(const float *__restrict__ X, int xstride, int64_t N,
                                        int E, const uint32_t *__restrict__ attr,
                                        float *__restrict__ cent, uint32_t *__restrict__ cattr) {
    const int j = blockIdx.x;
    const int64_t src = (int64_t)j * N / E;
    for (int i = threadIdx.x; i < xstride; i += blockDim.x)
        cent[(int64_t)j * xstride + i] = X[src * xstride + i];
    if (threadIdx.x == 0)
        cattr[j] = attr[src];
}

__global__ void cell_key_kernel(const uint32_t *__restrict__ attr, const uint32_t *__restrict__ cell,
                                int64_t N, unsigned long long *__restrict__ key,
                                uint32_t *__restrict__ iota) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N;
         v += (int64_t)gridDim.x * blockDim.x) {
        key[v] = ((unsigned long long)attr[v] << 16) | cell[v];
        iota[v] = (uint32_t)v;
    }
}

__device__ __forceinline__ int64_t lower_bound_u64(const unsigned long long *a, int64_t n,
                                                   unsigned long long x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t *a, int64_t n, uint32_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// ---- inference: Y[n][M] = act(s A[n][K] B[K][M] + bias[M]), k ascending per output ----
__device__ __forceinline__ float as_f32(float v) { return v; }
__device__ __forceinline__ float as_f32(__half v) { return __half2float(v); }

template <typename BT>
__global__ void __launch_bounds__(256) dense_kernel(const float *__restrict__ A, int64_t n, int K,
                                                    int64_t lda, const BT *__restrict__ B,
                                                    const BT *__restrict__ bias, int M,
                                                    const float *__restrict__ scale_ptr,
                                                    int relu, float *__restrict__ Y) {
    __shared__ float As[32][65];  // [k][row], padded: the tile loads are free of conflicts
    __shared__ float Bs[32][64];  // [k][col]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * 64;
    const int col0 = blockIdx.y * 64;
    const float sc = scale_ptr != nullptr ? *scale_ptr : 1.f;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            acc[i][j] = 0.f;
    for (int k0 = 0; k0 < K; k0 += 32) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = (tid >> 5) + 8 * i, kk = tid & 31;
            const int64_t gr = row0 + r;
            const int gk = k0 + kk;
            As[kk][r] = (gr < n && gk < K) ? __fmul_rn(sc, A[gr * lda + gk]) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int kk = (tid >> 6) + 4 * i, c = tid & 63;
            const int gk = k0 + kk, gc = col0 + c;
            Bs[kk][c] = (gk < K && gc < M) ? as_f32(B[(int64_t)gk * M + gc]) : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                b[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = row0 + ty * 4 + i;
        if (r >= n)
            continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = col0 + tx * 4 + j;
            if (c >= M)
                continue;
            float v = __fadd_rn(acc[i][j], as_f32(bias[c]));
            if (relu)
                v = fmaxf(v, 0.f);
            Y[r * M + c] = v;
        }
    }
}

template <typename BT>
cudaError_t launch_dense(const float *A, int64_t n, int K, int64_t lda, const BT *B,
                         const BT *bias, int M, const float *scale_ptr, int relu, float *Y,
                         cudaStream_t s) {
    if (n <= 0)
        return cudaSuccess;
    const int64_t gx = (n + 63) / 64;
    if (gx > 0x7FFFFFFF)
        return cudaErrorInvalidValue;
    dense_kernel<BT><<<dim3((unsigned)gx, (unsigned)((M + 63) / 64)), 256, 0, s>>>(
        A, n, K, lda, B, bias, M, scale_ptr, relu, Y);
    return cudaGetLastError();
}

// centroid columns for the nearest rule: cT[i][j] = cent[j][i], nh[j] = -|c_j|^2 / 2
__global__ void centroid_columns_kernel(const float *__restrict__ cent, int xstride, int d, int E,
                                        float *__restrict__ cT, float *__restrict__ nh) {
    const int j = blockIdx.x;
    for (int i = threadIdx.x; i < d; i += blockDim.x)
        cT[(int64_t)i * E + j] = cent[(int64_t)j * xstride + i];
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < d; ++i)
            s = fmaf(cent[(int64_t)j * xstride + i], cent[(int64_t)j * xstride + i], s);
        nh[j] = -0.5f * s;
    }
}

// a key whose ascending order is descending logit, then ascending cell
__device__ __forceinline__ unsigned long long logit_key(float t, int o) {
    uint32_t u = __float_as_uint(t);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);  // ascending map of the float order
    return ((unsigned long long)(~u) << 32) | (uint32_t)o;
}

__device__ __forceinline__ void topT_insert(unsigned long long *best, int T,
                                            unsigned long long k) {
    if (k >= best[T - 1])
        return;
    int i = T - 1;
    while (i > 0 && best[i - 1] > k) {
        best[i] = best[i - 1];
        --i;
    }
    best[i] = k;
}

struct CellSeedArgs {
    SearchArgs a;
    const uint32_t *attr_sorted, *id_sorted;         // tuple runs
    const unsigned long long *cell_key;              // (attribute word << 16 | cell), sorted
    const uint32_t *cell_id;                         // ids in that order
    int E, T;
    const float *scores;                             // [nq][E], the larger the better
    int32_t *cells_out;                              // [nq][T] or null
    uint32_t *seeds;                                 // [nq][32]
    uint8_t *bucket;                                 // [nq] or null
};

constexpr int kMaxT = 8;

// One warp per query: the T best cells from the query's score row, then its seeds.
__global__ void __launch_bounds__(256) cell_seeds_kernel(CellSeedArgs c) {
    const SearchArgs &a = c.a;
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= a.nq)
        return;
    const int T = c.T;
    {
        uint32_t qhi;
        const uint32_t qa = pack_query_word(a.qattr + q * a.w.m, a.w, &qhi);
        const int ef = a.ef_arr ? a.ef_arr[q] : a.ef;
        const int want = ef < 32 ? ef : 32;
        uint32_t *row = c.seeds + q * 32;
        const int64_t lo = lower_bound_u32(c.attr_sorted, a.N, qa);
        const int64_t hi = qa == 0xFFFFFFFFu ? a.N : lower_bound_u32(c.attr_sorted, a.N, qa + 1u);
        const int64_t P = hi - lo;
        if (lane == 0 && c.bucket != nullptr) {
            const int bits = 64 - __clzll((unsigned long long)P + 1ull);
            c.bucket[q] = (uint8_t)(bits >= 32 ? 0 : 32 - bits);
        }
        unsigned long long best[kMaxT];
#pragma unroll
        for (int t = 0; t < kMaxT; ++t)
            best[t] = ~0ull;
        const float *sr = c.scores + q * (int64_t)c.E;
        for (int o = lane; o < c.E; o += 32)
            topT_insert(best, T, logit_key(sr[o], o));
        int chosen[kMaxT];
        for (int t = 0; t < T; ++t) {
            unsigned long long m = best[0];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(FULL, m, o);
                m = other < m ? other : m;
            }
            chosen[t] = (int)(uint32_t)m;
            if (best[0] == m) {  // keys are unique: one owner pops its head
#pragma unroll
                for (int u = 0; u + 1 < kMaxT; ++u)
                    best[u] = best[u + 1];
                best[kMaxT - 1] = ~0ull;
            }
        }
        if (lane == 0) {
            if (c.cells_out != nullptr)
                for (int t = 0; t < T; ++t)
                    c.cells_out[q * T + t] = chosen[t];
            int j = 0;
            if (P > 0) {
                const int S = (int64_t)want < P ? want : (int)P;
                for (int t = 0; t < T && j < S; ++t) {
                    const unsigned long long key = ((unsigned long long)qa << 16) | (uint32_t)chosen[t];
                    int64_t r = lower_bound_u64(c.cell_key, a.N, key);
                    for (; r < a.N && c.cell_key[r] == key && j < S; ++r)
                        row[j++] = c.cell_id[r];
                }
                const int S2 = S - j;
                for (int jj = 0; jj < S2; ++jj)
                    row[j++] = c.id_sorted[lo + ((int64_t)jj * P) / S2];
            } else {  // the random stream of NHQ_SEED_RANDOM
                const uint64_t s0 = a.seed ^ mix64((uint64_t)q);
                for (int t = 0; t < 64 && j < want; ++t) {
                    const uint32_t v =
                        (uint32_t)(splitmix_at(s0, (uint64_t)t) % (unsigned long long)a.N);
                    bool dup = false;
                    for (int i = 0; i < j; ++i)
                        dup = dup || row[i] == v;
                    if (!dup)
                        row[j++] = v;
                }
            }
            for (; j < 32; ++j)
                row[j] = kNone;
        }
    }
}

__global__ void entry_to_half_kernel(const float *__restrict__ p, __half *__restrict__ h,
                                     int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        h[i] = __float2half_rn(p[i]);
}

// ---- training (f32 master weights) on a chunk of B samples ----
// Z[b][j] = b1[j] + sum_i W1[i][j] (s X[b][i]); 4 samples of 64 units per block
__global__ void train_hidden_kernel(const float *__restrict__ P, const float *__restrict__ X,
                                    int B, int d, float *__restrict__ Z, EntryLayout L) {
    const int b = blockIdx.x * 4 + (threadIdx.x >> 6), j = threadIdx.x & 63;
    if (b >= B)
        return;
    const float s = P[0];
    float z = P[L.oB1 + j];
    for (int i = 0; i < d; ++i)
        z = fmaf(P[L.oW1 + (int64_t)i * EH + j], s * X[(int64_t)b * d + i], z);
    Z[(int64_t)b * EH + j] = z;
}

// Tl[b][o] = b2[o] + sum_h W2[h][o] relu(Z[b][h]); grid (ceil(E/128), B)
__global__ void train_out_kernel(const float *__restrict__ P, const float *__restrict__ Z, int E,
                                 float *__restrict__ Tl, EntryLayout L) {
    __shared__ float h[EH];
    const int b = blockIdx.y;
    if (threadIdx.x < EH)
        h[threadIdx.x] = fmaxf(Z[(int64_t)b * EH + threadIdx.x], 0.f);
    __syncthreads();
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= E)
        return;
    float t = P[L.oB2 + o];
    for (int k = 0; k < EH; ++k)
        t = fmaf(P[L.oW2 + (int64_t)k * E + o], h[k], t);
    Tl[(int64_t)b * E + o] = t;
}

// dT = (softmax(T) - onehot(label)) * inv_n per sample (a warp each); loss += (lse - t_y) * inv_n.
// A label outside 0..E-1 contributes nothing.
__global__ void train_softmax_kernel(const float *__restrict__ Tl, const int32_t *__restrict__ y,
                                     int B, int E, float inv_n, float *__restrict__ dT,
                                     float *__restrict__ loss) {
    const int lane = threadIdx.x & 31;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= B)
        return;
    const float *t = Tl + (int64_t)b * E;
    float *g = dT + (int64_t)b * E;
    const int lab = y[b];
    if (lab < 0 || lab >= E) {
        for (int o = lane; o < E; o += 32)
            g[o] = 0.f;
        return;
    }
    float mx = -INFINITY;
    for (int o = lane; o < E; o += 32)
        mx = fmaxf(mx, t[o]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        mx = fmaxf(mx, __shfl_xor_sync(FULL, mx, o));
    float se = 0.f;
    for (int o = lane; o < E; o += 32)
        se += expf(t[o] - mx);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        se += __shfl_xor_sync(FULL, se, o);
    const float lse = mx + logf(se);
    for (int o = lane; o < E; o += 32)
        g[o] = (expf(t[o] - lse) - (o == lab ? 1.f : 0.f)) * inv_n;
    if (lane == 0)
        atomicAdd(loss, (lse - t[lab]) * inv_n);
}

// G[W2][h][o] += sum_b relu(Z[b][h]) dT[b][o]; row h = 64 is b2 (sum_b dT[b][o])
__global__ void train_gw2_kernel(const float *__restrict__ Z, const float *__restrict__ dT, int B,
                                 int E, float *__restrict__ G, EntryLayout L) {
    const int h = blockIdx.y;
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= E)
        return;
    float acc = 0.f;
    for (int b = 0; b < B; ++b) {
        const float hv = h < EH ? fmaxf(Z[(int64_t)b * EH + h], 0.f) : 1.f;
        acc = fmaf(hv, dT[(int64_t)b * E + o], acc);
    }
    if (h < EH)
        G[L.oW2 + (int64_t)h * E + o] += acc;
    else
        G[L.oB2 + o] += acc;
}

// dZ[b][h] = [Z > 0] sum_o dT[b][o] W2[h][o]; a warp per (b, h) pair group of 1
__global__ void train_dz_kernel(const float *__restrict__ P, const float *__restrict__ Z,
                                const float *__restrict__ dT, int B, int E,
                                float *__restrict__ dZ, EntryLayout L) {
    const int lane = threadIdx.x & 31;
    const int64_t pair = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (pair >= (int64_t)B * EH)
        return;
    const int b = (int)(pair / EH), h = (int)(pair % EH);
    float acc = 0.f;
    for (int o = lane; o < E; o += 32)
        acc = fmaf(dT[(int64_t)b * E + o], P[L.oW2 + (int64_t)h * E + o], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0)
        dZ[(int64_t)b * EH + h] = Z[(int64_t)b * EH + h] > 0.f ? acc : 0.f;
}

// G[W1][i][h] += sum_b s X[b][i] dZ[b][h]; row i = d is b1 (sum_b dZ[b][h]); 4 rows of 64
__global__ void train_gw1_kernel(const float *__restrict__ P, const float *__restrict__ X,
                                 const float *__restrict__ dZ, int B, int d,
                                 float *__restrict__ G, EntryLayout L) {
    const int i = blockIdx.x * 4 + (threadIdx.x >> 6), h = threadIdx.x & 63;
    if (i > d)
        return;
    const float s = P[0];
    float acc = 0.f;
    for (int b = 0; b < B; ++b) {
        const float x = i < d ? s * X[(int64_t)b * d + i] : 1.f;
        acc = fmaf(x, dZ[(int64_t)b * EH + h], acc);
    }
    if (i < d)
        G[L.oW1 + (int64_t)i * EH + h] += acc;
    else
        G[L.oB1 + h] += acc;
}

// Adam (beta1 0.9, beta2 0.999) on every parameter but the input scale (index 0)
__global__ void train_adam_kernel(float *__restrict__ p, const float *__restrict__ g,
                                  float *__restrict__ m, float *__restrict__ v, int64_t n,
                                  float lr, float c1, float c2) {
    for (int64_t i = 1 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        m[i] = b1 * m[i] + (1.f - b1) * g[i];
        v[i] = b2 * v[i] + (1.f - b2) * g[i] * g[i];
        p[i] -= lr * (m[i] * c1) / (sqrtf(v[i] * c2) + eps);
    }
}

__global__ void entry_labels_kernel(const uint32_t *__restrict__ ids, int k, int64_t n,
                                    const uint32_t *__restrict__ cell, int64_t N,
                                    int32_t *__restrict__ lab) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = ids[q * k];
        lab[q] = (v != kNone && (int64_t)v < N) ? (int32_t)cell[v] : -1;
    }
}

unsigned grid_for(int64_t n, int per) {
    int64_t g = (n + per - 1) / per;
    return (unsigned)(g < 1 ? 1 : (g > 65535 * 4 ? 65535 * 4 : g));
}

}  // namespace

int64_t entry_param_count(int d, int E) { return entry_layout(d, E).total; }

cudaError_t launch_gather_centroids(const float *X, int xstride, int64_t N, int E,
                                    const uint32_t *attr, float *cent, uint32_t *cattr,
                                    cudaStream_t s) {
    gather_centroids_kernel<<<E, 128, 0, s>>>(X, xstride, N, E, attr, cent, cattr);
    return cudaGetLastError();
}

size_t cell_sort_scratch_bytes(int64_t N) {
    size_t cub_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, cub_bytes, (const unsigned long long *)nullptr,
                                    (unsigned long long *)nullptr, (const uint32_t *)nullptr,
                                    (uint32_t *)nullptr, (int)N);
    return (sizeof(unsigned long long) + sizeof(uint32_t)) * (size_t)N + 512 + cub_bytes;
}

cudaError_t launch_cell_sort(const uint32_t *attr, const uint32_t *cell, int64_t N,
                             unsigned long long *key_sorted, uint32_t *id_sorted, void *scratch,
                             size_t scratch_bytes, cudaStream_t s) {
    unsigned long long *key = reinterpret_cast<unsigned long long *>(scratch);
    uintptr_t t = reinterpret_cast<uintptr_t>(key + N);
    t = (t + 255) & ~(uintptr_t)255;
    uint32_t *iota = reinterpret_cast<uint32_t *>(t);
    t = reinterpret_cast<uintptr_t>(iota + N);
    t = (t + 255) & ~(uintptr_t)255;
    void *tmp = reinterpret_cast<void *>(t);
    size_t cub_bytes = 0;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(nullptr, cub_bytes, key, key_sorted, iota,
                                                    id_sorted, (int)N, 0, 48);
    if (e != cudaSuccess)
        return e;
    if ((char *)tmp + cub_bytes > (char *)scratch + scratch_bytes)
        return cudaErrorInvalidValue;
    cell_key_kernel<<<grid_for(N, 256), 256, 0, s>>>(attr, cell, N, key, iota);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    return cub::DeviceRadixSort::SortPairs(tmp, cub_bytes, key, key_sorted, iota, id_sorted,
                                           (int)N, 0, 48, s);
}

cudaError_t launch_entry_to_half(const float *params, int64_t n, __half *w16, cudaStream_t s) {
    entry_to_half_kernel<<<grid_for(n, 256), 256, 0, s>>>(params, w16, n);
    return cudaGetLastError();
}

cudaError_t launch_cell_seeds(const SearchArgs &a, const uint32_t *attr_sorted,
                              const uint32_t *id_sorted, const unsigned long long *cell_key,
                              const uint32_t *cell_id, int E, int T, const float *scores,
                              int32_t *cells_out, uint32_t *seeds, uint8_t *bucket,
                              cudaStream_t s) {
    if (a.nq <= 0)
        return cudaSuccess;
    if (T < 1 || T > kMaxT || T > E)
        return cudaErrorInvalidValue;
    CellSeedArgs c;
    c.a = a;
    c.attr_sorted = attr_sorted;
    c.id_sorted = id_sorted;
    c.cell_key = cell_key;
    c.cell_id = cell_id;
    c.E = E;
    c.T = T;
    c.scores = scores;
    c.cells_out = cells_out;
    c.seeds = seeds;
    c.bucket = bucket;
    cell_seeds_kernel<<<(unsigned)((a.nq + 7) / 8), 256, 0, s>>>(c);
    return cudaGetLastError();
}

cudaError_t launch_centroid_columns(const float *cent, int xstride, int d, int E, float *cT,
                                    float *nh, cudaStream_t s) {
    centroid_columns_kernel<<<E, 128, 0, s>>>(cent, xstride, d, E, cT, nh);
    return cudaGetLastError();
}

cudaError_t launch_entry_scores_nearest(const float *cT, const float *nh, int d, int E,
                                        const float *Q, int64_t qstride, int64_t n, float *out,
                                        cudaStream_t s) {
    return launch_dense<float>(Q, n, d, qstride, cT, nh, E, nullptr, 0, out, s);
}

cudaError_t launch_entry_scores_learned(const __half *w16, const float *params, int d, int E,
                                        const float *Q, int64_t qstride, int64_t n,
                                        float *hidden, float *out, cudaStream_t s) {
    const EntryLayout L = entry_layout(d, E);
    cudaError_t e = launch_dense<__half>(Q, n, d, qstride, w16 + L.oW1, w16 + L.oB1, EH, params,
                                         1, hidden, s);
    if (e != cudaSuccess)
        return e;
    return launch_dense<__half>(hidden, n, EH, EH, w16 + L.oW2, w16 + L.oB2, E, nullptr, 0, out,
                                s);
}

cudaError_t launch_entry_labels(const uint32_t *ids, int k, int64_t n, const uint32_t *cell,
                                int64_t N, int32_t *labels, cudaStream_t s) {
    if (n <= 0)
        return cudaSuccess;
    entry_labels_kernel<<<grid_for(n, 256), 256, 0, s>>>(ids, k, n, cell, N, labels);
    return cudaGetLastError();
}

// Working memory of one chunk of B samples: Z, dZ [B][64], Tl, dT [B][E].
size_t entry_train_chunk_bytes(int B, int E) {
    return sizeof(float) * ((size_t)B * EH * 2 + (size_t)B * E * 2) + 1024;
}

// Adds the gradient of the loss over samples [0, n) (divided by `total`) to G and the loss
// to *loss, in chunks of B samples.
cudaError_t entry_grad_accumulate(const float *P, int d, int E, const float *X,
                                  const int32_t *y, int64_t n, int64_t total, int B, float *G,
                                  float *loss, void *work, cudaStream_t s) {
    const EntryLayout L = entry_layout(d, E);
    float *Z = reinterpret_cast<float *>(work);
    float *dZ = Z + (size_t)B * EH;
    float *Tl = dZ + (size_t)B * EH;
    float *dT = Tl + (size_t)B * E;
    const float inv = 1.f / (float)total;
    cudaError_t e = cudaSuccess;
    for (int64_t b0 = 0; b0 < n; b0 += B) {
        const int nb = (int)(n - b0 < B ? n - b0 : B);
        const float *Xb = X + b0 * d;
        train_hidden_kernel<<<(nb + 3) / 4, 256, 0, s>>>(P, Xb, nb, d, Z, L);
        train_out_kernel<<<dim3((E + 127) / 128, nb), 128, 0, s>>>(P, Z, E, Tl, L);
        train_softmax_kernel<<<(nb + 7) / 8, 256, 0, s>>>(Tl, y + b0, nb, E, inv, dT, loss);
        train_gw2_kernel<<<dim3((E + 127) / 128, EH + 1), 128, 0, s>>>(Z, dT, nb, E, G, L);
        train_dz_kernel<<<(unsigned)(((int64_t)nb * EH + 7) / 8), 256, 0, s>>>(P, Z, dT, nb, E,
                                                                               dZ, L);
        train_gw1_kernel<<<(d + 1 + 3) / 4, 256, 0, s>>>(P, Xb, dZ, nb, d, G, L);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
    }
    return e;
}

cudaError_t launch_entry_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr,
                              float c1, float c2, cudaStream_t s) {
    train_adam_kernel<<<grid_for(n, 256), 256, 0, s>>>(p, g, m, v, n, lr, c1, c2);
    return cudaGetLastError();
}

}  // namespace nhq
