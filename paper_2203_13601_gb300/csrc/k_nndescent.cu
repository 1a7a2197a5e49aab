// k_nndescent.cu -- candidate sets C(u) by NN-descent (Sec. 4.3: the NPG_kgraph
// recipe refines random neighbour lists with NN-descent instead of computing the
// exact K nearest), under the fusion distance Gamma of the index.
//
// Each vertex keeps its K best records (Gamma bits << 32 | id) sorted ascending and
// a "new" flag per record.  One iteration:
//   sample   per vertex (one warp): up to S of its new records (they become old)
//            and up to S of its old ones; every sampled id also records the vertex
//            in its own reverse sample (capped at S, atomics)
//   join     per vertex (one CTA): the candidates new = sample_new u reverse_new and
//            old = sample_old u reverse_old; their rows are copied into shared memory
//            and Gamma is computed for every new x new and new x old pair; a pair
//            closer than a vertex's current K-th record is offered to that vertex's
//            update table: U slots indexed by a hash of the record's id, each keeping
//            the smallest key offered to it (atomicMin), so the best candidates survive
//            however many arrive (a record lost to a collision only slows convergence)
//   merge    per vertex (one warp): list + updates sorted, repeated ids dropped, the
//            K smallest kept; records that entered are new; the number that entered
//            is added to a global count, and the host stops when it falls below
//            delta * N * K or after the iteration limit.
// The order in which updates arrive is not fixed, so two runs may end with lists
// that differ where the process had not converged; every record's Gamma is exact
// (the same f32 arithmetic as the other kernels).
#include "nhq_internal.cuh"

namespace nhq {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int NND_KMAX = 64;        // K
constexpr int NND_S = 16;           // sample size per side
constexpr int NND_U = 128;          // update slots per vertex (a power of two)
constexpr int NND_C = 4 * NND_S;    // candidates of one join (new 2S + old 2S)
constexpr int JOIN_THREADS = 128;

struct NndArgs {
    const float *X;
    int xstride;
    int64_t N;
    const uint32_t *attr;
    Fusion w;
    int K;
    unsigned long long *lists;  // [N][K]
    uint8_t *flags;             // [N][K] 1 = new
    uint32_t *snew, *sold;      // [N][S]
    uint32_t *rnew, *rold;      // [N][S]
    uint32_t *rcnt_new, *rcnt_old;  // [N]
    unsigned long long *upd;    // [N][U] hashed update table, +inf = empty
    unsigned long long *changes;
    uint64_t seed;
};

__device__ __forceinline__ unsigned long long rec_key(float g, uint32_t id) {
    return ((unsigned long long)__float_as_uint(g) << 32) | id;
}

// squared distance of two rows by a team of 4 lanes (f32, lane tl sums the float4
// chunks tl, tl + 4, ..., then the team reduces); every kernel here uses this order, so
// a pair gets the same Gamma bits wherever it is computed
__device__ __forceinline__ float team4_dist2(const float *a, const float *b, int xs4, int tl) {
    float acc = 0.f;
    for (int c = tl; c < xs4; c += 4) {
        const float4 x = reinterpret_cast<const float4 *>(a)[c];
        const float4 y = reinterpret_cast<const float4 *>(b)[c];
        float t;
        t = x.x - y.x; acc = fmaf(t, t, acc);
        t = x.y - y.y; acc = fmaf(t, t, acc);
        t = x.z - y.z; acc = fmaf(t, t, acc);
        t = x.w - y.w; acc = fmaf(t, t, acc);
    }
    acc += __shfl_xor_sync(FULL, acc, 1);
    acc += __shfl_xor_sync(FULL, acc, 2);
    return acc;
}

// ascending bitonic sort of n = 2^p <= 128 keys in shared memory by one warp, each key
// carrying one byte
__device__ void warp_sort_keys(unsigned long long *k, uint8_t *f, int n, int lane) {
    for (int size = 2; size <= n; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = lane; i < n / 2; i += 32) {
                const int lo = 2 * stride * (i / stride) + (i % stride), hi = lo + stride;
                const bool up = (lo & size) == 0;
                const unsigned long long x = k[lo], y = k[hi];
                if ((x > y) == up) {
                    k[lo] = y;
                    k[hi] = x;
                    const uint8_t t = f[lo];
                    f[lo] = f[hi];
                    f[hi] = t;
                }
            }
            __syncwarp();
        }
}

// ---------------------------------------------------------------- init
__global__ void nnd_init_kernel(NndArgs a) {
    __shared__ unsigned long long sk[8][2 * NND_KMAX];
    __shared__ uint8_t sf[8][2 * NND_KMAX];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t u = (int64_t)blockIdx.x * 8 + wib;
    if (u >= a.N)
        return;
    const int K = a.K, xs4 = a.xstride / 4;
    int P = 2;
    while (P < K)
        P <<= 1;
    unsigned long long *k = sk[wib];
    uint8_t *f = sf[wib];
    const uint64_t s0 = a.seed ^ mix64((uint64_t)u + 0x51ull);
    const float *xu = a.X + u * a.xstride;
    const uint32_t au = a.attr[u];
    const int team = lane >> 2, tl = lane & 3;
    for (int base = 0; base < K; base += 8) {  // 8 teams of 4 lanes, one random id each
        const int j = base + team;
        const int jj = j < K ? j : 0;
        // a random id other than u
        const uint32_t v = (uint32_t)((u + 1 + (int64_t)(splitmix_at(s0, (uint64_t)jj) %
                                                        (unsigned long long)(a.N - 1))) %
                                      a.N);
        const float d2 = team4_dist2(xu, a.X + (int64_t)v * a.xstride, xs4, tl);
        if (j < K && tl == 0) {
            k[j] = rec_key(fusion_gamma(__fsqrt_rn(d2), chi_packed(au, a.attr[v], a.w.hi, a.w.lo),
                                        a.w),
                           v);
            f[j] = 1;
        }
    }
    __syncwarp();
    for (int j = K + lane; j < P; j += 32) {
        k[j] = kInfKey;
        f[j] = 0;
    }
    __syncwarp();
    warp_sort_keys(k, f, P, lane);
    // repeated draws of one id are equal keys, now adjacent: keep the first
    for (int j = lane; j < K; j += 32) {
        const bool dup = j > 0 && k[j] == k[j - 1];
        a.lists[u * K + j] = dup ? kInfKey : k[j];
        a.flags[u * K + j] = dup ? 0 : 1;
    }
}

// ---------------------------------------------------------------- sample
__global__ void nnd_sample_kernel(NndArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t u = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (u >= a.N)
        return;
    const int K = a.K;
    int got_new = 0, got_old = 0;
    for (int base = 0; base < K; base += 32) {
        const int j = base + lane;
        const unsigned long long key = j < K ? a.lists[u * K + j] : kInfKey;
        const bool valid = key != kInfKey;
        const bool isnew = valid && a.flags[u * K + j] != 0;
        const bool isold = valid && !isnew;
        const unsigned bn = __ballot_sync(FULL, isnew), bo = __ballot_sync(FULL, isold);
        const int pn = got_new + __popc(bn & ((1u << lane) - 1u));
        const int po = got_old + __popc(bo & ((1u << lane) - 1u));
        const uint32_t id = (uint32_t)key;
        if (isnew && pn < NND_S) {
            a.snew[u * NND_S + pn] = id;
            a.flags[u * K + j] = 0;
            const uint32_t r = atomicAdd(&a.rcnt_new[id], 1u);
            if (r < NND_S)
                a.rnew[(int64_t)id * NND_S + r] = (uint32_t)u;
        }
        if (isold && po < NND_S) {
            a.sold[u * NND_S + po] = id;
            const uint32_t r = atomicAdd(&a.rcnt_old[id], 1u);
            if (r < NND_S)
                a.rold[(int64_t)id * NND_S + r] = (uint32_t)u;
        }
        got_new += __popc(bn);
        got_old += __popc(bo);
    }
    for (int p = (got_new < NND_S ? got_new : NND_S) + lane; p < NND_S; p += 32)
        a.snew[u * NND_S + p] = kNone;
    for (int p = (got_old < NND_S ? got_old : NND_S) + lane; p < NND_S; p += 32)
        a.sold[u * NND_S + p] = kNone;
}

// ---------------------------------------------------------------- local join
__device__ __forceinline__ void push_update(const NndArgs &a, uint32_t p, unsigned long long key) {
    // only records below p's current K-th can enter its list (a stale read is larger)
    if (key >= a.lists[(int64_t)p * a.K + a.K - 1])
        return;
    const uint32_t slot = ((uint32_t)key * 0x9E3779B1u) >> (32 - 7);  // 7 = log2(NND_U)
    atomicMin(&a.upd[(int64_t)p * NND_U + slot], key);
}

__global__ void __launch_bounds__(JOIN_THREADS) nnd_join_kernel(NndArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *cid = reinterpret_cast<uint32_t *>(smem);  // [NND_C] new ones first
    uint32_t *cat = cid + NND_C;                          // [NND_C]
    int *cnt = reinterpret_cast<int *>(cat + NND_C);      // [4]: new, total
    float *rows = reinterpret_cast<float *>(cnt + 4);     // [NND_C][xstride + 4]
    const int tid = threadIdx.x;
    const int64_t u = blockIdx.x;
    const int xs4 = a.xstride / 4, rs = a.xstride + 4;
    if (tid == 0) {
        // candidate ids: new = sample + reverse sample, old likewise; a repeat is dropped
        int n = 0;
        auto add = [&](uint32_t v) {
            if (v == kNone || (int64_t)v == u)
                return;
            for (int i = 0; i < n; ++i)
                if (cid[i] == v)
                    return;
            cid[n++] = v;
        };
        const uint32_t rn = a.rcnt_new[u] < NND_S ? a.rcnt_new[u] : NND_S;
        const uint32_t ro = a.rcnt_old[u] < NND_S ? a.rcnt_old[u] : NND_S;
        for (int i = 0; i < NND_S; ++i)
            add(a.snew[u * NND_S + i]);
        for (uint32_t i = 0; i < rn; ++i)
            add(a.rnew[u * NND_S + i]);
        cnt[0] = n;
        for (int i = 0; i < NND_S; ++i)
            add(a.sold[u * NND_S + i]);
        for (uint32_t i = 0; i < ro; ++i)
            add(a.rold[u * NND_S + i]);
        cnt[1] = n;
    }
    __syncthreads();
    const int nn = cnt[0], nt = cnt[1];
    if (nn == 0)
        return;  // nothing new around u: no pair can change a list
    for (int i = tid; i < nt; i += JOIN_THREADS)
        cat[i] = a.attr[cid[i]];
    for (int idx = tid; idx < nt * xs4; idx += JOIN_THREADS) {
        const int r = idx / xs4, c = idx % xs4;
        reinterpret_cast<float4 *>(rows + r * rs)[c] =
            __ldg(reinterpret_cast<const float4 *>(a.X + (int64_t)cid[r] * a.xstride) + c);
    }
    __syncthreads();
    // pairs (i, j): i < nn (new), j > i within all candidates: new x new and new x old
    const int team = tid >> 2, tl = tid & 3;
    constexpr int TEAMS = JOIN_THREADS / 4;
    const int64_t npairs = (int64_t)nn * nt - (int64_t)nn * (nn + 1) / 2;
    for (int64_t base = 0; base < npairs; base += TEAMS) {
        const int64_t pi = base + team;
        const bool live = pi < npairs;
        // pair index -> (i, j): row i holds nt - 1 - i pairs
        int i = 0;
        int64_t rem = live ? pi : 0;
        while (rem >= nt - 1 - i) {
            rem -= nt - 1 - i;
            ++i;
        }
        const int j = i + 1 + (int)rem;
        const float acc = team4_dist2(rows + i * rs, rows + j * rs, xs4, tl);
        if (live && tl == 0) {
            const float g = fusion_gamma(__fsqrt_rn(acc), chi_packed(cat[i], cat[j], a.w.hi, a.w.lo),
                                         a.w);
            push_update(a, cid[i], rec_key(g, cid[j]));
            push_update(a, cid[j], rec_key(g, cid[i]));
        }
    }
}

// ---------------------------------------------------------------- merge
__global__ void nnd_merge_kernel(NndArgs a) {
    __shared__ unsigned long long sk[4][256];
    __shared__ uint8_t sf[4][256];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t u = (int64_t)blockIdx.x * 4 + wib;
    if (u >= a.N)
        return;
    const int K = a.K;
    unsigned long long *k = sk[wib];
    uint8_t *f = sf[wib];
    const int nu = NND_U;
    // origin in bit 1 of the byte: 0 = list (bit 0 = its new flag), 2 = update; the
    // update table is read and cleared for the next iteration (empty slots are +inf)
    for (int j = lane; j < K; j += 32) {
        k[j] = a.lists[u * K + j];
        f[j] = a.flags[u * K + j];
    }
    for (int j = lane; j < nu; j += 32) {
        k[K + j] = a.upd[u * NND_U + j];
        a.upd[u * NND_U + j] = kInfKey;
        f[K + j] = 2;
    }
    int P = 2;
    while (P < K + nu)
        P <<= 1;
    for (int j = K + nu + lane; j < P; j += 32) {
        k[j] = kInfKey;
        f[j] = 2;
    }
    __syncwarp();
    warp_sort_keys(k, f, P, lane);
    // an id kept once: equal keys are the same record; a list copy wins over updates
    int kept = 0, entered = 0;
    for (int base = 0; base < P && kept < K; base += 32) {
        const int j = base + lane;
        bool first = false;
        uint8_t flag = 0;
        if (j < P && k[j] != kInfKey) {
            first = j == 0 || k[j - 1] != k[j];
            if (first) {
                // any list copy in this run of equal keys?
                bool from_list = false;
                uint8_t lf = 0;
                for (int t = j; t < P && k[t] == k[j]; ++t)
                    if ((f[t] & 2) == 0) {
                        from_list = true;
                        lf = f[t] & 1;
                    }
                flag = from_list ? (uint8_t)(lf | 4) : (uint8_t)1;
            }
        }
        const unsigned b = __ballot_sync(FULL, first);
        const int pos = kept + __popc(b & ((1u << lane) - 1u));
        if (first && pos < K) {
            a.lists[u * K + pos] = k[j];
            a.flags[u * K + pos] = flag & 1;
            if ((flag & 4) == 0)
                ++entered;
        }
        kept += __popc(b);
    }
    for (int p = (kept < K ? kept : K) + lane; p < K; p += 32) {
        a.lists[u * K + p] = kInfKey;
        a.flags[u * K + p] = 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        entered += __shfl_xor_sync(FULL, entered, o);
    if (lane == 0) {
        if (entered)
            atomicAdd(a.changes, (unsigned long long)entered);
        a.rcnt_new[u] = 0;
        a.rcnt_old[u] = 0;
    }
}

__global__ void nnd_output_kernel(const unsigned long long *__restrict__ lists, int64_t total,
                                  uint32_t *__restrict__ ids, float *__restrict__ dists) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = lists[i];
        ids[i] = key == kInfKey ? kNone : (uint32_t)key;
        if (dists)
            dists[i] = key == kInfKey ? __int_as_float(0x7f800000)
                                      : __uint_as_float((uint32_t)(key >> 32));
    }
}

}  // namespace

int nnd_kmax() { return NND_KMAX; }

size_t nnd_scratch_bytes(int64_t N, int K) {
    const size_t n = (size_t)N;
    return 8 * n * K + n * K + 4 * 4 * n * NND_S + 4 * 2 * n + 8 * n * NND_U + 64 + 16 * 256;
}

cudaError_t launch_nndescent(const float *X, int xstride, int64_t N, const uint32_t *attr,
                             const Fusion &w, int K, int max_iters, double delta, uint64_t seed,
                             void *scratch, uint32_t *ids, float *dists, int *iters_done,
                             cudaStream_t s) {
    auto align = [](size_t o) { return (o + 255) & ~(size_t)255; };
    char *p = reinterpret_cast<char *>(scratch);
    size_t o = 0;
    NndArgs a;
    a.X = X;
    a.xstride = xstride;
    a.N = N;
    a.attr = attr;
    a.w = w;
    a.K = K;
    a.seed = seed;
    const size_t n = (size_t)N;
    a.lists = reinterpret_cast<unsigned long long *>(p + o);
    o = align(o + 8 * n * K);
    a.flags = reinterpret_cast<uint8_t *>(p + o);
    o = align(o + n * K);
    a.snew = reinterpret_cast<uint32_t *>(p + o);
    o = align(o + 4 * n * NND_S);
    a.sold = reinterpret_cast<uint32_t *>(p + o);
    o = align(o + 4 * n * NND_S);
    a.rnew = reinterpret_cast<uint32_t *>(p + o);
    o = align(o + 4 * n * NND_S);
    a.rold = reinterpret_cast<uint32_t *>(p + o);
    o = align(o + 4 * n * NND_S);
    a.rcnt_new = reinterpret_cast<uint32_t *>(p + o);
    o = align(o + 4 * n);
    a.rcnt_old = reinterpret_cast<uint32_t *>(p + o);
    o = align(o + 4 * n);
    a.upd = reinterpret_cast<unsigned long long *>(p + o);
    o = align(o + 8 * n * NND_U);
    a.changes = reinterpret_cast<unsigned long long *>(p + o);
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.rcnt_new, 0, 4 * n, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(a.rcnt_old, 0, 4 * n, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(a.upd, 0xFF, 8 * n * NND_U, s)) != cudaSuccess)
        return e;
    nnd_init_kernel<<<(unsigned)((N + 7) / 8), 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    const size_t jsmem = 8 * NND_C + 16 + sizeof(float) * (size_t)NND_C * (xstride + 4);
    if ((e = cudaFuncSetAttribute(nnd_join_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)jsmem)) != cudaSuccess)
        return e;
    const double stop = delta * (double)N * (double)K;
    int it = 0;
    for (; it < max_iters; ++it) {
        if ((e = cudaMemsetAsync(a.changes, 0, 8, s)) != cudaSuccess)
            return e;
        nnd_sample_kernel<<<(unsigned)((N + 7) / 8), 256, 0, s>>>(a);
        nnd_join_kernel<<<(unsigned)N, JOIN_THREADS, jsmem, s>>>(a);
        nnd_merge_kernel<<<(unsigned)((N + 3) / 4), 128, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        unsigned long long ch = 0;
        if ((e = cudaMemcpyAsync(&ch, a.changes, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return e;
        if ((double)ch < stop) {
            ++it;
            break;
        }
    }
    if (iters_done)
        *iters_done = it;
    const int64_t total = N * (int64_t)K;
    nnd_output_kernel<<<(unsigned)((total + 255) / 256 > 8192 ? 8192 : (total + 255) / 256), 256,
                        0, s>>>(a.lists, total, ids, dists);
    return cudaGetLastError();
}

}  // namespace nhq
