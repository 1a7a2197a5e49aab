// k_search.cuh -- the search kernel's templates (Alg. 2 with the two-stage routing of
// Sec. 4.2 / Sec. 5.2); the description of the kernel is in k_search.cu.  Each scoring
// type instantiates them in a translation unit of its own (k_search_<type>.cu), so the
// variants compile in parallel.
#pragma once

#include <type_traits>

#include "nhq_internal.cuh"

namespace nhq {
namespace {  // internal to each translation unit that includes it

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int TEAM = 8;
constexpr int CAND = 64;

__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

__device__ __forceinline__ uint32_t hash_slot(uint32_t v, int bits) {
    return (v * 0x9E3779B1u) >> (32 - bits);
}

// true if v was not present (and is now); a plain read first, the atomic only on an empty slot
__device__ __forceinline__ bool hash_insert(uint32_t *h, int bits, uint32_t v) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t s = hash_slot(v, bits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        uint32_t x = h[s];
        if (x == v)
            return false;
        if (x == kNone) {
            x = atomicCAS(&h[s], kNone, v);
            if (x == kNone)
                return true;
            if (x == v)
                return false;
        }
        s = (s + 1) & mask;
    }
    return false;
}

__device__ __forceinline__ bool hash_contains(const uint32_t *h, int bits, uint32_t v) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t s = hash_slot(v, bits);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        uint32_t x = h[s];
        if (x == v)
            return true;
        if (x == kNone)
            return false;
        s = (s + 1) & mask;
    }
    return false;
}

__device__ __forceinline__ unsigned long long warp_sort_asc(unsigned long long x, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            unsigned long long y = __shfl_xor_sync(FULL, x, j);
            bool up = (lane & k) == 0;
            bool lower = (lane & j) == 0;
            unsigned long long lo = x < y ? x : y, hi = x < y ? y : x;
            x = (lower == up) ? lo : hi;
        }
    }
    return x;
}

// number of pool records whose (Gamma, id) is below key c (flag bits ignored)
__device__ __forceinline__ int pool_lower_bound(const unsigned long long *pool, int n,
                                                unsigned long long c) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((pool[mid] & ~1ull) < c)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int sorted_count_less(const unsigned long long *s, int n,
                                                 unsigned long long x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (s[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

template <typename VT>
struct VecTraits;
template <>
struct VecTraits<float> {
    static constexpr int kPerChunk = 4;  // 16-byte chunk = 4 f32
};
template <>
struct VecTraits<__nv_bfloat16> {
    static constexpr int kPerChunk = 8;  // 8 bf16
};
template <>
struct VecTraits<__nv_fp8_e4m3> {
    static constexpr int kPerChunk = 16;  // 16 fp8 e4m3
};
template <>
struct VecTraits<__half> {
    static constexpr int kPerChunk = 8;  // 8 f16
};

// the query values matching one 16-byte chunk of a stored row
template <int PC>
struct QChunk {
    float4 v[PC / 4];
};

template <int PC>
__device__ __forceinline__ QChunk<PC> load_qchunk(const float *qv, int c) {
    QChunk<PC> q;
#pragma unroll
    for (int i = 0; i < PC / 4; ++i)
        q.v[i] = reinterpret_cast<const float4 *>(qv)[c * (PC / 4) + i];
    return q;
}

__device__ __forceinline__ void sq4(float &acc, const float4 &q, float x0, float x1, float x2,
                                    float x3) {
    float t;
    t = q.x - x0; acc = fmaf(t, t, acc);
    t = q.y - x1; acc = fmaf(t, t, acc);
    t = q.z - x2; acc = fmaf(t, t, acc);
    t = q.w - x3; acc = fmaf(t, t, acc);
}

template <typename VT>
__device__ __forceinline__ void accum_chunk(float &acc, const QChunk<VecTraits<VT>::kPerChunk> &q,
                                            const VT *row, int c, bool live);

template <>
__device__ __forceinline__ void accum_chunk<float>(float &acc, const QChunk<4> &q,
                                                   const float *row, int c, bool live) {
    if (!live)
        return;
    const float4 x = __ldg(reinterpret_cast<const float4 *>(row) + c);
    sq4(acc, q.v[0], x.x, x.y, x.z, x.w);
}

template <>
__device__ __forceinline__ void accum_chunk<__nv_bfloat16>(float &acc, const QChunk<8> &q,
                                                           const __nv_bfloat16 *row, int c,
                                                           bool live) {
    if (!live)
        return;
    const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(row) + c);
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&raw);
    const float2 x0 = __bfloat1622float2(h[0]), x1 = __bfloat1622float2(h[1]);
    const float2 x2 = __bfloat1622float2(h[2]), x3 = __bfloat1622float2(h[3]);
    sq4(acc, q.v[0], x0.x, x0.y, x1.x, x1.y);
    sq4(acc, q.v[1], x2.x, x2.y, x3.x, x3.y);
}

template <>
__device__ __forceinline__ void accum_chunk<__half>(float &acc, const QChunk<8> &q,
                                                    const __half *row, int c, bool live) {
    if (!live)
        return;
    const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(row) + c);
    const __half2 *h = reinterpret_cast<const __half2 *>(&raw);
    const float2 x0 = __half22float2(h[0]), x1 = __half22float2(h[1]);
    const float2 x2 = __half22float2(h[2]), x3 = __half22float2(h[3]);
    sq4(acc, q.v[0], x0.x, x0.y, x1.x, x1.y);
    sq4(acc, q.v[1], x2.x, x2.y, x3.x, x3.y);
}

template <>
__device__ __forceinline__ void accum_chunk<__nv_fp8_e4m3>(float &acc, const QChunk<16> &q,
                                                           const __nv_fp8_e4m3 *row, int c,
                                                           bool live) {
    if (!live)
        return;
    const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(row) + c);
    const __nv_fp8x2_storage_t *p2 = reinterpret_cast<const __nv_fp8x2_storage_t *>(&raw);
    float2 f[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)  // e4m3 -> f16 -> f32 are exact
        f[i] = __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(p2[i], __NV_E4M3)));
#pragma unroll
    for (int i = 0; i < 4; ++i)
        sq4(acc, q.v[i], f[2 * i].x, f[2 * i].y, f[2 * i + 1].x, f[2 * i + 1].y);
}

// Ask L2 for a candidate's whole row as soon as the candidate is known to be
// evaluated: the passes of eval_dist2 below load 8 rows at a time, so without this
// every pass after the first would wait for HBM again.
template <typename VT>
__device__ __forceinline__ void prefetch_row(const VT *X, int xstride, uint32_t v) {
    const char *r = reinterpret_cast<const char *>(X + (int64_t)v * xstride);
    const int bytes = xstride * (int)sizeof(VT);
    for (int o = 0; o < bytes; o += 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(r + o));
}

// Squared distances of cnt candidates cid[0..cnt) into d2s[0..cnt).  Teams of 8
// lanes, two rows per team per pass (8 rows in flight per warp).  CPL > 0: each
// lane covers at most CPL chunks of a row (EXACT: exactly CPL, no bounds test);
// CPL == 0: a strided loop for wide rows.
// With wpq warps per query, warp wig of the group takes the passes wig, wig + wpq, ...
// A pass is RPT rows per team of 8 lanes (4 RPT rows per warp): RPT = 2 keeps 8 rows
// in flight per warp; RPT = 4 puts the usual expansion (about 15 candidates) in one
// pass at the price of registers (the tile_rows search parameter picks it).
template <typename VT, int CPL, bool EXACT, int RPT = 2>
__device__ __forceinline__ void eval_dist2(const VT *__restrict__ X, int xstride, const float *qv,
                                           const uint32_t *cid, float *d2s, int cnt, int lane,
                                           int wig = 0, int wpq = 1) {
    static_assert(RPT == 2 || RPT == 4, "two or four rows per team");
    constexpr int PC = VecTraits<VT>::kPerChunk;
    constexpr int ROWS = 4 * RPT;  // rows per warp and pass
    const int team = lane / TEAM, tl = lane % TEAM;
    const int nchunk = xstride / PC;
    for (int base = ROWS * wig; base < cnt; base += ROWS * wpq) {
        int jr[RPT];
        bool hr[RPT];
        const VT *rr[RPT];
        float acc[RPT];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            jr[r] = base + 4 * r + team;
            hr[r] = jr[r] < cnt;
            rr[r] = X + (int64_t)cid[hr[r] ? jr[r] : 0] * xstride;
            acc[r] = 0.f;
        }
        if (CPL > 0) {
#pragma unroll
            for (int i = 0; i < (CPL > 0 ? CPL : 1); ++i) {
                const int c = tl + i * TEAM;
                const bool live = EXACT || c < nchunk;
                const int cc = EXACT ? c : (live ? c : 0);
                const QChunk<PC> qc = load_qchunk<PC>(qv, cc);
#pragma unroll
                for (int r = 0; r < RPT; ++r)
                    accum_chunk<VT>(acc[r], qc, rr[r], cc, hr[r] && live);
            }
        } else {
            // wide rows: f32 chunks go 8 deep per row (measured faster at d = 960); the
            // 16- and 8-bit chunks carry their conversions and go 4 deep
#pragma unroll(std::is_same<VT, float>::value ? 8 : 4)
            for (int c = tl; c < nchunk; c += TEAM) {
                const QChunk<PC> qc = load_qchunk<PC>(qv, c);
#pragma unroll
                for (int r = 0; r < RPT; ++r)
                    accum_chunk<VT>(acc[r], qc, rr[r], c, hr[r]);
            }
        }
        if constexpr (RPT == 2) {
            // reduce both rows over the team: the first level swaps halves so that
            // lanes tl < 4 carry row jr[0] and lanes tl >= 4 row jr[1]
            const bool upper = (tl & 4) != 0;
            const float send = upper ? acc[0] : acc[1];
            const float keep = upper ? acc[1] : acc[0];
            float a = keep + __shfl_xor_sync(FULL, send, 4);
            a += __shfl_xor_sync(FULL, a, 2);
            a += __shfl_xor_sync(FULL, a, 1);
            if (tl == 0 && hr[0])
                d2s[jr[0]] = a;
            if (tl == 4 && hr[1])
                d2s[jr[1]] = a;
        } else {
            // four rows: each level halves the rows a lane carries; lane tl ends with row
            // 2 [tl & 4] + [tl & 2], summed over the 8 lanes of the team
            const bool up4 = (tl & 4) != 0, up2 = (tl & 2) != 0;
            const float s0 = up4 ? acc[0] : acc[2], s1 = up4 ? acc[1] : acc[3];
            const float k0 = (up4 ? acc[2] : acc[0]) + __shfl_xor_sync(FULL, s0, 4);
            const float k1 = (up4 ? acc[3] : acc[1]) + __shfl_xor_sync(FULL, s1, 4);
            float a = (up2 ? k1 : k0) + __shfl_xor_sync(FULL, up2 ? k0 : k1, 2);
            a += __shfl_xor_sync(FULL, a, 1);
            const int j = base + 4 * ((up4 ? 2 : 0) + (up2 ? 1 : 0)) + team;
            if ((tl & 1) == 0 && j < cnt)
                d2s[j] = a;
        }
    }
    __syncwarp();
}

// Record (Gamma, id) of candidate j, or kInfKey when j >= cnt (one lane per candidate).
__device__ __forceinline__ unsigned long long candidate_key(int j, int cnt, const float *d2s,
                                                            const uint32_t *cid, const int *cchi,
                                                            const Fusion &w) {
    if (j >= cnt)
        return kInfKey;
    return make_key(fusion_gamma(__fsqrt_rn(d2s[j]), cchi[j], w), cid[j]);
}

// smallest record over the warp from two 32-bit reductions (Gamma bits, then ids of ties)
__device__ __forceinline__ unsigned long long warp_min_key(unsigned long long x) {
    const unsigned hi = __reduce_min_sync(FULL, (unsigned)(x >> 32));
    const unsigned lo = __reduce_min_sync(FULL, (unsigned)(x >> 32) == hi ? (unsigned)x : ~0u);
    return ((unsigned long long)hi << 32) | lo;
}

// number of pool records below c, every lane passing the same c (ballot count)
__device__ __forceinline__ int pool_rank_uniform(const unsigned long long *pool, int n,
                                                 unsigned long long c, int lane) {
    int r = 0;
    for (int b = 0; b < n; b += 32) {
        const int i = b + lane;
        const unsigned m = __ballot_sync(FULL, i < n && (pool[i] & ~1ull) < c);
        r += __popc(m);
        if (m != FULL)
            break;  // sorted: the first record not below c ends the run
    }
    return r;
}

// Drop a candidate that cannot enter: above the last record of a full pool, or,
// after the visited filter was rebuilt, a record already in the pool.
__device__ __forceinline__ unsigned long long filter_key(unsigned long long c,
                                                         const unsigned long long *pool, int n,
                                                         int ef, bool dup_check) {
    if (c == kInfKey)
        return c;
    if (n == ef && c > (pool[ef - 1] & ~1ull))
        return kInfKey;
    if (dup_check) {
        const int lb = pool_lower_bound(pool, n, c);
        if (lb < n && (pool[lb] & ~1ull) == c)
            return kInfKey;
    }
    return c;
}

// Inserts the candidate records held one per lane (kInfKey = none) into the pool,
// keeping its ef smallest records; equals inserting them one at a time.
__device__ void merge_round(unsigned long long *pool, int &n, int ef, unsigned long long c,
                            unsigned long long *sorted32, int lane) {
    if (c != kInfKey && n == ef && c > (pool[ef - 1] & ~1ull))
        c = kInfKey;
    const unsigned vb = __ballot_sync(FULL, c != kInfKey);
    if (vb == 0)
        return;
    const int nv = __popc(vb);
    if (nv <= 8) {
        int rank = 0;
        for (unsigned mm = vb; mm; mm &= mm - 1) {
            const unsigned long long cj = __shfl_sync(FULL, c, __ffs(mm) - 1);
            rank += cj < c ? 1 : 0;
        }
        const int pos = c != kInfKey ? rank + pool_lower_bound(pool, n, c) : ef;
        const int p0 = (int)__reduce_min_sync(FULL, (unsigned)pos);
        if (p0 < ef) {
            for (int b = (n - 1) & ~31; n > 0 && b >= (p0 & ~31); b -= 32) {
                const int e = b + lane;
                const bool mv = e >= p0 && e < n;
                const unsigned long long val = mv ? pool[e] : 0ull;
                int sh = 0;
                for (unsigned mm = vb; mm; mm &= mm - 1) {
                    const unsigned long long cj = __shfl_sync(FULL, c, __ffs(mm) - 1);
                    sh += cj < (val & ~1ull) ? 1 : 0;
                }
                __syncwarp();
                if (mv && e + sh < ef)
                    pool[e + sh] = val;
                __syncwarp();
            }
            if (c != kInfKey && pos < ef)
                pool[pos] = c;
            __syncwarp();
            n = min(ef, n + nv);
        }
        return;
    }
    c = warp_sort_asc(c, lane);
    __syncwarp();
    sorted32[lane] = c;
    __syncwarp();
    const int pos = lane < nv ? lane + pool_lower_bound(pool, n, c) : ef;
    const int p0 = __shfl_sync(FULL, pos, 0);
    if (p0 < ef) {
        for (int b = (n - 1) & ~31; n > 0 && b >= (p0 & ~31); b -= 32) {
            const int e = b + lane;
            const bool mv = e >= p0 && e < n;
            unsigned long long val = 0;
            int dst = ef;
            if (mv) {
                val = pool[e];
                dst = e + sorted_count_less(sorted32, nv, val & ~1ull);
            }
            __syncwarp();
            if (mv && dst < ef)
                pool[dst] = val;
            __syncwarp();
        }
        if (lane < nv && pos < ef)
            pool[pos] = c;
        __syncwarp();
        n = min(ef, n + nv);
    }
}

// index of the first unexpanded record at or after `from`, or -1
__device__ __forceinline__ int first_unexpanded(const unsigned long long *pool, int n, int from,
                                                int lane) {
    for (int c = from; c < n; c += 32) {
        const int i = c + lane;
        const unsigned b = __ballot_sync(FULL, i < n && !(pool[i] & 1ull));
        if (b)
            return c + __ffs(b) - 1;
    }
    return -1;
}

// the neighbour ids and their attribute words of vertex u (slots lane, lane + 32)
struct Adjacency {
    uint32_t v0, v1, at0, at1;
};
template <bool TWO>
__device__ __forceinline__ Adjacency load_adjacency(const SearchArgs &a, uint32_t u, int lane) {
    Adjacency r{kNone, kNone, 0u, 0u};
    const int64_t row = (int64_t)u * a.R;
    if (lane < a.R) {
        r.v0 = __ldg(a.nbr + row + lane);
        r.at0 = __ldg(a.nbr_attr + row + lane);
    }
    if (TWO && lane + 32 < a.R) {
        r.v1 = __ldg(a.nbr + row + lane + 32);
        r.at1 = __ldg(a.nbr_attr + row + lane + 32);
    }
    return r;
}

// Hash of the first kk pool ids in order (equal hashes <=> same top-k, up to collisions).
__device__ __forceinline__ unsigned long long topk_hash(const unsigned long long *pool, int kk,
                                                        int lane) {
    unsigned long long h = 0ull;
    for (int j = lane; j < kk; j += 32)
        h ^= mix64((unsigned long long)key_id(pool[j]) * kGolden + (unsigned long long)(j + 1));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        h ^= __shfl_xor_sync(FULL, h, o);
    return h;
}

// Beam statistics fed to the learned early-stop model (warp-uniform).
__device__ __forceinline__ void stop_features(float *f, const unsigned long long *pool, int n,
                                              int k, int ef, int pidx, int iters, int last_surv,
                                              int since_change, int R) {
    // fast approximate operations are enough here: training traces and the
    // decisions both come from this same code
    const int kk = min(k, n);
    const float g0 = key_gamma(pool[0]);
    const float gk = key_gamma(pool[kk - 1]);
    const float gl = key_gamma(pool[n - 1]);
    const float gp = key_gamma(pool[pidx]);
    const float ik = __frcp_rn(gk + 1e-6f);
    f[0] = __logf(1.f + (float)iters) * 0.25f;                  // expansions so far
    f[1] = fminf(__fdividef(gk, g0 + 1e-6f) - 1.f, 10.f);        // spread of the top-k
    f[2] = fminf(gl * ik - 1.f, 10.f);                          // last record vs k-th
    f[3] = __fdividef((float)pidx, (float)ef);                  // depth of the next parent
    f[4] = fminf(gp * ik, 10.f);                                // next parent vs k-th
    f[5] = __fdividef((float)last_surv, (float)R);              // records inserted last time
    f[6] = __logf(1.f + (float)since_change) * 0.33f;           // expansions since a top-k change
    f[7] = __fdividef((float)n, (float)ef);                     // pool fill
}

__device__ __forceinline__ void clear_expanded(unsigned long long *pool, int n, int lane) {
    __syncwarp();
    for (int i = lane; i < n; i += 32)
        pool[i] &= ~1ull;
    __syncwarp();
}

// Several warps per query (wpq > 1): the group's warp 0 (the leader) runs the search;
// the others only share the distance passes.  For each batch of candidates the leader
// publishes the count and the row set in the group's control words and meets the other
// warps at the group's named barrier (1 + group index, wpq warps); all warps evaluate
// their passes and meet again, after which the leader reads every squared distance.  A
// negative count sends the other warps home.
__device__ __forceinline__ void group_bar(int grp, int wpq) {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(32 * wpq) : "memory");
}

template <typename VT, int CPL, bool EXACT, int RPT, bool GROUP>
__device__ __forceinline__ void group_eval(const VT *X, int xstride, const float *qv,
                                           const uint32_t *cid, float *d2s, int cnt, int lane,
                                           int wpq, int grp, volatile int *ctl, int rows_f32) {
    if (!GROUP) {
        eval_dist2<VT, CPL, EXACT, RPT>(X, xstride, qv, cid, d2s, cnt, lane);
        return;
    }
    if (lane == 0) {
        ctl[0] = cnt;
        ctl[1] = rows_f32;
    }
    __syncwarp();
    group_bar(grp, wpq);
    eval_dist2<VT, CPL, EXACT, RPT>(X, xstride, qv, cid, d2s, cnt, lane, 0, wpq);
    group_bar(grp, wpq);
}

struct WarpLayout {
    size_t pool, sorted, d2s, cid, cchi, hash, qv, ctl, total;
};

__host__ __device__ inline WarpLayout warp_layout(int ef_cap, int hash_bits, int xstride) {
    WarpLayout L;
    size_t o = 0;
    L.pool = o;
    o += sizeof(unsigned long long) * ef_cap;
    L.sorted = o;
    o += sizeof(unsigned long long) * 32;
    L.d2s = o;
    o += sizeof(float) * CAND;
    L.cid = o;
    o += sizeof(uint32_t) * CAND;
    L.cchi = o;
    o += sizeof(int) * CAND;
    o = (o + 15) & ~(size_t)15;
    L.hash = o;
    o += sizeof(uint32_t) * ((size_t)1 << hash_bits);
    o = (o + 15) & ~(size_t)15;
    L.qv = o;
    o += sizeof(float) * xstride;
    o = (o + 15) & ~(size_t)15;
    L.ctl = o;
    o += 16;
    L.total = o;
    return L;
}

// Rows too wide for a fixed chunk count per lane (CPL = 0) leave shared memory, not
// registers, to bound the resident warps (the query vector alone is 4 d bytes per warp,
// three blocks of eight warps at d = 960), so the f32 form of that variant may use the
// registers of three blocks (85 a thread) and keep twice the row loads in flight; the
// narrower types keep four blocks' worth, which a smaller visited filter can fill.
// GROUP: the form with several warps per query (wpq > 1); the one-warp form compiles
// without the group's bookkeeping.
template <typename VT, int CPL, bool EXACT, bool TWO, int RPT, bool GROUP>
__global__ void __launch_bounds__(
    256, ((CPL == 0 && std::is_same<VT, float>::value) || RPT == 4) ? 3 : 4) search_kernel(SearchArgs a, const VT *__restrict__ Xs,
                                                        int ef_cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wpq = GROUP ? a.wpq : 1, grp = GROUP ? wib / wpq : wib, wig = GROUP ? wib % wpq : 0;
    const WarpLayout L = warp_layout(ef_cap, a.hash_bits, a.xstride);
    unsigned char *base = smem + grp * L.total;
    unsigned long long *pool = reinterpret_cast<unsigned long long *>(base + L.pool);
    unsigned long long *sorted32 = reinterpret_cast<unsigned long long *>(base + L.sorted);
    float *d2s = reinterpret_cast<float *>(base + L.d2s);
    uint32_t *cid = reinterpret_cast<uint32_t *>(base + L.cid);
    int *cchi = reinterpret_cast<int *>(base + L.cchi);
    uint32_t *hash = reinterpret_cast<uint32_t *>(base + L.hash);
    float *qv = reinterpret_cast<float *>(base + L.qv);
    volatile int *ctl = reinterpret_cast<volatile int *>(base + L.ctl);
    const int H = 1 << a.hash_bits;
    const int R = a.R;
    const uint32_t alo = a.w.lo;
    // the learned stop's fp16 weights, staged once per block after the warps' areas
    __half *w16 = reinterpret_cast<__half *>(smem + ((blockDim.x >> 5) / wpq) * L.total);
    if (a.stop_w16 != nullptr) {
        for (int i = threadIdx.x; i < NHQ_MLP_PARAMS; i += blockDim.x)
            w16[i] = a.stop_w16[i];
        __syncthreads();
    }
    if (GROUP && wig != 0) {  // a helper warp of the group: distance passes only
        for (;;) {
            group_bar(grp, wpq);
            const int cnt = ctl[0];
            if (cnt < 0)
                break;
            if (ctl[1])
                eval_dist2<float, 0, false>(a.X, a.xstride, qv, cid, d2s, cnt, lane, wig, wpq);
            else
                eval_dist2<VT, CPL, EXACT, RPT>(Xs, a.xstride, qv, cid, d2s, cnt, lane, wig,
                                                wpq);
            group_bar(grp, wpq);
        }
        return;
    }

    for (;;) {
        unsigned long long qq = 0;
        if (lane == 0)
            qq = atomicAdd(a.counter, 1ull);
        qq = __shfl_sync(FULL, qq, 0);
        if (qq >= (unsigned long long)a.nq)
            break;
        const int64_t q = a.order ? (int64_t)a.order[qq] : (int64_t)qq;
        const int k = a.k_arr ? a.k_arr[q] : a.k;
        const int ef = a.ef_arr ? a.ef_arr[q] : a.ef;

        for (int i = lane; i < a.xstride; i += 32)
            qv[i] = i < a.d ? a.Q[q * a.qstride + i] : 0.f;
        uint32_t ahi;
        const uint32_t qa = pack_query_word(a.qattr + q * a.w.m, a.w, &ahi);
        for (int i = lane; i < H / 4; i += 32)
            reinterpret_cast<uint4 *>(hash)[i] = make_uint4(kNone, kNone, kNone, kNone);
        __syncwarp();

        int n = 0, cursor = 0, hcount = 0, iters = 0, ndc = 0;
        bool rebuilt = false;  // the visited filter forgot ids at least once
        int stage = a.h > 1 ? 1 : 2;
        int status = NHQ_OK;
        const uint64_t s0 = a.seed ^ mix64((uint64_t)q);

        // ---- seed set B, given: the valid distinct ids of the row, all evaluated
        for (int r = 0; a.seeds != nullptr && 32 * r < a.n_seeds; ++r) {
            const int j = 32 * r + lane;
            const uint32_t v = j < a.n_seeds ? a.seeds[q * a.n_seeds + j] : kNone;
            const bool valid = v != kNone && (int64_t)v < a.N;
            const unsigned same = __match_any_sync(FULL, v);
            bool take = valid && (__ffs(same) - 1) == lane;
            if (take)
                take = hash_insert(hash, a.hash_bits, v);  // false if an earlier round had it
            const unsigned kb = __ballot_sync(FULL, take);
            if (take) {
                prefetch_row(Xs, a.xstride, v);
                const int p = __popc(kb & lanemask_lt(lane));
                cid[p] = v;
                cchi[p] = chi_packed(a.attr[v], qa, ahi, alo);
            }
            __syncwarp();
            const int cnt = __popc(kb);
            hcount += cnt;
            ndc += cnt;
            if (cnt > 0) {
                group_eval<VT, CPL, EXACT, RPT, GROUP>(Xs, a.xstride, qv, cid, d2s, cnt, lane,
                                                       wpq, grp, ctl, 0);
                merge_round(pool, n, ef, candidate_key(lane, cnt, d2s, cid, cchi, a.w), sorted32,
                            lane);
            }
        }
        // ---- seed set B, random: first min(ef, 32) distinct ids of the stream, <= 64 draws
        const int want = a.seeds != nullptr ? 0 : min(ef, 32);
        int got = 0;
        for (int r = 0; r < 2 && got < want; ++r) {
            const uint32_t v = (uint32_t)(splitmix_at(s0, (uint64_t)(32 * r + lane)) %
                                          (unsigned long long)a.N);
            const unsigned same = __match_any_sync(FULL, v);
            bool first = (__ffs(same) - 1) == lane;
            if (r == 1 && first)
                first = !hash_contains(hash, a.hash_bits, v);
            const unsigned fb = __ballot_sync(FULL, first);
            const bool keep = first && __popc(fb & lanemask_lt(lane)) < want - got;
            const unsigned kb = __ballot_sync(FULL, keep);
            if (keep) {
                hash_insert(hash, a.hash_bits, v);
                prefetch_row(Xs, a.xstride, v);
                const int p = __popc(kb & lanemask_lt(lane));
                cid[p] = v;
                cchi[p] = chi_packed(a.attr[v], qa, ahi, alo);
            }
            __syncwarp();
            const int cnt = __popc(kb);
            got += cnt;
            hcount += cnt;
            ndc += cnt;
            if (cnt > 0) {
                group_eval<VT, CPL, EXACT, RPT, GROUP>(Xs, a.xstride, qv, cid, d2s, cnt, lane,
                                                       wpq, grp, ctl, 0);
                merge_round(pool, n, ef, candidate_key(lane, cnt, d2s, cid, cchi, a.w), sorted32,
                            lane);
            }
        }

        // ---- expansions.  The parent of the next expansion is known before the merge
        // (the smaller of the first unexpanded record and the smallest surviving new
        // candidate), so its adjacency loads are issued before the merge runs.
        cursor = 0;
        int pidx = first_unexpanded(pool, n, 0, lane);
        Adjacency adj{kNone, kNone, 0u, 0u};
        if (pidx >= 0)
            adj = load_adjacency<TWO>(a, key_id(pool[pidx]), lane);
        int last_surv = 0, since_change = 0;  // beam statistics of the learned stop
        for (;;) {
            if (pidx < 0) {
                if (stage == 1) {  // S1 exhausted C: S2 with C = C u R
                    stage = 2;
                    clear_expanded(pool, n, lane);
                    cursor = 0;
                    pidx = n > 0 ? 0 : -1;
                    if (pidx >= 0)
                        adj = load_adjacency<TWO>(a, key_id(pool[0]), lane);
                    continue;
                }
                break;
            }
            if (a.stop_every > 0 && iters >= a.stop_min &&
                (iters - a.stop_min) % a.stop_every == 0 && n >= k) {
                float f[NHQ_MLP_INPUTS];
                stop_features(f, pool, n, k, ef, pidx, iters, last_surv, since_change, R);
                if (a.tr_feat != nullptr) {  // training record: features now, label later
                    const unsigned long long th = topk_hash(pool, min(k, n), lane);
                    unsigned int slot = 0;
                    if (lane == 0)
                        slot = atomicAdd(a.tr_count, 1u);
                    slot = __shfl_sync(FULL, slot, 0);
                    if (lane == 0 && (int64_t)slot < a.tr_cap) {
#pragma unroll
                        for (int i = 0; i < NHQ_MLP_INPUTS; ++i)
                            a.tr_feat[(int64_t)slot * NHQ_MLP_INPUTS + i] = f[i];
                        a.tr_hash[slot] = th;
                        a.tr_q[slot] = (int32_t)q;
                    }
                }
                if (a.stop_w16 != nullptr && mlp_logit_warp(w16, f, lane) > a.stop_logit)
                    break;  // the model predicts the top-k will not change any more
            }
            if (iters >= a.max_iters) {
                status = NHQ_ERR_ITER_LIMIT;
                break;
            }
            ++iters;
            const unsigned long long pk = pool[pidx];
            __syncwarp();
            if (lane == 0)
                pool[pidx] = pk | 1ull;
            __syncwarp();
            cursor = pidx + 1;
            const uint32_t u = key_id(pk);

            if (hcount + R > (H >> 1)) {  // rebuild the visited filter from the pool
                rebuilt = true;
                __syncwarp();
                for (int i = lane; i < H / 4; i += 32)
                    reinterpret_cast<uint4 *>(hash)[i] = make_uint4(kNone, kNone, kNone, kNone);
                __syncwarp();
                for (int i = lane; i < n; i += 32)
                    hash_insert(hash, a.hash_bits, key_id(pool[i]));
                __syncwarp();
                hcount = n;
            }

            const uint32_t v0 = adj.v0, v1 = adj.v1, at0 = adj.at0, at1 = adj.at1;
            bool ok0 = v0 != kNone, ok1 = TWO && v1 != kNone;

            if (stage == 1) {  // S1: ceil(R/h) valid neighbours of smallest key
                const unsigned b0 = __ballot_sync(FULL, ok0), b1 = __ballot_sync(FULL, ok1);
                const int take = (R + a.h - 1) / a.h;
                if (__popc(b0) + __popc(b1) > take) {
                    const uint64_t su = mix64(s0 ^ mix64((uint64_t)u + 1));
                    const uint64_t k0 = splitmix_at(su, (uint64_t)lane);
                    const uint64_t k1 = splitmix_at(su, (uint64_t)(lane + 32));
                    int r0 = 0, r1 = 0;
                    for (int t = 0; t < R; ++t) {
                        const uint64_t kt = __shfl_sync(FULL, t < 32 ? k0 : k1, t & 31);
                        const bool okt = t < 32 ? ((b0 >> t) & 1u) : ((b1 >> (t - 32)) & 1u);
                        if (!okt)
                            continue;
                        r0 += (kt < k0 || (kt == k0 && t < lane)) ? 1 : 0;
                        r1 += (kt < k1 || (kt == k1 && t < lane + 32)) ? 1 : 0;
                    }
                    ok0 = ok0 && r0 < take;
                    ok1 = ok1 && r1 < take;
                }
            }

            bool nw0 = ok0 && hash_insert(hash, a.hash_bits, v0);
            bool nw1 = TWO && ok1 && hash_insert(hash, a.hash_bits, v1);
            // newly inserted ids fill the filter, pruned or not (they count as evaluated)
            hcount += __popc(__ballot_sync(FULL, nw0)) + (TWO ? __popc(__ballot_sync(FULL, nw1)) : 0);
            const int c0 = chi_packed(at0, qa, ahi, alo);
            const int c1 = TWO ? chi_packed(at1, qa, ahi, alo) : 0;
            if (a.w.mode == NHQ_W_CONSTANT && n == ef) {
                // Gamma >= w_l * chi in f32 (w_v * delta >= 0 and rounding is monotone)
                const unsigned long long worst = pool[ef - 1] & ~1ull;
                if (nw0 && make_key(__fmul_rn(a.w.wl, (float)c0), v0) > worst)
                    nw0 = false;
                if (TWO && nw1 && make_key(__fmul_rn(a.w.wl, (float)c1), v1) > worst)
                    nw1 = false;
            }
            if (nw0)
                prefetch_row(Xs, a.xstride, v0);
            if (TWO && nw1)
                prefetch_row(Xs, a.xstride, v1);
            const unsigned e0 = __ballot_sync(FULL, nw0);
            const unsigned e1 = TWO ? __ballot_sync(FULL, nw1) : 0u;
            if (nw0) {
                const int p = __popc(e0 & lanemask_lt(lane));
                cid[p] = v0;
                cchi[p] = c0;
            }
            if (TWO && nw1) {
                const int p = __popc(e0) + __popc(e1 & lanemask_lt(lane));
                cid[p] = v1;
                cchi[p] = c1;
            }
            __syncwarp();
            const int cnt = __popc(e0) + __popc(e1);
            ndc += cnt;
            unsigned long long k0 = kInfKey, k1 = kInfKey;
            if (cnt > 0) {
                group_eval<VT, CPL, EXACT, RPT, GROUP>(Xs, a.xstride, qv, cid, d2s, cnt, lane,
                                                       wpq, grp, ctl, 0);
                k0 = filter_key(candidate_key(lane, cnt, d2s, cid, cchi, a.w), pool, n, ef,
                                rebuilt);
                if (TWO)
                    k1 = filter_key(candidate_key(lane + 32, cnt, d2s, cid, cchi, a.w), pool, n,
                                    ef, rebuilt);
            }
            const unsigned long long cmin = warp_min_key(k0 < k1 ? k0 : k1);
            if (a.stop_every > 0)
                last_surv = __popc(__ballot_sync(FULL, k0 != kInfKey)) +
                            (TWO ? __popc(__ballot_sync(FULL, k1 != kInfKey)) : 0);
            // next parent and its adjacency, before the merge
            const int uo = first_unexpanded(pool, n, cursor, lane);
            const unsigned long long uo_key = uo >= 0 ? (pool[uo] & ~1ull) : kInfKey;
            int next = -1;
            uint32_t next_id = kNone;
            const int cpos = cmin != kInfKey ? pool_rank_uniform(pool, n, cmin, lane) : n;
            if (cmin != kInfKey && cmin < uo_key) {
                next = cpos;
                next_id = key_id(cmin);
            } else if (uo >= 0) {
                next = uo;
                next_id = key_id(uo_key);
            }
            if (next >= 0)
                adj = load_adjacency<TWO>(a, next_id, lane);
            since_change = (cmin != kInfKey && cpos < k) ? 0 : since_change + 1;
            if (cmin != kInfKey) {
                merge_round(pool, n, ef, k0, sorted32, lane);
                if (TWO)
                    merge_round(pool, n, ef, k1, sorted32, lane);
                cursor = min(cursor, cpos);
            }
            pidx = next;
            if (stage == 1 && cmin == kInfKey) {  // local optimum ends S1
                stage = 2;
                clear_expanded(pool, n, lane);
                cursor = 0;
                pidx = n > 0 ? 0 : -1;
                if (pidx >= 0 && key_id(pool[0]) != next_id)
                    adj = load_adjacency<TWO>(a, key_id(pool[0]), lane);
            }
        }

        __syncwarp();
        if (a.tr_final != nullptr) {
            const unsigned long long th = topk_hash(pool, min(k, n), lane);
            if (lane == 0)
                a.tr_final[q] = th;
        }
        int first_pad = 0;
        if (!std::is_same<VT, float>::value && a.rerank) {
            // re-score the final pool with the f32 vectors ...
            for (int b0 = 0; b0 < n; b0 += CAND) {
                const int cb = min(CAND, n - b0);
                for (int j = lane; j < cb; j += 32) {
                    const uint32_t id = key_id(pool[b0 + j]);
                    cid[j] = id;
                    cchi[j] = chi_packed(a.attr[id], qa, ahi, alo);
                }
                __syncwarp();
                group_eval<float, 0, false, 2, GROUP>(a.X, a.xstride, qv, cid, d2s, cb, lane,
                                                      wpq, grp, ctl, 1);
                for (int j = lane; j < cb; j += 32)
                    pool[b0 + j] = candidate_key(j, cb, d2s, cid, cchi, a.w);
                __syncwarp();
            }
            // ... and return its k smallest records by (Gamma, id), one minimum at a time
            const int kk = min(k, n);
            for (int j = 0; j < kk; ++j) {
                unsigned long long best = kInfKey;
                int bi = -1;
                for (int i = lane; i < n; i += 32) {
                    const unsigned long long v = pool[i];
                    if (v < best) {
                        best = v;
                        bi = i;
                    }
                }
                const unsigned long long m = warp_min_key(best);
                __syncwarp();
                if (bi >= 0 && best == m)
                    pool[bi] = kInfKey;
                if (lane == 0) {
                    const int64_t o = q * a.k_out + j;
                    const uint32_t id = key_id(m);
                    a.ids[o] = id;
                    if (a.dists)
                        a.dists[o] = key_gamma(m);
                    if (a.chi)
                        a.chi[o] = (uint8_t)chi_packed(a.attr[id], qa, ahi, alo);
                }
                __syncwarp();
            }
            first_pad = kk;
        }
        for (int j = first_pad + lane; j < a.k_out; j += 32) {
            const int64_t o = q * a.k_out + j;
            uint32_t id = kNone;
            float g = __int_as_float(0x7f800000);
            if (j < k && j < n) {
                id = key_id(pool[j]);
                g = key_gamma(pool[j]);
            }
            a.ids[o] = id;
            if (a.dists)
                a.dists[o] = g;
            if (a.chi)
                a.chi[o] = id == kNone ? (uint8_t)255 : (uint8_t)chi_packed(a.attr[id], qa, ahi, alo);
        }
        if (lane == 0) {
            if (a.status)
                a.status[q] = status;
            if (a.ndc)
                a.ndc[q] = ndc;
            if (a.expansions)
                a.expansions[q] = iters;
        }
        __syncwarp();
    }
    if (GROUP) {  // no query left: release the helper warps
        if (lane == 0)
            ctl[0] = -1;
        __syncwarp();
        group_bar(grp, wpq);
    }
}

// the smallest visited filter the rebuild rule allows (a rebuilt filter holds at most
// ef ids and takes R more per expansion before it is half full again): at large ef the
// filter is most of a warp's shared memory, and resident warps matter more than the
// rarer rebuilds a larger filter would save
int auto_hash_bits(int ef_cap, int R) {
    int need = 2 * (ef_cap + R) + 64;
    int bits = 10;  // 1024 slots: small enough for 32 resident warps per SM at small ef
    while ((1 << bits) < need)
        ++bits;
    return bits;
}

template <typename VT, int CPL, bool EXACT, bool TWO, int RPT, bool GROUP>
cudaError_t launch_kernel(const SearchArgs &a, const VT *X, int ef_cap, int wpb, size_t smem,
                          int sm_count, cudaStream_t s) {
    auto kfn = search_kernel<VT, CPL, EXACT, TWO, RPT, GROUP>;
    cudaError_t e =
        cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 32 * wpb, smem)) !=
        cudaSuccess)
        return e;
    if (per_sm < 1)
        per_sm = 1;
    int64_t blocks = (int64_t)per_sm * sm_count;
    const int64_t groups = wpb / a.wpq;  // queries in flight per block
    const int64_t need = (a.nq + groups - 1) / groups;
    if (blocks > need)
        blocks = need;
    kfn<<<(unsigned)blocks, 32 * wpb, smem, s>>>(a, X, ef_cap);
    return cudaGetLastError();
}

// one warp per query, or a group (four rows per team take one warp per query only)
template <typename VT, int CPL, bool EXACT, bool TWO, int RPT = 2>
cudaError_t launch_variant(const SearchArgs &a, const VT *X, int ef_cap, int wpb, size_t smem,
                           int sm_count, cudaStream_t s) {
    if (a.wpq == 1)
        return launch_kernel<VT, CPL, EXACT, TWO, RPT, false>(a, X, ef_cap, wpb, smem,
                                                               sm_count, s);
    if (RPT != 2)
        return cudaErrorInvalidValue;
    return launch_kernel<VT, CPL, EXACT, TWO, 2, true>(a, X, ef_cap, wpb, smem, sm_count, s);
}

template <typename VT, bool TWO>
cudaError_t launch_shape(const SearchArgs &a, const VT *X, int ef_cap, int wpb, size_t smem,
                         int sm_count, cudaStream_t s) {
    constexpr int PC = VecTraits<VT>::kPerChunk;
    const int nchunk = a.xstride / PC;
    const bool four = a.tile_rows == 4;  // rows per team and pass (wide rows: always 2)
    if (nchunk == 2 * TEAM)
        return four ? launch_variant<VT, 2, true, TWO, 4>(a, X, ef_cap, wpb, smem, sm_count, s)
                    : launch_variant<VT, 2, true, TWO>(a, X, ef_cap, wpb, smem, sm_count, s);
    if (nchunk == 4 * TEAM)
        return four ? launch_variant<VT, 4, true, TWO, 4>(a, X, ef_cap, wpb, smem, sm_count, s)
                    : launch_variant<VT, 4, true, TWO>(a, X, ef_cap, wpb, smem, sm_count, s);
    if (nchunk < 4 * TEAM)
        return four ? launch_variant<VT, 4, false, TWO, 4>(a, X, ef_cap, wpb, smem, sm_count, s)
                    : launch_variant<VT, 4, false, TWO>(a, X, ef_cap, wpb, smem, sm_count, s);
    return launch_variant<VT, 0, false, TWO>(a, X, ef_cap, wpb, smem, sm_count, s);
}

template <typename VT>
cudaError_t launch_dtype(const SearchArgs &a, const VT *X, int ef_cap, int wpb, size_t smem,
                         int sm_count, cudaStream_t s) {
    if (a.R > 32)
        return launch_shape<VT, true>(a, X, ef_cap, wpb, smem, sm_count, s);
    return launch_shape<VT, false>(a, X, ef_cap, wpb, smem, sm_count, s);
}


}  // namespace
}  // namespace nhq
