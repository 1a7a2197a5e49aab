// k_knn_tc.cu -- candidate sets C(u) of Sec. 4.1 (the exact K nearest by Gamma)
// with the dot products on the 5th-generation tensor cores.
//
// delta^2(u, v) = |u|^2 + |v|^2 - 2 u.v with u, v the bf16-rounded object rows
// (for integer components 0..255 the rounding is exact and every sum stays
// below 2^24, so delta^2, delta and Gamma equal the f32 path bit for bit).
//
// The objects are taken in the order of their packed attribute words (a stable
// sort, so the tuple runs are contiguous): a tile of 128 columns then mostly
// holds one attribute tuple, chi is one number per row and tile, and where the
// row's bound for that chi is already negative the tile costs no filtering.
// Records keep the original ids, so the result (ties by id included) does not
// depend on this order.
//
// One CTA owns 128 rows and sweeps all column tiles of 128, starting at its
// own (diagonal) tile so that each row first meets the objects of its own tuple
// (concurrent CTAs then read a sliding window of neighbouring tiles from L2):
//   warp 0              scheduler + TMA: decides for each tile whether any row
//                       can still take a record from it (skipped tiles are never
//                       loaded or multiplied), then one lane loads 128B-swizzled
//                       bf16 boxes of 128 rows x 64 dims; with d <= 128 the row
//                       operand is loaded once and stays resident
//   warp 1 (one lane)   tcgen05.mma kind::f16, M = 128, N = 128, K = 16, f32
//                       accumulators in four TMEM buffers of 128 columns
//   warps 2..9          epilogue, two groups of four warps taking the kept tiles
//                       alternately: tcgen05.ld of the warp's 32 lanes (= rows),
//                       delta^2 and chi of every pair against a per-row table of
//                       delta^2 bounds by chi (branch-free); the survivors wait in
//                       a per-row queue of the group and enter, with exact Gamma
//                       (Eq. 6), the row's max-heap of the K best records in
//                       shared memory (shared by the groups under a per-row lock,
//                       sorted once at the end)
// A tile is skipped when every row's bound for the smallest chi the tile can
// have with it is negative: in the constant and filter weightings a row whose K
// records all match its tuple rejects every other tuple.  The bounds only
// tighten, so a decision taken on older bounds is still correct.
// Every wait is bounded; a timeout records an error code, the other waits see it
// and return, the CTA drains its tensor-core work, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "nhq_internal.cuh"

namespace nhq {

namespace {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int KMAX = 64;
// u64 entries per row heap: slot 0 unused, 1..K the heap, K+1 a zero sentinel (so a
// node's two children are one aligned 16-byte pair); even, so every row is 16-byte aligned
constexpr int LSTRIDE = KMAX + 2;
constexpr int NTHREADS = 320;
constexpr uint32_t BOX_BYTES = BM * BK * 2;  // one operand box: 16 KB
// operand ring of 6 boxes: 3 stages of (A, B) boxes, or with d <= 128 the resident
// A boxes (2) and 4 single-box B stages
constexpr uint32_t RING_BYTES = 6 * BOX_BYTES;
constexpr int MAX_STAGES = 4;
constexpr int NBUF = 4;  // accumulator buffers in TMEM (two per epilogue group)
constexpr uint32_t TMEM_COLS = NBUF * BN;
constexpr long long kWaitLimit = 1ll << 26;
// survivors of the filter wait in a queue of QCAP records per row and enter the row's heap
// in flushes that every lane of the warp runs at once (a flush when some lane's queue is
// half full, every FLUSH_TILES kept tiles, and at the end)
constexpr int QCAP = 12;
constexpr int FLUSH_TILES = 16;

struct TcArgs {
    const float *norms;     // |x|^2 of the bf16-rounded rows, sorted order
    const uint32_t *attr;   // packed attribute words, sorted order
    const uint32_t *perm;   // sorted position -> original id
    int64_t N;
    int kblocks;
    Fusion w;
    int K;
    uint32_t *ids;
    float *dists;
    int *err;
};

// ---- PTX wrappers ----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t a, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false (and an error code recorded) if the phase never completes,
// or false early once another thread has recorded an error
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity, int *err, int code) {
    for (long long i = 0; i < kWaitLimit; ++i) {
        if (mbar_try_wait(a, parity))
            return true;
        if ((i & 1023) == 1023 && *reinterpret_cast<volatile int *>(err) != 0)
            return false;
    }
    atomicCAS(err, 0, code);
    return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
// shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups
// 1024 bytes apart (the layout TMA writes for a 64-element bf16 box width)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);  // start address
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused with swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
    d |= (uint64_t)1 << 46;                  // descriptor version
    d |= (uint64_t)2 << 61;                  // 128-byte swizzle
    return d;
}
// instruction descriptor: bf16 x bf16 -> f32, both K-major, N = 128, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
          "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// max-heap hp[1..n] with hp[n+1] == 0: sift `key` down from node i
__device__ __forceinline__ void heap_sift(unsigned long long *hp, int n, int i,
                                          unsigned long long key) {
    for (;;) {
        const int c = 2 * i;
        if (c > n)
            break;
        const ulonglong2 ch = *reinterpret_cast<const ulonglong2 *>(hp + c);
        const bool right = ch.y > ch.x;
        const unsigned long long big = right ? ch.y : ch.x;
        if (big <= key)
            break;
        hp[i] = big;
        i = c + (right ? 1 : 0);
    }
    hp[i] = key;
}

// v[j] for a runtime j by a tree of selects (the array stays in registers)
__device__ __forceinline__ uint32_t pick32(const uint32_t (&v)[32], int j) {
    uint32_t t16[16], t8[8], t4[4], t2[2];
#pragma unroll
    for (int i = 0; i < 16; ++i)
        t16[i] = (j & 16) ? v[i + 16] : v[i];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        t8[i] = (j & 8) ? t16[i + 8] : t16[i];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        t4[i] = (j & 4) ? t8[i + 4] : t8[i];
#pragma unroll
    for (int i = 0; i < 2; ++i)
        t2[i] = (j & 2) ? t4[i + 2] : t4[i];
    return (j & 1) ? t2[1] : t2[0];
}

// row of the bound table for a chi: the table holds chi = 0..4; Gamma grows with chi,
// so the bound of chi = 4 also holds (more loosely) for every larger chi
__device__ __forceinline__ int chi_level(int chi) { return chi < 4 ? chi : 4; }

// bounded wait for the scheduler's decision on the i-th tile of the sweep
__device__ __forceinline__ bool wait_decided(const int *decided, int i, int *err, int code) {
    for (long long it = 0; it < kWaitLimit; ++it) {
        if (*reinterpret_cast<const volatile int *>(decided) > i) {
            __threadfence_block();
            return true;
        }
        if ((it & 1023) == 1023 && *reinterpret_cast<volatile int *>(err) != 0)
            return false;
        __nanosleep(32);
    }
    atomicCAS(err, 0, code);
    return false;
}
// the first sweep index >= i that the scheduler kept (ntiles if none), scanning the
// published skip bits a word at a time; -1 if a wait failed
__device__ __forceinline__ int next_kept(const int *decided, const uint32_t *bits, int i,
                                         int ntiles, int *err, int code) {
    while (i < ntiles) {
        if (!wait_decided(decided, i, err, code))
            return -1;
        const int dec = *reinterpret_cast<const volatile int *>(decided);
        while (i < dec) {
            const int sh = i & 31;
            const int n = dec - i < 32 - sh ? dec - i : 32 - sh;
            const uint32_t w = reinterpret_cast<const volatile uint32_t *>(bits)[i >> 5] >> sh;
            const uint32_t keep = ~w & (n == 32 ? 0xFFFFFFFFu : ((1u << n) - 1u));
            if (keep != 0u)
                return i + __ffs((int)keep) - 1;
            i += n;
        }
    }
    return ntiles;
}

struct TcSmem {  // byte offsets in the dynamic shared memory (after 1024-byte alignment)
    uint32_t heaps, queue, qchi, rowcnt, rowlock, limtab, meta, bits, bars, misc, total;
};
__host__ __device__ inline TcSmem tc_smem_layout(int ntiles) {
    TcSmem L;
    L.heaps = RING_BYTES;
    L.queue = L.heaps + 8u * BM * LSTRIDE;                         // [2][QCAP][BM] u64
    L.qchi = L.queue + 8u * 2 * QCAP * BM;                         // [2][QCAP][BM] u8
    L.rowcnt = L.qchi + 1u * 2 * QCAP * BM;                        // [BM] records per heap
    L.rowlock = L.rowcnt + 4u * BM;                                // [BM] heap locks
    L.limtab = L.rowlock + 4u * BM;                                // [5][BM] f32
    L.meta = L.limtab + 4u * 5 * BM;                               // per epilogue warp: norm, attr, id [BN]
    L.bits = L.meta + 4u * 3 * 8 * BN;                             // skip bit per tile
    L.bars = L.bits + ((4u * (uint32_t)((ntiles + 31) / 32) + 15u) & ~15u);
    L.misc = L.bars + 8u * 32;                                     // decided counter, TMEM address
    L.total = L.misc + 16;
    return L;
}

// MODE: the weighting (NHQ_W_CONSTANT, NHQ_W_PROPORTIONAL or NHQ_W_HARMONIC), fixed at
// compile time so that each form carries only its own Gamma and bound code
template <int MODE>
__global__ void __launch_bounds__(NTHREADS, 1)
    knn_tc_kernel(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int ntiles = (int)((a.N + BN - 1) / BN);
    const TcSmem L = tc_smem_layout(ntiles);
    unsigned char *ring = sm;
    unsigned long long *heaps = reinterpret_cast<unsigned long long *>(sm + L.heaps);
    unsigned long long *queue = reinterpret_cast<unsigned long long *>(sm + L.queue);
    unsigned char *qchi = sm + L.qchi;
    int *rowcnt = reinterpret_cast<int *>(sm + L.rowcnt);
    int *rowlock = reinterpret_cast<int *>(sm + L.rowlock);
    float *limtab = reinterpret_cast<float *>(sm + L.limtab);
    unsigned char *meta = sm + L.meta;
    uint32_t *skipbits = reinterpret_cast<uint32_t *>(sm + L.bits);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(sm + L.bars);
    int *decided = reinterpret_cast<int *>(sm + L.misc);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(sm + L.misc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    const int kb_n = a.kblocks;
    const bool resA = kb_n <= 2;  // the row operand stays in shared memory
    const int nst = resA ? 4 : 3;
    const uint32_t sbytes = resA ? BOX_BYTES : 2 * BOX_BYTES;
    const uint32_t boff = resA ? 0u : BOX_BYTES;  // B box within a stage
    unsigned char *aregion = ring + 4 * BOX_BYTES;
    const int t0 = (int)blockIdx.x;  // the diagonal tile comes first
    auto tile_at = [&](int i) { return t0 + i < ntiles ? t0 + i : t0 + i - ntiles; };
    auto bar = [&](int i) { return smem_u32(bars + i); };
    const int FULL0 = 0, EMPTY0 = MAX_STAGES, TFULL0 = 2 * MAX_STAGES, TEMPTY0 = TFULL0 + NBUF,
              AFULL = TEMPTY0 + NBUF, DONE = AFULL + 1;
    // whole tiles are rejected only where a negative bound is possible
    constexpr bool skip_on = MODE == NHQ_W_CONSTANT;

    for (int i = threadIdx.x; i < (ntiles + 31) / 32; i += NTHREADS)
        skipbits[i] = 0u;
    for (int i = threadIdx.x; i < 5 * BM; i += NTHREADS)
        limtab[i] = __int_as_float(0x7f800000);
    for (int i = threadIdx.x; i < BM; i += NTHREADS) {
        rowcnt[i] = 0;
        rowlock[i] = 0;
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < MAX_STAGES; ++q) {
            mbar_init(bar(FULL0 + q), 1);
            mbar_init(bar(EMPTY0 + q), 1);
        }
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(bar(TFULL0 + b), 1);
            mbar_init(bar(TEMPTY0 + b), BM);  // the 128 threads of one epilogue group
        }
        mbar_init(bar(AFULL), 1);
        mbar_init(bar(DONE), 1);
        *decided = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                smem_u32(tmem_holder)),
            "r"(TMEM_COLS)
            : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        // ---------------- scheduler (all lanes) + TMA producer (lane 0)
        uint32_t ra[4];
        bool rv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t u = row0 + lane + 32 * k;
            rv[k] = u < a.N;
            ra[k] = rv[k] ? a.attr[u] : 0u;
        }
        int stage = 0;
        uint32_t phase = 0;
        bool ok = true;
        if (resA && lane == 0) {
            mbar_expect_tx(bar(AFULL), (uint32_t)kb_n * BOX_BYTES);
            for (int kb = 0; kb < kb_n; ++kb)
                tma_load_2d(smem_u32(aregion + kb * BOX_BYTES), &tmap, bar(AFULL), kb * BK,
                            (int)row0);
        }
        // first and last attribute word of tiles i..i+31 (lane l: tile i + l), loaded
        // one group of 32 ahead
        auto codes = [&](int base, uint32_t &f, uint32_t &l) {
            const int ii = base + lane;
            f = l = 0u;
            if (ii < ntiles) {
                const int64_t c0 = (int64_t)tile_at(ii) * BN;
                const int64_t c1 = (c0 + BN < a.N ? c0 + BN : a.N) - 1;
                f = __ldg(a.attr + c0);
                l = __ldg(a.attr + c1);
            }
        };
        uint32_t cf, cl, nf, nl;
        int gcur = 0;  // group of 32 tiles whose codes are in cf, cl
        codes(0, cf, cl);
        codes(32, nf, nl);
        uint32_t wbits = 0u;       // skip bits of the current word, published by lane 0
        uint32_t dead_tuple = 0u;  // a tuple whose tiles were found dead (stays dead)
        bool have_dead = false;
        int i = 0;
        while (i < ntiles && ok) {
            if ((i >> 5) != gcur) {
                cf = nf;
                cl = nl;
                ++gcur;
                codes((gcur + 1) * 32, nf, nl);
            }
            const int j = i & 31;
            const uint32_t tf = __shfl_sync(0xFFFFFFFFu, cf, j);
            const uint32_t tl = __shfl_sync(0xFFFFFFFFu, cl, j);
            bool need = true;
            if (skip_on) {
                if (have_dead && tf == tl && tf == dead_tuple) {
                    need = false;  // the bounds only tighten
                } else {
                    // the smallest chi a column of the tile can have with the row: 0 if
                    // the row's word lies in the tile's (sorted) range, that of the
                    // tile's one tuple if it has one, else at least 1
                    bool live = false;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (!rv[k])
                            continue;
                        const int ch = (ra[k] >= tf && ra[k] <= tl)
                                           ? 0
                                           : (tf == tl ? chi_level(chi_packed(ra[k], tf, a.w.hi,
                                                                              a.w.lo))
                                                       : 1);
                        const float lim = reinterpret_cast<const volatile float *>(
                            limtab)[ch * BM + lane + 32 * k];
                        live = live || !(lim < 0.f);
                    }
                    need = __any_sync(0xFFFFFFFFu, live);
                    if (!need && tf == tl) {
                        dead_tuple = tf;
                        have_dead = true;
                    }
                }
            }
            int step = 1;
            if (!need) {
                // the following tiles of this group with the same first and last word
                // are rejected by the same bounds
                const uint32_t same =
                    __ballot_sync(0xFFFFFFFFu, gcur * 32 + lane < ntiles && cf == tf && cl == tl) >>
                    j;
                step = (~same == 0u) ? 32 - j : __ffs((int)~same) - 1;
                wbits |= (step == 32 ? 0xFFFFFFFFu : ((1u << step) - 1u)) << j;
            }
            const int inext = i + step;
            // publish before loading (the consumers need the decision first) and at the
            // end of every word
            const bool word_end = (inext & 31) == 0 || inext >= ntiles;
            if (lane == 0 && (need || word_end)) {
                skipbits[i >> 5] = wbits;
                __threadfence_block();
                *reinterpret_cast<volatile int *>(decided) = need ? i + 1 : inext;
            }
            if (need && lane == 0) {
                const int t = tile_at(i);
                for (int kb = 0; kb < kb_n && ok; ++kb) {
                    ok = mbar_wait(bar(EMPTY0 + stage), phase ^ 1u, a.err, 1);
                    if (!ok)
                        break;
                    const uint32_t dst = smem_u32(ring + stage * sbytes);
                    mbar_expect_tx(bar(FULL0 + stage), sbytes);
                    if (!resA)
                        tma_load_2d(dst, &tmap, bar(FULL0 + stage), kb * BK, (int)row0);
                    tma_load_2d(dst + boff, &tmap, bar(FULL0 + stage), kb * BK, t * BN);
                    if (++stage == nst) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (word_end)
                wbits = 0u;
            ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
            i = inext;
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        int stage = 0, p = 0;
        uint32_t phase = 0;
        bool ok = true, issued = false;
        if (resA)
            ok = mbar_wait(bar(AFULL), 0, a.err, 6);
        for (int i = 0; ok; ++i) {
            if (skip_on) {  // otherwise every tile is kept
                i = next_kept(decided, skipbits, i, ntiles, a.err, 7);
                if (i < 0) {
                    ok = false;
                    break;
                }
            }
            if (i >= ntiles)
                break;
            const int b = p % NBUF;
            const uint32_t tph = (uint32_t)(p / NBUF) & 1u;
            ++p;
            ok = mbar_wait(bar(TEMPTY0 + b), tph ^ 1u, a.err, 2);
            if (!ok)
                break;
            tc_fence_after();
            const uint32_t d_tmem = tmem + (uint32_t)(b * BN);
            for (int kb = 0; kb < kb_n; ++kb) {
                ok = mbar_wait(bar(FULL0 + stage), phase, a.err, 3);
                if (!ok)
                    break;
                tc_fence_after();
                const uint32_t sS = smem_u32(ring + stage * sbytes);
                const uint32_t sA = resA ? smem_u32(aregion + kb * BOX_BYTES) : sS;
                const uint32_t sB = sS + boff;
#pragma unroll
                for (int k4 = 0; k4 < BK / 16; ++k4)
                    umma_bf16(d_tmem, sw128_desc(sA + 32u * k4), sw128_desc(sB + 32u * k4),
                              (kb | k4) != 0 ? 1u : 0u);
                issued = true;
                umma_commit(bar(EMPTY0 + stage));  // the stage is free once these complete
                if (++stage == nst) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (ok)
                umma_commit(bar(TFULL0 + b));  // accumulators of this tile are complete
        }
        if (issued) {  // wait for every issued MMA before TMEM can be released
            umma_commit(bar(DONE));
            mbar_wait(bar(DONE), 0, a.err, 4);
        }
    } else if (warp >= 2) {
        // ---------------- epilogue: two groups of four warps (g = (warp - 2) / 4) take
        // the kept tiles alternately (the k-th kept tile: group k mod 2, accumulator
        // buffer k mod NBUF).  Thread (warp, lane) serves row r = 32 (warp mod 4) + lane
        // (sorted position), warp mod 4 being the warp's TMEM lane quarter, so each row
        // has one thread in each group; the row's heap is shared, and a flush into it
        // holds the row's lock.
        const int g = (warp - 2) >> 2;
        const int ew = warp - 2;  // this warp's copy of the tile metadata
        const int r = (warp & 3) * 32 + lane;
        const int64_t u = row0 + r;
        const bool row_ok = u < a.N;
        const float nu = row_ok ? a.norms[u] : 0.f;
        const uint32_t au = row_ok ? a.attr[u] : 0u;
        unsigned long long *hp = heaps + r * LSTRIDE;
        unsigned long long *qk = queue + g * QCAP * BM + r;  // this group's queue of the row
        unsigned char *qc = qchi + g * QCAP * BM + r;        // their chi, stride BM
        volatile int *hcnt = rowcnt + r;                      // records in the row's heap
        int *hlock = rowlock + r;
        int qn = 0;  // records in this group's queue of the row
        float *mnorm = reinterpret_cast<float *>(meta) + ew * 3 * BN;
        uint32_t *mattr = reinterpret_cast<uint32_t *>(mnorm + BN);
        uint32_t *mid = mattr + BN;
        const int K = a.K;
        // delta^2 bound of chi = c for this row at limtab[c * BM + r]: a record with
        // this chi and a larger delta^2 cannot reach the row's current K-th record
        // (Gamma grows with delta and with chi); -1 where no delta can
        float fac[5];
#pragma unroll
        for (int c = 0; c < 5; ++c)
            fac[c] = MODE == NHQ_W_CONSTANT   ? a.w.wl * (float)c
                     : MODE == NHQ_W_HARMONIC // the attribute term h of the harmonic mean
                         ? (a.w.wl > 0.f ? (c == 0 ? 1.f : a.w.wl * (float)c) : (float)c)
                         : (float)a.w.m / (float)(a.w.m + c);
        const float inv_wv = a.w.wv > 0.f ? 1.f / a.w.wv : 0.f;
        Fusion wf = a.w;  // the weights with the mode as a constant
        wf.mode = MODE;
        auto update_lim = [&](unsigned long long thr) {  // thr: the row's K-th record
            // with slack 1e-5: the f32 roundings of Gamma and of these bounds stay far inside it
            const float gt = __uint_as_float((uint32_t)(thr >> 32)) * 1.00001f;
#pragma unroll
            for (int cc = 0; cc < 5; ++cc) {
                float tt;
                if constexpr (MODE == NHQ_W_CONSTANT) {
                    tt = a.w.wv > 0.f ? (gt - fac[cc]) * inv_wv
                                      : (gt >= fac[cc] ? __int_as_float(0x7f800000) : -1.f);
                } else if constexpr (MODE == NHQ_W_HARMONIC) {
                    // Gamma = 2 delta h / (delta + h) < 2 h for every delta: no bound while
                    // gt >= 2 h; below that, delta <= gt h / (2 h - gt)
                    const float h = fac[cc];
                    tt = (h == 0.f || gt >= 2.f * h) ? __int_as_float(0x7f800000)
                                                     : gt * h / (2.f * h - gt);
                } else {
                    tt = gt * fac[cc];
                }
                limtab[cc * BM + r] = tt < 0.f ? -1.f : tt * tt;
            }
        };
        // The queued records enter the heap under the row's lock: exact Gamma (Eq. 6) and
        // the key test, then the bounds once for the whole flush.  The lock's other user
        // is this row's thread of the other group, which holds it only for a flush (no
        // waits inside), so the bounded acquisition ends; a failure is recorded.
        auto flush = [&]() {
            if (qn == 0)
                return;
            bool locked = false;
            for (long long it = 0; it < kWaitLimit; ++it) {
                if (atomicCAS(hlock, 0, 1) == 0) {
                    locked = true;
                    break;
                }
                if ((it & 1023) == 1023 && *reinterpret_cast<volatile int *>(a.err) != 0)
                    break;
            }
            if (!locked) {
                atomicCAS(a.err, 0, 9);
                qn = 0;
                return;
            }
            __threadfence_block();
            int cnt = *hcnt;
            unsigned long long thr = cnt == K ? hp[1] : kInfKey;
            bool touched = false;
            for (int e = 0; e < qn; ++e) {
                const unsigned long long rec = qk[e * BM];
                const float gm = fusion_gamma(__fsqrt_rn(__uint_as_float((uint32_t)(rec >> 32))),
                                              (int)qc[e * BM], wf);
                const unsigned long long key =
                    ((unsigned long long)__float_as_uint(gm) << 32) | (uint32_t)rec;
                if (key >= thr)
                    continue;
                if (cnt < K) {  // filling: unordered, heapified once full
                    hp[1 + cnt] = key;
                    if (++cnt == K) {
                        hp[K + 1] = 0ull;
                        for (int h = K / 2; h >= 1; --h)
                            heap_sift(hp, K, h, hp[h]);
                        thr = hp[1];
                        touched = true;
                    }
                } else {  // replace the largest of the K records
                    heap_sift(hp, K, 1, key);
                    thr = hp[1];
                    touched = true;
                }
            }
            *hcnt = cnt;
            if (touched)
                update_lim(thr);
            __threadfence_block();
            atomicExch(hlock, 0);
            qn = 0;
        };
        const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
        const float *lt = limtab + r;
        bool ok = true;
        int k = -1;  // index of the current tile in the kept sequence
        int p = 0;   // tiles this group processed
        // a tile's column metadata in registers until it is stored to this warp's copy
        float rn[4];
        uint32_t rat[4], rid[4];
        auto load_meta = [&](int ii) {
            const int64_t cb = (int64_t)tile_at(ii) * BN;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int64_t col = cb + lane + 32 * kk;
                const bool in = col < a.N;
                rn[kk] = in ? __ldg(a.norms + col) : 0.f;
                rat[kk] = in ? __ldg(a.attr + col) : 0u;
                rid[kk] = in ? __ldg(a.perm + col) : 0u;
            }
        };
        // without tile skipping every tile is kept (k = i): there are no decisions to wait
        // for, and this group's next tile's metadata loads while this one is filtered
        if (!skip_on && g < ntiles)
            load_meta(g);
        for (int i = 0;; ++i) {
            if (skip_on) {
                i = next_kept(decided, skipbits, i, ntiles, a.err, 8);
                ok = i >= 0;
                if (!__all_sync(0xFFFFFFFFu, ok)) {
                    ok = false;
                    break;
                }
                i = __shfl_sync(0xFFFFFFFFu, i, 0);  // every lane saw the same published bits
            }
            const bool last = i >= ntiles;  // no tile left: the final flush
            if (!last) {
                ++k;
                if ((k & 1) != g)
                    continue;  // the other group's tile
                const int t = tile_at(i);
                const int b = k % NBUF;
                const uint32_t tph = (uint32_t)(k / NBUF) & 1u;
                ++p;
                const int64_t cbase = (int64_t)t * BN;
                // with skipping, the loads are issued here, before the accumulator wait
                if (skip_on)
                    load_meta(i);
                ok = mbar_wait(bar(TFULL0 + b), tph, a.err, 5);
                __syncwarp();  // every lane is done with the previous tile's metadata
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    mnorm[lane + 32 * kk] = rn[kk];
                    mattr[lane + 32 * kk] = rat[kk];
                    mid[lane + 32 * kk] = rid[kk];
                }
                __syncwarp();  // metadata visible; tcgen05.ld below needs the warp converged
                // the tile's largest |v|^2 (norms are >= 0, so their bits order like them)
                const float ncmax = __uint_as_float(__reduce_max_sync(
                    0xFFFFFFFFu,
                    __float_as_uint(fmaxf(fmaxf(rn[0], rn[1]), fmaxf(rn[2], rn[3])))));
                if (!__all_sync(0xFFFFFFFFu, ok)) {
                    ok = false;
                    break;
                }
                if (!skip_on && i + 2 < ntiles)
                    load_meta(i + 2);
                tc_fence_after();
                const int nvalid = a.N - cbase < BN ? (int)(a.N - cbase) : BN;
                const uint32_t tf = mattr[0], tl = mattr[nvalid - 1];
                const bool uni = tf == tl;  // one tuple in the whole tile (sorted order)
                const int ch_t = chi_level(chi_packed(au, tf, a.w.hi, a.w.lo));
                const int ch_min = (au >= tf && au <= tl) ? 0 : (uni ? ch_t : 1);
                for (int c0 = 0; c0 < BN; c0 += 32) {
                    // the bounds only tighten: a row whose bound for the smallest chi of
                    // this tile is negative rejects every column of it (negative bounds
                    // arise only under constant weights, where tiles are skipped)
                    const bool dead = !row_ok || (skip_on && lt[ch_min * BM] < 0.f);
                    if (__all_sync(0xFFFFFFFFu, dead))
                        break;
                    uint32_t v[32];
                    tmem_ld32(tmem + lane_base + (uint32_t)(b * BN + c0), v);
                    // branch-free filter: a pass mask of the columns within the bound of their
                    // chi (a dead row passes none and stays with the warp for its votes)
                    uint32_t pass = 0;
                    const float4 *cn4 = reinterpret_cast<const float4 *>(mnorm + c0);
                    if (dead) {
                    } else if (uni) {
                        // delta^2 = |u|^2 + |v|^2 - 2 u.v <= Lb tested as u.v >= |v|^2 / 2 + h,
                        // h = (|u|^2 - Lb) / 2 lowered by 2^-20 (|u|^2 + max |v|^2 + |Lb|):
                        // sixteen times the f32 rounding of either form, so every pair
                        // within the bound passes (a few more do, and fail the exact key
                        // test); two operations per pair instead of three
                        const float Lb = lt[ch_t * BM];
                        const float marg = 9.5367431640625e-07f * (nu + ncmax + fabsf(Lb));
                        const float h = 0.5f * (nu - Lb) - marg;
#pragma unroll
                        for (int j4 = 0; j4 < 8; ++j4) {
                            const float4 n4 = cn4[j4];
                            const float nc[4] = {n4.x, n4.y, n4.z, n4.w};
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int j = j4 * 4 + q;
                                const float dot = __uint_as_float(v[j]);
                                pass |= (dot >= fmaf(0.5f, nc[q], h) ? 1u : 0u) << j;
                            }
                        }
                    } else {
                        const uint4 *ca4 = reinterpret_cast<const uint4 *>(mattr + c0);
#pragma unroll
                        for (int j4 = 0; j4 < 8; ++j4) {
                            const float4 n4 = cn4[j4];
                            const uint4 at4 = ca4[j4];
                            const float nc[4] = {n4.x, n4.y, n4.z, n4.w};
                            const uint32_t ac[4] = {at4.x, at4.y, at4.z, at4.w};
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int j = j4 * 4 + q;
                                const float d2 =
                                    __fmaf_rn(-2.f, __uint_as_float(v[j]), __fadd_rn(nu, nc[q]));
                                const int ch = chi_level(chi_packed(au, ac[q], a.w.hi, a.w.lo));
                                pass |= (d2 <= lt[ch * BM] ? 1u : 0u) << j;
                            }
                        }
                    }
                    // the passing columns join this group's queue of the row (delta^2 picked
                    // from the registers by the column's index); every lane flushes together
                    // once some queue is half full, or full with columns of the chunk left
                    // (one call site, so the flush is compiled twice in all, not four times)
                    uint32_t pm = pass;
                    for (;;) {
                        for (; pm != 0u && qn < QCAP; pm &= pm - 1u) {
                            const int j = __ffs((int)pm) - 1;
                            const int c = c0 + j;
                            const int64_t col = cbase + c;
                            if (col >= a.N || col == u)
                                continue;
                            // the pair's delta^2 as the filters define it (unclamped there: a
                            // rounding below zero passes as it would at zero)
                            const float d2 = __fmaf_rn(-2.f, __uint_as_float(pick32(v, j)),
                                                       __fadd_rn(nu, mnorm[c]));
                            qk[qn * BM] =
                                ((unsigned long long)__float_as_uint(fmaxf(d2, 0.f)) << 32) | mid[c];
                            qc[qn * BM] = (unsigned char)chi_packed(au, mattr[c], a.w.hi, a.w.lo);
                            ++qn;
                        }
                        if (!__any_sync(0xFFFFFFFFu, qn >= QCAP / 2 || pm != 0u))
                            break;
                        flush();
                    }
                }
                tc_fence_before();
                mbar_arrive(bar(TEMPTY0 + b));
                // and every FLUSH_TILES tiles of the group, so that the bounds (and the
                // scheduler's skip decisions) follow the heaps; at the end, the rest
                if ((p % FLUSH_TILES) != 0)
                    continue;
            }
            if (__any_sync(0xFFFFFFFFu, qn > 0))
                flush();
            if (last)
                break;
        }
        // both groups have flushed (named barrier 1 over the eight epilogue warps); group
        // 0 writes the rows
        asm volatile("bar.sync 1, 256;" ::: "memory");
        const int cnt = *hcnt;
        if (g == 0 && row_ok) {
            // heap sort: pop the largest into the last open output slot of the
            // object's own (original) row
            const int64_t orow = (int64_t)a.perm[u] * K;
            if (cnt < K) {
                hp[cnt + 1] = 0ull;
                for (int h = cnt / 2; h >= 1; --h)
                    heap_sift(hp, cnt, h, hp[h]);
            }
            for (int j = K - 1; j >= 0; --j) {
                const int64_t o = orow + j;
                if (j >= cnt) {
                    a.ids[o] = kNone;
                    if (a.dists)
                        a.dists[o] = __int_as_float(0x7f800000);
                    continue;
                }
                const unsigned long long top = hp[1];
                a.ids[o] = (uint32_t)top;
                if (a.dists)
                    a.dists[o] = __uint_as_float((uint32_t)(top >> 32));
                const unsigned long long last = hp[j + 1];
                hp[j + 1] = 0ull;  // sentinel of the heap of size j
                if (j > 0)
                    heap_sift(hp, j, 1, last);
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

// bf16 rows padded to kpad (multiple of 64) and the squared norms of the rounded rows,
// row r taken from object perm[r]
__global__ void bf16_rows_norms_kernel(const float *__restrict__ X, int xstride, int d,
                                       int64_t N, int kpad, const uint32_t *__restrict__ perm,
                                       __nv_bfloat16 *__restrict__ Xk,
                                       float *__restrict__ norms) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= N)
        return;
    const int64_t src = perm[r];
    float acc = 0.f;
    for (int c = lane; c < kpad; c += 32) {
        const __nv_bfloat16 h = __float2bfloat16_rn(c < d ? X[src * xstride + c] : 0.f);
        Xk[r * kpad + c] = h;
        const float f = __bfloat162float(h);
        acc = fmaf(f, f, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0)
        norms[r] = acc;
}

size_t tc_smem_bytes(int ntiles) { return 1024 + tc_smem_layout(ntiles).total; }

}  // namespace

int knn_tc_kmax() { return KMAX; }

cudaError_t launch_knn_tc_prepare(const float *X, int xstride, int d, int64_t N, int kpad,
                                  const uint32_t *perm, __nv_bfloat16 *Xk, float *norms,
                                  cudaStream_t s) {
    const int wpb = 8;
    bf16_rows_norms_kernel<<<(unsigned)((N + wpb - 1) / wpb), 32 * wpb, 0, s>>>(
        X, xstride, d, N, kpad, perm, Xk, norms);
    return cudaGetLastError();
}

cudaError_t launch_knn_tc(const __nv_bfloat16 *Xk, int kpad, const float *norms,
                          const uint32_t *attr, const uint32_t *perm, int64_t N, const Fusion &w,
                          int K, uint32_t *ids, float *dists, int *err, cudaStream_t s) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (encode == nullptr) {
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion(
            "cuTensorMapEncodeTiled", reinterpret_cast<void **>(&encode), 12000,
            cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || encode == nullptr) {
            encode = nullptr;
            return e != cudaSuccess ? e : cudaErrorNotSupported;
        }
    }
    CUtensorMap tmap;
    const cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)kpad * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult cr = encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(Xk),
                         dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    TcArgs a;
    a.norms = norms;
    a.attr = attr;
    a.perm = perm;
    a.N = N;
    a.kblocks = kpad / BK;
    a.w = w;
    a.K = K;
    a.ids = ids;
    a.dists = dists;
    a.err = err;
    const int ntiles = (int)((N + BN - 1) / BN);
    const size_t smem = tc_smem_bytes(ntiles);
    int dev = 0, smax = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess)
        return e;
    if (smem > (size_t)smax)  // one skip bit per tile: N up to about 2.2e7
        return cudaErrorInvalidValue;
    void (*kfn)(const CUtensorMap, TcArgs) =
        w.mode == NHQ_W_CONSTANT   ? knn_tc_kernel<NHQ_W_CONSTANT>
        : w.mode == NHQ_W_HARMONIC ? knn_tc_kernel<NHQ_W_HARMONIC>
                                   : knn_tc_kernel<NHQ_W_PROPORTIONAL>;
    if (w.mode != NHQ_W_CONSTANT && w.mode != NHQ_W_HARMONIC && w.mode != NHQ_W_PROPORTIONAL)
        return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    kfn<<<(unsigned)ntiles, NTHREADS, smem, s>>>(tmap, a);
    return cudaGetLastError();
}

}  // namespace nhq
