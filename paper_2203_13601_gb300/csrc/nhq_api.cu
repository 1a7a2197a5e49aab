// nhq_api.cu -- the C ABI declared in include/nhq.h: argument checks, index
// ownership, host/device pointer handling, and the launches of the kernels in
// k_util.cu, k_bruteforce.cu, k_edge.cu and k_search.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "nhq_internal.cuh"

using namespace nhq;

namespace {

thread_local std::string g_err;

nhq_status fail(nhq_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

nhq_status fail_cuda(cudaError_t e, const char *what) {
    nhq_status s = e == cudaErrorMemoryAllocation ? NHQ_ERR_OOM : NHQ_ERR_CUDA;
    return fail(s, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail_cuda(e_, #call);                                                           \
    } while (0)

#define CKS(expr)                                                                                  \
    do {                                                                                           \
        nhq_status s_ = (expr);                                                                    \
        if (s_ != NHQ_OK)                                                                          \
            return s_;                                                                             \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

bool is_device_ptr(const void *p) {
    if (p == nullptr)
        return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

nhq_status grow(void **buf, size_t *cap, size_t need) {
    if (*cap >= need)
        return NHQ_OK;
    if (*buf) {
        CK(cudaDeviceSynchronize());
        CK(cudaFree(*buf));
        *buf = nullptr;
        *cap = 0;
    }
    size_t sz = need < 4096 ? 4096 : need;
    CK(cudaMalloc(buf, sz));
    *cap = sz;
    return NHQ_OK;
}

// Host pointers are copied through one device staging allocation per call.
struct Stager {
    struct Req {
        void *user;
        size_t bytes;
        bool input;
        bool host;
        size_t off;
    };
    std::vector<Req> reqs;
    void *base = nullptr;
    bool any_host = false;

    int add(const void *p, size_t bytes, bool input) {
        Req r{const_cast<void *>(p), bytes, input, p != nullptr && !is_device_ptr(p), 0};
        any_host = any_host || r.host;
        reqs.push_back(r);
        return (int)reqs.size() - 1;
    }
    nhq_status commit(void **arena, size_t *cap, cudaStream_t s) {
        size_t off = 0;
        for (auto &r : reqs)
            if (r.host) {
                r.off = off;
                off += (r.bytes + 255) & ~(size_t)255;
            }
        if (off == 0)
            return NHQ_OK;
        CKS(grow(arena, cap, off));
        base = *arena;
        for (auto &r : reqs)
            if (r.host && r.input && r.bytes)
                CK(cudaMemcpyAsync((char *)base + r.off, r.user, r.bytes, cudaMemcpyHostToDevice, s));
        return NHQ_OK;
    }
    void *dev(int i) const {
        const Req &r = reqs[i];
        if (r.user == nullptr)
            return nullptr;
        return r.host ? (char *)base + r.off : r.user;
    }
    nhq_status finish(cudaStream_t s) {
        if (!any_host)
            return NHQ_OK;
        for (auto &r : reqs)
            if (r.host && !r.input && r.bytes)
                CK(cudaMemcpyAsync(r.user, (char *)base + r.off, r.bytes, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        return NHQ_OK;
    }
};

nhq_status check_weights(const nhq_weights &w, bool allow_filter) {
    if (w.mode != NHQ_W_PROPORTIONAL && w.mode != NHQ_W_CONSTANT && w.mode != NHQ_W_HARMONIC &&
        !(allow_filter && w.mode == NHQ_W_FILTER))
        return fail(NHQ_ERR_ARG, "unknown weight mode %d", w.mode);
    // curve ii's adjusted chi (1, c, 2c, ...) must grow with chi: c = 0 (curve i) or c >= 1
    if (w.mode == NHQ_W_HARMONIC && !(std::isfinite(w.w_l) && (w.w_l == 0.f || w.w_l >= 1.f)))
        return fail(NHQ_ERR_ARG, "harmonic weights need w_l = 0 (curve i) or w_l >= 1 (curve ii)");
    if (w.mode == NHQ_W_CONSTANT &&
        (!std::isfinite(w.w_v) || !std::isfinite(w.w_l) || w.w_v < 0.f || w.w_l < 0.f))
        return fail(NHQ_ERR_ARG, "constant weights must be finite and >= 0");
    return NHQ_OK;
}

nhq_status scratch(nhq_index *ix, size_t need) { return grow(&ix->scratch, &ix->scratch_bytes, need); }

struct StageArena {
    void *p = nullptr;
    size_t cap = 0;
};
thread_local StageArena g_stage;  // host-pointer staging (per host thread)

nhq_status install_graph(nhq_index *ix, const uint32_t *nbr_dev, int R, cudaStream_t s) {
    const size_t bytes = sizeof(uint32_t) * (size_t)ix->N * R;
    if (ix->R != R || ix->nbr == nullptr) {
        if (ix->nbr)
            CK(cudaFree(ix->nbr));
        if (ix->nbr_attr)
            CK(cudaFree(ix->nbr_attr));
        ix->nbr = ix->nbr_attr = nullptr;
        CK(cudaMalloc(&ix->nbr, bytes));
        CK(cudaMalloc(&ix->nbr_attr, bytes));
    }
    if (nbr_dev != ix->nbr)
        CK(cudaMemcpyAsync(ix->nbr, nbr_dev, bytes, cudaMemcpyDeviceToDevice, s));
    CKS(scratch(ix, 256));
    int *bad = reinterpret_cast<int *>(ix->scratch);
    CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
    CK(launch_gather_nbr_attr(ix->nbr, ix->attr, ix->N, R, ix->nbr_attr, bad, s));
    int hbad = 0;
    CK(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ix->R = R;
    if (hbad)
        return fail(NHQ_ERR_ARG, "graph holds an id that is neither 0xFFFFFFFF nor < N");
    return NHQ_OK;
}

}  // namespace

namespace nhq {
// Lets other translation units of the library report an error through nhq_last_error.
nhq_status report_error(nhq_status s, const char *message) {
    g_err = message;
    return s;
}
// The weight rules of every entry point, for the entry points defined in other units.
nhq_status validate_weights(const nhq_weights &w, bool allow_filter) {
    return check_weights(w, allow_filter);
}
}  // namespace nhq

extern "C" {

const char *nhq_last_error(void) { return g_err.c_str(); }

int32_t nhq_version(void) { return 1; }

static nhq_status index_create_impl(const void *vectors, int dtype, int64_t N, int32_t d,
                                    const uint8_t *attributes, int32_t m, nhq_weights w,
                                    void *stream, nhq_index **out) {
    if (dtype != NHQ_F32 && dtype != NHQ_F16 && dtype != NHQ_BF16)
        return fail(NHQ_ERR_ARG, "dtype must be NHQ_F32, NHQ_F16 or NHQ_BF16 (got %d)", dtype);
    if (out == nullptr)
        return fail(NHQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (N < 1 || N > 0x7FFFFFFE)
        return fail(NHQ_ERR_ARG, "N must be in 1..2^31-2 (got %lld)", (long long)N);
    if (d < 1 || d > 16384)
        return fail(NHQ_ERR_ARG, "d must be in 1..16384 (got %d)", d);
    if (m < 1 || m > kMaxAttr)
        return fail(NHQ_ERR_ARG, "m must be in 1..%d (got %d)", kMaxAttr, m);
    if (vectors == nullptr || attributes == nullptr)
        return fail(NHQ_ERR_ARG, "vectors and attributes are required");
    CKS(check_weights(w, false));
    cudaStream_t s = as_stream(stream);
    nhq_index *ix = new nhq_index();
    ix->N = N;
    ix->d = d;
    ix->m = m;
    ix->xstride = (d + 15) & ~15;
    ix->w = w;
    auto bail = [&](nhq_status st) {
        nhq_free(ix);
        return st;
    };
    cudaError_t e;
    if ((e = cudaGetDevice(&ix->device)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaGetDevice"));
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, ix->device)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaGetDeviceProperties"));
    ix->sm_count = prop.multiProcessorCount;
    ix->smem_optin = prop.sharedMemPerBlockOptin;
    if ((e = cudaMalloc(&ix->X, sizeof(float) * (size_t)N * ix->xstride)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaMalloc(vectors)"));
    if ((e = cudaMalloc(&ix->attr, sizeof(uint32_t) * (size_t)N)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaMalloc(attributes)"));
    Stager st;
    const size_t esz = dtype == NHQ_F32 ? sizeof(float) : 2;
    int iv = st.add(vectors, esz * (size_t)N * d, true);
    int ia = st.add(attributes, (size_t)N * m, true);
    nhq_status rs = st.commit(&g_stage.p, &g_stage.cap, s);
    if (rs != NHQ_OK)
        return bail(rs);
    if ((rs = scratch(ix, 256)) != NHQ_OK)
        return bail(rs);
    int *bad = reinterpret_cast<int *>(ix->scratch);
    if ((e = cudaMemsetAsync(bad, 0, sizeof(int), s)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaMemsetAsync"));
    e = dtype == NHQ_F32
            ? launch_copy_rows((const float *)st.dev(iv), N, d, ix->xstride, ix->X, bad, s)
            : launch_copy_rows_typed(st.dev(iv), dtype, N, d, ix->xstride, ix->X, bad, s);
    if (e != cudaSuccess)
        return bail(fail_cuda(e, "copy_rows"));
    // an f16 / bf16 input is also the scoring copy of its type (the round trip is exact)
    if (dtype == NHQ_F16) {
        if ((e = cudaMalloc(&ix->Xf, sizeof(__half) * (size_t)N * ix->xstride)) != cudaSuccess ||
            (e = launch_rows_to_f16(ix->X, (int64_t)N * ix->xstride, ix->Xf, s)) != cudaSuccess)
            return bail(fail_cuda(e, "f16 copy"));
    } else if (dtype == NHQ_BF16) {
        if ((e = cudaMalloc(&ix->Xh, sizeof(__nv_bfloat16) * (size_t)N * ix->xstride)) !=
                cudaSuccess ||
            (e = launch_rows_to_bf16(ix->X, (int64_t)N * ix->xstride, ix->Xh, s)) != cudaSuccess)
            return bail(fail_cuda(e, "bf16 copy"));
    }
    // the largest code of each attribute: the field widths for m > 4, and the codes an
    // open query position ranges over
    unsigned int *amax = reinterpret_cast<unsigned int *>((char *)ix->scratch + 128);
    unsigned int hmax[kMaxAttr];
    if ((e = launch_attr_max((const uint8_t *)st.dev(ia), N, m, amax, s)) != cudaSuccess)
        return bail(fail_cuda(e, "attr_max"));
    if ((e = cudaMemcpyAsync(hmax, amax, sizeof(hmax), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return bail(fail_cuda(e, "attr_max copy"));
    uint8_t mc[kMaxAttr] = {};
    for (int j = 0; j < m; ++j)
        mc[j] = (uint8_t)hmax[j];
    if (m <= 4) {
        ix->layout = byte_layout(m);
        for (int j = 0; j < m; ++j)
            ix->layout.amax[j] = mc[j];
    } else {  // fields as narrow as the largest codes allow
        if (!compact_layout(m, mc, &ix->layout))
            return bail(fail(NHQ_ERR_ARG, "the codes of the %d attributes need more than 32 bits "
                                          "packed (each takes the bits of its largest code + 1)",
                             m));
    }
    if ((e = launch_pack_attributes((const uint8_t *)st.dev(ia), N, ix->layout, ix->attr, s)) !=
        cudaSuccess)
        return bail(fail_cuda(e, "pack_attributes"));
    int hbad = 0;
    if ((e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaMemcpyAsync"));
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess)
        return bail(fail_cuda(e, "cudaStreamSynchronize"));
    if (hbad)
        return bail(fail(NHQ_ERR_ARG, "vectors contain a non-finite component"));
    *out = ix;
    return NHQ_OK;
}

nhq_status nhq_index_create(const float *vectors, int64_t N, int32_t d, const uint8_t *attributes,
                            int32_t m, nhq_weights w, void *stream, nhq_index **out) {
    return index_create_impl(vectors, NHQ_F32, N, d, attributes, m, w, stream, out);
}

nhq_status nhq_index_create_typed(const void *vectors, int32_t dtype, int64_t N, int32_t d,
                                  const uint8_t *attributes, int32_t m, nhq_weights w,
                                  void *stream, nhq_index **out) {
    return index_create_impl(vectors, dtype, N, d, attributes, m, w, stream, out);
}

void nhq_free(nhq_index *ix) {
    if (ix == nullptr)
        return;
    cudaDeviceSynchronize();
    cudaFree(ix->X);
    cudaFree(ix->Xh);
    cudaFree(ix->X8);
    cudaFree(ix->Xf);
    cudaFree(ix->attr);
    cudaFree(ix->nbr);
    cudaFree(ix->nbr_attr);
    cudaFree(ix->Xk);
    cudaFree(ix->normk);
    cudaFree(ix->attr_sorted);
    cudaFree(ix->id_sorted);
    cudaFree(ix->cent);
    cudaFree(ix->centT);
    cudaFree(ix->cnh);
    cudaFree(ix->cell);
    cudaFree(ix->cell_key);
    cudaFree(ix->cell_id);
    cudaFree(ix->scratch);
    delete ix;
}

nhq_status nhq_index_info(const nhq_index *ix, int64_t *N, int32_t *d, int32_t *m, int32_t *R) {
    if (ix == nullptr)
        return fail(NHQ_ERR_ARG, "index is NULL");
    if (N)
        *N = ix->N;
    if (d)
        *d = ix->d;
    if (m)
        *m = ix->m;
    if (R)
        *R = ix->R;
    return NHQ_OK;
}

nhq_status nhq_pack_attributes(const uint8_t *attributes, int64_t n, int32_t m, uint32_t *packed,
                               void *stream) {
    if (n < 0 || m < 1 || m > 4)
        return fail(NHQ_ERR_ARG, "n must be >= 0 and m in 1..4");
    if (n == 0)
        return NHQ_OK;
    if (!is_device_ptr(attributes) || !is_device_ptr(packed))
        return fail(NHQ_ERR_ARG, "nhq_pack_attributes takes device pointers");
    CK(launch_pack_attributes(attributes, n, byte_layout(m), packed, as_stream(stream)));
    return NHQ_OK;
}

nhq_status nhq_knn(const nhq_index *cix, int32_t K, uint32_t *cand_ids, float *cand_dist,
                   void *stream) {
    nhq_index *ix = const_cast<nhq_index *>(cix);
    if (ix == nullptr || cand_ids == nullptr)
        return fail(NHQ_ERR_ARG, "index and cand_ids are required");
    if (K < 1 || K > kMaxK || K >= ix->N)
        return fail(NHQ_ERR_ARG, "K must be in 1..min(256, N-1) (got %d)", K);
    cudaStream_t s = as_stream(stream);
    Stager st;
    int io = st.add(cand_ids, sizeof(uint32_t) * (size_t)ix->N * K, false);
    int id = st.add(cand_dist, sizeof(float) * (size_t)ix->N * K, false);
    CKS(st.commit(&g_stage.p, &g_stage.cap, s));
    TopkArgs a;
    a.X = ix->X;
    a.xstride = ix->xstride;
    a.d = ix->d;
    a.N = ix->N;
    a.attr = ix->attr;
    a.Q = ix->X;
    a.qstride = ix->xstride;
    a.qattr = ix->attr;
    a.qhi = nullptr;
    a.nq = ix->N;
    a.k = K;
    a.exclude_self = 1;
    a.w = make_fusion(ix->w, ix->layout);
    a.ids = (uint32_t *)st.dev(io);
    a.dists = (float *)st.dev(id);
    a.chi = nullptr;
    size_t need = topk_scratch_bytes(a, ix->sm_count);
    CKS(scratch(ix, need + 256));
    CK(launch_topk(a, ix->scratch, ix->scratch_bytes, ix->sm_count, s));
    return st.finish(s);
}

// the packed attribute words sorted ascending with their ids (stable), built once
static nhq_status ensure_attribute_order(nhq_index *ix, cudaStream_t s) {
    if (ix->attr_sorted != nullptr)
        return NHQ_OK;
    CK(cudaMalloc(&ix->attr_sorted, sizeof(uint32_t) * (size_t)ix->N));
    CK(cudaMalloc(&ix->id_sorted, sizeof(uint32_t) * (size_t)ix->N));
    CKS(scratch(ix, attribute_sort_scratch_bytes(ix->N)));
    CK(launch_attribute_sort(ix->attr, ix->N, ix->attr_sorted, ix->id_sorted, ix->scratch,
                             ix->scratch_bytes, s));
    return NHQ_OK;
}

nhq_status nhq_knn_bf16(const nhq_index *cix, int32_t K, uint32_t *cand_ids, float *cand_dist,
                        void *stream) {
    nhq_index *ix = const_cast<nhq_index *>(cix);
    if (ix == nullptr || cand_ids == nullptr)
        return fail(NHQ_ERR_ARG, "index and cand_ids are required");
    if (K < 1 || K > knn_tc_kmax() || K >= ix->N)
        return fail(NHQ_ERR_ARG, "K must be in 1..min(64, N-1) (got %d)", K);
    cudaStream_t s = as_stream(stream);
    CKS(ensure_attribute_order(ix, s));
    if (ix->Xk == nullptr) {  // bf16 rows in attribute order
        ix->kpad = (ix->d + 63) & ~63;
        CK(cudaMalloc(&ix->Xk, sizeof(__nv_bfloat16) * (size_t)ix->N * ix->kpad));
        CK(cudaMalloc(&ix->normk, sizeof(float) * (size_t)ix->N));
        CK(launch_knn_tc_prepare(ix->X, ix->xstride, ix->d, ix->N, ix->kpad, ix->id_sorted,
                                 ix->Xk, ix->normk, s));
    }
    Stager st;
    int io = st.add(cand_ids, sizeof(uint32_t) * (size_t)ix->N * K, false);
    int id = st.add(cand_dist, sizeof(float) * (size_t)ix->N * K, false);
    CKS(st.commit(&g_stage.p, &g_stage.cap, s));
    CKS(scratch(ix, 256));
    int *err = reinterpret_cast<int *>(ix->scratch);
    CK(cudaMemsetAsync(err, 0, sizeof(int), s));
    cudaError_t e = launch_knn_tc(ix->Xk, ix->kpad, ix->normk, ix->attr_sorted, ix->id_sorted,
                                  ix->N, make_fusion(ix->w, ix->layout), K, (uint32_t *)st.dev(io),
                                  (float *)st.dev(id), err, s);
    if (e != cudaSuccess)
        return fail_cuda(e, "tensor-core candidate kernel launch");
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CKS(st.finish(s));
    CK(cudaStreamSynchronize(s));
    if (herr)
        return fail(NHQ_ERR_CUDA, "tensor-core candidate pipeline timed out (stage %d)", herr);
    return NHQ_OK;
}

nhq_status nhq_knn_nndescent(const nhq_index *ix, int32_t K, int32_t max_iters, uint64_t seed,
                             uint32_t *cand_ids, float *cand_dist, int32_t *iterations,
                             void *stream) {
    if (ix == nullptr || cand_ids == nullptr)
        return fail(NHQ_ERR_ARG, "index and cand_ids are required");
    if (K < 1 || K > nnd_kmax() || K >= ix->N)
        return fail(NHQ_ERR_ARG, "K must be in 1..min(64, N-1) (got %d)", K);
    if (max_iters < 1 || max_iters > 100)
        return fail(NHQ_ERR_ARG, "max_iters must be in 1..100 (got %d)", max_iters);
    cudaStream_t s = as_stream(stream);
    Stager st;
    int io = st.add(cand_ids, sizeof(uint32_t) * (size_t)ix->N * K, false);
    int id = st.add(cand_dist, sizeof(float) * (size_t)ix->N * K, false);
    CKS(st.commit(&g_stage.p, &g_stage.cap, s));
    void *work = nullptr;
    CK(cudaMalloc(&work, nnd_scratch_bytes(ix->N, K)));
    int done = 0;
    cudaError_t e = launch_nndescent(ix->X, ix->xstride, ix->N, ix->attr, make_fusion(ix->w, ix->layout),
                                     K, max_iters, 1e-3, seed, work, (uint32_t *)st.dev(io),
                                     (float *)st.dev(id), &done, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    cudaFree(work);
    if (e != cudaSuccess)
        return fail_cuda(e, "NN-descent");
    if (iterations)
        *iterations = done;
    return st.finish(s);
}

nhq_status nhq_edge_select(const nhq_index *cix, const uint32_t *cand_ids, int32_t L, int32_t R,
                           uint32_t *nbr_out, void *stream) {
    const nhq_index *ix = cix;
    if (ix == nullptr || cand_ids == nullptr || nbr_out == nullptr)
        return fail(NHQ_ERR_ARG, "index, cand_ids and nbr_out are required");
    if (L < 1 || L > kMaxCand)
        return fail(NHQ_ERR_ARG, "L must be in 1..128 (got %d)", L);
    if (R < 1 || R > kMaxDegree)
        return fail(NHQ_ERR_ARG, "R must be in 1..64 (got %d)", R);
    cudaStream_t s = as_stream(stream);
    Stager st;
    int ic = st.add(cand_ids, sizeof(uint32_t) * (size_t)ix->N * L, true);
    int io = st.add(nbr_out, sizeof(uint32_t) * (size_t)ix->N * R, false);
    CKS(st.commit(&g_stage.p, &g_stage.cap, s));
    CK(launch_edge_select(ix, (const uint32_t *)st.dev(ic), L, R, (uint32_t *)st.dev(io), s));
    return st.finish(s);
}

nhq_status nhq_reverse_candidates(const nhq_index *cix, const uint32_t *nbr, int32_t R, int32_t cap,
                                  uint32_t *out, void *stream) {
    nhq_index *ix = const_cast<nhq_index *>(cix);
    if (ix == nullptr || nbr == nullptr || out == nullptr)
        return fail(NHQ_ERR_ARG, "index, nbr and out are required");
    if (R < 1 || R > kMaxDegree || cap < 0 || cap > kMaxDegree)
        return fail(NHQ_ERR_ARG, "R must be in 1..64 and cap in 0..64");
    cudaStream_t s = as_stream(stream);
    Stager st;
    int in = st.add(nbr, sizeof(uint32_t) * (size_t)ix->N * R, true);
    int io = st.add(out, sizeof(uint32_t) * (size_t)ix->N * (R + cap), false);
    CKS(st.commit(&g_stage.p, &g_stage.cap, s));
    CKS(scratch(ix, reverse_scratch_bytes(ix->N, R)));
    CK(launch_reverse_candidates((const uint32_t *)st.dev(in), ix->N, R, cap,
                                 (uint32_t *)st.dev(io), ix->scratch, s));
    return st.finish(s);
}

nhq_status nhq_index_set_graph(nhq_index *ix, const uint32_t *nbr, int32_t R, void *stream) {
    if (ix == nullptr || nbr == nullptr)
        return fail(NHQ_ERR_ARG, "index and nbr are required");
    if (R < 1 || R > kMaxDegree)
        return fail(NHQ_ERR_ARG, "R must be in 1..64 (got %d)", R);
    cudaStream_t s = as_stream(stream);
    Stager st;
    int in = st.add(nbr, sizeof(uint32_t) * (size_t)ix->N * R, true);
    CKS(st.commit(&g_stage.p, &g_stage.cap, s));
    return install_graph(ix, (const uint32_t *)st.dev(in), R, s);
}

nhq_status nhq_index_get_graph(const nhq_index *ix, uint32_t *nbr, void *stream) {
    if (ix == nullptr || nbr == nullptr)
        return fail(NHQ_ERR_ARG, "index and nbr are required");
    if (ix->nbr == nullptr)
        return fail(NHQ_ERR_ARG, "the index has no graph");
    cudaStream_t s = as_stream(stream);
    Stager st;
    int io = st.add(nbr, sizeof(uint32_t) * (size_t)ix->N * ix->R, false);
    CKS(st.commit(&g_stage.p, &g_stage.cap, s));
    CK(cudaMemcpyAsync(st.dev(io), ix->nbr, sizeof(uint32_t) * (size_t)ix->N * ix->R,
                       cudaMemcpyDeviceToDevice, s));
    return st.finish(s);
}

nhq_status nhq_index_build(nhq_index *ix, int32_t degree, const nhq_build_params *p,
                           void *stream) {
    if (ix == nullptr)
        return fail(NHQ_ERR_ARG, "index is NULL");
    if (degree < 1 || degree > kMaxDegree)
        return fail(NHQ_ERR_ARG, "degree must be in 1..64 (got %d)", degree);
    if (ix->N < 2)
        return fail(NHQ_ERR_ARG, "a graph needs N >= 2");
    int K = p && p->K > 0 ? p->K : 64;
    int rev = p ? p->reverse : 1;
    int cap = p && p->reverse_cap > 0 ? p->reverse_cap : 64;
    if (K > kMaxCand)
        return fail(NHQ_ERR_ARG, "K must be in 1..128 for the build (got %d)", K);
    if (cap > kMaxDegree)
        return fail(NHQ_ERR_ARG, "reverse_cap must be in 1..64");
    if (K >= ix->N)
        K = (int)(ix->N - 1);
    if (rev && degree + cap > kMaxCand)
        cap = kMaxCand - degree;
    cudaStream_t s = as_stream(stream);
    uint32_t *cand = nullptr, *nbr = nullptr, *rc = nullptr;
    const size_t N = (size_t)ix->N;
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);
        cudaFree(cand);
        cudaFree(nbr);
        cudaFree(rc);
    };
    cudaError_t e;
    if ((e = cudaMalloc(&cand, sizeof(uint32_t) * N * K)) != cudaSuccess ||
        (e = cudaMalloc(&nbr, sizeof(uint32_t) * N * degree)) != cudaSuccess) {
        cleanup();
        return fail_cuda(e, "cudaMalloc(build buffers)");
    }
    const int tc = p ? p->knn_dtype : 0;
    if (tc < 0 || tc > 2)
        return fail(NHQ_ERR_ARG,
                    "knn_dtype must be 0 (f32), 1 (bf16 tensor cores) or 2 (NN-descent)");
    if (tc == 1 && K > knn_tc_kmax())
        K = knn_tc_kmax();
    if (tc == 2 && K > nnd_kmax())
        K = nnd_kmax();
    nhq_status st = tc == 1   ? nhq_knn_bf16(ix, K, cand, nullptr, stream)
                    : tc == 2 ? nhq_knn_nndescent(ix, K, 12, 0x2203ull, cand, nullptr, nullptr,
                                                  stream)
                              : nhq_knn(ix, K, cand, nullptr, stream);
    if (st == NHQ_OK)
        st = nhq_edge_select(ix, cand, K, degree, nbr, stream);
    if (st == NHQ_OK && rev) {
        if ((e = cudaMalloc(&rc, sizeof(uint32_t) * N * (degree + cap))) != cudaSuccess) {
            cleanup();
            return fail_cuda(e, "cudaMalloc(reverse candidates)");
        }
        st = nhq_reverse_candidates(ix, nbr, degree, cap, rc, stream);
        if (st == NHQ_OK)
            st = nhq_edge_select(ix, rc, degree + cap, degree, nbr, stream);
    }
    if (st == NHQ_OK)
        st = install_graph(ix, nbr, degree, s);
    cleanup();
    return st;
}

nhq_status nhq_index_build_nsw(nhq_index *ix, int32_t degree, int32_t L, int32_t wave_max,
                               int32_t rev_cap, int32_t entry, uint64_t seed, void *stream) {
    if (ix == nullptr)
        return fail(NHQ_ERR_ARG, "index is NULL");
    if (degree < 1 || degree > kMaxDegree)
        return fail(NHQ_ERR_ARG, "degree must be in 1..64 (got %d)", degree);
    if (L < degree || L > kMaxCand)
        return fail(NHQ_ERR_ARG, "L must be in degree..128 (got %d)", L);
    if (rev_cap < 0 || degree + rev_cap > kMaxCand)
        return fail(NHQ_ERR_ARG, "degree + rev_cap must be at most 128");
    if (wave_max < 1 || wave_max > 65536)
        return fail(NHQ_ERR_ARG, "wave_max must be in 1..65536 (got %d)", wave_max);
    if (entry != 0 && entry != 1)
        return fail(NHQ_ERR_ARG, "entry must be 0 (by id) or 1 (by attributes)");
    cudaStream_t s = as_stream(stream);
    if (entry == 1)
        CKS(ensure_attribute_order(ix, s));
    const int64_t N = ix->N, R = degree;
    const int64_t Bmax = std::min<int64_t>(wave_max, std::max<int64_t>(N - 1, 1));
    const int W = R + rev_cap;
    const int ns = nsw_seed_count();
    // the empty graph, then the wave buffers
    uint32_t *empty = nullptr;
    CK(cudaMalloc(&empty, sizeof(uint32_t) * (size_t)N * R));
    CK(cudaMemsetAsync(empty, 0xFF, sizeof(uint32_t) * (size_t)N * R, s));
    nhq_status st = install_graph(ix, empty, (int)R, s);
    cudaFree(empty);
    if (st != NHQ_OK)
        return st;
    const int64_t np = Bmax * R;
    const size_t sort_bytes = nsw_sort_scratch_bytes(np);
    std::vector<void *> bufs;
    auto get = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes < 256 ? 256 : bytes) != cudaSuccess)
            return nullptr;
        bufs.push_back(p);
        return p;
    };
    auto release = [&]() {
        cudaStreamSynchronize(s);
        for (void *p : bufs)
            cudaFree(p);
    };
    float *q = (float *)get(sizeof(float) * Bmax * ix->d);
    uint8_t *qa = (uint8_t *)get((size_t)Bmax * ix->m);
    uint32_t *seeds = (uint32_t *)get(sizeof(uint32_t) * Bmax * ns);
    uint32_t *cand = (uint32_t *)get(sizeof(uint32_t) * Bmax * L);
    uint32_t *rows = (uint32_t *)get(sizeof(uint32_t) * Bmax * R);
    unsigned long long *keys = (unsigned long long *)get(8 * np);
    unsigned long long *sorted = (unsigned long long *)get(8 * np);
    void *tmp = get(sort_bytes);
    uint32_t *seg = (uint32_t *)get(sizeof(uint32_t) * np);
    int *nseg_dev = (int *)get(sizeof(int));
    uint32_t *U = (uint32_t *)get(sizeof(uint32_t) * np);
    uint32_t *candU = (uint32_t *)get(sizeof(uint32_t) * np * W);
    uint32_t *upd = (uint32_t *)get(sizeof(uint32_t) * np * R);
    for (void *p : bufs)
        if (p == nullptr) {
            release();
            return fail(NHQ_ERR_OOM, "cudaMalloc(incremental build buffers)");
        }
    if (bufs.size() != 13) {
        release();
        return fail(NHQ_ERR_OOM, "cudaMalloc(incremental build buffers)");
    }
    nhq_search_params P{};
    P.h = 1;
    P.seed_mode = NHQ_SEED_GIVEN;
    P.n_seeds = ns;
    P.seeds = seeds;
    cudaError_t e = cudaSuccess;
    for (int64_t s0 = 1; s0 < N && st == NHQ_OK && e == cudaSuccess;) {
        const int64_t B = std::min<int64_t>(std::min<int64_t>(s0, wave_max), N - s0);
        if ((e = entry == 1 ? launch_nsw_attr_seeds(ix, s0, B, seed, seeds, s)
                            : launch_nsw_seeds(s0, B, seed, seeds, s)) != cudaSuccess ||
            (e = launch_nsw_queries(ix, s0, B, q, qa, s)) != cudaSuccess)
            break;
        st = nhq_search(ix, q, qa, B, L, L, &P, cand, nullptr, nullptr, nullptr, nullptr, nullptr,
                        stream);
        if (st != NHQ_OK)
            break;
        if ((e = launch_edge_select_rows(ix, cand, L, (int)R, nullptr, s0, B, rows, s)) !=
                cudaSuccess ||
            (e = launch_nsw_pairs(rows, (int)R, s0, B, keys, sorted, tmp, sort_bytes, seg,
                                  nseg_dev, s)) != cudaSuccess)
            break;
        int nseg = 0;
        if ((e = cudaMemcpyAsync(&nseg, nseg_dev, sizeof(int), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            break;
        if (nseg > 0 &&
            ((e = launch_nsw_reverse(sorted, B * R, seg, nseg, ix->nbr, (int)R, rev_cap, U,
                                     candU, s)) != cudaSuccess ||
             (e = launch_edge_select_rows(ix, candU, W, (int)R, U, 0, nseg, upd, s)) !=
                 cudaSuccess))
            break;
        // both selections read the graph as the wave began; now write the rows
        if ((e = launch_nsw_install(rows, nullptr, s0, B, (int)R, ix->attr, ix->nbr,
                                    ix->nbr_attr, s)) != cudaSuccess ||
            (e = launch_nsw_install(upd, U, 0, nseg, (int)R, ix->attr, ix->nbr, ix->nbr_attr,
                                    s)) != cudaSuccess)
            break;
        s0 += B;
    }
    release();
    if (st != NHQ_OK)
        return st;
    if (e != cudaSuccess)
        return fail_cuda(e, "incremental build");
    return NHQ_OK;
}

nhq_status nhq_index_build_cells(nhq_index *ix, int32_t E, void *stream) {
    if (ix == nullptr)
        return fail(NHQ_ERR_ARG, "index is NULL");
    if (E < 1 || (int64_t)E > ix->N || E > 65535)
        return fail(NHQ_ERR_ARG, "E must be in 1..min(N, 65535) (got %d)", E);
    cudaStream_t s = as_stream(stream);
    CK(cudaStreamSynchronize(s));
    cudaFree(ix->cent);
    cudaFree(ix->centT);
    cudaFree(ix->cnh);
    cudaFree(ix->cell);
    cudaFree(ix->cell_key);
    cudaFree(ix->cell_id);
    ix->cent = ix->centT = ix->cnh = nullptr;
    ix->cell = ix->cell_id = nullptr;
    ix->cell_key = nullptr;
    ix->E = 0;
    CK(cudaMalloc(&ix->cent, sizeof(float) * (size_t)E * ix->xstride));
    CK(cudaMalloc(&ix->centT, sizeof(float) * (size_t)E * ix->d));
    CK(cudaMalloc(&ix->cnh, sizeof(float) * (size_t)E));
    CK(cudaMalloc(&ix->cell, sizeof(uint32_t) * (size_t)ix->N));
    CK(cudaMalloc(&ix->cell_key, sizeof(unsigned long long) * (size_t)ix->N));
    CK(cudaMalloc(&ix->cell_id, sizeof(uint32_t) * (size_t)ix->N));
    CKS(ensure_attribute_order(ix, s));
    // the centroid rows and their attribute words, then every object's nearest centroid
    // (Gamma = 1 * delta + 0 * chi: plain L2, ties to the smaller centroid index)
    TopkArgs a;
    a.X = ix->cent;
    a.xstride = ix->xstride;
    a.d = ix->d;
    a.N = E;
    a.Q = ix->X;
    a.qstride = ix->xstride;
    a.qattr = ix->attr;
    a.qhi = nullptr;
    a.nq = ix->N;
    a.k = 1;
    a.exclude_self = 0;
    nhq_weights l2{NHQ_W_CONSTANT, 1.f, 0.f};
    a.w = make_fusion(l2, ix->layout);
    a.ids = ix->cell;
    a.dists = nullptr;
    a.chi = nullptr;
    const size_t cattr_bytes = ((sizeof(uint32_t) * (size_t)E) + 255) & ~(size_t)255;
    CKS(scratch(ix, cattr_bytes + topk_scratch_bytes(a, ix->sm_count)));
    uint32_t *cattr = reinterpret_cast<uint32_t *>(ix->scratch);
    a.attr = cattr;
    CK(launch_gather_centroids(ix->X, ix->xstride, ix->N, E, ix->attr, ix->cent, cattr, s));
    CK(launch_centroid_columns(ix->cent, ix->xstride, ix->d, E, ix->centT, ix->cnh, s));
    CK(launch_topk(a, (char *)ix->scratch + cattr_bytes, ix->scratch_bytes - cattr_bytes,
                   ix->sm_count, s));
    CKS(scratch(ix, cell_sort_scratch_bytes(ix->N)));
    CK(launch_cell_sort(ix->attr, ix->cell, ix->N, ix->cell_key, ix->cell_id, ix->scratch,
                        ix->scratch_bytes, s));
    ix->E = E;
    return NHQ_OK;
}

nhq_status nhq_index_cells(const nhq_index *ix, int32_t *E, uint32_t *cell_of, void *stream) {
    if (ix == nullptr)
        return fail(NHQ_ERR_ARG, "index is NULL");
    if (E)
        *E = ix->E;
    if (cell_of != nullptr) {
        if (ix->E == 0)
            return fail(NHQ_ERR_ARG, "the index has no entry cells (nhq_index_build_cells)");
        cudaStream_t s = as_stream(stream);
        CK(cudaMemcpyAsync(cell_of, ix->cell, sizeof(uint32_t) * (size_t)ix->N, cudaMemcpyDefault,
                           s));
        CK(cudaStreamSynchronize(s));
    }
    return NHQ_OK;
}

int64_t nhq_entry_param_count(int32_t d, int32_t E) {
    if (d < 1 || E < 1)
        return 0;
    return entry_param_count(d, E);
}

static nhq_status check_entry(const float *params, int32_t d, int32_t E, const float *queries,
                              int64_t n) {
    if (d < 1 || d > 16384 || E < 1 || E > 65535 || n < 0)
        return fail(NHQ_ERR_ARG, "need d in 1..16384, E in 1..65535, n >= 0");
    if (!is_device_ptr(params) || (n > 0 && !is_device_ptr(queries)))
        return fail(NHQ_ERR_ARG, "the entry-model calls take device pointers");
    return NHQ_OK;
}

nhq_status nhq_entry_forward(const float *params, int32_t d, int32_t E, const float *queries,
                             int64_t n, float *logits, void *stream) {
    CKS(check_entry(params, d, E, queries, n));
    if (n > 0 && !is_device_ptr(logits))
        return fail(NHQ_ERR_ARG, "logits must be device memory");
    cudaStream_t s = as_stream(stream);
    const int64_t np = entry_param_count(d, E);
    __half *w16 = nullptr;
    float *hidden = nullptr;
    CK(cudaMallocAsync(&w16, sizeof(__half) * (size_t)np, s));
    cudaError_t e = cudaMallocAsync(&hidden, sizeof(float) * NHQ_ENTRY_HIDDEN * (size_t)(n + 1), s);
    if (e == cudaSuccess)
        e = launch_entry_to_half(params, np, w16, s);
    if (e == cudaSuccess)
        e = launch_entry_scores_learned(w16, params, d, E, queries, d, n, hidden, logits, s);
    if (hidden)
        cudaFreeAsync(hidden, s);
    cudaFreeAsync(w16, s);
    if (e != cudaSuccess)
        return fail_cuda(e, "nhq_entry_forward");
    return NHQ_OK;
}

nhq_status nhq_entry_grad(const float *params, int32_t d, int32_t E, const float *queries,
                          const int32_t *labels, int64_t n, float *grad, float *loss,
                          void *stream) {
    CKS(check_entry(params, d, E, queries, n));
    if (!is_device_ptr(grad) || !is_device_ptr(loss) || (n > 0 && !is_device_ptr(labels)))
        return fail(NHQ_ERR_ARG, "the entry-model calls take device pointers");
    cudaStream_t s = as_stream(stream);
    const int64_t np = entry_param_count(d, E);
    CK(cudaMemsetAsync(grad, 0, sizeof(float) * (size_t)np, s));
    CK(cudaMemsetAsync(loss, 0, sizeof(float), s));
    if (n == 0)
        return NHQ_OK;
    const int B = 2048;
    void *work = nullptr;
    CK(cudaMallocAsync(&work, entry_train_chunk_bytes(B, E), s));
    cudaError_t e = entry_grad_accumulate(params, d, E, queries, labels, n, n, B, grad, loss,
                                          work, s);
    cudaFreeAsync(work, s);
    if (e != cudaSuccess)
        return fail_cuda(e, "nhq_entry_grad");
    return NHQ_OK;
}

nhq_status nhq_entry_train(float *params, int32_t d, int32_t E, const float *queries,
                           const int32_t *labels, int64_t n, int32_t epochs, int32_t batch,
                           float lr, void *stream) {
    CKS(check_entry(params, d, E, queries, n));
    if (batch < 1 || batch > 65536 || epochs < 0)
        return fail(NHQ_ERR_ARG, "batch must be in 1..65536 and epochs >= 0");
    if (n > 0 && !is_device_ptr(labels))
        return fail(NHQ_ERR_ARG, "the entry-model calls take device pointers");
    if (n == 0 || epochs == 0)
        return NHQ_OK;
    cudaStream_t s = as_stream(stream);
    const int64_t np = entry_param_count(d, E);
    const int B = batch < 2048 ? batch : 2048;  // chunk of one gradient pass
    float *buf = nullptr;  // gradient, first and second moments, loss
    void *work = nullptr;
    CK(cudaMallocAsync(&buf, sizeof(float) * (size_t)(3 * np + 1), s));
    cudaError_t e = cudaMallocAsync(&work, entry_train_chunk_bytes(B, E), s);
    float *g = buf, *m = buf + np, *v = m + np, *loss = v + np;
    if (e == cudaSuccess)
        e = cudaMemsetAsync(m, 0, sizeof(float) * (size_t)(2 * np), s);
    int t = 0;
    for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
        for (int64_t b = 0; b < n && e == cudaSuccess; b += batch) {
            const int64_t nb = n - b < batch ? n - b : batch;
            e = cudaMemsetAsync(g, 0, sizeof(float) * (size_t)(np + 1), s);
            if (e == cudaSuccess)
                e = entry_grad_accumulate(params, d, E, queries + b * d, labels + b, nb, nb, B,
                                          g, loss, work, s);
            ++t;
            const float c1 = 1.f / (1.f - powf(0.9f, (float)t));
            const float c2 = 1.f / (1.f - powf(0.999f, (float)t));
            if (e == cudaSuccess)
                e = launch_entry_adam(params, g, m, v, np, lr, c1, c2, s);
        }
    }
    if (work)
        cudaFreeAsync(work, s);
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess)
        return fail_cuda(e, "nhq_entry_train");
    return NHQ_OK;
}

nhq_status nhq_entry_labels(const nhq_index *ix, const uint32_t *ids, int32_t k, int64_t n,
                            int32_t *labels, void *stream) {
    if (ix == nullptr || ix->E == 0)
        return fail(NHQ_ERR_ARG, "the index has no entry cells (nhq_index_build_cells)");
    if (k < 1 || n < 0)
        return fail(NHQ_ERR_ARG, "need k >= 1, n >= 0");
    if (n > 0 && (!is_device_ptr(ids) || !is_device_ptr(labels)))
        return fail(NHQ_ERR_ARG, "nhq_entry_labels takes device pointers");
    CK(launch_entry_labels(ids, k, n, ix->cell, ix->N, labels, as_stream(stream)));
    return NHQ_OK;
}

nhq_status nhq_build(const float *vectors, int64_t N, int32_t d, const uint8_t *attributes,
                     int32_t m, int32_t degree, nhq_weights w, const nhq_build_params *params,
                     void *stream, nhq_index **out) {
    return nhq_build_typed(vectors, NHQ_F32, N, d, attributes, m, degree, w, params, stream, out);
}

nhq_status nhq_build_typed(const void *vectors, int32_t dtype, int64_t N, int32_t d,
                           const uint8_t *attributes, int32_t m, int32_t degree, nhq_weights w,
                           const nhq_build_params *params, void *stream, nhq_index **out) {
    if (out == nullptr)
        return fail(NHQ_ERR_ARG, "out is NULL");
    nhq_index *ix = nullptr;
    CKS(nhq_index_create_typed(vectors, dtype, N, d, attributes, m, w, stream, &ix));
    nhq_status st = nhq_index_build(ix, degree, params, stream);
    if (st != NHQ_OK) {
        std::string keep = g_err;
        nhq_free(ix);
        g_err = keep;
        *out = nullptr;
        return st;
    }
    *out = ix;
    return NHQ_OK;
}

nhq_status nhq_brute_force(const nhq_index *cix, const float *queries,
                           const uint8_t *query_attributes, int64_t Q, int32_t k,
                           const nhq_weights *w, uint32_t *ids, float *dists, uint8_t *chi,
                           void *stream) {
    return nhq_brute_force_wildcard(cix, queries, query_attributes, Q, k, w, 0, ids, dists, chi,
                                    stream);
}

nhq_status nhq_brute_force_wildcard(const nhq_index *cix, const float *queries,
                                    const uint8_t *query_attributes, int64_t Q, int32_t k,
                                    const nhq_weights *w, int32_t wildcard, uint32_t *ids,
                                    float *dists, uint8_t *chi, void *stream) {
    nhq_index *ix = const_cast<nhq_index *>(cix);
    if (wildcard != 0 && wildcard != 1)
        return fail(NHQ_ERR_ARG, "wildcard must be 0 or 1 (got %d)", wildcard);
    if (ix == nullptr)
        return fail(NHQ_ERR_ARG, "index is NULL");
    if (Q < 0)
        return fail(NHQ_ERR_ARG, "Q must be >= 0");
    if (k < 1 || k > kMaxK)
        return fail(NHQ_ERR_ARG, "k must be in 1..256 (got %d)", k);
    if (Q == 0)
        return NHQ_OK;
    if (queries == nullptr || query_attributes == nullptr || ids == nullptr)
        return fail(NHQ_ERR_ARG, "queries, query_attributes and ids are required");
    nhq_weights ww = w ? *w : ix->w;
    CKS(check_weights(ww, true));
    cudaStream_t s = as_stream(stream);
    Stager st;
    int iq = st.add(queries, sizeof(float) * (size_t)Q * ix->d, true);
    int ia = st.add(query_attributes, (size_t)Q * ix->m, true);
    int io = st.add(ids, sizeof(uint32_t) * (size_t)Q * k, false);
    int id = st.add(dists, sizeof(float) * (size_t)Q * k, false);
    int ic = st.add(chi, (size_t)Q * k, false);
    CKS(st.commit(&g_stage.p, &g_stage.cap, s));
    TopkArgs a;
    a.X = ix->X;
    a.xstride = ix->xstride;
    a.d = ix->d;
    a.N = ix->N;
    a.attr = ix->attr;
    a.Q = (const float *)st.dev(iq);
    a.qstride = ix->d;
    a.nq = Q;
    a.k = k;
    a.exclude_self = 0;
    a.w = make_fusion(ww, ix->layout);
    a.w.wild = wildcard;
    a.ids = (uint32_t *)st.dev(io);
    a.dists = (float *)st.dev(id);
    a.chi = (uint8_t *)st.dev(ic);
    // query words, then (with a wildcard) their chi masks
    size_t qa_bytes = ((sizeof(uint32_t) * (size_t)Q) + 255) & ~(size_t)255;
    const size_t words = wildcard ? 2 * qa_bytes : qa_bytes;
    size_t need = words + topk_scratch_bytes(a, ix->sm_count);
    CKS(scratch(ix, need));
    uint32_t *qa = reinterpret_cast<uint32_t *>(ix->scratch);
    uint32_t *qh = wildcard ? reinterpret_cast<uint32_t *>((char *)ix->scratch + qa_bytes) : nullptr;
    CK(launch_pack_queries((const uint8_t *)st.dev(ia), Q, a.w, qa, qh, s));
    a.qattr = qa;
    a.qhi = qh;
    qa_bytes = words;
    CK(launch_topk(a, (char *)ix->scratch + qa_bytes, ix->scratch_bytes - qa_bytes, ix->sm_count,
                   s));
    return st.finish(s);
}

nhq_status nhq_postfilter(int64_t Q, int32_t k_in, int32_t k_out, const uint32_t *ids,
                          const float *dists, const uint8_t *chi, uint32_t *out_ids,
                          float *out_dists, void *stream) {
    if (k_in < 1 || k_in > 1024 || k_out < 1 || k_out > 1024)
        return fail(NHQ_ERR_ARG, "k_in and k_out must be in 1..1024");
    if (Q < 0)
        return fail(NHQ_ERR_ARG, "Q must be >= 0");
    if (Q == 0)
        return NHQ_OK;
    if (ids == nullptr || dists == nullptr || chi == nullptr || out_ids == nullptr ||
        out_dists == nullptr)
        return fail(NHQ_ERR_ARG, "ids, dists, chi, out_ids and out_dists are required");
    cudaStream_t s = as_stream(stream);
    const size_t in_n = (size_t)Q * k_in, out_n = (size_t)Q * k_out;
    Stager st;
    int ii = st.add(ids, sizeof(uint32_t) * in_n, true);
    int idd = st.add(dists, sizeof(float) * in_n, true);
    int ic = st.add(chi, in_n, true);
    int oi = st.add(out_ids, sizeof(uint32_t) * out_n, false);
    int od = st.add(out_dists, sizeof(float) * out_n, false);
    CKS(st.commit(&g_stage.p, &g_stage.cap, s));
    CK(launch_postfilter(Q, k_in, k_out, (const uint32_t *)st.dev(ii), (const float *)st.dev(idd),
                         (const uint8_t *)st.dev(ic), (uint32_t *)st.dev(oi),
                         (float *)st.dev(od), s));
    return st.finish(s);
}

nhq_status nhq_merge_topk(int32_t P, int64_t Q, int32_t k_in, int32_t k_out,
                          const uint32_t *ids, const float *dists, const uint8_t *chi,
                          const uint32_t *offsets, uint32_t *out_ids, float *out_dists,
                          uint8_t *out_chi, void *stream) {
    if (P < 1 || P > 4096)
        return fail(NHQ_ERR_ARG, "P must be in 1..4096 (got %d)", P);
    if (k_in < 1 || k_in > 1024 || k_out < 1 || k_out > 1024)
        return fail(NHQ_ERR_ARG, "k_in and k_out must be in 1..1024");
    if (Q < 0)
        return fail(NHQ_ERR_ARG, "Q must be >= 0");
    if (Q == 0)
        return NHQ_OK;
    if (ids == nullptr || dists == nullptr || offsets == nullptr || out_ids == nullptr ||
        out_dists == nullptr)
        return fail(NHQ_ERR_ARG, "ids, dists, offsets, out_ids and out_dists are required");
    if (out_chi != nullptr && chi == nullptr)
        return fail(NHQ_ERR_ARG, "out_chi needs the shards' chi");
    cudaStream_t s = as_stream(stream);
    const size_t in_n = (size_t)P * (size_t)Q * (size_t)k_in, out_n = (size_t)Q * (size_t)k_out;
    Stager st;
    int ii = st.add(ids, sizeof(uint32_t) * in_n, true);
    int idd = st.add(dists, sizeof(float) * in_n, true);
    int ic = st.add(out_chi ? chi : nullptr, in_n, true);
    int io = st.add(offsets, sizeof(uint32_t) * (size_t)P, true);
    int oi = st.add(out_ids, sizeof(uint32_t) * out_n, false);
    int od = st.add(out_dists, sizeof(float) * out_n, false);
    int oc = st.add(out_chi, out_n, false);
    CKS(st.commit(&g_stage.p, &g_stage.cap, s));
    CK(launch_merge_topk(P, Q, k_in, k_out, (const uint32_t *)st.dev(ii),
                         (const float *)st.dev(idd), (const uint8_t *)st.dev(ic),
                         (const uint32_t *)st.dev(io), (uint32_t *)st.dev(oi),
                         (float *)st.dev(od), (uint8_t *)st.dev(oc), s));
    return st.finish(s);
}

struct TraceOut {
    float *features = nullptr;
    uint8_t *labels = nullptr;
    int32_t *query = nullptr;
    int64_t cap = 0;
    int64_t *n_traces = nullptr;
};

static nhq_status search_common(const nhq_index *cix, const float *queries,
                                const uint8_t *query_attributes, int64_t Q, const int32_t *k_arr,
                                const int32_t *ef_arr, int32_t k, int32_t ef, int32_t k_out,
                                const nhq_search_params *p, uint32_t *ids, float *dists,
                                uint8_t *chi, int32_t *status, int32_t *ndc, int32_t *expansions,
                                void *stream, const TraceOut *trace = nullptr) {
    nhq_index *ix = const_cast<nhq_index *>(cix);
    cudaStream_t s = as_stream(stream);
    nhq_search_params P{};
    if (p)
        P = *p;
    if (P.h < 1)
        P.h = 1;
    if (P.h > kMaxDegree)
        return fail(NHQ_ERR_ARG, "h must be in 1..64");
    if (P.max_iters <= 0)
        P.max_iters = 1 << 20;
    if (P.vec_dtype != NHQ_VEC_F32 && P.vec_dtype != NHQ_VEC_BF16 &&
        P.vec_dtype != NHQ_VEC_FP8E4M3 && P.vec_dtype != NHQ_VEC_F16)
        return fail(NHQ_ERR_ARG, "unknown vec_dtype %d", P.vec_dtype);
    if (P.hash_bits < 0 || P.hash_bits > 16)
        return fail(NHQ_ERR_ARG, "hash_bits must be in 0..16");
    if (P.wildcard != 0 && P.wildcard != 1)
        return fail(NHQ_ERR_ARG, "wildcard must be 0 or 1 (got %d)", P.wildcard);
    if (P.warps_per_block < 0 || P.warps_per_block > 8)
        return fail(NHQ_ERR_ARG, "warps_per_block must be in 0..8");
    if (P.warps_per_query == 0)
        P.warps_per_query = 1;
    if (P.warps_per_query != 1 && P.warps_per_query != 2 && P.warps_per_query != 4)
        return fail(NHQ_ERR_ARG, "warps_per_query must be 0, 1, 2 or 4 (got %d)",
                    P.warps_per_query);
    if (P.warps_per_block != 0 && P.warps_per_block % P.warps_per_query != 0)
        return fail(NHQ_ERR_ARG, "warps_per_block must be a multiple of warps_per_query");
    if (P.tile_rows == 0)
        P.tile_rows = 2;
    if (P.tile_rows != 2 && P.tile_rows != 4)
        return fail(NHQ_ERR_ARG, "tile_rows must be 0, 2 or 4 (got %d)", P.tile_rows);
    if (P.tile_rows == 4 && P.warps_per_query != 1)
        return fail(NHQ_ERR_ARG, "tile_rows 4 takes one warp per query");
    if (P.seed_mode < NHQ_SEED_RANDOM || P.seed_mode > NHQ_SEED_CELL_LEARNED)
        return fail(NHQ_ERR_ARG, "unknown seed_mode %d", P.seed_mode);
    const bool cell_mode =
        P.seed_mode == NHQ_SEED_CELL_NEAREST || P.seed_mode == NHQ_SEED_CELL_LEARNED;
    if (cell_mode) {
        if (ix->E == 0)
            return fail(NHQ_ERR_ARG, "seed modes 4/5 need entry cells (nhq_index_build_cells)");
        if (P.entry_cells == 0)
            P.entry_cells = 2;
        if (P.entry_cells < 1 || P.entry_cells > 8 || P.entry_cells > ix->E)
            return fail(NHQ_ERR_ARG, "entry_cells must be in 1..min(8, E)");
        if (P.wildcard != 0)
            return fail(NHQ_ERR_ARG, "seed modes 4/5 take closed queries (wildcard = 0)");
        if (P.seed_mode == NHQ_SEED_CELL_LEARNED && !is_device_ptr(P.entry_model))
            return fail(NHQ_ERR_ARG, "NHQ_SEED_CELL_LEARNED needs entry_model in device memory");
        if (P.cells_out != nullptr && !is_device_ptr(P.cells_out))
            return fail(NHQ_ERR_ARG, "cells_out must be device memory");
    }
    if (P.seed_mode == NHQ_SEED_GIVEN && (P.seeds == nullptr || P.n_seeds < 1 || P.n_seeds > 64))
        return fail(NHQ_ERR_ARG, "NHQ_SEED_GIVEN needs seeds and n_seeds in 1..64");
    const bool use_model = P.stop_model != nullptr && trace == nullptr;
    if (use_model || trace != nullptr) {
        if (P.stop_min < 0 || P.stop_every < 1)
            return fail(NHQ_ERR_ARG, "stop_min must be >= 0 and stop_every >= 1");
    }
    if (use_model) {
        if (!is_device_ptr(P.stop_model))
            return fail(NHQ_ERR_ARG, "stop_model must be device memory");
        if (!(P.stop_threshold > 0.f && P.stop_threshold < 1.f))
            return fail(NHQ_ERR_ARG, "stop_threshold must be a probability in (0, 1)");
    }
    if (P.seed_mode == NHQ_SEED_ATTRIBUTE || P.seed_mode == NHQ_SEED_ATTRIBUTE_NEAR || cell_mode)
        CKS(ensure_attribute_order(ix, s));
    if (P.vec_dtype == NHQ_VEC_BF16 && ix->Xh == nullptr) {
        CK(cudaMalloc(&ix->Xh, sizeof(__nv_bfloat16) * (size_t)ix->N * ix->xstride));
        CK(launch_rows_to_bf16(ix->X, (int64_t)ix->N * ix->xstride, ix->Xh, s));
    }
    if (P.vec_dtype == NHQ_VEC_F16 && ix->Xf == nullptr) {
        CK(cudaMalloc(&ix->Xf, sizeof(__half) * (size_t)ix->N * ix->xstride));
        CK(launch_rows_to_f16(ix->X, (int64_t)ix->N * ix->xstride, ix->Xf, s));
    }
    if (P.vec_dtype == NHQ_VEC_FP8E4M3 && ix->X8 == nullptr) {
        CK(cudaMalloc(&ix->X8, sizeof(__nv_fp8_e4m3) * (size_t)ix->N * ix->xstride));
        CK(launch_rows_to_fp8(ix->X, (int64_t)ix->N * ix->xstride, ix->X8, s));
    }
    Stager st;
    int iq = st.add(queries, sizeof(float) * (size_t)Q * ix->d, true);
    int ia = st.add(query_attributes, (size_t)Q * ix->m, true);
    int ik = st.add(k_arr, sizeof(int32_t) * (size_t)Q, true);
    int ie = st.add(ef_arr, sizeof(int32_t) * (size_t)Q, true);
    int io = st.add(ids, sizeof(uint32_t) * (size_t)Q * k_out, false);
    int id = st.add(dists, sizeof(float) * (size_t)Q * k_out, false);
    int ic = st.add(chi, (size_t)Q * k_out, false);
    int is = st.add(status, sizeof(int32_t) * (size_t)Q, false);
    int in = st.add(ndc, sizeof(int32_t) * (size_t)Q, false);
    int ix_ = st.add(expansions, sizeof(int32_t) * (size_t)Q, false);
    int isd = st.add(P.seed_mode == NHQ_SEED_GIVEN ? P.seeds : nullptr,
                     sizeof(uint32_t) * (size_t)Q * (P.seed_mode == NHQ_SEED_GIVEN ? P.n_seeds : 0),
                     true);
    CKS(st.commit(&g_stage.p, &g_stage.cap, s));
    SearchArgs a{};
    a.X = ix->X;
    a.Xh = ix->Xh;
    a.X8 = ix->X8;
    a.Xf = ix->Xf;
    a.xstride = ix->xstride;
    a.d = ix->d;
    a.N = ix->N;
    a.attr = ix->attr;
    a.nbr = ix->nbr;
    a.nbr_attr = ix->nbr_attr;
    a.R = ix->R;
    a.w = make_fusion(ix->w, ix->layout);
    a.w.wild = P.wildcard;
    a.Q = (const float *)st.dev(iq);
    a.qstride = ix->d;
    a.qattr = (const uint8_t *)st.dev(ia);
    a.nq = Q;
    a.k_arr = (const int32_t *)st.dev(ik);
    a.ef_arr = (const int32_t *)st.dev(ie);
    a.k = k;
    a.ef = ef;
    a.k_out = k_out;
    a.h = P.h;
    a.seed = P.seed;
    a.max_iters = P.max_iters;
    a.vec_dtype = P.vec_dtype;
    a.rerank = P.vec_dtype != NHQ_VEC_F32 && P.rerank != 0;
    a.ids = (uint32_t *)st.dev(io);
    a.dists = (float *)st.dev(id);
    a.chi = (uint8_t *)st.dev(ic);
    a.status = (int32_t *)st.dev(is);
    a.ndc = (int32_t *)st.dev(in);
    a.expansions = (int32_t *)st.dev(ix_);
    a.warps_per_block = P.warps_per_block;
    a.hash_bits = P.hash_bits;
    a.wpq = P.warps_per_query;
    a.tile_rows = P.tile_rows;
    // scratch: work counter and seeds | fp16 model | trace counter, hashes, final hashes
    const size_t off_w16 = (search_scratch_bytes(Q) + 255) & ~(size_t)255;
    const size_t off_tr = off_w16 + 2048;
    const size_t tr_bytes = trace ? 256 + sizeof(unsigned long long) * ((size_t)trace->cap + Q) : 0;
    // the fp16 copy of the entry model after the trace records
    const size_t off_entry = (off_tr + tr_bytes + 255) & ~(size_t)255;
    const size_t entry_bytes = P.seed_mode == NHQ_SEED_CELL_LEARNED
                                   ? sizeof(__half) * (size_t)entry_param_count(ix->d, ix->E)
                                   : 0;
    // the cell scores of every query [Q][E] and the model's hidden values [Q][64]
    const size_t off_scores = (off_entry + entry_bytes + 255) & ~(size_t)255;
    const size_t scores_bytes = cell_mode ? sizeof(float) * (size_t)Q * ix->E : 0;
    const size_t off_hidden = (off_scores + scores_bytes + 255) & ~(size_t)255;
    const size_t hidden_bytes = P.seed_mode == NHQ_SEED_CELL_LEARNED
                                    ? sizeof(float) * (size_t)Q * NHQ_ENTRY_HIDDEN
                                    : 0;
    CKS(scratch(ix, off_hidden + hidden_bytes));
    a.stop_w16 = nullptr;
    a.stop_every = 0;
    a.stop_min = P.stop_min;
    a.tr_feat = nullptr;
    a.tr_hash = nullptr;
    a.tr_q = nullptr;
    a.tr_count = nullptr;
    a.tr_cap = 0;
    a.tr_final = nullptr;
    if (use_model) {
        __half *w16 = reinterpret_cast<__half *>((char *)ix->scratch + off_w16);
        CK(launch_mlp_to_half(P.stop_model, w16, s));
        a.stop_w16 = w16;
        a.stop_logit = logf(P.stop_threshold / (1.f - P.stop_threshold));
        a.stop_every = P.stop_every;
    }
    if (trace != nullptr) {
        char *t = (char *)ix->scratch + off_tr;
        a.tr_count = reinterpret_cast<unsigned int *>(t);
        a.tr_hash = reinterpret_cast<unsigned long long *>(t + 256);
        a.tr_final = a.tr_hash + trace->cap;
        a.tr_feat = trace->features;
        a.tr_q = trace->query;
        a.tr_cap = trace->cap;
        a.stop_every = P.stop_every;
        CK(cudaMemsetAsync(a.tr_count, 0, sizeof(unsigned int), s));
    }
    a.seeds = nullptr;
    a.n_seeds = 0;
    a.order = nullptr;
    if (P.seed_mode == NHQ_SEED_GIVEN) {
        a.seeds = (const uint32_t *)st.dev(isd);
        a.n_seeds = P.n_seeds;
    } else if (P.seed_mode == NHQ_SEED_ATTRIBUTE || P.seed_mode == NHQ_SEED_ATTRIBUTE_NEAR ||
               cell_mode) {
        uint32_t *sd = reinterpret_cast<uint32_t *>((char *)ix->scratch + 256);
        uint32_t *order = sd + (size_t)32 * Q;
        uint8_t *bucket = reinterpret_cast<uint8_t *>(order + Q);
        if (P.seed_mode == NHQ_SEED_ATTRIBUTE) {
            CK(launch_attribute_seeds(a, ix->attr_sorted, ix->id_sorted, sd, bucket, s));
        } else if (P.seed_mode == NHQ_SEED_ATTRIBUTE_NEAR) {
            CK(launch_attribute_near_seeds(a, ix->attr_sorted, ix->id_sorted, sd, bucket, s));
        } else {
            float *scores = reinterpret_cast<float *>((char *)ix->scratch + off_scores);
            if (P.seed_mode == NHQ_SEED_CELL_LEARNED) {
                __half *ew16 = reinterpret_cast<__half *>((char *)ix->scratch + off_entry);
                float *hidden = reinterpret_cast<float *>((char *)ix->scratch + off_hidden);
                CK(launch_entry_to_half(P.entry_model, entry_param_count(ix->d, ix->E), ew16, s));
                CK(launch_entry_scores_learned(ew16, P.entry_model, ix->d, ix->E, a.Q, a.qstride,
                                               Q, hidden, scores, s));
            } else {
                CK(launch_entry_scores_nearest(ix->centT, ix->cnh, ix->d, ix->E, a.Q, a.qstride,
                                               Q, scores, s));
            }
            CK(launch_cell_seeds(a, ix->attr_sorted, ix->id_sorted, ix->cell_key, ix->cell_id,
                                 ix->E, P.entry_cells, scores, P.cells_out, sd, bucket, s));
        }
        CK(launch_query_order(bucket, Q, order, s));
        a.seeds = sd;
        a.n_seeds = 32;
        a.order = order;
    }
    cudaError_t e = launch_search(a, ix->scratch, ix->sm_count, ix->smem_optin, s);
    if (e == cudaErrorInvalidValue)
        return fail(NHQ_ERR_ARG, "search launch: ef/hash_bits/warps_per_block do not fit shared memory");
    if (e != cudaSuccess)
        return fail_cuda(e, "search kernel launch");
    if (trace != nullptr) {
        unsigned int cnt = 0;
        CK(cudaMemcpyAsync(&cnt, a.tr_count, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const int64_t nt = (int64_t)cnt < trace->cap ? (int64_t)cnt : trace->cap;
        CK(launch_trace_labels(a.tr_hash, a.tr_q, a.tr_final, nt, trace->labels, s));
        *trace->n_traces = nt;
    }
    return st.finish(s);
}

nhq_status nhq_search(const nhq_index *ix, const float *queries, const uint8_t *query_attributes,
                      int64_t Q, int32_t k, int32_t ef, const nhq_search_params *params,
                      uint32_t *ids, float *dists, uint8_t *chi, int32_t *status, int32_t *ndc,
                      int32_t *expansions, void *stream) {
    if (ix == nullptr)
        return fail(NHQ_ERR_ARG, "index is NULL");
    if (ix->nbr == nullptr)
        return fail(NHQ_ERR_ARG, "the index has no graph (build or set one first)");
    if (Q < 0)
        return fail(NHQ_ERR_ARG, "Q must be >= 0");
    if (k < 1 || k > kMaxK)
        return fail(NHQ_ERR_ARG, "k must be in 1..256 (got %d)", k);
    if (ef < k || ef > kMaxEf)
        return fail(NHQ_ERR_ARG, "ef must be in k..1024 (got %d)", ef);
    if (Q == 0)
        return NHQ_OK;
    if (queries == nullptr || query_attributes == nullptr || ids == nullptr)
        return fail(NHQ_ERR_ARG, "queries, query_attributes and ids are required");
    return search_common(ix, queries, query_attributes, Q, nullptr, nullptr, k, ef, k, params, ids,
                         dists, chi, status, ndc, expansions, stream);
}

nhq_status nhq_search_batched(const nhq_index *ix, const float *queries,
                              const uint8_t *query_attributes, int64_t Q, const int32_t *k_arr,
                              const int32_t *ef_arr, int32_t k_max,
                              const nhq_search_params *params, uint32_t *ids, float *dists,
                              uint8_t *chi, int32_t *status, int32_t *ndc, int32_t *expansions,
                              void *stream) {
    if (ix == nullptr)
        return fail(NHQ_ERR_ARG, "index is NULL");
    if (ix->nbr == nullptr)
        return fail(NHQ_ERR_ARG, "the index has no graph (build or set one first)");
    if (Q < 0)
        return fail(NHQ_ERR_ARG, "Q must be >= 0");
    if (k_max < 1 || k_max > kMaxK)
        return fail(NHQ_ERR_ARG, "k_max must be in 1..256 (got %d)", k_max);
    if (Q == 0)
        return NHQ_OK;
    if (queries == nullptr || query_attributes == nullptr || ids == nullptr || k_arr == nullptr ||
        ef_arr == nullptr)
        return fail(NHQ_ERR_ARG, "queries, query_attributes, k_arr, ef_arr and ids are required");
    // the per-query values bound the pool size, so they are read on the host
    std::vector<int32_t> hk((size_t)Q), he((size_t)Q);
    cudaStream_t s = as_stream(stream);
    CK(cudaMemcpyAsync(hk.data(), k_arr, sizeof(int32_t) * Q, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(he.data(), ef_arr, sizeof(int32_t) * Q, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    int ef_max = 1;
    for (int64_t i = 0; i < Q; ++i) {
        if (hk[i] < 1 || hk[i] > k_max)
            return fail(NHQ_ERR_ARG, "k_arr[%lld] = %d outside 1..k_max", (long long)i, hk[i]);
        if (he[i] < hk[i] || he[i] > kMaxEf)
            return fail(NHQ_ERR_ARG, "ef_arr[%lld] = %d outside k..1024", (long long)i, he[i]);
        ef_max = he[i] > ef_max ? he[i] : ef_max;
    }
    return search_common(ix, queries, query_attributes, Q, k_arr, ef_arr, k_max, ef_max, k_max,
                         params, ids, dists, chi, status, ndc, expansions, stream);
}

}  // extern "C"

// Times run(P) for every launch shape (rows per team, warps per query, warps per block,
// visited-filter size from the smallest legal one) with CUDA events, one warm-up and
// three timed calls each, and writes the fastest shape into params.
template <typename Run>
static nhq_status autotune_shapes(const nhq_index *ix, int ef, nhq_search_params *params,
                                  float *best_ms, cudaStream_t s, Run run) {
    const int ef_cap = (ef + 31) & ~31;
    int bmin = 6;  // the smallest filter the rebuild rule allows, then three larger ones
    while ((1 << bmin) < 2 * (ef_cap + ix->R) + 64)
        ++bmin;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    nhq_search_params best = *params;
    float best_t = 1e30f;
    bool any = false;
    const int wpbs[3] = {2, 4, 8}, wpqs[3] = {1, 2, 4}, rows[2] = {2, 4};
    for (int tr : rows) {
        for (int wpq : wpqs) {
            for (int wpb : wpbs) {
                if (wpb < wpq)
                    continue;
                for (int b = bmin; b <= bmin + 3 && b <= 16; ++b) {
                    nhq_search_params P = *params;
                    P.tile_rows = tr;
                    P.warps_per_query = wpq;
                    P.warps_per_block = wpb;
                    P.hash_bits = b;
                    nhq_status st = run(P);
                    if (st == NHQ_ERR_ARG)
                        continue;  // this shape does not fit shared memory
                    if (st != NHQ_OK) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return st;
                    }
                    CK(cudaEventRecord(e0, s));
                    for (int r = 0; r < 3; ++r)
                        run(P);
                    CK(cudaEventRecord(e1, s));
                    CK(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, e0, e1));
                    ms /= 3.f;
                    if (ms < best_t) {
                        best_t = ms;
                        best = P;
                        any = true;
                    }
                }
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!any)
        return fail(NHQ_ERR_ARG, "no launch shape fits shared memory for ef = %d", ef);
    params->warps_per_query = best.warps_per_query;
    params->tile_rows = best.tile_rows;
    params->warps_per_block = best.warps_per_block;
    params->hash_bits = best.hash_bits;
    if (best_ms)
        *best_ms = best_t;
    return NHQ_OK;
}

extern "C" {

nhq_status nhq_autotune_search(const nhq_index *ix, const float *queries,
                               const uint8_t *query_attributes, int64_t Q, int32_t k, int32_t ef,
                               nhq_search_params *params, uint32_t *ids, float *best_ms,
                               void *stream) {
    if (ix == nullptr || params == nullptr || ids == nullptr || Q < 1)
        return fail(NHQ_ERR_ARG, "index, params, ids and Q >= 1 are required");
    if (!is_device_ptr(queries) || !is_device_ptr(query_attributes) || !is_device_ptr(ids))
        return fail(NHQ_ERR_ARG, "nhq_autotune_search takes device pointers");
    return autotune_shapes(ix, ef, params, best_ms, as_stream(stream),
                           [&](const nhq_search_params &P) {
                               return nhq_search(ix, queries, query_attributes, Q, k, ef, &P,
                                                 ids, nullptr, nullptr, nullptr, nullptr,
                                                 nullptr, stream);
                           });
}

nhq_status nhq_autotune_batched(const nhq_index *ix, const float *queries,
                                const uint8_t *query_attributes, int64_t Q,
                                const int32_t *k_arr, const int32_t *ef_arr, int32_t k_max,
                                nhq_search_params *params, uint32_t *ids, float *best_ms,
                                void *stream) {
    if (ix == nullptr || params == nullptr || ids == nullptr || Q < 1 || k_arr == nullptr ||
        ef_arr == nullptr)
        return fail(NHQ_ERR_ARG, "index, params, ids, k_arr, ef_arr and Q >= 1 are required");
    if (!is_device_ptr(queries) || !is_device_ptr(query_attributes) || !is_device_ptr(ids) ||
        !is_device_ptr(k_arr) || !is_device_ptr(ef_arr))
        return fail(NHQ_ERR_ARG, "nhq_autotune_batched takes device pointers");
    std::vector<int32_t> he((size_t)Q);
    cudaStream_t s = as_stream(stream);
    CK(cudaMemcpyAsync(he.data(), ef_arr, sizeof(int32_t) * Q, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int ef_max = 1;
    for (int32_t e : he)
        ef_max = e > ef_max ? e : ef_max;
    return autotune_shapes(ix, ef_max, params, best_ms, s, [&](const nhq_search_params &P) {
        return nhq_search_batched(ix, queries, query_attributes, Q, k_arr, ef_arr, k_max, &P,
                                  ids, nullptr, nullptr, nullptr, nullptr, nullptr, stream);
    });
}

nhq_status nhq_recall(const uint32_t *ids, int32_t k, const uint32_t *truth, int32_t k_truth,
                      int64_t Q, float *recall, void *stream) {
    if (ids == nullptr || truth == nullptr || recall == nullptr || Q < 0 || k < 1 ||
        k_truth < 1 || k_truth > k)
        return fail(NHQ_ERR_ARG, "nhq_recall: need ids, truth, recall, Q >= 0, 1 <= k_truth <= k");
    if (!is_device_ptr(ids) || !is_device_ptr(truth))
        return fail(NHQ_ERR_ARG, "nhq_recall takes device ids and truth");
    cudaStream_t s = as_stream(stream);
    double *acc = nullptr;
    CK(cudaMallocAsync(&acc, 2 * sizeof(double), s));
    double h[2] = {0.0, 0.0};
    cudaError_t e = launch_recall(ids, k, truth, k_truth, Q, acc, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(acc, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return fail_cuda(e, "nhq_recall");
    *recall = h[1] > 0.0 ? (float)(h[0] / h[1]) : 0.f;
    return NHQ_OK;
}

nhq_status nhq_autotune_beam(const nhq_index *ix, const float *queries,
                             const uint8_t *query_attributes, int64_t Q, int32_t k,
                             const int32_t *ef_list, int32_t n_ef, const uint32_t *truth,
                             float target, nhq_search_params *params, uint32_t *ids,
                             int32_t *ef_out, float *recall_out, float *best_ms, void *stream) {
    if (ix == nullptr || params == nullptr || ids == nullptr || truth == nullptr ||
        ef_list == nullptr || ef_out == nullptr || Q < 1)
        return fail(NHQ_ERR_ARG, "index, params, ids, truth, ef_list, ef_out and Q >= 1 are "
                                 "required");
    if (n_ef < 1 || n_ef > 64)
        return fail(NHQ_ERR_ARG, "n_ef must be in 1..64");
    if (!(target > 0.f && target <= 1.f))
        return fail(NHQ_ERR_ARG, "target must be in (0, 1]");
    for (int i = 0; i < n_ef; ++i)
        if (ef_list[i] < k || ef_list[i] > kMaxEf || (i > 0 && ef_list[i] <= ef_list[i - 1]))
            return fail(NHQ_ERR_ARG, "ef_list must ascend within k..1024");
    int chosen = ef_list[n_ef - 1];
    float rec = 0.f;
    for (int i = 0; i < n_ef; ++i) {
        CKS(nhq_search(ix, queries, query_attributes, Q, k, ef_list[i], params, ids, nullptr,
                       nullptr, nullptr, nullptr, nullptr, stream));
        CKS(nhq_recall(ids, k, truth, k, Q, &rec, stream));
        if (rec >= target || i == n_ef - 1) {
            chosen = ef_list[i];
            break;
        }
    }
    *ef_out = chosen;
    if (recall_out)
        *recall_out = rec;
    return nhq_autotune_search(ix, queries, query_attributes, Q, k, chosen, params, ids, best_ms,
                               stream);
}

}  // extern "C"

struct nhq_search_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// One ordinary call of run(stream) first (it builds the lazily made index parts and sizes
// the scratch), then the same call captured on a private stream and instantiated.
template <typename Run>
static nhq_status capture_search(Run run, nhq_search_graph **out) {
    cudaStream_t cs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    nhq_status st = run(cs);
    cudaError_t e = cudaStreamSynchronize(cs);
    if (st == NHQ_OK && e != cudaSuccess)
        st = fail_cuda(e, "cudaStreamSynchronize");
    nhq_search_graph *g = nullptr;
    if (st == NHQ_OK) {
        g = new nhq_search_graph();
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            st = fail_cuda(e, "cudaStreamBeginCapture");
        } else {
            st = run(cs);
            e = cudaStreamEndCapture(cs, &g->graph);
            if (st == NHQ_OK && e != cudaSuccess)
                st = fail_cuda(e, "cudaStreamEndCapture");
            if (st == NHQ_OK && (e = cudaGraphInstantiate(&g->exec, g->graph, 0)) != cudaSuccess)
                st = fail_cuda(e, "cudaGraphInstantiate");
        }
    }
    cudaStreamDestroy(cs);
    if (st != NHQ_OK) {
        nhq_search_graph_free(g);
        return st;
    }
    *out = g;
    return NHQ_OK;
}

extern "C" {

nhq_status nhq_search_graph_create(const nhq_index *ix, const float *queries,
                                   const uint8_t *query_attributes, int64_t Q, int32_t k,
                                   int32_t ef, const nhq_search_params *params, uint32_t *ids,
                                   float *dists, uint8_t *chi, nhq_search_graph **out) {
    if (out == nullptr)
        return fail(NHQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!is_device_ptr(queries) || !is_device_ptr(query_attributes) || !is_device_ptr(ids) ||
        (dists && !is_device_ptr(dists)) || (chi && !is_device_ptr(chi)))
        return fail(NHQ_ERR_ARG, "nhq_search_graph_create takes device pointers");
    return capture_search(
        [&](cudaStream_t cs) {
            return nhq_search(ix, queries, query_attributes, Q, k, ef, params, ids, dists, chi,
                              nullptr, nullptr, nullptr, cs);
        },
        out);
}

nhq_status nhq_search_graph_create_batched(const nhq_index *ix, const float *queries,
                                           const uint8_t *query_attributes, int64_t Q,
                                           const int32_t *k_arr, const int32_t *ef_arr,
                                           int32_t k_max, const nhq_search_params *params,
                                           uint32_t *ids, float *dists, uint8_t *chi,
                                           nhq_search_graph **out) {
    if (out == nullptr)
        return fail(NHQ_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (ix == nullptr || ix->nbr == nullptr)
        return fail(NHQ_ERR_ARG, "the index has no graph (build or set one first)");
    if (Q < 1 || k_max < 1 || k_max > kMaxK)
        return fail(NHQ_ERR_ARG, "need Q >= 1 and k_max in 1..256");
    if (!is_device_ptr(queries) || !is_device_ptr(query_attributes) || !is_device_ptr(ids) ||
        !is_device_ptr(k_arr) || !is_device_ptr(ef_arr) || (dists && !is_device_ptr(dists)) ||
        (chi && !is_device_ptr(chi)))
        return fail(NHQ_ERR_ARG, "nhq_search_graph_create_batched takes device pointers");
    // the per-query values are checked (and the pool sized) once, here
    std::vector<int32_t> hk((size_t)Q), he((size_t)Q);
    CK(cudaMemcpy(hk.data(), k_arr, sizeof(int32_t) * Q, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(he.data(), ef_arr, sizeof(int32_t) * Q, cudaMemcpyDeviceToHost));
    int ef_max = 1;
    for (int64_t i = 0; i < Q; ++i) {
        if (hk[i] < 1 || hk[i] > k_max)
            return fail(NHQ_ERR_ARG, "k_arr[%lld] = %d outside 1..k_max", (long long)i, hk[i]);
        if (he[i] < hk[i] || he[i] > kMaxEf)
            return fail(NHQ_ERR_ARG, "ef_arr[%lld] = %d outside k..1024", (long long)i, he[i]);
        ef_max = he[i] > ef_max ? he[i] : ef_max;
    }
    return capture_search(
        [&](cudaStream_t cs) {
            return search_common(ix, queries, query_attributes, Q, k_arr, ef_arr, k_max, ef_max,
                                 k_max, params, ids, dists, chi, nullptr, nullptr, nullptr, cs);
        },
        out);
}

nhq_status nhq_search_graph_launch(nhq_search_graph *g, void *stream) {
    if (g == nullptr || g->exec == nullptr)
        return fail(NHQ_ERR_ARG, "graph is NULL");
    CK(cudaGraphLaunch(g->exec, as_stream(stream)));
    return NHQ_OK;
}

void nhq_search_graph_free(nhq_search_graph *g) {
    if (g == nullptr)
        return;
    if (g->exec)
        cudaGraphExecDestroy(g->exec);
    if (g->graph)
        cudaGraphDestroy(g->graph);
    delete g;
}

nhq_status nhq_search_trace(const nhq_index *ix, const float *queries,
                            const uint8_t *query_attributes, int64_t Q, int32_t k, int32_t ef,
                            const nhq_search_params *params, float *features, uint8_t *labels,
                            int32_t *query, int64_t cap, int64_t *n_traces, void *stream) {
    if (ix == nullptr || ix->nbr == nullptr)
        return fail(NHQ_ERR_ARG, "index with a graph is required");
    if (Q < 1 || k < 1 || k > kMaxK || ef < k || ef > kMaxEf || cap < 1 || n_traces == nullptr)
        return fail(NHQ_ERR_ARG, "need Q >= 1, k in 1..256, ef in k..1024, cap >= 1, n_traces");
    if (!is_device_ptr(queries) || !is_device_ptr(query_attributes) || !is_device_ptr(features) ||
        !is_device_ptr(labels) || !is_device_ptr(query))
        return fail(NHQ_ERR_ARG, "nhq_search_trace takes device pointers");
    if (params == nullptr)
        return fail(NHQ_ERR_ARG, "params (stop_min, stop_every) are required");
    uint32_t *ids = nullptr;
    CK(cudaMallocAsync((void **)&ids, sizeof(uint32_t) * (size_t)Q * k, as_stream(stream)));
    TraceOut t;
    t.features = features;
    t.labels = labels;
    t.query = query;
    t.cap = cap;
    t.n_traces = n_traces;
    nhq_status st = search_common(ix, queries, query_attributes, Q, nullptr, nullptr, k, ef, k,
                                  params, ids, nullptr, nullptr, nullptr, nullptr, nullptr,
                                  stream, &t);
    cudaFreeAsync(ids, as_stream(stream));
    return st;
}

nhq_status nhq_mlp_forward(const float *params, const float *features, int64_t n, float *logits,
                           void *stream) {
    if (n < 0 || params == nullptr || (n > 0 && (features == nullptr || logits == nullptr)))
        return fail(NHQ_ERR_ARG, "params, features and logits are required, n >= 0");
    if (!is_device_ptr(params) || (n > 0 && (!is_device_ptr(features) || !is_device_ptr(logits))))
        return fail(NHQ_ERR_ARG, "nhq_mlp_forward takes device pointers");
    CK(mlp_forward(params, features, n, logits, as_stream(stream)));
    return NHQ_OK;
}

nhq_status nhq_mlp_grad(const float *params, const float *features, const float *labels,
                        int64_t n, float *grad, float *loss, void *stream) {
    if (n < 1 || !params || !features || !labels || !grad || !loss)
        return fail(NHQ_ERR_ARG, "params, features, labels, grad and loss are required, n >= 1");
    if (!is_device_ptr(params) || !is_device_ptr(features) || !is_device_ptr(labels) ||
        !is_device_ptr(grad) || !is_device_ptr(loss))
        return fail(NHQ_ERR_ARG, "nhq_mlp_grad takes device pointers");
    cudaStream_t s = as_stream(stream);
    CK(cudaMemsetAsync(grad, 0, sizeof(float) * NHQ_MLP_PARAMS, s));
    CK(cudaMemsetAsync(loss, 0, sizeof(float), s));
    CK(mlp_grad(params, features, labels, n, n, grad, loss, s));
    return NHQ_OK;
}

nhq_status nhq_mlp_train(float *params, const float *features, const float *labels, int64_t n,
                         int32_t epochs, int32_t batch, float lr, void *stream) {
    if (n < 1 || epochs < 0 || batch < 1 || !(lr > 0.f) || !params || !features || !labels)
        return fail(NHQ_ERR_ARG, "need n >= 1, epochs >= 0, batch >= 1, lr > 0 and arrays");
    if (!is_device_ptr(params) || !is_device_ptr(features) || !is_device_ptr(labels))
        return fail(NHQ_ERR_ARG, "nhq_mlp_train takes device pointers");
    CK(mlp_train(params, features, labels, n, epochs, batch, lr, as_stream(stream)));
    return NHQ_OK;
}

static const char kMagic[8] = {'N', 'H', 'Q', 'I', 'D', 'X', '0', '1'};

nhq_status nhq_save(const nhq_index *ix, const char *path) {
    if (ix == nullptr || path == nullptr)
        return fail(NHQ_ERR_ARG, "index and path are required");
    FILE *f = fopen(path, "wb");
    if (!f)
        return fail(NHQ_ERR_IO, "cannot open %s for writing", path);
    const size_t N = (size_t)ix->N;
    std::vector<float> row((size_t)ix->xstride * 4096);
    std::vector<uint32_t> attr(N), nbr(N * (size_t)ix->R);
    // version 2: version 1 followed by the attribute layout (shift[32], width[32])
    int32_t hdr[8] = {2, (int32_t)(ix->N & 0x7FFFFFFF), ix->d, ix->m, ix->R, ix->w.mode, 0, 0};
    float wts[2] = {ix->w.w_v, ix->w.w_l};
    uint8_t lay[2 * kMaxAttr];
    memcpy(lay, ix->layout.shift, kMaxAttr);
    memcpy(lay + kMaxAttr, ix->layout.width, kMaxAttr);
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              fwrite(wts, sizeof(wts), 1, f) == 1 && fwrite(lay, sizeof(lay), 1, f) == 1;
    cudaError_t e = cudaSuccess;
    for (size_t r0 = 0; ok && r0 < N; r0 += 4096) {
        size_t nr = N - r0 < 4096 ? N - r0 : 4096;
        e = cudaMemcpy(row.data(), ix->X + r0 * ix->xstride, sizeof(float) * nr * ix->xstride,
                       cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            break;
        for (size_t r = 0; ok && r < nr; ++r)
            ok = fwrite(row.data() + r * ix->xstride, sizeof(float), ix->d, f) == (size_t)ix->d;
    }
    if (e == cudaSuccess && ok)
        e = cudaMemcpy(attr.data(), ix->attr, sizeof(uint32_t) * N, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && ok && ix->R > 0)
        e = cudaMemcpy(nbr.data(), ix->nbr, sizeof(uint32_t) * nbr.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && ok)
        ok = fwrite(attr.data(), sizeof(uint32_t), N, f) == N &&
             fwrite(nbr.data(), sizeof(uint32_t), nbr.size(), f) == nbr.size();
    bool closed = fclose(f) == 0;
    if (e != cudaSuccess)
        return fail_cuda(e, "nhq_save copy");
    if (!ok || !closed)
        return fail(NHQ_ERR_IO, "write to %s failed", path);
    return NHQ_OK;
}

nhq_status nhq_load(const char *path, void *stream, nhq_index **out) {
    if (path == nullptr || out == nullptr)
        return fail(NHQ_ERR_ARG, "path and out are required");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f)
        return fail(NHQ_ERR_IO, "cannot open %s", path);
    char magic[8];
    int32_t hdr[8];
    float wts[2];
    uint8_t lay[2 * kMaxAttr];
    bool hdr_ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, kMagic, 8) == 0 &&
                  fread(hdr, sizeof(hdr), 1, f) == 1 && fread(wts, sizeof(wts), 1, f) == 1 &&
                  (hdr[0] == 1 || hdr[0] == 2) && hdr[1] >= 1 && hdr[2] >= 1 && hdr[3] >= 1 &&
                  hdr[3] <= (hdr[0] == 1 ? 4 : kMaxAttr) && hdr[4] >= 0 && hdr[4] <= kMaxDegree;
    if (hdr_ok && hdr[0] == 2)
        hdr_ok = fread(lay, sizeof(lay), 1, f) == 1;
    if (hdr_ok && hdr[0] == 1) {  // a byte per attribute
        for (int j = 0; j < kMaxAttr; ++j) {
            lay[j] = (uint8_t)(8 * j);
            lay[kMaxAttr + j] = 8;
        }
    }
    for (int j = 0; hdr_ok && j < hdr[3]; ++j)
        hdr_ok = lay[kMaxAttr + j] >= 1 && lay[kMaxAttr + j] <= 8 + 1 &&
                 lay[j] + lay[kMaxAttr + j] <= 32;
    if (!hdr_ok) {
        fclose(f);
        return fail(NHQ_ERR_IO, "%s is not an index file of version 1 or 2", path);
    }
    const size_t N = (size_t)hdr[1], d = (size_t)hdr[2], m = (size_t)hdr[3], R = (size_t)hdr[4];
    std::vector<float> X(N * d);
    std::vector<uint32_t> attr(N), nbr(N * R);
    bool ok = fread(X.data(), sizeof(float), X.size(), f) == X.size() &&
              fread(attr.data(), sizeof(uint32_t), N, f) == N &&
              fread(nbr.data(), sizeof(uint32_t), nbr.size(), f) == nbr.size();
    fclose(f);
    if (!ok)
        return fail(NHQ_ERR_IO, "%s is truncated", path);
    std::vector<uint8_t> a8(N * m);
    for (size_t i = 0; i < N; ++i)
        for (size_t j = 0; j < m; ++j)
            a8[i * m + j] = (uint8_t)((attr[i] >> lay[j]) & ((1u << lay[kMaxAttr + j]) - 1u));
    nhq_weights w{hdr[5], wts[0], wts[1]};
    nhq_index *ix = nullptr;
    CKS(nhq_index_create(X.data(), (int64_t)N, (int32_t)d, a8.data(), (int32_t)m, w, stream, &ix));
    if (R > 0) {
        nhq_status st = nhq_index_set_graph(ix, nbr.data(), (int32_t)R, stream);
        if (st != NHQ_OK) {
            nhq_free(ix);
            return st;
        }
    }
    *out = ix;
    return NHQ_OK;
}

}  // extern "C"
