// k_util.cu -- data-layout kernels: ordinal attribute packing (Sec. 3.2),
// padded row copies of the object vectors, the BF16 scoring copy, and the
// per-edge attribute words stored beside the adjacency.
#include "nhq_internal.cuh"

namespace nhq {

namespace {

// code j of row i at bits shift[j]; codes above maxc[j] (queries only) as maxc[j] + 1
__global__ void pack_attr_kernel(const uint8_t *__restrict__ a, int64_t n, AttrLayout L,
                                 uint32_t *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t w = 0;
        for (int j = 0; j < L.m; ++j) {
            const uint32_t v = a[i * L.m + j];
            w |= (v <= L.maxc[j] ? v : (uint32_t)L.maxc[j] + 1u) << L.shift[j];
        }
        out[i] = w;
    }
}

__global__ void pack_query_kernel(const uint8_t *__restrict__ a, int64_t n, Fusion w,
                                  uint32_t *__restrict__ out, uint32_t *__restrict__ hi_out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t hi;
        out[i] = pack_query_word(a + i * w.m, w, &hi);
        if (hi_out)
            hi_out[i] = hi;
    }
}

// out[j] = the largest code of attribute j over the n rows (out zeroed by the caller)
__global__ void attr_max_kernel(const uint8_t *__restrict__ a, int64_t n, int m,
                                unsigned int *__restrict__ out) {
    __shared__ unsigned int smax[kMaxAttr];
    if (threadIdx.x < kMaxAttr)
        smax[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t total = n * m;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        atomicMax(&smax[(int)(i % m)], (unsigned int)a[i]);
    __syncthreads();
    if (threadIdx.x < m)
        atomicMax(&out[threadIdx.x], smax[threadIdx.x]);
}

// dst[r][0..xstride) = src[r][0..d) followed by zeros; flags non-finite input.
__global__ void copy_rows_kernel(const float *__restrict__ src, int64_t N, int d, int xstride,
                                 float *__restrict__ dst, int *__restrict__ bad) {
    int64_t total = N * (int64_t)xstride;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i / xstride;
        int c = (int)(i - r * xstride);
        float v = c < d ? src[r * d + c] : 0.0f;
        if (!isfinite(v))
            *bad = 1;
        dst[i] = v;
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ src, int64_t n,
                               __nv_bfloat16 *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn(src[i]);
}

__global__ void to_fp8_kernel(const float *__restrict__ src, int64_t n,
                              __nv_fp8_e4m3 *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        __nv_fp8_e4m3 v;
        v.__x = __nv_cvt_float_to_fp8(src[i], __NV_SATFINITE, __NV_E4M3);
        dst[i] = v;
    }
}

// Also validates the adjacency: an id that is neither kNone nor < N sets *bad.
__global__ void gather_nbr_attr_kernel(const uint32_t *__restrict__ nbr,
                                       const uint32_t *__restrict__ attr, int64_t N,
                                       int64_t total, uint32_t *__restrict__ out,
                                       int *__restrict__ bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = nbr[i];
        if (v != kNone && (int64_t)v >= N) {
            *bad = 1;
            v = kNone;
        }
        out[i] = v == kNone ? 0u : attr[v];
    }
}

inline int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 8192 ? 8192 : g));
}

}  // namespace

cudaError_t launch_pack_attributes(const uint8_t *a, int64_t n, const AttrLayout &L,
                                   uint32_t *out, cudaStream_t s) {
    if (n <= 0)
        return cudaSuccess;
    pack_attr_kernel<<<grid_for(n), 256, 0, s>>>(a, n, L, out);
    return cudaGetLastError();
}

cudaError_t launch_pack_queries(const uint8_t *a, int64_t n, const Fusion &w, uint32_t *out,
                                uint32_t *hi_out, cudaStream_t s) {
    if (n <= 0)
        return cudaSuccess;
    pack_query_kernel<<<grid_for(n), 256, 0, s>>>(a, n, w, out, hi_out);
    return cudaGetLastError();
}

cudaError_t launch_attr_max(const uint8_t *a, int64_t n, int m, unsigned int *out,
                            cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned int) * kMaxAttr, s);
    if (e != cudaSuccess || n <= 0)
        return e;
    attr_max_kernel<<<grid_for(n * m), 256, 0, s>>>(a, n, m, out);
    return cudaGetLastError();
}

template <typename T>
__global__ void copy_rows_typed_kernel(const T *__restrict__ src, int64_t N, int d, int xstride,
                                       float *__restrict__ dst, int *__restrict__ bad) {
    int64_t total = N * (int64_t)xstride;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = i / xstride;
        int c = (int)(i - r * xstride);
        float v = c < d ? (float)src[r * d + c] : 0.0f;  // exact: every f16 / bf16 is an f32
        if (!isfinite(v))
            *bad = 1;
        dst[i] = v;
    }
}

__global__ void to_f16_kernel(const float *__restrict__ src, int64_t n, __half *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2half_rn(src[i]);
}

cudaError_t launch_copy_rows_typed(const void *src, int dtype, int64_t N, int d, int xstride,
                                   float *dst, int *bad, cudaStream_t s) {
    if (dtype == NHQ_F16)
        copy_rows_typed_kernel<__half><<<grid_for(N * xstride), 256, 0, s>>>(
            (const __half *)src, N, d, xstride, dst, bad);
    else
        copy_rows_typed_kernel<__nv_bfloat16><<<grid_for(N * xstride), 256, 0, s>>>(
            (const __nv_bfloat16 *)src, N, d, xstride, dst, bad);
    return cudaGetLastError();
}

cudaError_t launch_rows_to_f16(const float *src, int64_t n, __half *dst, cudaStream_t s) {
    to_f16_kernel<<<grid_for(n), 256, 0, s>>>(src, n, dst);
    return cudaGetLastError();
}

cudaError_t launch_copy_rows(const float *src, int64_t N, int d, int xstride, float *dst,
                             int *bad, cudaStream_t s) {
    copy_rows_kernel<<<grid_for(N * xstride), 256, 0, s>>>(src, N, d, xstride, dst, bad);
    return cudaGetLastError();
}

cudaError_t launch_rows_to_bf16(const float *src, int64_t n, __nv_bfloat16 *dst, cudaStream_t s) {
    to_bf16_kernel<<<grid_for(n), 256, 0, s>>>(src, n, dst);
    return cudaGetLastError();
}

cudaError_t launch_rows_to_fp8(const float *src, int64_t n, __nv_fp8_e4m3 *dst, cudaStream_t s) {
    to_fp8_kernel<<<grid_for(n), 256, 0, s>>>(src, n, dst);
    return cudaGetLastError();
}

cudaError_t launch_gather_nbr_attr(const uint32_t *nbr, const uint32_t *attr, int64_t N, int R,
                                   uint32_t *out, int *bad, cudaStream_t s) {
    gather_nbr_attr_kernel<<<grid_for(N * R), 256, 0, s>>>(nbr, attr, N, N * (int64_t)R, out, bad);
    return cudaGetLastError();
}

static void finish_masks(AttrLayout *L) {
    L->hi = L->lo = 0u;
    for (int j = 0; j < L->m; ++j) {
        const uint32_t top = 1u << (L->shift[j] + L->width[j] - 1);
        const uint32_t field = (L->width[j] >= 32 ? 0xFFFFFFFFu : ((1u << L->width[j]) - 1u))
                               << L->shift[j];
        L->hi |= top;
        L->lo |= field & ~top;
    }
}

AttrLayout byte_layout(int m) {
    AttrLayout L;
    L.m = m;
    for (int j = 0; j < m && j < 4; ++j) {
        L.shift[j] = (uint8_t)(8 * j);
        L.width[j] = 8;
        L.maxc[j] = 255;
        L.amax[j] = 255;
    }
    finish_masks(&L);
    return L;
}

bool compact_layout(int m, const uint8_t *maxc, AttrLayout *out) {
    AttrLayout L;
    L.m = m;
    int bits = 0;
    for (int j = 0; j < m; ++j) {
        int w = 1;  // bits for 0..maxc + 1
        while ((1 << w) <= (int)maxc[j] + 1)
            ++w;
        if (bits + w > 32)
            return false;
        L.shift[j] = (uint8_t)bits;
        L.width[j] = (uint8_t)w;
        L.maxc[j] = maxc[j];
        L.amax[j] = maxc[j];
        bits += w;
    }
    finish_masks(&L);
    *out = L;
    return true;
}

Fusion make_fusion(const nhq_weights &w, const AttrLayout &L) {
    Fusion f;
    f.mode = w.mode;
    f.wv = w.w_v;
    f.wl = w.w_l;
    f.m = L.m;
    f.hi = L.hi;
    f.lo = L.lo;
    f.wild = 0;
    for (int j = 0; j < kMaxAttr; ++j) {
        f.shift[j] = L.shift[j];
        f.maxc[j] = L.maxc[j];
        f.amax[j] = L.amax[j];
    }
    return f;
}

Fusion make_fusion(const nhq_weights &w, int m) { return make_fusion(w, byte_layout(m)); }

}  // namespace nhq
