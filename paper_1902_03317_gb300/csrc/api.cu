// C ABI of libpasta (include/pasta.h): argument checking, ownership of the
// stored copies, the bounds/finiteness scan, and dispatch to the kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <new>

#include "host_copy.cuh"
#include "pasta_internal.cuh"
#include "stream_kernels.cuh"

namespace pasta {

namespace {
thread_local char g_err[512] = "";
constexpr int kPartialsCap = 4096;
std::atomic<int> g_grid_cap{0};
}  // namespace

int grid_cap() { return g_grid_cap.load(std::memory_order_relaxed); }

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

pasta_status cuda_fail(cudaError_t e, const char *where) {
    set_error("%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? PASTA_ERR_NOMEM : PASTA_ERR_CUDA;
}

// Device buffers: cudaMalloc/cudaFree unless the caller installed an
// allocator (pasta_set_allocator).  The number of live blocks guards against
// swapping allocators while blocks of the old one are held.
namespace {
std::mutex g_alloc_mu;
pasta_alloc_fn g_alloc = nullptr;
pasta_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;
std::atomic<long long> g_live{0};
}  // namespace

cudaError_t dev_malloc(void **p, size_t bytes, cudaStream_t s) {
    pasta_alloc_fn a;
    void *ctx;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        a = g_alloc;
        ctx = g_alloc_ctx;
    }
    cudaError_t e = cudaSuccess;
    if (!a) {
        e = cudaMalloc(p, bytes);
    } else {
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e == cudaSuccess) {
            *p = a(bytes, dev, static_cast<void *>(s), ctx);
            if (!*p) e = cudaErrorMemoryAllocation;
            else if ((reinterpret_cast<uintptr_t>(*p) & 255u) != 0) {
                pasta_free_fn f;
                {
                    std::lock_guard<std::mutex> lock(g_alloc_mu);
                    f = g_free;
                }
                if (f) f(*p, ctx);
                *p = nullptr;
                e = cudaErrorMisalignedAddress;
            }
        }
    }
    if (e == cudaSuccess) ++g_live;
    return e;
}

void dev_free(void *p) {
    if (!p) return;
    pasta_free_fn f;
    void *ctx;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        f = g_free;
        ctx = g_alloc_ctx;
    }
    if (f)
        f(p, ctx);
    else
        cudaFree(p);
    --g_live;
}

// Scratch of one handle (sort keys and histograms, CP-ALS buffers): one
// plain device allocation that only grows, kept until pasta_coo_destroy, so
// successive sorts and sweeps on a handle reuse it.  Growing it waits for the
// device.  Calls on one handle are stream-ordered, so its users never
// overlap.
pasta_status handle_scratch(pasta_coo_s *X, size_t bytes, void **out) {
    if (bytes > X->scratch_bytes) {
        if (X->scratch) {
            cudaDeviceSynchronize();  // kernels may still use the old buffer
            dev_free(X->scratch);
        }
        X->scratch = nullptr;
        X->scratch_bytes = 0;
        const size_t grow = (bytes + ((size_t)1 << 20) - 1) & ~(((size_t)1 << 20) - 1);
        cudaError_t e = dev_malloc(&X->scratch, grow, 0);
        if (e != cudaSuccess) {
            X->scratch = nullptr;
            cudaGetLastError();
            set_error("cudaMalloc of %zu bytes of scratch failed", grow);
            return PASTA_ERR_NOMEM;
        }
        X->scratch_bytes = grow;
    }
    *out = X->scratch;
    return PASTA_OK;
}

size_t dtype_size(pasta_dtype t) {
    switch (t) {
        case PASTA_F32: return 4;
        case PASTA_BF16: return 2;
        case PASTA_F16: return 2;
        case PASTA_F64: return 8;
    }
    return 0;
}

Geometry make_geometry(int R, int vec, int elem_bytes) {
    (void)elem_bytes;
    Geometry g{};
    g.vec = vec;
    g.slots = (R + vec - 1) / vec;
    int L = 1, sh = 0;
    while (L < g.slots && L < 32) {
        L <<= 1;
        ++sh;
    }
    g.L = L;
    g.lshift = sh;
    g.J = (g.slots + L - 1) / L;
    g.tile = std::max(4 * L, 512);
    return g;
}

CooView view_of(const pasta_coo_s *X, const StoredCopy &c) {
    CooView v{};
    for (int k = 0; k < X->order; ++k) v.idx[k] = c.idx[k];
    v.val = c.val;
    v.nnz = X->nnz;
    v.order = X->order;
    return v;
}

namespace {

bool ok_dtype(int t) { return t >= PASTA_F32 && t <= PASTA_F64; }

pasta_status alloc_copy(pasta_coo_s *X, StoredCopy &c, bool with_perm) {
    const size_t arr = (size_t)X->nnz_pad * 4;  // multiple of 4096 bytes
    const int narr = X->order + 1 + (with_perm ? 1 : 0);
    void *block = nullptr;
    cudaError_t e = dev_malloc(&block, arr * (size_t)narr, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc of %zu bytes for a stored copy failed", arr * (size_t)narr);
        return PASTA_ERR_NOMEM;
    }
    char *p = static_cast<char *>(block);
    for (int k = 0; k < X->order; ++k, p += arr) c.idx[k] = reinterpret_cast<uint32_t *>(p);
    c.val = reinterpret_cast<float *>(p);
    p += arr;
    c.perm = with_perm ? reinterpret_cast<uint32_t *>(p) : nullptr;
    c.block = block;
    return PASTA_OK;
}

void free_copy(StoredCopy &c) {
    if (c.block) dev_free(c.block);
    c = StoredCopy{};
}

// counts[0]: indices >= dims[k] (any mode); counts[1]: non-finite values.
__global__ void k_validate(CooView v, const uint64_t *dims_unused, unsigned long long *counts,
                           uint64_t d0, uint64_t d1, uint64_t d2, uint64_t d3, uint64_t d4,
                           uint64_t d5, uint64_t d6, uint64_t d7) {
    const uint64_t dims[kMaxOrder] = {d0, d1, d2, d3, d4, d5, d6, d7};
    unsigned long long bad_i = 0, bad_v = 0;
    for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < v.nnz;
         m += (uint64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < kMaxOrder; ++k)
            if (k < v.order && (uint64_t)v.idx[k][m] >= dims[k]) ++bad_i;
        if (!isfinite(v.val[m])) ++bad_v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        bad_i += __shfl_xor_sync(0xFFFFFFFFu, bad_i, o);
        bad_v += __shfl_xor_sync(0xFFFFFFFFu, bad_v, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad_i) atomicAdd(&counts[0], bad_i);
        if (bad_v) atomicAdd(&counts[1], bad_v);
    }
    (void)dims_unused;
}

}  // namespace

pasta_status validate_coo(const pasta_coo_s *X, void *stream, uint64_t *bad_index,
                          uint64_t *bad_value) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long *d_counts = nullptr;
    PASTA_CUDA(cudaMallocAsync((void **)&d_counts, 2 * sizeof(unsigned long long), s));
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(d_counts, 0, sizeof(h), s);
    if (e == cudaSuccess && X->nnz > 0) {
        const CooView v = view_of(X, X->orig);
        const int blocks = (int)std::min<uint64_t>((X->nnz + 255) / 256, (uint64_t)X->num_sms * 8);
        const uint64_t *d = X->dims;
        k_validate<<<blocks, 256, 0, s>>>(v, nullptr, d_counts, d[0], d[1], d[2], d[3], d[4], d[5],
                                          d[6], d[7]);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_counts, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(d_counts, s);
    if (e != cudaSuccess) return cuda_fail(e, "validate_coo");
    *bad_index = h[0];
    *bad_value = h[1];
    return PASTA_OK;
}

// n 32-bit words from src to dst, 16 bytes per access where possible; either
// side may be pinned host memory (the SMs then move the data over the host
// link).  Each thread keeps four 16-byte loads in flight, so a small grid
// covers the link's latency and leaves most SMs to kernels running beside it.
constexpr int kCopyThreads = 512;
constexpr int kCopyIlp = 4;
__global__ void __launch_bounds__(kCopyThreads) k_copy_words(const uint32_t *src, uint32_t *dst, uint64_t n) {
    const uint64_t n4 = n / 4;
    const uint64_t stride = (uint64_t)gridDim.x * kCopyThreads;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (uint64_t i = (uint64_t)blockIdx.x * kCopyThreads + threadIdx.x; i < n4; i += stride * kCopyIlp) {
        uint4 v[kCopyIlp];
#pragma unroll
        for (int k = 0; k < kCopyIlp; ++k)
            if (i + k * stride < n4) v[k] = s4[i + k * stride];
#pragma unroll
        for (int k = 0; k < kCopyIlp; ++k)
            if (i + k * stride < n4) d4[i + k * stride] = v[k];
    }
    for (uint64_t i = 4 * n4 + (uint64_t)blockIdx.x * kCopyThreads + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

// Device-side address of p if it is pinned host memory the device can reach,
// else NULL (device memory, pageable memory, or an unknown pointer).
const void *pinned_device_address(const void *p) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
        cudaGetLastError();  // clear the failed query
        return nullptr;
    }
    return pa.type == cudaMemoryTypeHost ? pa.devicePointer : nullptr;
}

// Copy of `bytes` on stream s.  Where one side is pinned host memory, both
// sides are 16-byte aligned and the size is whole words, a kernel moves the
// data (SM loads and stores over the host link) instead of the copy engine:
// measured on GB300, copy-engine transfers stalled for 20-90 ms about every
// 0.4 s in some runs while SM-driven ones at the same ~210 GB/s did not.
// Anything else goes through cudaMemcpyAsync (direction from the pointers).
cudaError_t copy_bytes(void *dst, const void *src, uint64_t bytes, int num_sms, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    const bool aligned = ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0;
    if (aligned && bytes % 4 == 0) {
        const void *hs = pinned_device_address(src);
        void *hd = const_cast<void *>(pinned_device_address(dst));
        if (hs || hd) {
            // one block per 8 SMs: 4 x 16 bytes in flight per thread is enough
            // for the host link's ~210 GB/s
            const uint64_t n = bytes / 4;
            const uint64_t want = (n / 4 + (uint64_t)kCopyThreads * kCopyIlp - 1) / ((uint64_t)kCopyThreads * kCopyIlp);
            const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)std::max(1, num_sms / 8)));
            k_copy_words<<<blocks, kCopyThreads, 0, s>>>(static_cast<const uint32_t *>(hs ? hs : src),
                                                        static_cast<uint32_t *>(hd ? hd : dst), n);
            return cudaGetLastError();
        }
    }
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s);
}

// make_handle flag (never accepted from callers): allocate and pad the
// creation-order copy but leave the copy-in and the validation to the caller.
constexpr unsigned kCreateDeferCopy = 1u << 30;

// Handle construction shared by pasta_coo_create and the operations that
// return a new tensor: copies the caller's (device or host) coordinates and, when
// d_val is not NULL, values into a new creation-order copy (zero padding);
// validates unless PASTA_CREATE_NO_VALIDATE.
pasta_status make_handle(pasta_coo *out, int order, const uint64_t *dims, uint64_t nnz,
                         const uint32_t *const *d_idx, const float *d_val, unsigned flags,
                         void *stream) {
    if (!out) {
        set_error("out is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (order < 2 || order > PASTA_MAX_ORDER || !dims) {
        set_error("order must be in [2, %d] and dims non-NULL", PASTA_MAX_ORDER);
        return PASTA_ERR_INVALID_ARG;
    }
    for (int k = 0; k < order; ++k) {
        if (dims[k] < 1 || dims[k] > 0xFFFFFFFFull) {
            set_error("dims[%d] = %llu out of [1, 2^32)", k, (unsigned long long)dims[k]);
            return PASTA_ERR_INVALID_ARG;
        }
    }
    if (nnz >= 0xFFFF0000ull) {
        set_error("nnz must be < 2^32 - 2^16");
        return PASTA_ERR_INVALID_ARG;
    }
    if (nnz > 0) {
        if (!d_idx) {
            set_error("d_idx is NULL");
            return PASTA_ERR_INVALID_ARG;
        }
        for (int k = 0; k < order; ++k)
            if (!d_idx[k]) {
                set_error("d_idx[%d] is NULL", k);
                return PASTA_ERR_INVALID_ARG;
            }
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    pasta_coo_s *X = new (std::nothrow) pasta_coo_s();
    if (!X) return PASTA_ERR_NOMEM;
    X->order = order;
    for (int k = 0; k < order; ++k) X->dims[k] = dims[k];
    X->nnz = nnz;
    X->nnz_pad = std::max<uint64_t>(kPadEntries, (nnz + kPadEntries - 1) / kPadEntries * kPadEntries);
    pasta_status st = PASTA_OK;
    cudaError_t e = cudaGetDevice(&X->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&X->num_sms, cudaDevAttrMultiProcessorCount, X->device);
    if (e != cudaSuccess) st = cuda_fail(e, "device query");
    if (st == PASTA_OK) st = alloc_copy(X, X->orig, false);
    if (st == PASTA_OK) {
        e = dev_malloc(reinterpret_cast<void **>(&X->partials), kPartialsCap * sizeof(double), s);
        if (e != cudaSuccess) st = cuda_fail(e, "allocation of partials");
        X->partials_cap = kPartialsCap;
    }
    if (st == PASTA_OK) {
        // only the padding past nnz needs zeros; the copies below fill the rest
        // (without values, the value array is zeroed whole)
        const size_t arr = (size_t)X->nnz_pad * 4;
        const size_t tail = (size_t)(X->nnz_pad - nnz) * 4;
        e = cudaSuccess;
        for (int k = 0; k < order && e == cudaSuccess; ++k)
            e = cudaMemsetAsync(X->orig.idx[k] + nnz, 0, tail, s);
        if (e == cudaSuccess)
            e = d_val ? cudaMemsetAsync(X->orig.val + nnz, 0, tail, s) : cudaMemsetAsync(X->orig.val, 0, arr, s);
        // the source may be device memory or host memory (copy_bytes); with
        // kCreateDeferCopy the caller copies (and validates) itself
        const bool copy = !(flags & kCreateDeferCopy);
        for (int k = 0; k < order && e == cudaSuccess && nnz > 0 && copy; ++k)
            e = copy_bytes(X->orig.idx[k], d_idx[k], nnz * 4, X->num_sms, s);
        if (e == cudaSuccess && nnz > 0 && d_val && copy)
            e = copy_bytes(X->orig.val, d_val, nnz * 4, X->num_sms, s);
        if (e != cudaSuccess) st = cuda_fail(e, "copy-in");
    }
    if (st == PASTA_OK) X->orig.present = true;
    if (st == PASTA_OK && !(flags & (PASTA_CREATE_NO_VALIDATE | kCreateDeferCopy))) {
        uint64_t bi = 0, bv = 0;
        st = validate_coo(X, stream, &bi, &bv);
        if (st == PASTA_OK && bi) {
            set_error("%llu index entries are >= their mode size", (unsigned long long)bi);
            st = PASTA_ERR_INDEX_OOB;
        } else if (st == PASTA_OK && bv) {
            set_error("%llu values are NaN or Inf", (unsigned long long)bv);
            st = PASTA_ERR_NONFINITE;
        }
    }
    if (st != PASTA_OK) {
        pasta_coo_destroy(X);
        return st;
    }
    *out = X;
    return PASTA_OK;
}

}  // namespace pasta

using namespace pasta;

extern "C" {

const char *pasta_status_str(pasta_status s) {
    switch (s) {
        case PASTA_OK: return "PASTA_OK";
        case PASTA_ERR_INVALID_ARG: return "PASTA_ERR_INVALID_ARG";
        case PASTA_ERR_ALIGNMENT: return "PASTA_ERR_ALIGNMENT";
        case PASTA_ERR_INDEX_OOB: return "PASTA_ERR_INDEX_OOB";
        case PASTA_ERR_NONFINITE: return "PASTA_ERR_NONFINITE";
        case PASTA_ERR_NOT_SORTED: return "PASTA_ERR_NOT_SORTED";
        case PASTA_ERR_NOMEM: return "PASTA_ERR_NOMEM";
        case PASTA_ERR_CUDA: return "PASTA_ERR_CUDA";
        case PASTA_ERR_UNSUPPORTED: return "PASTA_ERR_UNSUPPORTED";
        case PASTA_ERR_SINGULAR: return "PASTA_ERR_SINGULAR";
    }
    return "PASTA_ERR_UNKNOWN";
}

const char *pasta_last_error(void) { return g_err; }

int pasta_version(void) { return PASTA_VERSION; }

pasta_status pasta_coo_create(pasta_coo *out, int order, const uint64_t *dims, uint64_t nnz,
                              const uint32_t *const *d_idx, const float *d_val, unsigned flags,
                              void *stream) {
    if (flags & ~PASTA_CREATE_NO_VALIDATE) {
        set_error("unknown flags 0x%x", flags);
        return PASTA_ERR_INVALID_ARG;
    }
    if (nnz > 0 && !d_val) {
        set_error("d_val is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    return pasta::make_handle(out, order, dims, nnz, d_idx, d_val, flags, stream);
}

pasta_status pasta_coo_create_sorted(pasta_coo *out, int order, const uint64_t *dims, uint64_t nnz,
                                     const uint32_t *const *d_idx, const float *d_val, unsigned flags, int mode,
                                     void *stream) {
    if (flags & ~PASTA_CREATE_NO_VALIDATE) {
        set_error("unknown flags 0x%x", flags);
        return PASTA_ERR_INVALID_ARG;
    }
    if (!out) {
        set_error("out is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (order < 2 || order > PASTA_MAX_ORDER || !dims || mode < 0 || mode >= order) {
        set_error("order must be in [2, %d], dims non-NULL and mode in [0, order)", PASTA_MAX_ORDER);
        return PASTA_ERR_INVALID_ARG;
    }
    if (nnz > 0 && (!d_val || !d_idx)) {
        set_error("d_idx or d_val is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    // the overlapped path: large tensors in pinned host memory (16-byte
    // aligned) whose sort key holds every index
    int key_bits = 0;
    for (int k = 0; k < order; ++k) {
        uint64_t d = dims[k] ? dims[k] - 1 : 0;
        while (d) {
            ++key_bits;
            d >>= 1;
        }
    }
    bool overlap = nnz >= (1ull << 22) && key_bits <= 64;
    for (int k = 0; k < order && overlap; ++k)
        overlap = d_idx[k] && (reinterpret_cast<uintptr_t>(d_idx[k]) & 15) == 0 && pinned_device_address(d_idx[k]);
    overlap = overlap && (reinterpret_cast<uintptr_t>(d_val) & 15) == 0 && pinned_device_address(d_val);
    if (!overlap) {
        pasta_status st = pasta_coo_create(out, order, dims, nnz, d_idx, d_val, flags, stream);
        if (st != PASTA_OK) return st;
        st = pasta_coo_sort_by_mode(*out, mode, stream);
        if (st != PASTA_OK) {
            pasta_coo_destroy(*out);
            *out = nullptr;
        }
        return st;
    }
    pasta_status st = pasta::make_handle(out, order, dims, nnz, d_idx, d_val, flags | kCreateDeferCopy, stream);
    if (st != PASTA_OK) return st;
    pasta_coo_s *X = *out;
    StoredCopy &c = X->sorted[mode];
    st = alloc_copy(X, c, true);
    if (st == PASTA_OK)
        st = copy_in_and_sort(X, mode, reinterpret_cast<const void *const *>(d_idx), d_val,
                              static_cast<cudaStream_t>(stream));
    if (st == PASTA_OK) c.present = true;
    if (st == PASTA_OK && !(flags & PASTA_CREATE_NO_VALIDATE)) {
        uint64_t bi = 0, bv = 0;
        st = validate_coo(X, stream, &bi, &bv);
        if (st == PASTA_OK && bi) {
            set_error("%llu index entries are >= their mode size", (unsigned long long)bi);
            st = PASTA_ERR_INDEX_OOB;
        } else if (st == PASTA_OK && bv) {
            set_error("%llu values are NaN or Inf", (unsigned long long)bv);
            st = PASTA_ERR_NONFINITE;
        }
    }
    if (st != PASTA_OK) {
        pasta_coo_destroy(X);
        *out = nullptr;
    }
    return st;
}

pasta_status pasta_coo_destroy(pasta_coo X) {
    if (!X) return PASTA_OK;
    cudaDeviceSynchronize();
    free_copy(X->orig);
    for (int k = 0; k < PASTA_MAX_ORDER; ++k) free_copy(X->sorted[k]);
    for (int k = 0; k < PASTA_MAX_ORDER; ++k) free_fibers(X->fibers[k]);
    free_hicoo(X->hicoo);
    dev_free(X->partials);
    dev_free(X->als_normsq);
    dev_free(X->scratch);
    delete X;
    return PASTA_OK;
}

pasta_status pasta_coo_info(pasta_coo X, int *order, uint64_t *dims, uint64_t *nnz) {
    if (!X) {
        set_error("X is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    if (order) *order = X->order;
    if (dims)
        for (int k = 0; k < X->order; ++k) dims[k] = X->dims[k];
    if (nnz) *nnz = X->nnz;
    return PASTA_OK;
}

pasta_status pasta_coo_sort_by_mode(pasta_coo X, int mode, void *stream) {
    if (!X || mode < 0 || mode >= X->order) {
        set_error("bad handle or mode");
        return PASTA_ERR_INVALID_ARG;
    }
    StoredCopy &c = X->sorted[mode];
    if (c.present) return PASTA_OK;
    pasta_status st = alloc_copy(X, c, true);
    if (st != PASTA_OK) return st;
    st = sort_copy(X, mode, static_cast<cudaStream_t>(stream));
    if (st != PASTA_OK) {
        cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        free_copy(c);
        return st;
    }
    c.present = true;
    return PASTA_OK;
}

pasta_status pasta_coo_view(pasta_coo X, int mode, const uint32_t **d_idx, const float **d_val,
                            const uint32_t **d_perm) {
    if (!X || mode < -1 || mode >= X->order) {
        set_error("bad handle or mode");
        return PASTA_ERR_INVALID_ARG;
    }
    const StoredCopy &c = mode < 0 ? X->orig : X->sorted[mode];
    if (!c.present) {
        set_error("mode %d has no sorted copy", mode);
        return PASTA_ERR_NOT_SORTED;
    }
    if (d_idx)
        for (int k = 0; k < X->order; ++k) d_idx[k] = c.idx[k];
    if (d_val) *d_val = c.val;
    if (d_perm && mode >= 0 && !c.perm_ready) {
        // built on first request, on the legacy default stream, and waited for
        pasta_status st = ensure_perm(X, mode, nullptr);
        if (st != PASTA_OK) return st;
        PASTA_CUDA(cudaStreamSynchronize(nullptr));
    }
    if (d_perm) *d_perm = c.perm;
    return PASTA_OK;
}

pasta_status pasta_coo_copy_out(pasta_coo X, int mode, uint32_t *const *d_idx_out,
                                float *d_val_out, uint32_t *d_perm_out, void *stream) {
    if (!X || mode < -1 || mode >= X->order || (mode < 0 && d_perm_out)) {
        set_error("bad handle or mode");
        return PASTA_ERR_INVALID_ARG;
    }
    const StoredCopy &c = mode < 0 ? X->orig : X->sorted[mode];
    if (!c.present) {
        set_error("mode %d has no sorted copy", mode);
        return PASTA_ERR_NOT_SORTED;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)X->nnz * 4;
    if (bytes == 0) return PASTA_OK;
    if (d_idx_out)
        for (int k = 0; k < X->order; ++k)
            if (d_idx_out[k])
                PASTA_CUDA(cudaMemcpyAsync(d_idx_out[k], c.idx[k], bytes, cudaMemcpyDeviceToDevice, s));
    if (d_val_out) PASTA_CUDA(cudaMemcpyAsync(d_val_out, c.val, bytes, cudaMemcpyDeviceToDevice, s));
    if (d_perm_out) {
        pasta_status st = ensure_perm(X, mode, s);
        if (st != PASTA_OK) return st;
        PASTA_CUDA(cudaMemcpyAsync(d_perm_out, c.perm, bytes, cudaMemcpyDeviceToDevice, s));
    }
    return PASTA_OK;
}

static pasta_status check_factors(pasta_coo X, const void *const *d_U, int dt, int R, int skip) {
    if (!X) {
        set_error("X is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    if (!ok_dtype(dt)) {
        set_error("unknown dtype %d", dt);
        return PASTA_ERR_INVALID_ARG;
    }
    if (R < 1 || R > PASTA_MAX_RANK) {
        set_error("R = %d out of [1, %d]", R, PASTA_MAX_RANK);
        return PASTA_ERR_INVALID_ARG;
    }
    if (!d_U) {
        set_error("d_U is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    for (int k = 0; k < X->order; ++k)
        if (k != skip && !d_U[k]) {
            set_error("d_U[%d] is NULL", k);
            return PASTA_ERR_INVALID_ARG;
        }
    return PASTA_OK;
}

pasta_status pasta_mttkrp(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int mode,
                          int R, void *d_M, void *stream) {
    if (X && (mode < 0 || mode >= X->order)) {
        set_error("mode %d out of range", mode);
        return PASTA_ERR_INVALID_ARG;
    }
    pasta_status st = check_factors(X, d_U, u_dtype, R, mode);
    if (st != PASTA_OK) return st;
    if (!d_M) {
        set_error("d_M is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    if (!X->sorted[mode].present) {
        set_error("mode %d has no sorted copy (call pasta_coo_sort_by_mode)", mode);
        return PASTA_ERR_NOT_SORTED;
    }
    return launch_mttkrp(X, X->sorted[mode], d_U, u_dtype, mode, R, d_M,
                         static_cast<cudaStream_t>(stream));
}

pasta_status pasta_gather_probe(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int mode,
                                int R, float *d_sink, uint64_t sink_len, void *stream) {
    if (X && (mode < 0 || mode >= X->order)) {
        set_error("mode %d out of range", mode);
        return PASTA_ERR_INVALID_ARG;
    }
    pasta_status st = check_factors(X, d_U, u_dtype, R, mode);
    if (st != PASTA_OK) return st;
    if (!d_sink || sink_len < (uint64_t)stream::kThreads) {
        set_error("d_sink is NULL or holds fewer than %d floats", stream::kThreads);
        return PASTA_ERR_INVALID_ARG;
    }
    if (!X->sorted[mode].present) {
        set_error("mode %d has no sorted copy (call pasta_coo_sort_by_mode)", mode);
        return PASTA_ERR_NOT_SORTED;
    }
    if (!stream_supported(u_dtype, X->order, R, d_U, mode, d_sink, 2)) {
        set_error("the gather probe covers the streaming MTTKRP cases only");
        return PASTA_ERR_UNSUPPORTED;
    }
    if (X->nnz == 0) return PASTA_OK;
    const StoredCopy &c = X->sorted[mode];
    StreamLaunch l;
    l.order = X->order;
    l.R = R;
    l.dtype = u_dtype;
    for (int p = 0; p < X->order; ++p) {
        const int k = (mode + p) % X->order;
        l.idx[p] = c.idx[k];
        l.U[p] = d_U[k];
    }
    l.val = c.val;
    l.out = d_sink;
    l.nnz = X->nnz;
    l.num_sms = X->num_sms;
    l.max_blocks = (int)std::min<uint64_t>(sink_len / stream::kThreads, 1u << 30);
    return launch_stream(stream::kGather, l, static_cast<cudaStream_t>(stream));
}

pasta_status pasta_cp_loss_fwd(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int R,
                               int mode, double *d_loss, void *d_resid, void *stream) {
    pasta_status st = check_factors(X, d_U, u_dtype, R, -1);
    if (st != PASTA_OK) return st;
    if (mode < -1 || mode >= X->order || !d_loss) {
        set_error("bad mode or d_loss is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    const StoredCopy &c = mode < 0 ? X->orig : X->sorted[mode];
    if (!c.present) {
        set_error("mode %d has no sorted copy", mode);
        return PASTA_ERR_NOT_SORTED;
    }
    return launch_cp_loss_fwd(view_of(X, c), mode < 0 ? 0 : mode, X->num_sms, d_U, u_dtype, R,
                              d_loss, d_resid, X->partials, X->partials_cap,
                              static_cast<cudaStream_t>(stream));
}

pasta_status pasta_cp_loss_bwd(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int R,
                               int mode, const double *d_gscale, void *const *d_G,
                               void *stream) {
    pasta_status st = check_factors(X, d_U, u_dtype, R, -1);
    if (st != PASTA_OK) return st;
    if (mode < PASTA_BWD_PER_MODE || mode >= X->order || !d_G) {
        set_error("bad mode or d_G is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    for (int k = 0; k < X->order; ++k)
        if (!d_G[k]) {
            set_error("d_G[%d] is NULL", k);
            return PASTA_ERR_INVALID_ARG;
        }
    for (int k = 0; k < X->order; ++k) {
        const bool need = mode == PASTA_BWD_PER_MODE || mode == k;
        if (need && !X->sorted[k].present) {
            set_error("mode %d has no sorted copy", k);
            return PASTA_ERR_NOT_SORTED;
        }
    }
    return launch_cp_loss_bwd(X, mode, d_U, u_dtype, R, d_gscale, d_G,
                              static_cast<cudaStream_t>(stream));
}

pasta_status pasta_convert(const void *d_src, pasta_dtype src_dtype, void *d_dst,
                           pasta_dtype dst_dtype, uint64_t n, void *stream) {
    return pasta_convert_scaled(d_src, src_dtype, d_dst, dst_dtype, n, nullptr, stream);
}

pasta_status pasta_convert_scaled(const void *d_src, pasta_dtype src_dtype, void *d_dst,
                                  pasta_dtype dst_dtype, uint64_t n, const double *d_scale,
                                  void *stream) {
    if (!ok_dtype(src_dtype) || !ok_dtype(dst_dtype) || (n > 0 && (!d_src || !d_dst))) {
        set_error("bad dtype or NULL pointer");
        return PASTA_ERR_INVALID_ARG;
    }
    if (d_src == d_dst && src_dtype != dst_dtype) {
        set_error("in-place conversion needs equal source and destination types");
        return PASTA_ERR_INVALID_ARG;
    }
    return launch_convert(d_src, src_dtype, d_dst, dst_dtype, n, d_scale,
                          static_cast<cudaStream_t>(stream));
}

pasta_status pasta_cp_loss_fwd_bwd(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype,
                                   int R, double *d_loss, const double *d_gscale,
                                   void *const *d_G, void *stream) {
    pasta_status st = check_factors(X, d_U, u_dtype, R, -1);
    if (st != PASTA_OK) return st;
    if (!d_loss || !d_G) {
        set_error("d_loss or d_G is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    for (int k = 0; k < X->order; ++k) {
        if (!d_G[k]) {
            set_error("d_G[%d] is NULL", k);
            return PASTA_ERR_INVALID_ARG;
        }
        if (!X->sorted[k].present) {
            set_error("mode %d has no sorted copy", k);
            return PASTA_ERR_NOT_SORTED;
        }
    }
    return launch_cp_loss_fwd_bwd(X, d_U, u_dtype, R, d_loss, d_gscale, d_G,
                                  static_cast<cudaStream_t>(stream));
}

namespace {

pasta_status check_als(pasta_coo X, float *const *d_U, int R, const double *d_lambda) {
    pasta_status st = check_factors(X, reinterpret_cast<const void *const *>(d_U), PASTA_F32, R, -1);
    if (st != PASTA_OK) return st;
    if (R > PASTA_ALS_MAX_RANK) {
        set_error("CP-ALS supports R <= %d (got %d)", PASTA_ALS_MAX_RANK, R);
        return PASTA_ERR_UNSUPPORTED;
    }
    if (!d_lambda) {
        set_error("d_lambda is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    for (int k = 0; k < X->order; ++k)
        if (!X->sorted[k].present) {
            set_error("mode %d has no sorted copy", k);
            return PASTA_ERR_NOT_SORTED;
        }
    if (X->nnz == 0) {
        set_error("CP-ALS needs at least one stored entry");
        return PASTA_ERR_INVALID_ARG;
    }
    return PASTA_OK;
}

}  // namespace

pasta_status pasta_cp_als_sweep(pasta_coo X, float *const *d_U, int R, double *d_lambda,
                                double *d_fit, void *stream) {
    const pasta_status st = check_als(X, d_U, R, d_lambda);
    if (st != PASTA_OK) return st;
    return run_cp_als(X, d_U, R, 1, -1.0, d_lambda, d_fit, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

pasta_status pasta_cp_als(pasta_coo X, float *const *d_U, int R, int max_sweeps, double tol,
                          double *d_lambda, double *h_fits, int *h_sweeps, void *stream) {
    const pasta_status st = check_als(X, d_U, R, d_lambda);
    if (st != PASTA_OK) return st;
    if (max_sweeps < 1 || !h_fits || !h_sweeps || !(tol == tol)) {
        set_error("pasta_cp_als: need max_sweeps >= 1, h_fits, h_sweeps and a tolerance that is a number");
        return PASTA_ERR_INVALID_ARG;
    }
    return run_cp_als(X, d_U, R, max_sweeps, tol, d_lambda, nullptr, h_fits, h_sweeps,
                      static_cast<cudaStream_t>(stream));
}

// Output handle of TEW-eq / TS: a new handle with X's coordinates, or the
// caller's same-shaped handle with X's coordinates copied over its
// creation-order copy and its derived data (sorted copies, cached norm)
// dropped.  *created tells the caller whether to destroy it on failure.
static pasta_status elementwise_output(pasta_coo X, pasta_coo Y, pasta_coo *Z, cudaStream_t s,
                                       bool *created) {
    *created = false;
    if (!*Z) {
        pasta_status st = pasta::make_handle(Z, X->order, X->dims, X->nnz, X->orig.idx, nullptr,
                                             PASTA_CREATE_NO_VALIDATE, s);
        *created = (st == PASTA_OK);
        return st;
    }
    pasta_coo O = *Z;
    if (O == X || O == Y) {
        set_error("the output handle must differ from the inputs");
        return PASTA_ERR_INVALID_ARG;
    }
    if (O->order != X->order || O->nnz != X->nnz) {
        set_error("the output handle's order/nnz differ from the input's");
        return PASTA_ERR_INVALID_ARG;
    }
    for (int k = 0; k < X->order; ++k)
        if (O->dims[k] != X->dims[k]) {
            set_error("the output handle's dims differ from the input's");
            return PASTA_ERR_INVALID_ARG;
        }
    bool derived = O->als_normsq != nullptr;
    for (int k = 0; k < PASTA_MAX_ORDER; ++k)
        derived = derived || O->sorted[k].block != nullptr || O->fibers[k].present;
    if (derived) {
        cudaStreamSynchronize(s);  // earlier work on O may still read what is freed here
        for (int k = 0; k < PASTA_MAX_ORDER; ++k) free_copy(O->sorted[k]);
        for (int k = 0; k < PASTA_MAX_ORDER; ++k) free_fibers(O->fibers[k]);
        free_hicoo(O->hicoo);
        if (O->als_normsq) {
            dev_free(O->als_normsq);
            O->als_normsq = nullptr;
        }
    }
    for (int k = 0; k < X->order; ++k)
        PASTA_CUDA(cudaMemcpyAsync(O->orig.idx[k], X->orig.idx[k], (size_t)X->nnz_pad * 4,
                                   cudaMemcpyDeviceToDevice, s));
    return PASTA_OK;
}

static bool ok_op(int op) { return op >= PASTA_OP_ADD && op <= PASTA_OP_DIV; }

pasta_status pasta_tew_eq(pasta_coo X, pasta_coo Y, pasta_op op, pasta_coo *Z, void *stream) {
    if (!X || !Y || !Z || !ok_op(op)) {
        set_error("NULL handle/output or unknown op");
        return PASTA_ERR_INVALID_ARG;
    }
    if (X->order != Y->order || X->nnz != Y->nnz) {
        set_error("X and Y differ in order or nnz");
        return PASTA_ERR_INVALID_ARG;
    }
    for (int k = 0; k < X->order; ++k)
        if (X->dims[k] != Y->dims[k]) {
            set_error("X and Y differ in dims[%d]", k);
            return PASTA_ERR_INVALID_ARG;
        }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool same = false;
    pasta_status st = same_coordinates(X, Y, s, &same);
    if (st != PASTA_OK) return st;
    if (!same) {
        set_error("X and Y do not store the same coordinates in the same order");
        return PASTA_ERR_INVALID_ARG;
    }
    bool created = false;
    st = elementwise_output(X, Y, Z, s, &created);
    if (st == PASTA_OK)
        st = launch_elementwise(X->orig.val, Y->orig.val, 0.0, (*Z)->orig.val, X->nnz_pad, op, X->num_sms, s);
    if (st != PASTA_OK && created) {
        pasta_coo_destroy(*Z);
        *Z = nullptr;
    }
    return st;
}

pasta_status pasta_ts(pasta_coo X, pasta_op op, double sc, pasta_coo *Z, void *stream) {
    if (!X || !Z || !ok_op(op)) {
        set_error("NULL handle/output or unknown op");
        return PASTA_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bool created = false;
    pasta_status st = elementwise_output(X, nullptr, Z, s, &created);
    if (st == PASTA_OK)
        st = launch_elementwise(X->orig.val, nullptr, sc, (*Z)->orig.val, X->nnz_pad, op, X->num_sms, s);
    if (st != PASTA_OK && created) {
        pasta_coo_destroy(*Z);
        *Z = nullptr;
    }
    return st;
}

pasta_status pasta_coo_fibers(pasta_coo X, int mode, uint64_t *nfibs, void *stream) {
    if (!X || mode < 0 || mode >= X->order) {
        set_error("bad handle or mode");
        return PASTA_ERR_INVALID_ARG;
    }
    pasta_status st = build_fibers(X, mode, static_cast<cudaStream_t>(stream));
    if (st == PASTA_OK && nfibs) *nfibs = X->fibers[mode].nfibs;
    return st;
}

pasta_status pasta_coo_fiber_coords(pasta_coo X, int mode, uint32_t *const *d_coords, void *stream) {
    if (!X || mode < 0 || mode >= X->order || !d_coords) {
        set_error("bad handle, mode or d_coords");
        return PASTA_ERR_INVALID_ARG;
    }
    const pasta::FiberTable &F = X->fibers[mode];
    if (!F.present) {
        set_error("mode %d has no fiber table (pasta_coo_fibers)", mode);
        return PASTA_ERR_NOT_SORTED;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    for (int j = 0; j < X->order - 1; ++j) {
        if (!d_coords[j]) continue;
        if (F.nfibs)
            PASTA_CUDA(cudaMemcpyAsync(d_coords[j], F.coords[j], F.nfibs * 4, cudaMemcpyDeviceToDevice, s));
    }
    return PASTA_OK;
}

pasta_status pasta_ttm(pasta_coo X, int mode, const void *d_U, pasta_dtype u_dtype, int R, void *d_Y,
                       void *stream) {
    if (!X || mode < 0 || mode >= X->order || !d_U || !ok_dtype(u_dtype) || R < 1 ||
        R > PASTA_MAX_RANK) {
        set_error("bad handle, mode, U, dtype or R");
        return PASTA_ERR_INVALID_ARG;
    }
    if (!X->fibers[mode].present) {
        set_error("mode %d has no fiber table (pasta_coo_fibers)", mode);
        return PASTA_ERR_NOT_SORTED;
    }
    if (X->fibers[mode].nfibs == 0) return PASTA_OK;  // nothing to write; d_Y may be NULL
    if (!d_Y) {
        set_error("d_Y is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    return launch_ttm(X, mode, d_U, u_dtype, R, d_Y, static_cast<cudaStream_t>(stream));
}

pasta_status pasta_ttv(pasta_coo X, int mode, const void *d_v, pasta_dtype v_dtype, void *d_y,
                       void *stream) {
    return pasta_ttm(X, mode, d_v, v_dtype, 1, d_y, stream);
}

// A shallow copy of X whose stored copies start at entry lo and hold hi - lo
// entries (the arrays stay X's; nothing is owned).
static pasta_status range_view(pasta_coo X, uint64_t lo, uint64_t hi, pasta_coo_s *out) {
    if (lo > hi || hi > X->nnz) {
        set_error("range [%llu, %llu) outside [0, %llu)", (unsigned long long)lo, (unsigned long long)hi,
                  (unsigned long long)X->nnz);
        return PASTA_ERR_INVALID_ARG;
    }
    if (lo % 4 != 0) {
        set_error("range start %llu is not a multiple of 4 entries", (unsigned long long)lo);
        return PASTA_ERR_ALIGNMENT;
    }
    *out = *X;
    out->nnz = hi - lo;
    auto shift = [&](StoredCopy &c) {
        if (!c.present) return;
        for (int k = 0; k < X->order; ++k) c.idx[k] += lo;
        c.val += lo;
        if (c.perm) c.perm += lo;
    };
    shift(out->orig);
    for (int k = 0; k < X->order; ++k) shift(out->sorted[k]);
    out->hicoo = HicooCopy{};
    for (int k = 0; k < PASTA_MAX_ORDER; ++k) out->fibers[k] = FiberTable{};
    return PASTA_OK;
}

pasta_status pasta_mttkrp_range(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int mode, int R,
                                uint64_t lo, uint64_t hi, void *d_M, void *stream) {
    if (X && (mode < 0 || mode >= X->order)) {
        set_error("mode %d out of range", mode);
        return PASTA_ERR_INVALID_ARG;
    }
    pasta_status st = check_factors(X, d_U, u_dtype, R, mode);
    if (st != PASTA_OK) return st;
    if (!d_M) {
        set_error("d_M is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    if (!X->sorted[mode].present) {
        set_error("mode %d has no sorted copy (call pasta_coo_sort_by_mode)", mode);
        return PASTA_ERR_NOT_SORTED;
    }
    pasta_coo_s V;
    st = range_view(X, lo, hi, &V);
    if (st != PASTA_OK) return st;
    return launch_mttkrp(&V, V.sorted[mode], d_U, u_dtype, mode, R, d_M, static_cast<cudaStream_t>(stream));
}

pasta_status pasta_cp_loss_fwd_bwd_range(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int R,
                                         uint64_t lo, uint64_t hi, double *d_loss, const double *d_gscale,
                                         void *const *d_G, void *stream) {
    pasta_status st = check_factors(X, d_U, u_dtype, R, -1);
    if (st != PASTA_OK) return st;
    if (!d_loss || !d_G) {
        set_error("d_loss/d_G is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    for (int k = 0; k < X->order; ++k) {
        if (!d_G[k]) {
            set_error("d_G[%d] is NULL", k);
            return PASTA_ERR_INVALID_ARG;
        }
        if (!X->sorted[k].present) {
            set_error("mode %d has no sorted copy", k);
            return PASTA_ERR_NOT_SORTED;
        }
    }
    pasta_coo_s V;
    st = range_view(X, lo, hi, &V);
    if (st != PASTA_OK) return st;
    return launch_cp_loss_fwd_bwd(&V, d_U, u_dtype, R, d_loss, d_gscale, d_G, static_cast<cudaStream_t>(stream));
}

pasta_status pasta_coo_hicoo(pasta_coo X, int block_bits, uint64_t *nblocks, void *stream) {
    if (!X || block_bits < 1 || block_bits > 8) {
        set_error("NULL handle or block_bits out of [1, 8]");
        return PASTA_ERR_INVALID_ARG;
    }
    pasta_status st = build_hicoo(X, block_bits, static_cast<cudaStream_t>(stream));
    if (st == PASTA_OK && nblocks) *nblocks = X->hicoo.nb;
    return st;
}

pasta_status pasta_hicoo_copy_out(pasta_coo X, uint32_t *d_bptr, uint32_t *const *d_binds,
                                  uint8_t *const *d_einds, float *d_val, void *stream) {
    if (!X) {
        set_error("NULL handle");
        return PASTA_ERR_INVALID_ARG;
    }
    const HicooCopy &H = X->hicoo;
    if (!H.present) {
        set_error("no HiCOO copy (call pasta_coo_hicoo)");
        return PASTA_ERR_NOT_SORTED;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (d_bptr) PASTA_CUDA(cudaMemcpyAsync(d_bptr, H.bptr, (H.nb + 1) * 4, cudaMemcpyDeviceToDevice, s));
    for (int k = 0; k < X->order; ++k) {
        if (d_binds && d_binds[k] && H.nb)
            PASTA_CUDA(cudaMemcpyAsync(d_binds[k], H.binds[k], H.nb * 4, cudaMemcpyDeviceToDevice, s));
        if (d_einds && d_einds[k] && X->nnz)
            PASTA_CUDA(cudaMemcpyAsync(d_einds[k], H.einds[k], X->nnz, cudaMemcpyDeviceToDevice, s));
    }
    if (d_val && X->nnz) PASTA_CUDA(cudaMemcpyAsync(d_val, H.val, X->nnz * 4, cudaMemcpyDeviceToDevice, s));
    return PASTA_OK;
}

pasta_status pasta_hicoo_mttkrp(pasta_coo X, const void *const *d_U, pasta_dtype u_dtype, int mode, int R,
                                void *d_M, void *stream) {
    if (X && (mode < 0 || mode >= X->order)) {
        set_error("mode %d out of range", mode);
        return PASTA_ERR_INVALID_ARG;
    }
    pasta_status st = check_factors(X, d_U, u_dtype, R, mode);
    if (st != PASTA_OK) return st;
    if (!d_M) {
        set_error("d_M is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    if (!X->hicoo.present) {
        set_error("no HiCOO copy (call pasta_coo_hicoo)");
        return PASTA_ERR_NOT_SORTED;
    }
    return launch_hicoo_mttkrp(X, d_U, u_dtype, mode, R, d_M, static_cast<cudaStream_t>(stream));
}

pasta_status pasta_memcpy(void *dst, const void *src, uint64_t bytes, void *stream) {
    if (bytes == 0) return PASTA_OK;
    if (!dst || !src) {
        set_error("dst or src is NULL");
        return PASTA_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = copy_bytes(dst, src, bytes, sms, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "pasta_memcpy");
    return PASTA_OK;
}

pasta_status pasta_set_grid_cap(int max_blocks) {
    if (max_blocks < 0) {
        set_error("pasta_set_grid_cap: max_blocks %d < 0", max_blocks);
        return PASTA_ERR_INVALID_ARG;
    }
    pasta::g_grid_cap.store(max_blocks, std::memory_order_relaxed);
    return PASTA_OK;
}

int pasta_get_grid_cap(void) { return pasta::grid_cap(); }

pasta_status pasta_set_allocator(pasta_alloc_fn alloc, pasta_free_fn free_fn, void *ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        set_error("give both alloc and free, or neither");
        return PASTA_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(pasta::g_alloc_mu);
    if (pasta::g_live.load() != 0) {
        set_error("%lld library blocks are still held; destroy the handles first",
                  (long long)pasta::g_live.load());
        return PASTA_ERR_INVALID_ARG;
    }
    pasta::g_alloc = alloc;
    pasta::g_free = free_fn;
    pasta::g_alloc_ctx = ctx;
    return PASTA_OK;
}

}  // extern "C"
