// Internal declarations shared by the translation units of libpasta.
// Not installed; the public boundary is include/pasta.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "pasta.h"

namespace pasta {

constexpr int kMaxOrder = PASTA_MAX_ORDER;
constexpr uint32_t kNoRow = 0xFFFFFFFFu;  // no open segment (indices are < 2^32 - 1)
constexpr uint64_t kPadEntries = 1024;    // stored arrays are padded to this multiple

// ---------------------------------------------------------------- errors ---

void set_error(const char *fmt, ...);
pasta_status cuda_fail(cudaError_t e, const char *where);

// Upper bound on the thread blocks of one MTTKRP / CP-loss launch
// (pasta_set_grid_cap; 0 = none), and `blocks` limited by it.
int grid_cap();
inline unsigned long long apply_grid_cap(unsigned long long blocks) {
    const int c = grid_cap();
    return (c > 0 && blocks > (unsigned long long)c) ? (unsigned long long)c : blocks;
}

// The library's device buffers go through these (pasta_set_allocator).
cudaError_t dev_malloc(void **p, size_t bytes, cudaStream_t stream);
void dev_free(void *p);

#define PASTA_CUDA(call)                                         \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return ::pasta::cuda_fail(e_, #call); \
    } while (0)

// ----------------------------------------------------------------- handle ---

// One stored copy of the tensor: SoA, every array padded to kPadEntries and
// 256-byte aligned inside one allocation.
struct StoredCopy {
    uint32_t *idx[kMaxOrder] = {};
    float *val = nullptr;
    uint32_t *perm = nullptr;  // sorted position -> creation-order entry (sorted copies)
    bool perm_ready = false;   // perm computed (built on request when the sort did not need it)
    void *block = nullptr;     // the allocation holding all arrays
    bool present = false;
};

// Mode-n fibers (the preprocessing of Algorithms 4 and 5): the stored
// entries that share every index but i_n.  They are contiguous in the
// mode-(n+1) sorted copy, whose key ends with mode n.
struct FiberTable {
    uint64_t nfibs = 0;
    uint32_t *fid = nullptr;             // per entry of that copy: its fiber (padded to nnz_pad)
    uint32_t *coords[kMaxOrder] = {};    // nfibs each: indices in modes n+1, ..., n-1 (cyclic)
    void *block = nullptr;               // fid
    void *cblock = nullptr;              // coords
    bool present = false;
};

// HiCOO copy (hicoo.cu): blocks of 2^bits cells per mode, one copy for
// every mode.
constexpr uint32_t kHTile = 512;  // entries per work tile of the HiCOO MTTKRP
struct HicooCopy {
    int bits = 0;
    uint64_t nb = 0;                     // nonempty blocks
    uint64_t ntiles = 0;                 // kHTile-entry tiles
    uint32_t *bptr = nullptr;            // nb + 1: first entry of each block, then nnz
    uint32_t *binds[kMaxOrder] = {};     // nb each: block coordinates
    uint8_t *einds[kMaxOrder] = {};      // per entry (padded): offset inside the block
    float *val = nullptr;                // per entry (padded)
    uint32_t *tile_block = nullptr;      // ntiles: block holding each tile's first entry
    void *block = nullptr;               // einds, val
    void *bblock = nullptr;              // bptr, binds, tile_block
    bool present = false;
};

}  // namespace pasta

struct pasta_coo_s {
    int order = 0;
    uint64_t dims[PASTA_MAX_ORDER] = {};
    uint64_t nnz = 0;
    uint64_t nnz_pad = 0;
    int device = 0;
    int num_sms = 0;
    pasta::StoredCopy orig;
    pasta::StoredCopy sorted[PASTA_MAX_ORDER];
    double *partials = nullptr;  // per-block FP64 partial sums of the loss
    int partials_cap = 0;
    double *als_normsq = nullptr;  // CP-ALS: sum of squared values (device), computed once
    void *scratch = nullptr;       // grow-only scratch (handle_scratch)
    size_t scratch_bytes = 0;
    pasta::FiberTable fibers[PASTA_MAX_ORDER];  // per mode, built by pasta_coo_fibers
    pasta::HicooCopy hicoo;                     // built by pasta_coo_hicoo
};

namespace pasta {
// At least `bytes` of the handle's scratch (see api.cu); PASTA_ERR_NOMEM on failure.
pasta_status handle_scratch(pasta_coo_s *X, size_t bytes, void **out);
// New handle from device coordinates (and values unless d_val is NULL); see api.cu.
pasta_status make_handle(pasta_coo *out, int order, const uint64_t *dims, uint64_t nnz,
                         const uint32_t *const *d_idx, const float *d_val, unsigned flags,
                         void *stream);
}  // namespace pasta

namespace pasta {

// Read-only description of one stored copy, passed by value to kernels.
struct CooView {
    const uint32_t *idx[kMaxOrder];
    const float *val;
    uint64_t nnz;
    int order;
};

CooView view_of(const pasta_coo_s *X, const StoredCopy &c);

// --------------------------------------------------------- lane geometry ---
//
// Work is spread warp-wide with the lanes across the rank: a factor row of R
// elements is cut into S "slots" of VEC elements (16 bytes on the fast path).
// L = min(32, next_pow2(S)) lanes serve one entry and each lane owns J =
// ceil(S / L) slots, so a warp works on G = 32 / L entries at a time, one per
// lane group.  Each lane group walks a contiguous run ("tile") of the stream.
struct Geometry {
    int vec;     // elements per slot
    int slots;   // S
    int L;       // lanes per entry (power of two)
    int lshift;  // log2(L)
    int J;       // slots per lane
    int tile;    // entries per lane-group tile (multiple of 4L)
};

Geometry make_geometry(int R, int vec, int elem_bytes);

size_t dtype_size(pasta_dtype t);

// ---------------------------------------------------------------- launchers --

pasta_status validate_coo(const pasta_coo_s *X, void *stream, uint64_t *bad_index,
                          uint64_t *bad_value);

pasta_status sort_copy(pasta_coo_s *X, int mode, cudaStream_t stream);
// Computes the mode's sorted-copy permutation if the sort left it out.
pasta_status ensure_perm(pasta_coo_s *X, int mode, cudaStream_t stream);
// The mode sort's stable LSD radix sort on other keys: `make` writes n keys
// (bits [0, used) significant) and n 32-bit payloads into the two device
// buffers it is given (the handle's scratch); the sorted payloads land in
// payload_out and *keys_sorted points at the sorted keys (in the scratch,
// valid until its next use).
using MakeKeysFn = pasta_status (*)(void *ctx, uint64_t *keys, uint32_t *payload, cudaStream_t s);
pasta_status radix_sort_keys(pasta_coo_s *X, uint64_t n, int used, MakeKeysFn make, void *ctx,
                             uint32_t *payload_out, const uint64_t **keys_sorted, cudaStream_t s);

// every_row_touched: every row of M has at least one entry (the TTM view,
// whose rows are fibers), so the streaming kernel's output needs zeros only
// where it adds atomically instead of a full clear.
pasta_status launch_mttkrp(const pasta_coo_s *X, const StoredCopy &c, const void *const *U,
                           pasta_dtype dt, int mode, int R, void *M, cudaStream_t stream,
                           bool every_row_touched = false);

// Streaming kernels (stream.cu and its per-kind units): one launch over a stored copy with the modes
// rotated so that position 0 is the copy's sorted mode.
struct StreamLaunch {
    int order = 0;
    int R = 0;
    pasta_dtype dtype = PASTA_F32;
    const uint32_t *idx[kMaxOrder] = {};  // by position
    const void *U[kMaxOrder] = {};        // by position
    const float *val = nullptr;
    float *out = nullptr;           // MTTKRP: M; loss bwd: G of position 0; loss fwd: residuals or null
    double *partials = nullptr;     // loss fwd
    const double *gscale = nullptr; // loss bwd
    uint64_t nnz = 0;
    int num_sms = 0;
    int max_blocks = 0;          // 0 = no cap
    int *blocks_used = nullptr;  // optional
    // MTTKRP whose every output row has an entry (the TTM view): instead of
    // a cleared output, zero only the rows open at a group-tile end, the
    // ones the kernel adds into atomically
    bool zero_tile_end_rows = false;
};
// True when the streaming kernels cover this case (see stream.cu); the loss
// kinds need order >= 3, MTTKRP (min_order 2) also takes order 2.
bool stream_supported(pasta_dtype dt, int order, int R, const void *const *U, int skip,
                      const void *out, int min_order = 3);
// kind: 0 MTTKRP, 1 loss forward, 2 loss backward (one mode)
pasta_status launch_stream(int kind, const StreamLaunch &l, cudaStream_t s);

// Loss forward over an arbitrary stored copy; `rot` is the copy's sorted mode
// (0 for the creation-order copy); `partials` must hold at least
// `partials_cap` doubles (the grid is capped to it).
pasta_status launch_cp_loss_fwd(const CooView &v, int rot, int num_sms, const void *const *U,
                                pasta_dtype dt, int R, double *loss, void *resid,
                                double *partials, int partials_cap, cudaStream_t stream);

// seg_mode: >= 0 one pass over that sorted copy, -1 one pass over the
// creation-order copy, -2 one pass per mode over each mode's sorted copy.
pasta_status launch_cp_loss_bwd(const pasta_coo_s *X, int seg_mode, const void *const *U,
                                pasta_dtype dt, int R, const double *gscale, void *const *G,
                                cudaStream_t stream);

// Loss and every factor's gradient (one pass per mode over its sorted copy;
// the first pass also sums the loss).  All sorted copies must exist.
pasta_status launch_cp_loss_fwd_bwd(const pasta_coo_s *X, const void *const *U, pasta_dtype dt,
                                    int R, double *loss, const double *gscale, void *const *G,
                                    cudaStream_t stream);

// Up to max_sweeps CP-ALS sweeps (cp_als.cu); arguments checked by the
// caller.  fit: device double for the last sweep's fit, or NULL; h_fits:
// host array of max_sweeps fits, or NULL; stops early once two consecutive
// fits differ by less than tol (tol >= 0, with h_fits); *h_sweeps = sweeps
// completed.  Synchronises `stream` once per sweep.
pasta_status run_cp_als(pasta_coo_s *X, float *const *U, int R, int max_sweeps, double tol, double *lambda,
                        double *fit, double *h_fits, int *h_sweeps, cudaStream_t stream);

// TEW-eq / TS (tew.cu): coordinate equality of two creation-order copies
// (synchronises `stream`), and z = x op y (y == NULL: z = x op s) over n_pad
// padded values.
pasta_status same_coordinates(const pasta_coo_s *X, const pasta_coo_s *Y, cudaStream_t stream,
                              bool *same);
pasta_status launch_elementwise(const float *x, const float *y, double s, float *z, uint64_t n_pad,
                                int op, int num_sms, cudaStream_t stream);

// Fiber tables and mode-n products (fibers.cu).
pasta_status build_fibers(pasta_coo_s *X, int mode, cudaStream_t stream);
void free_fibers(pasta::FiberTable &F);
pasta_status launch_ttm(pasta_coo_s *X, int mode, const void *U, pasta_dtype dt, int R, void *Y,
                        cudaStream_t stream);

// HiCOO copy and its MTTKRP (hicoo.cu).
pasta_status build_hicoo(pasta_coo_s *X, int bits, cudaStream_t stream);
void free_hicoo(HicooCopy &H);
pasta_status launch_hicoo_mttkrp(pasta_coo_s *X, const void *const *U, pasta_dtype dt, int mode, int R,
                                 void *M, cudaStream_t stream);

pasta_status launch_convert(const void *src, pasta_dtype st, void *dst, pasta_dtype dt,
                            uint64_t n, const double *scale, cudaStream_t stream);

// ------------------------------------------------------ device primitives ---

template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

// L2 policy for data streamed once (the COO arrays).
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 16-byte streaming load of read-only data: no L1 allocation, evict-first in L2.
__device__ __forceinline__ uint4 ld_stream_u4(const uint32_t *p, uint64_t pol) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p), "l"(pol));
    return r;
}

__device__ __forceinline__ float4 ld_stream_f4(const float *p, uint64_t pol) {
    float4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(p), "l"(pol));
    return r;
}

template <int Q> __device__ __forceinline__ uint32_t comp(const uint4 &v) {
    return Q == 0 ? v.x : Q == 1 ? v.y : Q == 2 ? v.z : v.w;
}
template <int Q> __device__ __forceinline__ float compf(const float4 &v) {
    return Q == 0 ? v.x : Q == 1 ? v.y : Q == 2 ? v.z : v.w;
}

// Load VEC consecutive factor elements (one slot) and widen to the
// accumulation type.  The fast-path forms are 16-byte vector loads through
// the read-only path.
template <typename T, int VEC> struct RowLoad;

template <> struct RowLoad<float, 4> {
    __device__ __forceinline__ static void run(const float *p, float (&o)[4]) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <> struct RowLoad<float, 1> {
    __device__ __forceinline__ static void run(const float *p, float (&o)[1]) { o[0] = __ldg(p); }
};
template <> struct RowLoad<__nv_bfloat16, 8> {
    __device__ __forceinline__ static void run(const __nv_bfloat16 *p, float (&o)[8]) {
        uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&w[i]);
            float2 f = __bfloat1622float2(h);
            o[2 * i] = f.x; o[2 * i + 1] = f.y;
        }
    }
};
template <> struct RowLoad<__nv_bfloat16, 1> {
    __device__ __forceinline__ static void run(const __nv_bfloat16 *p, float (&o)[1]) {
        o[0] = __bfloat162float(__ldg(p));
    }
};
template <> struct RowLoad<__half, 8> {
    __device__ __forceinline__ static void run(const __half *p, float (&o)[8]) {
        uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h = *reinterpret_cast<const __half2 *>(&w[i]);
            float2 f = __half22float2(h);
            o[2 * i] = f.x; o[2 * i + 1] = f.y;
        }
    }
};
template <> struct RowLoad<__half, 1> {
    __device__ __forceinline__ static void run(const __half *p, float (&o)[1]) {
        o[0] = __half2float(__ldg(p));
    }
};
template <> struct RowLoad<double, 2> {
    __device__ __forceinline__ static void run(const double *p, double (&o)[2]) {
        double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        o[0] = v.x; o[1] = v.y;
    }
};
template <> struct RowLoad<double, 1> {
    __device__ __forceinline__ static void run(const double *p, double (&o)[1]) { o[0] = __ldg(p); }
};

// Split form of RowLoad for software pipelining: load_raw issues the load
// (16 bytes on the fast path, kept as raw bits so a pending load costs four
// registers whatever the element type), widen converts after it lands.
template <typename T, int VEC> struct Raw { using type = uint4; };
template <typename T> struct Raw<T, 1> { using type = T; };

template <typename T, int VEC>
__device__ __forceinline__ typename Raw<T, VEC>::type load_raw(const T *p) {
    if constexpr (VEC == 1)
        return __ldg(p);
    else
        return __ldg(reinterpret_cast<const uint4 *>(p));
}

template <typename T, int VEC>
__device__ __forceinline__ void widen(const typename Raw<T, VEC>::type &r,
                                      typename AccOf<T>::type (&o)[VEC]) {
    if constexpr (VEC == 1) {
        if constexpr (std::is_same<T, __nv_bfloat16>::value)
            o[0] = __bfloat162float(r);
        else if constexpr (std::is_same<T, __half>::value)
            o[0] = __half2float(r);
        else
            o[0] = r;
    } else if constexpr (std::is_same<T, float>::value) {
        o[0] = __uint_as_float(r.x); o[1] = __uint_as_float(r.y);
        o[2] = __uint_as_float(r.z); o[3] = __uint_as_float(r.w);
    } else if constexpr (std::is_same<T, double>::value) {
        o[0] = __hiloint2double((int)r.y, (int)r.x);
        o[1] = __hiloint2double((int)r.w, (int)r.z);
    } else {
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float2 f;
            if constexpr (std::is_same<T, __nv_bfloat16>::value)
                f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&w[i]));
            else
                f = __half22float2(*reinterpret_cast<const __half2 *>(&w[i]));
            o[2 * i] = f.x; o[2 * i + 1] = f.y;
        }
    }
}

// Add VEC accumulators into global memory without reading the old value.
// The 4-wide FP32 form is one red.global.add.v4.f32 (16-byte aligned).
template <typename A, int VEC> struct RedAdd;
template <> struct RedAdd<float, 4> {
    __device__ __forceinline__ static void run(float *d, const float (&a)[4]) {
        asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(d), "f"(a[0]), "f"(a[1]),
                     "f"(a[2]), "f"(a[3]));
    }
};
template <> struct RedAdd<float, 8> {
    __device__ __forceinline__ static void run(float *d, const float (&a)[8]) {
        asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(d), "f"(a[0]), "f"(a[1]),
                     "f"(a[2]), "f"(a[3]));
        asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(d + 4), "f"(a[4]),
                     "f"(a[5]), "f"(a[6]), "f"(a[7]));
    }
};
template <> struct RedAdd<float, 1> {
    __device__ __forceinline__ static void run(float *d, const float (&a)[1]) {
        asm volatile("red.global.add.f32 [%0], %1;" ::"l"(d), "f"(a[0]));
    }
};
template <> struct RedAdd<double, 2> {
    __device__ __forceinline__ static void run(double *d, const double (&a)[2]) {
        asm volatile("red.global.add.f64 [%0], %1;" ::"l"(d), "d"(a[0]));
        asm volatile("red.global.add.f64 [%0], %1;" ::"l"(d + 1), "d"(a[1]));
    }
};
template <> struct RedAdd<double, 1> {
    __device__ __forceinline__ static void run(double *d, const double (&a)[1]) {
        asm volatile("red.global.add.f64 [%0], %1;" ::"l"(d), "d"(a[0]));
    }
};

// Plain (non-atomic) store of VEC accumulators.
template <typename A, int VEC> struct Store;
template <> struct Store<float, 4> {
    __device__ __forceinline__ static void run(float *d, const float (&a)[4]) {
        asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(d), "f"(a[0]), "f"(a[1]),
                     "f"(a[2]), "f"(a[3]));
    }
};
template <> struct Store<float, 8> {
    __device__ __forceinline__ static void run(float *d, const float (&a)[8]) {
        asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(d), "f"(a[0]), "f"(a[1]),
                     "f"(a[2]), "f"(a[3]));
        asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(d + 4), "f"(a[4]), "f"(a[5]),
                     "f"(a[6]), "f"(a[7]));
    }
};
template <> struct Store<float, 1> {
    __device__ __forceinline__ static void run(float *d, const float (&a)[1]) {
        asm volatile("st.global.f32 [%0], %1;" ::"l"(d), "f"(a[0]));
    }
};
template <> struct Store<double, 2> {
    __device__ __forceinline__ static void run(double *d, const double (&a)[2]) {
        asm volatile("st.global.v2.f64 [%0], {%1,%2};" ::"l"(d), "d"(a[0]), "d"(a[1]));
    }
};
template <> struct Store<double, 1> {
    __device__ __forceinline__ static void run(double *d, const double (&a)[1]) {
        asm volatile("st.global.f64 [%0], %1;" ::"l"(d), "d"(a[0]));
    }
};

}  // namespace pasta
