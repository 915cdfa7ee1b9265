// Sparse CP least-squares loss and its gradient over the stored entries.
//
// The paper lists gradient-descent CPD among the methods whose bottleneck is
// MTTKRP (Sec. 2.2); its CP model is a sum of R rank-one terms.  Over the
// stored entries:
//     model(m) = sum_r prod_k U_k(i_k(m), r),   e(m) = val(m) - model(m),
//     loss     = 1/2 sum_m e(m)^2,
//     dloss/dU_k(i, r) = -sum_{m : i_k(m) = i} e(m) prod_{j != k} U_j(i_j(m), r),
// i.e. minus the mode-k MTTKRP of the residual tensor.
//
// Forward: the same warp geometry as MTTKRP (lanes across R, lane groups
// walking contiguous tiles); the model value is reduced across the lane
// group with xor shuffles, e^2 is summed in FP64 per block and the block
// partials are summed in a fixed order by a one-block kernel, so the loss is
// reproducible bit for bit for the same inputs and launch.
//
// Backward: one pass over the stream computes e(m) again and, for every mode,
// the leave-one-out product; the mode the stream is sorted by is reduced in
// registers along runs of equal index (plain stores inside a tile,
// red.global.add at tile edges), every other mode is added with 16-byte
// vector atomics.
#include <algorithm>
#include <type_traits>

#include "pasta_internal.cuh"

namespace pasta {
namespace {

constexpr int kThreads = 256;
constexpr unsigned FULL = 0xFFFFFFFFu;

template <typename T, int NM>
struct LossArgs {
    const uint32_t *idx[NM];  // position p: mode (rot + p) % order
    const T *U[NM];
    typename AccOf<T>::type *G[NM];
    const float *val;
    typename AccOf<T>::type *resid;  // forward only, optional
    double *partials;                // forward only
    const double *gscale;            // backward only, optional
    uint64_t nnz;
    int order;
    int seg;       // backward: position 0 is the sorted mode, reduced along runs
    int seg_only;  // backward: compute only position 0's gradient (no atomics)
    int R, S, L, lshift, tile;
};

template <int NM>
struct EntryIdx {
    uint32_t v[NM];
};

// Shared tile walk: calls body(m, ok, ci_q[], v) for every entry slot of the
// warp's tiles, with the entry's indices (positions 0..NM-1) and value
// broadcast to its lane group.  All lanes run the same trip counts, so the
// shuffles inside are always converged; `ok` marks real entries.
template <int NM, typename Args, typename Body>
__device__ __forceinline__ void walk_tiles(const Args &a, Body &body) {
    const uint64_t nnz = a.nnz;
    const int order = a.order, L = a.L, lshift = a.lshift, tile = a.tile;
    const int lane = threadIdx.x & 31;
    const int lig = lane & (L - 1);
    const int grp = lane >> lshift;
    const int G = 32 >> lshift;
    const int chunk = 4 * L;
    const uint64_t pol = policy_evict_first();
    const uint64_t warp_span = (uint64_t)tile * (uint64_t)G;
    const uint64_t nwt = (nnz + warp_span - 1) / warp_span;
    const uint64_t wpb = blockDim.x >> 5;
    for (uint64_t wt = (uint64_t)blockIdx.x * wpb + (threadIdx.x >> 5); wt < nwt;
         wt += (uint64_t)gridDim.x * wpb) {
        const uint64_t t0 = wt * warp_span + (uint64_t)grp * (uint64_t)tile;
        const uint64_t t1 = min(t0 + (uint64_t)tile, nnz);
        for (int c = 0; c < tile; c += chunk) {
            const uint64_t base = t0 + (uint64_t)c;
            if (!__any_sync(FULL, base < t1)) break;
            const uint64_t my = base + 4u * (uint64_t)lig;
            const bool ld = my < t1;
            uint32_t ci[NM][4];
            float cv[4];
#pragma unroll
            for (int k = 0; k < NM; ++k) {
                uint4 w = make_uint4(0u, 0u, 0u, 0u);
                if (ld && k < order) w = ld_stream_u4(a.idx[k] + my, pol);
                ci[k][0] = w.x; ci[k][1] = w.y; ci[k][2] = w.z; ci[k][3] = w.w;
            }
            {
                float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
                if (ld) w = ld_stream_f4(a.val + my, pol);
                cv[0] = w.x; cv[1] = w.y; cv[2] = w.z; cv[3] = w.w;
            }
            for (int src = 0; src < L; ++src) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint64_t m = base + 4u * (uint64_t)src + (uint64_t)q;
                    EntryIdx<NM> iq;
#pragma unroll
                    for (int k = 0; k < NM; ++k)
                        iq.v[k] = (k < order) ? __shfl_sync(FULL, ci[k][q], src, L) : 0u;
                    const float v = __shfl_sync(FULL, cv[q], src, L);
                    body(m, m < t1, iq, v);
                }
            }
        }
        body.tile_end();
    }
}

template <typename A>
__device__ __forceinline__ A group_sum(A x, int L) {
    for (int o = L >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o, L);
    return x;
}

// Lane-slot bookkeeping shared by the loss kernels: this lane owns slots
// lig + j*L (j < J) of the factor rows, VEC elements each.
template <int J>
struct Slots {
    int lig;
    int slot[J];
    bool act[J];
    __device__ __forceinline__ Slots(int L, int S) {
        lig = (threadIdx.x & 31) & (L - 1);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            slot[j] = lig + j * L;
            act[j] = slot[j] < S;
        }
    }
};

// Gather the factor rows of one entry (every mode) into u; rows of modes
// >= order and of absent entries stay 1.
template <typename T, int VEC, int J, int NM>
__device__ __forceinline__ void gather_rows(const LossArgs<T, NM> &a, const Slots<J> &sl, bool ok,
                                            const EntryIdx<NM> &iq,
                                            typename AccOf<T>::type (&u)[NM][J][VEC]) {
    using A = typename AccOf<T>::type;
#pragma unroll
    for (int k = 0; k < NM; ++k)
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int e = 0; e < VEC; ++e) u[k][j][e] = A(1);
    if (!ok) return;
#pragma unroll
    for (int k = 0; k < NM; ++k) {
        if (k >= a.order) continue;
        const T *row = a.U[k] + (uint64_t)iq.v[k] * (uint64_t)a.R;
#pragma unroll
        for (int j = 0; j < J; ++j)
            if (sl.act[j]) RowLoad<T, VEC>::run(row + sl.slot[j] * VEC, u[k][j]);
    }
}

// model(m) = sum over this lane group's slots of prod_k u[k], reduced across
// the L lanes of the group (every lane of the group gets the same value).
template <typename A, int VEC, int J, int NM>
__device__ __forceinline__ A model_value(const A (&u)[NM][J][VEC], const Slots<J> &sl, int L) {
    A part = A(0);
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
            A p = u[0][j][e];
#pragma unroll
            for (int k = 1; k < NM; ++k) p *= u[k][j][e];
            if (sl.act[j]) part += p;
        }
    return group_sum(part, L);
}

template <typename T, int VEC, int J, int NM>
struct FwdBody {
    using A = typename AccOf<T>::type;
    const LossArgs<T, NM> &a;
    Slots<J> sl;
    double sq;
    __device__ __forceinline__ FwdBody(const LossArgs<T, NM> &args)
        : a(args), sl(args.L, args.S), sq(0.0) {}
    __device__ __forceinline__ void operator()(uint64_t m, bool ok, const EntryIdx<NM> &iq,
                                               float v) {
        A u[NM][J][VEC];
        gather_rows<T, VEC, J, NM>(a, sl, ok, iq, u);
        const A model = model_value<A, VEC, J, NM>(u, sl, a.L);
        if (ok && sl.lig == 0) {
            const A e = A(v) - model;
            sq += (double)e * (double)e;
            if (a.resid) a.resid[m] = e;
        }
    }
    __device__ __forceinline__ void tile_end() {}
};

template <typename T, int VEC, int J, int NM>
__global__ void __launch_bounds__(kThreads) k_loss_fwd(const LossArgs<T, NM> a) {
    FwdBody<T, VEC, J, NM> body(a);
    walk_tiles<NM>(a, body);
    // Fixed-order block reduction of the FP64 partial sums.
    double sq = body.sq;
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(FULL, sq, o);
    __shared__ double ws[kThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
        a.partials[blockIdx.x] = s;
    }
}

// loss = 1/2 * sum of the block partials, summed in a fixed order.
__global__ void __launch_bounds__(256) k_loss_finalize(const double *partials, int n,
                                                       double *loss) {
    __shared__ double s[256];
    double x = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) x += partials[i];
    s[threadIdx.x] = x;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = 0.5 * s[0];
}

template <typename T, int VEC, int J, int NM>
struct BwdBody {
    using A = typename AccOf<T>::type;
    const LossArgs<T, NM> &a;
    Slots<J> sl;
    A g;
    A acc[J][VEC];
    uint32_t cur;
    bool first;

    __device__ __forceinline__ BwdBody(const LossArgs<T, NM> &args)
        : a(args), sl(args.L, args.S), cur(kNoRow), first(true) {
        g = a.gscale ? A(*a.gscale) : A(1);
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc[j][e] = A(0);
    }

    __device__ __forceinline__ void flush(uint32_t row, bool atomic) {
        A *dst = a.G[0] + (uint64_t)row * (uint64_t)a.R;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            if (!sl.act[j]) continue;
            if (atomic)
                RedAdd<A, VEC>::run(dst + sl.slot[j] * VEC, acc[j]);
            else
                Store<A, VEC>::run(dst + sl.slot[j] * VEC, acc[j]);
        }
    }

    __device__ __forceinline__ void operator()(uint64_t m, bool ok, const EntryIdx<NM> &iq,
                                               float v) {
        (void)m;
        A u[NM][J][VEC];
        gather_rows<T, VEC, J, NM>(a, sl, ok, iq, u);
        const A model = model_value<A, VEC, J, NM>(u, sl, a.L);
        if (!ok) return;
        const A w = -g * (A(v) - model);
#pragma unroll
        for (int k = 0; k < NM; ++k) {
            if (k >= a.order) continue;
            A t[J][VEC];  // w * prod_{q != k} u[q]
#pragma unroll
            for (int j = 0; j < J; ++j)
#pragma unroll
                for (int e = 0; e < VEC; ++e) {
                    A p = w;
#pragma unroll
                    for (int q = 0; q < NM; ++q)
                        if (q != k) p *= u[q][j][e];
                    t[j][e] = p;
                }
            if (k == 0 && a.seg) {
                if (iq.v[0] != cur) {
                    if (cur != kNoRow) {
                        flush(cur, first);
                        first = false;
                    }
                    cur = iq.v[0];
#pragma unroll
                    for (int j = 0; j < J; ++j)
#pragma unroll
                        for (int e = 0; e < VEC; ++e) acc[j][e] = t[j][e];
                } else {
#pragma unroll
                    for (int j = 0; j < J; ++j)
#pragma unroll
                        for (int e = 0; e < VEC; ++e) acc[j][e] += t[j][e];
                }
            } else if (!a.seg_only) {
                A *dst = a.G[k] + (uint64_t)iq.v[k] * (uint64_t)a.R;
#pragma unroll
                for (int j = 0; j < J; ++j)
                    if (sl.act[j]) RedAdd<A, VEC>::run(dst + sl.slot[j] * VEC, t[j]);
            }
        }
    }

    __device__ __forceinline__ void tile_end() {
        if (a.seg && cur != kNoRow) flush(cur, true);
        cur = kNoRow;
        first = true;
    }
};

template <typename T, int VEC, int J, int NM>
__global__ void __launch_bounds__(kThreads) k_loss_bwd(const LossArgs<T, NM> a) {
    BwdBody<T, VEC, J, NM> body(a);
    walk_tiles<NM>(a, body);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename T> constexpr pasta_dtype dtype_of();
template <> constexpr pasta_dtype dtype_of<float>() { return PASTA_F32; }
template <> constexpr pasta_dtype dtype_of<__nv_bfloat16>() { return PASTA_BF16; }
template <> constexpr pasta_dtype dtype_of<__half>() { return PASTA_F16; }
template <> constexpr pasta_dtype dtype_of<double>() { return PASTA_F64; }

template <typename T, int NM>
LossArgs<T, NM> make_args(const CooView &v, int rot, const void *const *U, void *const *G,
                          int R, const Geometry &g) {
    LossArgs<T, NM> a{};
    for (int p = 0; p < v.order && p < NM; ++p) {
        const int k = (rot + p) % v.order;
        a.idx[p] = v.idx[k];
        a.U[p] = static_cast<const T *>(U[k]);
        if (G) a.G[p] = static_cast<typename AccOf<T>::type *>(G[k]);
    }
    a.val = v.val;
    a.nnz = v.nnz;
    a.order = v.order;
    a.R = R;
    a.S = g.slots;
    a.L = g.L;
    a.lshift = g.lshift;
    a.tile = g.tile;
    return a;
}

template <typename K>
int grid_for(K kernel, uint64_t nnz, const Geometry &g, int num_sms, int cap) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const uint64_t G = 32u >> g.lshift;
    const uint64_t nwt = (nnz + (uint64_t)g.tile * G - 1) / ((uint64_t)g.tile * G);
    const uint64_t want = std::max<uint64_t>(1, (nwt + kThreads / 32 - 1) / (kThreads / 32));
    uint64_t b = std::min<uint64_t>(want, (uint64_t)num_sms * (uint64_t)per_sm);
    if (cap > 0) b = std::min<uint64_t>(b, (uint64_t)cap);
    return (int)apply_grid_cap(b);
}

template <typename T, int VEC, int J, int NM>
pasta_status fwd_run(const CooView &v, int num_sms, const void *const *U, int R,
                     const Geometry &g, double *loss, void *resid, double *partials, int cap,
                     cudaStream_t s) {
    using A = typename AccOf<T>::type;
    LossArgs<T, NM> a = make_args<T, NM>(v, 0, U, nullptr, R, g);
    a.resid = static_cast<A *>(resid);
    a.partials = partials;
    const int blocks = grid_for(k_loss_fwd<T, VEC, J, NM>, v.nnz, g, num_sms, cap);
    k_loss_fwd<T, VEC, J, NM><<<blocks, kThreads, 0, s>>>(a);
    PASTA_CUDA(cudaGetLastError());
    k_loss_finalize<<<1, 256, 0, s>>>(partials, blocks, loss);
    PASTA_CUDA(cudaGetLastError());
    return PASTA_OK;
}

template <typename T, int VEC, int J, int NM>
pasta_status bwd_run(const pasta_coo_s *X, int seg_mode, const void *const *U, int R,
                     const Geometry &g, const double *gscale, void *const *G, cudaStream_t s) {
    using A = typename AccOf<T>::type;
    for (int k = 0; k < X->order; ++k)
        PASTA_CUDA(cudaMemsetAsync(G[k], 0, (size_t)X->dims[k] * (size_t)R * sizeof(A), s));
    if (X->nnz == 0) return PASTA_OK;
    // seg_mode >= 0: one pass over that mode's sorted copy; -1: one pass over
    // the creation-order copy (atomics for every mode); -2: one pass per mode,
    // each over its own sorted copy, reducing only that mode's gradient.
    const int passes = seg_mode == -2 ? X->order : 1;
    for (int p = 0; p < passes; ++p) {
        const int mode = seg_mode == -2 ? p : seg_mode;
        const StoredCopy &c = mode < 0 ? X->orig : X->sorted[mode];
        const CooView v = view_of(X, c);
        if (seg_mode == -2 && stream_supported(dtype_of<T>(), X->order, R, U, -1, G[mode])) {
            StreamLaunch l;
            l.order = X->order;
            l.R = R;
            l.dtype = dtype_of<T>();
            for (int q = 0; q < X->order; ++q) {
                const int k = (mode + q) % X->order;
                l.idx[q] = v.idx[k];
                l.U[q] = U[k];
            }
            l.val = v.val;
            l.out = static_cast<float *>(G[mode]);
            l.gscale = gscale;
            l.nnz = v.nnz;
            l.num_sms = X->num_sms;
            pasta_status st = launch_stream(2, l, s);
            if (st != PASTA_OK) return st;
            continue;
        }
        LossArgs<T, NM> a = make_args<T, NM>(v, mode < 0 ? 0 : mode, U, G, R, g);
        a.gscale = gscale;
        a.seg = mode >= 0 ? 1 : 0;
        a.seg_only = seg_mode == -2 ? 1 : 0;
        const int blocks = grid_for(k_loss_bwd<T, VEC, J, NM>, v.nnz, g, X->num_sms, 0);
        k_loss_bwd<T, VEC, J, NM><<<blocks, kThreads, 0, s>>>(a);
        PASTA_CUDA(cudaGetLastError());
    }
    return PASTA_OK;
}

// Dispatch on element type, vector width, slots per lane and order.
template <template <typename, int, int, int> class Fn, typename... Args>
pasta_status dispatch(pasta_dtype dt, bool fast, int J, int order, Args &&...args) {
    if (!fast) {
        switch (dt) {
            case PASTA_F32: return Fn<float, 1, 8, 8>::run(args...);
            case PASTA_BF16: return Fn<__nv_bfloat16, 1, 8, 8>::run(args...);
            case PASTA_F16: return Fn<__half, 1, 8, 8>::run(args...);
            case PASTA_F64: return Fn<double, 1, 8, 8>::run(args...);
        }
        return PASTA_ERR_UNSUPPORTED;
    }
    switch (dt) {
        case PASTA_F32:
            if (J == 1) {
                if (order <= 3) return Fn<float, 4, 1, 3>::run(args...);
                if (order == 4) return Fn<float, 4, 1, 4>::run(args...);
                if (order == 5) return Fn<float, 4, 1, 5>::run(args...);
                return Fn<float, 4, 1, 8>::run(args...);
            }
            return Fn<float, 4, 2, 8>::run(args...);
        case PASTA_BF16:
            if (order <= 3) return Fn<__nv_bfloat16, 8, 1, 3>::run(args...);
            if (order == 4) return Fn<__nv_bfloat16, 8, 1, 4>::run(args...);
            if (order == 5) return Fn<__nv_bfloat16, 8, 1, 5>::run(args...);
            return Fn<__nv_bfloat16, 8, 1, 8>::run(args...);
        case PASTA_F16:
            if (order <= 3) return Fn<__half, 8, 1, 3>::run(args...);
            if (order == 4) return Fn<__half, 8, 1, 4>::run(args...);
            return Fn<__half, 8, 1, 8>::run(args...);
        case PASTA_F64:
            if (J == 1) return Fn<double, 2, 1, 8>::run(args...);
            if (J == 2) return Fn<double, 2, 2, 8>::run(args...);
            return Fn<double, 2, 4, 8>::run(args...);
    }
    return PASTA_ERR_UNSUPPORTED;
}

template <typename T, int VEC, int J, int NM>
struct FwdFn {
    template <typename... Args>
    static pasta_status run(Args &&...args) { return fwd_run<T, VEC, J, NM>(args...); }
};
template <typename T, int VEC, int J, int NM>
struct BwdFn {
    template <typename... Args>
    static pasta_status run(Args &&...args) { return bwd_run<T, VEC, J, NM>(args...); }
};

bool fast_path(pasta_dtype dt, int R, int order, const void *const *U, const void *const *G,
               const void *resid) {
    const int es = (int)dtype_size(dt);
    bool fast = ((R * es) % 16) == 0;
    for (int k = 0; k < order; ++k) {
        fast = fast && aligned16(U[k]);
        if (G) fast = fast && aligned16(G[k]);
    }
    (void)resid;
    return fast;
}

// ------------------------------------------------------------- convert ---

template <typename S, typename D>
__device__ __forceinline__ D cvt(S x);
template <> __device__ __forceinline__ float cvt<float, float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<float, __nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ __half cvt<float, __half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ double cvt<float, double>(float x) { return (double)x; }
template <> __device__ __forceinline__ float cvt<double, float>(double x) { return __double2float_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<double, __nv_bfloat16>(double x) { return __double2bfloat16(x); }
template <> __device__ __forceinline__ __half cvt<double, __half>(double x) { return __double2half(x); }
template <> __device__ __forceinline__ double cvt<double, double>(double x) { return x; }

template <typename S> __device__ __forceinline__ float widen(S x);
template <> __device__ __forceinline__ float widen<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <> __device__ __forceinline__ float widen<__half>(__half x) { return __half2float(x); }

// dst[i] = (D)(scale * src[i]) (scale = 1 when null), rounded to nearest
// even; FP32 arithmetic except for FP64 sources.
template <typename S, typename D>
__global__ void k_convert(const S *src, D *dst, uint64_t n, const double *scale) {
    const double sd = scale ? *scale : 1.0;
    const float sf = (float)sd;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if constexpr (std::is_same<S, double>::value) {
            dst[i] = cvt<double, D>(scale ? sd * src[i] : src[i]);
        } else {
            float v;
            if constexpr (std::is_same<S, float>::value)
                v = src[i];
            else
                v = widen<S>(src[i]);
            dst[i] = cvt<float, D>(scale ? sf * v : v);
        }
    }
}

template <typename S>
pasta_status convert_from(const S *src, void *dst, pasta_dtype dt, uint64_t n, cudaStream_t s,
                          int blocks, const double *sc) {
    switch (dt) {
        case PASTA_F32: k_convert<S, float><<<blocks, 256, 0, s>>>(src, (float *)dst, n, sc); break;
        case PASTA_BF16: k_convert<S, __nv_bfloat16><<<blocks, 256, 0, s>>>(src, (__nv_bfloat16 *)dst, n, sc); break;
        case PASTA_F16: k_convert<S, __half><<<blocks, 256, 0, s>>>(src, (__half *)dst, n, sc); break;
        case PASTA_F64: k_convert<S, double><<<blocks, 256, 0, s>>>(src, (double *)dst, n, sc); break;
        default: return PASTA_ERR_INVALID_ARG;
    }
    PASTA_CUDA(cudaGetLastError());
    return PASTA_OK;
}

}  // namespace

pasta_status launch_cp_loss_fwd(const CooView &v, int rot, int num_sms, const void *const *U,
                                pasta_dtype dt, int R, double *loss, void *resid,
                                double *partials, int cap, cudaStream_t s) {
    if (v.nnz == 0) {
        PASTA_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s));
        return PASTA_OK;
    }
    if (stream_supported(dt, v.order, R, U, -1, nullptr)) {
        StreamLaunch l;
        l.order = v.order;
        l.R = R;
        l.dtype = dt;
        for (int p = 0; p < v.order; ++p) {
            const int k = (rot + p) % v.order;
            l.idx[p] = v.idx[k];
            l.U[p] = U[k];
        }
        l.val = v.val;
        l.out = static_cast<float *>(resid);
        l.partials = partials;
        l.nnz = v.nnz;
        l.num_sms = num_sms;
        l.max_blocks = cap;
        int blocks = 0;
        l.blocks_used = &blocks;
        pasta_status st = launch_stream(1, l, s);
        if (st != PASTA_OK) return st;
        k_loss_finalize<<<1, 256, 0, s>>>(partials, blocks, loss);
        PASTA_CUDA(cudaGetLastError());
        return PASTA_OK;
    }
    const bool fast = fast_path(dt, R, v.order, U, nullptr, resid);
    const int es = (int)dtype_size(dt);
    const Geometry g = make_geometry(R, fast ? 16 / es : 1, es);
    return dispatch<FwdFn>(dt, fast, g.J, v.order, v, num_sms, U, R, g, loss, resid, partials,
                           cap, s);
}

pasta_status launch_cp_loss_bwd(const pasta_coo_s *X, int seg_mode, const void *const *U,
                                pasta_dtype dt, int R, const double *gscale, void *const *G,
                                cudaStream_t s) {
    const bool fast = fast_path(dt, R, X->order, U, G, nullptr);
    const int es = (int)dtype_size(dt);
    const Geometry g = make_geometry(R, fast ? 16 / es : 1, es);
    return dispatch<BwdFn>(dt, fast, g.J, X->order, X, seg_mode, U, R, g, gscale, G, s);
}

pasta_status launch_cp_loss_fwd_bwd(const pasta_coo_s *X, const void *const *U, pasta_dtype dt,
                                    int R, double *loss, const double *gscale, void *const *G,
                                    cudaStream_t s) {
    bool fast = stream_supported(dt, X->order, R, U, -1, nullptr);
    for (int k = 0; k < X->order; ++k) fast = fast && aligned16(G[k]);
    if (!fast) {
        // general kernels: forward over the mode-0 copy, then one pass per mode
        pasta_status st = launch_cp_loss_fwd(view_of(X, X->sorted[0]), 0, X->num_sms, U, dt, R,
                                             loss, nullptr, X->partials, X->partials_cap, s);
        if (st != PASTA_OK) return st;
        return launch_cp_loss_bwd(X, -2, U, dt, R, gscale, G, s);
    }
    for (int k = 0; k < X->order; ++k)
        PASTA_CUDA(cudaMemsetAsync(G[k], 0, (size_t)X->dims[k] * (size_t)R * sizeof(float), s));
    if (X->nnz == 0) {
        PASTA_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), s));
        return PASTA_OK;
    }
    for (int p = 0; p < X->order; ++p) {
        const CooView v = view_of(X, X->sorted[p]);
        StreamLaunch l;
        l.order = X->order;
        l.R = R;
        l.dtype = dt;
        for (int q = 0; q < X->order; ++q) {
            const int k = (p + q) % X->order;
            l.idx[q] = v.idx[k];
            l.U[q] = U[k];
        }
        l.val = v.val;
        l.out = static_cast<float *>(G[p]);
        l.gscale = gscale;
        l.nnz = v.nnz;
        l.num_sms = X->num_sms;
        int blocks = 0;
        if (p == 0) {  // the first pass also sums the squared residuals
            l.partials = X->partials;
            l.max_blocks = X->partials_cap;
            l.blocks_used = &blocks;
        }
        pasta_status st = launch_stream(2, l, s);
        if (st != PASTA_OK) return st;
        if (p == 0) {
            k_loss_finalize<<<1, 256, 0, s>>>(X->partials, blocks, loss);
            PASTA_CUDA(cudaGetLastError());
        }
    }
    return PASTA_OK;
}

pasta_status launch_convert(const void *src, pasta_dtype st, void *dst, pasta_dtype dt,
                            uint64_t n, const double *scale, cudaStream_t s) {
    if (n == 0) return PASTA_OK;
    const int blocks = (int)std::min<uint64_t>((n + 255) / 256, 4096);
    switch (st) {
        case PASTA_F32: return convert_from<float>((const float *)src, dst, dt, n, s, blocks, scale);
        case PASTA_BF16: return convert_from<__nv_bfloat16>((const __nv_bfloat16 *)src, dst, dt, n, s, blocks, scale);
        case PASTA_F16: return convert_from<__half>((const __half *)src, dst, dt, n, s, blocks, scale);
        case PASTA_F64: return convert_from<double>((const double *)src, dst, dt, n, s, blocks, scale);
    }
    return PASTA_ERR_INVALID_ARG;
}

}  // namespace pasta
