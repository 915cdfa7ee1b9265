// Mode-n COO MTTKRP on the mode-n sorted copy (arXiv:1902.03317, Eq.
// (mttkrp-init) and Algorithm 6):
//     M(i, r) = sum_{m : i_n(m) = i} val(m) * prod_{k != n} U_k(i_k(m), r).
//
// The paper's parallel loop over nonzeros races on the output row (Sec. 5.3),
// which it resolves with atomics or with per-thread private copies of the
// output plus a final reduction.  Here the stream is sorted by the output
// index, so all contributions to one row are contiguous: each lane group
// (L lanes spanning the rank) walks a contiguous tile of the stream and keeps
// the running row sum in registers.  A run that starts and ends inside the
// tile is the whole row and is written with a plain 16-byte store; only the
// first and last run of a tile, which may continue in a neighbouring tile,
// are added with red.global.add.v4.f32 into the zero-filled output.
//
// Per entry: one 16-byte load per COO array per four entries (streamed,
// evict-first), the N-1 gathered factor rows (16-byte loads, lanes across R),
// and (N-1)*R multiplies.
#include <algorithm>

#include "pasta_internal.cuh"

namespace pasta {
namespace {

constexpr int kThreads = 256;

template <typename T, int NM>
struct MttkrpArgs {
    const uint32_t *idx[NM];  // idx[0]: output mode; idx[1..nother]: the other modes
    const T *U[NM];           // U[p] is the factor of the mode at position p (U[0] unused)
    const float *val;
    typename AccOf<T>::type *M;
    uint64_t nnz;
    int nother;
    int R, S, L, lshift, tile;
};

// Load this lane's four consecutive entries of a chunk: one 16-byte streamed
// load per COO array (arrays are padded, so the load stays in bounds).
template <int NM>
__device__ __forceinline__ void load_chunk(const uint32_t *const (&idx)[NM], const float *val,
                                           int nother, uint64_t my, bool ld, uint64_t pol,
                                           uint32_t (&ci)[NM][4], float (&cv)[4]) {
#pragma unroll
    for (int k = 0; k < NM; ++k) {
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (ld && k <= nother) w = ld_stream_u4(idx[k] + my, pol);
        ci[k][0] = w.x; ci[k][1] = w.y; ci[k][2] = w.z; ci[k][3] = w.w;
    }
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ld) w = ld_stream_f4(val + my, pol);
    cv[0] = w.x; cv[1] = w.y; cv[2] = w.z; cv[3] = w.w;
}

template <typename T, int VEC, int J, int NM>
__global__ void __launch_bounds__(kThreads) k_mttkrp(const MttkrpArgs<T, NM> a) {
    using A = typename AccOf<T>::type;
    using RawT = typename Raw<T, VEC>::type;
    constexpr unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const int L = a.L;
    const int lig = lane & (L - 1);
    const int grp = lane >> a.lshift;
    const int G = 32 >> a.lshift;
    const int chunk = 4 * L;
    const uint64_t pol = policy_evict_first();

    int slot[J];
    bool act[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        slot[j] = lig + j * L;
        act[j] = slot[j] < a.S;
    }

    const uint64_t warp_span = (uint64_t)a.tile * (uint64_t)G;
    const uint64_t nwt = (a.nnz + warp_span - 1) / warp_span;
    const uint64_t wpb = blockDim.x >> 5;

    for (uint64_t wt = (uint64_t)blockIdx.x * wpb + (threadIdx.x >> 5); wt < nwt;
         wt += (uint64_t)gridDim.x * wpb) {
        const uint64_t t0 = wt * warp_span + (uint64_t)grp * (uint64_t)a.tile;
        const uint64_t t1 = min(t0 + (uint64_t)a.tile, a.nnz);

        A acc[J][VEC];
#pragma unroll
        for (int j = 0; j < J; ++j)
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc[j][e] = A(0);
        uint32_t cur = kNoRow;
        bool first = true;

        auto flush = [&](uint32_t row, bool atomic) {
            A *dst = a.M + (uint64_t)row * (uint64_t)a.R;
#pragma unroll
            for (int j = 0; j < J; ++j) {
                if (!act[j]) continue;
                if (atomic)
                    RedAdd<A, VEC>::run(dst + slot[j] * VEC, acc[j]);
                else
                    Store<A, VEC>::run(dst + slot[j] * VEC, acc[j]);
            }
        };

        // COO words of the current chunk; the next chunk's are requested
        // before the current one is processed.
        uint32_t ci[NM][4];
        float cv[4];
        {
            const uint64_t my = t0 + 4u * (uint64_t)lig;
            load_chunk<NM>(a.idx, a.val, a.nother, my, my < t1, pol, ci, cv);
        }
        for (int c = 0; c < a.tile; c += chunk) {
            const uint64_t base = t0 + (uint64_t)c;
            if (!__any_sync(FULL, base < t1)) break;
            uint32_t ni[NM][4];
            float nv[4];
            {
                const uint64_t my = base + (uint64_t)chunk + 4u * (uint64_t)lig;
                load_chunk<NM>(a.idx, a.val, a.nother, my, c + chunk < a.tile && my < t1, pol, ni, nv);
            }

            for (int src = 0; src < L; ++src) {
                // Phase A: indices, values and every gathered row of the four
                // entries held by lane `src` of the group, all loads in flight
                // before any is used.
                uint32_t io[4];
                float v[4];
                bool ok[4];
                RawT rows[4][NM > 1 ? NM - 1 : 1][J];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ok[q] = base + 4u * (uint64_t)src + (uint64_t)q < t1;  // uniform per group
                    io[q] = __shfl_sync(FULL, ci[0][q], src, L);
                    v[q] = __shfl_sync(FULL, cv[q], src, L);
#pragma unroll
                    for (int k = 1; k < NM; ++k) {
                        if (k > a.nother) continue;
                        const uint32_t ik = __shfl_sync(FULL, ci[k][q], src, L);
                        const T *row = a.U[k] + (uint64_t)ik * (uint64_t)a.R;
#pragma unroll
                        for (int j = 0; j < J; ++j)
                            if (ok[q] && act[j]) rows[q][k - 1][j] = load_raw<T, VEC>(row + slot[j] * VEC);
                    }
                }
                // Phase B: Hadamard product scaled by the value, then the run
                // reduction along equal output rows.
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (!ok[q]) continue;
                    A t[J][VEC];
#pragma unroll
                    for (int j = 0; j < J; ++j)
#pragma unroll
                        for (int e = 0; e < VEC; ++e) t[j][e] = A(v[q]);
#pragma unroll
                    for (int k = 1; k < NM; ++k) {
                        if (k > a.nother) continue;
#pragma unroll
                        for (int j = 0; j < J; ++j) {
                            if (!act[j]) continue;
                            A r[VEC];
                            widen<T, VEC>(rows[q][k - 1][j], r);
#pragma unroll
                            for (int e = 0; e < VEC; ++e) t[j][e] *= r[e];
                        }
                    }
                    if (io[q] != cur) {
                        if (cur != kNoRow) {
                            flush(cur, first);
                            first = false;
                        }
                        cur = io[q];
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
                }
            }
#pragma unroll
            for (int k = 0; k < NM; ++k)
#pragma unroll
                for (int q = 0; q < 4; ++q) ci[k][q] = ni[k][q];
#pragma unroll
            for (int q = 0; q < 4; ++q) cv[q] = nv[q];
        }
        if (cur != kNoRow) flush(cur, true);
    }
}

template <typename T, int VEC, int J, int NM>
pasta_status run(const pasta_coo_s *X, const StoredCopy &c, const void *const *U, int mode, int R,
                 const Geometry &g, void *M, cudaStream_t s) {
    using A = typename AccOf<T>::type;
    MttkrpArgs<T, NM> a{};
    const int N = X->order;
    for (int p = 0; p < N && p < NM; ++p) {
        const int k = (mode + p) % N;
        a.idx[p] = c.idx[k];
        a.U[p] = static_cast<const T *>(U[k]);
    }
    a.val = c.val;
    a.M = static_cast<A *>(M);
    a.nnz = X->nnz;
    a.nother = N - 1;
    a.R = R;
    a.S = g.slots;
    a.L = g.L;
    a.lshift = g.lshift;
    a.tile = g.tile;

    PASTA_CUDA(cudaMemsetAsync(M, 0, (size_t)X->dims[mode] * (size_t)R * sizeof(A), s));
    if (X->nnz == 0) return PASTA_OK;

    int per_sm = 0;  // queried per call: no shared state between host threads
    PASTA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mttkrp<T, VEC, J, NM>, kThreads, 0));
    if (per_sm < 1) per_sm = 1;
    const uint64_t G = 32u >> g.lshift;
    const uint64_t nwt = (X->nnz + (uint64_t)g.tile * G - 1) / ((uint64_t)g.tile * G);
    const uint64_t wpb = kThreads / 32;
    const uint64_t want = (nwt + wpb - 1) / wpb;
    const int blocks = (int)apply_grid_cap(std::min<uint64_t>(want, (uint64_t)X->num_sms * (uint64_t)per_sm));
    k_mttkrp<T, VEC, J, NM><<<blocks, kThreads, 0, s>>>(a);
    PASTA_CUDA(cudaGetLastError());
    return PASTA_OK;
}

template <typename T, int VEC, int J>
pasta_status by_order(const pasta_coo_s *X, const StoredCopy &c, const void *const *U, int mode,
                      int R, const Geometry &g, void *M, cudaStream_t s) {
    if (X->order <= 3) return run<T, VEC, J, 3>(X, c, U, mode, R, g, M, s);
    if (X->order == 4) return run<T, VEC, J, 4>(X, c, U, mode, R, g, M, s);
    if (X->order == 5) return run<T, VEC, J, 5>(X, c, U, mode, R, g, M, s);
    return run<T, VEC, J, 8>(X, c, U, mode, R, g, M, s);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

pasta_status launch_mttkrp(const pasta_coo_s *X, const StoredCopy &c, const void *const *U,
                           pasta_dtype dt, int mode, int R, void *M, cudaStream_t s,
                           bool every_row_touched) {
    if (stream_supported(dt, X->order, R, U, mode, M, 2)) {
        if (!every_row_touched || X->nnz == 0)
            PASTA_CUDA(cudaMemsetAsync(M, 0, (size_t)X->dims[mode] * (size_t)R * sizeof(float), s));
        if (X->nnz == 0) return PASTA_OK;
        StreamLaunch l;
        l.order = X->order;
        l.R = R;
        l.dtype = dt;
        for (int p = 0; p < X->order; ++p) {
            const int k = (mode + p) % X->order;
            l.idx[p] = c.idx[k];
            l.U[p] = U[k];
        }
        l.val = c.val;
        l.out = static_cast<float *>(M);
        l.nnz = X->nnz;
        l.num_sms = X->num_sms;
        l.zero_tile_end_rows = every_row_touched;
        return launch_stream(0, l, s);
    }
    const int es = (int)dtype_size(dt);
    bool fast = ((R * es) % 16) == 0 && aligned16(M);
    for (int k = 0; k < X->order; ++k)
        if (k != mode) fast = fast && aligned16(U[k]);
    const int vec = fast ? 16 / es : 1;
    const Geometry g = make_geometry(R, vec, es);
    if (!fast) {
        switch (dt) {
            case PASTA_F32: return run<float, 1, 8, 8>(X, c, U, mode, R, g, M, s);
            case PASTA_BF16: return run<__nv_bfloat16, 1, 8, 8>(X, c, U, mode, R, g, M, s);
            case PASTA_F16: return run<__half, 1, 8, 8>(X, c, U, mode, R, g, M, s);
            case PASTA_F64: return run<double, 1, 8, 8>(X, c, U, mode, R, g, M, s);
        }
        return PASTA_ERR_UNSUPPORTED;
    }
    switch (dt) {
        case PASTA_F32:
            if (g.J == 1) return by_order<float, 4, 1>(X, c, U, mode, R, g, M, s);
            return by_order<float, 4, 2>(X, c, U, mode, R, g, M, s);
        case PASTA_BF16: return by_order<__nv_bfloat16, 8, 1>(X, c, U, mode, R, g, M, s);
        case PASTA_F16: return by_order<__half, 8, 1>(X, c, U, mode, R, g, M, s);
        case PASTA_F64:
            if (g.J == 1) return run<double, 2, 1, 8>(X, c, U, mode, R, g, M, s);
            if (g.J == 2) return run<double, 2, 2, 8>(X, c, U, mode, R, g, M, s);
            return run<double, 2, 4, 8>(X, c, U, mode, R, g, M, s);
    }
    return PASTA_ERR_UNSUPPORTED;
}

}  // namespace pasta
