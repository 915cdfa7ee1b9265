// Streaming kernels over a mode-sorted COO copy: MTTKRP (Eq. (mttkrp-init),
// Algorithm 6), the CP-loss forward and the per-mode CP-loss backward share
// one walk.
//
// Geometry: lanes span the rank (L lanes x 16 bytes cover a factor row, so
// R * sizeof(T) == 16 L), G = 32/L lane groups per warp, each group owns a
// contiguous "group tile" of the stream, and a block owns a contiguous "block
// tile" made of its warps' group tiles in order.  COO words reach shared
// memory by cp.async (one 16-byte copy per lane per array per 4 entries,
// STAGES chunks in flight per warp); each batch of four entries is read back
// with one 16-byte broadcast load per array, so no index shuffles are needed.
// All factor-row loads of a batch are issued before any is used.
//
// Run reduction: the stream is sorted by position 0's mode, so the entries of
// one output row are contiguous.  Each group keeps the running row sum in
// registers.  A run that opens and closes inside its group tile is the whole
// row: one plain 16-byte store per lane.  The first closed run of a group tile
// is added with red.global.add.v4.f32 if it began in an earlier tile (the
// entry before the tile has the same row), else stored as a whole row;
// the run still open at the tile end goes to a shared-memory slot, and after
// the warp's group tiles equal rows among its slots are summed and added
// once.  A row spanning many tiles thus costs one atomic per warp tile (G
// group tiles, 2048 entries at R = 32 FP32), which also keeps its FP32
// rounding chain short; the add is red.global.add.v4.f32, four columns per
// lane.
//
// L2 policy: factor rows are re-read across the whole launch (evict-last).
#pragma once

#include "pasta_internal.cuh"

namespace pasta {
namespace stream {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }

// kGather: a diagnostic that gathers exactly the rows MTTKRP gathers, with
// the same staging, batches and launch, but neither scales nor reduces them
// into output rows (each thread writes one float of what it summed): the
// gather ceiling of the MTTKRP kind on the same tensor.
enum Kind : int { kMttkrp = 0, kLossFwd = 1, kLossBwd = 2, kGather = 3 };

// Longest lane-group tile (at least one chunk of 4L); the launch may pick a
// shorter multiple of the chunk to balance the grid.  A block tile is kWarps
// * G group tiles, a warp tile the warp's G of them.
#ifndef PASTA_STREAM_GROUP_TILE
#define PASTA_STREAM_GROUP_TILE 512
#endif
constexpr int kGroupTile = PASTA_STREAM_GROUP_TILE;
__host__ __device__ constexpr int group_tile(int L) { return 4 * L > kGroupTile ? 4 * L : kGroupTile; }

template <typename T, int N>
struct Args {
    const uint32_t *idx[N];  // position p holds mode (rot + p) % N; position 0 is the sorted mode
    const T *U[N];           // factor of position p (position 0 unused by MTTKRP)
    const float *val;
    float *out;              // MTTKRP: M; loss bwd: gradient of position 0; loss fwd: residuals or null
    double *partials;        // loss fwd (and fused loss bwd, else null): per-block FP64 partial sums
    const double *gscale;    // loss bwd: incoming gradient (null = 1)
    uint64_t nnz;
    uint32_t R;
    int L, lshift;
    int tile;  // entries per group tile, a multiple of 4L
};

// 16-byte asynchronous copy global -> shared, L1 bypassed; src_bytes < 16
// fills the rest with zeros.  (The form with an L2 cache-policy operand
// raised an illegal-instruction fault on GB300 together with src_bytes, so
// the COO stream is copied without a policy.)
__device__ __forceinline__ void cp_async16(uint32_t *smem, const void *gmem, int src_bytes) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem),
                 "r"(src_bytes));
}

__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// 16-byte read-only load of a factor row slice, kept in L2 preferentially
// (measured: 1-1.5% faster MTTKRP than without the hint; an L1 evict-last
// hint on top changed nothing).
__device__ __forceinline__ uint4 ld_row(const uint4 *p, uint64_t pol) {
    uint4 r;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int K> __device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(K));
}

// ---- per-lane vector arithmetic on VEC FP32 values.  The pairs go through
// the packed FP32x2 instructions of sm_100 and later (__fmul2_rn,
// __ffma2_rn: one instruction per two values, each rounded as the scalar
// FMUL/FFMA would).  Measured 1-2% faster on zipf3d, neutral elsewhere.
// PASTA_STREAM_F2=0 builds the scalar form.
#ifndef PASTA_STREAM_F2
#define PASTA_STREAM_F2 1
#endif
constexpr bool kF2 = PASTA_STREAM_F2 != 0;
#ifndef PASTA_SHFL_CONST
#define PASTA_SHFL_CONST 1
#endif
constexpr bool kShflConst = PASTA_SHFL_CONST != 0;
#ifndef PASTA_FAST_BATCH
#define PASTA_FAST_BATCH 1
#endif
constexpr bool kFastBatch = PASTA_FAST_BATCH != 0;

template <int VEC> __device__ __forceinline__ void v_scale(float (&y)[VEC], float a, const float (&x)[VEC]) {
    if constexpr (kF2 && VEC % 2 == 0) {
#pragma unroll
        for (int e = 0; e < VEC; e += 2) {
            const float2 r = __fmul2_rn(make_float2(a, a), make_float2(x[e], x[e + 1]));
            y[e] = r.x;
            y[e + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) y[e] = a * x[e];
    }
}
template <int VEC> __device__ __forceinline__ void v_mul(float (&y)[VEC], const float (&x)[VEC]) {
    if constexpr (kF2 && VEC % 2 == 0) {
#pragma unroll
        for (int e = 0; e < VEC; e += 2) {
            const float2 r = __fmul2_rn(make_float2(y[e], y[e + 1]), make_float2(x[e], x[e + 1]));
            y[e] = r.x;
            y[e + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) y[e] *= x[e];
    }
}
// acc += a * b (element-wise)
template <int VEC>
__device__ __forceinline__ void v_fma(float (&acc)[VEC], const float (&a)[VEC], const float (&b)[VEC]) {
    if constexpr (kF2 && VEC % 2 == 0) {
#pragma unroll
        for (int e = 0; e < VEC; e += 2) {
            const float2 r = __ffma2_rn(make_float2(a[e], a[e + 1]), make_float2(b[e], b[e + 1]),
                                        make_float2(acc[e], acc[e + 1]));
            acc[e] = r.x;
            acc[e + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = fmaf(a[e], b[e], acc[e]);
    }
}
// acc += w * b
template <int VEC> __device__ __forceinline__ void v_fma_s(float (&acc)[VEC], float w, const float (&b)[VEC]) {
    if constexpr (kF2 && VEC % 2 == 0) {
#pragma unroll
        for (int e = 0; e < VEC; e += 2) {
            const float2 r = __ffma2_rn(make_float2(w, w), make_float2(b[e], b[e + 1]),
                                        make_float2(acc[e], acc[e + 1]));
            acc[e] = r.x;
            acc[e + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = fmaf(w, b[e], acc[e]);
    }
}
// sum_e a[e] * b[e]
template <int VEC> __device__ __forceinline__ float v_dot(const float (&a)[VEC], const float (&b)[VEC]) {
    if constexpr (kF2 && VEC % 2 == 0) {
        float2 t = __fmul2_rn(make_float2(a[0], a[1]), make_float2(b[0], b[1]));
#pragma unroll
        for (int e = 2; e < VEC; e += 2) t = __ffma2_rn(make_float2(a[e], a[e + 1]), make_float2(b[e], b[e + 1]), t);
        return t.x + t.y;
    } else {
        float part = 0.f;
#pragma unroll
        for (int e = 0; e < VEC; ++e) part = fmaf(a[e], b[e], part);
        return part;
    }
}

// Shared memory per block: the COO stages of every warp.  After a warp has
// drained its stages at the end of a warp tile, the same words hold its
// groups' end-of-tile slots: G row indices (padded to 4 words), then G rows
// of R FP32 partials (G * (R + 1) words <= the stage words for every covered
// geometry).
__host__ __device__ constexpr int coo_words_per_warp(int N, int stages, int L) {
    return stages * (N + 1) * (32 / L) * (4 * L + 4);
}
__host__ __device__ constexpr size_t smem_bytes(int N, int stages, int L, int R) {
    (void)R;
    return (size_t)kWarps * coo_words_per_warp(N, stages, L) * 4;
}

// Per-group running state.
template <int VEC>
struct GroupState {
    float acc[VEC];
    uint32_t cur;   // row of the open run (kNoRow before the first entry)
    bool first;     // the open run continues a run of the previous tile
    uint4 row0;     // loss kinds: position-0 factor row of the open run
    float sq32;     // loss fwd: FP32 sum of squared residuals of the current chunk
    double sq;      // loss fwd: FP64 sum of the chunk sums
};

template <typename T, int N, int KIND>
struct Ctx {
    static constexpr int VEC = 16 / sizeof(T);
    const Args<T, N> &a;
    const char *ub[N];  // this lane's first byte of row 0 of every factor
    uint32_t stride;    // bytes per factor row
    int lane_off;       // this lane's first element of a row
    int L, lig, gslot;
    uint64_t t0;
    uint64_t pol_rows;  // L2 evict-last policy for factor rows
    float g_scale;
    bool sq_lane;       // this lane adds the squared residuals (loss fwd, or bwd with partials)
};

// Close the open run: a run continuing one of the previous tile (only the
// tile's first) is added atomically; any other is a whole row and is stored.
template <typename T, int N, int KIND>
__device__ __forceinline__ void close_run(const Ctx<T, N, KIND> &c,
                                          GroupState<Ctx<T, N, KIND>::VEC> &s) {
    constexpr int VEC = Ctx<T, N, KIND>::VEC;
    float *d = c.a.out + (uint64_t)s.cur * c.a.R + c.lane_off;
#pragma unroll
    for (int e = 0; e < VEC; e += 4) {
        const float v4[4] = {s.acc[e], s.acc[e + 1], s.acc[e + 2], s.acc[e + 3]};
        if (s.first)
            RedAdd<float, 4>::run(d + e, v4);  // may continue a run of an earlier tile
        else
            Store<float, 4>::run(d + e, v4);   // the whole row
    }
    s.first = false;
}

// One batch: the four entries held at position `src` of the group's chunk.
// CHECK = false when all four are real entries (every full chunk).
// R0L (loss kinds): 0 = position 0's row, needed where a run starts, is
// gathered with the others in phase A (a register row per entry); 1 = it is
// loaded in phase B when the run changes (fewer registers, a dependent load).

// One batch's staged inputs between its two phases: position 0's indices and
// the values of the four entries, and the rows gathered in phase A.
template <int N, int NR>
struct Staged {
    uint32_t i0[4];
    float v[4];
    uint4 rows[4][NR];
    bool need0[4];
};

template <int N, int KIND, int R0L>
struct Shape {
    static constexpr bool MT = (KIND == kMttkrp || KIND == kGather);
    static constexpr int P0 = (MT || R0L) ? 1 : 0;  // first position gathered in phase A
    static constexpr int NR = N - P0;               // rows gathered per entry in phase A
};

// Phase A of the four entries held at position `src` of the group's chunk:
// indices and values from shared memory, then every gathered row (position
// 0, loss kinds, only where the run changes; prev0 = the row of the entry
// before the batch).  CHECK = false when all four are real entries.
template <bool CHECK, int R0L, typename T, int N, int KIND>
__device__ __forceinline__ void batch_load(const Ctx<T, N, KIND> &c, uint32_t prev0, const uint32_t *sb, int AS,
                                           int src, int lim, Staged<N, Shape<N, KIND, R0L>::NR> &b) {
    constexpr int P0 = Shape<N, KIND, R0L>::P0;
    uint32_t iw[N][4];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const uint4 w = *reinterpret_cast<const uint4 *>(sb + k * AS + 4 * src);
        iw[k][0] = w.x; iw[k][1] = w.y; iw[k][2] = w.z; iw[k][3] = w.w;
    }
    {
        const float4 w = *reinterpret_cast<const float4 *>(sb + N * AS + 4 * src);
        b.v[0] = w.x; b.v[1] = w.y; b.v[2] = w.z; b.v[3] = w.w;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        b.i0[q] = iw[0][q];
        const bool ok = !CHECK || q < lim;
        // Only R0L = 0 loads position 0 here.  R0L = 1 tests the run change
        // in phase B, where it is the same test (the entries of a batch are
        // in stream order and invalid ones only trail it); not carrying the
        // flags across the phases made the loss pass 1-6% faster.
        if (P0 == 0) b.need0[q] = ok && iw[0][q] != (q == 0 ? prev0 : iw[0][q - 1]);
#pragma unroll
        for (int p = P0; p < N; ++p) {
            const uint4 *ptr = reinterpret_cast<const uint4 *>(c.ub[p] + (uint64_t)iw[p][q] * c.stride);
            if (p == 0) {
                if (b.need0[q]) b.rows[q][0] = ld_row(ptr, c.pol_rows);
            } else if (CHECK) {
                b.rows[q][p - P0] = ok ? ld_row(ptr, c.pol_rows) : make_uint4(0u, 0u, 0u, 0u);
            } else {
                b.rows[q][p - P0] = ld_row(ptr, c.pol_rows);
            }
        }
    }
}

// Phase B: the four entries' arithmetic in stream order.
// R0L (loss kinds): 0 = position 0's row, needed where a run starts, was
// gathered in phase A (a register row per entry); 1 = it is loaded here when
// the run changes (fewer registers, a dependent load).
template <bool CHECK, int R0L, int LC, typename T, int N, int KIND>
__device__ __forceinline__ void batch_compute(const Ctx<T, N, KIND> &c, GroupState<Ctx<T, N, KIND>::VEC> &s,
                                              const Staged<N, Shape<N, KIND, R0L>::NR> &b, int lim,
                                              uint64_t pos) {
    constexpr int VEC = Ctx<T, N, KIND>::VEC;
    constexpr bool MT = Shape<N, KIND, R0L>::MT;
    constexpr int P0 = Shape<N, KIND, R0L>::P0;
    constexpr int NR = Shape<N, KIND, R0L>::NR;
    // The arithmetic of entry q with the run state as it stands.
    auto math = [&](int q, bool ok) {
        float p[VEC], r[VEC];
        if constexpr (KIND == kGather) {
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                widen<T, VEC>(b.rows[q][k], r);
                if (ok) {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) s.acc[e] += r[e];
                }
            }
        } else if constexpr (KIND == kMttkrp && NR == 1) {  // order 2: val times one row
            widen<T, VEC>(b.rows[q][0], r);
            if (ok) v_fma_s<VEC>(s.acc, b.v[q], r);
        } else if (KIND == kMttkrp) {
            widen<T, VEC>(b.rows[q][0], r);
            v_scale<VEC>(p, b.v[q], r);
#pragma unroll
            for (int k = 1; k < NR - 1; ++k) {
                widen<T, VEC>(b.rows[q][k], r);
                v_mul<VEC>(p, r);
            }
            widen<T, VEC>(b.rows[q][NR - 1], r);
            if (ok) v_fma<VEC>(s.acc, p, r);
        } else {
            // p = prod over positions 1..N-1; model = sum_r p * row0
            widen<T, VEC>(b.rows[q][1 - P0], p);
#pragma unroll
            for (int k = 2; k < N; ++k) {
                widen<T, VEC>(b.rows[q][k - P0], r);
                v_mul<VEC>(p, r);
            }
            widen<T, VEC>(s.row0, r);
            float part = v_dot<VEC>(p, r);
            if constexpr (LC > 0 && kShflConst) {  // the lane count compiled in: an unrolled tree
#pragma unroll
                for (int o = LC >> 1; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o, LC);
            } else {
                for (int o = c.L >> 1; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o, c.L);
            }
            const float e_m = b.v[q] - part;
            if (KIND == kLossFwd) {
                if (ok && c.lig == 0) {
                    // FP32 within a chunk (at most 4L <= 128 positive terms,
                    // relative error <= 127 u); FP64 across chunks.  GB300's
                    // FP64 pipe is too narrow for one FP64 add per entry.
                    s.sq32 = fmaf(e_m, e_m, s.sq32);
                    if (c.a.out) c.a.out[pos + q] = e_m;
                }
            } else if (ok) {
                // fused forward: the backward pass over the first copy also
                // sums the squared residuals (Args::partials set)
                if (c.sq_lane) s.sq32 = fmaf(e_m, e_m, s.sq32);
                const float w = -c.g_scale * e_m;
                v_fma_s<VEC>(s.acc, w, p);
            }
        }
    };
    if constexpr (KIND == kGather) {
#pragma unroll
        for (int q = 0; q < 4; ++q) math(q, !CHECK || q < lim);
        return;
    }
    if constexpr (kFastBatch) {
        // No lane group of the warp starts a run in this batch (the common
        // case on long runs): one vote instead of one per entry.
        bool any = false;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            any |= (!CHECK || q < lim) && b.i0[q] != (q == 0 ? s.cur : b.i0[q - 1]);
        if (!__any_sync(kFull, any)) {
#pragma unroll
            for (int q = 0; q < 4; ++q) math(q, !CHECK || q < lim);
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const bool ok = !CHECK || q < lim;
        const bool changed = ok && b.i0[q] != s.cur;
        if (KIND != kLossFwd) {
            if (__any_sync(kFull, changed)) {
                if (changed) {
                    if (s.cur != kNoRow) close_run(c, s);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) s.acc[e] = 0.f;
                }
            }
        }
        if (changed) s.cur = b.i0[q];
        if constexpr (!MT && R0L) {
            // the run's row where it starts (a divergent branch measured faster
            // than a predicated load on every lane group)
            if (changed)
                s.row0 = ld_row(reinterpret_cast<const uint4 *>(c.ub[0] + (uint64_t)b.i0[q] * c.stride),
                                c.pol_rows);
        } else if (!MT && b.need0[q]) {
            s.row0 = b.rows[q][0];
        }
        math(q, ok);
    }
}

// One batch, both phases.
template <bool CHECK, int R0L, int LC, typename T, int N, int KIND>
__device__ __forceinline__ void batch(const Ctx<T, N, KIND> &c, GroupState<Ctx<T, N, KIND>::VEC> &s,
                                      const uint32_t *sb, int AS, int src, int lim, uint64_t pos) {
    Staged<N, Shape<N, KIND, R0L>::NR> b;
    batch_load<CHECK, R0L>(c, s.cur, sb, AS, src, lim, b);
    batch_compute<CHECK, R0L, LC>(c, s, b, lim, pos);
}

// LC: lanes per entry fixed at compile time (0 = read from Args), which turns
// every lane-group stride, shared-memory offset and shuffle width into a
// constant.
template <typename T, int N, int KIND, int STAGES, int MINB, int LC = 0, int R0L = 0>
__global__ void __launch_bounds__(kThreads, MINB) k_stream(const Args<T, N> a) {
    constexpr int VEC = 16 / sizeof(T);
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int L = LC ? LC : a.L;
    const int lshift = LC ? ilog2(LC) : a.lshift;
    const int lig = lane & (L - 1);
    const int grp = lane >> lshift;
    const int G = 32 >> lshift;
    const int tile = a.tile;
    const int chunk = 4 * L;
    const int GS = 4 * L + 4;  // padded words per group chunk (bank spread)
    const int AS = G * GS;     // words per array per stage
    const int SS = (N + 1) * AS;
    uint32_t *wbuf = smem + (size_t)warp * STAGES * SS;
    const int nchunks = tile / chunk;

    Ctx<T, N, KIND> c{a};
    c.stride = a.R * (uint32_t)sizeof(T);
    c.lane_off = lig * VEC;
#pragma unroll
    for (int p = 0; p < N; ++p) c.ub[p] = reinterpret_cast<const char *>(a.U[p] + c.lane_off);
    c.L = L;
    c.lig = lig;
    c.pol_rows = policy_evict_last();
    // end-of-tile slots (overlaid on each warp's drained COO stages)
    const int G4 = (G + 3) & ~3;
    auto slot_row = [&](int sidx) { return smem + (size_t)(sidx / G) * STAGES * SS + (sidx % G); };
    auto slot_val = [&](int sidx) {
        return reinterpret_cast<float *>(smem + (size_t)(sidx / G) * STAGES * SS + G4) +
               (size_t)(sidx % G) * a.R;
    };
    c.g_scale = (KIND == kLossBwd && a.gscale) ? (float)*a.gscale : 1.f;
    c.sq_lane = lig == 0 && (KIND == kLossFwd || a.partials != nullptr);

    GroupState<VEC> s;
#pragma unroll
    for (int e = 0; e < VEC; ++e) s.acc[e] = 0.f;
    s.sq = 0.0;
    s.sq32 = 0.f;
    s.row0 = make_uint4(0u, 0u, 0u, 0u);

    const uint64_t block_span = (uint64_t)tile * (uint64_t)(G * kWarps);
    const uint64_t nbt = (a.nnz + block_span - 1) / block_span;

    for (uint64_t bt = blockIdx.x; bt < nbt; bt += gridDim.x) {
        c.gslot = warp * G + grp;
        c.t0 = bt * block_span + (uint64_t)c.gslot * (uint64_t)tile;
        const uint64_t t0 = c.t0;
        const int len = (int)(t0 < a.nnz ? min((uint64_t)tile, a.nnz - t0) : 0);
        if (KIND != kGather) {
#pragma unroll
            for (int e = 0; e < VEC; ++e) s.acc[e] = 0.f;
        }
        s.cur = kNoRow;
        // the tile's first run continues a run of the previous tile
        s.first = t0 > 0 && t0 < a.nnz && a.idx[0][t0 - 1] == a.idx[0][t0];


        auto issue = [&](int ci, int stage) {
            const int off = ci * chunk + 4 * lig;
            const bool ld = ci < nchunks && off < len;
            const uint64_t my = t0 + (uint64_t)off;
            uint32_t *sb = wbuf + stage * SS + grp * GS + 4 * lig;
#pragma unroll
            for (int k = 0; k < N; ++k)
                cp_async16(sb + k * AS, ld ? (const void *)(a.idx[k] + my) : (const void *)a.idx[k],
                           ld ? 16 : 0);
            cp_async16(sb + N * AS, ld ? (const void *)(a.val + my) : (const void *)a.val, ld ? 16 : 0);
            cp_commit();
        };
#pragma unroll
        for (int st = 0; st < STAGES - 1; ++st) issue(st, st);
        for (int i = 0;; ++i) {
            const int rem = len - i * chunk;
            if (!__any_sync(kFull, i < nchunks && rem > 0)) break;
            issue(i + STAGES - 1, (i + STAGES - 1) % STAGES);
            cp_wait<STAGES - 1>();
            __syncwarp();
            const uint32_t *sb = wbuf + (i % STAGES) * SS + grp * GS;
            const uint64_t pos = t0 + (uint64_t)(i * chunk);
            if (__all_sync(kFull, rem >= chunk)) {
                for (int src = 0; src < L; ++src)
                    batch<false, R0L, LC>(c, s, sb, AS, src, 4, pos + 4u * (uint64_t)src);
            } else {
                for (int src = 0; src < L; ++src)
                    batch<true, R0L, LC>(c, s, sb, AS, src, rem - 4 * src, pos + 4u * (uint64_t)src);
            }
            if (KIND == kLossFwd || (KIND == kLossBwd && a.partials)) {
                s.sq += (double)s.sq32;
                s.sq32 = 0.f;
            }
            __syncwarp();
        }
        cp_wait<0>();
        __syncwarp();

        if (KIND != kLossFwd && KIND != kGather) {
            // The run still open at the tile end goes to this group's slot
            // (the warp's stages are drained, so their words are free).
            if (lig == 0) *slot_row(c.gslot) = s.cur;
            if (s.cur != kNoRow) {
                float *d = slot_val(c.gslot) + c.lane_off;
#pragma unroll
                for (int e = 0; e < VEC; e += 4)
                    *reinterpret_cast<float4 *>(d + e) =
                        make_float4(s.acc[e], s.acc[e + 1], s.acc[e + 2], s.acc[e + 3]);
            }
            __syncwarp();
            // Sum the warp's consecutive slots of equal row (in stream order)
            // and add each sum once; lanes span the row.  (Combining over the
            // whole block tile instead cost a block barrier per tile: 1-7%
            // slower, the block waiting for its slowest warp.)
            const int s_lo = warp * G;
            const int s_hi = warp * G + G;
            for (int h = s_lo; h < s_hi; ++h) {
                const uint32_t row = *slot_row(h);
                if (row == kNoRow) continue;
                int prev = h - 1;
                while (prev >= s_lo && *slot_row(prev) == kNoRow) --prev;
                if (prev >= s_lo && *slot_row(prev) == row) continue;  // not the first slot of its run
                int end = h;
                for (int u = h + 1; u < s_hi; ++u) {
                    const uint32_t ru = *slot_row(u);
                    if (ru == kNoRow) continue;
                    if (ru != row) break;
                    end = u;
                }
                // R is a multiple of 4 (R * sizeof(T) = 16 L) and the slot rows
                // and the output are 16-byte aligned: one vector add per 4 columns.
                for (int t = 4 * lane; t < (int)a.R; t += 128) {
                    float sum[4] = {0.f, 0.f, 0.f, 0.f};
                    for (int u = h; u <= end; ++u)
                        if (*slot_row(u) == row) {
                            const float4 v = *reinterpret_cast<const float4 *>(slot_val(u) + t);
                            sum[0] += v.x;
                            sum[1] += v.y;
                            sum[2] += v.z;
                            sum[3] += v.w;
                        }
                    RedAdd<float, 4>::run(a.out + (uint64_t)row * a.R + t, sum);
                }
            }
            __syncwarp();  // the slots are staging words again in the next tile
        }
    }

    if (KIND == kGather) {
        float t = 0.f;
#pragma unroll
        for (int e = 0; e < VEC; ++e) t += s.acc[e];
        a.out[(uint64_t)blockIdx.x * kThreads + threadIdx.x] = t;
    }
    if (KIND == kLossFwd || (KIND == kLossBwd && a.partials)) {
        double sq = s.sq;
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(kFull, sq, o);
        __shared__ double ws[kWarps];
        if (lane == 0) ws[warp] = sq;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kWarps; ++w) t += ws[w];
            a.partials[blockIdx.x] = t;
        }
    }
}

}  // namespace stream
}  // namespace pasta
