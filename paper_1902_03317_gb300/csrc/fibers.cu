// Mode-n fibers and the mode-n products TTV and TTM (Sec. 3.3 and 3.4,
// Algorithms 4 and 5).
//
// A mode-n fiber is the set of stored entries sharing every index but i_n.
// In the mode-(n+1) sorted copy the key runs through modes n+1, ..., N-1,
// 0, ..., n-1 and ends with n, so each fiber is one contiguous run there
// (when those N-1 modes fit the key's 64 bits, checked here).  The fiber
// table is that copy's run structure: fid[p] = the fiber of sorted position
// p (the paper's fptr, inverted) and each fiber's N-1 coordinates.
//
// Built in three launches: per-tile head counts (a head is a position whose
// fiber coordinates differ from its predecessor's), one block scanning the
// tile counts, and a pass that ranks the heads inside each tile (a lane takes
// four consecutive positions with 16-byte loads; per round of 1024 positions a
// warp scan of the lanes' head counts plus the block's warp totals) to write
// fid and the head coordinates.
//
// With the table, Y = X x_n U is exactly an MTTKRP of the order-2 tensor with
// coordinates (fid, i_n) and the same values: Y(f, r) = sum_{p in f}
// val(p) U(i_n(p), r), and fid is non-decreasing along the copy.  So TTM runs
// the MTTKRP kernels on that two-mode view.  TTV (R = 1) has its own kernel
// (k_ttv): with one value per entry the MTTKRP lane layout idles, and fibers
// are short, so each lane sums four entries and a warp scan joins them.
#include <algorithm>

#include "pasta_internal.cuh"

namespace pasta {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;  // positions per thread per tile
constexpr int kTile = kThreads * kItems;
constexpr int kRounds = kItems / 4;  // a lane takes 4 consecutive positions per round
constexpr unsigned FULL = 0xFFFFFFFFu;

struct FiberView {
    const uint32_t *idx[kMaxOrder];  // position j: mode (n + 1 + j) % N, j < N - 1
    int nm;                          // N - 1
    uint64_t nnz;
};

struct FiberCoords {
    uint32_t *idx[kMaxOrder];  // nfibs each, same positions as FiberView
};

// Head flags of the four positions p .. p + 3 held by this lane (p = q0 + 4
// lane, q0 the warp's first position of the round, q0 < nnz so the whole
// warp calls this together): bit e is set when position p + e < nnz has fiber
// coordinates that differ from its predecessor's (position 0 is a head).
// The lane's N-1 coordinate quads are left in w (16-byte loads: the arrays
// are padded to a multiple of kPadEntries, so a quad starting below nnz is
// inside them); a lane's first predecessor is the previous lane's last
// position, and lane 0 loads its own.
__device__ __forceinline__ unsigned head_quad(const FiberView &v, uint64_t q0, uint4 *w) {
    const int lane = threadIdx.x & 31;
    const uint64_t p = q0 + 4 * (uint64_t)lane;
    const bool live = p < v.nnz;
    unsigned diff = 0;  // bit e: position p + e differs from its predecessor
#pragma unroll
    for (int j = 0; j < kMaxOrder - 1; ++j) {
        if (j < v.nm) {
            w[j] = live ? *reinterpret_cast<const uint4 *>(v.idx[j] + p) : make_uint4(0u, 0u, 0u, 0u);
            uint32_t prev = __shfl_up_sync(FULL, w[j].w, 1);
            if (lane == 0) prev = q0 > 0 ? v.idx[j][q0 - 1] : ~w[j].x;
            diff |= (unsigned)(w[j].x != prev) | ((unsigned)(w[j].y != w[j].x) << 1) |
                    ((unsigned)(w[j].z != w[j].y) << 2) | ((unsigned)(w[j].w != w[j].z) << 3);
        }
    }
    if (p == 0) diff |= 1u;
    const uint64_t left = live ? v.nnz - p : 0;  // positions of the quad below nnz
    const unsigned valid = left >= 4 ? 0xFu : (1u << left) - 1u;
    return diff & valid;
}

// counts[t] = heads in tile t (kTile positions: kRounds rounds of 1024, a
// warp taking 128 consecutive positions of a round, a lane 4 of them).
__global__ void __launch_bounds__(kThreads) k_fiber_count(FiberView v, uint32_t *counts) {
    __shared__ uint32_t ws[kThreads / 32];
    const int warp = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * kTile;
    uint32_t c = 0;
    uint4 w[kMaxOrder - 1];
    for (int r = 0; r < kRounds; ++r) {
        const uint64_t q0 = base + (uint64_t)r * (kThreads * 4) + (uint64_t)warp * 128;
        if (q0 >= v.nnz) break;  // warp-uniform
        c += __popc(head_quad(v, q0, w));
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0) ws[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kThreads / 32; ++i) t += ws[i];
        counts[blockIdx.x] = t;
    }
}

// Exclusive scan of counts (one block); total -> *total.
__global__ void __launch_bounds__(1024) k_scan_counts(const uint32_t *counts, uint32_t n, uint32_t *offsets,
                                                      uint64_t *total) {
    __shared__ uint32_t wsum[32];
    __shared__ uint64_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t b = 0; b < n; b += 1024) {
        const uint32_t i = b + threadIdx.x;
        const uint32_t x = i < n ? counts[i] : 0u;
        uint32_t inc = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            uint32_t s = wsum[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, s, o);
                if (lane >= o) s += y;
            }
            wsum[lane] = s;
        }
        __syncthreads();
        const uint64_t before = carry + (warp > 0 ? wsum[warp - 1] : 0u);
        if (i < n) offsets[i] = (uint32_t)(before + inc - x);
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// fid[p] = (heads at or before p) - 1, written as 16-byte quads (zeros past
// nnz); each head writes its fiber's coordinates.  Same position layout as
// k_fiber_count; heads are ranked per round by a warp scan of the lanes'
// head counts and the block's warp totals.
__global__ void __launch_bounds__(kThreads) k_fiber_write(FiberView v, const uint32_t *offsets,
                                                          uint32_t *fid, FiberCoords out) {
    __shared__ uint32_t wsum[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t base = (uint64_t)blockIdx.x * kTile;
    uint32_t running = offsets[blockIdx.x];  // heads before this round
    uint4 w[kMaxOrder - 1];
    for (int r = 0; r < kRounds; ++r) {
        const uint64_t r0 = base + (uint64_t)r * (kThreads * 4);
        if (r0 >= v.nnz) break;  // block-uniform
        const uint64_t q0 = r0 + (uint64_t)warp * 128;
        const unsigned m = q0 < v.nnz ? head_quad(v, q0, w) : 0u;
        const uint32_t c = __popc(m);
        uint32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        uint32_t before = running, round_total = 0;
        for (int i = 0; i < kThreads / 32; ++i) {
            if (i < warp) before += wsum[i];
            round_total += wsum[i];
        }
        const uint64_t p = q0 + 4 * (uint64_t)lane;
        if (p < v.nnz) {
            uint32_t k = before + inc - c;  // heads before this lane's quad
            uint32_t f[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if ((m >> e) & 1u) {
#pragma unroll
                    for (int j = 0; j < kMaxOrder - 1; ++j) {
                        if (j < v.nm) {
                            const uint32_t x = e == 0 ? w[j].x : e == 1 ? w[j].y : e == 2 ? w[j].z : w[j].w;
                            out.idx[j][k] = x;
                        }
                    }
                    ++k;
                }
                f[e] = p + e < v.nnz ? k - 1u : 0u;
            }
            *reinterpret_cast<uint4 *>(fid + p) = make_uint4(f[0], f[1], f[2], f[3]);
        }
        running += round_total;
        __syncthreads();  // wsum is rewritten next round
    }
}

// TTV: y(f) = sum over fiber f of val * v(i_n).  Each warp takes a chunk of
// kTtvChunk consecutive entries in rounds of 128: lane l holds entries
// 4l .. 4l + 3 of the round (16-byte loads of fid, i_n and val; the next
// round's are loaded while this one is summed).  Fiber ids are
// non-decreasing, so each lane first sums its own entries fiber by fiber:
// fibers that begin and end inside the lane are complete; the lane's first
// fiber (head) may continue from the lanes before it and its last (tail)
// into the lanes after it.  A segmented inclusive scan over the lanes'
// tail sums then joins the pieces, and the fiber open at lane 31 is carried
// into the next round.  A complete fiber is stored plainly unless it is the
// chunk's first or last fiber (those may be shared with the neighbouring
// chunks), which is added atomically.  y must be zero-filled.
constexpr int kTtvChunk = 2048;

template <typename A>
__device__ __forceinline__ void ttv_put(A *y, uint32_t f, A x, uint32_t first_f, uint32_t last_f) {
    if (f == first_f || f == last_f)
        atomicAdd(&y[f], x);
    else
        y[f] = x;
}

template <typename T, typename A>
__global__ void __launch_bounds__(256) k_ttv(const uint32_t *fid, const uint32_t *in, const float *val,
                                             const T *v, A *y, uint64_t nnz) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t c0 = warp * kTtvChunk;
    if (c0 >= nnz) return;
    const uint64_t c1 = min(nnz, c0 + kTtvChunk);
    const uint32_t first_f = fid[c0], last_f = fid[c1 - 1];
    // arrays are padded to a multiple of 4 entries, so a 16-byte load at a
    // position below nnz stays inside them; entries at or past c1 are masked
    uint4 nf, ni;
    float4 nv;
    auto load = [&](uint64_t r0) {
        const uint64_t p = r0 + 4 * (uint64_t)lane;
        if (p < c1) {
            nf = *reinterpret_cast<const uint4 *>(fid + p);
            ni = *reinterpret_cast<const uint4 *>(in + p);
            nv = *reinterpret_cast<const float4 *>(val + p);
        }
    };
    load(c0);
    uint32_t carry_f = kNoRow;  // fiber open at the end of the previous round
    A carry_t = 0;
    for (uint64_t r0 = c0; r0 < c1; r0 += 128) {
        const uint64_t p = r0 + 4 * (uint64_t)lane;
        uint32_t f[4] = {nf.x, nf.y, nf.z, nf.w};
        const uint32_t ix[4] = {ni.x, ni.y, ni.z, ni.w};
        const float xv[4] = {nv.x, nv.y, nv.z, nv.w};
        const bool last_round = r0 + 128 >= c1;
        if (!last_round) load(r0 + 128);
        A t[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool ok = p + k < c1;
            if (!ok) f[k] = kNoRow;  // masked entries form a trailing pseudo-fiber, never written
            t[k] = ok ? (A)xv[k] * (A)v[ix[k]] : (A)0;
        }
        // this lane's entries, fiber by fiber
        const uint32_t hf = f[0], tf = f[3];
        A run = t[0], head = 0;
        bool whole = true;  // all four entries in one fiber
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            if (f[k] != f[k - 1]) {
                if (whole) {
                    head = run;
                    whole = false;
                } else if (f[k - 1] != kNoRow) {
                    ttv_put(y, f[k - 1], run, first_f, last_f);  // begins and ends in this lane
                }
                run = t[k];
            } else {
                run += t[k];
            }
        }
        if (lane == 0 && carry_f != kNoRow) {
            if (carry_f == hf) {  // continues the fiber open at the previous round's end
                if (whole)
                    run += carry_t;
                else
                    head += carry_t;
            } else {  // that fiber ended with the previous round
                ttv_put(y, carry_f, carry_t, first_f, last_f);
            }
        }
        // segmented inclusive scan of the tail sums over lanes; a lane starts
        // a segment unless it is wholly inside the previous lane's tail fiber
        const uint32_t tf_prev = __shfl_up_sync(FULL, tf, 1);
        bool B = lane == 0 || !whole || tf_prev != tf;
        A S = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const A Sp = __shfl_up_sync(FULL, S, o);
            const bool Bp = __shfl_up_sync(FULL, (int)B, o) != 0;
            if (lane >= o) {
                if (!B) S += Sp;
                B = B || Bp;
            }
        }
        const A S_prev = __shfl_up_sync(FULL, S, 1);
        const uint32_t hf_next = __shfl_down_sync(FULL, hf, 1);
        if (!whole) {
            if (lane > 0 && tf_prev == hf) head += S_prev;
            if (hf != kNoRow) ttv_put(y, hf, head, first_f, last_f);
        }
        // the tail is complete unless the next lane continues it (lane 31:
        // unless the next round may)
        const bool tail_done = lane < 31 ? hf_next != tf : last_round;
        if (tail_done && tf != kNoRow) ttv_put(y, tf, S, first_f, last_f);
        carry_f = __shfl_sync(FULL, tf, 31);
        carry_t = __shfl_sync(FULL, S, 31);
    }
}

int bits_for(uint64_t dim) {
    int b = 0;
    while (b < 64 && (dim - 1) >> b) ++b;
    return b;
}

}  // namespace

void free_fibers(FiberTable &F) {
    dev_free(F.block);
    dev_free(F.cblock);
    F = FiberTable{};
}

pasta_status build_fibers(pasta_coo_s *X, int n, cudaStream_t s) {
    FiberTable &F = X->fibers[n];
    if (F.present) return PASTA_OK;
    const int N = X->order;
    const int m = (n + 1) % N;
    const StoredCopy &c = X->sorted[m];
    if (!c.present) {
        set_error("mode-%d fibers need the mode-%d sorted copy (pasta_coo_sort_by_mode)", n, m);
        return PASTA_ERR_NOT_SORTED;
    }
    int bits = 0;
    for (int k = 0; k < N; ++k)
        if (k != n) bits += bits_for(X->dims[k]);
    if (bits > 64) {
        set_error("mode-%d fibers: the other modes need %d key bits (at most 64 supported)", n, bits);
        return PASTA_ERR_UNSUPPORTED;
    }
    FiberView v{};
    v.nm = N - 1;
    v.nnz = X->nnz;
    for (int j = 0; j < N - 1; ++j) v.idx[j] = c.idx[(n + 1 + j) % N];

    const uint32_t ntiles = (uint32_t)std::max<uint64_t>(1, (X->nnz + kTile - 1) / kTile);
    // fid (padded like a stored array, zero tail) + per-tile counts/offsets + total
    const size_t fid_b = (size_t)X->nnz_pad * 4;
    const size_t cnt_b = ((size_t)ntiles * 4 + 255) & ~(size_t)255;
    char *blk = nullptr;
    cudaError_t e = dev_malloc((void **)&blk, fid_b + 2 * cnt_b + 256, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("cudaMalloc for the mode-%d fiber table failed", n);
        return PASTA_ERR_NOMEM;
    }
    F.block = blk;
    F.fid = reinterpret_cast<uint32_t *>(blk);
    uint32_t *counts = reinterpret_cast<uint32_t *>(blk + fid_b);
    uint32_t *offsets = reinterpret_cast<uint32_t *>(blk + fid_b + cnt_b);
    uint64_t *total = reinterpret_cast<uint64_t *>(blk + fid_b + 2 * cnt_b);
    uint64_t nfibs = 0;
    {
        // zero tail of fid: k_fiber_write writes every quad that starts below nnz
        const size_t written = (size_t)((X->nnz + 3) / 4) * 16;
        e = cudaMemsetAsync(reinterpret_cast<char *>(F.fid) + written, 0, fid_b - written, s);
    }
    if (e == cudaSuccess && X->nnz > 0) {
        k_fiber_count<<<ntiles, kThreads, 0, s>>>(v, counts);
        k_scan_counts<<<1, 1024, 0, s>>>(counts, ntiles, offsets, total);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&nfibs, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e == cudaSuccess && nfibs > 0) {
        const size_t per = ((size_t)nfibs * 4 + 255) & ~(size_t)255;
        e = dev_malloc(&F.cblock, per * (size_t)(N - 1), s);
        if (e == cudaSuccess) {
            FiberCoords out{};
            for (int j = 0; j < N - 1; ++j) {
                F.coords[j] = reinterpret_cast<uint32_t *>(static_cast<char *>(F.cblock) + per * j);
                out.idx[j] = F.coords[j];
            }
            k_fiber_write<<<ntiles, kThreads, 0, s>>>(v, offsets, F.fid, out);
            e = cudaGetLastError();
        }
    }
    if (e != cudaSuccess) {
        pasta_status st = cuda_fail(e, "fiber table");
        cudaStreamSynchronize(s);
        free_fibers(F);
        return st;
    }
    F.nfibs = nfibs;
    F.present = true;
    return PASTA_OK;
}

pasta_status launch_ttm(pasta_coo_s *X, int n, const void *U, pasta_dtype dt, int R, void *Y,
                        cudaStream_t s) {
    const FiberTable &F = X->fibers[n];
    const int m = (n + 1) % X->order;
    const StoredCopy &c = X->sorted[m];
    if (R == 1) {  // TTV
        const size_t acc = dt == PASTA_F64 ? 8 : 4;
        PASTA_CUDA(cudaMemsetAsync(Y, 0, F.nfibs * acc, s));
        if (X->nnz == 0) return PASTA_OK;
        const uint64_t warps = (X->nnz + kTtvChunk - 1) / kTtvChunk;
        const int blocks = (int)((warps + 7) / 8);
        switch (dt) {
            case PASTA_F32:
                k_ttv<float, float><<<blocks, 256, 0, s>>>(F.fid, c.idx[n], c.val, static_cast<const float *>(U),
                                                            static_cast<float *>(Y), X->nnz);
                break;
            case PASTA_BF16:
                k_ttv<__nv_bfloat16, float><<<blocks, 256, 0, s>>>(
                    F.fid, c.idx[n], c.val, static_cast<const __nv_bfloat16 *>(U), static_cast<float *>(Y), X->nnz);
                break;
            case PASTA_F16:
                k_ttv<__half, float><<<blocks, 256, 0, s>>>(F.fid, c.idx[n], c.val, static_cast<const __half *>(U),
                                                             static_cast<float *>(Y), X->nnz);
                break;
            case PASTA_F64:
                k_ttv<double, double><<<blocks, 256, 0, s>>>(F.fid, c.idx[n], c.val, static_cast<const double *>(U),
                                                              static_cast<double *>(Y), X->nnz);
                break;
        }
        PASTA_CUDA(cudaGetLastError());
        return PASTA_OK;
    }
    // the order-2 view (fiber, i_n) of the mode-(n+1) sorted copy
    pasta_coo_s V;
    V.order = 2;
    V.dims[0] = F.nfibs;
    V.dims[1] = X->dims[n];
    V.nnz = X->nnz;
    V.nnz_pad = X->nnz_pad;
    V.device = X->device;
    V.num_sms = X->num_sms;
    StoredCopy vc;
    vc.idx[0] = F.fid;
    vc.idx[1] = c.idx[n];
    vc.val = c.val;
    vc.present = true;
    const void *Us[2] = {nullptr, U};
    return launch_mttkrp(&V, vc, Us, dt, 0, R, Y, s, /*every_row_touched=*/true);
}

}  // namespace pasta
