// Mode-order sort of the COO stream (arXiv:1902.03317, Sec. 5.2.2: tensors
// are sorted lexicographically "in the order of mode 1 > 2 > 3"; Sec. 2.3:
// each iteration order wants its own sorted copy).
//
// The key of entry m is its coordinate in cyclic mode order starting at the
// sorted mode, each mode taking ceil(log2(dims[k])) bits, cut to the leading
// 64 bits.  A stable least-significant-digit radix sort (8-bit digits) of
// (key, entry number) pairs gives the permutation; a final pass writes the
// sorted SoA copy, decoding every index the key holds whole from the sorted
// keys and gathering only the rest (and the values) through the permutation.
// Equal keys keep creation order, so the result is unique.
//
// Radix pass = histogram per 4096-entry tile (digit-major table), exclusive
// scan of each digit's row over tiles, stable scatter: inside a tile the
// entries are ranked round by round (256 at a time) with __match_any_sync
// peer groups and per-warp digit counts, which keeps storage order.
#include <algorithm>

#include "pasta_internal.cuh"

namespace pasta {
namespace {

constexpr int kThreads = 256;
constexpr int kRounds = 16;
constexpr int kTile = kThreads * kRounds;
constexpr unsigned FULL = 0xFFFFFFFFu;

struct KeySpec {
    int order;
    int mode[kMaxOrder];  // mode at cyclic position p
    int shl[kMaxOrder];   // contribution = (idx >> shr) << shl
    int shr[kMaxOrder];
    int use[kMaxOrder];   // 0: this position contributes nothing
    int final_shift;      // key >>= final_shift (right-aligns the used bits)
};

__global__ void k_make_keys(CooView v, KeySpec ks, uint64_t *keys, uint32_t *perm) {
    for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < v.nnz;
         m += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t key = 0;
#pragma unroll
        for (int p = 0; p < kMaxOrder; ++p) {
            if (p < ks.order && ks.use[p]) {
                const uint64_t ix = v.idx[ks.mode[p]][m];
                key |= (ix >> ks.shr[p]) << ks.shl[p];
            }
        }
        keys[m] = ks.final_shift >= 64 ? 0 : (key >> ks.final_shift);
        perm[m] = (uint32_t)m;
    }
}

// hist[d * ntiles + tile] = number of entries of `tile` whose digit is d.
__global__ void __launch_bounds__(kThreads) k_hist(const uint64_t *keys, uint64_t n, int shift,
                                                   uint32_t ntiles, uint32_t *hist) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kTile;
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < kRounds; ++r) {
        const uint64_t i = base + (uint64_t)r * kThreads + threadIdx.x;
        const bool valid = i < n;
        const uint32_t d = valid ? (uint32_t)((keys[i] >> shift) & 255u) : 0u;
        const unsigned peers = __match_any_sync(FULL, valid ? d : 256u + lane);
        if (valid && (peers & ((1u << lane) - 1u)) == 0) atomicAdd(&cnt[d], __popc(peers));
    }
    __syncthreads();
    hist[(uint64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive scan of row d (one block per digit) of the digit-major table;
// totals[d] receives the row sum.
__global__ void __launch_bounds__(1024) k_rowscan(uint32_t *hist, uint32_t ntiles,
                                                  uint32_t *totals) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    uint32_t *row = hist + (uint64_t)blockIdx.x * ntiles;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t b = 0; b < ntiles; b += 1024) {
        const uint32_t i = b + threadIdx.x;
        const uint32_t x = i < ntiles ? row[i] : 0u;
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
            wsum[lane] = s;  // inclusive over warps
        }
        __syncthreads();
        const uint32_t before = (warp > 0 ? wsum[warp - 1] : 0u) + carry;
        if (i < ntiles) row[i] = before + inc - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = carry;
}

__global__ void __launch_bounds__(kThreads) k_scatter(const uint64_t *kin, const uint32_t *vin,
                                                      uint64_t *kout, uint32_t *vout, uint64_t n,
                                                      int shift, uint32_t ntiles,
                                                      const uint32_t *hist,
                                                      const uint32_t *totals) {
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_w[kThreads / 32][256];
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    // Digit bases: exclusive scan of the digit totals (256 entries).
    {
        uint32_t x = totals[t];
        uint32_t inc = x;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[0][warp] = inc;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += s_w[0][w];
        s_base[t] = before + inc - x + hist[(uint64_t)t * ntiles + blockIdx.x];
        __syncthreads();
    }
    const uint64_t base = (uint64_t)blockIdx.x * kTile;
    for (int r = 0; r < kRounds; ++r) {
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) s_w[w][t] = 0;
        __syncthreads();
        const uint64_t i = base + (uint64_t)r * kThreads + t;
        const bool valid = i < n;
        const uint64_t key = valid ? kin[i] : 0ull;
        const uint32_t val = valid ? vin[i] : 0u;
        const uint32_t d = (uint32_t)((key >> shift) & 255u);
        const unsigned peers = __match_any_sync(FULL, valid ? d : 256u + lane);
        const uint32_t below = __popc(peers & ((1u << lane) - 1u));
        if (valid && below == 0) s_w[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            const uint32_t c = s_w[w][t];
            s_w[w][t] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            const uint64_t pos = (uint64_t)s_base[d] + s_w[warp][d] + below;
            kout[pos] = key;
            vout[pos] = val;
        }
        __syncthreads();
        s_base[t] += run;
        __syncthreads();
    }
}

struct GatherDst {
    uint32_t *idx[kMaxOrder];
    float *val;
    // Mode k whose index sits whole in the sorted key: decode it from the key
    // (shift[k] >= 0, mask[k]); else (shift[k] < 0) gather it through perm.
    int shift[kMaxOrder];
    uint32_t mask[kMaxOrder];
};

// Writes the sorted copy: indices held whole by the key are decoded from the
// sorted keys (coalesced), the rest and the values are gathered through the
// permutation (one random 4-byte read each).
__global__ void k_gather(CooView src, const uint32_t *perm, const uint64_t *keys, GatherDst dst) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < src.nnz;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t o = perm[p];
        const uint64_t key = keys[p];
#pragma unroll
        for (int k = 0; k < kMaxOrder; ++k) {
            if (k >= src.order) continue;
            dst.idx[k][p] = dst.shift[k] >= 0 ? (uint32_t)(key >> dst.shift[k]) & dst.mask[k]
                                              : src.idx[k][o];
        }
        dst.val[p] = src.val[o];
    }
}

int bits_for(uint64_t dim) {
    int b = 0;
    while (b < 64 && (dim - 1) >> b) ++b;
    return b;
}

}  // namespace

pasta_status sort_copy(pasta_coo_s *X, int mode, cudaStream_t s) {
    StoredCopy &dst = X->sorted[mode];
    const uint64_t n = X->nnz;
    if (n == 0) return PASTA_OK;

    KeySpec ks{};
    ks.order = X->order;
    int used = 0;
    for (int p = 0; p < X->order; ++p) {
        const int k = (mode + p) % X->order;
        const int b = bits_for(X->dims[k]);
        ks.mode[p] = k;
        if (b == 0 || used >= 64) continue;
        ks.use[p] = 1;
        if (used + b <= 64) {
            ks.shl[p] = 64 - used - b;
            ks.shr[p] = 0;
            used += b;
        } else {
            ks.shl[p] = 0;
            ks.shr[p] = b - (64 - used);
            used = 64;
        }
    }
    ks.final_shift = 64 - used;
    const int passes = (used + 7) / 8;

    const uint32_t ntiles = (uint32_t)((n + kTile - 1) / kTile);
    uint64_t *keys = nullptr;
    uint32_t *tmpv = nullptr, *hist = nullptr;
    const size_t hist_n = (size_t)256 * ntiles + 256;
    PASTA_CUDA(cudaMallocAsync((void **)&keys, 2 * n * sizeof(uint64_t), s));
    cudaError_t e1 = cudaMallocAsync((void **)&tmpv, n * sizeof(uint32_t), s);
    cudaError_t e2 = cudaMallocAsync((void **)&hist, hist_n * sizeof(uint32_t), s);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaFreeAsync(keys, s);
        if (tmpv) cudaFreeAsync(tmpv, s);
        if (hist) cudaFreeAsync(hist, s);
        set_error("cudaMallocAsync of sort scratch failed");
        return PASTA_ERR_NOMEM;
    }
    uint64_t *kb[2] = {keys, keys + n};
    uint32_t *vb[2];
    vb[passes % 2] = dst.perm;  // the last pass writes into the copy's perm
    vb[1 - passes % 2] = tmpv;
    uint32_t *totals = hist + (size_t)256 * ntiles;

    const CooView src = view_of(X, X->orig);
    const int gblocks = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)X->num_sms * 16);
    pasta_status st = PASTA_OK;
    k_make_keys<<<gblocks, 256, 0, s>>>(src, ks, kb[0], vb[0]);
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_hist<<<ntiles, kThreads, 0, s>>>(kb[p % 2], n, shift, ntiles, hist);
        k_rowscan<<<256, 1024, 0, s>>>(hist, ntiles, totals);
        k_scatter<<<ntiles, kThreads, 0, s>>>(kb[p % 2], vb[p % 2], kb[(p + 1) % 2],
                                              vb[(p + 1) % 2], n, shift, ntiles, hist, totals);
    }
    GatherDst gd{};
    for (int k = 0; k < X->order; ++k) {
        gd.idx[k] = dst.idx[k];
        gd.shift[k] = -1;
    }
    for (int p = 0; p < X->order; ++p) {
        const int k = ks.mode[p];
        const int b = bits_for(X->dims[k]);
        if (b == 0) {  // a mode of size 1: every index is 0
            gd.shift[k] = 0;
            gd.mask[k] = 0u;
        } else if (ks.use[p] && ks.shr[p] == 0) {  // held whole, right-aligned by final_shift
            gd.shift[k] = ks.shl[p] - ks.final_shift;
            gd.mask[k] = b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u);
        }
    }
    gd.val = dst.val;
    k_gather<<<gblocks, 256, 0, s>>>(src, dst.perm, kb[passes % 2], gd);
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) st = cuda_fail(le, "sort kernels");
    cudaFreeAsync(keys, s);
    cudaFreeAsync(tmpv, s);
    cudaFreeAsync(hist, s);
    return st;
}

}  // namespace pasta
