// Mode-order sort of the COO stream (arXiv:1902.03317, Sec. 5.2.2: the
// tensors are sorted lexicographically, the first mode most significant;
// Sec. 2.3: each iteration order wants its own sorted copy).
//
// The key of entry m is its coordinate in cyclic mode order starting at the
// sorted mode, each mode taking ceil(log2(dims[k])) bits, cut to the leading
// 64 bits.  A stable least-significant-digit radix sort (digits of up to 9 bits) of
// (key, payload) pairs orders the entries; equal keys keep creation order, so
// the result is unique.  When the key holds every index whole (the common
// case: the modes' bits fit 64), the payload is the value itself and the
// indices are decoded from the sorted keys, so nothing is gathered; the
// permutation (sorted position -> creation-order entry), which no kernel
// needs, is sorted for only when a caller asks for it.  Otherwise the
// payload is the entry number and a final pass gathers the indices the key
// does not hold, and the values, through the resulting permutation.
//
// Digits have up to 9 bits, balanced over the fewest passes.
// Radix pass = histogram per 4096-entry tile (digit-major table), exclusive
// scan of each digit's row over tiles, stable scatter: each warp ranks its
// 512-entry sub-tile by digit in storage order, the tile is reordered by
// digit in shared memory and written out in runs of equal digit.
#include <algorithm>

#include "host_copy.cuh"
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

// keys[m] = the key of entry m; payload[m] = its value's bits (payload_val)
// or its creation-order number.  A thread takes four consecutive entries:
// 16-byte loads of each index array and the values (stored arrays are
// 16-byte aligned and padded past nnz), 16-byte stores where all four are
// real entries.
__global__ void k_make_keys(CooView v, KeySpec ks, uint64_t *keys, uint32_t *payload, bool payload_val) {
    const uint64_t n4 = (v.nnz + 3) / 4;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t m = 4 * q;
        uint64_t key[4] = {0, 0, 0, 0};
#pragma unroll
        for (int p = 0; p < kMaxOrder; ++p) {
            if (p < ks.order && ks.use[p]) {
                const uint4 ix = *reinterpret_cast<const uint4 *>(v.idx[ks.mode[p]] + m);
                key[0] |= ((uint64_t)ix.x >> ks.shr[p]) << ks.shl[p];
                key[1] |= ((uint64_t)ix.y >> ks.shr[p]) << ks.shl[p];
                key[2] |= ((uint64_t)ix.z >> ks.shr[p]) << ks.shl[p];
                key[3] |= ((uint64_t)ix.w >> ks.shr[p]) << ks.shl[p];
            }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) key[e] = ks.final_shift >= 64 ? 0 : (key[e] >> ks.final_shift);
        uint4 pl;
        if (payload_val) {
            const float4 x = *reinterpret_cast<const float4 *>(v.val + m);
            pl = make_uint4(__float_as_uint(x.x), __float_as_uint(x.y), __float_as_uint(x.z), __float_as_uint(x.w));
        } else {
            pl = make_uint4((uint32_t)m, (uint32_t)m + 1u, (uint32_t)m + 2u, (uint32_t)m + 3u);
        }
        if (m + 3 < v.nnz) {
            reinterpret_cast<ulonglong2 *>(keys + m)[0] = make_ulonglong2(key[0], key[1]);
            reinterpret_cast<ulonglong2 *>(keys + m)[1] = make_ulonglong2(key[2], key[3]);
            *reinterpret_cast<uint4 *>(payload + m) = pl;
        } else {
            const uint32_t pv[4] = {pl.x, pl.y, pl.z, pl.w};
            for (int e = 0; e < 4 && m + e < v.nnz; ++e) {
                keys[m + e] = key[e];
                payload[m + e] = pv[e];
            }
        }
    }
}

// A tile is kThreads x kItems entries; warp w of its block owns the
// contiguous sub-tile [w * kWarpSpan, (w + 1) * kWarpSpan), read in rounds
// of 32 consecutive entries.  Both radix kernels use this arrangement, so
// every entry is loaded by one coalesced 8-byte access per lane.
constexpr int kWarpsPerBlock = kThreads / 32;
constexpr int kItems = kTile / kThreads;
constexpr int kWarpSpan = 32 * kItems;
constexpr int kMaxBins = 512;  // digits of up to 9 bits
static_assert(kWarpSpan <= 65536, "warp ranks are packed as 16-bit values");

// hist[d * ntiles + tile] = number of entries of `tile` whose digit
// ((key >> shift) & mask, below BINS) is d.  Plain shared atomics per entry
// (one sub-histogram per warp); measured faster than aggregating equal digits
// with __match_any_sync first.
template <int BINS>
__global__ void __launch_bounds__(kThreads) k_hist(const uint64_t *keys, uint64_t n, int shift,
                                                   uint32_t mask, uint32_t ntiles, uint32_t *hist) {
    __shared__ uint32_t cnt[kWarpsPerBlock][BINS];
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    for (int i = t; i < kWarpsPerBlock * BINS; i += kThreads) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * kTile + (uint64_t)warp * kWarpSpan + lane;
    const int64_t rem = (int64_t)n - (int64_t)base;  // entry j is real iff 32 j < rem
    const uint64_t *kp = keys + base;
    uint64_t k[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) k[j] = 32 * j < rem ? kp[32 * j] : 0ull;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const uint32_t d = (uint32_t)(k[j] >> shift) & mask;
        if (32 * j < rem) atomicAdd(&cnt[warp][d], 1u);
    }
    __syncthreads();
    for (int d = t; d < BINS; d += kThreads) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < kWarpsPerBlock; ++w) c += cnt[w][d];
        hist[(uint64_t)d * ntiles + blockIdx.x] = c;
    }
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

// Shared memory of k_scatter: the tile's keys and values in digit order.
constexpr size_t kScatterSmem = (size_t)kTile * (sizeof(uint64_t) + sizeof(uint32_t));

// Exclusive scan over the block of one value per thread (thread order);
// every thread must call it.  wsum: kWarpsPerBlock words of shared memory.
__device__ __forceinline__ uint32_t block_exclusive(uint32_t x, uint32_t *wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, inc, o);
        if (lane >= o) inc += y;
    }
    __syncthreads();  // wsum may still be read from a previous call
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    return before + inc - x;
}

// Stable scatter of one tile.  (1) Each warp ranks its sub-tile round by
// round: __match_any_sync finds the lanes of equal digit (measured faster
// here than a shared-memory mask word per digit), the lowest of them reads
// and advances the warp's running count of that digit, so an entry's warp
// rank counts the equal digits before it in storage order.  (2) Per
// digit, warp offsets and the tile-local start follow from those counts.
// (3) The tile is reordered by digit in shared memory, and (4) written out in
// that order: consecutive threads write consecutive positions of one digit's
// output range, so the writes coalesce.  Thread t owns digits t * PER ...
// t * PER + PER - 1 in the per-digit steps.
template <int BINS>
__global__ void __launch_bounds__(kThreads, 2)
    k_scatter(const uint64_t *kin, const uint32_t *vin, uint64_t *kout, uint32_t *vout,
              uint64_t n, int shift, uint32_t mask, uint32_t ntiles, const uint32_t *hist,
              const uint32_t *totals) {
    constexpr int PER = BINS / kThreads;
    static_assert(PER >= 1 && PER * kThreads == BINS, "BINS must be a multiple of the block");
    extern __shared__ __align__(16) unsigned char sm_raw[];
    uint64_t *sk = reinterpret_cast<uint64_t *>(sm_raw);
    uint32_t *sv = reinterpret_cast<uint32_t *>(sm_raw + (size_t)kTile * sizeof(uint64_t));
    __shared__ uint32_t wcnt[kWarpsPerBlock][BINS];  // per-warp counts, then warp offsets
    __shared__ uint32_t lstart[BINS];                // tile-local start of each digit
    __shared__ uint32_t gbase[BINS];                 // output position of that start
    __shared__ uint32_t wsum[kWarpsPerBlock];
    const int t = threadIdx.x;
    const int lane = t & 31;
    const int warp = t >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int i = t; i < kWarpsPerBlock * BINS; i += kThreads) (&wcnt[0][0])[i] = 0;

    const uint64_t tbase = (uint64_t)blockIdx.x * kTile;
    const int tlen = (int)min((uint64_t)kTile, n - tbase);
    const uint64_t base = tbase + (uint64_t)warp * kWarpSpan + lane;
    const int64_t rem = (int64_t)n - (int64_t)base;  // entry j is real iff 32 j < rem
    const uint64_t *kp = kin + base;
    const uint32_t *vp = vin + base;
    uint64_t k[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) k[j] = 32 * j < rem ? kp[32 * j] : 0ull;
    // Exclusive scan of the digit totals (digit base of this pass) plus this
    // tile's scanned count: where the tile's first entry of each digit goes.
    {
        uint32_t x[PER], sum = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            x[u] = totals[t * PER + u];
            sum += x[u];
        }
        uint32_t ex = block_exclusive(sum, wsum);  // its barriers also order the zeroing above
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int d = t * PER + u;
            gbase[d] = ex + hist[(uint64_t)d * ntiles + blockIdx.x];
            ex += x[u];
        }
    }
    // (1) warp ranks (< kWarpSpan, two per register)
    uint32_t r[kItems / 2];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        const bool valid = 32 * j < rem;
        const uint32_t d = (uint32_t)(k[j] >> shift) & mask;
        const unsigned peers = __match_any_sync(FULL, valid ? d : BINS + lane);
        const int leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (valid && lane == leader) {
            old = wcnt[warp][d];
            wcnt[warp][d] = old + __popc(peers);
        }
        const uint32_t rank = __shfl_sync(FULL, old, leader) + __popc(peers & lt);
        if (j & 1)
            r[j / 2] |= rank << 16;
        else
            r[j / 2] = rank;
        __syncwarp();
    }
    // the values are loaded now, so the ranking holds fewer registers
    uint32_t v[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) v[j] = 32 * j < rem ? vp[32 * j] : 0u;
    __syncthreads();
    // (2) warp offsets per digit, then the tile-local digit starts
    {
        uint32_t tot[PER], sum = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int d = t * PER + u;
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < kWarpsPerBlock; ++w) {
                const uint32_t c = wcnt[w][d];
                wcnt[w][d] = run;
                run += c;
            }
            tot[u] = run;
            sum += run;
        }
        uint32_t ex = block_exclusive(sum, wsum);
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            lstart[t * PER + u] = ex;
            ex += tot[u];
        }
    }
    __syncthreads();
    // (3) reorder the tile by digit in shared memory
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        if (32 * j < rem) {
            const uint32_t d = (uint32_t)(k[j] >> shift) & mask;
            const uint32_t lp = lstart[d] + wcnt[warp][d] + ((r[j / 2] >> (16 * (j & 1))) & 0xFFFFu);
            sk[lp] = k[j];
            sv[lp] = v[j];
        }
    }
    __syncthreads();
    // (4) coalesced write-out
#pragma unroll 4
    for (int q = t; q < tlen; q += kThreads) {
        const uint64_t key = sk[q];
        const uint32_t d = (uint32_t)(key >> shift) & mask;
        const uint64_t gp = (uint64_t)gbase[d] + (uint32_t)(q - (int)lstart[d]);
        kout[gp] = key;
        vout[gp] = sv[q];
    }
}

struct GatherDst {
    uint32_t *idx[kMaxOrder];
    float *val;
    // Mode k whose index sits whole in the sorted key: decode it from the key
    // (shift[k] >= 0, mask[k]); else (shift[k] < 0) gather it through perm.
    int shift[kMaxOrder];
    uint32_t mask[kMaxOrder];
    int order;
};

// Writes the sorted copy: indices held whole by the key are decoded from the
// sorted keys (coalesced), the rest and the values are gathered through the
// permutation (one random 4-byte read each).  Each thread takes kGatherItems
// positions a grid stride apart and issues all their loads before any use,
// so several random reads are in flight per thread.
constexpr int kGatherItems = 4;

__global__ void __launch_bounds__(256) k_gather(CooView src, const uint32_t *perm,
                                                const uint64_t *keys, GatherDst dst) {
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t p0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p0 < src.nnz;
         p0 += step * kGatherItems) {
        uint32_t o[kGatherItems];
        uint64_t key[kGatherItems];
#pragma unroll
        for (int j = 0; j < kGatherItems; ++j) {
            const uint64_t p = p0 + (uint64_t)j * step;
            o[j] = p < src.nnz ? perm[p] : 0u;
            key[j] = p < src.nnz ? keys[p] : 0ull;
        }
        float v[kGatherItems];
#pragma unroll
        for (int j = 0; j < kGatherItems; ++j) v[j] = src.val[o[j]];
#pragma unroll
        for (int k = 0; k < kMaxOrder; ++k) {
            if (k >= src.order) continue;
            uint32_t x[kGatherItems];
#pragma unroll
            for (int j = 0; j < kGatherItems; ++j)
                x[j] = dst.shift[k] >= 0 ? (uint32_t)(key[j] >> dst.shift[k]) & dst.mask[k]
                                         : src.idx[k][o[j]];
#pragma unroll
            for (int j = 0; j < kGatherItems; ++j) {
                const uint64_t p = p0 + (uint64_t)j * step;
                if (p < src.nnz) dst.idx[k][p] = x[j];
            }
        }
#pragma unroll
        for (int j = 0; j < kGatherItems; ++j) {
            const uint64_t p = p0 + (uint64_t)j * step;
            if (p < src.nnz) dst.val[p] = v[j];
        }
    }
}

// Writes the sorted copy's indices when the key holds every one of them
// (the values arrived as the sort's payload).
__global__ void k_decode(const uint64_t *keys, uint64_t n, int order, GatherDst dst) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t key = keys[p];
#pragma unroll
        for (int k = 0; k < kMaxOrder; ++k)
            if (k < order) dst.idx[k][p] = (uint32_t)(key >> dst.shift[k]) & dst.mask[k];
    }
}

// ----------------------------------------------------------- two runs ---

// Number of elements of A among the first d of the stable merge of sorted
// A and B (ties: A first): the first i in [max(0, d - nB), min(d, nA)] whose
// A[i] is above B[d - i - 1].
template <typename KA, typename KB>
__device__ __forceinline__ uint64_t merge_split(KA A, uint64_t nA, KB B, uint64_t nB, uint64_t d) {
    uint64_t lo = d > nB ? d - nB : 0;
    uint64_t hi = d < nA ? d : nA;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) / 2;
        if (A[mid] <= B[d - mid - 1])
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Dynamic shared memory of k_merge: a tile of input pairs, then the
// tile merged.
constexpr size_t kMergeSmem = 2 * (size_t)kTile * (sizeof(uint64_t) + sizeof(uint32_t));

// Stable merge of the sorted runs (kA, vA) and (kB, vB) (ties: A first, A
// holding the earlier entries).  DECODE: written as the sorted copy, position
// p getting the indices decoded from its key and the value whose bits are its
// payload; else written as merged pairs (kO, vO).
// Block b writes positions [b kTile, (b + 1) kTile): split[b] and
// split[b + 1] (k_merge_splits) say where that range starts and ends in A and
// B; it loads both pieces into shared memory, each thread merges kItems
// outputs from its own split point, and the block writes the tile out in
// order.
// split[b] = merge_split(A, B, min(b kTile, nA + nB)) for b in [0, nblocks]:
// where each merge block's output range starts in A (one thread per block
// boundary, so the searches' dependent loads overlap across threads).
__global__ void k_merge_splits(const uint64_t *kA, uint64_t nA, const uint64_t *kB, uint64_t nB, uint64_t nblocks,
                               uint64_t *split) {
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nblocks) return;
    const uint64_t d = min(b * (uint64_t)kTile, nA + nB);
    split[b] = merge_split(kA, nA, kB, nB, d);
}

template <bool DECODE>
__global__ void __launch_bounds__(kThreads) k_merge(const uint64_t *kA, const uint32_t *vA, uint64_t nA,
                                                    const uint64_t *kB, const uint32_t *vB, uint64_t nB,
                                                    const uint64_t *split, GatherDst dst, uint64_t *kO, uint32_t *vO) {
    extern __shared__ __align__(16) unsigned char sm_raw[];
    uint64_t *ik = reinterpret_cast<uint64_t *>(sm_raw);
    uint32_t *iv = reinterpret_cast<uint32_t *>(sm_raw + (size_t)kTile * sizeof(uint64_t));
    uint64_t *ok = reinterpret_cast<uint64_t *>(sm_raw + (size_t)kTile * (sizeof(uint64_t) + sizeof(uint32_t)));
    uint32_t *ov = reinterpret_cast<uint32_t *>(sm_raw + (size_t)kTile * (2 * sizeof(uint64_t) + sizeof(uint32_t)));
    const int t = threadIdx.x;
    const uint64_t n = nA + nB;
    const uint64_t d0 = (uint64_t)blockIdx.x * kTile;
    const uint64_t d1 = min(n, d0 + kTile);
    const uint64_t i0 = split[blockIdx.x], i1 = split[blockIdx.x + 1];
    const int lenA = (int)(i1 - i0);
    const int len = (int)(d1 - d0);
    const int lenB = len - lenA;
    const uint64_t j0 = d0 - i0;
    for (int q = t; q < lenA; q += kThreads) {
        ik[q] = kA[i0 + q];
        iv[q] = vA[i0 + q];
    }
    for (int q = t; q < lenB; q += kThreads) {
        ik[lenA + q] = kB[j0 + q];
        iv[lenA + q] = vB[j0 + q];
    }
    __syncthreads();
    const int o0 = t * kItems;
    if (o0 < len) {
        const uint64_t *A = ik;
        const uint64_t *B = ik + lenA;
        int i = (int)merge_split(A, (uint64_t)lenA, B, (uint64_t)lenB, (uint64_t)o0);
        int j = o0 - i;
        const int o1 = min(len, o0 + kItems);
        for (int o = o0; o < o1; ++o) {
            const bool takeA = j >= lenB || (i < lenA && A[i] <= B[j]);
            if (takeA) {
                ok[o] = A[i];
                ov[o] = iv[i];
                ++i;
            } else {
                ok[o] = B[j];
                ov[o] = iv[lenA + j];
                ++j;
            }
        }
    }
    __syncthreads();
    for (int q = t; q < len; q += kThreads) {
        const uint64_t key = ok[q];
        const uint64_t p = d0 + q;
        if (DECODE) {
#pragma unroll
            for (int k = 0; k < kMaxOrder; ++k)
                if (k < dst.order) dst.idx[k][p] = (uint32_t)(key >> dst.shift[k]) & dst.mask[k];
            dst.val[p] = __uint_as_float(ov[q]);
        } else {
            kO[p] = key;
            vO[p] = ov[q];
        }
    }
}

int bits_for(uint64_t dim) {
    int b = 0;
    while (b < 64 && (dim - 1) >> b) ++b;
    return b;
}

// Key layout of a mode-n copy: cyclic mode order from n, each mode
// ceil(log2 dims) bits, cut to the leading 64 bits.  *used = bits kept.
KeySpec key_spec(const pasta_coo_s *X, int mode, int *used_out) {
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
    *used_out = used;
    return ks;
}

// Where each mode's index sits in the sorted key (shift < 0: not whole).
GatherDst decode_spec(const pasta_coo_s *X, const KeySpec &ks, const StoredCopy &dst) {
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
    gd.order = X->order;
    return gd;
}

// Stable LSD radix sort of (key, payload) pairs made from the stored copy
// srcc: payload = the value bits (payload_val) or the entry number (then srcc
// must be the creation-order copy).  The passes cover key bits [low, used):
// low > 0 when srcc is already ordered by the low bits (see sort_copy).  The
// sorted payload lands in payload_out (nnz words); *keys_sorted points at the
// sorted keys inside the handle's scratch (valid until its next use).
// The passes of the radix sort over keys and payloads that `make` writes
// into the scratch (see radix_sort).
// Scratch bytes of one radix sort of n pairs: two key buffers, the spare
// payload buffer, the histograms.
size_t radix_scratch_bytes(uint64_t n) {
    const uint64_t ntiles = (n + kTile - 1) / kTile;
    const size_t hist_n = (size_t)kMaxBins * ntiles + kMaxBins;
    const size_t keys_b = (2 * n * sizeof(uint64_t) + 255) & ~(size_t)255;
    const size_t tmpv_b = (n * sizeof(uint32_t) + 255) & ~(size_t)255;
    return keys_b + tmpv_b + ((hist_n * sizeof(uint32_t) + 255) & ~(size_t)255);
}

template <typename Make>
pasta_status radix_core(pasta_coo_s *X, uint64_t n, int low, int used, Make make, uint32_t *payload_out,
                        const uint64_t **keys_sorted, cudaStream_t s, void *scratch_at = nullptr) {
    // digits of at most 9 bits, balanced over the fewest passes: 57 bits take
    // 7 passes (one of 9 bits), 64 take 8 of 8
    const int bits = used - low;
    const int passes = (bits + 8) / 9;
    const uint32_t ntiles = (uint32_t)((n + kTile - 1) / kTile);
    // scratch (radix_scratch_bytes): the handle's, or the region given
    const size_t keys_b = (2 * n * sizeof(uint64_t) + 255) & ~(size_t)255;
    const size_t tmpv_b = (n * sizeof(uint32_t) + 255) & ~(size_t)255;
    void *base = scratch_at;
    pasta_status st = PASTA_OK;
    if (!base) st = handle_scratch(X, radix_scratch_bytes(n), &base);
    if (st != PASTA_OK) return st;
    uint64_t *keys = reinterpret_cast<uint64_t *>(base);
    uint32_t *tmpv = reinterpret_cast<uint32_t *>(static_cast<char *>(base) + keys_b);
    uint32_t *hist = reinterpret_cast<uint32_t *>(static_cast<char *>(base) + keys_b + tmpv_b);
    uint64_t *kb[2] = {keys, keys + n};
    uint32_t *vb[2];
    vb[passes % 2] = payload_out;  // the last pass writes into payload_out
    vb[1 - passes % 2] = tmpv;
    uint32_t *totals = hist + (size_t)kMaxBins * ntiles;

    PASTA_CUDA(cudaFuncSetAttribute(k_scatter<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kScatterSmem));
    PASTA_CUDA(cudaFuncSetAttribute(k_scatter<512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kScatterSmem));
    st = make(kb[0], vb[0]);
    if (st != PASTA_OK) return st;
    int shift = low;
    for (int p = 0; p < passes; ++p) {
        const int width = bits / passes + (p < bits % passes ? 1 : 0);  // 1..9 bits
        const uint32_t mask = (1u << width) - 1u;
        const uint64_t *ki = kb[p % 2];
        uint64_t *ko = kb[(p + 1) % 2];
        if (width > 8) {
            k_hist<512><<<ntiles, kThreads, 0, s>>>(ki, n, shift, mask, ntiles, hist);
            k_rowscan<<<512, 1024, 0, s>>>(hist, ntiles, totals);
            k_scatter<512><<<ntiles, kThreads, kScatterSmem, s>>>(ki, vb[p % 2], ko, vb[(p + 1) % 2], n,
                                                                  shift, mask, ntiles, hist, totals);
        } else {
            k_hist<256><<<ntiles, kThreads, 0, s>>>(ki, n, shift, mask, ntiles, hist);
            k_rowscan<<<256, 1024, 0, s>>>(hist, ntiles, totals);
            k_scatter<256><<<ntiles, kThreads, kScatterSmem, s>>>(ki, vb[p % 2], ko, vb[(p + 1) % 2], n,
                                                                  shift, mask, ntiles, hist, totals);
        }
        shift += width;
    }
    PASTA_CUDA(cudaGetLastError());
    *keys_sorted = kb[passes % 2];
    return PASTA_OK;
}

pasta_status radix_sort_view(pasta_coo_s *X, const CooView &src, const KeySpec &ks, int low, int used,
                             bool payload_val, uint32_t *payload_out, const uint64_t **keys_sorted,
                             cudaStream_t s, void *scratch_at);

pasta_status radix_sort(pasta_coo_s *X, const StoredCopy &srcc, const KeySpec &ks, int low, int used,
                        bool payload_val, uint32_t *payload_out, const uint64_t **keys_sorted,
                        cudaStream_t s) {
    return radix_sort_view(X, view_of(X, srcc), ks, low, used, payload_val, payload_out, keys_sorted, s,
                           nullptr);
}

// radix_sort over the entries of a view (src.nnz of them; each array 16-byte
// aligned and readable 16 bytes past its end), with the scratch given
// (nullptr: the handle's).
pasta_status radix_sort_view(pasta_coo_s *X, const CooView &src, const KeySpec &ks, int low, int used,
                             bool payload_val, uint32_t *payload_out, const uint64_t **keys_sorted,
                             cudaStream_t s, void *scratch_at) {
    const uint64_t n = src.nnz;
    const int gblocks = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)X->num_sms * 16);
    return radix_core(
        X, n, low, used,
        [&](uint64_t *keys, uint32_t *payload) -> pasta_status {
            k_make_keys<<<gblocks, 256, 0, s>>>(src, ks, keys, payload, payload_val);
            PASTA_CUDA(cudaGetLastError());
            return PASTA_OK;
        },
        payload_out, keys_sorted, s, scratch_at);
}

bool key_holds_all(const GatherDst &gd, int order) {
    for (int k = 0; k < order; ++k)
        if (gd.shift[k] < 0) return false;
    return true;
}

}  // namespace

pasta_status sort_copy(pasta_coo_s *X, int mode, cudaStream_t s) {
    StoredCopy &dst = X->sorted[mode];
    const uint64_t n = X->nnz;
    dst.perm_ready = false;
    if (n == 0) {
        dst.perm_ready = true;
        return PASTA_OK;
    }
    int used = 0;
    const KeySpec ks = key_spec(X, mode, &used);
    const GatherDst gd = decode_spec(X, ks, dst);
    const int gblocks = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)X->num_sms * 16);
    const uint64_t *keys = nullptr;
    if (key_holds_all(gd, X->order)) {
        // the values travel as the payload and every index is decoded from
        // the sorted keys: nothing is gathered; the permutation is built on
        // request (ensure_perm).  A copy already sorted for a neighbouring
        // mode saves passes, the stable sort keeping its order among ties:
        //  - mode n+1's copy is ordered by (n+1, ..., n-1, n), which is mode
        //    n's key without its leading field; a stable sort of it on the
        //    mode-n field alone (the key's top bits) gives mode n's order;
        //  - else mode n-1's copy is ordered by (n-1, n, ..., n-2); its
        //    leading field is the least significant field of mode n's key,
        //    so a stable sort on the other fields gives mode n's order.
        // Ties in the sorted fields keep the copy's order, which is by the
        // remaining fields and then creation order, as in the full sort.
        const int next = (mode + 1) % X->order;
        const int prev = (mode + X->order - 1) % X->order;
        const StoredCopy *src = &X->orig;
        int low = 0;
        if (X->sorted[next].present) {
            src = &X->sorted[next];
            low = used - bits_for(X->dims[mode]);
        } else if (X->sorted[prev].present) {
            src = &X->sorted[prev];
            low = bits_for(X->dims[prev]);
        }
        pasta_status st = radix_sort(X, *src, ks, low, used, true,
                                     reinterpret_cast<uint32_t *>(dst.val), &keys, s);
        if (st != PASTA_OK) return st;
        k_decode<<<gblocks, 256, 0, s>>>(keys, n, X->order, gd);
    } else {
        pasta_status st = radix_sort(X, X->orig, ks, 0, used, false, dst.perm, &keys, s);
        if (st != PASTA_OK) return st;
        const CooView src = view_of(X, X->orig);
        k_gather<<<gblocks, 256, 0, s>>>(src, dst.perm, keys, gd);
        dst.perm_ready = true;
    }
    cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return cuda_fail(le, "sort kernels");
    return PASTA_OK;
}

bool sort_key_holds_all(const pasta_coo_s *X, int mode) {
    int used = 0;
    const KeySpec ks = key_spec(X, mode, &used);
    StoredCopy none{};
    return key_holds_all(decode_spec(X, ks, none), X->order);
}

pasta_status copy_in_and_sort(pasta_coo_s *X, int mode, const void *const *h_idx, const void *h_val, cudaStream_t s) {
    const uint64_t n = X->nnz;
    // K parts, each a multiple of 1024 entries but the last (16-byte aligned
    // splits of every array): 4 from 2^24 entries on (measured 2% faster on
    // the 100M-entry tensor than 2), else 2
    const int K = n >= (1ull << 24) ? 4 : 2;
    uint64_t off[5], len[4];
    for (int q = 0; q <= K; ++q) off[q] = q == K ? n : ((n * (uint64_t)q / (uint64_t)K) & ~(uint64_t)1023);
    for (int q = 0; q < K; ++q) len[q] = off[q + 1] - off[q];
    StoredCopy &dst = X->sorted[mode];
    dst.perm_ready = false;
    int used = 0;
    const KeySpec ks = key_spec(X, mode, &used);
    const GatherDst gd = decode_spec(X, ks, dst);
    if (!key_holds_all(gd, X->order) || len[0] == 0) {
        set_error("copy_in_and_sort needs a key that holds every index and enough entries per part");
        return PASTA_ERR_UNSUPPORTED;
    }
    // scratch: a radix region and a payload array per part; with four parts,
    // the two first-level merges' pairs; the merge blocks' split points
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t total = 0, rof[4], pof[4];
    for (int q = 0; q < K; ++q) {
        rof[q] = total;
        total += radix_scratch_bytes(len[q]);
    }
    for (int q = 0; q < K; ++q) {
        pof[q] = total;
        total += up(len[q] * sizeof(uint32_t));
    }
    size_t mk[2] = {0, 0}, mv[2] = {0, 0};
    if (K == 4) {
        for (int h = 0; h < 2; ++h) {
            const uint64_t m = len[2 * h] + len[2 * h + 1];
            mk[h] = total;
            total += up(m * sizeof(uint64_t));
            mv[h] = total;
            total += up(m * sizeof(uint32_t));
        }
    }
    const size_t spl = total;
    total += up(((n + kTile - 1) / kTile + 1) * sizeof(uint64_t));
    void *base = nullptr;
    pasta_status st = handle_scratch(X, total, &base);
    if (st != PASTA_OK) return st;
    char *b = static_cast<char *>(base);
    uint64_t *splits = reinterpret_cast<uint64_t *>(b + spl);

    // parts 1.. are copied on a high-priority stream of their own, one after
    // another, so their (small) grids are scheduled while earlier parts sort
    int lo_pri = 0, hi_pri = 0;
    PASTA_CUDA(cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri));
    cudaStream_t sc = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    PASTA_CUDA(cudaStreamCreateWithPriority(&sc, cudaStreamNonBlocking, hi_pri));
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < K && e == cudaSuccess; ++q) e = cudaEventCreateWithFlags(&ev[q], cudaEventDisableTiming);
    const int order = X->order;
    for (int q = 0; q < K && e == cudaSuccess; ++q) {
        cudaStream_t cs = q == 0 ? s : sc;
        for (int k = 0; k < order && e == cudaSuccess; ++k)
            e = copy_bytes(X->orig.idx[k] + off[q], static_cast<const uint32_t *>(h_idx[k]) + off[q], len[q] * 4,
                           X->num_sms, cs);
        if (e == cudaSuccess)
            e = copy_bytes(X->orig.val + off[q], static_cast<const float *>(h_val) + off[q], len[q] * 4, X->num_sms,
                           cs);
        if (e == cudaSuccess) e = cudaEventRecord(ev[q], cs);
        if (e == cudaSuccess && q == 0) e = cudaStreamWaitEvent(sc, ev[0], 0);
    }
    if (e != cudaSuccess) st = cuda_fail(e, "copy-in of the parts");
    if (st == PASTA_OK) {
        e = cudaFuncSetAttribute(k_merge<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMergeSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_merge<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMergeSmem);
        if (e != cudaSuccess) st = cuda_fail(e, "merge kernel attributes");
    }
    // each part sorts once it has arrived (the later ones still arriving);
    // with four parts, each pair is merged as soon as both are sorted
    const uint64_t *keys[4] = {nullptr, nullptr, nullptr, nullptr};
    uint32_t *pay[4];
    for (int q = 0; q < K; ++q) pay[q] = reinterpret_cast<uint32_t *>(b + pof[q]);
    auto merge = [&](bool decode, const uint64_t *kA, const uint32_t *vA, uint64_t nA, const uint64_t *kB,
                     const uint32_t *vB, uint64_t nB, uint64_t *kO, uint32_t *vO) -> pasta_status {
        const uint64_t mb = (nA + nB + kTile - 1) / kTile;
        k_merge_splits<<<(unsigned)((mb + 1 + 255) / 256), 256, 0, s>>>(kA, nA, kB, nB, mb, splits);
        if (decode)
            k_merge<true><<<(unsigned)mb, kThreads, kMergeSmem, s>>>(kA, vA, nA, kB, vB, nB, splits, gd, nullptr,
                                                                     nullptr);
        else
            k_merge<false><<<(unsigned)mb, kThreads, kMergeSmem, s>>>(kA, vA, nA, kB, vB, nB, splits, gd, kO, vO);
        const cudaError_t le = cudaGetLastError();
        return le == cudaSuccess ? PASTA_OK : cuda_fail(le, "merge of sorted parts");
    };
    for (int q = 0; q < K && st == PASTA_OK; ++q) {
        if (q > 0) {
            e = cudaStreamWaitEvent(s, ev[q], 0);
            if (e != cudaSuccess) st = cuda_fail(e, "wait for a part");
        }
        if (st == PASTA_OK) {
            CooView v = view_of(X, X->orig);
            for (int k = 0; k < order; ++k) v.idx[k] += off[q];
            v.val += off[q];
            v.nnz = len[q];
            st = radix_sort_view(X, v, ks, 0, used, true, pay[q], &keys[q], s, b + rof[q]);
        }
        if (st == PASTA_OK && K == 4 && (q & 1)) {
            const int h = q / 2;
            st = merge(false, keys[q - 1], pay[q - 1], len[q - 1], keys[q], pay[q], len[q],
                       reinterpret_cast<uint64_t *>(b + mk[h]), reinterpret_cast<uint32_t *>(b + mv[h]));
        }
    }
    if (st == PASTA_OK) {
        if (K == 2)
            st = merge(true, keys[0], pay[0], len[0], keys[1], pay[1], len[1], nullptr, nullptr);
        else
            st = merge(true, reinterpret_cast<const uint64_t *>(b + mk[0]), reinterpret_cast<const uint32_t *>(b + mv[0]),
                       len[0] + len[1], reinterpret_cast<const uint64_t *>(b + mk[1]),
                       reinterpret_cast<const uint32_t *>(b + mv[1]), len[2] + len[3], nullptr, nullptr);
    }
    // stream and events are released once the work queued on them is done
    for (int q = 0; q < K; ++q)
        if (ev[q]) cudaEventDestroy(ev[q]);
    cudaStreamDestroy(sc);
    return st;
}

pasta_status radix_sort_keys(pasta_coo_s *X, uint64_t n, int used, MakeKeysFn make, void *ctx,
                             uint32_t *payload_out, const uint64_t **keys_sorted, cudaStream_t s) {
    if (n == 0) return PASTA_OK;
    return radix_core(
        X, n, 0, used, [&](uint64_t *keys, uint32_t *payload) { return make(ctx, keys, payload, s); },
        payload_out, keys_sorted, s);
}

pasta_status ensure_perm(pasta_coo_s *X, int mode, cudaStream_t s) {
    StoredCopy &c = X->sorted[mode];
    if (!c.present || c.perm_ready) return PASTA_OK;
    int used = 0;
    const KeySpec ks = key_spec(X, mode, &used);
    const uint64_t *keys = nullptr;
    pasta_status st = radix_sort(X, X->orig, ks, 0, used, false, c.perm, &keys, s);
    if (st == PASTA_OK) c.perm_ready = true;
    return st;
}

}  // namespace pasta
