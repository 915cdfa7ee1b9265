// HiCOO: the hierarchical COO format (Li, Choi and Vuduc, SC'18) that
// Sec. 8 names, with CSF, as the compressed formats to add, and its MTTKRP.
//
// Format.  The index space is cut into blocks of B^N cells (B = 2^bits,
// bits <= 8).  Entry coordinates i_k split into a block coordinate
// b_k = i_k >> bits and an in-block offset e_k = i_k & (B - 1).  The copy is
// one array of nonempty blocks (bptr: where each block's entries start, nb + 1
// words; binds[k]: the block coordinates, nb words per mode) and the entries
// in block order (einds[k]: one byte per mode per entry; val: FP32).  Blocks
// are in lexicographic order of (b_0, ..., b_{N-1}); inside a block, entries
// are in lexicographic order of (e_0, ..., e_{N-1}).  Both orders come from
// one stable sort of the key (block coordinates, each mode taking the bits
// of its block count, then the offsets, bits each), cut to its leading 64
// bits: the block part must fit (else PASTA_ERR_UNSUPPORTED), and where
// offset bits are cut, entries with equal leading bits keep creation order.
// Index bytes per entry: N + 4 (value) instead of 4N + 4, plus 4N + 4 per
// block.  One copy serves every mode.
//
// Build: key kernel, the mode sort's radix sort (payload = entry number),
// per-tile block-head counts, a one-block scan (one synchronisation for the
// block count), a pass writing bptr / binds at the heads and the einds / val
// of every entry through the permutation, and, per tile of kHTile entries,
// the block holding its first entry (a binary search in bptr).
//
// MTTKRP (Eq. (mttkrp-init) on this copy).  Lanes span the rank as in the
// streaming kernels (L lanes x 16 bytes = one factor row, G = 32/L lane groups
// per warp); each group walks tiles of kHTile consecutive entries
// (grid-strided).  A batch of four entries reads one 32-bit word of offsets
// per mode and a float4 of values; the group advances its block (bptr, binds)
// when an entry passes the next block start, forms i_k = (b_k << bits) + e_k,
// issues the N-1 row gathers of all four entries, then adds
// val * prod(rows) into one of two register row slots keyed by the output
// row.  The copy is not sorted by the output mode, so rows recur across the
// stream: a slot is flushed with red.global.add.v4.f32 when a third row
// evicts it (least recently used) and at the tile end, into an output
// cleared first.
#include <algorithm>

#include "pasta_internal.cuh"

namespace pasta {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // build: entries per head-count tile
constexpr unsigned FULL = 0xFFFFFFFFu;

struct HKeySpec {
    int order;
    int bits;
    int bshl[kMaxOrder];  // block field of mode k at bit bshl[k] of the block key
    int bbits[kMaxOrder];
    int block_bits;       // sum of bbits
    int elem_keep;        // offset bits kept below the block key (<= order * bits)
    int elem_total;       // order * bits
};

int bits_of(uint64_t x) {
    int b = 0;
    while (b < 64 && (x >> b)) ++b;
    return b;
}

// key of entry m: (block key << elem_keep) | (offset key >> (elem_total - elem_keep))
__device__ __forceinline__ uint64_t hkey(const CooView &v, const HKeySpec &ks, uint64_t m) {
    uint64_t bk = 0, ek = 0;
    const uint32_t emask = (1u << ks.bits) - 1u;
    for (int k = 0; k < ks.order; ++k) {
        const uint32_t i = v.idx[k][m];
        bk |= (uint64_t)(i >> ks.bits) << ks.bshl[k];
        ek = (ek << ks.bits) | (uint64_t)(i & emask);
    }
    const int drop = ks.elem_total - ks.elem_keep;
    const uint64_t e = drop >= 64 ? 0 : (ek >> drop);
    const uint64_t hi = ks.elem_keep >= 64 ? 0 : (bk << ks.elem_keep);  // bk = 0 when elem_keep = 64
    return hi | e;
}

__global__ void k_hkeys(CooView v, HKeySpec ks, uint64_t *keys, uint32_t *payload) {
    for (uint64_t m = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; m < v.nnz;
         m += (uint64_t)gridDim.x * blockDim.x) {
        keys[m] = hkey(v, ks, m);
        payload[m] = (uint32_t)m;
    }
}

struct KeyCtx {
    CooView v;
    HKeySpec ks;
    int grid;
};

pasta_status make_hkeys(void *ctx, uint64_t *keys, uint32_t *payload, cudaStream_t s) {
    const KeyCtx *c = static_cast<const KeyCtx *>(ctx);
    k_hkeys<<<c->grid, 256, 0, s>>>(c->v, c->ks, keys, payload);
    PASTA_CUDA(cudaGetLastError());
    return PASTA_OK;
}

__device__ __forceinline__ bool is_head(const uint64_t *keys, uint64_t p, int elem_keep) {
    if (p == 0) return true;
    const uint64_t a = elem_keep >= 64 ? 0 : keys[p] >> elem_keep;
    const uint64_t b = elem_keep >= 64 ? 0 : keys[p - 1] >> elem_keep;
    return a != b;
}

// counts[t] = block heads among entries [t * kTile, (t + 1) * kTile)
__global__ void __launch_bounds__(kThreads) k_hhead_count(const uint64_t *keys, uint64_t n, int elem_keep,
                                                          uint32_t *counts) {
    __shared__ uint32_t wsum[kThreads / 32];
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
    uint32_t c = 0;
    for (int j = 0; j < kItems; ++j) {
        const uint64_t p = t0 + (uint64_t)j * kThreads + threadIdx.x;
        if (p < n && is_head(keys, p, elem_keep)) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += wsum[w];
        counts[blockIdx.x] = t;
    }
}

// offsets = exclusive scan of counts (one block); *total = the sum
__global__ void __launch_bounds__(1024) k_hscan(const uint32_t *counts, uint32_t n, uint32_t *offsets,
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

struct HWrite {
    const uint64_t *keys;
    const uint32_t *perm;
    CooView src;  // creation-order copy
    HKeySpec ks;
    uint64_t n;
    uint32_t *bptr;
    uint32_t *binds[kMaxOrder];
    uint8_t *einds[kMaxOrder];
    float *val;
};

// Ranks the block heads of each tile (block offsets from k_hscan) and writes
// bptr / binds there; writes every entry's offsets and value.
__global__ void __launch_bounds__(kThreads) k_hwrite(HWrite w, const uint32_t *offsets) {
    __shared__ uint32_t wsum[kThreads / 32];
    __shared__ uint32_t base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
    if (threadIdx.x == 0) base = offsets[blockIdx.x];
    __syncthreads();
    const uint32_t emask = (1u << w.ks.bits) - 1u;
    for (int j = 0; j < kItems; ++j) {
        // round j: positions t0 + j * kThreads + threadIdx.x, in order
        const uint64_t p = t0 + (uint64_t)j * kThreads + threadIdx.x;
        const bool live = p < w.n;
        const bool h = live && is_head(w.keys, p, w.ks.elem_keep);
        const unsigned bal = __ballot_sync(FULL, h);
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        uint32_t before = base;
        for (int v = 0; v < warp; ++v) before += wsum[v];
        if (h) {
            const uint32_t r = before + __popc(bal & ((1u << lane) - 1u));
            w.bptr[r] = (uint32_t)p;
            const uint64_t bk = w.ks.elem_keep >= 64 ? 0 : w.keys[p] >> w.ks.elem_keep;
            for (int k = 0; k < w.ks.order; ++k) {
                const uint64_t m = w.ks.bbits[k] >= 64 ? ~0ull : ((1ull << w.ks.bbits[k]) - 1ull);
                w.binds[k][r] = (uint32_t)((bk >> w.ks.bshl[k]) & m);
            }
        }
        if (live) {
            const uint32_t src = w.perm[p];
            for (int k = 0; k < w.ks.order; ++k) w.einds[k][p] = (uint8_t)(w.src.idx[k][src] & emask);
            w.val[p] = w.src.val[src];
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int v = 0; v < kThreads / 32; ++v) base += wsum[v];
        __syncthreads();
    }
}

// tile_block[t] = the block holding entry t * tile (last b with bptr[b] <= t * tile)
__global__ void k_tile_block(const uint32_t *bptr, uint64_t nb, uint64_t ntiles, uint32_t tile,
                             uint32_t *tile_block) {
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p = t * tile;
        uint64_t lo = 0, hi = nb;  // bptr[lo] <= p < bptr[hi] (bptr[nb] = nnz)
        while (hi - lo > 1) {
            const uint64_t mid = (lo + hi) / 2;
            if (bptr[mid] <= p) lo = mid; else hi = mid;
        }
        tile_block[t] = (uint32_t)lo;
    }
}

}  // namespace

void free_hicoo(HicooCopy &H) {
    dev_free(H.block);
    dev_free(H.bblock);
    H = HicooCopy{};
}

pasta_status build_hicoo(pasta_coo_s *X, int bits, cudaStream_t s) {
    HicooCopy &H = X->hicoo;
    if (H.present && H.bits == bits) return PASTA_OK;
    if (H.present) {
        cudaStreamSynchronize(s);  // kernels may still read the old copy
        free_hicoo(H);
    }
    const int N = X->order;
    HKeySpec ks{};
    ks.order = N;
    ks.bits = bits;
    int bb = 0;
    for (int k = N - 1; k >= 0; --k) {  // mode 0 most significant
        const uint64_t nblk = (X->dims[k] + ((uint64_t)1 << bits) - 1) >> bits;
        ks.bbits[k] = bits_of(nblk - 1);
        ks.bshl[k] = bb;
        bb += ks.bbits[k];
    }
    if (bb > 64) {
        set_error("HiCOO block coordinates need %d key bits (more than 64)", bb);
        return PASTA_ERR_UNSUPPORTED;
    }
    ks.block_bits = bb;
    ks.elem_total = N * bits;
    ks.elem_keep = std::min(64 - bb, ks.elem_total);
    const int used = bb + ks.elem_keep;
    const uint64_t n = X->nnz;

    // entry arrays: N offset bytes and a value per entry, padded like the stored copies
    const size_t e_b = ((size_t)X->nnz_pad + 255) & ~(size_t)255;
    const size_t v_b = ((size_t)X->nnz_pad * 4 + 255) & ~(size_t)255;
    H.bits = bits;
    cudaError_t e = dev_malloc(&H.block, e_b * N + v_b, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        H = HicooCopy{};
        set_error("device allocation of the HiCOO entry arrays failed");
        return PASTA_ERR_NOMEM;
    }
    char *blk = static_cast<char *>(H.block);
    for (int k = 0; k < N; ++k) H.einds[k] = reinterpret_cast<uint8_t *>(blk + e_b * k);
    H.val = reinterpret_cast<float *>(blk + e_b * N);
    PASTA_CUDA(cudaMemsetAsync(H.block, 0, e_b * N + v_b, s));  // padding words read by 4-entry loads
    if (n == 0) {
        H.nb = 0;
        H.ntiles = 0;
        e = dev_malloc(&H.bblock, 256, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_hicoo(H);
            return PASTA_ERR_NOMEM;
        }
        H.bptr = static_cast<uint32_t *>(H.bblock);
        PASTA_CUDA(cudaMemsetAsync(H.bptr, 0, 4, s));
        H.present = true;
        return PASTA_OK;
    }

    // build temporaries: the permutation, per-tile head counts and offsets, the block count
    const uint32_t ntile = (uint32_t)((n + kTile - 1) / kTile);
    const size_t perm_b = ((size_t)n * 4 + 255) & ~(size_t)255;
    void *tmp = nullptr;
    e = dev_malloc(&tmp, perm_b + (size_t)ntile * 8 + 64, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_hicoo(H);
        return PASTA_ERR_NOMEM;
    }
    uint32_t *perm = static_cast<uint32_t *>(tmp);
    uint32_t *counts = reinterpret_cast<uint32_t *>(static_cast<char *>(tmp) + perm_b);
    uint32_t *offsets = counts + ntile;
    uint64_t *total =
        reinterpret_cast<uint64_t *>(static_cast<char *>(tmp) + perm_b + (((size_t)ntile * 8 + 7) & ~(size_t)7));
    KeyCtx kc{view_of(X, X->orig), ks, (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)X->num_sms * 16)};
    const uint64_t *keys = nullptr;
    pasta_status st = radix_sort_keys(X, n, used, make_hkeys, &kc, perm, &keys, s);
    if (st != PASTA_OK) {
        cudaStreamSynchronize(s);
        dev_free(tmp);
        free_hicoo(H);
        return st;
    }
    // block heads: counts per tile, scan, one synchronisation for nb
    uint64_t nb = 0;
    k_hhead_count<<<ntile, kThreads, 0, s>>>(keys, n, ks.elem_keep, counts);
    k_hscan<<<1, 1024, 0, s>>>(counts, ntile, offsets, total);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nb, total, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        dev_free(tmp);
        free_hicoo(H);
        return cuda_fail(e, "HiCOO block count");
    }
    H.nb = nb;
    H.ntiles = (n + kHTile - 1) / kHTile;
    const size_t bp_b = (((size_t)nb + 1) * 4 + 255) & ~(size_t)255;
    const size_t bi_b = ((size_t)nb * 4 + 255) & ~(size_t)255;
    const size_t tb_b = ((size_t)H.ntiles * 4 + 255) & ~(size_t)255;
    e = dev_malloc(&H.bblock, bp_b + bi_b * N + tb_b, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        dev_free(tmp);
        free_hicoo(H);
        return PASTA_ERR_NOMEM;
    }
    char *bb_ = static_cast<char *>(H.bblock);
    H.bptr = reinterpret_cast<uint32_t *>(bb_);
    for (int k = 0; k < N; ++k) H.binds[k] = reinterpret_cast<uint32_t *>(bb_ + bp_b + bi_b * k);
    H.tile_block = reinterpret_cast<uint32_t *>(bb_ + bp_b + bi_b * N);
    HWrite w{};
    w.keys = keys;
    w.perm = perm;
    w.src = view_of(X, X->orig);
    w.ks = ks;
    w.n = n;
    w.bptr = H.bptr;
    for (int k = 0; k < N; ++k) {
        w.binds[k] = H.binds[k];
        w.einds[k] = H.einds[k];
    }
    w.val = H.val;
    k_hwrite<<<ntile, kThreads, 0, s>>>(w, offsets);
    const uint32_t nnz32 = (uint32_t)n;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(H.bptr + nb, &nnz32, 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_tile_block<<<(unsigned)std::min<uint64_t>((H.ntiles + 255) / 256, 4096), 256, 0, s>>>(
            H.bptr, nb, H.ntiles, (uint32_t)kHTile, H.tile_block);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // nnz32 is a host temporary; tmp is freed next
    dev_free(tmp);
    if (e != cudaSuccess) {
        free_hicoo(H);
        return cuda_fail(e, "HiCOO write");
    }
    H.present = true;
    return PASTA_OK;
}

// ------------------------------------------------------------- MTTKRP ---

namespace {

template <typename T, int N>
struct HArgs {
    const uint32_t *bptr;
    const uint32_t *binds[N];  // by position: position 0 is the output mode
    const uint8_t *einds[N];
    const T *U[N];
    const float *val;
    const uint32_t *tile_block;
    double *M;  // FP64 images of the output: `copies` of dims[mode] x R (summed into FP32 after)
    uint64_t nnz, ntiles;
    uint64_t copy_stride;  // elements per image
    uint32_t copies;       // block b adds into image b % copies
    uint32_t R;
    int bits, L, lshift;
};

__device__ __forceinline__ uint64_t policy_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint4 ld_row16(const void *p, uint64_t pol) {
    uint4 r;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p), "l"(pol));
    return r;
}

// A row slot's FP32 partial sums (at most one 512-entry tile's) are added
// into an FP64 image of the output: an output row can receive a partial
// from every tile (millions, for the short modes), and FP32 atomic sums of
// that many terms drift beyond the FP32 MTTKRP's error bar.  Blocks spread
// over several images (Sec. 5.3's privatization, per block instead of per
// thread), so a hot row's additions queue on several addresses, not one.
template <int VEC> __device__ __forceinline__ void flush_row(double *M, uint32_t row, uint32_t R, int off,
                                                             const float (&acc)[VEC]) {
    double *d = M + (uint64_t)row * R + off;
#pragma unroll
    for (int e = 0; e < VEC; ++e) atomicAdd(d + e, (double)acc[e]);
}

// dst[i] = FP32 of the sum over the images of element i.
__global__ void k_images_to_f32(const double *src, uint32_t copies, uint64_t n, float *dst) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (uint32_t c = 0; c < copies; ++c) acc += src[(uint64_t)c * n + i];
        dst[i] = (float)acc;
    }
}

template <typename T, int N, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_hicoo_mttkrp(const HArgs<T, N> a) {
    constexpr int VEC = 16 / sizeof(T);
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int L = a.L;
    const int lig = lane & (L - 1);
    const int grp = lane >> a.lshift;
    const int G = 32 >> a.lshift;
    const int off = lig * VEC;
    const uint64_t pol = policy_last();
    const uint32_t stride = a.R * (uint32_t)sizeof(T);
    const char *ub[N];
#pragma unroll
    for (int p = 1; p < N; ++p) ub[p] = reinterpret_cast<const char *>(a.U[p] + off);
    const uint64_t gid = ((uint64_t)blockIdx.x * (kThreads / 32) + warp) * G + grp;
    const uint64_t gstride = (uint64_t)gridDim.x * (kThreads / 32) * G;
    double *const Mimg = a.M + (uint64_t)(blockIdx.x % a.copies) * a.copy_stride;

    for (uint64_t t = gid; t < a.ntiles; t += gstride) {
        uint64_t p = t * kHTile;
        const uint64_t pend = min(p + kHTile, a.nnz);
        uint32_t blk = a.tile_block[t];
        uint32_t next = a.bptr[blk + 1];
        uint32_t base[N];
#pragma unroll
        for (int k = 0; k < N; ++k) base[k] = a.binds[k][blk] << a.bits;
        // two row slots, [0] most recently used
        uint32_t srow[2] = {kNoRow, kNoRow};
        float sacc[2][VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) sacc[0][e] = sacc[1][e] = 0.f;
        for (; p < pend; p += 4) {
            uint32_t ew[N];
#pragma unroll
            for (int k = 0; k < N; ++k) ew[k] = *reinterpret_cast<const uint32_t *>(a.einds[k] + p);
            const float4 v4 = *reinterpret_cast<const float4 *>(a.val + p);
            const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
            uint32_t ix[4][N];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (p + q < pend) {
                    while (p + q >= next) {  // the entry starts a later block
                        ++blk;
                        next = a.bptr[blk + 1];
#pragma unroll
                        for (int k = 0; k < N; ++k) base[k] = a.binds[k][blk] << a.bits;
                    }
                }
#pragma unroll
                for (int k = 0; k < N; ++k) ix[q][k] = base[k] + ((ew[k] >> (8 * q)) & 0xFFu);
            }
            uint4 rows[4][N - 1];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 1; k < N; ++k)
                    rows[q][k - 1] = p + q < pend ? ld_row16(ub[k] + (uint64_t)ix[q][k] * stride, pol)
                                                  : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (p + q >= pend) continue;
                float t1[VEC], r[VEC];
                widen<T, VEC>(rows[q][0], r);
#pragma unroll
                for (int e = 0; e < VEC; ++e) t1[e] = vv[q] * r[e];
#pragma unroll
                for (int k = 2; k < N; ++k) {
                    widen<T, VEC>(rows[q][k - 1], r);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) t1[e] *= r[e];
                }
                const uint32_t o = ix[q][0];
                if (o == srow[0]) {
#pragma unroll
                    for (int e = 0; e < VEC; ++e) sacc[0][e] += t1[e];
                } else if (o == srow[1]) {  // swap: slot 1 becomes the most recent
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        const float x = sacc[1][e] + t1[e];
                        sacc[1][e] = sacc[0][e];
                        sacc[0][e] = x;
                    }
                    srow[1] = srow[0];
                    srow[0] = o;
                } else {  // evict slot 1, shift slot 0 down
                    if (srow[1] != kNoRow) flush_row<VEC>(Mimg, srow[1], a.R, off, sacc[1]);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) {
                        sacc[1][e] = sacc[0][e];
                        sacc[0][e] = t1[e];
                    }
                    srow[1] = srow[0];
                    srow[0] = o;
                }
            }
        }
        if (srow[0] != kNoRow) flush_row<VEC>(Mimg, srow[0], a.R, off, sacc[0]);
        if (srow[1] != kNoRow) flush_row<VEC>(Mimg, srow[1], a.R, off, sacc[1]);
    }
}

template <typename T, int N>
pasta_status hrun(const pasta_coo_s *X, const void *const *U, int mode, int R, double *M, uint32_t copies,
                  cudaStream_t s) {
    const HicooCopy &H = X->hicoo;
    HArgs<T, N> a{};
    for (int p = 0; p < N; ++p) {
        const int k = (mode + p) % N;
        a.binds[p] = H.binds[k];
        a.einds[p] = H.einds[k];
        a.U[p] = static_cast<const T *>(U[k]);
    }
    a.bptr = H.bptr;
    a.val = H.val;
    a.tile_block = H.tile_block;
    a.M = M;
    a.copies = copies;
    a.copy_stride = X->dims[mode] * (uint64_t)R;
    a.nnz = X->nnz;
    a.ntiles = H.ntiles;
    a.R = (uint32_t)R;
    a.bits = H.bits;
    const Geometry g = make_geometry(R, 16 / (int)sizeof(T), (int)sizeof(T));
    a.L = g.L;
    a.lshift = g.lshift;
    constexpr int MINB = (N <= 3 && sizeof(T) == 4) ? 3 : 2;  // 16-bit rows widen to 8 FP64 adds per flush
    auto kern = k_hicoo_mttkrp<T, N, MINB>;
    int per_sm = 0;
    PASTA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0));
    per_sm = std::max(per_sm, 1);
    const uint64_t groups_per_block = (uint64_t)(kThreads / 32) * (32u >> g.lshift);
    const uint64_t want = (H.ntiles + groups_per_block - 1) / groups_per_block;
    const uint64_t blocks = apply_grid_cap(std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)X->num_sms * per_sm)));
    kern<<<(unsigned)blocks, kThreads, 0, s>>>(a);
    PASTA_CUDA(cudaGetLastError());
    return PASTA_OK;
}

template <typename T>
pasta_status hby_order(const pasta_coo_s *X, const void *const *U, int mode, int R, double *M, uint32_t copies,
                       cudaStream_t s) {
    switch (X->order) {
        case 2: return hrun<T, 2>(X, U, mode, R, M, copies, s);
        case 3: return hrun<T, 3>(X, U, mode, R, M, copies, s);
        case 4: return hrun<T, 4>(X, U, mode, R, M, copies, s);
        case 5: return hrun<T, 5>(X, U, mode, R, M, copies, s);
    }
    return PASTA_ERR_UNSUPPORTED;
}

}  // namespace

pasta_status launch_hicoo_mttkrp(pasta_coo_s *X, const void *const *U, pasta_dtype dt, int mode, int R,
                                 void *M, cudaStream_t s) {
    if (!stream_supported(dt, X->order, R, U, mode, M, 2)) {
        set_error("the HiCOO MTTKRP covers FP32/BF16/FP16 factors, order 2..5, R * sizeof(element) = 16 L "
                  "(L a power of two) and 16-byte aligned factors and output");
        return PASTA_ERR_UNSUPPORTED;
    }
    const uint64_t n = X->dims[mode] * (uint64_t)R;
    if (X->nnz == 0) {
        PASTA_CUDA(cudaMemsetAsync(M, 0, n * sizeof(float), s));
        return PASTA_OK;
    }
    // The FP64 images of M live in the handle's scratch (calls on one handle
    // are ordered, so it is not in use by a sort): as many as fit 256 MB, at
    // most 64, at least one.
    const uint64_t img_bytes = n * sizeof(double);
    const uint32_t copies = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(64, (256ull << 20) / img_bytes));
    void *img = nullptr;
    pasta_status st = handle_scratch(X, img_bytes * copies, &img);
    if (st != PASTA_OK) return st;
    double *M64 = static_cast<double *>(img);
    PASTA_CUDA(cudaMemsetAsync(M64, 0, img_bytes * copies, s));
    switch (dt) {
        case PASTA_F32: st = hby_order<float>(X, U, mode, R, M64, copies, s); break;
        case PASTA_BF16: st = hby_order<__nv_bfloat16>(X, U, mode, R, M64, copies, s); break;
        case PASTA_F16: st = hby_order<__half>(X, U, mode, R, M64, copies, s); break;
        default: st = PASTA_ERR_UNSUPPORTED;
    }
    if (st != PASTA_OK) return st;
    const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, (uint64_t)X->num_sms * 8));
    k_images_to_f32<<<blocks, 256, 0, s>>>(M64, copies, n, static_cast<float *>(M));
    PASTA_CUDA(cudaGetLastError());
    return PASTA_OK;
}

}  // namespace pasta
