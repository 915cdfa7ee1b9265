// Launch templates of the streaming kernels (stream_kernels.cuh), shared by
// the three translation units that instantiate them: stream_mttkrp.cu (MTTKRP),
// stream_loss_fwd.cu (CP-loss forward) and stream_loss_bwd.cu (per-mode
// CP-loss backward).  One unit per kind keeps each compile short and lets the
// build run them in parallel.
#pragma once

#include <algorithm>

#include "stream_kernels.cuh"

namespace pasta {
namespace stream_launch {

using stream::Args;
using stream::k_stream;
using stream::kThreads;
using stream::kWarps;

constexpr int kStages = 2;

// Zeros the output row of the last entry of every group tile of `tile`
// entries: the streaming kernel adds atomically only into rows open at a
// group-tile end (the run reaching the end, and the same row's continuation
// in the next tile) and stores every other row whole.  One warp per tile,
// lanes across R.  (Internal linkage: every unit that includes this header
// gets its own copy.)
namespace {
__global__ void __launch_bounds__(256) k_zero_tile_end_rows(const uint32_t *idx0, uint64_t nnz, uint32_t tile,
                                                            uint32_t R, float *out) {
    const uint64_t w = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t ntiles = (nnz + tile - 1) / tile;
    if (w >= ntiles) return;
    const uint64_t p = min(nnz, (w + 1) * (uint64_t)tile) - 1;
    float *row = out + (uint64_t)idx0[p] * R;
    for (uint32_t r = threadIdx.x & 31; r < R; r += 32) row[r] = 0.f;
}
}  // namespace

// Blocks per SM each instantiation is compiled for (register budget
// 65536 / (256 * blocks)), chosen by measurement on the order-3 workloads:
// occupancy outweighs a few spilled registers, not many; higher orders need
// two blocks' budget.
template <typename T, int N, int KIND>
constexpr int min_blocks() {
    if (KIND == stream::kGather) return min_blocks<T, N, stream::kMttkrp>();  // MTTKRP's launch
    if (N == 2) return 4;
    if (N != 3) return 2;
    if (KIND == stream::kLossBwd) return sizeof(T) == 4 ? 4 : 3;  // with the late row-0 load
    return sizeof(T) == 4 ? 4 : 3;
}

// The backward kind loads the sorted mode's row where a run starts, in phase
// B (R0L = 1), instead of holding a register row per entry of the batch: that
// let the FP32 order-3 kernel fit 4 blocks per SM with 24 bytes of spills
// (88 with the row held), 2.24 -> 2.09 ms per zipf3d pass.  It costs uniform
// cploss3d 5% (0.46 -> 0.48 ms), whose runs and rows sit in L2 anyway.
template <int KIND>
constexpr int row0_late() {
    return KIND == stream::kLossBwd ? 1 : 0;
}

// LC > 0 compiles the lane count of a row in (LC must equal the geometry's
// L); LC = 0 reads it from the arguments.
template <typename T, int N, int KIND, int LC>
pasta_status run(const StreamLaunch &l, cudaStream_t s) {
    constexpr int MINB = min_blocks<T, N, KIND>();
    Args<T, N> a{};
    for (int p = 0; p < N; ++p) {
        a.idx[p] = l.idx[p];
        a.U[p] = static_cast<const T *>(l.U[p]);
    }
    a.val = l.val;
    a.out = l.out;
    a.partials = l.partials;
    a.gscale = l.gscale;
    a.nnz = l.nnz;
    a.R = (uint32_t)l.R;
    const Geometry g = make_geometry(l.R, 16 / (int)sizeof(T), (int)sizeof(T));
    if (LC != 0 && g.L != LC) return PASTA_ERR_UNSUPPORTED;  // by_lanes picks LC = L
    a.L = g.L;
    a.lshift = g.lshift;
    const size_t smem = stream::smem_bytes(N, kStages, g.L, l.R);
    auto kern = k_stream<T, N, KIND, kStages, MINB, LC, row0_late<KIND>()>;
    PASTA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PASTA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    per_sm = std::max(per_sm, 1);
    // Block tiles go round-robin over the resident grid.  With the longest
    // group tile the last round may leave most blocks idle, so the tile is
    // shortened (to a multiple of the chunk) until the block tiles just fill
    // the same number of rounds.
    const uint64_t per_bt = (uint64_t)(32 >> g.lshift) * kWarps;  // group tiles per block tile
    const uint64_t chunk = 4 * (uint64_t)g.L;
    const uint64_t longest = (uint64_t)stream::group_tile(g.L);
    const uint64_t nbt0 = std::max<uint64_t>(1, (l.nnz + longest * per_bt - 1) / (longest * per_bt));
    uint64_t blocks = std::min<uint64_t>(nbt0, (uint64_t)l.num_sms * (uint64_t)per_sm);
    if (l.max_blocks > 0) blocks = std::min<uint64_t>(blocks, (uint64_t)l.max_blocks);
    blocks = apply_grid_cap(blocks);
    const uint64_t rounds = (nbt0 + blocks - 1) / blocks;
    const uint64_t need = (l.nnz + blocks * rounds * per_bt - 1) / (blocks * rounds * per_bt);
    a.tile = (int)std::min<uint64_t>(longest, std::max<uint64_t>(chunk, (need + chunk - 1) / chunk * chunk));
    if (l.zero_tile_end_rows) {
        const uint64_t ntiles = (l.nnz + a.tile - 1) / a.tile;
        k_zero_tile_end_rows<<<(unsigned)((ntiles + 7) / 8), 256, 0, s>>>(l.idx[0], l.nnz, (uint32_t)a.tile,
                                                                       (uint32_t)l.R, l.out);
    }
    kern<<<(int)blocks, kThreads, smem, s>>>(a);
    PASTA_CUDA(cudaGetLastError());
    if (l.blocks_used) *l.blocks_used = (int)blocks;
    return PASTA_OK;
}

// MTTKRP and the loss kinds get a compiled-in lane count for the common row
// widths (32..256 bytes: R = 8..64 in FP32, 16..128 in 16-bit); it turns the
// lane group's strides, shared-memory offsets and shuffle widths into
// constants and unrolls the chunk's batches (loss passes 4-6% faster, MTTKRP
// 0.2-1.2%).  The gather probe is compiled the same way as MTTKRP.
template <typename T, int N, int KIND>
pasta_status by_lanes(const StreamLaunch &l, cudaStream_t s) {
    {
        switch (l.R * (int)sizeof(T) / 16) {
            case 2: return run<T, N, KIND, 2>(l, s);
            case 4: return run<T, N, KIND, 4>(l, s);
            case 8: return run<T, N, KIND, 8>(l, s);
            case 16: return run<T, N, KIND, 16>(l, s);
            default: return run<T, N, KIND, 0>(l, s);
        }
    }
}

template <typename T, int KIND>
pasta_status by_order(const StreamLaunch &l, cudaStream_t s) {
    switch (l.order) {
        case 2:  // MTTKRP only (TTM/TTV run as an order-2 MTTKRP)
            if constexpr (KIND == stream::kMttkrp || KIND == stream::kGather) return by_lanes<T, 2, KIND>(l, s);
            return PASTA_ERR_UNSUPPORTED;
        case 3: return by_lanes<T, 3, KIND>(l, s);
        case 4: return by_lanes<T, 4, KIND>(l, s);
        case 5: return by_lanes<T, 5, KIND>(l, s);
    }
    return PASTA_ERR_UNSUPPORTED;
}

template <int KIND>
pasta_status by_type(const StreamLaunch &l, cudaStream_t s) {
    switch (l.dtype) {
        case PASTA_F32: return by_order<float, KIND>(l, s);
        case PASTA_BF16: return by_order<__nv_bfloat16, KIND>(l, s);
        case PASTA_F16: return by_order<__half, KIND>(l, s);
        default: return PASTA_ERR_UNSUPPORTED;
    }
}

}  // namespace stream_launch

// One per kind, each defined in its own translation unit.
pasta_status launch_stream_mttkrp(const StreamLaunch &l, cudaStream_t s);
pasta_status launch_stream_loss_fwd(const StreamLaunch &l, cudaStream_t s);
pasta_status launch_stream_loss_bwd(const StreamLaunch &l, cudaStream_t s);
pasta_status launch_stream_gather(const StreamLaunch &l, cudaStream_t s);

}  // namespace pasta
