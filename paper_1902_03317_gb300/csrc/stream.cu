// Launchers of the streaming kernels (stream_kernels.cuh) for MTTKRP, the
// CP-loss forward and the per-mode CP-loss backward.
//
// Covered: FP32/BF16/FP16 factors, order 3..5, 16-byte aligned factors and
// outputs, and R * sizeof(element) = 16 * L with L a power of two <= 32 (so
// the L lanes of a group cover a row exactly).  Anything else returns
// PASTA_ERR_UNSUPPORTED and the caller uses the general kernels.
#include <algorithm>

#include "stream_kernels.cuh"

namespace pasta {
namespace {

using stream::Args;
using stream::k_stream;
using stream::kThreads;
using stream::kWarps;

constexpr int kStages = 2;

// Blocks per SM each instantiation is compiled for (register budget
// 65536 / (256 * blocks)), chosen by measurement on the order-3 workloads:
// occupancy outweighs a few spilled registers for MTTKRP and the forward,
// not for the backward; higher orders need two blocks' budget.
template <typename T, int N, int KIND>
constexpr int min_blocks() {
    if (N != 3) return 2;
    if (KIND == 2) return 3;  // the backward spills too much at 4
    return sizeof(T) == 4 ? 4 : 3;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename T, int N, int KIND>
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
    a.L = g.L;
    a.lshift = g.lshift;
    a.tile = g.tile;
    const size_t smem = stream::smem_bytes(N, kStages, g.L, l.R);
    auto kern = k_stream<T, N, KIND, kStages, MINB>;
    PASTA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    PASTA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    per_sm = std::max(per_sm, 1);
    const uint64_t span = (uint64_t)g.tile * (uint64_t)(32 >> g.lshift) * kWarps;
    const uint64_t nbt = std::max<uint64_t>(1, (l.nnz + span - 1) / span);
    uint64_t blocks = std::min<uint64_t>(nbt, (uint64_t)l.num_sms * (uint64_t)per_sm);
    if (l.max_blocks > 0) blocks = std::min<uint64_t>(blocks, (uint64_t)l.max_blocks);
    kern<<<(int)blocks, kThreads, smem, s>>>(a);
    PASTA_CUDA(cudaGetLastError());
    if (l.blocks_used) *l.blocks_used = (int)blocks;
    return PASTA_OK;
}

template <typename T, int KIND>
pasta_status by_order(const StreamLaunch &l, cudaStream_t s) {
    switch (l.order) {
        case 3: return run<T, 3, KIND>(l, s);
        case 4: return run<T, 4, KIND>(l, s);
        case 5: return run<T, 5, KIND>(l, s);
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

}  // namespace

bool stream_supported(pasta_dtype dt, int order, int R, const void *const *U, int skip,
                      const void *out) {
    if (dt != PASTA_F32 && dt != PASTA_BF16 && dt != PASTA_F16) return false;
    if (order < 3 || order > 5) return false;
    const int bytes = R * (int)dtype_size(dt);
    if (bytes % 16 != 0) return false;
    const int L = bytes / 16;
    if (L < 1 || L > 32 || (L & (L - 1)) != 0) return false;
    for (int k = 0; k < order; ++k)
        if (k != skip && !aligned16(U[k])) return false;
    if (out && !aligned16(out)) return false;
    return true;
}

pasta_status launch_stream(int kind, const StreamLaunch &l, cudaStream_t s) {
    switch (kind) {
        case stream::kMttkrp: return by_type<stream::kMttkrp>(l, s);
        case stream::kLossFwd: return by_type<stream::kLossFwd>(l, s);
        case stream::kLossBwd: return by_type<stream::kLossBwd>(l, s);
    }
    return PASTA_ERR_UNSUPPORTED;
}

}  // namespace pasta
