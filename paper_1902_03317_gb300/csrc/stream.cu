// Entry to the streaming kernels (stream_kernels.cuh) for MTTKRP, the CP-loss
// forward and the per-mode CP-loss backward: the coverage test and the
// dispatch to the per-kind launchers (stream_mttkrp.cu, stream_loss_fwd.cu,
// stream_loss_bwd.cu).
//
// Covered: FP32/BF16/FP16 factors, order 3..5 (2..5 for MTTKRP), 16-byte aligned factors and
// outputs, and R * sizeof(element) = 16 * L with L a power of two <= 32 (so
// the L lanes of a group cover a row exactly).  Anything else returns
// PASTA_ERR_UNSUPPORTED and the caller uses the general kernels.
#include "stream_launch.cuh"

namespace pasta {
namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

bool stream_supported(pasta_dtype dt, int order, int R, const void *const *U, int skip,
                      const void *out, int min_order) {
    if (dt != PASTA_F32 && dt != PASTA_BF16 && dt != PASTA_F16) return false;
    if (order < min_order || order > 5) return false;
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
        case stream::kMttkrp: return launch_stream_mttkrp(l, s);
        case stream::kLossFwd: return launch_stream_loss_fwd(l, s);
        case stream::kLossBwd: return launch_stream_loss_bwd(l, s);
        case stream::kGather: return launch_stream_gather(l, s);
    }
    return PASTA_ERR_UNSUPPORTED;
}

}  // namespace pasta
