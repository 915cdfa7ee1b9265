// CP-loss backward instantiations of the streaming kernel (one factor's
// gradient per launch, optionally also the loss partial sums); see
// stream_launch.cuh.
#include "stream_launch.cuh"

namespace pasta {

pasta_status launch_stream_loss_bwd(const StreamLaunch &l, cudaStream_t s) {
    return stream_launch::by_type<stream::kLossBwd>(l, s);
}

}  // namespace pasta
