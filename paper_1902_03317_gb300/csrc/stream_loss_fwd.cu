// CP-loss forward instantiations of the streaming kernel (residuals and the
// loss partial sums); see stream_launch.cuh.
#include "stream_launch.cuh"

namespace pasta {

pasta_status launch_stream_loss_fwd(const StreamLaunch &l, cudaStream_t s) {
    return stream_launch::by_type<stream::kLossFwd>(l, s);
}

}  // namespace pasta
