// MTTKRP instantiations of the streaming kernel (Algorithm 6 over a
// mode-sorted copy); see stream_launch.cuh.
#include "stream_launch.cuh"

namespace pasta {

pasta_status launch_stream_mttkrp(const StreamLaunch &l, cudaStream_t s) {
    return stream_launch::by_type<stream::kMttkrp>(l, s);
}

}  // namespace pasta
