// Gather-only instantiations of the streaming kernel (the diagnostic behind
// pasta_gather_probe: MTTKRP's row gathers without its arithmetic or output);
// see stream_launch.cuh.
#include "stream_launch.cuh"

namespace pasta {

pasta_status launch_stream_gather(const StreamLaunch &l, cudaStream_t s) {
    return stream_launch::by_type<stream::kGather>(l, s);
}

}  // namespace pasta
