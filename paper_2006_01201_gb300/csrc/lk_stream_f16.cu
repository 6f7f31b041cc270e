// lk_stream_f16.cu -- the streamed LK kernel (lk_stream_impl.cuh) for
// __half pyramid planes.
#include "lk_stream_impl.cuh"

namespace pano {
namespace lks {
PANO_LKS_INSTANTIATE(__half)
}  // namespace lks
PANO_BOUNDS_READER(bounds_read_lk_stream_f16)
}  // namespace pano
