// lk_stream_bf16.cu -- the streamed LK kernel (lk_stream_impl.cuh) for
// __nv_bfloat16 pyramid planes.
#include "lk_stream_impl.cuh"

namespace pano {
namespace lks {
PANO_LKS_INSTANTIATE(__nv_bfloat16)
}  // namespace lks
PANO_BOUNDS_READER(bounds_read_lk_stream_bf16)
}  // namespace pano
