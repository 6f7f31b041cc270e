// lk_stream.cu -- the streamed LK kernel (lk_stream_impl.cuh) for float32
// pyramid planes, and the dispatch over storage types. The bfloat16 and
// binary16 instantiations live in lk_stream_bf16.cu and lk_stream_f16.cu so
// that the three compile in parallel.
#include "lk_stream_impl.cuh"

namespace pano {

namespace lks {
PANO_LKS_INSTANTIATE(float)
PANO_LKS_EXTERN(__nv_bfloat16)
PANO_LKS_EXTERN(__half)
}  // namespace lks

PANO_BOUNDS_READER(bounds_read_lk_stream)

bool lk_stream_supports(int iters, int radius) { return iters >= 1 && iters <= 5 && radius >= 1 && radius <= 3; }

cudaError_t lk_stream_prepare(int max_smem_bytes) {
    cudaError_t e;
    if ((e = lks::stream_prepare<float>(max_smem_bytes)) != cudaSuccess) return e;
    if ((e = lks::stream_prepare<__nv_bfloat16>(max_smem_bytes)) != cudaSuccess) return e;
    return lks::stream_prepare<__half>(max_smem_bytes);
}

cudaError_t launch_lk_stream_batch(const LkBatch& b, int n_ctas, cudaStream_t s) {
    if (b.n < 1 || b.n > kMaxBatch) return cudaErrorInvalidValue;
    for (int p = 1; p < b.n; ++p)
        if (b.pair[p].pyr != b.pair[0].pyr || b.pair[p].iters != b.pair[0].iters ||
            b.pair[p].radius != b.pair[0].radius)
            return cudaErrorInvalidValue;
    switch (b.pair[0].pyr) {
        case kPyrF32: return lks::stream_launch_batch<float>(b, n_ctas, s);
        case kPyrBF16: return lks::stream_launch_batch<__nv_bfloat16>(b, n_ctas, s);
        case kPyrF16: return lks::stream_launch_batch<__half>(b, n_ctas, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_lk_stream(const LkArgs& a, int ndirs, cudaStream_t s) {
    switch (a.pyr) {
        case kPyrF32: return lks::stream_launch<float>(a, ndirs, s);
        case kPyrBF16: return lks::stream_launch<__nv_bfloat16>(a, ndirs, s);
        case kPyrF16: return lks::stream_launch<__half>(a, ndirs, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pano
