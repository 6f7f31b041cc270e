// pyramid.cu -- luma and Gaussian pyramid REDUCE kernels.
//
// The flow of Section III-C-1 is estimated with the "LK pyramid algorithm";
// the pyramid is the Burt-Adelson REDUCE: the binomial [1 4 6 4 1]/16
// along y, then along x, replicate border, keeping the even rows and
// columns (level size ceil(h/2) x ceil(w/2)). Level 0 is the BT.601 luma of
// the unit-scaled strip.
#include "common.cuh"

namespace pano {

namespace {

constexpr float kInv255 = 1.0f / 255.0f;

// ---------------------------------------------------------------------------
// Level 0: one thread per pixel. Both strips in one launch (blockIdx.z).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) luma_kernel(LumaArgs a) {
    const ImageDesc& in = a.in[blockIdx.z];
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= in.w || y >= in.h) return;
    float v;
    if (in.dtype == 0) {
        const uint8_t* row = static_cast<const uint8_t*>(in.data) + (long long)y * in.pitch_bytes;
        if (in.c == 3) {
            const uint8_t* px = row + 3 * x;
            v = (0.299f * px[0] + 0.587f * px[1] + 0.114f * px[2]) * kInv255;
        } else {
            v = row[x] * kInv255;
        }
    } else {
        const float* row = reinterpret_cast<const float*>(
            static_cast<const char*>(in.data) + (long long)y * in.pitch_bytes);
        if (in.c == 3) {
            const float* px = row + 3 * x;
            v = 0.299f * px[0] + 0.587f * px[1] + 0.114f * px[2];
        } else {
            v = row[x];
        }
    }
    a.out[blockIdx.z][(long long)y * a.out_pitch[blockIdx.z] + x] = v;
}

// ---------------------------------------------------------------------------
// REDUCE: a 32 x 8 tile of the destination per 256-thread block. The source
// footprint (2*8+3 rows x 2*32+3 columns, clamped) is staged in shared
// memory, blurred along y at the even rows, then along x at the even
// columns.
// ---------------------------------------------------------------------------
constexpr int kPdTW = 32, kPdTH = 8;
constexpr int kPdSW = 2 * kPdTW + 3;  // source columns 2*x0-2 .. 2*(x0+31)+2
constexpr int kPdSH = 2 * kPdTH + 3;

__global__ void __launch_bounds__(256) pyr_down_kernel(PyrDownArgs a) {
    __shared__ float s_src[kPdSH][kPdSW + 1];
    __shared__ float s_v[kPdTH][kPdSW + 1];
    const float* __restrict__ src = a.src[blockIdx.z];
    float* __restrict__ dst = a.dst[blockIdx.z];
    const int hd = (a.h + 1) >> 1, wd = (a.w + 1) >> 1;
    const int xd0 = blockIdx.x * kPdTW, yd0 = blockIdx.y * kPdTH;
    const int sx0 = 2 * xd0 - 2, sy0 = 2 * yd0 - 2;
    const int tid = threadIdx.y * kPdTW + threadIdx.x;
    for (int i = tid; i < kPdSH * kPdSW; i += 256) {
        int r = i / kPdSW, c = i - r * kPdSW;
        int sy = min(max(sy0 + r, 0), a.h - 1);
        int sx = min(max(sx0 + c, 0), a.w - 1);
        s_src[r][c] = __ldg(src + (long long)sy * a.src_pitch[blockIdx.z] + sx);
    }
    __syncthreads();
    const float k0 = 1.0f / 16, k1 = 4.0f / 16, k2 = 6.0f / 16;
    for (int i = tid; i < kPdTH * kPdSW; i += 256) {
        int r = i / kPdSW, c = i - r * kPdSW;
        int sr = 2 * r + 2;
        s_v[r][c] = k0 * s_src[sr - 2][c] + k1 * s_src[sr - 1][c] + k2 * s_src[sr][c] +
                    k1 * s_src[sr + 1][c] + k0 * s_src[sr + 2][c];
    }
    __syncthreads();
    int xd = xd0 + threadIdx.x, yd = yd0 + threadIdx.y;
    if (xd < wd && yd < hd) {
        int c = 2 * threadIdx.x + 2;
        const float* v = s_v[threadIdx.y];
        dst[(long long)yd * a.dst_pitch[blockIdx.z] + xd] =
            k0 * v[c - 2] + k1 * v[c - 1] + k2 * v[c] + k1 * v[c + 1] + k0 * v[c + 2];
    }
}

}  // namespace

cudaError_t launch_luma(const LumaArgs& a, cudaStream_t s) {
    int h = max(a.in[0].h, a.count > 1 ? a.in[1].h : 0);
    int w = max(a.in[0].w, a.count > 1 ? a.in[1].w : 0);
    dim3 block(32, 8);
    dim3 grid((w + 31) / 32, (h + 7) / 8, a.count);
    luma_kernel<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pyr_down(const PyrDownArgs& a, cudaStream_t s) {
    int hd = (a.h + 1) / 2, wd = (a.w + 1) / 2;
    dim3 block(kPdTW, kPdTH);
    dim3 grid((wd + kPdTW - 1) / kPdTW, (hd + kPdTH - 1) / kPdTH, a.count);
    pyr_down_kernel<<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pano
