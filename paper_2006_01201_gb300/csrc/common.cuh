// common.cuh -- internal declarations shared by the kernels and the C ABI of
// the optical-flow blend (Section III-C of the paper). Not a public header.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pano {

constexpr int kMaxLevels = 12;

// Storage type of the pyramid planes. Arithmetic is FP32 throughout; a
// 16-bit plane is widened on load and rounded to nearest even on store.
enum PyrType : int { kPyrF32 = 0, kPyrBF16 = 1, kPyrF16 = 2 };

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }

template <class Ts>
__device__ __forceinline__ Ts from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }

// Read-only load of one stored element, widened to FP32.
template <class Ts>
__device__ __forceinline__ float ld_f32(const Ts* p) { return to_f32(__ldg(p)); }

// A float32 plane in device memory: rows of `pitch` elements.
struct Plane {
    const float* p;
    int pitch;
};

// ---------------------------------------------------------------------------
// Bilinear sample of a float plane at (qx + ox, qy + oy), pixel centres on
// integer coordinates, each of the four taps clamped to [0, w-1] x [0, h-1].
// The integer base (qx, qy) and the real offset (ox, oy) are kept apart so
// that the fractional weights come from the offset alone: their rounding
// error does not grow with the position in a large strip.
// ---------------------------------------------------------------------------
struct Taps {
    int o00, o10, o01, o11;  // element offsets of the four taps
    float ax, ay;            // weights of the second column / second row
};

__device__ __forceinline__ Taps bilinear_taps(int qx, int qy, float ox, float oy, int w, int h,
                                              int pitch_elems, int elem_stride) {
    // Beyond +-(size + 2) every tap clamps to the same edge pixel, so limiting
    // the offset first changes no result and keeps the conversion defined.
    ox = fminf(fmaxf(ox, -(float)(w + 2)), (float)(w + 2));
    oy = fminf(fmaxf(oy, -(float)(h + 2)), (float)(h + 2));
    float fx = floorf(ox), fy = floorf(oy);
    Taps t;
    t.ax = ox - fx;
    t.ay = oy - fy;
    int x0 = qx + (int)fx, y0 = qy + (int)fy;
    int xa = min(max(x0, 0), w - 1), xb = min(max(x0 + 1, 0), w - 1);
    int ya = min(max(y0, 0), h - 1), yb = min(max(y0 + 1, 0), h - 1);
    t.o00 = ya * pitch_elems + xa * elem_stride;
    t.o10 = ya * pitch_elems + xb * elem_stride;
    t.o01 = yb * pitch_elems + xa * elem_stride;
    t.o11 = yb * pitch_elems + xb * elem_stride;
    return t;
}

__device__ __forceinline__ float bilinear_mix(const Taps& t, float i00, float i10, float i01,
                                              float i11) {
    float top = fmaf(t.ax, i10 - i00, i00);
    float bot = fmaf(t.ax, i11 - i01, i01);
    return fmaf(t.ay, bot - top, top);
}

template <class Ts>
__device__ __forceinline__ float sample_plane(const Ts* __restrict__ img, int pitch, int w, int h,
                                              int qx, int qy, float ox, float oy) {
    Taps t = bilinear_taps(qx, qy, ox, oy, w, h, pitch, 1);
    return bilinear_mix(t, ld_f32(img + t.o00), ld_f32(img + t.o10), ld_f32(img + t.o01),
                        ld_f32(img + t.o11));
}

// ---------------------------------------------------------------------------
// Launch descriptors (host fills, kernels read by value).
// ---------------------------------------------------------------------------
struct ImageDesc {
    const void* data;
    int h, w, c;
    long long pitch_bytes;
    int dtype;  // 0 = u8, 1 = f32
};

// Strip pairs in one batched launch, and the planes (two per pair) they hold.
constexpr int kMaxBatch = 8;
constexpr int kMaxPlanes = 2 * kMaxBatch;

// Level-0 luma of up to kMaxPlanes images in one launch (blockIdx.z selects
// one; kernels take the descriptor as a __grid_constant__ parameter and index
// it in place).
struct LumaArgs {
    ImageDesc in[kMaxPlanes];
    void* out[kMaxPlanes];          // planes of type pyr
    int out_pitch[kMaxPlanes];      // elements
    int count;
    int pyr;                        // PyrType of the output planes
};

// Level 0 (luma) and level 1 (its REDUCE) of up to kMaxPlanes images in one
// launch.
struct LumaReduceArgs {
    ImageDesc in[kMaxPlanes];
    void* l0[kMaxPlanes];           // planes of type pyr
    void* l1[kMaxPlanes];
    int l0_pitch[kMaxPlanes], l1_pitch[kMaxPlanes];  // elements
    int count;
    int pyr;
};

// Several REDUCE steps of up to kMaxPlanes planes in one launch: levels
// s+1 .. s+levels from level s (pyramid.cu, pyr_tail_kernel).
constexpr int kTailMaxLevels = 4;
struct PyrTailArgs {
    const void* src[kMaxPlanes];    // level s, planes of type pyr
    int src_pitch[kMaxPlanes];
    int h[kMaxPlanes], w[kMaxPlanes];  // size of level s
    void* dst[kMaxPlanes][kTailMaxLevels];  // levels s+1 .. s+levels
    int dst_pitch[kMaxPlanes][kTailMaxLevels];
    int count, levels, pyr;
};

// One REDUCE step of up to kMaxPlanes planes of any sizes in one launch.
struct PyrDownArgs {
    const void* src[kMaxPlanes];    // planes of type pyr
    void* dst[kMaxPlanes];
    int src_pitch[kMaxPlanes], dst_pitch[kMaxPlanes];  // elements
    int h[kMaxPlanes], w[kMaxPlanes];  // source sizes
    int count;
    int pyr;                        // PyrType of every plane
};

// One pyramid level of Lucas-Kanade in up to two directions (blockIdx.z).
struct LkDir {
    const void* T;    // template level (PyrType of LkArgs::pyr)
    const void* J;    // target level
    const float* uin; // starting / coarse flow (float2 elements), may be null
    float* uout;      // result (float2 elements)
    int pitchT, pitchJ;  // in elements
    int uin_pitch;    // in float2 elements
    int uout_pitch;   // in float2 elements
};

struct LkArgs {
    LkDir dir[2];
    int h, w;            // level size
    int in_h, in_w;      // size of uin
    int mode;            // 0 zero start, 1 upsample coarse uin, 2 uin as is
    int iters, radius;
    float lambda;
    int tile_w, tile_h;  // tiled kernel
    int seg_rows;        // streamed kernel: segment height (0 = automatic)
    int pyr;             // PyrType of T and J
};

// The same pyramid level of several strip pairs in one launch (all share
// iters and radius): persistent for the streamed kernel, one grid over every
// pair and direction for the tiled one (all pairs then share the tile shape).
struct LkBatch {
    LkArgs pair[kMaxBatch];
    int n;
    int nb[kMaxBatch], seg[kMaxBatch], nseg[kMaxBatch];  // filled by the launcher
    int start[kMaxBatch + 1];                             // item prefix sums
    unsigned* counter;                                    // device work counter
};

// Code 1 blend or the plain flow warp.
struct BlendArgs {
    ImageDesc L, R;
    const float2* flowLR;
    const float2* flowRL;
    const float* blend;  // (h, w) or null -> Eq. (1) strip ramp
    void* F;
    long long F_pitch_bytes;
    float k_sharp, k_mag;
    float inv_w, inv_w1;  // 1 / w and 1 / (w + 1), rounded to nearest (the launchers set them)
};

// The reciprocals a blend launch multiplies by instead of dividing.
inline void set_blend_scales(BlendArgs* a) {
    a->inv_w = 1.0f / (float)a->L.w;
    a->inv_w1 = 1.0f / (float)(a->L.w + 1);
}

// Blend of every pair of a rig into one canvas (F of each pair is the canvas
// row of strip row 0; the column comes from x0).
struct RigBlendArgs {
    BlendArgs pair[kMaxBatch];
    int x0[kMaxBatch];  // canvas column of strip column 0, in [0, canvas_w)
    int n;
    int canvas_w;
};

// Code 1 on a whole canvas (every branch).
struct ComposeArgs {
    ImageDesc L, R;                 // canvas images (same h, w, c, dtype)
    const unsigned char* label;     // (h, w): 1 Area1, 2 Area2, 3 Area3, else neither
    long long label_pitch;          // bytes
    const float* blend;             // (h, w) Eq. (1)
    int blend_pitch;                // floats
    const float2* flowLR;           // (fh, fw) flows of the overlap crop
    const float2* flowRL;
    int fy0, fx0, fh, fw;           // canvas position and size of the crop
    void* F;
    long long F_pitch_bytes;
    float k_sharp, k_mag;
    float inv_fw;                   // 1 / fw, rounded to nearest
};

struct WarpArgs {
    ImageDesc src;
    const float2* flow;
    float scale;
    float* dst;
    long long dst_pitch_bytes;
};

// Energy and gradients of the differentiable refinement (refine.cu).
struct EnergyArgs {
    const float* T;
    const float* J;
    const float* u;      // (h, w, 2)
    int h, w, pitch;     // pitch of T and J in floats
    float alpha;
    double* energy;      // one double, or null
    float* grad_u;       // (h, w, 2) or null
    float* grad_T;       // (h, w) or null
    float* grad_J;       // (h, w) or null (zeroed by the launcher)
};

// Launchers: enqueue on `s`, return the launch error (cudaSuccess if none).
cudaError_t launch_luma(const LumaArgs& a, cudaStream_t s);
cudaError_t launch_pyr_down(const PyrDownArgs& a, cudaStream_t s);
cudaError_t launch_luma_reduce(const LumaReduceArgs& a, cudaStream_t s);
cudaError_t launch_pyr_tail(const PyrTailArgs& a, cudaStream_t s);
cudaError_t pyr_tail_prepare(int max_smem_bytes);
// One LK level: streamed (lk_stream.cu) for levels of at least
// kStreamMinPixels pixels and 1 <= iters <= 5, tiled (lk.cu) otherwise.
// Levels below kSmallTilePixels use small tiles (kSmallTileW x kSmallTileH):
// their few large tiles would leave most SMs idle, and the time of such a
// level is the latency of one tile. (Measured on GB300: a 94k-pixel level
// takes 38 us streamed and 51 us tiled; a 5.9k-pixel level 15 us on 16x8
// tiles and 21 us on 32x16.)
constexpr long long kStreamMinPixels = 50000;
constexpr long long kSmallTilePixels = 16000;
constexpr int kSmallTileW = 16, kSmallTileH = 8;
// Tile of the tiled kernel for a level of w x h pixels, given the default.
inline void lk_level_tile(int w, int h, int def_w, int def_h, int* tw, int* th) {
    const bool small = (long long)w * h < kSmallTilePixels;
    *tw = small ? kSmallTileW : def_w;
    *th = small ? kSmallTileH : def_h;
}
cudaError_t launch_lk_level(const LkArgs& a, int ndirs, cudaStream_t s);
cudaError_t launch_lk_tile(const LkArgs& a, int ndirs, cudaStream_t s);
cudaError_t launch_lk_tile_batch(const LkBatch& b, cudaStream_t s);
// Streamed form of the same level (lk_stream.cu), used for 1 <= iters <= 5.
bool lk_stream_supports(int iters, int radius);
cudaError_t lk_stream_prepare(int max_smem_bytes);
cudaError_t launch_lk_stream(const LkArgs& a, int ndirs, cudaStream_t s);
cudaError_t launch_lk_stream_batch(const LkBatch& b, int n_ctas, cudaStream_t s);
size_t lk_smem_bytes(int tile_w, int tile_h, int iters, int radius);
cudaError_t lk_prepare(int max_smem_bytes);
cudaError_t launch_blend(const BlendArgs& a, cudaStream_t s);
cudaError_t launch_rig_blend(const RigBlendArgs& r, cudaStream_t s);
cudaError_t launch_warp(const WarpArgs& a, cudaStream_t s);
cudaError_t launch_compose(const ComposeArgs& a, cudaStream_t s);

// Eq. (1) on a labelled canvas through an exact distance transform (edt.cu).
size_t blend_coeff_scratch_bytes(int h, int w);
size_t blend_coeff_row_smem(int w);
cudaError_t blend_coeff_prepare(int max_smem_bytes);
cudaError_t launch_blend_coeff(const unsigned char* label, int h, int w, long long pitch, float* blend,
                               int blend_pitch, void* scratch, cudaStream_t s);

cudaError_t launch_energy_grad(const EnergyArgs& a, cudaStream_t s);
cudaError_t launch_pyr_down_adjoint(const float* gdst, int h, int w, int dst_pitch, float* gsrc, int src_pitch,
                                    cudaStream_t s);

// Index-check records of the debug build (bounds.cuh), one per translation
// unit: each adds its record to out[4] and clears it (no-ops in the normal
// build).
cudaError_t bounds_read_lk_stream(unsigned* out);
cudaError_t bounds_read_lk_stream_bf16(unsigned* out);
cudaError_t bounds_read_lk_stream_f16(unsigned* out);
cudaError_t bounds_read_lk_tile(unsigned* out);
cudaError_t bounds_read_pyramid(unsigned* out);
cudaError_t bounds_read_blend(unsigned* out);
cudaError_t bounds_read_edt(unsigned* out);
cudaError_t bounds_read_refine(unsigned* out);

// Stores the message that pano_last_error() returns on the calling thread.
void set_last_error(const char* msg);

}  // namespace pano
