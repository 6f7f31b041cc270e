// blend.cu -- the asymmetric softmax blend of Code 1 (Section III-C-3) with
// the global blending coefficient of Eq. (1) (Section III-C-2): on overlap
// strips, on a rig's canvas and on a whole canvas with every branch of
// Code 1; and the plain bilinear flow warp.
//
// Code 1, Area3 branch, at pixel p = (x, y) of the overlap strips:
//   BlendL = 1 - Blend(p), BlendR = Blend(p)
//   ColorL = L(p + (1 - BlendL) FlowRtoL(p)),  ColorR = R(p + (1 - BlendR) FlowLtoR(p))
//   FlowL = 1 + kFlowMagCoef FlowMagRL,  FlowR = 1 + kFlowMagCoef FlowMagLR
//   F = (ColorL e^{k BlendL FlowL} + ColorR e^{k BlendR FlowR}) / (e^{k BlendL FlowL} + e^{k BlendR FlowR})
// FlowMagRL / FlowMagLR are |FlowRtoL(p)| / w and |FlowLtoR(p)| / w. With no
// Blend array the strip value of Eq. (1) is used, (x + 1) / (w + 1). The
// softmax is evaluated as the equal logistic form 1 / (1 + e^{sR - sL}).
#include "bounds.cuh"
#include "common.cuh"

namespace pano {

namespace {

// A stored sample as float. A byte b becomes exactly b through the float
// whose bits are those of 2^23 with b in the low mantissa bits, minus 2^23:
// one logic operation and one add instead of an integer-to-float conversion.
__device__ __forceinline__ float sample_f(float v) { return v; }
__device__ __forceinline__ float sample_f(uint8_t b) {
    return __uint_as_float(0x4B000000u | (unsigned)b) - 8388608.0f;
}

// round(f) to [0, 255], ties to even: after clamping, f + 2^23 is rounded by
// the add to the nearest integer (ties to even) and that integer is the low
// mantissa byte. Clamping first gives what rounding and then clamping gives.
__device__ __forceinline__ uint8_t to_u8_rn(float f) {
    f = fminf(fmaxf(f, 0.f), 255.f);  // a NaN becomes 0
    return (uint8_t)(__float_as_uint(f + 8388608.0f) & 0xFFu);
}

// Bilinear sample of channel k of an interleaved image, raw sample scale
// (0..255 for u8, as stored for f32).
template <typename Tv>
__device__ __forceinline__ float sample_channel(const Tv* __restrict__ base, const Taps& t, int k, long long n) {
    (void)n;  // elements of the image ((h - 1) rows of its pitch and w C): the bound of the index checks
    return bilinear_mix(t, sample_f(PANO_AT(base, t.o00 + k, n, 401)), sample_f(PANO_AT(base, t.o10 + k, n, 402)),
                        sample_f(PANO_AT(base, t.o01 + k, n, 403)), sample_f(PANO_AT(base, t.o11 + k, n, 404)));
}

// Code 1, Area3 branch, at pixel (x, y) of images L, R (h x w, row pitches
// in elements): Blend B, flows rl = FlowRtoL(p) and lr = FlowLtoR(p),
// inv_w = 1 / (width of the overlap strip); C channels to out.
template <typename Tv, int C>
__device__ __forceinline__ void code1_area3(const Tv* __restrict__ Lb, int pitchL, const Tv* __restrict__ Rb,
                                            int pitchR, int w, int h, int x, int y, float B, float2 rl,
                                            float2 lr, float inv_w, float k_sharp, float k_mag, Tv* out) {
    const float blendL = 1.f - B, blendR = B;
    // ColorL at p + (1 - BlendL) FlowRtoL, ColorR at p + (1 - BlendR) FlowLtoR
    const Taps tl = bilinear_taps(x, y, (1.f - blendL) * rl.x, (1.f - blendL) * rl.y, w, h, pitchL, C);
    const Taps tr = bilinear_taps(x, y, (1.f - blendR) * lr.x, (1.f - blendR) * lr.y, w, h, pitchR, C);
    const float magRL = sqrtf(fmaf(rl.x, rl.x, rl.y * rl.y)) * inv_w;
    const float magLR = sqrtf(fmaf(lr.x, lr.x, lr.y * lr.y)) * inv_w;
    const float sL = k_sharp * blendL * fmaf(k_mag, magRL, 1.f);
    const float sR = k_sharp * blendR * fmaf(k_mag, magLR, 1.f);
    const float e = expf(fminf(fmaxf(sR - sL, -80.f), 80.f));
    const float wL = 1.f / (1.f + e);
    const float wR = e * wL;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        const float cl = sample_channel(Lb, tl, k, (long long)(h - 1) * pitchL + (long long)w * C);
        const float cr = sample_channel(Rb, tr, k, (long long)(h - 1) * pitchR + (long long)w * C);
        const float f = fmaf(cl, wL, cr * wR);
        if constexpr (sizeof(Tv) == 1) {
            out[k] = to_u8_rn(f);
        } else {
            out[k] = (Tv)f;
        }
    }
}

// F at strip pixel (x, y), stored at column `fx` of row y of a.F.
template <typename Tv, int C>
__device__ __forceinline__ void blend_pixel(const BlendArgs& a, int x, int y, int fx) {
    const int w = a.L.w, h = a.L.h;
    const long long p = (long long)y * w + x;
    const float B = a.blend ? a.blend[p] : (float)(x + 1) * a.inv_w1;
    const int pitchL = (int)(a.L.pitch_bytes / sizeof(Tv)), pitchR = (int)(a.R.pitch_bytes / sizeof(Tv));
    Tv* out = reinterpret_cast<Tv*>(static_cast<char*>(a.F) + (long long)y * a.F_pitch_bytes) + (long long)fx * C;
    code1_area3<Tv, C>(static_cast<const Tv*>(a.L.data), pitchL, static_cast<const Tv*>(a.R.data), pitchR, w, h,
                       x, y, B, a.flowRL[p], a.flowLR[p], a.inv_w, a.k_sharp, a.k_mag, out);
}

template <typename Tv, int C>
__global__ void __launch_bounds__(256, 8) blend_kernel(BlendArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.L.w || y >= a.L.h) return;
    blend_pixel<Tv, C>(a, x, y, x);
}

// Every pair of a rig blended straight into the panorama canvas (Code 1's
// final placement of Area3): strip column x of pair p lands on canvas column
// (x0[p] + x) mod canvas_w. Where the spans of several pairs cover a canvas
// column, the pair with the highest index owns it; the others skip it, so
// every canvas pixel has one writer and the result is deterministic.
template <typename Tv, int C>
__global__ void __launch_bounds__(256, 8) rig_blend_kernel(const __grid_constant__ RigBlendArgs r) {
    const int p = blockIdx.z;
    const BlendArgs& a = r.pair[p];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.L.w || y >= a.L.h) return;
    const int W = r.canvas_w;
    int cx = r.x0[p] + x;
    if (cx >= W) cx -= W;
    for (int q = p + 1; q < r.n; ++q) {
        int d = cx - r.x0[q];
        if (d < 0) d += W;
        if (d < r.pair[q].L.w) return;
    }
    blend_pixel<Tv, C>(a, x, y, cx);
}

// Code 1 on a whole canvas, every branch: Area1 (label 1) copies L, Area2
// (label 2) copies R, Area3 (label 3) blends with the flows of the overlap
// crop (zero outside it), any other label writes 0.
template <typename Tv, int C>
__global__ void __launch_bounds__(256, 8) compose_kernel(ComposeArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int w = a.L.w, h = a.L.h;
    if (x >= w || y >= h) return;
    const int pitchL = (int)(a.L.pitch_bytes / sizeof(Tv)), pitchR = (int)(a.R.pitch_bytes / sizeof(Tv));
    const Tv* __restrict__ Lb = static_cast<const Tv*>(a.L.data);
    const Tv* __restrict__ Rb = static_cast<const Tv*>(a.R.data);
    Tv* out = reinterpret_cast<Tv*>(static_cast<char*>(a.F) + (long long)y * a.F_pitch_bytes) + (long long)x * C;
    const unsigned char area = a.label[(long long)y * a.label_pitch + x];
    if (area == 1 || area == 2) {
        const Tv* src = area == 1 ? Lb : Rb;
        const long long o = (long long)y * (area == 1 ? pitchL : pitchR) + (long long)x * C;
        const long long n = (long long)(h - 1) * (area == 1 ? pitchL : pitchR) + (long long)w * C;
        (void)n;
#pragma unroll
        for (int k = 0; k < C; ++k) out[k] = PANO_AT(src, o + k, n, 405);
    } else if (area == 3) {
        float2 rl = make_float2(0.f, 0.f), lr = make_float2(0.f, 0.f);
        const int qy = y - a.fy0, qx = x - a.fx0;
        if ((unsigned)qy < (unsigned)a.fh && (unsigned)qx < (unsigned)a.fw) {
            const long long q = (long long)qy * a.fw + qx, nq = (long long)a.fh * a.fw;
            (void)nq;
            rl = PANO_AT(a.flowRL, q, nq, 406);
            lr = PANO_AT(a.flowLR, q, nq, 407);
        }
        code1_area3<Tv, C>(Lb, pitchL, Rb, pitchR, w, h, x, y, a.blend[(long long)y * a.blend_pitch + x], rl, lr,
                           a.inv_fw, a.k_sharp, a.k_mag, out);
    } else {
#pragma unroll
        for (int k = 0; k < C; ++k) out[k] = (Tv)0;
    }
}

template <typename Tv>
__global__ void __launch_bounds__(256) warp_kernel(WarpArgs a) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int w = a.src.w, h = a.src.h, C = a.src.c;
    if (x >= w || y >= h) return;
    const float2 f = a.flow[(long long)y * w + x];
    const int pitch = (int)(a.src.pitch_bytes / sizeof(Tv));
    const Taps t = bilinear_taps(x, y, a.scale * f.x, a.scale * f.y, w, h, pitch, C);
    const Tv* __restrict__ base = static_cast<const Tv*>(a.src.data);
    float* out = reinterpret_cast<float*>(reinterpret_cast<char*>(a.dst) + (long long)y * a.dst_pitch_bytes) + x * C;
    const float scale = sizeof(Tv) == 1 ? 1.0f / 255.0f : 1.0f;  // samples widened by sample_f
    for (int k = 0; k < C; ++k) out[k] = sample_channel(base, t, k, (long long)(h - 1) * pitch + (long long)w * C) * scale;
}

}  // namespace

cudaError_t launch_blend(const BlendArgs& args, cudaStream_t s) {
    BlendArgs a = args;
    set_blend_scales(&a);
    dim3 block(32, 8);
    dim3 grid((a.L.w + 31) / 32, (a.L.h + 7) / 8);
    if (a.L.dtype == 0) {
        if (a.L.c == 3) blend_kernel<uint8_t, 3><<<grid, block, 0, s>>>(a);
        else blend_kernel<uint8_t, 1><<<grid, block, 0, s>>>(a);
    } else {
        if (a.L.c == 3) blend_kernel<float, 3><<<grid, block, 0, s>>>(a);
        else blend_kernel<float, 1><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_rig_blend(const RigBlendArgs& args, cudaStream_t s) {
    if (args.n < 1 || args.n > kMaxBatch) return cudaErrorInvalidValue;
    RigBlendArgs r = args;
    for (int p = 0; p < r.n; ++p) set_blend_scales(&r.pair[p]);
    int h = 0, w = 0;
    for (int p = 0; p < r.n; ++p) {
        h = max(h, r.pair[p].L.h);
        w = max(w, r.pair[p].L.w);
    }
    dim3 block(32, 8);
    dim3 grid((w + 31) / 32, (h + 7) / 8, r.n);
    const ImageDesc& d = r.pair[0].L;
    if (d.dtype == 0) {
        if (d.c == 3) rig_blend_kernel<uint8_t, 3><<<grid, block, 0, s>>>(r);
        else rig_blend_kernel<uint8_t, 1><<<grid, block, 0, s>>>(r);
    } else {
        if (d.c == 3) rig_blend_kernel<float, 3><<<grid, block, 0, s>>>(r);
        else rig_blend_kernel<float, 1><<<grid, block, 0, s>>>(r);
    }
    return cudaGetLastError();
}

PANO_BOUNDS_READER(bounds_read_blend)

cudaError_t launch_compose(const ComposeArgs& a, cudaStream_t s) {
    dim3 block(32, 8);
    dim3 grid((a.L.w + 31) / 32, (a.L.h + 7) / 8);
    if (a.L.dtype == 0) {
        if (a.L.c == 3) compose_kernel<uint8_t, 3><<<grid, block, 0, s>>>(a);
        else compose_kernel<uint8_t, 1><<<grid, block, 0, s>>>(a);
    } else {
        if (a.L.c == 3) compose_kernel<float, 3><<<grid, block, 0, s>>>(a);
        else compose_kernel<float, 1><<<grid, block, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_warp(const WarpArgs& a, cudaStream_t s) {
    dim3 block(32, 8);
    dim3 grid((a.src.w + 31) / 32, (a.src.h + 7) / 8);
    if (a.src.dtype == 0) warp_kernel<uint8_t><<<grid, block, 0, s>>>(a);
    else warp_kernel<float><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pano
