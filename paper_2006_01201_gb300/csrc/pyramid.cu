// pyramid.cu -- luma and Gaussian pyramid REDUCE kernels.
//
// The flow of Section III-C-1 is estimated with the "LK pyramid algorithm";
// the pyramid is the Burt-Adelson REDUCE: the binomial [1 4 6 4 1]/16
// along y, then along x, replicate border, keeping the even rows and
// columns (level size ceil(h/2) x ceil(w/2)). Level 0 is the BT.601 luma of
// the unit-scaled strip. Levels are stored as float32, bfloat16 or binary16
// (rounded to nearest even); every sum is formed in FP32.
#include "bounds.cuh"
#include "common.cuh"

namespace pano {

namespace {

constexpr float kInv255 = 1.0f / 255.0f;

// ---------------------------------------------------------------------------
// Level 0: each thread converts 4 consecutive pixels of one row, a block
// 256 x 4 pixels. All strips
// in one launch (blockIdx.z selects the strip; the grid-constant descriptor
// is indexed in parameter space, without a local copy).
// ---------------------------------------------------------------------------
// A byte value as float, exactly: the bits of 2^23 with the byte in the low
// mantissa bits, minus 2^23 (no integer-to-float conversion).
__device__ __forceinline__ float byte_f(uint32_t b) { return __uint_as_float(0x4B000000u | b) - 8388608.0f; }

// BT.601 luma with a fixed order of operations, shared by every kernel that
// forms level 0 (so that all of them give the same bits).
__device__ __forceinline__ float luma3(float r, float g, float b) { return fmaf(0.114f, b, fmaf(0.587f, g, 0.299f * r)); }

__device__ __forceinline__ float luma_at(const ImageDesc& in, const unsigned char* row, int x) {
    x = PANO_IDX(x, in.w, 315);
    if (in.dtype == 0) {
        if (in.c == 3) {
            const uint8_t* px = row + 3 * x;
            return luma3(byte_f(px[0]), byte_f(px[1]), byte_f(px[2])) * kInv255;
        }
        return byte_f(row[x]) * kInv255;
    }
    const float* r = reinterpret_cast<const float*>(row);
    if (in.c == 3) return luma3(r[3 * x], r[3 * x + 1], r[3 * x + 2]);
    return r[x];
}

// Luma of the four pixels x .. x+3 of a row (all inside the row): 12 aligned
// bytes for u8 RGB when the address allows it, else one pixel at a time.
__device__ __forceinline__ void luma4(const ImageDesc& in, const unsigned char* row, int x, float (&v)[4]) {
    x = PANO_IDX(x, in.w - 3, 316);  // pixels x .. x+3
    if (in.dtype == 0 && in.c == 3 && ((((uintptr_t)row) + 3 * x) & 3) == 0) {
        const uint32_t* p = reinterpret_cast<const uint32_t*>(row + 3 * x);
        const uint32_t w0 = __ldg(p), w1 = __ldg(p + 1), w2 = __ldg(p + 2);
        const uint32_t b[12] = {w0 & 255, (w0 >> 8) & 255, (w0 >> 16) & 255, w0 >> 24,
                                w1 & 255, (w1 >> 8) & 255, (w1 >> 16) & 255, w1 >> 24,
                                w2 & 255, (w2 >> 8) & 255, (w2 >> 16) & 255, w2 >> 24};
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = luma3(byte_f(b[3 * k]), byte_f(b[3 * k + 1]), byte_f(b[3 * k + 2])) * kInv255;
        return;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = luma_at(in, row, x + k);
}

// Four consecutive outputs: one 16-byte store for float32 rows, one 8-byte
// store for 16-bit rows, when the address allows it.
__device__ __forceinline__ void store4(float* o, const float (&v)[4]) {
    if ((((uintptr_t)o) & 15) == 0) {
        *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = v[k];
    }
}
template <class To>
__device__ __forceinline__ void store4(To* o, const float (&v)[4]) {
    To q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = from_f32<To>(v[k]);
    if ((((uintptr_t)o) & 7) == 0) {
        *reinterpret_cast<uint2*>(o) = *reinterpret_cast<const uint2*>(q);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = q[k];
    }
}

template <class To>
__global__ void __launch_bounds__(256) luma_kernel(const __grid_constant__ LumaArgs a) {
    const ImageDesc& in = a.in[blockIdx.z];
    To* out = static_cast<To*>(a.out[blockIdx.z]);
    const int out_pitch = a.out_pitch[blockIdx.z];
    const int x = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= in.w || y >= in.h) return;
    const unsigned char* row = static_cast<const unsigned char*>(in.data) + (long long)y * in.pitch_bytes;
    To* orow = out + (long long)y * out_pitch;
    if (x + 4 <= in.w) {
        float v[4];
        luma4(in, row, x, v);
        store4(orow + x, v);
        return;
    }
    const int n = min(4, in.w - x);
    for (int k = 0; k < n; ++k) orow[x + k] = from_f32<To>(luma_at(in, row, x + k));
}

// ---------------------------------------------------------------------------
// REDUCE: a 64 x 16 tile of the destination per 256-thread block. The source
// footprint (2*16+3 rows x 2*64+3 columns, clamped) is staged in shared
// memory -- with 16-byte (float) or 8-byte (16-bit) loads of four aligned
// elements where the four lie inside the row and the plane is aligned, else
// one element at a time -- then blurred along y at the even rows and along x
// at the even columns.
// ---------------------------------------------------------------------------
constexpr int kPdTW = 64, kPdTH = 16;

// One 5-tap binomial sum [1 4 6 4 1]/16 with a fixed order of operations.
__device__ __forceinline__ float reduce5(float a, float b, float c, float d, float e) {
    const float k0 = 1.0f / 16, k1 = 4.0f / 16, k2 = 6.0f / 16;
    return fmaf(k0, e, fmaf(k1, d, fmaf(k2, c, fmaf(k1, b, k0 * a))));
}
constexpr int kPdSH = 2 * kPdTH + 3;  // source rows 2*y0-2 .. 2*(y0+15)+2
constexpr int kPdQ = (2 * kPdTW + 8) / 4;  // groups of four source columns from 2*x0-4
constexpr int kPdSW = 4 * kPdQ;            // staged columns 2*x0-4 .. 2*x0+131

template <class Ts>
struct Vec4Of;
template <>
struct Vec4Of<float> { using type = float4; };
template <>
struct Vec4Of<__nv_bfloat16> { using type = uint2; };
template <>
struct Vec4Of<__half> { using type = uint2; };

__device__ __forceinline__ void widen4(const float4& v, float* o) {
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
}
template <class Ts>
__device__ __forceinline__ void widen4(const uint2& v, float* o) {
    const Ts* e = reinterpret_cast<const Ts*>(&v);
#pragma unroll
    for (int k = 0; k < 4; ++k) o[k] = to_f32(e[k]);
}

// Blur the staged footprint along y at the even rows and along x at the even
// columns, and store the 64 x 16 destination tile (one barrier inside).
template <class Ts>
__device__ __forceinline__ void reduce_staged(const float (*s_src)[kPdSW], float (*s_v)[kPdSW + 1], int xd0, int yd0,
                                              int wd, int hd, Ts* __restrict__ dst, int dst_pitch) {
    const int tid = threadIdx.x;
    for (int i = tid; i < kPdTH * kPdSW; i += 256) {
        int r = i / kPdSW, c = i - r * kPdSW;
        int sr = 2 * r + 2;
        const float* S = &s_src[0][0];
        constexpr int NS = kPdSH * kPdSW;
        PANO_AT(&s_v[0][0], r * (kPdSW + 1) + c, kPdTH * (kPdSW + 1), 311) =
            reduce5(PANO_AT(S, (sr - 2) * kPdSW + c, NS, 312), PANO_AT(S, (sr - 1) * kPdSW + c, NS, 312),
                    PANO_AT(S, sr * kPdSW + c, NS, 312), PANO_AT(S, (sr + 1) * kPdSW + c, NS, 312),
                    PANO_AT(S, (sr + 2) * kPdSW + c, NS, 312));
    }
    __syncthreads();
    const int x = tid & (kPdTW - 1);
    const int xd = xd0 + x;
    if (xd < wd) {
        const int c = 2 * x + 4;  // staged column of source column 2 * xd
#pragma unroll
        for (int r = tid / kPdTW; r < kPdTH; r += 256 / kPdTW) {
            const int yd = yd0 + r;
            if (yd >= hd) break;
            const float* V = &s_v[0][0];
            const int o = r * (kPdSW + 1) + c, NV = kPdTH * (kPdSW + 1);
            PANO_AT(dst, (long long)yd * dst_pitch + xd, (long long)hd * dst_pitch, 313) = from_f32<Ts>(
                reduce5(PANO_AT(V, o - 2, NV, 314), PANO_AT(V, o - 1, NV, 314), PANO_AT(V, o, NV, 314),
                        PANO_AT(V, o + 1, NV, 314), PANO_AT(V, o + 2, NV, 314)));
        }
    }
}

template <class Ts>
__global__ void __launch_bounds__(256) pyr_down_kernel(const __grid_constant__ PyrDownArgs a) {
    __shared__ __align__(16) float s_src[kPdSH][kPdSW];
    __shared__ float s_v[kPdTH][kPdSW + 1];
    const int z = blockIdx.z;
    const Ts* __restrict__ src = static_cast<const Ts*>(a.src[z]);
    Ts* __restrict__ dst = static_cast<Ts*>(a.dst[z]);
    const int src_pitch = a.src_pitch[z], dst_pitch = a.dst_pitch[z];
    const int h = a.h[z], w = a.w[z];
    const int hd = (h + 1) >> 1, wd = (w + 1) >> 1;
    const int xd0 = blockIdx.x * kPdTW, yd0 = blockIdx.y * kPdTH;
    if (xd0 >= wd || yd0 >= hd) return;  // a smaller plane of the batch
    const int cx0 = 2 * xd0 - 4, sy0 = 2 * yd0 - 2;
    const int tid = threadIdx.x;
    // four-element loads need a plane whose rows start on 4-element boundaries
    const bool vec = ((((uintptr_t)src) & (4 * sizeof(Ts) - 1)) == 0) && (src_pitch & 3) == 0;
    for (int i = tid; i < kPdSH * kPdQ; i += 256) {
        const int r = i / kPdQ, q = i - r * kPdQ;
        const int sy = PANO_IDX(min(max(sy0 + r, 0), h - 1), h, 317);
        const int sx = cx0 + 4 * q;
        const long long ro = (long long)sy * src_pitch;
        const long long ns = (long long)(h - 1) * src_pitch + w;  // elements of the plane
        (void)ns;
        float* o = &PANO_VEC(float, &s_src[0][0], r * kPdSW + 4 * q, 4, kPdSH * kPdSW, 318);
        if (vec && sx >= 0 && sx + 3 < w) {
            using V = typename Vec4Of<Ts>::type;
            const V v = __ldg(&PANO_VEC(const V, src, ro + sx, 4, ns, 319));
            if constexpr (sizeof(Ts) == 4) widen4(v, o);
            else widen4<Ts>(v, o);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = ld_f32(&PANO_AT(src, ro + min(max(sx + k, 0), w - 1), ns, 320));
        }
    }
    __syncthreads();
    __syncthreads();
    reduce_staged<Ts>(s_src, s_v, xd0, yd0, wd, hd, dst, dst_pitch);
}

// Level 0 and level 1 in one pass: a block computes the luma of the footprint
// of its 64 x 16 level-1 tile (35 rows x 136 columns, clamped), rounded to
// the storage type as level 0 is stored, writes the level-0 pixels it owns
// (rows 2*y0 .. 2*y0+31, columns 2*x0 .. 2*x0+127; the blocks tile level 0
// exactly) and reduces the footprint to the level-1 tile. Same values as
// luma_kernel followed by pyr_down_kernel.
template <class Ts>
__global__ void __launch_bounds__(256) luma_reduce_kernel(const __grid_constant__ LumaReduceArgs a) {
    __shared__ __align__(16) float s_src[kPdSH][kPdSW];
    __shared__ float s_v[kPdTH][kPdSW + 1];
    const int z = blockIdx.z;
    const ImageDesc& in = a.in[z];
    const int h = in.h, w = in.w;
    const int hd = (h + 1) >> 1, wd = (w + 1) >> 1;
    const int xd0 = blockIdx.x * kPdTW, yd0 = blockIdx.y * kPdTH;
    if (xd0 >= wd || yd0 >= hd) return;  // a smaller plane of the batch
    const int cx0 = 2 * xd0 - 4, sy0 = 2 * yd0 - 2;
    Ts* __restrict__ l0 = static_cast<Ts*>(a.l0[z]);
    const int p0 = a.l0_pitch[z];
    const int tid = threadIdx.x;
    for (int i = tid; i < kPdSH * kPdQ; i += 256) {
        const int r = i / kPdQ, q = i - r * kPdQ;
        const int yy = sy0 + r;
        const int sy = PANO_IDX(min(max(yy, 0), h - 1), h, 321);
        const int sx = cx0 + 4 * q;
        const unsigned char* row = static_cast<const unsigned char*>(in.data) + (long long)sy * in.pitch_bytes;
        float v[4];
        if (sx >= 0 && sx + 3 < w) {
            luma4(in, row, sx, v);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = luma_at(in, row, min(max(sx + k, 0), w - 1));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = to_f32(from_f32<Ts>(v[k]));  // the stored level-0 value
        float* o = &PANO_VEC(float, &s_src[0][0], r * kPdSW + 4 * q, 4, kPdSH * kPdSW, 322);
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = v[k];
        // level-0 pixels owned by this block
        if (r >= 2 && r < 2 + 2 * kPdTH && yy < h && q >= 1 && q <= kPdTW / 2 && sx < w) {
            const long long ro = (long long)yy * p0;
            const long long n0 = (long long)(h - 1) * p0 + w;  // elements of level 0
            (void)n0;
            if (sx + 3 < w) {
                store4(&PANO_VEC(Ts, l0, ro + sx, 1, n0 - 3, 323), v);   // elements sx .. sx+3
            } else {
                for (int k = 0; k < 4 && sx + k < w; ++k) PANO_AT(l0, ro + sx + k, n0, 324) = from_f32<Ts>(v[k]);
            }
        }
    }
    __syncthreads();
    reduce_staged<Ts>(s_src, s_v, xd0, yd0, wd, hd, static_cast<Ts*>(a.l1[z]), a.l1_pitch[z]);
}

// ---------------------------------------------------------------------------
// Levels s+1 .. s+M in one launch. A block owns a kTailTC x kTailTC tile of
// the coarsest level and, at distance d from it, the 2^d-times larger tile;
// the blocks tile every level exactly once. It stages the footprint of
// level s that its tile needs (clamped), then forms each coarser level on
// the region the next one needs: in-range pixels by the same two 5-tap
// passes as pyr_down_kernel (each value rounded to the storage type, as it
// is stored), pixels outside the level by copying the clamped in-range
// pixel (the replicate border), and writes the pixels it owns. Same values
// as M launches of pyr_down_kernel.
// ---------------------------------------------------------------------------
constexpr int kTailTC = 8;
// side of the region needed at distance d: n(0) = TC, n(d) = 2 n(d-1) + 3
__host__ __device__ constexpr int tail_n(int d) { return (kTailTC + 3) * (1 << d) - 3; }
// offset of the buffer of distance d (the buffers of distances 0 .. d-1 before it)
__host__ __device__ constexpr int tail_off(int d) {
    int o = 0;
    for (int e = 0; e < d; ++e) o += tail_n(e) * tail_n(e);
    return o;
}
// the vertical-pass buffer: the largest n(d) x n(d+1), d < m
__host__ __device__ constexpr int tail_tmp(int m) {
    int t = 0;
    for (int d = 0; d < m; ++d) t = tail_n(d) * tail_n(d + 1) > t ? tail_n(d) * tail_n(d + 1) : t;
    return t;
}
template <int M>
struct TailSmem {
    static constexpr int floats = tail_off(M + 1) + tail_tmp(M);
    static constexpr size_t bytes = sizeof(float) * floats;
};

template <class Ts, int M>
__global__ void __launch_bounds__(256) pyr_tail_kernel(const __grid_constant__ PyrTailArgs a) {
    extern __shared__ float tsm[];
    const int z = blockIdx.z;
    // level sizes at distance d from the coarsest (ceil of repeated halving
    // is the ceil of one division), and the first row / column of the
    // region a block needs there: 2^d Yc - 2 (2^d - 1)
    const int hs = a.h[z], ws = a.w[z];
    auto H = [&](int d) { return (hs + (1 << (M - d)) - 1) >> (M - d); };
    auto W = [&](int d) { return (ws + (1 << (M - d)) - 1) >> (M - d); };
    const int Yc = blockIdx.y * kTailTC, Xc = blockIdx.x * kTailTC;
    if (Yc >= H(0) || Xc >= W(0)) return;  // a smaller plane of the batch
    auto Oy = [&](int d) { return (Yc << d) - 2 * ((1 << d) - 1); };
    auto Ox = [&](int d) { return (Xc << d) - 2 * ((1 << d) - 1); };
    const int tid = threadIdx.x;
    float* tmp = tsm + tail_off(M + 1);
    {
        // footprint of level s, clamped
        const Ts* __restrict__ src = static_cast<const Ts*>(a.src[z]);
        const int pitch = a.src_pitch[z];
        constexpr int n = tail_n(M);
        float* b = tsm + tail_off(M);
        for (int i = tid; i < n * n; i += 256) {
            const int r = i / n, c = i - r * n;
            const int y = min(max(Oy(M) + r, 0), H(M) - 1), x = min(max(Ox(M) + c, 0), W(M) - 1);
            PANO_AT(b, i, n * n, 301) = ld_f32(&PANO_AT(src, (long long)y * pitch + x, (long long)H(M) * pitch, 302));
        }
    }
    __syncthreads();
#pragma unroll
    for (int d = M - 1; d >= 0; --d) {
        const int nf = tail_n(d + 1), nc = tail_n(d);
        const float* f = tsm + tail_off(d + 1);
        float* c = tsm + tail_off(d);
        // along y at the even rows of the finer level
        for (int i = tid; i < nc * nf; i += 256) {
            const int r = i / nf, q = i - r * nf;
            const int o = 2 * r * nf + q, nn = nf * nf;
            PANO_AT(tmp, i, tail_tmp(M), 303) =
                reduce5(PANO_AT(f, o, nn, 304), PANO_AT(f, o + nf, nn, 304), PANO_AT(f, o + 2 * nf, nn, 304),
                        PANO_AT(f, o + 3 * nf, nn, 304), PANO_AT(f, o + 4 * nf, nn, 304));
        }
        __syncthreads();
        // along x at the even columns, for the pixels inside the level
        for (int i = tid; i < nc * nc; i += 256) {
            const int r = i / nc, q = i - r * nc;
            const int y = Oy(d) + r, x = Ox(d) + q;
            if (y < 0 || y >= H(d) || x < 0 || x >= W(d)) continue;
            const int o = r * nf + 2 * q, nt = tail_tmp(M);
            PANO_AT(c, i, nc * nc, 305) = to_f32(from_f32<Ts>(
                reduce5(PANO_AT(tmp, o, nt, 306), PANO_AT(tmp, o + 1, nt, 306), PANO_AT(tmp, o + 2, nt, 306),
                        PANO_AT(tmp, o + 3, nt, 306), PANO_AT(tmp, o + 4, nt, 306))));
        }
        __syncthreads();
        // the replicate border: pixels outside the level take the clamped pixel
        for (int i = tid; i < nc * nc; i += 256) {
            const int r = i / nc, q = i - r * nc;
            const int y = Oy(d) + r, x = Ox(d) + q;
            if (y >= 0 && y < H(d) && x >= 0 && x < W(d)) continue;
            const int cy = min(max(y, 0), H(d) - 1), cx = min(max(x, 0), W(d) - 1);
            PANO_AT(c, i, nc * nc, 307) = PANO_AT(c, (cy - Oy(d)) * nc + (cx - Ox(d)), nc * nc, 308);
        }
        // the owned pixels of this level
        Ts* __restrict__ dst = static_cast<Ts*>(a.dst[z][M - 1 - d]);
        const int dp = a.dst_pitch[z][M - 1 - d];
        const int t = kTailTC << d;
        const int y0 = Yc << d, x0 = Xc << d;
        for (int i = tid; i < t * t; i += 256) {
            const int r = i / t, q = i - r * t;
            const int y = y0 + r, x = x0 + q;
            if (y >= H(d) || x >= W(d)) continue;
            PANO_AT(dst, (long long)y * dp + x, (long long)H(d) * dp, 309) =
                from_f32<Ts>(PANO_AT(c, (y - Oy(d)) * nc + (x - Ox(d)), nc * nc, 310));
        }
        __syncthreads();
    }
}

template <class Ts, int M>
cudaError_t launch_tail_m(const PyrTailArgs& a, cudaStream_t s) {
    int hc = 0, wc = 0;
    for (int i = 0; i < a.count; ++i) {
        int h = a.h[i], w = a.w[i];
        for (int d = 0; d < M; ++d) {
            h = (h + 1) / 2;
            w = (w + 1) / 2;
        }
        hc = max(hc, h);
        wc = max(wc, w);
    }
    dim3 grid((wc + kTailTC - 1) / kTailTC, (hc + kTailTC - 1) / kTailTC, a.count);
    pyr_tail_kernel<Ts, M><<<grid, 256, TailSmem<M>::bytes, s>>>(a);
    return cudaGetLastError();
}

template <class Ts>
cudaError_t launch_tail_t(const PyrTailArgs& a, cudaStream_t s) {
    switch (a.levels) {
        case 1: return launch_tail_m<Ts, 1>(a, s);
        case 2: return launch_tail_m<Ts, 2>(a, s);
        case 3: return launch_tail_m<Ts, 3>(a, s);
        case 4: return launch_tail_m<Ts, 4>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class Ts>
cudaError_t prepare_tail_t(int max_smem) {
    const void* fns[] = {(const void*)pyr_tail_kernel<Ts, 1>, (const void*)pyr_tail_kernel<Ts, 2>,
                         (const void*)pyr_tail_kernel<Ts, 3>, (const void*)pyr_tail_kernel<Ts, 4>};
    const size_t need[] = {TailSmem<1>::bytes, TailSmem<2>::bytes, TailSmem<3>::bytes, TailSmem<4>::bytes};
    for (int i = 0; i < 4; ++i) {
        if (need[i] > (size_t)max_smem) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need[i]);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_pyr_tail(const PyrTailArgs& a, cudaStream_t s) {
    if (a.count < 1 || a.count > kMaxPlanes || a.levels < 1 || a.levels > kTailMaxLevels) return cudaErrorInvalidValue;
    switch (a.pyr) {
        case kPyrF32: return launch_tail_t<float>(a, s);
        case kPyrBF16: return launch_tail_t<__nv_bfloat16>(a, s);
        case kPyrF16: return launch_tail_t<__half>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t pyr_tail_prepare(int max_smem_bytes) {
    cudaError_t e;
    if ((e = prepare_tail_t<float>(max_smem_bytes)) != cudaSuccess) return e;
    if ((e = prepare_tail_t<__nv_bfloat16>(max_smem_bytes)) != cudaSuccess) return e;
    return prepare_tail_t<__half>(max_smem_bytes);
}

cudaError_t launch_luma_reduce(const LumaReduceArgs& a, cudaStream_t s) {
    if (a.count < 1 || a.count > kMaxPlanes) return cudaErrorInvalidValue;
    int hd = 0, wd = 0;
    for (int i = 0; i < a.count; ++i) {
        hd = max(hd, (a.in[i].h + 1) / 2);
        wd = max(wd, (a.in[i].w + 1) / 2);
    }
    dim3 block(256);
    dim3 grid((wd + kPdTW - 1) / kPdTW, (hd + kPdTH - 1) / kPdTH, a.count);
    switch (a.pyr) {
        case kPyrF32: luma_reduce_kernel<float><<<grid, block, 0, s>>>(a); break;
        case kPyrBF16: luma_reduce_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(a); break;
        case kPyrF16: luma_reduce_kernel<__half><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

PANO_BOUNDS_READER(bounds_read_pyramid)

cudaError_t launch_luma(const LumaArgs& a, cudaStream_t s) {
    if (a.count < 1 || a.count > kMaxPlanes) return cudaErrorInvalidValue;
    int h = 0, w = 0;
    for (int i = 0; i < a.count; ++i) {
        h = max(h, a.in[i].h);
        w = max(w, a.in[i].w);
    }
    // 64 x 4 threads, four pixels each: 256 x 4 pixels per block
    dim3 block(64, 4);
    dim3 grid((w + 4 * 64 - 1) / (4 * 64), (h + 3) / 4, a.count);
    switch (a.pyr) {
        case kPyrF32: luma_kernel<float><<<grid, block, 0, s>>>(a); break;
        case kPyrBF16: luma_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(a); break;
        case kPyrF16: luma_kernel<__half><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_pyr_down(const PyrDownArgs& a, cudaStream_t s) {
    if (a.count < 1 || a.count > kMaxPlanes) return cudaErrorInvalidValue;
    int hd = 0, wd = 0;
    for (int i = 0; i < a.count; ++i) {
        hd = max(hd, (a.h[i] + 1) / 2);
        wd = max(wd, (a.w[i] + 1) / 2);
    }
    dim3 block(256);
    dim3 grid((wd + kPdTW - 1) / kPdTW, (hd + kPdTH - 1) / kPdTH, a.count);
    switch (a.pyr) {
        case kPyrF32: pyr_down_kernel<float><<<grid, block, 0, s>>>(a); break;
        case kPyrBF16: pyr_down_kernel<__nv_bfloat16><<<grid, block, 0, s>>>(a); break;
        case kPyrF16: pyr_down_kernel<__half><<<grid, block, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace pano
