// lk.cu -- one pyramid level of dense Lucas-Kanade flow (Section III-C-1,
// "LK pyramid algorithm"; the local least-squares flow of [20]).
//
// Every pixel p solves for a flow v that is constant over the (2r+1)^2 box
// W(p); each box sample q is linearised at its own current flow u(q):
//   (G(p) + lambda I) v = sum_{q in W(p)} grad T(q) (grad T(q) . u(q) - It(q)) + lambda u(p)
//   It(q) = J(q + u(q)) - T(q),   G(p) = sum_{q in W(p)} grad T(q) grad T(q)^T
// with the box clipped to the image, central-difference gradients of T and
// bilinear clamp-to-edge sampling of J; then u(p) <- v. K such steps run per
// level, starting from twice the bilinearly upsampled flow of the coarser
// level (or zero at the coarsest level).
//
// GPU design: one CTA owns an output tile and iterates all K steps of the
// level on chip. Because step k at p reads the flows of step k-1 on W(p),
// the tile carries a halo of K*r pixels that shrinks by r per step; the
// template, its gradient, the flow and the inverse normal matrices stay in
// shared memory for the whole level, and so does a box of J around the
// region (shifted by the tile's reference flow); a sample outside the box is
// gathered from L1/L2. Each
// step is: per-sample residual products -> column box sums -> row box sums
// and the 2x2 solve. Both flow directions run in the same launch
// (blockIdx.z). To keep FP32 rounding independent of the size of the flow,
// the kernel works with flows relative to one reference flow per tile (the
// starting flow at the tile centre); the equations above are unchanged by
// that shift.
#include "bounds.cuh"
#include "common.cuh"

namespace pano {

namespace {

constexpr int kLkThreads = 512;
constexpr int kTileJM = 4;  // margin of the staged target box around the region, pixels

// The target box of a tile: the region shifted by the integer part of the
// reference flow, widened by kTileJM on every side (one more column and row
// for the second bilinear tap).
__host__ __device__ __forceinline__ int tile_jbw(int rw) { return rw + 2 * kTileJM + 1; }
__host__ __device__ __forceinline__ int tile_jbh(int rh) { return rh + 2 * kTileJM + 1; }

// J at (qx + ox, qy + oy) as sample_plane computes it (same taps, same
// weights, same arithmetic), from the staged box when all four taps lie in
// it and from global memory otherwise.
template <class Ts>
__device__ __forceinline__ float sample_box(const float* __restrict__ sJ, int jbw, int jbh, int jx0, int jy0,
                                            const Ts* __restrict__ J, int pitchJ, int w, int h, int qx, int qy,
                                            float ox, float oy) {
    const float cx = fminf(fmaxf(ox, -(float)(w + 2)), (float)(w + 2));
    const float cy = fminf(fmaxf(oy, -(float)(h + 2)), (float)(h + 2));
    const float fx = floorf(cx), fy = floorf(cy);
    const int bx = qx + (int)fx - jx0, by = qy + (int)fy - jy0;
    if ((unsigned)bx < (unsigned)(jbw - 1) && (unsigned)by < (unsigned)(jbh - 1)) {
        Taps t;
        t.ax = cx - fx;
        t.ay = cy - fy;
        const int o = by * jbw + bx, nj = jbw * jbh;
        return bilinear_mix(t, PANO_AT(sJ, o, nj, 201), PANO_AT(sJ, o + 1, nj, 202), PANO_AT(sJ, o + jbw, nj, 203),
                            PANO_AT(sJ, o + jbw + 1, nj, 204));
    }
    return sample_plane(J, pitchJ, w, h, qx, qy, ox, oy);
}

__device__ __forceinline__ float2 start_flow(const LkArgs& a, const LkDir& D, int x, int y) {
    if (a.mode == 0 || D.uin == nullptr) return make_float2(0.f, 0.f);
    const float2* __restrict__ u = reinterpret_cast<const float2*>(D.uin);
    if (a.mode == 2) return u[(long long)y * D.uin_pitch + x];
    // coarse-to-fine: 2 * bilinear(u_coarse)(x/2, y/2); fine pixel 2i sits on
    // coarse pixel i, so the weights are 0 or 1/2
    int x0 = x >> 1, y0 = y >> 1;
    float fx = (x & 1) ? 0.5f : 0.f, fy = (y & 1) ? 0.5f : 0.f;
    int xa = min(x0, a.in_w - 1), xb = min(x0 + 1, a.in_w - 1);
    int ya = min(y0, a.in_h - 1), yb = min(y0 + 1, a.in_h - 1);
    float2 u00 = u[(long long)ya * D.uin_pitch + xa], u10 = u[(long long)ya * D.uin_pitch + xb];
    float2 u01 = u[(long long)yb * D.uin_pitch + xa], u11 = u[(long long)yb * D.uin_pitch + xb];
    float tx = fmaf(fx, u10.x - u00.x, u00.x), bx = fmaf(fx, u11.x - u01.x, u01.x);
    float ty = fmaf(fx, u10.y - u00.y, u00.y), by = fmaf(fx, u11.y - u01.y, u01.y);
    return make_float2(2.f * fmaf(fy, bx - tx, tx), 2.f * fmaf(fy, by - ty, ty));
}

// One output tile (bx, by) of direction `dir` of one level; T and J stored
// as Ts.
template <int RAD, class Ts>
__device__ __forceinline__ void lk_tile_item(const LkArgs& a, int dir, int bx, int by, float4* smem4) {
    const LkDir& D = a.dir[dir];
    const int K = a.iters;
    const int halo = K * RAD;
    const int RW = a.tile_w + 2 * halo, RH = a.tile_h + 2 * halo;
    const int N = RW * RH;
    float4* sGi = smem4;                                  // inverse normal matrix (i11, i12, i22)
    float2* sG = reinterpret_cast<float2*>(sGi + N);      // grad T
    float2* sU = sG + N;                                  // flow relative to the reference
    float2* sP = sU + N;                                  // per-sample products
    float2* sV = sP + N;                                  // column box sums
    float* sT = reinterpret_cast<float*>(sV + N);         // template
    float* sJ = sT + N;                                   // staged target box
    const int ox = bx * a.tile_w - halo, oy = by * a.tile_h - halo;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int w = a.w, h = a.h, pitchT = D.pitchT, pitchJ = D.pitchJ;
    const Ts* __restrict__ T = static_cast<const Ts*>(D.T);
    const Ts* __restrict__ J = static_cast<const Ts*>(D.J);

    // Phase 0: template, its gradient and the starting flow on the region.
    for (int ry = warp; ry < RH; ry += nwarps) {
        const int y = oy + ry;
        for (int rx = lane; rx < RW; rx += 32) {
            const int x = ox + rx;
            float t = 0.f;
            float2 g = make_float2(0.f, 0.f), u = make_float2(0.f, 0.f);
            if (x >= 0 && x < w && y >= 0 && y < h) {
                const Ts* row = T + (long long)y * pitchT;
                t = ld_f32(row + x);
                g.x = 0.5f * (ld_f32(row + min(x + 1, w - 1)) - ld_f32(row + max(x - 1, 0)));
                g.y = 0.5f * (ld_f32(T + (long long)min(y + 1, h - 1) * pitchT + x) -
                              ld_f32(T + (long long)max(y - 1, 0) * pitchT + x));
                u = start_flow(a, D, x, y);
            }
            const int i = ry * RW + rx;
            PANO_AT(sT, i, N, 205) = t;
            PANO_AT(sG, i, N, 206) = g;
            PANO_AT(sU, i, N, 207) = u;
        }
    }
    __syncthreads();

    // Reference flow: the starting flow at the tile centre (inside the image).
    const int cx = min(bx * a.tile_w + a.tile_w / 2, w - 1);
    const int cy = min(by * a.tile_h + a.tile_h / 2, h - 1);
    const float2 ref = PANO_AT(sU, (cy - oy) * RW + (cx - ox), N, 208);

    // the staged target box (clamped values), shifted by the reference flow
    const int jbw = tile_jbw(RW), jbh = tile_jbh(RH);
    const int jx0 = ox + (int)floorf(fminf(fmaxf(ref.x, -(float)(w + 2)), (float)(w + 2))) - kTileJM;
    const int jy0 = oy + (int)floorf(fminf(fmaxf(ref.y, -(float)(h + 2)), (float)(h + 2))) - kTileJM;

    if (K > 0) {
        __syncthreads();  // everyone has read ref before it is overwritten
        for (int i = threadIdx.x; i < jbw * jbh; i += blockDim.x) {
            const int r = i / jbw, c = i - r * jbw;
            const int yy = min(max(jy0 + r, 0), h - 1), xx = min(max(jx0 + c, 0), w - 1);
            PANO_AT(sJ, i, jbw * jbh, 209) = ld_f32(&PANO_AT(J, (long long)yy * pitchJ + xx, (long long)h * pitchJ, 210));
        }
        // Relative flows and the inverse normal matrices on R_1 (margin RAD).
        for (int ry = warp; ry < RH; ry += nwarps) {
            for (int rx = lane; rx < RW; rx += 32) {
                const int i = ry * RW + rx;
                float2 u = PANO_AT(sU, i, N, 211);
                PANO_AT(sU, i, N, 211) = make_float2(u.x - ref.x, u.y - ref.y);
                if (ry < RAD || ry >= RH - RAD || rx < RAD || rx >= RW - RAD) continue;
                float g11 = 0.f, g12 = 0.f, g22 = 0.f;
#pragma unroll
                for (int dy = -RAD; dy <= RAD; ++dy)
#pragma unroll
                    for (int dx = -RAD; dx <= RAD; ++dx) {
                        float2 g = PANO_AT(sG, i + dy * RW + dx, N, 212);
                        g11 = fmaf(g.x, g.x, g11);
                        g12 = fmaf(g.x, g.y, g12);
                        g22 = fmaf(g.y, g.y, g22);
                    }
                const float a11 = g11 + a.lambda, a22 = g22 + a.lambda;
                const float inv = 1.0f / (a11 * a22 - g12 * g12);
                PANO_AT(sGi, i, N, 213) = make_float4(a22 * inv, -g12 * inv, a11 * inv, 0.f);
            }
        }
        __syncthreads();

        for (int k = 1; k <= K; ++k) {
            const int mA = (k - 1) * RAD, mC = k * RAD;
            // A: products grad T(q) * s(q), s = grad T . u(q) - It(q), on R_{k-1}
            for (int ry = mA + warp; ry < RH - mA; ry += nwarps) {
                const int y = oy + ry;
                for (int rx = mA + lane; rx < RW - mA; rx += 32) {
                    const int x = ox + rx;
                    const int i = ry * RW + rx;
                    float2 P = make_float2(0.f, 0.f);
                    if (x >= 0 && x < w && y >= 0 && y < h) {
                        const float2 u = PANO_AT(sU, i, N, 214);
                        const float2 g = PANO_AT(sG, i, N, 215);
                        const float Jw = sample_box(sJ, jbw, jbh, jx0, jy0, J, pitchJ, w, h, x, y, ref.x + u.x,
                                                    ref.y + u.y);
                        const float It = Jw - PANO_AT(sT, i, N, 216);
                        const float s = fmaf(g.x, u.x, fmaf(g.y, u.y, -It));
                        P = make_float2(g.x * s, g.y * s);
                    }
                    PANO_AT(sP, i, N, 217) = P;
                }
            }
            __syncthreads();
            // B: sums over the column window, rows of R_k, columns of R_{k-1}
            for (int ry = mC + warp; ry < RH - mC; ry += nwarps) {
                for (int rx = mA + lane; rx < RW - mA; rx += 32) {
                    const int i = ry * RW + rx;
                    float2 v = PANO_AT(sP, i - RAD * RW, N, 218);
#pragma unroll
                    for (int dy = -RAD + 1; dy <= RAD; ++dy) {
                        float2 q = PANO_AT(sP, i + dy * RW, N, 219);
                        v.x += q.x;
                        v.y += q.y;
                    }
                    PANO_AT(sV, i, N, 220) = v;
                }
            }
            __syncthreads();
            // C: sums over the row window and the 2x2 solve on R_k
            for (int ry = mC + warp; ry < RH - mC; ry += nwarps) {
                const int y = oy + ry;
                for (int rx = mC + lane; rx < RW - mC; rx += 32) {
                    const int x = ox + rx;
                    if (x < 0 || x >= w || y < 0 || y >= h) continue;
                    const int i = ry * RW + rx;
                    float2 m = PANO_AT(sV, i - RAD, N, 221);
#pragma unroll
                    for (int dx = -RAD + 1; dx <= RAD; ++dx) {
                        float2 q = PANO_AT(sV, i + dx, N, 222);
                        m.x += q.x;
                        m.y += q.y;
                    }
                    const float2 u = PANO_AT(sU, i, N, 223);
                    const float4 gi = PANO_AT(sGi, i, N, 224);
                    const float r1 = fmaf(a.lambda, u.x, m.x), r2 = fmaf(a.lambda, u.y, m.y);
                    PANO_AT(sU, i, N, 225) = make_float2(fmaf(gi.x, r1, gi.y * r2), fmaf(gi.y, r1, gi.z * r2));
                }
            }
            __syncthreads();
        }
    }

    // Write the tile (relative flows back to absolute).
    const float2 add = (K > 0) ? ref : make_float2(0.f, 0.f);
    float2* __restrict__ uo = reinterpret_cast<float2*>(D.uout);
    for (int ty = warp; ty < a.tile_h; ty += nwarps) {
        const int y = by * a.tile_h + ty;
        if (y >= h) break;
        for (int tx = lane; tx < a.tile_w; tx += 32) {
            const int x = bx * a.tile_w + tx;
            if (x >= w) break;
            const float2 u = PANO_AT(sU, (ty + halo) * RW + (tx + halo), N, 226);
            PANO_AT(uo, (long long)y * D.uout_pitch + x, (long long)h * D.uout_pitch, 227) =
                make_float2(u.x + add.x, u.y + add.y);
        }
    }
}

template <int RAD, class Ts>
__global__ void __launch_bounds__(kLkThreads) lk_level_kernel(const __grid_constant__ LkArgs a) {
    extern __shared__ float4 smem4[];
    lk_tile_item<RAD, Ts>(a, blockIdx.z, blockIdx.x, blockIdx.y, smem4);
}

// The same level of several strip pairs: blockIdx.z = 2 * pair + direction,
// the x/y grid covers the largest pair and tiles beyond a smaller pair exit.
template <int RAD, class Ts>
__global__ void __launch_bounds__(kLkThreads) lk_level_batch_kernel(const __grid_constant__ LkBatch b) {
    extern __shared__ float4 smem4[];
    const LkArgs& a = b.pair[blockIdx.z >> 1];
    if ((int)blockIdx.x * a.tile_w >= a.w || (int)blockIdx.y * a.tile_h >= a.h) return;
    lk_tile_item<RAD, Ts>(a, blockIdx.z & 1, blockIdx.x, blockIdx.y, smem4);
}

template <int RAD, class Ts>
cudaError_t launch_rad(const LkArgs& a, int ndirs, cudaStream_t s) {
    size_t smem = lk_smem_bytes(a.tile_w, a.tile_h, a.iters, a.radius);
    dim3 grid((a.w + a.tile_w - 1) / a.tile_w, (a.h + a.tile_h - 1) / a.tile_h, ndirs);
    lk_level_kernel<RAD, Ts><<<grid, kLkThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int RAD, class Ts>
cudaError_t launch_rad_batch(const LkBatch& b, cudaStream_t s) {
    const LkArgs& a0 = b.pair[0];
    size_t smem = lk_smem_bytes(a0.tile_w, a0.tile_h, a0.iters, a0.radius);
    int gx = 0, gy = 0;
    for (int p = 0; p < b.n; ++p) {
        const LkArgs& a = b.pair[p];
        if (a.tile_w != a0.tile_w || a.tile_h != a0.tile_h || a.iters != a0.iters || a.radius != a0.radius ||
            a.pyr != a0.pyr)
            return cudaErrorInvalidValue;
        gx = max(gx, (a.w + a.tile_w - 1) / a.tile_w);
        gy = max(gy, (a.h + a.tile_h - 1) / a.tile_h);
    }
    dim3 grid(gx, gy, 2 * b.n);
    lk_level_batch_kernel<RAD, Ts><<<grid, kLkThreads, smem, s>>>(b);
    return cudaGetLastError();
}

template <class Ts>
cudaError_t launch_tile_t(const LkArgs& a, int ndirs, cudaStream_t s) {
    switch (a.radius) {
        case 1: return launch_rad<1, Ts>(a, ndirs, s);
        case 2: return launch_rad<2, Ts>(a, ndirs, s);
        case 3: return launch_rad<3, Ts>(a, ndirs, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class Ts>
cudaError_t launch_tile_batch_t(const LkBatch& b, cudaStream_t s) {
    switch (b.pair[0].radius) {
        case 1: return launch_rad_batch<1, Ts>(b, s);
        case 2: return launch_rad_batch<2, Ts>(b, s);
        case 3: return launch_rad_batch<3, Ts>(b, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class Ts>
cudaError_t prepare_tile_t(int max_smem_bytes) {
    const void* fns[] = {(const void*)lk_level_kernel<1, Ts>,       (const void*)lk_level_kernel<2, Ts>,
                         (const void*)lk_level_kernel<3, Ts>,       (const void*)lk_level_batch_kernel<1, Ts>,
                         (const void*)lk_level_batch_kernel<2, Ts>, (const void*)lk_level_batch_kernel<3, Ts>};
    for (const void* f : fns) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem_bytes);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

size_t lk_smem_bytes(int tile_w, int tile_h, int iters, int radius) {
    size_t halo = (size_t)iters * radius;
    size_t n = (tile_w + 2 * halo) * (tile_h + 2 * halo);
    const size_t box = sizeof(float) * (size_t)tile_jbw((int)(tile_w + 2 * halo)) * tile_jbh((int)(tile_h + 2 * halo));
    return n * (sizeof(float4) + 4 * sizeof(float2) + sizeof(float)) + box;
}

cudaError_t lk_prepare(int max_smem_bytes) {
    cudaError_t e;
    if ((e = lk_stream_prepare(max_smem_bytes)) != cudaSuccess) return e;
    if ((e = prepare_tile_t<float>(max_smem_bytes)) != cudaSuccess) return e;
    if ((e = prepare_tile_t<__nv_bfloat16>(max_smem_bytes)) != cudaSuccess) return e;
    return prepare_tile_t<__half>(max_smem_bytes);
}

cudaError_t launch_lk_level(const LkArgs& a, int ndirs, cudaStream_t s) {
    // Small levels have too few rows to fill the streamed schedule; tiles
    // run them in one short wave.
    if (lk_stream_supports(a.iters, a.radius) && (long long)a.w * a.h >= kStreamMinPixels)
        return launch_lk_stream(a, ndirs, s);
    return launch_lk_tile(a, ndirs, s);
}

PANO_BOUNDS_READER(bounds_read_lk_tile)

cudaError_t launch_lk_tile_batch(const LkBatch& b, cudaStream_t s) {
    if (b.n < 1 || b.n > kMaxBatch) return cudaErrorInvalidValue;
    switch (b.pair[0].pyr) {
        case kPyrF32: return launch_tile_batch_t<float>(b, s);
        case kPyrBF16: return launch_tile_batch_t<__nv_bfloat16>(b, s);
        case kPyrF16: return launch_tile_batch_t<__half>(b, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_lk_tile(const LkArgs& a, int ndirs, cudaStream_t s) {
    switch (a.pyr) {
        case kPyrF32: return launch_tile_t<float>(a, ndirs, s);
        case kPyrBF16: return launch_tile_t<__nv_bfloat16>(a, ndirs, s);
        case kPyrF16: return launch_tile_t<__half>(a, ndirs, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pano
