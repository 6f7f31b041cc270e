// refine.cu -- energy and adjoint kernels for differentiable flow refinement.
//
// Not a step of the paper's method: a build extension that refines a flow by
// gradient steps on the energy
//   E(u) = sum_p (J(p + u(p)) - T(p))^2
//        + alpha sum_p sum_c [ (u_c(p + e_x) - u_c(p))^2 [x < w-1] + (u_c(p + e_y) - u_c(p))^2 [y < h-1] ]
// (data term of the LK step, smoothness term of the Horn-Schunck half of
// [20]). J is sampled with the bilinear clamp-to-edge sampler of the flow
// path. The kernels give E (reduced in FP64 -- the only FP64 arithmetic on
// the GPU, used by finite-difference checks), dE/du, dE/dT and dE/dJ, and the
// transpose of the pyramid REDUCE so that gradients can be carried to
// full-resolution images without storing the pyramid.
#include "bounds.cuh"
#include "common.cuh"

namespace pano {

namespace {

constexpr int kEgThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kEgThreads) energy_grad_kernel(EnergyArgs a) {
    __shared__ double s_part[kEgThreads / 32];
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * (kEgThreads / 32) + (threadIdx.x >> 5);
    const int w = a.w, h = a.h;
    double e = 0.0;
    if (x < w && y < h) {
        const long long p = (long long)y * w + x;
        const long long nf = (long long)h * w;                      // flow / gradient elements
        const long long nj = (long long)(h - 1) * a.pitch + w;      // elements of T and J
        (void)nf;
        (void)nj;
        const float2* U = reinterpret_cast<const float2*>(a.u);
        const float2 u = PANO_AT(U, p, nf, 601);
        // bilinear sample of J at p + u and its derivative along x and y
        const float ox = fminf(fmaxf(u.x, -(float)(w + 2)), (float)(w + 2));
        const float oy = fminf(fmaxf(u.y, -(float)(h + 2)), (float)(h + 2));
        const float fxf = floorf(ox), fyf = floorf(oy);
        const float fx = ox - fxf, fy = oy - fyf;
        const int x0 = x + (int)fxf, y0 = y + (int)fyf;
        const int xa = min(max(x0, 0), w - 1), xb = min(max(x0 + 1, 0), w - 1);
        const int ya = min(max(y0, 0), h - 1), yb = min(max(y0 + 1, 0), h - 1);
        const long long ra = (long long)ya * a.pitch, rb = (long long)yb * a.pitch;
        const float i00 = __ldg(&PANO_AT(a.J, ra + xa, nj, 602)), i10 = __ldg(&PANO_AT(a.J, ra + xb, nj, 602));
        const float i01 = __ldg(&PANO_AT(a.J, rb + xa, nj, 602)), i11 = __ldg(&PANO_AT(a.J, rb + xb, nj, 602));
        const float top = fmaf(fx, i10 - i00, i00), bot = fmaf(fx, i11 - i01, i01);
        const float Jw = fmaf(fy, bot - top, top);
        const float r = Jw - __ldg(&PANO_AT(a.T, (long long)y * a.pitch + x, nj, 603));
        e = (double)r * (double)r;
        // smoothness: forward differences to the right and downwards
        float2 lap = make_float2(0.f, 0.f);
        double es = 0.0;
        if (x < w - 1) {
            const float2 n = PANO_AT(U, p + 1, nf, 604);
            const float dx0 = n.x - u.x, dx1 = n.y - u.y;
            es += (double)dx0 * dx0 + (double)dx1 * dx1;
            lap.x -= dx0;
            lap.y -= dx1;
        }
        if (y < h - 1) {
            const float2 n = PANO_AT(U, p + w, nf, 605);
            const float dy0 = n.x - u.x, dy1 = n.y - u.y;
            es += (double)dy0 * dy0 + (double)dy1 * dy1;
            lap.x -= dy0;
            lap.y -= dy1;
        }
        if (x > 0) {
            const float2 n = PANO_AT(U, p - 1, nf, 606);
            lap.x += u.x - n.x;
            lap.y += u.y - n.y;
        }
        if (y > 0) {
            const float2 n = PANO_AT(U, p - w, nf, 607);
            lap.x += u.x - n.x;
            lap.y += u.y - n.y;
        }
        e += (double)a.alpha * es;
        if (a.grad_u) {
            const float jdx = fmaf(fy, (i11 - i01) - (i10 - i00), i10 - i00);
            const float jdy = fmaf(fx, (i11 - i10) - (i01 - i00), i01 - i00);
            PANO_AT(reinterpret_cast<float2*>(a.grad_u), p, nf, 608) =
                make_float2(2.f * r * jdx + 2.f * a.alpha * lap.x, 2.f * r * jdy + 2.f * a.alpha * lap.y);
        }
        if (a.grad_T) PANO_AT(a.grad_T, p, nf, 609) = -2.f * r;
        if (a.grad_J) {
            const float g = 2.f * r;
            float* GJ = a.grad_J;
            atomicAdd(&PANO_AT(GJ, (long long)ya * w + xa, nf, 610), g * (1.f - fy) * (1.f - fx));
            atomicAdd(&PANO_AT(GJ, (long long)ya * w + xb, nf, 610), g * (1.f - fy) * fx);
            atomicAdd(&PANO_AT(GJ, (long long)yb * w + xa, nf, 610), g * fy * (1.f - fx));
            atomicAdd(&PANO_AT(GJ, (long long)yb * w + xb, nf, 610), g * fy * fx);
        }
    }
    if (a.energy) {
        e = warp_sum(e);
        if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = e;
        __syncthreads();
        if (threadIdx.x < 32) {
            double v = threadIdx.x < kEgThreads / 32 ? s_part[threadIdx.x] : 0.0;
            v = warp_sum(v);
            if (threadIdx.x == 0) atomicAdd(a.energy, v);
        }
    }
}

// Rows (or columns) of the level below that a source row feeds, with their
// REDUCE weights: source index s receives weight k[t] from destination index
// d whenever clamp(2 d + t, 0, n - 1) == s, t in [-2, 2]. At most four
// destination indices qualify: d in [s/2 - 1, s/2 + 2] (border clamping adds
// weight, never indices); a weight of zero marks an unused candidate.
__device__ __forceinline__ void reduce_taps(int s, int n, int nd, int (&d)[4], float (&wt)[4]) {
    const float k[5] = {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16};
    const int base = (s >> 1) - 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int dd = base + i;
        float acc = 0.f;
#pragma unroll
        for (int t = -2; t <= 2; ++t)
            if (min(max(2 * dd + t, 0), n - 1) == s) acc += k[t + 2];
        const bool ok = dd >= 0 && dd < nd;
        d[i] = min(max(dd, 0), nd - 1);
        wt[i] = ok ? acc : 0.f;
    }
}

__global__ void __launch_bounds__(256) pyr_down_adjoint_kernel(const float* __restrict__ gdst, int h, int w,
                                                               int dst_pitch, float* __restrict__ gsrc,
                                                               int src_pitch) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= w || y >= h) return;
    const int hd = (h + 1) / 2, wd = (w + 1) / 2;
    int dy[4], dx[4];
    float wy[4], wx[4];
    reduce_taps(y, h, hd, dy, wy);
    reduce_taps(x, w, wd, dx, wx);
    const long long nd = (long long)(hd - 1) * dst_pitch + wd;  // elements of the gradient of the output
    (void)nd;
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const long long ro = (long long)dy[i] * dst_pitch;
        float racc = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) racc = fmaf(wx[j], __ldg(&PANO_AT(gdst, ro + dx[j], nd, 611)), racc);
        acc = fmaf(wy[i], racc, acc);
    }
    PANO_AT(gsrc, (long long)y * src_pitch + x, (long long)(h - 1) * src_pitch + w, 612) = acc;
}

}  // namespace

PANO_BOUNDS_READER(bounds_read_refine)

cudaError_t launch_energy_grad(const EnergyArgs& a, cudaStream_t s) {
    cudaError_t e;
    if (a.energy && (e = cudaMemsetAsync(a.energy, 0, sizeof(double), s)) != cudaSuccess) return e;
    if (a.grad_J && (e = cudaMemsetAsync(a.grad_J, 0, sizeof(float) * (size_t)a.h * a.w, s)) != cudaSuccess)
        return e;
    dim3 grid((a.w + 31) / 32, (a.h + kEgThreads / 32 - 1) / (kEgThreads / 32));
    energy_grad_kernel<<<grid, kEgThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pyr_down_adjoint(const float* gdst, int h, int w, int dst_pitch, float* gsrc, int src_pitch,
                                    cudaStream_t s) {
    dim3 block(32, 8);
    dim3 grid((w + 31) / 32, (h + 7) / 8);
    pyr_down_adjoint_kernel<<<grid, block, 0, s>>>(gdst, h, w, dst_pitch, gsrc, src_pitch);
    return cudaGetLastError();
}

}  // namespace pano
