// edt.cu -- the global blending coefficient of Eq. (1) (Section III-C-2) on
// a labelled canvas of any shape, through an exact Euclidean distance
// transform.
//
// Eq. (1): Blend = 0 in Area1, 1 in Area2 and Lmin / (Lmin + Rmin) in
// Area3, where Lmin / Rmin are the distances from the pixel to the nearest
// Area1 / Area2 pixel (Euclidean, between pixel centres). Pixels in none of
// the areas get 0.5. A canvas without any Area1 pixel gives Blend = 1 in
// Area3 (the limit as Lmin grows without bound), without Area2 0, with
// neither 0.5.
//
// Distances are computed exactly, as integers, in two separable passes
// (Felzenszwalb & Huttenlocher, "Distance transforms of sampled functions",
// 2012):
//   columns: g(x, y) = |y - y'| to the nearest feature pixel (x, y') of the
//            same column, or "none";
//   rows:    d2(x, y) = min over columns x' of (x - x')^2 + g(x', y)^2, the
//            lower envelope of one parabola per column that has a feature.
// The envelope of a row is built by one thread per area; the intersection
// abscissae of neighbouring parabolas are rationals, compared exactly by
// cross-multiplication in 64-bit integers, so d2 is exact. Only the final
// ratio is rounded (FP32 square roots and one division).
#include <stdio.h>
#include <string.h>

#include <climits>

#include "bounds.cuh"
#include "common.cuh"
#include "ctx.h"
#include "pano_flow.h"

namespace pano {

namespace {

constexpr int kNone = 1 << 29;      // no feature pixel in the column
constexpr int kColThreads = 128;
constexpr int kRowThreads = 128;

// Column pass: one thread per column, a downward and an upward sweep.
__global__ void __launch_bounds__(kColThreads) edt_cols_kernel(const unsigned char* __restrict__ label, int h,
                                                               int w, long long pitch, int* __restrict__ gL,
                                                               int* __restrict__ gR) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= w) return;
    const long long nl = (long long)(h - 1) * pitch + w, ng = (long long)h * w;  // label and g elements
    (void)nl;
    (void)ng;
    int dl = kNone, dr = kNone;
    for (int y = 0; y < h; ++y) {
        const unsigned char a = __ldg(&PANO_AT(label, (long long)y * pitch + x, nl, 501));
        dl = a == 1 ? 0 : min(dl + 1, kNone);
        dr = a == 2 ? 0 : min(dr + 1, kNone);
        PANO_AT(gL, (long long)y * w + x, ng, 502) = dl;
        PANO_AT(gR, (long long)y * w + x, ng, 502) = dr;
    }
    dl = dr = kNone;
    for (int y = h - 1; y >= 0; --y) {
        const unsigned char a = __ldg(&PANO_AT(label, (long long)y * pitch + x, nl, 503));
        dl = a == 1 ? 0 : min(dl + 1, kNone);
        dr = a == 2 ? 0 : min(dr + 1, kNone);
        const long long o = (long long)y * w + x;
        PANO_AT(gL, o, ng, 504) = min(PANO_AT(gL, o, ng, 504), dl);
        PANO_AT(gR, o, ng, 504) = min(PANO_AT(gR, o, ng, 504), dr);
    }
}

// Parabola of site q of a row of w columns: f(q) + (x - q)^2 with f = g^2.
__device__ __forceinline__ long long site_f(const int* __restrict__ g, int w, int q) {
    (void)w;
    const long long v = PANO_AT(g, q, w, 505);
    return v * v;
}

// Intersection abscissa of the parabolas of sites p < q as num / den (den > 0).
__device__ __forceinline__ void intersect(const int* __restrict__ g, int w, int p, int q, long long* num,
                                          long long* den) {
    *num = (site_f(g, w, q) + (long long)q * q) - (site_f(g, w, p) + (long long)p * p);
    *den = 2LL * (q - p);
}

// Lower envelope of one row: v[0..k] are the sites whose parabolas form it,
// from left to right; returns k (-1 when the row has no site).
__device__ int build_envelope(const int* __restrict__ g, int w, int* __restrict__ v) {
    int k = -1;
    for (int q = 0; q < w; ++q) {
        if (PANO_AT(g, q, w, 506) >= kNone) continue;
        if (k < 0) {
            PANO_AT(v, ++k, w, 507) = q;
            continue;
        }
        // drop envelope parabolas that the new one hides: while the new
        // intersection lies at or left of the start of the last parabola
        while (k >= 1) {
            long long n1, d1, n0, d0;
            intersect(g, w, PANO_AT(v, k, w, 508), q, &n1, &d1);  // s(v[k], q)
            intersect(g, w, PANO_AT(v, k - 1, w, 508), PANO_AT(v, k, w, 508), &n0, &d0);  // z[k] = s(v[k-1], v[k])
            if (n1 * d0 <= n0 * d1) --k;
            else break;
        }
        PANO_AT(v, ++k, w, 507) = q;
    }
    return k;
}

// Squared distance at column x from an envelope of k + 1 sites.
__device__ __forceinline__ long long envelope_at(const int* __restrict__ g, const int* __restrict__ v, int w, int k,
                                                int x) {
    // largest j with z[j] <= x, z[0] = -infinity, z[j] = s(v[j-1], v[j])
    int lo = 0, hi = k;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        long long n, d;
        intersect(g, w, PANO_AT(v, mid - 1, w, 509), PANO_AT(v, mid, w, 509), &n, &d);
        if (n <= (long long)x * d) lo = mid;
        else hi = mid - 1;
    }
    const int q = PANO_AT(v, lo, w, 509);
    const long long dx = x - q;
    return dx * dx + site_f(g, w, q);
}

// Row pass and Eq. (1): one CTA per row. Warp 0 builds the Area1 envelope,
// warp 1 the Area2 envelope (one thread each); then every thread fills
// columns.
__global__ void __launch_bounds__(kRowThreads) edt_rows_blend_kernel(const unsigned char* __restrict__ label, int h,
                                                                     int w, long long pitch,
                                                                     const int* __restrict__ gL,
                                                                     const int* __restrict__ gR,
                                                                     float* __restrict__ blend, int blend_pitch) {
    // dynamic shared memory only (the kernel's limit is set to the device
    // maximum): the two envelope sizes, then the sites of each envelope
    extern __shared__ int s_dyn[];
    int* s_k = s_dyn;
    int* vL = s_dyn + 2;
    int* vR = vL + w;
    const int y = blockIdx.x;
    const int* rowL = gL + (long long)y * w;
    const int* rowR = gR + (long long)y * w;
    if (threadIdx.x == 0) s_k[0] = build_envelope(rowL, w, vL);
    if (threadIdx.x == 32) s_k[1] = build_envelope(rowR, w, vR);
    __syncthreads();
    const int kL = s_k[0], kR = s_k[1];
    const unsigned char* lab = label + (long long)y * pitch;
    float* out = blend + (long long)y * blend_pitch;
    for (int x = threadIdx.x; x < w; x += blockDim.x) {
        const unsigned char a = PANO_AT(lab, x, w, 510);
        float b;
        if (a == 1) {
            b = 0.f;
        } else if (a == 2) {
            b = 1.f;
        } else if (a == 3) {
            if (kL < 0 && kR < 0) b = 0.5f;
            else if (kL < 0) b = 1.f;
            else if (kR < 0) b = 0.f;
            else {
                const float dl = sqrtf((float)envelope_at(rowL, vL, w, kL, x));
                const float dr = sqrtf((float)envelope_at(rowR, vR, w, kR, x));
                b = dl / (dl + dr);
            }
        } else {
            b = 0.5f;
        }
        PANO_AT(out, x, w, 511) = b;
    }
}

}  // namespace

PANO_BOUNDS_READER(bounds_read_edt)

size_t blend_coeff_scratch_bytes(int h, int w) { return (size_t)2 * h * w * sizeof(int); }

size_t blend_coeff_row_smem(int w) { return (size_t)(2 * w + 2) * sizeof(int); }

cudaError_t blend_coeff_prepare(int max_smem_bytes) {
    return cudaFuncSetAttribute(edt_rows_blend_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem_bytes);
}

cudaError_t launch_blend_coeff(const unsigned char* label, int h, int w, long long pitch, float* blend,
                               int blend_pitch, void* scratch, cudaStream_t s) {
    int* gL = static_cast<int*>(scratch);
    int* gR = gL + (size_t)h * w;
    edt_cols_kernel<<<(w + kColThreads - 1) / kColThreads, kColThreads, 0, s>>>(label, h, w, pitch, gL, gR);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    edt_rows_blend_kernel<<<h, kRowThreads, blend_coeff_row_smem(w), s>>>(label, h, w, pitch, gL, gR, blend,
                                                                          blend_pitch);
    return cudaGetLastError();
}

}  // namespace pano

using namespace pano;

extern "C" {

size_t pano_blend_coeff_scratch_bytes(int h, int w) {
    if (h < 1 || w < 1) return 0;
    return blend_coeff_scratch_bytes(h, w);
}

pano_status pano_blend_coeff(const unsigned char* label, int h, int w, size_t label_pitch, float* blend,
                             int blend_pitch, void* scratch, size_t scratch_bytes, void* cuda_stream) {
    if (!label || !blend || !scratch) return fail(PANO_ERR_INVALID_ARG, "label, blend or scratch is NULL");
    if (h < 1 || w < 1) return fail(PANO_ERR_INVALID_ARG, "canvas size %dx%d", h, w);
    if (h > 65535 || w > 65535)
        return fail(PANO_ERR_UNSUPPORTED, "canvas %dx%d: sides above 65535 (64-bit envelope products)", h, w);
    if (label_pitch < (size_t)w) return fail(PANO_ERR_INVALID_ARG, "label_pitch %zu < w %d", label_pitch, w);
    if (blend_pitch < w) return fail(PANO_ERR_INVALID_ARG, "blend_pitch %d < w %d", blend_pitch, w);
    if (((uintptr_t)blend) % 4 || ((uintptr_t)scratch) % 4)
        return fail(PANO_ERR_INVALID_ARG, "blend or scratch not 4-byte aligned");
    const size_t need = blend_coeff_scratch_bytes(h, w);
    if (scratch_bytes < need) return fail(PANO_ERR_INVALID_ARG, "scratch of %zu bytes < %zu", scratch_bytes, need);
    if ((double)h * (double)w > (double)INT_MAX * 8.0) return fail(PANO_ERR_UNSUPPORTED, "canvas too large");
    const size_t bb = (size_t)h * blend_pitch * sizeof(float), lb = (size_t)h * label_pitch;
    if (overlaps(blend, bb, label, lb) || overlaps(scratch, need, label, lb) || overlaps(scratch, need, blend, bb))
        return fail(PANO_ERR_INVALID_ARG, "label, blend and scratch must not overlap");
    int max_smem = 0;
    pano_status st;
    if ((st = ensure_lk_ready(&max_smem)) != PANO_OK) return st;
    if (blend_coeff_row_smem(w) > (size_t)max_smem)
        return fail(PANO_ERR_UNSUPPORTED, "canvas width %d needs %zu bytes of shared memory per row (device: %d)", w,
                    blend_coeff_row_smem(w), max_smem);
    cudaError_t e = launch_blend_coeff(label, h, w, (long long)label_pitch, blend, blend_pitch, scratch,
                                       static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? PANO_OK : cuda_fail(e, "blend coefficient launch");
}

}  // extern "C"
