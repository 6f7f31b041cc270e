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
// Distances are computed exactly, as integers, in two separable passes:
//   columns: g(x, y) = |y - y'| to the nearest feature pixel (x, y') of the
//            same column, or "none";
//   rows:    d2(x, y) = min over columns x' of (x - x')^2 + g(x', y)^2, the
//            lower envelope of one parabola per column that has a feature
//            (edt_row.cuh: banded envelopes merged in a tree).
// Only the final ratio is rounded (FP32 square roots and one division).
#include <stdio.h>
#include <string.h>

#include <climits>

#include "bounds.cuh"
#include "common.cuh"
#include "ctx.h"
#include "edt_row.cuh"
#include "pano_flow.h"

namespace pano {

namespace {

// ---------------------------------------------------------------------------
// Column pass. A CTA of 32 x 32 threads owns 32 columns and walks down them
// in blocks of 1024 rows; thread (tx, ty) holds rows ty*32 .. ty*32+31 of a
// block of column tx as two 32-bit masks (Area1, Area2 pixels). A first pass
// over the labels finds, per column and block, the first feature row; a
// suffix minimum gives the first feature row at or after each block. The
// second pass finds each row's nearest feature above and below from the
// bits of its own mask, the masks of the other threads of its block (shared
// memory), the last feature row of the blocks above and the first of the
// blocks below. g of each area goes to a plane of 16-bit values (coalesced
// 2-byte stores; edt::kNoSite where the column has no feature pixel).
// ---------------------------------------------------------------------------
constexpr int kColW = 32;                     // columns per CTA
constexpr int kColTY = 32;                    // threads along y, 32 rows each
constexpr int kColBlock = 32 * kColTY;        // rows per block
constexpr int kMaxBlocks = (65535 + kColBlock - 1) / kColBlock;
constexpr int kAboveNone = -(1 << 20);        // y - kAboveNone > any distance
constexpr int kBelowNone = INT_MAX;

__device__ __forceinline__ void col_masks(const unsigned char* __restrict__ label, long long pitch, long long nl,
                                          int h, int x, int y0, uint32_t* m1, uint32_t* m2) {
    uint32_t a = 0, b = 0;
    const int n = min(32, h - y0);
    const unsigned char* p = label + (long long)y0 * pitch + x;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
        if (i < n) {
            const unsigned char c = __ldg(&PANO_AT(p, (long long)i * pitch, nl - ((long long)y0 * pitch + x), 501));
            a |= (uint32_t)(c == 1) << i;
            b |= (uint32_t)(c == 2) << i;
        }
    }
    *m1 = a;
    *m2 = b;
}

__global__ void __launch_bounds__(kColW * kColTY, 2) edt_cols_kernel(const unsigned char* __restrict__ label, int h,
                                                                    int w, long long pitch, uint16_t* __restrict__ g1,
                                                                    uint16_t* __restrict__ g2) {
    __shared__ int s_next[2][kMaxBlocks + 1][kColW];  // first feature row at or after block rb's first row
    __shared__ uint32_t s_mask[2][kColTY][kColW];
    __shared__ int s_above[2][kColW];                 // last feature row above the current block
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kColW + tx;
    const int x = blockIdx.x * kColW + tx;
    const bool col_in = x < w;
    const int nblk = (h + kColBlock - 1) / kColBlock;
    const long long nl = (long long)(h - 1) * pitch + w, ng = (long long)h * w;  // label and g elements
    (void)nl;
    (void)ng;
    constexpr int NN = 2 * (kMaxBlocks + 1) * kColW;
    for (int i = tid; i < NN; i += kColW * kColTY) PANO_AT(&s_next[0][0][0], i, NN, 502) = kBelowNone;
    if (tid < 2 * kColW) PANO_AT(&s_above[0][0], tid, 2 * kColW, 503) = kAboveNone;
    __syncthreads();
    for (int rb = 0; rb < nblk; ++rb) {
        const int y0 = rb * kColBlock + ty * 32;
        uint32_t m1 = 0, m2 = 0;
        if (col_in && y0 < h) col_masks(label, pitch, nl, h, x, y0, &m1, &m2);
        if (m1) atomicMin(&s_next[0][rb][tx], y0 + __ffs(m1) - 1);
        if (m2) atomicMin(&s_next[1][rb][tx], y0 + __ffs(m2) - 1);
    }
    __syncthreads();
    if (ty < 2)
        for (int rb = nblk - 1; rb >= 0; --rb) s_next[ty][rb][tx] = min(s_next[ty][rb][tx], s_next[ty][rb + 1][tx]);
    __syncthreads();
    for (int rb = 0; rb < nblk; ++rb) {
        const int yb = rb * kColBlock, y0 = yb + ty * 32;
        uint32_t m[2] = {0, 0};
        if (col_in && y0 < h) col_masks(label, pitch, nl, h, x, y0, &m[0], &m[1]);
        s_mask[0][ty][tx] = m[0];
        s_mask[1][ty][tx] = m[1];
        __syncthreads();
        int above[2], below[2];  // nearest feature rows above and below this thread's 32 rows
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            int p = s_above[a][tx];
            for (int k = ty - 1; k >= 0; --k) {
                const uint32_t v = s_mask[a][k][tx];
                if (v) {
                    p = yb + k * 32 + 31 - __clz(v);
                    break;
                }
            }
            int n = s_next[a][rb + 1][tx];
            for (int k = ty + 1; k < kColTY; ++k) {
                const uint32_t v = s_mask[a][k][tx];
                if (v) {
                    n = yb + k * 32 + __ffs(v) - 1;
                    break;
                }
            }
            above[a] = p;
            below[a] = n;
        }
        if (col_in && y0 < h) {
            const int n = min(32, h - y0);
#pragma unroll 8
            for (int i = 0; i < 32; ++i) {
                if (i >= n) break;
                const int yy = y0 + i;
                uint32_t g[2];
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const uint32_t up = m[a] << (31 - i);  // rows y0 .. yy, row yy in bit 31
                    const uint32_t dn = m[a] >> i;         // rows yy .. y0 + 31, row yy in bit 0
                    // distances above and below (ints: rows < 2^16, the no-feature
                    // values keep both differences below 2^31)
                    const int da = up ? __clz(up) : yy - above[a];
                    const int db = dn ? __ffs(dn) - 1 : below[a] - yy;
                    const int d = min(da, db);
                    g[a] = d >= (int)edt::kNoSite ? edt::kNoSite : (uint32_t)d;
                }
                PANO_AT(g1, (long long)yy * w + x, ng, 504) = (uint16_t)g[0];
                PANO_AT(g2, (long long)yy * w + x, ng, 504) = (uint16_t)g[1];
            }
        }
        __syncthreads();  // the masks and s_above are read
        if (ty == kColTY - 1) {
            s_above[0][tx] = m[0] ? y0 + 31 - __clz(m[0]) : above[0];
            s_above[1][tx] = m[1] ? y0 + 31 - __clz(m[1]) : above[1];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Row pass: one CTA of kRowThreads per row and area, one band of
// ceil(w / kRowThreads) columns per thread (edt_row.cuh for the steps).
// The Area1 launch writes the distances to Area1 (FP32 square roots of the
// exact squared distances, +inf with no Area1 pixel on the canvas) of the
// Area3 pixels to a plane; the Area2 launch reads them there and writes
// Eq. (1).
// Shared memory, all dynamic (the kernel's limit is set to the device
// maximum): the row's g (2 B per column), the kept sites (2 B per column),
// five ints per band and 33 ints for the scans; five CTAs fit on an SM at
// 9000 columns.
// ---------------------------------------------------------------------------
constexpr int kRowThreads = 256;
constexpr int kRowWarps = kRowThreads / 32;
constexpr int kRowCtas = 5;

// inclusive prefix maximum over the threads of the block
__device__ __forceinline__ int block_prefix_max(int v, int* s_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v = max(v, t);
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int t = lane < kRowWarps ? s_warp[lane] : INT_MIN;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t = max(t, u);
        }
        if (lane < kRowWarps) s_warp[lane] = t;
    }
    __syncthreads();
    if (wid > 0) v = max(v, s_warp[wid - 1]);
    __syncthreads();
    return v;
}

// inclusive suffix minimum over the threads of the block
__device__ __forceinline__ int block_suffix_min(int v, int* s_warp) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_down_sync(0xffffffffu, v, o);
        if (lane + o < 32) v = min(v, t);
    }
    if (lane == 0) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int t = lane < kRowWarps ? s_warp[lane] : INT_MAX;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_down_sync(0xffffffffu, t, o);
            if (lane + o < 32) t = min(t, u);
        }
        if (lane < kRowWarps) s_warp[lane] = t;
    }
    __syncthreads();
    if (wid + 1 < kRowWarps) v = min(v, s_warp[wid + 1]);
    __syncthreads();
    return v;
}

// kFinal false: Area1 (g = g1), writes dist1; true: Area2, writes Blend
template <bool kFinal>
__global__ void __launch_bounds__(kRowThreads, kRowCtas) edt_row_kernel(const unsigned char* __restrict__ label,
                                                                        int h, int w, long long pitch,
                                                                        const uint16_t* __restrict__ gplane,
                                                                        float* __restrict__ dist1,
                                                                        float* __restrict__ blend, int blend_pitch) {
    using namespace edt;
    constexpr int NB = kRowThreads;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint16_t* gs = reinterpret_cast<uint16_t*>(s_dyn);                  // [w]
    uint16_t* st = gs + w;                                              // [w]
    int* lo = reinterpret_cast<int*>(s_dyn + 4 * (size_t)w);            // [NB]
    int* hi = lo + NB;                                                  // [NB]
    int* gfirst = hi + NB;   // [NB] first band of a group; then the last band <= b with a site
    int* glast = gfirst + NB;  // [NB] last band of a group; then the first band >= b with a site
    int* zs = glast + NB;      // [NB] start of the region of band b's first site
    int* s_warp = zs + NB;     // [32] warp totals of the scans
    int* s_any = s_warp + 32;  // [1] the row has a site
    const int tid = threadIdx.x, y = blockIdx.x;
    const int bw = (w + NB - 1) / NB;
    const long long ng = (long long)h * w;
    (void)ng;
    for (int i = tid; i < w; i += NB) PANO_AT(gs, i, w, 505) = PANO_AT(gplane, (long long)y * w + i, ng, 506);
    __syncthreads();
    const int x0 = min(w, tid * bw), x1 = min(w, x0 + bw);
    {
        // step 0: the runs of equal g at the band's edges, against the
        // columns before and after them (found by scans over the bands)
        int ls, fe;
        band_run_edges(gs, w, x0, x1, &ls, &fe);
        const int ps = block_prefix_max(ls, s_warp);
        const int sf = block_suffix_min(fe, s_warp);
        zs[tid] = ps;
        glast[tid] = sf;
        __syncthreads();
        int L = -1, R = w;
        if (x0 < x1) {
            const int u = (x0 == 0 || gs[x0] != gs[x0 - 1]) ? x0 : (tid > 0 ? zs[tid - 1] : 0);
            const int v = (x1 == w || gs[x1 - 1] != gs[x1]) ? x1 - 1 : (tid + 1 < NB ? glast[tid + 1] : w - 1);
            L = u - 1;
            R = v + 1;
        }
        edge_runs_hidden(gs, st, w, x0, x1, L, R);
        __syncthreads();
        for (int q = x0; q < x1; ++q)
            if (st[q]) gs[q] = (uint16_t)kNoSite;
        __syncthreads();
    }
    {
        const int k = band_envelope(gs, st, w, x0, x1);
        PANO_AT(lo, tid, NB, 507) = x0;
        PANO_AT(hi, tid, NB, 507) = x0 + k;
        PANO_AT(gfirst, tid, NB, 507) = k ? tid : -1;
        PANO_AT(glast, tid, NB, 507) = k ? tid : -1;
    }
    __syncthreads();
    // merge tree: in the round of stride s, thread lg (a multiple of 2 s)
    // merges the groups lg and lg + s
    for (int s = 1; s < NB; s <<= 1) {
        const int lg = tid;
        if ((lg & (2 * s - 1)) == 0 && lg + s < NB) {
            const int lf = PANO_AT(gfirst, lg, NB, 508), ll = PANO_AT(glast, lg, NB, 508);
            const int rf = PANO_AT(gfirst, lg + s, NB, 508), rl = PANO_AT(glast, lg + s, NB, 508);
            if (rf >= 0) {
                if (lf < 0) {
                    gfirst[lg] = rf;
                } else {
                    const bool ok = merge_groups(gs, st, lo, hi, w, NB, lf, ll, rf, rl);
                    PANO_FLAG(!ok, 509);  // the merge reached its iteration limit
                    (void)ok;
                }
                glast[lg] = rl;
            }
        }
        __syncthreads();
    }
    if (tid == 0) s_any[0] = gfirst[0] >= 0;
    // the last band <= b and the first band >= b that keep a site
    {
        const bool kept = hi[tid] > lo[tid];
        const int pv = block_prefix_max(kept ? tid : -1, s_warp);
        const int nx = block_suffix_min(kept ? tid : NB, s_warp);
        gfirst[tid] = pv;
        glast[tid] = nx;
    }
    __syncthreads();
    if (hi[tid] > lo[tid]) {
        const int pb = tid > 0 ? gfirst[tid - 1] : -1;
        int z = -1;
        if (pb >= 0) {
            const int p = PANO_AT(st, hi[pb] - 1, w, 510), q = PANO_AT(st, lo[tid], w, 510);
            z = region_start(f_of(gs, w, p), p, f_of(gs, w, q), q, w);
        }
        zs[tid] = z;
    }
    __syncthreads();
    if (hi[tid] <= lo[tid]) {
        const int n = glast[tid];
        zs[tid] = n < NB ? PANO_AT(zs, n, NB, 511) : w;
    }
    __syncthreads();
    if (x0 >= x1) return;
    const bool any = s_any[0] != 0;
    Walker k = {0, 0, 0, 0, 0};
    if (any) k = walk_start(gs, st, lo, hi, zs, w, NB, x0);
    const long long ro = (long long)y * w;
    const unsigned char* lab = label + (long long)y * pitch;
    if constexpr (!kFinal) {
        // only Area3 pixels read the distances to Area1
        for (int x = x0; x < x1; ++x)
            if (PANO_AT(lab, x, w, 512) == 3)
                PANO_AT(dist1, ro + x, ng, 512) =
                    any ? sqrtf((float)walk_to(gs, st, lo, hi, glast, w, NB, x, &k)) : INFINITY;
    } else {
        float* out = blend + (long long)y * blend_pitch;
        for (int x = x0; x < x1; ++x) {
            const unsigned char c = PANO_AT(lab, x, w, 513);
            float b;
            if (c == 1) {
                b = 0.f;
            } else if (c == 2) {
                b = 1.f;
            } else if (c == 3) {
                const float dl = PANO_AT(dist1, ro + x, ng, 514);
                const float dr = any ? sqrtf((float)walk_to(gs, st, lo, hi, glast, w, NB, x, &k)) : INFINITY;
                const bool no1 = isinf(dl), no2 = !any;
                if (no1 && no2) b = 0.5f;
                else if (no1) b = 1.f;
                else if (no2) b = 0.f;
                else b = dl / (dl + dr);
            } else {
                b = 0.5f;
            }
            PANO_AT(out, x, w, 515) = b;
        }
    }
}

}  // namespace

PANO_BOUNDS_READER(bounds_read_edt)

size_t blend_coeff_scratch_bytes(int h, int w) {
    return (size_t)h * w * (2 * sizeof(uint16_t) + sizeof(float));  // g of both areas, distances to Area1
}

size_t blend_coeff_row_smem(int w) { return (size_t)4 * w + (size_t)(5 * kRowThreads + 33) * sizeof(int); }

cudaError_t blend_coeff_prepare(int max_smem_bytes) {
    cudaError_t e = cudaFuncSetAttribute(edt_row_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         max_smem_bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(edt_row_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem_bytes);
}

cudaError_t launch_blend_coeff(const unsigned char* label, int h, int w, long long pitch, float* blend,
                               int blend_pitch, void* scratch, cudaStream_t s) {
    uint16_t* g1 = static_cast<uint16_t*>(scratch);
    uint16_t* g2 = g1 + (size_t)h * w;
    float* dist1 = reinterpret_cast<float*>(g2 + (size_t)h * w);
    edt_cols_kernel<<<(w + kColW - 1) / kColW, dim3(kColW, kColTY), 0, s>>>(label, h, w, pitch, g1, g2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = blend_coeff_row_smem(w);
    edt_row_kernel<false><<<h, kRowThreads, smem, s>>>(label, h, w, pitch, g1, dist1, blend, blend_pitch);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    edt_row_kernel<true><<<h, kRowThreads, smem, s>>>(label, h, w, pitch, g2, dist1, blend, blend_pitch);
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
        return fail(PANO_ERR_UNSUPPORTED, "canvas %dx%d: sides above 65535 (16-bit distances and columns)", h, w);
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
