// lk_stream_impl.cuh -- internal: the streamed LK kernel, templated on the
// storage type of the pyramid planes. One pyramid level of dense
// Lucas-Kanade flow (Section III-C-1), all K steps fused, streamed down
// column bands. Included once per storage type (lk_stream.cu: float,
// lk_stream_bf16.cu, lk_stream_f16.cu), each of which instantiates the entry
// points at the end of this file for its type only.
//
// Same arithmetic as lk_level_kernel (lk.cu): per step and pixel p
//   (G(p) + lambda I) v = sum_{q in W(p)} grad T(q) (grad T(q) . u(q) - It(q)) + lambda u(p),
//   It(q) = J(q + u(q)) - T(q), u(p) <- v,
// over the (2r+1)^2 box clipped to the image.
//
// Schedule. A CTA owns a band of BW output columns and a segment of output
// rows, plus a halo of K*r columns on each side. It walks down the segment in
// chunks of CH rows. Step k of the iteration ("stage k") runs r rows behind
// stage k-1, so that when stage k updates rows [a_k, a_k + CH) the flows it
// needs from stage k-1 (rows up to a_k + CH + r) are already final. Within a
// chunk the stages run in order:
//   X_0 : load T, grad T and the starting flow of the CH newest rows and form
//         the residual products P = grad T (grad T . u - It) of stage 1;
//   B_k : column sums of P over 2r+1 rows (stage k); B_1 also forms the
//         column sums of grad T grad T^T of the newest complete rows;
//   X_k : row sums, the 2x2 solve and the update of stage k (X_1 first
//         completes the normal matrices and inverts them), then, for the
//         same pixels, the products P of stage k+1; X_K writes the output
//         and loads the target rows of the next chunk.
// Per-row state (T, grad T, flow, inverse normal matrix) lives in a ring of
// kRing rows in shared memory; each stage keeps the last 2r rows of its
// products for the next chunk. The target image J is staged in a second ring
// of kRing rows: a box of the band shifted by the CTA's reference flow, with
// a margin of kMX columns and kMY rows, holding clamp-to-edge values; a sample
// whose four taps fall outside the box is read from global memory instead.
// The first chunks of a segment start ceil(2 K r / CH) chunks early, so every
// row a stage must produce is computed from complete windows; the rows before
// that are discarded. Flows are kept relative to the reference flow (the
// starting flow at the centre of the band and segment) so that FP32 rounding
// does not grow with the size of the flow.
//
// T and J are read as Ts and widened to FP32: float planes are fetched with
// cp.async, 16-bit planes with plain loads (their elements are narrower than
// the 4-byte copies), the target rows of the next chunk into registers before
// X_K and stored to the ring after it.
#pragma once

#include <type_traits>

#include "bounds.cuh"
#include "common.cuh"

namespace pano {
namespace lks {

constexpr int kStreamThreads = 768;
constexpr int kRing = 32;
constexpr int kRingOff = 1 << 20;  // keeps ring slots of negative rows non-negative
constexpr int kMX = 8;             // target box margin, columns
constexpr int kMY = 3;             // target box margin, rows
constexpr int kCsT0 = 256;         // first thread of the normal-matrix column sums in B_1

template <int RAD, int K, int BW, int CH>
struct StreamGeom {
    static constexpr int RW = BW + 2 * K * RAD;  // region columns
    static constexpr int JW = RW + 2 * kMX + 2;  // target box columns
    static constexpr int PR = CH + 2 * RAD;      // rows of the product buffer
    static_assert(CH >= 2 * RAD, "chunk must cover the column-sum history");
    static_assert(CH + (K + 1) * RAD <= kRing, "row ring too small");
    static_assert((K - 1) * RAD + CH + 2 * kMY + 2 <= kRing, "target ring too small");
    static constexpr size_t kT = 0;
    static constexpr size_t kG = kT + sizeof(float) * kRing * RW;
    static constexpr size_t kU = kG + sizeof(float2) * kRing * RW;
    static constexpr size_t kGiA = kU + sizeof(float2) * kRing * RW;
    static constexpr size_t kGiB = kGiA + sizeof(float2) * kRing * RW;
    static constexpr size_t kJ = kGiB + sizeof(float) * kRing * RW;
    static constexpr size_t kP = kJ + sizeof(float) * kRing * JW;
    static constexpr size_t kH = kP + sizeof(float2) * PR * RW;
    // sV, sCSA and sCSB are padded by kPad elements on both sides: the row
    // sums of the column pair at a stage's edge read a window of up to
    // kPad elements beyond the first or last column (values of pixels the
    // stage does not update, never used), which then stays in the array
    static constexpr int kPad = 4;
    static constexpr size_t kV = kH + sizeof(float2) * K * 2 * RAD * RW + sizeof(float2) * kPad;
    static constexpr size_t kCSA = kV + sizeof(float2) * (CH * RW + kPad) + sizeof(float2) * kPad;
    static constexpr size_t kCSB = kCSA + sizeof(float2) * (CH * RW + kPad) + sizeof(float) * kPad;
    // next chunk's template rows (with a 1-pixel ring) and coarse flow rows
    static constexpr int TSW = RW + 2, TSH = CH + 2;
    static constexpr int FSW = RW / 2 + 3, FSH = CH / 2 + 3;
    static constexpr size_t kTS = kCSB + sizeof(float) * (CH * RW + kPad);
    static constexpr size_t kFS = (kTS + sizeof(float) * TSH * TSW + 7) / 8 * 8;
    static constexpr size_t bytes = kFS + sizeof(float2) * FSH * FSW;
};

__device__ __forceinline__ int ring_slot(int y) { return (y + kRingOff) & (kRing - 1); }

// Paired FP32 arithmetic (one instruction for the two lanes of a float2;
// each lane rounds exactly as the scalar operation would).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ void copy_async4(void* dst_smem, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void copy_async8(void* dst_smem, const void* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void copy_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void copy_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ float2 start_flow_s(const LkArgs& a, const LkDir& D, int x, int y) {
    if (a.mode == 0 || D.uin == nullptr) return make_float2(0.f, 0.f);
    const float2* __restrict__ u = reinterpret_cast<const float2*>(D.uin);
    if (a.mode == 2) return u[(long long)y * D.uin_pitch + x];
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

// What every stage needs to sample J around pixel q.
template <class Ts>
struct TargetBox {
    const float* sJ;   // ring of staged target rows
    const Ts* J;       // global target plane (fallback)
    int pitchJ, w, h;
    int fref_x, fref_y;  // integer part of the reference flow
};

// J(q + ref + u) with clamp-to-edge taps: from the staged box when all four
// taps lie in it, else from global memory. Both paths read the same values.
template <int JW, class Ts>
__device__ __forceinline__ float sample_target(const TargetBox<Ts>& b, int x, int y, int rx, float2 ref, float2 u) {
    const float2 o = add2(ref, u);
    const float ox = o.x, oy = o.y;
    // floor(o) through the FP adder: o + 1.5 * 2^23 rounded down holds floor(o)
    // in its low mantissa bits while |o| < 2^22; larger or non-finite offsets
    // give integer parts far outside the box and take the global path
    const float tx = __fadd_rd(ox, 12582912.0f), ty = __fadd_rd(oy, 12582912.0f);
    const float fx = tx - 12582912.0f, fy = ty - 12582912.0f;
    const unsigned uix = __float_as_uint(tx) - 0x4B400000u, uiy = __float_as_uint(ty) - 0x4B400000u;
    const int ix = (int)uix, iy = (int)uiy;
    const unsigned bcol_u = (unsigned)rx + uix - (unsigned)b.fref_x + (unsigned)kMX;
    const int bcol = (int)bcol_u;
    if (bcol_u < (unsigned)(JW - 1) && uiy - (unsigned)(b.fref_y - kMY) <= (unsigned)(2 * kMY)) {
        Taps t;
        t.ax = ox - fx;
        t.ay = oy - fy;
        const int o0 = ring_slot(y + iy) * JW + bcol, o1 = ring_slot(y + iy + 1) * JW + bcol;
        constexpr int NJ = kRing * JW;
        return bilinear_mix(t, PANO_AT(b.sJ, o0, NJ, 101), PANO_AT(b.sJ, o0 + 1, NJ, 102), PANO_AT(b.sJ, o1, NJ, 103),
                            PANO_AT(b.sJ, o1 + 1, NJ, 104));
    }
    // outside the staged box (large or non-finite offsets): clamped global taps
    return sample_plane(b.J, b.pitchJ, b.w, b.h, x, y, ox, oy);
}

// Residual product of one sample q at flow u (relative to ref).
template <int JW, class Ts>
__device__ __forceinline__ float2 residual_product(const TargetBox<Ts>& b, int x, int y, int rx, float2 ref,
                                                   float2 u, float2 g, float t) {
    const float Jw = sample_target<JW, Ts>(b, x, y, rx, ref, u);
    const float s = fmaf(g.x, u.x, fmaf(g.y, u.y, t - Jw));
    return mul2(g, make_float2(s, s));
}

// Column sums over 2R+1 rows of the product buffer for the output rows
// [part * CH / S, (part + 1) * CH / S) of one column: the CH / S + 2R values
// are read once into registers and every output row is summed directly from
// them (no running sums, which would carry rounding from one row into the
// next). The part with the last rows also saves the last 2R product rows as
// the history of this stage for the next chunk.
template <int RAD, int CH, int RW, int S>
__device__ __forceinline__ void column_sums(const float2* __restrict__ sP, float2* __restrict__ sV,
                                            float2* __restrict__ hist, int rx, int part) {
    static_assert(CH % S == 0, "parts must split the chunk rows evenly");
    constexpr int HC = CH / S;
    const int r0 = part * HC;
    float2 p[HC + 2 * RAD];
#pragma unroll
    for (int d = 0; d < HC + 2 * RAD; ++d) p[d] = PANO_AT(sP, (r0 + d) * RW + rx, (CH + 2 * RAD) * RW, 105);
#pragma unroll
    for (int yy = 0; yy < HC; ++yy) {
        float2 v = p[yy];
#pragma unroll
        for (int d = 1; d <= 2 * RAD; ++d) v = add2(v, p[yy + d]);
        PANO_AT(sV, (r0 + yy) * RW + rx, CH * RW, 106) = v;
    }
    if (part == S - 1) {
#pragma unroll
        for (int d = 0; d < 2 * RAD; ++d) PANO_AT(hist, d * RW + rx, 2 * RAD * RW, 107) = p[HC + d];
    }
}

// One work item: direction `dir`, band `bx` (BW output columns) and segment
// `by` (rows [by * seg, by * seg + seg)) of the level described by `a`.
template <int RAD, int K, int BW, int CH, class Ts>
__device__ __forceinline__ void lk_stream_item(const LkArgs& a, int dir, int bx, int by, int seg,
                                               unsigned char* smem) {
    constexpr bool kAsyncT = std::is_same<Ts, float>::value;  // cp.async of 4-byte elements
    using Geo = StreamGeom<RAD, K, BW, CH>;
    constexpr int RW = Geo::RW;
    constexpr int JW = Geo::JW;
    // Thread layout: thread (ty, tx) works on row ty of every chunk-sized
    // block of rows and on the columns tx, tx + TX, tx + 2 TX, ...
    constexpr int TX = kStreamThreads / CH;
    static_assert(TX * CH == kStreamThreads, "threads must tile the chunk rows");
    constexpr int kJPT = (Geo::JW + TX - 1) / TX;  // target-row elements per thread (16-bit planes)
    float jnext[kJPT];
    (void)jnext;
    static_assert(2 * RW <= kCsT0 && kCsT0 + 2 * RW <= kStreamThreads && CH % 2 == 0, "B_1 thread groups");
    float* sT = reinterpret_cast<float*>(smem + Geo::kT);
    float2* sG = reinterpret_cast<float2*>(smem + Geo::kG);
    float2* sU = reinterpret_cast<float2*>(smem + Geo::kU);
    float2* sGiA = reinterpret_cast<float2*>(smem + Geo::kGiA);  // (i11, i12)
    float* sGiB = reinterpret_cast<float*>(smem + Geo::kGiB);    // i22
    float* sJ = reinterpret_cast<float*>(smem + Geo::kJ);
    float2* sP = reinterpret_cast<float2*>(smem + Geo::kP);
    float2* sH = reinterpret_cast<float2*>(smem + Geo::kH);
    float2* sV = reinterpret_cast<float2*>(smem + Geo::kV);
    float2* sCSA = reinterpret_cast<float2*>(smem + Geo::kCSA);  // (c11, c12)
    float* sCSB = reinterpret_cast<float*>(smem + Geo::kCSB);    // c22
    float* sTS = reinterpret_cast<float*>(smem + Geo::kTS);      // staged template rows
    float2* sFS = reinterpret_cast<float2*>(smem + Geo::kFS);    // staged coarse flow rows
    constexpr int TSW = Geo::TSW, TSH = Geo::TSH, FSW = Geo::FSW, FSH = Geo::FSH;
    // element counts of the shared arrays (for the debug build's index checks)
    constexpr int NR = kRing * RW, NJ = kRing * JW, NP = (CH + 2 * RAD) * RW, NHIST = K * 2 * RAD * RW;
    constexpr int NCH = CH * RW, NTS = TSH * TSW, NFS = FSH * FSW;
    (void)NR, (void)NJ, (void)NP, (void)NHIST, (void)NCH, (void)NTS, (void)NFS;

    const LkDir D = dir ? a.dir[1] : a.dir[0];
    const int w = a.w, h = a.h;
    const float lam = a.lambda;
    const Ts* __restrict__ T = static_cast<const Ts*>(D.T);
    const int pitchT = D.pitchT;
    const int X0 = bx * BW;
    const int ox = X0 - K * RAD;
    const int Y0 = by * seg;
    const int Y1 = min(h, Y0 + seg);
    const int tid = threadIdx.x;
    const int ty = tid / TX, tx = tid - ty * TX;
    // region columns that lie inside the image: [cmin, cmax)
    const int cmin = max(0, -ox), cmax = min(RW, w - ox);

    // reference flow: starting flow at the centre of the band and segment
    const float2 ref = start_flow_s(a, D, min(X0 + BW / 2, w - 1), min((Y0 + Y1) / 2, h - 1));
    TargetBox<Ts> box;
    box.sJ = sJ;
    box.J = static_cast<const Ts*>(D.J);
    box.pitchJ = D.pitchJ;
    box.w = w;
    box.h = h;
    box.fref_x = (int)floorf(fminf(fmaxf(ref.x, -(float)(w + 2)), (float)(w + 2)));
    box.fref_y = (int)floorf(fminf(fmaxf(ref.y, -(float)(h + 2)), (float)(h + 2)));
    const int jx0 = ox + box.fref_x - kMX;  // image column of box column 0

    const bool stage_flow = a.mode == 1 && D.uin != nullptr;
    const float2* __restrict__ ucoarse = reinterpret_cast<const float2*>(D.uin);
    // Asynchronous copies of what X_0 of the chunk with newest rows
    // [a0n, a0n + CH) reads from global memory: template rows a0n-1 .. a0n+CH
    // (columns ox-1 .. ox+RW, clamp-to-edge) and, when the level starts from
    // the coarser level, the coarse flow rows and columns its upsampling taps.
    // Staged by nw workers, this thread being worker wi.
    auto stage_inputs = [&](int a0n, int wi, int nw) {
        for (int i = wi; i < TSH * TSW; i += nw) {
            const int r = i / TSW, cc = i - r * TSW;
            const int ys = min(max(a0n - 1 + r, 0), h - 1), xs = min(max(ox - 1 + cc, 0), w - 1);
            const Ts* src = &PANO_AT(T, (long long)ys * pitchT + xs, (long long)h * pitchT, 110);
            if constexpr (kAsyncT) copy_async4(&PANO_AT(sTS, i, NTS, 111), src);
            else PANO_AT(sTS, i, NTS, 111) = ld_f32(src);
        }
        if (stage_flow) {
            const int cy0 = a0n >> 1, cx0 = ox >> 1;
            for (int i = wi; i < FSH * FSW; i += nw) {
                const int r = i / FSW, cc = i - r * FSW;
                const int ys = min(max(cy0 + r, 0), a.in_h - 1), xs = min(max(cx0 + cc, 0), a.in_w - 1);
                copy_async8(&PANO_AT(sFS, i, NFS, 112),
                            &PANO_AT(ucoarse, (long long)ys * D.uin_pitch + xs, (long long)a.in_h * D.uin_pitch, 113));
            }
        }
        copy_async_commit();
    };

    const int c_first = -((2 * K * RAD + CH - 1) / CH);
    const int c_last = (Y1 - Y0 + CH - 1) / CH - 1;
    stage_inputs(Y0 + K * RAD + c_first * CH, tid, kStreamThreads);
    // Rings start at zero: the column sums of the first chunk read ring rows
    // that no earlier chunk wrote (their results are discarded, but must
    // stay finite).
    for (int i = tid; i < K * 2 * RAD * RW; i += kStreamThreads) PANO_AT(sH, i, NHIST, 114) = make_float2(0.f, 0.f);
    for (int i = tid; i < kRing * RW; i += kStreamThreads) {
        PANO_AT(sT, i, NR, 115) = 0.f;
        PANO_AT(sG, i, NR, 116) = make_float2(0.f, 0.f);
        PANO_AT(sU, i, NR, 117) = make_float2(0.f, 0.f);
    }
    {
        // target rows of the first chunk
        const int a0f = Y0 + K * RAD + c_first * CH;
        const int yb = a0f - (K - 1) * RAD + box.fref_y - kMY;
        const int n = ((K - 1) * RAD + CH + 2 * kMY + 1) * JW;
        for (int i = tid; i < n; i += kStreamThreads) {
            const int yy = i / JW, bc = i - yy * JW;
            const int yj = yb + yy;
            const int ys = min(max(yj, 0), h - 1), xs = min(max(jx0 + bc, 0), w - 1);
            PANO_AT(sJ, ring_slot(yj) * JW + bc, NJ, 118) =
                ld_f32(&PANO_AT(box.J, (long long)ys * box.pitchJ + xs, (long long)h * box.pitchJ, 119));
        }
    }
    copy_async_wait_all();
    __syncthreads();

    for (int c = c_first; c <= c_last; ++c) {
        const int a0 = Y0 + K * RAD + c * CH;  // newest rows [a0, a0 + CH)
        // ---- X_0: state of the new rows and the products of stage 1
        for (int i = tid; i < 2 * RAD * RW; i += kStreamThreads) PANO_AT(sP, i, NP, 120) = PANO_AT(sH, i, NHIST, 121);
        {
            const int y = a0 + ty;
            const bool row_in = y >= 0 && y < h;
            const int srow = ring_slot(y) * RW;
            const int tso = (ty + 1) * TSW + 1;  // staged row of y: column rx at sTS[tso + rx]
            const int cy0 = a0 >> 1, cx0 = ox >> 1;
            const int fr0 = (y >> 1) - cy0;               // staged coarse row of y / 2
            const float fy = (y & 1) ? 0.5f : 0.f;
            const int pro = (2 * RAD + ty) * RW;  // this row's products at sP[pro + rx]
            for (int rx = tx; rx < RW; rx += TX) {
                const int x = ox + rx;
                float t = 0.f;
                float2 g = make_float2(0.f, 0.f), u = make_float2(0.f, 0.f), P = make_float2(0.f, 0.f);
                if (row_in && rx >= cmin && rx < cmax) {
                    t = PANO_AT(sTS, tso + rx, NTS, 122);
                    g.x = 0.5f * (PANO_AT(sTS, tso + rx + 1, NTS, 123) - PANO_AT(sTS, tso + rx - 1, NTS, 124));
                    g.y = 0.5f * (PANO_AT(sTS, tso + rx + TSW, NTS, 125) - PANO_AT(sTS, tso + rx - TSW, NTS, 126));
                    float2 u0;
                    if (stage_flow) {
                        // 2 * bilinear(u_coarse)(x/2, y/2) from the staged rows
                        const int fc0 = (x >> 1) - cx0;
                        const float fx = (x & 1) ? 0.5f : 0.f;
                        const int f0 = fr0 * FSW + fc0, f1 = f0 + FSW;
                        const float2 u00 = PANO_AT(sFS, f0, NFS, 127), u10 = PANO_AT(sFS, f0 + 1, NFS, 128);
                        const float2 u01 = PANO_AT(sFS, f1, NFS, 129), u11 = PANO_AT(sFS, f1 + 1, NFS, 130);
                        const float tx0 = fmaf(fx, u10.x - u00.x, u00.x), bx0 = fmaf(fx, u11.x - u01.x, u01.x);
                        const float ty0 = fmaf(fx, u10.y - u00.y, u00.y), by0 = fmaf(fx, u11.y - u01.y, u01.y);
                        u0 = make_float2(2.f * fmaf(fy, bx0 - tx0, tx0), 2.f * fmaf(fy, by0 - ty0, ty0));
                    } else {
                        u0 = start_flow_s(a, D, x, y);
                    }
                    u = make_float2(u0.x - ref.x, u0.y - ref.y);
                    P = residual_product<JW, Ts>(box, x, y, rx, ref, u, g, t);
                }
                PANO_AT(sT, srow + rx, NR, 131) = t;
                PANO_AT(sG, srow + rx, NR, 132) = g;
                PANO_AT(sU, srow + rx, NR, 133) = u;
                PANO_AT(sP, pro + rx, NP, 134) = P;
            }
        }
        __syncthreads();
        // the staging buffers are free again: every thread starts fetching
        // part of the next chunk's inputs
        if (c < c_last) stage_inputs(a0 + CH, tid, kStreamThreads);
        // ---- B_1: column sums of stage 1 (two threads per column, the
        //      column's values read once into registers) and its history;
        //      column sums of grad T grad T^T for the normal matrices of rows
        //      [a1, a1 + CH)
        if (tid < 2 * RW) {
            const int part = tid >= RW;
            column_sums<RAD, CH, RW, 2>(sP, sV, sH, tid - part * RW, part);
        } else if (tid >= kCsT0 && tid < kCsT0 + 2 * RW) {
            // normal-matrix column sums: two threads per column, CH/2 rows each
            const int rx = (tid - kCsT0) % RW, half = (tid - kCsT0) / RW;
            constexpr int HC = CH / 2;
            const int yb = a0 - 2 * RAD + half * HC;   // first ring row of this half's windows
            float2 g[HC + 2 * RAD];
#pragma unroll
            for (int d = 0; d < HC + 2 * RAD; ++d) g[d] = PANO_AT(sG, ring_slot(yb + d) * RW + rx, NR, 135);
#pragma unroll
            for (int yy = 0; yy < HC; ++yy) {
                float2 c1 = make_float2(0.f, 0.f);  // (c11, c12)
                float c22 = 0.f;
#pragma unroll
                for (int d = 0; d <= 2 * RAD; ++d) {
                    c1 = fma2(make_float2(g[yy + d].x, g[yy + d].x), g[yy + d], c1);
                    c22 = fmaf(g[yy + d].y, g[yy + d].y, c22);
                }
                const int o = (half * HC + yy) * RW + rx;
                PANO_AT(sCSA, o, NCH, 136) = c1;
                PANO_AT(sCSB, o, NCH, 137) = c22;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 1; k <= K; ++k) {
            const int c0 = k * RAD;            // columns [c0, RW - c0)
            if (k == K) {
                // target rows that the next chunk's products reach for the
                // first time: asynchronous copies, issued first so that they
                // overlap this phase (no products are sampled in it)
                const int yj = a0 + CH + box.fref_y + kMY + 1 + ty;
                const long long jso = (long long)min(max(yj, 0), h - 1) * box.pitchJ;  // source row
                const long long NJG = (long long)h * box.pitchJ;
                (void)NJG;
                if constexpr (kAsyncT) {
                    const int jdo = ring_slot(yj) * JW;
                    for (int bc = tx; bc < JW; bc += TX)
                        copy_async4(&PANO_AT(sJ, jdo + bc, NJ, 138),
                                    &PANO_AT(box.J, jso + min(max(jx0 + bc, 0), w - 1), NJG, 139));
                    copy_async_commit();
                } else {
#pragma unroll
                    for (int q = 0; q < kJPT; ++q) {
                        const int bc = tx + q * TX;
                        jnext[q] = bc < JW ? ld_f32(&PANO_AT(box.J, jso + min(max(jx0 + bc, 0), w - 1), NJG, 139)) : 0.f;
                    }
                }
            }
            // ---- X_k: row sums, solve, update; products of stage k+1
            if (k < K) {
                const int hko = k * 2 * RAD * RW;  // this stage's history in sH
                const int width = RW - 2 * c0;
                for (int i = tid; i < 2 * RAD * width; i += kStreamThreads) {
                    const int yy = i / width, rx = c0 + (i - yy * width);
                    PANO_AT(sP, yy * RW + rx, NP, 140) = PANO_AT(sH, hko + yy * RW + rx, NHIST, 141);
                }
            }
            {
                // this thread: row ty of stage k, the column pair (xp, xp + 1)
                constexpr int HR = (RAD + 1) / 2 * 2;      // even halo >= RAD
                constexpr int NPAIR = (2 * HR + 2) / 2;     // float4 loads for the row sums
                const int c0e = c0 & ~1;
                const int xp = c0e + 2 * tx;
                const int y = a0 - k * RAD + ty;
                const bool row_in = y >= 0 && y < h;
                const bool on0 = xp >= c0 && xp < RW - c0, on1 = xp + 1 >= c0 && xp + 1 < RW - c0;
                if (xp < RW - c0) {
                    const int srow = ring_slot(y) * RW;
                    const bool in0 = on0 && row_in && xp >= cmin && xp < cmax;
                    const bool in1 = on1 && row_in && xp + 1 >= cmin && xp + 1 < cmax;
                    // row sums of the column sums for both pixels
                    const int vqo = ty * RW + xp - HR;  // first column pair at sV[vqo]
                    float2 vv[2 * HR + 2];
#pragma unroll
                    for (int q = 0; q < NPAIR; ++q) {
                        const float4 t4 = PANO_VEC(const float4, sV - Geo::kPad, vqo + 2 * q + Geo::kPad, 2,
                                                   NCH + 2 * Geo::kPad, 142);
                        vv[2 * q] = make_float2(t4.x, t4.y);
                        vv[2 * q + 1] = make_float2(t4.z, t4.w);
                    }
                    float2 m0 = vv[HR - RAD], m1 = vv[HR - RAD + 1];
#pragma unroll
                    for (int d = 1; d <= 2 * RAD; ++d) {
                        m0 = add2(m0, vv[HR - RAD + d]);
                        m1 = add2(m1, vv[HR - RAD + d + 1]);
                    }
                    float2 ga0, ga1;
                    float gb0, gb1;
                    if (k == 1) {
                        const int co = ty * RW + xp;  // column sums of column xp at sCSA[co], sCSB[co]
                        float2 a1 = make_float2(0.f, 0.f), b1 = make_float2(0.f, 0.f);  // (x11, x12)
                        float a22 = 0.f, b22 = 0.f;
#pragma unroll
                        for (int d = -RAD; d <= RAD; ++d) {
                            constexpr int NCP = NCH + 2 * Geo::kPad, PD = Geo::kPad;
                            a1 = add2(a1, PANO_AT(sCSA - PD, co + d + PD, NCP, 143));
                            a22 += PANO_AT(sCSB - PD, co + d + PD, NCP, 144);
                            b1 = add2(b1, PANO_AT(sCSA - PD, co + d + 1 + PD, NCP, 145));
                            b22 += PANO_AT(sCSB - PD, co + d + 1 + PD, NCP, 146);
                        }
                        const float a11 = a1.x, a12 = a1.y, b11 = b1.x, b12 = b1.y;
                        const float p11 = a11 + lam, p22 = a22 + lam;
                        const float ip = 1.0f / (p11 * p22 - a12 * a12);
                        const float q11 = b11 + lam, q22 = b22 + lam;
                        const float iq = 1.0f / (q11 * q22 - b12 * b12);
                        ga0 = make_float2(p22 * ip, -a12 * ip);
                        gb0 = p11 * ip;
                        ga1 = make_float2(q22 * iq, -b12 * iq);
                        gb1 = q11 * iq;
                        PANO_VEC(float4, sGiA, srow + xp, 2, NR, 147) = make_float4(ga0.x, ga0.y, ga1.x, ga1.y);
                        PANO_VEC(float2, sGiB, srow + xp, 2, NR, 148) = make_float2(gb0, gb1);
                    } else {
                        const float4 a4 = PANO_VEC(const float4, sGiA, srow + xp, 2, NR, 149);
                        const float2 b2 = PANO_VEC(const float2, sGiB, srow + xp, 2, NR, 150);
                        ga0 = make_float2(a4.x, a4.y);
                        ga1 = make_float2(a4.z, a4.w);
                        gb0 = b2.x;
                        gb1 = b2.y;
                    }
                    const float4 u4 = PANO_VEC(const float4, sU, srow + xp, 2, NR, 151);
                    float2 v0 = make_float2(u4.x, u4.y), v1 = make_float2(u4.z, u4.w);
                    const float2 lam2 = make_float2(lam, lam);
                    if (in0) {
                        const float2 r = fma2(lam2, v0, m0);
                        v0 = fma2(ga0, make_float2(r.x, r.x), mul2(make_float2(ga0.y, gb0), make_float2(r.y, r.y)));
                    }
                    if (in1) {
                        const float2 r = fma2(lam2, v1, m1);
                        v1 = fma2(ga1, make_float2(r.x, r.x), mul2(make_float2(ga1.y, gb1), make_float2(r.y, r.y)));
                    }
                    PANO_VEC(float4, sU, srow + xp, 2, NR, 152) = make_float4(v0.x, v0.y, v1.x, v1.y);
                    if (k == K) {
                        if (row_in && y >= Y0 && y < Y1) {
                            float2* uo = reinterpret_cast<float2*>(D.uout);
                            const long long uoo = (long long)y * D.uout_pitch + ox + xp;
                            const long long NUO = (long long)h * D.uout_pitch;
                            (void)NUO;
                            if (in0 && xp >= K * RAD && xp < K * RAD + BW) PANO_AT(uo, uoo, NUO, 153) = add2(v0, ref);
                            if (in1 && xp + 1 >= K * RAD && xp + 1 < K * RAD + BW)
                                PANO_AT(uo, uoo + 1, NUO, 154) = add2(v1, ref);
                        }
                    } else {
                        // products of stage k+1 at the same two pixels
                        const float4 g4 = PANO_VEC(const float4, sG, srow + xp, 2, NR, 155);
                        const float2 t2 = PANO_VEC(const float2, sT, srow + xp, 2, NR, 156);
                        float2 P0 = make_float2(0.f, 0.f), P1 = make_float2(0.f, 0.f);
                        if (in0) P0 = residual_product<JW, Ts>(box, ox + xp, y, xp, ref, v0, make_float2(g4.x, g4.y), t2.x);
                        if (in1) P1 = residual_product<JW, Ts>(box, ox + xp + 1, y, xp + 1, ref, v1, make_float2(g4.z, g4.w), t2.y);
                        PANO_VEC(float4, sP, (2 * RAD + ty) * RW + xp, 2, NP, 157) = make_float4(P0.x, P0.y, P1.x, P1.y);
                    }
                }
            }
            if (k == K) {
                // the coarse-flow rows (and for float planes the template and
                // target rows) copied asynchronously since B_1
                copy_async_wait_all();
                if constexpr (!kAsyncT) {
                    // the target loads issued before X_K land in the ring now
                    const int yj = a0 + CH + box.fref_y + kMY + 1 + ty;
                    const int jdo = ring_slot(yj) * JW;
#pragma unroll
                    for (int q = 0; q < kJPT; ++q) {
                        const int bc = tx + q * TX;
                        if (bc < JW) PANO_AT(sJ, jdo + bc, NJ, 158) = jnext[q];
                    }
                }
            }
            __syncthreads();
            if (k < K) {
                // ---- B_{k+1}: column sums of stage k+1 and its history (two
                //      threads per column)
                const int ncol = RW - 2 * c0;
                if (tid < 2 * ncol) {
                    const int part = tid >= ncol;
                    column_sums<RAD, CH, RW, 2>(sP, sV, sH + (size_t)k * 2 * RAD * RW, c0 + tid - part * ncol, part);
                }
                __syncthreads();
            }
        }
    }
}

template <int RAD, int K, int BW, int CH, class Ts>
__global__ void __launch_bounds__(kStreamThreads, 1) lk_stream_kernel(const __grid_constant__ LkArgs a, int seg) {
    extern __shared__ __align__(16) unsigned char smem[];
    lk_stream_item<RAD, K, BW, CH, Ts>(a, blockIdx.z, blockIdx.x, blockIdx.y, seg, smem);
}

// Persistent form over several strip pairs at once: a fixed grid of CTAs
// takes (pair, direction, band, segment) items from an atomic counter until
// none are left. The counter only hands out indices; nothing waits on it.
template <int RAD, int K, int BW, int CH, class Ts>
__global__ void __launch_bounds__(kStreamThreads, 1) lk_stream_batch_kernel(const __grid_constant__ LkBatch b) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int)atomicAdd(b.counter, 1u);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= b.start[b.n]) break;
        int p = 0;
        while (p + 1 < b.n && item >= b.start[p + 1]) ++p;
        const int local = item - b.start[p];
        const int per_dir = b.nb[p] * b.nseg[p];
        const int dir = local / per_dir, rem = local - dir * per_dir;
        const int by = rem / b.nb[p], bx = rem - by * b.nb[p];
        lk_stream_item<RAD, K, BW, CH, Ts>(b.pair[p], dir, bx, by, b.seg[p], smem);
        __syncthreads();
    }
}

// Segment height and count for one level: about 256+ rows per segment (the
// first chunks of a segment are discarded work), in whole waves of one CTA
// per SM; seg_rows > 0 overrides the target height. (On the 4000 x 1500
// pair's level 0 that is 3 waves of 286-row segments; 4 waves of 211 rows
// measured 0.8% slower for the step, 2 waves of 445 rows 1.6% slower.)
template <int CH>
void stream_segments(int h, int per_row, int seg_rows, int* seg_out, int* nseg_out) {
    const int sms = 152;
    int seg;
    if (seg_rows > 0) {
        seg = seg_rows;
    } else {
        long long waves = (long long)per_row * h / (256LL * sms);
        if (waves < 1) waves = 1;
        int nseg = (int)(waves * sms / per_row);
        if (nseg < 1) nseg = 1;
        seg = (h + nseg - 1) / nseg;
    }
    if (seg < 2 * CH) seg = 2 * CH;
    *seg_out = seg;
    *nseg_out = (h + seg - 1) / seg;
}

template <int RAD, int K, int BW, int CH, class Ts>
cudaError_t launch_one(const LkArgs& a, int ndirs, cudaStream_t s) {
    using Geo = StreamGeom<RAD, K, BW, CH>;
    const int nb = (a.w + BW - 1) / BW;
    int seg = 0, nseg = 0;
    stream_segments<CH>(a.h, nb * ndirs, a.seg_rows, &seg, &nseg);
    dim3 grid(nb, nseg, ndirs);
    lk_stream_kernel<RAD, K, BW, CH, Ts><<<grid, kStreamThreads, Geo::bytes, s>>>(a, seg);
    return cudaGetLastError();
}

template <int RAD, int K, int BW, int CH, class Ts>
cudaError_t prepare_one(int max_smem) {
    using Geo = StreamGeom<RAD, K, BW, CH>;
    if (Geo::bytes > (size_t)max_smem) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(lk_stream_kernel<RAD, K, BW, CH, Ts>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Geo::bytes);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(lk_stream_batch_kernel<RAD, K, BW, CH, Ts>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Geo::bytes);
}

constexpr int kBW = 96;

template <int RAD>
struct RadCfg;
template <>
struct RadCfg<1> { static constexpr int CH = 12; };
template <>
struct RadCfg<2> { static constexpr int CH = 12; };
template <>
struct RadCfg<3> { static constexpr int CH = 8; };

template <int RAD, int K, int BW, int CH, class Ts>
cudaError_t launch_batch_one(LkBatch b, int n_ctas, cudaStream_t s) {
    using Geo = StreamGeom<RAD, K, BW, CH>;
    b.start[0] = 0;
    for (int p = 0; p < b.n; ++p) {
        b.nb[p] = (b.pair[p].w + BW - 1) / BW;
        stream_segments<CH>(b.pair[p].h, b.nb[p] * 2, b.pair[p].seg_rows, &b.seg[p], &b.nseg[p]);
        b.start[p + 1] = b.start[p] + 2 * b.nb[p] * b.nseg[p];
    }
    int grid = n_ctas > 0 ? n_ctas : 152;
    if (grid > b.start[b.n]) grid = b.start[b.n];
    cudaError_t e = cudaMemsetAsync(b.counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    lk_stream_batch_kernel<RAD, K, BW, CH, Ts><<<grid, kStreamThreads, Geo::bytes, s>>>(b);
    return cudaGetLastError();
}

template <int RAD, class Ts>
cudaError_t launch_rad_batch(const LkBatch& b, int n_ctas, cudaStream_t s) {
    constexpr int CH = RadCfg<RAD>::CH;
    switch (b.pair[0].iters) {
        case 1: return launch_batch_one<RAD, 1, kBW, CH, Ts>(b, n_ctas, s);
        case 2: return launch_batch_one<RAD, 2, kBW, CH, Ts>(b, n_ctas, s);
        case 3: return launch_batch_one<RAD, 3, kBW, CH, Ts>(b, n_ctas, s);
        case 4: return launch_batch_one<RAD, 4, kBW, CH, Ts>(b, n_ctas, s);
        case 5: return launch_batch_one<RAD, 5, kBW, CH, Ts>(b, n_ctas, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int RAD, class Ts>
cudaError_t launch_rad_stream(const LkArgs& a, int ndirs, cudaStream_t s) {
    constexpr int CH = RadCfg<RAD>::CH;
    switch (a.iters) {
        case 1: return launch_one<RAD, 1, kBW, CH, Ts>(a, ndirs, s);
        case 2: return launch_one<RAD, 2, kBW, CH, Ts>(a, ndirs, s);
        case 3: return launch_one<RAD, 3, kBW, CH, Ts>(a, ndirs, s);
        case 4: return launch_one<RAD, 4, kBW, CH, Ts>(a, ndirs, s);
        case 5: return launch_one<RAD, 5, kBW, CH, Ts>(a, ndirs, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int RAD, class Ts>
cudaError_t prepare_rad_stream(int max_smem) {
    constexpr int CH = RadCfg<RAD>::CH;
    cudaError_t e;
    if ((e = prepare_one<RAD, 1, kBW, CH, Ts>(max_smem)) != cudaSuccess) return e;
    if ((e = prepare_one<RAD, 2, kBW, CH, Ts>(max_smem)) != cudaSuccess) return e;
    if ((e = prepare_one<RAD, 3, kBW, CH, Ts>(max_smem)) != cudaSuccess) return e;
    if ((e = prepare_one<RAD, 4, kBW, CH, Ts>(max_smem)) != cudaSuccess) return e;
    return prepare_one<RAD, 5, kBW, CH, Ts>(max_smem);
}

// Entry points for one storage type (instantiated by exactly one .cu file).
template <class Ts>
cudaError_t stream_launch(const LkArgs& a, int ndirs, cudaStream_t s) {
    switch (a.radius) {
        case 1: return launch_rad_stream<1, Ts>(a, ndirs, s);
        case 2: return launch_rad_stream<2, Ts>(a, ndirs, s);
        case 3: return launch_rad_stream<3, Ts>(a, ndirs, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class Ts>
cudaError_t stream_launch_batch(const LkBatch& b, int n_ctas, cudaStream_t s) {
    switch (b.pair[0].radius) {
        case 1: return launch_rad_batch<1, Ts>(b, n_ctas, s);
        case 2: return launch_rad_batch<2, Ts>(b, n_ctas, s);
        case 3: return launch_rad_batch<3, Ts>(b, n_ctas, s);
        default: return cudaErrorInvalidValue;
    }
}

template <class Ts>
cudaError_t stream_prepare(int max_smem_bytes) {
    cudaError_t e;
    if ((e = prepare_rad_stream<1, Ts>(max_smem_bytes)) != cudaSuccess) return e;
    if ((e = prepare_rad_stream<2, Ts>(max_smem_bytes)) != cudaSuccess) return e;
    return prepare_rad_stream<3, Ts>(max_smem_bytes);
}

#define PANO_LKS_INSTANTIATE(Ts)                                                          \
    template cudaError_t stream_launch<Ts>(const LkArgs&, int, cudaStream_t);            \
    template cudaError_t stream_launch_batch<Ts>(const LkBatch&, int, cudaStream_t);     \
    template cudaError_t stream_prepare<Ts>(int);

#define PANO_LKS_EXTERN(Ts)                                                                  \
    extern template cudaError_t stream_launch<Ts>(const LkArgs&, int, cudaStream_t);        \
    extern template cudaError_t stream_launch_batch<Ts>(const LkBatch&, int, cudaStream_t); \
    extern template cudaError_t stream_prepare<Ts>(int);

}  // namespace lks
}  // namespace pano
