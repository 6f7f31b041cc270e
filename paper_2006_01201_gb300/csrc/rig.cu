// rig.cu -- the C ABI of include/pano_rig.h: all overlap pairs of a
// 360-degree rig (Section III: the panorama is stitched from the pairs of
// adjacent cameras) through the flow-blend path of Section III-C in a fixed
// sequence of batched launches, optionally replayed from a CUDA graph, with
// per-level kernel tuning measured on the device.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <new>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "pano_flow.h"
#include "pano_rig.h"

using namespace pano;

namespace {

// What a captured graph depends on: every pointer and pitch of the call and
// the tuning generation.
struct GraphKey {
    const void* L[kMaxBatch];
    const void* R[kMaxBatch];
    size_t Lp[kMaxBatch], Rp[kMaxBatch];
    float* lr[kMaxBatch];
    float* rl[kMaxBatch];
    void* canvas;
    size_t canvas_pitch;
    unsigned long long tune_gen;
};

// A captured graph and what it was captured for.
struct GraphSlot {
    GraphKey key;
    cudaGraphExec_t exec;
    int kernels;
    unsigned long long last_use;
};
constexpr int kGraphSlots = 4;  // e.g. the buffer sets of a double-buffered pipeline

struct RunCall {
    const pano_image* L;
    const pano_image* R;
    float* lr[kMaxBatch];
    float* rl[kMaxBatch];
    const pano_image* canvas;
};

}  // namespace

struct pano_rig {
    pano_flow_params p;
    pano_rig_desc d;
    int device;
    int nlev;
    int max_smem;
    int n_ctas;                    // persistent grid of the streamed kernel
    int def_tile_w, def_tile_h;    // default tile of the tiled kernel
    int hs[kMaxLevels];            // level heights (shared by all pairs)
    int ws[kMaxBatch][kMaxLevels]; // level widths per pair
    int lev_pitch[kMaxBatch][kMaxLevels];   // elements of the pyramid dtype
    int flow_pitch[kMaxBatch][kMaxLevels];  // float2 elements
    void* pyr[kMaxBatch][2][kMaxLevels];    // luma pyramids of L and R (pyr_dtype elements)
    float* flw[kMaxBatch][2][kMaxLevels];   // flows per direction; level 0 = the rig's own output flows
    unsigned* counters;                     // work counters of the persistent launches, one per level
    void* buf;
    size_t buf_bytes;
    pano_rig_tuning tune[kMaxLevels];
    unsigned long long tune_gen;
    cudaStream_t cap_stream;
    GraphSlot graphs[kGraphSlots];
    unsigned long long graph_clock;
    int captures;
    unsigned long long launches;
    Trace tr;
};

namespace {

pano_status check_desc(const pano_rig_desc* d) {
    if (!d) return fail(PANO_ERR_INVALID_ARG, "desc is NULL");
    if (d->n_pairs < 1 || d->n_pairs > PANO_RIG_MAX_PAIRS)
        return fail(PANO_ERR_INVALID_ARG, "n_pairs %d not in 1..%d", d->n_pairs, PANO_RIG_MAX_PAIRS);
    if (d->h < 1) return fail(PANO_ERR_INVALID_ARG, "strip height %d", d->h);
    if (d->c != 1 && d->c != 3) return fail(PANO_ERR_UNSUPPORTED, "%d channels (1 or 3 supported)", d->c);
    if (d->dtype != PANO_U8 && d->dtype != PANO_F32)
        return fail(d->dtype == PANO_BF16 || d->dtype == PANO_F16 ? PANO_ERR_UNSUPPORTED : PANO_ERR_INVALID_ARG,
                    "strip dtype %d (PANO_U8 or PANO_F32)", d->dtype);
    if (d->canvas_w < 1 || d->canvas_h < 1) return fail(PANO_ERR_INVALID_ARG, "canvas size %dx%d", d->canvas_h, d->canvas_w);
    if (d->canvas_y0 < 0 || (long long)d->canvas_y0 + d->h > d->canvas_h)
        return fail(PANO_ERR_INVALID_ARG, "strip rows %d..%d outside the canvas (%d rows)", d->canvas_y0,
                    d->canvas_y0 + d->h - 1, d->canvas_h);
    for (int k = 0; k < d->n_pairs; ++k) {
        if (d->w[k] < 1 || d->w[k] > d->canvas_w)
            return fail(PANO_ERR_INVALID_ARG, "pair %d: width %d not in 1..canvas_w (%d)", k, d->w[k], d->canvas_w);
        if (d->canvas_x0[k] < 0 || d->canvas_x0[k] >= d->canvas_w)
            return fail(PANO_ERR_INVALID_ARG, "pair %d: canvas_x0 %d not in [0, %d)", k, d->canvas_x0[k], d->canvas_w);
        if ((double)d->h * (double)align_up((size_t)d->w[k] * 3, 64) > (double)INT_MAX)
            return fail(PANO_ERR_UNSUPPORTED, "pair %d: strip too large for 32-bit offsets", k);
    }
    if ((double)d->canvas_h * (double)d->canvas_w * d->c > (double)INT_MAX * 4.0)
        return fail(PANO_ERR_UNSUPPORTED, "canvas too large");
    return PANO_OK;
}

pano_status check_tuning(const pano_rig* r, const pano_rig_tuning* t) {
    if (!t) return fail(PANO_ERR_INVALID_ARG, "tuning is NULL");
    if (t->kernel < PANO_LK_AUTO || t->kernel > PANO_LK_TILE)
        return fail(PANO_ERR_INVALID_ARG, "kernel %d is not a PANO_LK_* value", t->kernel);
    if (t->kernel == PANO_LK_STREAM && !lk_stream_supports(r->p.iters, r->p.radius))
        return fail(PANO_ERR_UNSUPPORTED, "the streamed kernel needs 1 <= iters <= 5");
    if (t->seg_rows < 0 || t->seg_rows > (1 << 20)) return fail(PANO_ERR_INVALID_ARG, "seg_rows %d", t->seg_rows);
    if ((t->tile_w == 0) != (t->tile_h == 0))
        return fail(PANO_ERR_INVALID_ARG, "tile %dx%d: set both sides or neither", t->tile_w, t->tile_h);
    if (t->tile_w) {
        if (t->tile_w < 1 || t->tile_h < 1 || t->tile_w > 1024 || t->tile_h > 1024)
            return fail(PANO_ERR_INVALID_ARG, "tile %dx%d", t->tile_w, t->tile_h);
        if (lk_smem_bytes(t->tile_w, t->tile_h, r->p.iters, r->p.radius) > (size_t)r->max_smem)
            return fail(PANO_ERR_UNSUPPORTED, "tile %dx%d needs more shared memory than the device has", t->tile_w,
                        t->tile_h);
    }
    return PANO_OK;
}

pano_status check_strips(const pano_rig* r, const pano_image* L, const pano_image* R) {
    if (!L || !R) return fail(PANO_ERR_INVALID_ARG, "L or R array is NULL");
    pano_status st;
    char nl[16], nr[16];
    for (int k = 0; k < r->d.n_pairs; ++k) {
        snprintf(nl, sizeof(nl), "L[%d]", k);
        snprintf(nr, sizeof(nr), "R[%d]", k);
        if ((st = check_image(&L[k], nl)) != PANO_OK) return st;
        if ((st = check_image(&R[k], nr)) != PANO_OK) return st;
        if ((st = check_same(&L[k], &R[k], nl, nr)) != PANO_OK) return st;
        if (L[k].h != r->d.h || L[k].w != r->d.w[k] || L[k].c != r->d.c || L[k].dtype != r->d.dtype)
            return fail(PANO_ERR_INVALID_ARG, "%s is %dx%dx%d dtype %d; the rig expects %dx%dx%d dtype %d", nl, L[k].h,
                        L[k].w, L[k].c, L[k].dtype, r->d.h, r->d.w[k], r->d.c, r->d.dtype);
    }
    return PANO_OK;
}

pano_status check_device(const pano_rig* r) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != r->device) return fail(PANO_ERR_INVALID_ARG, "device %d is current; the rig lives on device %d", dev, r->device);
    return PANO_OK;
}

// Whether strip side `s` of pair k is its own level 0: a one-channel float
// strip with float32 pyramids.
bool own_level0(const pano_rig* r, const pano_image& im) {
    return im.dtype == PANO_F32 && im.c == 1 && r->p.pyr_dtype == PANO_F32;
}

// Level-0 plane of strip side `s` (0 = L, 1 = R) of pair k.
const void* level0(const pano_rig* r, const RunCall& c, int k, int s, int* pitch) {
    const pano_image& im = s == 0 ? c.L[k] : c.R[k];
    if (own_level0(r, im)) {
        *pitch = (int)(im.pitch_bytes / sizeof(float));
        return im.data;
    }
    *pitch = r->lev_pitch[k][0];
    return r->pyr[k][s][0];
}

LkArgs pair_level_args(const pano_rig* r, const RunCall& c, int k, int l, const pano_rig_tuning& t) {
    LkArgs a;
    memset(&a, 0, sizeof(a));
    const int nlev = r->nlev;
    for (int d = 0; d < 2; ++d) {
        // direction 0: FlowLtoR (template L, target R); 1: FlowRtoL
        int pt = r->lev_pitch[k][l], pj = r->lev_pitch[k][l];
        const void* T = r->pyr[k][d][l];
        const void* J = r->pyr[k][1 - d][l];
        if (l == 0) {
            T = level0(r, c, k, d, &pt);
            J = level0(r, c, k, 1 - d, &pj);
        }
        a.dir[d].T = T;
        a.dir[d].pitchT = pt;
        a.dir[d].J = J;
        a.dir[d].pitchJ = pj;
        a.dir[d].uin = l == nlev - 1 ? nullptr : r->flw[k][d][l + 1];
        a.dir[d].uin_pitch = l == nlev - 1 ? 0 : r->flow_pitch[k][l + 1];
        float* out0 = d == 0 ? c.lr[k] : c.rl[k];
        a.dir[d].uout = l == 0 ? out0 : r->flw[k][d][l];
        a.dir[d].uout_pitch = l == 0 ? r->d.w[k] : r->flow_pitch[k][l];
    }
    a.h = r->hs[l];
    a.w = r->ws[k][l];
    a.in_h = l == nlev - 1 ? 0 : r->hs[l + 1];
    a.in_w = l == nlev - 1 ? 0 : r->ws[k][l + 1];
    a.mode = l == nlev - 1 ? 0 : 1;
    a.iters = r->p.iters;
    a.radius = r->p.radius;
    a.lambda = r->p.lambda;
    if (t.tile_w) {
        a.tile_w = t.tile_w;
        a.tile_h = t.tile_h;
    } else {
        lk_level_tile(a.w, a.h, r->def_tile_w, r->def_tile_h, &a.tile_w, &a.tile_h);  // the rule of pano_flow_pair
    }
    a.seg_rows = t.seg_rows;
    a.pyr = pyr_type(r->p.pyr_dtype);
    return a;
}

bool uses_stream(const pano_rig* r, const LkArgs& a, int kernel) {
    if (!lk_stream_supports(r->p.iters, r->p.radius)) return false;
    if (kernel == PANO_LK_STREAM) return true;
    if (kernel == PANO_LK_TILE) return false;
    return (long long)a.w * a.h >= kStreamMinPixels;  // the rule of launch_lk_level
}

// LK level l of every pair with tuning t: one persistent launch of the
// streamed kernel for the pairs that use it, then one tiled launch per tile
// shape (in the order of the first pair with that shape). Returns the first
// launch error and adds the kernels launched to *kernels.
cudaError_t enqueue_lk_level(pano_rig* r, const RunCall& c, int l, const pano_rig_tuning& t, cudaStream_t s,
                             bool trace, int* kernels) {
    LkBatch sb;
    memset(&sb, 0, sizeof(sb));
    LkBatch tb[kMaxBatch];
    int ntb = 0;
    for (int k = 0; k < r->d.n_pairs; ++k) {
        LkArgs a = pair_level_args(r, c, k, l, t);
        if (uses_stream(r, a, t.kernel)) {
            sb.pair[sb.n++] = a;
            continue;
        }
        int g = 0;
        while (g < ntb && (tb[g].pair[0].tile_w != a.tile_w || tb[g].pair[0].tile_h != a.tile_h)) ++g;
        if (g == ntb) {
            memset(&tb[g], 0, sizeof(tb[g]));
            ++ntb;
        }
        tb[g].pair[tb[g].n++] = a;
    }
    cudaError_t e;
    if (sb.n) {
        sb.counter = r->counters + l;
        int slot = trace ? trace_begin(r->tr, PANO_TRACE_LK, l, s) : -1;
        if ((e = launch_lk_stream_batch(sb, r->n_ctas, s)) != cudaSuccess) return e;
        if (slot >= 0) trace_end(r->tr, slot, s);
        ++*kernels;
    }
    for (int g = 0; g < ntb; ++g) {
        int slot = trace ? trace_begin(r->tr, PANO_TRACE_LK, l, s) : -1;
        if ((e = launch_lk_tile_batch(tb[g], s)) != cudaSuccess) return e;
        if (slot >= 0) trace_end(r->tr, slot, s);
        ++*kernels;
    }
    return cudaSuccess;
}

// The whole rig step on stream s. Kernel launches are added to *kernels.
cudaError_t enqueue_all(pano_rig* r, const RunCall& c, cudaStream_t s, bool trace, int* kernels) {
    const int n = r->d.n_pairs;
    cudaError_t e;
    // work counters of the persistent launches start at zero
    if ((e = cudaMemsetAsync(r->counters, 0, sizeof(unsigned) * kMaxLevels, s)) != cudaSuccess) return e;
    // luma of every strip that is not its own level 0
    LumaArgs la;
    memset(&la, 0, sizeof(la));
    for (int k = 0; k < n; ++k)
        for (int si = 0; si < 2; ++si) {
            const pano_image& im = si == 0 ? c.L[k] : c.R[k];
            if (own_level0(r, im)) continue;
            la.in[la.count] = desc(&im);
            la.out[la.count] = r->pyr[k][si][0];
            la.out_pitch[la.count] = r->lev_pitch[k][0];
            la.count++;
        }
    la.pyr = pyr_type(r->p.pyr_dtype);
    int first = 1;  // first level left to REDUCE
    if (la.count == 2 * n && r->nlev >= 2) {
        // level 0 and level 1 of every strip in one launch (as pano_flow_pair)
        LumaReduceArgs lr;
        memset(&lr, 0, sizeof(lr));
        int i = 0;
        for (int k = 0; k < n; ++k)
            for (int si = 0; si < 2; ++si, ++i) {
                lr.in[i] = la.in[i];
                lr.l0[i] = la.out[i];
                lr.l0_pitch[i] = la.out_pitch[i];
                lr.l1[i] = r->pyr[k][si][1];
                lr.l1_pitch[i] = r->lev_pitch[k][1];
            }
        lr.count = la.count;
        lr.pyr = la.pyr;
        int slot = trace ? trace_begin(r->tr, PANO_TRACE_LUMA_REDUCE, 1, s) : -1;
        if ((e = launch_luma_reduce(lr, s)) != cudaSuccess) return e;
        if (slot >= 0) trace_end(r->tr, slot, s);
        ++*kernels;
        first = 2;
    } else if (la.count) {
        int slot = trace ? trace_begin(r->tr, PANO_TRACE_LUMA, 0, s) : -1;
        if ((e = launch_luma(la, s)) != cudaSuccess) return e;
        if (slot >= 0) trace_end(r->tr, slot, s);
        ++*kernels;
    }
    // the other levels of every strip (the same launch sequence as pano_flow_pair)
    PyrSet ps;
    memset(&ps, 0, sizeof(ps));
    for (int k = 0; k < n; ++k)
        for (int si = 0; si < 2; ++si) {
            const int i = 2 * k + si;
            for (int l = 0; l < r->nlev; ++l) {
                int sp = r->lev_pitch[k][l];
                ps.plane[i][l] = l == 0 ? level0(r, c, k, si, &sp) : r->pyr[k][si][l];
                ps.pitch[i][l] = sp;
            }
            ps.h0[i] = r->hs[0];
            ps.w0[i] = r->ws[k][0];
        }
    ps.count = 2 * n;
    ps.nlev = r->nlev;
    ps.pyr = pyr_type(r->p.pyr_dtype);
    if ((e = launch_pyramid_rest(ps, first, trace ? &r->tr : nullptr, s, kernels)) != cudaSuccess) return e;
    // LK from the coarsest level to the finest
    for (int l = r->nlev - 1; l >= 0; --l)
        if ((e = enqueue_lk_level(r, c, l, r->tune[l], s, trace, kernels)) != cudaSuccess) return e;
    // blend of every pair straight into the canvas
    if (c.canvas) {
        RigBlendArgs ba;
        memset(&ba, 0, sizeof(ba));
        ba.n = n;
        ba.canvas_w = r->d.canvas_w;
        for (int k = 0; k < n; ++k) {
            BlendArgs& a = ba.pair[k];
            a.L = desc(&c.L[k]);
            a.R = desc(&c.R[k]);
            a.flowLR = reinterpret_cast<const float2*>(c.lr[k]);
            a.flowRL = reinterpret_cast<const float2*>(c.rl[k]);
            a.blend = nullptr;  // Eq. (1) for a full-height strip
            a.F = static_cast<char*>(c.canvas->data) + (size_t)r->d.canvas_y0 * c.canvas->pitch_bytes;
            a.F_pitch_bytes = (long long)c.canvas->pitch_bytes;
            a.k_sharp = r->p.soft_sharpness;
            a.k_mag = r->p.flow_mag_coef;
            ba.x0[k] = r->d.canvas_x0[k];
        }
        int slot = trace ? trace_begin(r->tr, PANO_TRACE_BLEND, 0, s) : -1;
        if ((e = launch_rig_blend(ba, s)) != cudaSuccess) return e;
        if (slot >= 0) trace_end(r->tr, slot, s);
        ++*kernels;
    }
    return cudaSuccess;
}

GraphKey make_key(const pano_rig* r, const RunCall& c) {
    GraphKey k;
    memset(&k, 0, sizeof(k));
    for (int i = 0; i < r->d.n_pairs; ++i) {
        k.L[i] = c.L[i].data;
        k.R[i] = c.R[i].data;
        k.Lp[i] = c.L[i].pitch_bytes;
        k.Rp[i] = c.R[i].pitch_bytes;
        k.lr[i] = c.lr[i];
        k.rl[i] = c.rl[i];
    }
    k.canvas = c.canvas ? c.canvas->data : nullptr;
    k.canvas_pitch = c.canvas ? c.canvas->pitch_bytes : 0;
    k.tune_gen = r->tune_gen;
    return k;
}

// Capture the call's launch sequence into slot `g` (replacing its graph).
pano_status capture(pano_rig* r, const RunCall& c, int g) {
    GraphSlot& slot = r->graphs[g];
    if (slot.exec) {
        cudaGraphExecDestroy(slot.exec);
        slot.exec = nullptr;
    }
    cudaError_t e = cudaStreamBeginCapture(r->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    int kernels = 0;
    cudaError_t le = enqueue_all(r, c, r->cap_stream, false, &kernels);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(r->cap_stream, &graph);  // always ends the capture
    if (le != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(le, "launch during graph capture");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&slot.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        slot.exec = nullptr;
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    slot.key = make_key(r, c);
    slot.kernels = kernels;
    r->captures++;
    return PANO_OK;
}

void free_rig(pano_rig* r) {
    trace_free(r->tr);
    for (GraphSlot& g : r->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (r->cap_stream) cudaStreamDestroy(r->cap_stream);
    if (r->buf) cudaFree(r->buf);
    delete r;
}

pano_status fill_call(const pano_rig* r, const pano_image* L, const pano_image* R, float* const* lr, float* const* rl,
                      const pano_image* canvas, RunCall* c) {
    pano_status st;
    if ((st = check_strips(r, L, R)) != PANO_OK) return st;
    if ((lr == nullptr) != (rl == nullptr))
        return fail(PANO_ERR_INVALID_ARG, "pass both flow arrays or neither");
    memset(c, 0, sizeof(*c));
    c->L = L;
    c->R = R;
    for (int k = 0; k < r->d.n_pairs; ++k) {
        c->lr[k] = lr ? lr[k] : r->flw[k][0][0];
        c->rl[k] = rl ? rl[k] : r->flw[k][1][0];
        char n1[24], n2[24];
        snprintf(n1, sizeof(n1), "flow_LtoR[%d]", k);
        snprintf(n2, sizeof(n2), "flow_RtoL[%d]", k);
        if ((st = check_flow(c->lr[k], n1)) != PANO_OK) return st;
        if ((st = check_flow(c->rl[k], n2)) != PANO_OK) return st;
        const size_t fb = (size_t)r->d.h * r->d.w[k] * 2 * sizeof(float);
        if (overlaps(c->lr[k], fb, c->rl[k], fb)) return fail(PANO_ERR_INVALID_ARG, "the flows of pair %d overlap", k);
    }
    if (canvas) {
        if ((st = check_image(canvas, "canvas")) != PANO_OK) return st;
        if (canvas->h != r->d.canvas_h || canvas->w != r->d.canvas_w || canvas->c != r->d.c ||
            canvas->dtype != r->d.dtype)
            return fail(PANO_ERR_INVALID_ARG, "canvas is %dx%dx%d dtype %d; the rig expects %dx%dx%d dtype %d",
                        canvas->h, canvas->w, canvas->c, canvas->dtype, r->d.canvas_h, r->d.canvas_w, r->d.c,
                        r->d.dtype);
        const size_t cb = (size_t)canvas->h * canvas->pitch_bytes;
        for (int k = 0; k < r->d.n_pairs; ++k) {
            if (overlaps(canvas->data, cb, L[k].data, (size_t)L[k].h * L[k].pitch_bytes) ||
                overlaps(canvas->data, cb, R[k].data, (size_t)R[k].h * R[k].pitch_bytes))
                return fail(PANO_ERR_INVALID_ARG, "the canvas overlaps the strips of pair %d", k);
            const size_t fb = (size_t)r->d.h * r->d.w[k] * 2 * sizeof(float);
            if (overlaps(canvas->data, cb, c->lr[k], fb) || overlaps(canvas->data, cb, c->rl[k], fb))
                return fail(PANO_ERR_INVALID_ARG, "the canvas overlaps the flows of pair %d", k);
        }
        c->canvas = canvas;
    }
    return PANO_OK;
}

}  // namespace

extern "C" {

pano_status pano_rig_create(const pano_flow_params* p, const pano_rig_desc* d, pano_rig** out) {
    if (!out) return fail(PANO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    pano_status st;
    if ((st = check_params(p)) != PANO_OK) return st;
    if ((st = check_desc(d)) != PANO_OK) return st;
    int max_smem = 0;
    if ((st = ensure_lk_ready(&max_smem)) != PANO_OK) return st;
    int tw = 0, th = 0;
    if (!pick_tile(p->iters, p->radius, max_smem, &tw, &th))
        return fail(PANO_ERR_UNSUPPORTED, "iters * radius = %d needs more shared memory than the device has",
                    p->iters * p->radius);
    pano_rig* r = new (std::nothrow) pano_rig;
    if (!r) return fail(PANO_ERR_OOM, "host allocation failed");
    memset(r, 0, sizeof(*r));
    r->p = *p;
    r->d = *d;
    r->nlev = p->levels;
    r->max_smem = max_smem;
    r->def_tile_w = tw;
    r->def_tile_h = th;
    cudaError_t e = cudaGetDevice(&r->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, r->device);
    if (e != cudaSuccess) {
        free_rig(r);
        return cuda_fail(e, "device query");
    }
    r->n_ctas = sms;  // the streamed kernel runs one 768-thread CTA per SM
    const int n = d->n_pairs;
    for (int l = 0; l < r->nlev; ++l) r->hs[l] = l == 0 ? d->h : (r->hs[l - 1] + 1) / 2;
    size_t total = align_up(sizeof(unsigned) * kMaxLevels, 256);
    std::vector<size_t> offs;
    for (int k = 0; k < n; ++k)
        for (int l = 0; l < r->nlev; ++l) {
            r->ws[k][l] = l == 0 ? d->w[k] : (r->ws[k][l - 1] + 1) / 2;
            r->lev_pitch[k][l] = (int)align_up(r->ws[k][l], 32);
            r->flow_pitch[k][l] = l == 0 ? d->w[k] : (int)align_up(r->ws[k][l], 16);
            for (int s = 0; s < 2; ++s) {
                offs.push_back(total);
                total += align_up((size_t)r->lev_pitch[k][l] * r->hs[l] * (size_t)elem_size(p->pyr_dtype), 256);
            }
            for (int s = 0; s < 2; ++s) {
                offs.push_back(total);
                total += align_up((size_t)r->flow_pitch[k][l] * r->hs[l] * 2 * sizeof(float), 256);
            }
        }
    e = device_alloc(&r->buf, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        r->buf = nullptr;
        free_rig(r);
        return fail(PANO_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", total, cudaGetErrorString(e));
    }
    r->buf_bytes = total;
    char* b = static_cast<char*>(r->buf);
    r->counters = reinterpret_cast<unsigned*>(b);
    size_t i = 0;
    for (int k = 0; k < n; ++k)
        for (int l = 0; l < r->nlev; ++l) {
            for (int s = 0; s < 2; ++s) r->pyr[k][s][l] = b + offs[i++];
            for (int s = 0; s < 2; ++s) r->flw[k][s][l] = reinterpret_cast<float*>(b + offs[i++]);
        }
    if ((e = cudaStreamCreateWithFlags(&r->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        r->cap_stream = nullptr;
        free_rig(r);
        return cuda_fail(e, "cudaStreamCreate");
    }
    for (int l = 0; l < kMaxLevels; ++l) r->tune[l].kernel = PANO_LK_AUTO;
    *out = r;
    return PANO_OK;
}

pano_status pano_rig_destroy(pano_rig* r) {
    if (!r) return PANO_OK;
    free_rig(r);
    return PANO_OK;
}

pano_status pano_rig_run(pano_rig* r, const pano_image* L, const pano_image* R, float* const* flow_LtoR,
                         float* const* flow_RtoL, pano_image* canvas, int use_graph, void* cuda_stream) {
    if (!r) return fail(PANO_ERR_INVALID_ARG, "rig is NULL");
    pano_status st;
    if ((st = check_device(r)) != PANO_OK) return st;
    RunCall c;
    if ((st = fill_call(r, L, R, flow_LtoR, flow_RtoL, canvas, &c)) != PANO_OK) return st;
    NvtxRange range(use_graph ? "pano_rig_run (graph)" : "pano_rig_run");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (!use_graph) {
        int kernels = 0;
        cudaError_t e = enqueue_all(r, c, s, true, &kernels);
        r->launches += kernels;
        if (e == cudaSuccess) e = debug_check(s);
        return e == cudaSuccess ? PANO_OK : cuda_fail(e, "rig launch");
    }
    // a graph captured for these pointers, pitches and tuning, else a new
    // capture in the least recently used slot
    GraphKey k = make_key(r, c);
    int g = -1, lru = 0;
    for (int i = 0; i < kGraphSlots; ++i) {
        if (r->graphs[i].exec && memcmp(&k, &r->graphs[i].key, sizeof(k)) == 0) g = i;
        if (!r->graphs[i].exec) {
            if (r->graphs[lru].exec) lru = i;
        } else if (r->graphs[lru].exec && r->graphs[i].last_use < r->graphs[lru].last_use) {
            lru = i;
        }
    }
    if (g < 0) {
        g = lru;
        if ((st = capture(r, c, g)) != PANO_OK) return st;
    }
    r->graphs[g].last_use = ++r->graph_clock;
    cudaError_t e = cudaGraphLaunch(r->graphs[g].exec, s);
    if (e == cudaSuccess) e = debug_check(s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    r->launches += r->graphs[g].kernels;
    return PANO_OK;
}

pano_status pano_rig_autotune(pano_rig* r, const pano_image* L, const pano_image* R, int reps, void* cuda_stream) {
    if (!r) return fail(PANO_ERR_INVALID_ARG, "rig is NULL");
    if (reps < 1 || reps > 1000) return fail(PANO_ERR_INVALID_ARG, "reps %d not in 1..1000", reps);
    pano_status st;
    if ((st = check_device(r)) != PANO_OK) return st;
    RunCall c;
    if ((st = fill_call(r, L, R, nullptr, nullptr, nullptr, &c)) != PANO_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int kernels = 0;
    cudaError_t e = enqueue_all(r, c, s, false, &kernels);  // pyramids and every level's flows
    r->launches += kernels;
    if (e != cudaSuccess) return cuda_fail(e, "rig launch");

    std::vector<pano_rig_tuning> cand;
    pano_rig_tuning t;
    memset(&t, 0, sizeof(t));
    cand.push_back(t);  // PANO_LK_AUTO
    if (lk_stream_supports(r->p.iters, r->p.radius)) {
        static const int segs[] = {0, 64, 96, 128, 192, 256, 384};
        for (int sg : segs) {
            t.kernel = PANO_LK_STREAM;
            t.seg_rows = sg;
            cand.push_back(t);
        }
    }
    static const int tiles[][2] = {{32, 8}, {32, 16}, {16, 16}, {64, 8}, {64, 16}, {32, 32}};
    for (auto& tl : tiles) {
        memset(&t, 0, sizeof(t));
        t.kernel = PANO_LK_TILE;
        t.tile_w = tl[0];
        t.tile_h = tl[1];
        if (lk_smem_bytes(t.tile_w, t.tile_h, r->p.iters, r->p.radius) <= (size_t)r->max_smem) cand.push_back(t);
    }

    cudaEvent_t ev[2] = {nullptr, nullptr};
    if ((e = cudaEventCreate(&ev[0])) != cudaSuccess || (e = cudaEventCreate(&ev[1])) != cudaSuccess) {
        if (ev[0]) cudaEventDestroy(ev[0]);
        return cuda_fail(e, "cudaEventCreate");
    }
    pano_status out = PANO_OK;
    std::vector<float> times(reps);
    for (int l = 0; l < r->nlev && out == PANO_OK; ++l) {
        float best = -1.f;
        pano_rig_tuning pick = cand[0];
        for (const pano_rig_tuning& ct : cand) {
            int dummy = 0;
            // the counter of this level is reset before every launch
            if ((e = cudaMemsetAsync(r->counters + l, 0, sizeof(unsigned), s)) != cudaSuccess ||
                (e = enqueue_lk_level(r, c, l, ct, s, false, &dummy)) != cudaSuccess) {
                out = cuda_fail(e, "autotune launch");
                break;
            }
            for (int i = 0; i < reps && out == PANO_OK; ++i) {
                if ((e = cudaMemsetAsync(r->counters + l, 0, sizeof(unsigned), s)) != cudaSuccess ||
                    (e = cudaEventRecord(ev[0], s)) != cudaSuccess ||
                    (e = enqueue_lk_level(r, c, l, ct, s, false, &dummy)) != cudaSuccess ||
                    (e = cudaEventRecord(ev[1], s)) != cudaSuccess || (e = cudaEventSynchronize(ev[1])) != cudaSuccess ||
                    (e = cudaEventElapsedTime(&times[i], ev[0], ev[1])) != cudaSuccess)
                    out = cuda_fail(e, "autotune timing");
            }
            if (out != PANO_OK) break;
            r->launches += (unsigned long long)dummy;
            std::vector<float> sorted(times);
            std::sort(sorted.begin(), sorted.end());
            const float med = sorted[reps / 2];
            if (best < 0.f || med < best) {
                best = med;
                pick = ct;
            }
        }
        if (out == PANO_OK) {
            pick.ms = best;
            r->tune[l] = pick;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    r->tune_gen++;
    return out;
}

pano_status pano_rig_get_tuning(const pano_rig* r, int level, pano_rig_tuning* out) {
    if (!r || !out) return fail(PANO_ERR_INVALID_ARG, "NULL argument");
    if (level < 0 || level >= r->nlev) return fail(PANO_ERR_INVALID_ARG, "level %d not in 0..%d", level, r->nlev - 1);
    *out = r->tune[level];
    return PANO_OK;
}

pano_status pano_rig_set_tuning(pano_rig* r, int level, const pano_rig_tuning* t) {
    if (!r) return fail(PANO_ERR_INVALID_ARG, "rig is NULL");
    if (level < 0 || level >= r->nlev) return fail(PANO_ERR_INVALID_ARG, "level %d not in 0..%d", level, r->nlev - 1);
    pano_status st;
    if ((st = check_tuning(r, t)) != PANO_OK) return st;
    r->tune[level] = *t;
    r->tune[level].ms = 0.f;
    r->tune_gen++;
    return PANO_OK;
}

pano_status pano_rig_flows(const pano_rig* r, int k, float** lr, float** rl) {
    if (!r || !lr || !rl) return fail(PANO_ERR_INVALID_ARG, "NULL argument");
    if (k < 0 || k >= r->d.n_pairs) return fail(PANO_ERR_INVALID_ARG, "pair %d not in 0..%d", k, r->d.n_pairs - 1);
    *lr = r->flw[k][0][0];
    *rl = r->flw[k][1][0];
    return PANO_OK;
}

pano_status pano_rig_trace_enable(pano_rig* r, unsigned kind_mask, int capacity) {
    if (!r) return fail(PANO_ERR_INVALID_ARG, "rig is NULL");
    return trace_enable(r->tr, kind_mask, capacity);
}

pano_status pano_rig_trace_read(pano_rig* r, pano_trace_record* out, int max_records, int* n_out) {
    if (!r) return fail(PANO_ERR_INVALID_ARG, "rig is NULL");
    return trace_read(r->tr, out, max_records, n_out);
}

unsigned long long pano_rig_launches(const pano_rig* r) { return r ? r->launches : 0ull; }

int pano_rig_graph_captures(const pano_rig* r) { return r ? r->captures : 0; }

}  // extern "C"
