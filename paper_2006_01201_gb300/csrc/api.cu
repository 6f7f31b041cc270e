// api.cu -- the C ABI declared in include/pano_flow.h: argument checks, the
// context (scratch pyramids and coarse flows), and the launch sequence of the
// blend path of Section III-C:
//   pano_flow_pair : luma (level 0) -> REDUCE x (levels-1) -> LK level
//                    (both directions per launch) from coarse to fine
//   pano_blend_pair: Code 1 with Eq. (1)
// Every call only enqueues kernels on the caller's stream.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <climits>
#include <cstdlib>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "pano_flow.h"

using namespace pano;

#include "ctx.h"

namespace {
thread_local char g_err[512] = "";
}  // namespace

namespace pano {

pano_status fail(pano_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

pano_status cuda_fail(cudaError_t e, const char* what) {
    return fail(PANO_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int elem_size(int dtype) { return dtype == PANO_U8 ? 1 : (dtype == PANO_F32 ? 4 : 2); }

int pyr_type(int pyr_dtype) {
    return pyr_dtype == PANO_BF16 ? kPyrBF16 : (pyr_dtype == PANO_F16 ? kPyrF16 : kPyrF32);
}

pano_status check_image(const pano_image* im, const char* name) {
    if (!im) return fail(PANO_ERR_INVALID_ARG, "%s is NULL", name);
    if (!im->data) return fail(PANO_ERR_INVALID_ARG, "%s->data is NULL", name);
    if (im->h < 1 || im->w < 1) return fail(PANO_ERR_INVALID_ARG, "%s size %dx%d", name, im->h, im->w);
    if (im->dtype == PANO_BF16 || im->dtype == PANO_F16)
        return fail(PANO_ERR_UNSUPPORTED, "%s: 16-bit images are not supported", name);
    if (im->dtype != PANO_U8 && im->dtype != PANO_F32)
        return fail(PANO_ERR_INVALID_ARG, "%s: unknown dtype %d", name, im->dtype);
    if (im->c != 1 && im->c != 3)
        return fail(PANO_ERR_UNSUPPORTED, "%s: %d channels (1 or 3 supported)", name, im->c);
    size_t es = (size_t)elem_size(im->dtype);
    if (im->pitch_bytes < (size_t)im->w * im->c * es)
        return fail(PANO_ERR_INVALID_ARG, "%s: pitch %zu < row size %zu", name, im->pitch_bytes,
                    (size_t)im->w * im->c * es);
    if (im->pitch_bytes % es || ((uintptr_t)im->data) % es)
        return fail(PANO_ERR_INVALID_ARG, "%s: pitch or data not aligned to the element size", name);
    if ((double)im->h * (double)(im->pitch_bytes / es) > (double)INT_MAX)
        return fail(PANO_ERR_UNSUPPORTED, "%s: more than 2^31 elements", name);
    return PANO_OK;
}

pano_status check_same(const pano_image* a, const pano_image* b, const char* na, const char* nb) {
    if (a->h != b->h || a->w != b->w || a->c != b->c || a->dtype != b->dtype)
        return fail(PANO_ERR_INVALID_ARG, "%s and %s differ in size, channels or dtype", na, nb);
    return PANO_OK;
}

pano_status check_flow(const void* f, const char* name) {
    if (!f) return fail(PANO_ERR_INVALID_ARG, "%s is NULL", name);
    if (((uintptr_t)f) % 8) return fail(PANO_ERR_INVALID_ARG, "%s is not 8-byte aligned", name);
    return PANO_OK;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

pano_status check_params(const pano_flow_params* p) {
    if (!p) return fail(PANO_ERR_INVALID_ARG, "params is NULL");
    if (p->levels < 1 || p->levels > kMaxLevels)
        return fail(PANO_ERR_INVALID_ARG, "levels %d not in 1..%d", p->levels, kMaxLevels);
    if (p->iters < 0 || p->iters > 16) return fail(PANO_ERR_INVALID_ARG, "iters %d not in 0..16", p->iters);
    if (p->radius < 1 || p->radius > 3) return fail(PANO_ERR_INVALID_ARG, "radius %d not in 1..3", p->radius);
    if (!(p->lambda >= 0.f) || !(p->lambda < 1e30f))
        return fail(PANO_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    if (!(p->soft_sharpness == p->soft_sharpness) || !(p->flow_mag_coef == p->flow_mag_coef))
        return fail(PANO_ERR_INVALID_ARG, "softmax parameters must not be NaN");
    if (p->pyr_dtype != PANO_F32 && p->pyr_dtype != PANO_BF16 && p->pyr_dtype != PANO_F16)
        return fail(PANO_ERR_INVALID_ARG, "pyramid dtype %d (PANO_F32, PANO_BF16 or PANO_F16)", p->pyr_dtype);
    return PANO_OK;
}

int max_optin_smem() {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return -1;
    return v;
}

// Largest tile from a fixed list whose shared-memory footprint fits.
bool pick_tile(int iters, int radius, int max_smem, int* tw, int* th) {
    static const int cand[][2] = {{32, 16}, {32, 8}, {16, 16}, {16, 8}, {8, 8}};
    for (auto& c : cand) {
        if (lk_smem_bytes(c[0], c[1], iters, radius) <= (size_t)max_smem) {
            *tw = c[0];
            *th = c[1];
            return true;
        }
    }
    return false;
}

// Sets the dynamic shared-memory limit of the LK kernel once per device.
pano_status ensure_lk_ready(int* max_smem_out) {
    static int prepared[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    int ms = max_optin_smem();
    if (ms <= 0) return fail(PANO_ERR_CUDA, "cannot query the shared-memory limit");
    if (dev >= 0 && dev < 64 && !prepared[dev]) {
        if ((e = lk_prepare(ms)) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        if ((e = blend_coeff_prepare(ms)) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        if ((e = pyr_tail_prepare(ms)) != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        prepared[dev] = 1;
    }
    *max_smem_out = ms;
    return PANO_OK;
}

void trace_free(Trace& t) {
    if (t.ev) {
        for (int i = 0; i < 2 * t.cap; ++i)
            if (t.ev[i]) cudaEventDestroy(t.ev[i]);
        delete[] t.ev;
    }
    delete[] t.rec;
    t.ev = nullptr;
    t.rec = nullptr;
    t.cap = t.n = 0;
    t.mask = 0;
}

int trace_begin(Trace& t, unsigned kind, int level, cudaStream_t s) {
    if (!(t.mask & kind) || t.n >= t.cap) return -1;
    int i = t.n++;
    t.rec[i].kind = (int)kind;
    t.rec[i].level = level;
    t.rec[i].ms = 0.f;
    cudaEventRecord(t.ev[2 * i], s);
    return i;
}

void trace_end(Trace& t, int slot, cudaStream_t s) {
    if (slot >= 0) cudaEventRecord(t.ev[2 * slot + 1], s);
}

pano_status trace_enable(Trace& t, unsigned kind_mask, int capacity) {
    if (capacity < 0 || capacity > (1 << 20)) return fail(PANO_ERR_INVALID_ARG, "capacity %d", capacity);
    trace_free(t);
    if (capacity == 0 || kind_mask == 0) return PANO_OK;
    t.ev = new (std::nothrow) cudaEvent_t[2 * (size_t)capacity]();
    t.rec = new (std::nothrow) pano_trace_record[capacity];
    if (!t.ev || !t.rec) {
        delete[] t.ev;
        delete[] t.rec;
        t.ev = nullptr;
        t.rec = nullptr;
        return fail(PANO_ERR_OOM, "host allocation failed");
    }
    t.cap = capacity;
    for (int i = 0; i < 2 * capacity; ++i) {
        cudaError_t e = cudaEventCreate(&t.ev[i]);
        if (e != cudaSuccess) {
            trace_free(t);
            return cuda_fail(e, "cudaEventCreate");
        }
    }
    t.mask = kind_mask;
    t.n = 0;
    return PANO_OK;
}

pano_status trace_read(Trace& t, pano_trace_record* out, int max_records, int* n_out) {
    if (!n_out || (max_records > 0 && !out)) return fail(PANO_ERR_INVALID_ARG, "NULL argument");
    *n_out = 0;
    int n = t.n < max_records ? t.n : max_records;
    for (int i = 0; i < n; ++i) {
        cudaError_t e = cudaEventSynchronize(t.ev[2 * i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t.rec[i].ms, t.ev[2 * i], t.ev[2 * i + 1]);
        if (e != cudaSuccess) return cuda_fail(e, "reading trace events");
        out[i] = t.rec[i];
    }
    *n_out = n;
    t.n = 0;
    return PANO_OK;
}

ImageDesc desc(const pano_image* im) {
    ImageDesc d;
    d.data = im->data;
    d.h = im->h;
    d.w = im->w;
    d.c = im->c;
    d.pitch_bytes = (long long)im->pitch_bytes;
    d.dtype = im->dtype == PANO_U8 ? 0 : 1;
    return d;
}

void set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg ? msg : ""); }

unsigned debug_flags() {
    const char* v = getenv("PANO_DEBUG");
    if (!v) return 0;
    unsigned f = 0;
    const char* p = v;
    while (*p) {
        const char* q = p;
        while (*q && *q != ',') ++q;
        const size_t n = (size_t)(q - p);
        if (n == 4 && strncmp(p, "sync", 4) == 0) f |= kDebugSync;
        if (n == 10 && strncmp(p, "fail_alloc", 10) == 0) f |= kDebugFailAlloc;
        p = *q ? q + 1 : q;
    }
    return f;
}

cudaError_t device_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (debug_flags() & kDebugFailAlloc) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t debug_check(cudaStream_t s) {
    if (!(debug_flags() & kDebugSync)) return cudaSuccess;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(s);
    return e != cudaSuccess ? e : cudaGetLastError();
}

NvtxRange::NvtxRange(const char* name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

pano_status check_pair_call(const pano_flow_ctx* c, const pano_image* L, const pano_image* R, const float* lr,
                            const float* rl) {
    if (!c) return fail(PANO_ERR_INVALID_ARG, "context is NULL");
    pano_status st;
    if ((st = check_image(L, "L")) != PANO_OK) return st;
    if ((st = check_image(R, "R")) != PANO_OK) return st;
    if ((st = check_same(L, R, "L", "R")) != PANO_OK) return st;
    if ((st = check_flow(lr, "flow_LtoR")) != PANO_OK) return st;
    if ((st = check_flow(rl, "flow_RtoL")) != PANO_OK) return st;
    if (L->h > c->max_h || L->w > c->max_w || L->c > c->max_c)
        return fail(PANO_ERR_INVALID_ARG, "strip %dx%dx%d exceeds the context maximum %dx%dx%d", L->h, L->w,
                    L->c, c->max_h, c->max_w, c->max_c);
    const size_t fbytes = (size_t)L->h * L->w * 2 * sizeof(float);
    if (overlaps(lr, fbytes, rl, fbytes)) return fail(PANO_ERR_INVALID_ARG, "the two flows overlap");
    return PANO_OK;
}

void pair_planes(const pano_flow_ctx* c, const pano_image* L, const pano_image* R, PairPlanes* pp) {
    memset(pp, 0, sizeof(*pp));
    const int nlev = c->nlev;
    pp->hs[0] = L->h;
    pp->ws[0] = L->w;
    for (int l = 1; l < nlev; ++l) {
        pp->hs[l] = (pp->hs[l - 1] + 1) / 2;
        pp->ws[l] = (pp->ws[l - 1] + 1) / 2;
    }
    const pano_image* img[2] = {L, R};
    for (int si = 0; si < 2; ++si) {
        for (int l = 0; l < nlev; ++l) {
            pp->plane[si][l] = c->pyr[si][l];
            pp->pitch[si][l] = c->lev_pitch[l];
        }
        if (img[si]->dtype == PANO_F32 && img[si]->c == 1 && c->p.pyr_dtype == PANO_F32) {
            // a one-channel float strip is its own luma (float32 pyramids only)
            pp->plane[si][0] = img[si]->data;
            pp->pitch[si][0] = (int)(img[si]->pitch_bytes / sizeof(float));
        } else {
            LumaArgs& la = pp->luma;
            la.in[la.count] = desc(img[si]);
            la.out[la.count] = c->pyr[si][0];
            la.out_pitch[la.count] = c->lev_pitch[0];
            la.count++;
        }
    }
    pp->luma.pyr = pyr_type(c->p.pyr_dtype);
}

cudaError_t launch_pyramid_rest(const PyrSet& ps, int first, Trace* tr, cudaStream_t s, int* kernels) {
    auto size = [&](int i, int l, int* h, int* w) {
        *h = ps.h0[i];
        *w = ps.w0[i];
        for (int k = 0; k < l; ++k) {
            *h = (*h + 1) / 2;
            *w = (*w + 1) / 2;
        }
    };
    cudaError_t e;
    int l = first;
    while (l < ps.nlev) {
        const int m = ps.nlev - l < kTailMaxLevels ? ps.nlev - l : kTailMaxLevels;
        if (l >= 3 && m >= 2) {
            // levels l .. l+m-1 from level l-1 in one launch
            PyrTailArgs ta;
            memset(&ta, 0, sizeof(ta));
            for (int i = 0; i < ps.count; ++i) {
                ta.src[i] = ps.plane[i][l - 1];
                ta.src_pitch[i] = ps.pitch[i][l - 1];
                size(i, l - 1, &ta.h[i], &ta.w[i]);
                for (int j = 0; j < m; ++j) {
                    ta.dst[i][j] = const_cast<void*>(ps.plane[i][l + j]);
                    ta.dst_pitch[i][j] = ps.pitch[i][l + j];
                }
            }
            ta.count = ps.count;
            ta.levels = m;
            ta.pyr = ps.pyr;
            const int t = tr ? trace_begin(*tr, PANO_TRACE_PYR_TAIL, l, s) : -1;
            if ((e = launch_pyr_tail(ta, s)) != cudaSuccess) return e;
            if (tr) trace_end(*tr, t, s);
            ++*kernels;
            l += m;
            continue;
        }
        PyrDownArgs pa;
        memset(&pa, 0, sizeof(pa));
        for (int i = 0; i < ps.count; ++i) {
            pa.src[i] = ps.plane[i][l - 1];
            pa.src_pitch[i] = ps.pitch[i][l - 1];
            pa.dst[i] = const_cast<void*>(ps.plane[i][l]);
            pa.dst_pitch[i] = ps.pitch[i][l];
            size(i, l - 1, &pa.h[i], &pa.w[i]);
        }
        pa.count = ps.count;
        pa.pyr = ps.pyr;
        const int t = tr ? trace_begin(*tr, PANO_TRACE_PYR_DOWN, l, s) : -1;
        if ((e = launch_pyr_down(pa, s)) != cudaSuccess) return e;
        if (tr) trace_end(*tr, t, s);
        ++*kernels;
        ++l;
    }
    return cudaSuccess;
}

cudaError_t launch_pair_pyramid(pano_flow_ctx* c, const PairPlanes& pp, cudaStream_t s) {
    cudaError_t e;
    int first = 1;  // first level left to REDUCE
    if (pp.luma.count == 2 && c->nlev >= 2) {
        // level 0 and level 1 of both strips in one launch
        LumaReduceArgs lr;
        memset(&lr, 0, sizeof(lr));
        for (int i = 0; i < 2; ++i) {
            lr.in[i] = pp.luma.in[i];
            lr.l0[i] = pp.luma.out[i];
            lr.l0_pitch[i] = pp.luma.out_pitch[i];
            lr.l1[i] = c->pyr[i][1];
            lr.l1_pitch[i] = c->lev_pitch[1];
        }
        lr.count = 2;
        lr.pyr = pp.luma.pyr;
        int t = trace_begin(c->tr, PANO_TRACE_LUMA_REDUCE, 1, s);
        if ((e = launch_luma_reduce(lr, s)) != cudaSuccess) return e;
        trace_end(c->tr, t, s);
        c->launches++;
        first = 2;
    } else if (pp.luma.count > 0) {
        int t = trace_begin(c->tr, PANO_TRACE_LUMA, 0, s);
        if ((e = launch_luma(pp.luma, s)) != cudaSuccess) return e;
        trace_end(c->tr, t, s);
        c->launches++;
    }
    PyrSet ps;
    memset(&ps, 0, sizeof(ps));
    for (int si = 0; si < 2; ++si) {
        for (int l = 0; l < c->nlev; ++l) {
            ps.plane[si][l] = pp.plane[si][l];
            ps.pitch[si][l] = pp.pitch[si][l];
        }
        ps.h0[si] = pp.hs[0];
        ps.w0[si] = pp.ws[0];
    }
    ps.count = 2;
    ps.nlev = c->nlev;
    ps.pyr = pyr_type(c->p.pyr_dtype);
    int kernels = 0;
    e = launch_pyramid_rest(ps, first, &c->tr, s, &kernels);
    c->launches += kernels;
    return e;
}

void pair_lk_args(const pano_flow_ctx* c, const PairPlanes& pp, int l, float* flow_LtoR, float* flow_RtoL,
                  LkArgs* ka) {
    const int nlev = c->nlev;
    float* out[2] = {flow_LtoR, flow_RtoL};
    memset(ka, 0, sizeof(*ka));
    for (int d = 0; d < 2; ++d) {
        // direction 0: FlowLtoR (template L, target R); 1: FlowRtoL
        ka->dir[d].T = pp.plane[d][l];
        ka->dir[d].pitchT = pp.pitch[d][l];
        ka->dir[d].J = pp.plane[1 - d][l];
        ka->dir[d].pitchJ = pp.pitch[1 - d][l];
        ka->dir[d].uin = l == nlev - 1 ? nullptr : c->flw[d][l + 1];
        ka->dir[d].uin_pitch = l == nlev - 1 ? 0 : c->flow_pitch[l + 1];
        ka->dir[d].uout = l == 0 ? out[d] : c->flw[d][l];
        ka->dir[d].uout_pitch = l == 0 ? pp.ws[0] : c->flow_pitch[l];
    }
    ka->h = pp.hs[l];
    ka->w = pp.ws[l];
    ka->in_h = l == nlev - 1 ? 0 : pp.hs[l + 1];
    ka->in_w = l == nlev - 1 ? 0 : pp.ws[l + 1];
    ka->mode = l == nlev - 1 ? 0 : 1;
    ka->iters = c->p.iters;
    ka->radius = c->p.radius;
    ka->lambda = c->p.lambda;
    lk_level_tile(ka->w, ka->h, c->tile_w, c->tile_h, &ka->tile_w, &ka->tile_h);
    ka->pyr = pyr_type(c->p.pyr_dtype);
}

}  // namespace pano

extern "C" {

void pano_flow_params_default(pano_flow_params* p) {
    if (!p) return;
    p->levels = 4;
    p->iters = 5;
    p->radius = 2;
    p->lambda = 1e-2f;
    p->soft_sharpness = 10.0f;
    p->flow_mag_coef = 20.0f;
    p->pyr_dtype = PANO_F32;
}

const char* pano_last_error(const pano_flow_ctx*) { return g_err; }

pano_status pano_flow_create(const pano_flow_params* p, int max_h, int max_w, int max_c,
                             pano_flow_ctx** out) {
    if (!out) return fail(PANO_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    pano_status st = check_params(p);
    if (st != PANO_OK) return st;
    if (max_h < 1 || max_w < 1) return fail(PANO_ERR_INVALID_ARG, "max size %dx%d", max_h, max_w);
    if (max_c != 1 && max_c != 3) return fail(PANO_ERR_INVALID_ARG, "max_c %d (1 or 3)", max_c);
    if ((double)max_h * (double)align_up((size_t)max_w * 3, 64) > (double)INT_MAX)
        return fail(PANO_ERR_UNSUPPORTED, "strip too large for 32-bit offsets");
    int max_smem = 0;
    if ((st = ensure_lk_ready(&max_smem)) != PANO_OK) return st;
    int tw = 0, th = 0;
    if (!pick_tile(p->iters, p->radius, max_smem, &tw, &th))
        return fail(PANO_ERR_UNSUPPORTED, "iters * radius = %d needs more shared memory than the device has",
                    p->iters * p->radius);

    pano_flow_ctx* c = new (std::nothrow) pano_flow_ctx;
    if (!c) return fail(PANO_ERR_OOM, "host allocation failed");
    memset(c, 0, sizeof(*c));
    c->p = *p;
    c->max_h = max_h;
    c->max_w = max_w;
    c->max_c = max_c;
    c->nlev = p->levels;
    c->tile_w = tw;
    c->tile_h = th;
    cudaGetDevice(&c->device);
    size_t off[2][2][kMaxLevels];
    size_t total = 0;
    for (int l = 0; l < c->nlev; ++l) {
        c->lev_h[l] = l == 0 ? max_h : (c->lev_h[l - 1] + 1) / 2;
        c->lev_w[l] = l == 0 ? max_w : (c->lev_w[l - 1] + 1) / 2;
        c->lev_pitch[l] = (int)align_up(c->lev_w[l], 32);
        c->flow_pitch[l] = (int)align_up(c->lev_w[l], 16);
    }
    for (int s = 0; s < 2; ++s)
        for (int l = 0; l < c->nlev; ++l) {
            off[0][s][l] = total;
            total += align_up((size_t)c->lev_pitch[l] * c->lev_h[l] * (size_t)elem_size(p->pyr_dtype), 256);
        }
    for (int d = 0; d < 2; ++d)
        for (int l = 1; l < c->nlev; ++l) {
            off[1][d][l] = total;
            total += align_up((size_t)c->flow_pitch[l] * c->lev_h[l] * sizeof(float2), 256);
        }
    cudaError_t e = device_alloc(&c->buf, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return fail(PANO_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", total, cudaGetErrorString(e));
    }
    c->buf_bytes = total;
    char* b = static_cast<char*>(c->buf);
    for (int s = 0; s < 2; ++s)
        for (int l = 0; l < c->nlev; ++l) c->pyr[s][l] = b + off[0][s][l];
    for (int d = 0; d < 2; ++d)
        for (int l = 1; l < c->nlev; ++l) c->flw[d][l] = reinterpret_cast<float*>(b + off[1][d][l]);
    *out = c;
    return PANO_OK;
}

pano_status pano_flow_destroy(pano_flow_ctx* c) {
    if (!c) return PANO_OK;
    trace_free(c->tr);
    cudaError_t e = c->buf ? cudaFree(c->buf) : cudaSuccess;
    delete c;
    if (e != cudaSuccess) return cuda_fail(e, "cudaFree");
    return PANO_OK;
}

pano_status pano_flow_pair(pano_flow_ctx* c, const pano_image* L, const pano_image* R,
                           float* flow_LtoR, float* flow_RtoL, void* cuda_stream) {
    pano_status st = check_pair_call(c, L, R, flow_LtoR, flow_RtoL);
    if (st != PANO_OK) return st;
    NvtxRange range("pano_flow_pair");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    PairPlanes pp;
    pair_planes(c, L, R, &pp);
    cudaError_t e;
    {
        NvtxRange r("pyramid");
        if ((e = launch_pair_pyramid(c, pp, s)) != cudaSuccess) return cuda_fail(e, "pyramid launch");
        if ((e = debug_check(s)) != cudaSuccess) return cuda_fail(e, "pyramid (PANO_DEBUG=sync)");
    }
    for (int l = c->nlev - 1; l >= 0; --l) {
        NvtxRange r("LK level");
        LkArgs ka;
        pair_lk_args(c, pp, l, flow_LtoR, flow_RtoL, &ka);
        int t = trace_begin(c->tr, PANO_TRACE_LK, l, s);
        if ((e = launch_lk_level(ka, 2, s)) != cudaSuccess) return cuda_fail(e, "LK launch");
        trace_end(c->tr, t, s);
        c->launches++;
        if ((e = debug_check(s)) != cudaSuccess) return cuda_fail(e, "LK level (PANO_DEBUG=sync)");
    }
    return PANO_OK;
}

pano_status pano_blend_pair(pano_flow_ctx* c, const pano_image* L, const pano_image* R,
                            const float* flow_LtoR, const float* flow_RtoL, const float* blend,
                            pano_image* F, void* cuda_stream) {
    if (!c) return fail(PANO_ERR_INVALID_ARG, "context is NULL");
    pano_status st;
    if ((st = check_image(L, "L")) != PANO_OK) return st;
    if ((st = check_image(R, "R")) != PANO_OK) return st;
    if ((st = check_image(F, "F")) != PANO_OK) return st;
    if ((st = check_same(L, R, "L", "R")) != PANO_OK) return st;
    if ((st = check_same(L, F, "L", "F")) != PANO_OK) return st;
    if ((st = check_flow(flow_LtoR, "flow_LtoR")) != PANO_OK) return st;
    if ((st = check_flow(flow_RtoL, "flow_RtoL")) != PANO_OK) return st;
    if (blend && ((uintptr_t)blend) % 4) return fail(PANO_ERR_INVALID_ARG, "blend is not 4-byte aligned");
    const size_t fb = (size_t)F->h * F->pitch_bytes;
    if (overlaps(F->data, fb, L->data, (size_t)L->h * L->pitch_bytes) ||
        overlaps(F->data, fb, R->data, (size_t)R->h * R->pitch_bytes))
        return fail(PANO_ERR_INVALID_ARG, "F overlaps an input strip");
    BlendArgs a;
    a.L = desc(L);
    a.R = desc(R);
    a.flowLR = reinterpret_cast<const float2*>(flow_LtoR);
    a.flowRL = reinterpret_cast<const float2*>(flow_RtoL);
    a.blend = blend;
    a.F = F->data;
    a.F_pitch_bytes = (long long)F->pitch_bytes;
    a.k_sharp = c->p.soft_sharpness;
    a.k_mag = c->p.flow_mag_coef;
    NvtxRange range("pano_blend_pair");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int t = trace_begin(c->tr, PANO_TRACE_BLEND, 0, s);
    cudaError_t e = launch_blend(a, s);
    if (e != cudaSuccess) return cuda_fail(e, "blend launch");
    trace_end(c->tr, t, s);
    c->launches++;
    if ((e = debug_check(s)) != cudaSuccess) return cuda_fail(e, "blend (PANO_DEBUG=sync)");
    return PANO_OK;
}

pano_status pano_compose_pair(const pano_flow_params* p, const pano_image* L, const pano_image* R,
                              const unsigned char* label, size_t label_pitch, const float* blend, int blend_pitch,
                              const float* flow_LtoR, const float* flow_RtoL, int flow_y0, int flow_x0,
                              int flow_h, int flow_w, pano_image* F, void* cuda_stream) {
    if (!p) return fail(PANO_ERR_INVALID_ARG, "params is NULL");
    if (!(p->soft_sharpness > -1e30f && p->soft_sharpness < 1e30f) || !(p->flow_mag_coef > -1e30f && p->flow_mag_coef < 1e30f))
        return fail(PANO_ERR_INVALID_ARG, "soft_sharpness and flow_mag_coef must be finite");
    pano_status st;
    if ((st = check_image(L, "L")) != PANO_OK) return st;
    if ((st = check_image(R, "R")) != PANO_OK) return st;
    if ((st = check_image(F, "F")) != PANO_OK) return st;
    if ((st = check_same(L, R, "L", "R")) != PANO_OK) return st;
    if ((st = check_same(L, F, "L", "F")) != PANO_OK) return st;
    const int h = L->h, w = L->w;
    if (!label || label_pitch < (size_t)w) return fail(PANO_ERR_INVALID_ARG, "label is NULL or its pitch < w");
    if (!blend || ((uintptr_t)blend) % 4 || blend_pitch < w)
        return fail(PANO_ERR_INVALID_ARG, "blend is NULL, not 4-byte aligned or its pitch < w");
    if (flow_h < 1 || flow_w < 1 || flow_y0 < 0 || flow_x0 < 0 || flow_h > h - flow_y0 || flow_w > w - flow_x0)
        return fail(PANO_ERR_INVALID_ARG, "flow crop %dx%d at (%d, %d) is not inside the %dx%d canvas", flow_h,
                    flow_w, flow_y0, flow_x0, h, w);
    if ((st = check_flow(flow_LtoR, "flow_LtoR")) != PANO_OK) return st;
    if ((st = check_flow(flow_RtoL, "flow_RtoL")) != PANO_OK) return st;
    const size_t fb = (size_t)F->h * F->pitch_bytes, nflow = (size_t)flow_h * flow_w * 8;
    if (overlaps(F->data, fb, L->data, (size_t)L->h * L->pitch_bytes) ||
        overlaps(F->data, fb, R->data, (size_t)R->h * R->pitch_bytes) ||
        overlaps(F->data, fb, label, (size_t)h * label_pitch) ||
        overlaps(F->data, fb, blend, (size_t)h * blend_pitch * sizeof(float)) ||
        overlaps(F->data, fb, flow_LtoR, nflow) || overlaps(F->data, fb, flow_RtoL, nflow))
        return fail(PANO_ERR_INVALID_ARG, "F overlaps an input");
    ComposeArgs a;
    a.L = desc(L);
    a.R = desc(R);
    a.label = label;
    a.label_pitch = (long long)label_pitch;
    a.blend = blend;
    a.blend_pitch = blend_pitch;
    a.flowLR = reinterpret_cast<const float2*>(flow_LtoR);
    a.flowRL = reinterpret_cast<const float2*>(flow_RtoL);
    a.fy0 = flow_y0;
    a.fx0 = flow_x0;
    a.fh = flow_h;
    a.fw = flow_w;
    a.F = F->data;
    a.F_pitch_bytes = (long long)F->pitch_bytes;
    a.k_sharp = p->soft_sharpness;
    a.k_mag = p->flow_mag_coef;
    a.inv_fw = 1.0f / (float)flow_w;
    NvtxRange range("pano_compose_pair");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = launch_compose(a, s);
    if (e != cudaSuccess) return cuda_fail(e, "compose launch");
    if ((e = debug_check(s)) != cudaSuccess) return cuda_fail(e, "compose (PANO_DEBUG=sync)");
    return PANO_OK;
}

pano_status pano_debug_bounds(unsigned* out) {
    if (!out) return fail(PANO_ERR_INVALID_ARG, "out is NULL");
    out[0] = out[1] = out[2] = out[3] = 0;
#ifdef PANO_BOUNDS_CHECK
    cudaError_t e;
    if ((e = bounds_read_lk_stream(out)) != cudaSuccess || (e = bounds_read_lk_stream_bf16(out)) != cudaSuccess ||
        (e = bounds_read_lk_stream_f16(out)) != cudaSuccess || (e = bounds_read_lk_tile(out)) != cudaSuccess ||
        (e = bounds_read_pyramid(out)) != cudaSuccess || (e = bounds_read_blend(out)) != cudaSuccess ||
        (e = bounds_read_edt(out)) != cudaSuccess || (e = bounds_read_refine(out)) != cudaSuccess)
        return cuda_fail(e, "reading the index-check records");
    return PANO_OK;
#else
    return fail(PANO_ERR_UNSUPPORTED, "this build has no index checks (build the check variant)");
#endif
}

pano_status pano_trace_enable(pano_flow_ctx* c, unsigned kind_mask, int capacity) {
    if (!c) return fail(PANO_ERR_INVALID_ARG, "context is NULL");
    return trace_enable(c->tr, kind_mask, capacity);
}

pano_status pano_trace_read(pano_flow_ctx* c, pano_trace_record* out, int max_records, int* n_out) {
    if (!c) return fail(PANO_ERR_INVALID_ARG, "NULL argument");
    return trace_read(c->tr, out, max_records, n_out);
}

unsigned long long pano_flow_launches(const pano_flow_ctx* c) { return c ? c->launches : 0ull; }

// ---------------------------------------------------------------------------
// Stage entry points
// ---------------------------------------------------------------------------

pano_status pano_stage_luma(const pano_image* in, float* Y, int y_pitch, void* cuda_stream) {
    pano_status st;
    if ((st = check_image(in, "in")) != PANO_OK) return st;
    if (!Y || ((uintptr_t)Y) % 4) return fail(PANO_ERR_INVALID_ARG, "Y is NULL or misaligned");
    if (y_pitch < in->w) return fail(PANO_ERR_INVALID_ARG, "y_pitch %d < w %d", y_pitch, in->w);
    LumaArgs la;
    memset(&la, 0, sizeof(la));
    la.in[0] = desc(in);
    la.out[0] = Y;
    la.out_pitch[0] = y_pitch;
    la.count = 1;
    cudaError_t e = launch_luma(la, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? PANO_OK : cuda_fail(e, "luma launch");
}

pano_status pano_stage_luma_pyr(const pano_image* in, float* Y, int y_pitch, float* Y1, int y1_pitch,
                                void* cuda_stream) {
    pano_status st;
    if ((st = check_image(in, "in")) != PANO_OK) return st;
    if (!Y || !Y1 || ((uintptr_t)Y) % 4 || ((uintptr_t)Y1) % 4)
        return fail(PANO_ERR_INVALID_ARG, "Y or Y1 is NULL or misaligned");
    if (y_pitch < in->w || y1_pitch < (in->w + 1) / 2)
        return fail(PANO_ERR_INVALID_ARG, "y_pitch %d or y1_pitch %d too small", y_pitch, y1_pitch);
    LumaReduceArgs lr;
    memset(&lr, 0, sizeof(lr));
    lr.in[0] = desc(in);
    lr.l0[0] = Y;
    lr.l0_pitch[0] = y_pitch;
    lr.l1[0] = Y1;
    lr.l1_pitch[0] = y1_pitch;
    lr.count = 1;
    cudaError_t e = launch_luma_reduce(lr, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? PANO_OK : cuda_fail(e, "luma/REDUCE launch");
}

pano_status pano_stage_pyramid(const float* Y, int h, int w, int pitch, float* const* levels, const int* pitches,
                               int nlev, void* cuda_stream) {
    if (!Y || ((uintptr_t)Y) % 4) return fail(PANO_ERR_INVALID_ARG, "Y is NULL or misaligned");
    if (h < 1 || w < 1 || pitch < w) return fail(PANO_ERR_INVALID_ARG, "bad size or pitch");
    if (nlev < 2 || nlev > kMaxLevels) return fail(PANO_ERR_INVALID_ARG, "nlev %d not in 2..%d", nlev, kMaxLevels);
    if (!levels || !pitches) return fail(PANO_ERR_INVALID_ARG, "levels or pitches is NULL");
    PyrSet ps;
    memset(&ps, 0, sizeof(ps));
    ps.plane[0][0] = Y;
    ps.pitch[0][0] = pitch;
    int lh = h, lw = w;
    for (int l = 1; l < nlev; ++l) {
        lh = (lh + 1) / 2;
        lw = (lw + 1) / 2;
        if (!levels[l - 1] || ((uintptr_t)levels[l - 1]) % 4)
            return fail(PANO_ERR_INVALID_ARG, "level %d is NULL or misaligned", l);
        if (pitches[l - 1] < lw) return fail(PANO_ERR_INVALID_ARG, "pitch of level %d < %d", l, lw);
        ps.plane[0][l] = levels[l - 1];
        ps.pitch[0][l] = pitches[l - 1];
    }
    ps.h0[0] = h;
    ps.w0[0] = w;
    ps.count = 1;
    ps.nlev = nlev;
    int st_ms = 0;
    pano_status st;
    if ((st = ensure_lk_ready(&st_ms)) != PANO_OK) return st;
    int kernels = 0;
    cudaError_t e = launch_pyramid_rest(ps, 1, nullptr, static_cast<cudaStream_t>(cuda_stream), &kernels);
    return e == cudaSuccess ? PANO_OK : cuda_fail(e, "pyramid launch");
}

pano_status pano_stage_pyr_down(const float* src, int h, int w, int src_pitch, float* dst, int dst_pitch,
                                void* cuda_stream) {
    if (!src || !dst || ((uintptr_t)src) % 4 || ((uintptr_t)dst) % 4)
        return fail(PANO_ERR_INVALID_ARG, "src or dst NULL or misaligned");
    if (h < 1 || w < 1 || src_pitch < w || dst_pitch < (w + 1) / 2)
        return fail(PANO_ERR_INVALID_ARG, "bad size or pitch");
    PyrDownArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.src[0] = src;
    pa.dst[0] = dst;
    pa.src_pitch[0] = src_pitch;
    pa.dst_pitch[0] = dst_pitch;
    pa.h[0] = h;
    pa.w[0] = w;
    pa.count = 1;
    cudaError_t e = launch_pyr_down(pa, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? PANO_OK : cuda_fail(e, "pyramid launch");
}

pano_status pano_stage_lk(const float* T, const float* J, int h, int w, int pitch, const float* flow_in,
                          int in_h, int in_w, int upsample, float* flow_out, int iters, int radius,
                          float lambda, void* cuda_stream) {
    // the stage entry point runs the streamed kernel whenever it applies
    return pano_stage_lk_kernel(T, J, h, w, pitch, flow_in, in_h, in_w, upsample, flow_out, iters, radius, lambda,
                                lk_stream_supports(iters, radius) ? PANO_LK_STREAM : PANO_LK_TILE, cuda_stream);
}

pano_status pano_stage_lk_kernel(const float* T, const float* J, int h, int w, int pitch, const float* flow_in,
                                 int in_h, int in_w, int upsample, float* flow_out, int iters, int radius,
                                 float lambda, int kernel, void* cuda_stream) {
    if (kernel < PANO_LK_AUTO || kernel > PANO_LK_TILE)
        return fail(PANO_ERR_INVALID_ARG, "kernel %d is not a PANO_LK_* value", kernel);
    if (!T || !J || ((uintptr_t)T) % 4 || ((uintptr_t)J) % 4)
        return fail(PANO_ERR_INVALID_ARG, "T or J NULL or misaligned");
    if (h < 1 || w < 1 || pitch < w) return fail(PANO_ERR_INVALID_ARG, "bad size or pitch");
    pano_status st;
    if ((st = check_flow(flow_out, "flow_out")) != PANO_OK) return st;
    if (flow_in && ((uintptr_t)flow_in) % 8) return fail(PANO_ERR_INVALID_ARG, "flow_in is not 8-byte aligned");
    if (iters < 0 || iters > 16 || radius < 1 || radius > 3 || !(lambda >= 0.f))
        return fail(PANO_ERR_INVALID_ARG, "iters, radius or lambda out of range");
    if (kernel == PANO_LK_STREAM && !lk_stream_supports(iters, radius))
        return fail(PANO_ERR_UNSUPPORTED, "the streamed kernel needs 1 <= iters <= 5");
    int ih = h, iw = w;
    if (flow_in && upsample) {
        if (in_h < 1 || in_w < 1) return fail(PANO_ERR_INVALID_ARG, "coarse flow size %dx%d", in_h, in_w);
        ih = in_h;
        iw = in_w;
    }
    if (flow_in && overlaps(flow_in, (size_t)ih * iw * 8, flow_out, (size_t)h * w * 8))
        return fail(PANO_ERR_INVALID_ARG, "flow_in and flow_out overlap");
    int max_smem = 0;
    if ((st = ensure_lk_ready(&max_smem)) != PANO_OK) return st;
    LkArgs ka;
    memset(&ka, 0, sizeof(ka));
    if (!pick_tile(iters, radius, max_smem, &ka.tile_w, &ka.tile_h))
        return fail(PANO_ERR_UNSUPPORTED, "iters * radius too large for shared memory");
    ka.dir[0].T = T;
    ka.dir[0].J = J;
    ka.dir[0].pitchT = ka.dir[0].pitchJ = pitch;
    ka.dir[0].uin = flow_in;
    ka.dir[0].uin_pitch = iw;
    ka.dir[0].uout = flow_out;
    ka.dir[0].uout_pitch = w;
    ka.h = h;
    ka.w = w;
    ka.in_h = ih;
    ka.in_w = iw;
    ka.mode = flow_in ? (upsample ? 1 : 2) : 0;
    ka.iters = iters;
    ka.radius = radius;
    ka.lambda = lambda;
    ka.pyr = kPyrF32;
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e;
    switch (kernel) {
        case PANO_LK_AUTO: e = launch_lk_level(ka, 1, s); break;
        case PANO_LK_STREAM: e = launch_lk_stream(ka, 1, s); break;
        default: e = launch_lk_tile(ka, 1, s); break;
    }
    return e == cudaSuccess ? PANO_OK : cuda_fail(e, "LK launch");
}

pano_status pano_stage_warp(const pano_image* src, const float* flow, float scale, pano_image* dst,
                            void* cuda_stream) {
    pano_status st;
    if ((st = check_image(src, "src")) != PANO_OK) return st;
    if ((st = check_image(dst, "dst")) != PANO_OK) return st;
    if ((st = check_flow(flow, "flow")) != PANO_OK) return st;
    if (dst->dtype != PANO_F32 || dst->h != src->h || dst->w != src->w || dst->c != src->c)
        return fail(PANO_ERR_INVALID_ARG, "dst must be float32 with the size and channels of src");
    WarpArgs a;
    a.src = desc(src);
    a.flow = reinterpret_cast<const float2*>(flow);
    a.scale = scale;
    a.dst = static_cast<float*>(dst->data);
    a.dst_pitch_bytes = (long long)dst->pitch_bytes;
    cudaError_t e = launch_warp(a, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? PANO_OK : cuda_fail(e, "warp launch");
}

pano_status pano_energy_grad(const float* T, const float* J, int h, int w, int pitch, const float* u, float alpha,
                             double* energy, float* grad_u, float* grad_T, float* grad_J, void* cuda_stream) {
    if (!T || !J || !u) return fail(PANO_ERR_INVALID_ARG, "T, J or u is NULL");
    if (h < 1 || w < 1 || pitch < w) return fail(PANO_ERR_INVALID_ARG, "bad size or pitch");
    if (((uintptr_t)T) % 4 || ((uintptr_t)J) % 4 || ((uintptr_t)u) % 8)
        return fail(PANO_ERR_INVALID_ARG, "T, J or u misaligned");
    if ((energy && ((uintptr_t)energy) % 8) || (grad_u && ((uintptr_t)grad_u) % 8) ||
        (grad_T && ((uintptr_t)grad_T) % 4) || (grad_J && ((uintptr_t)grad_J) % 4))
        return fail(PANO_ERR_INVALID_ARG, "output misaligned");
    if (!(alpha >= 0.f) || !(alpha < 1e30f)) return fail(PANO_ERR_INVALID_ARG, "alpha must be finite and >= 0");
    if ((double)h * (double)pitch > (double)INT_MAX) return fail(PANO_ERR_UNSUPPORTED, "more than 2^31 elements");
    EnergyArgs a;
    a.T = T;
    a.J = J;
    a.u = u;
    a.h = h;
    a.w = w;
    a.pitch = pitch;
    a.alpha = alpha;
    a.energy = energy;
    a.grad_u = grad_u;
    a.grad_T = grad_T;
    a.grad_J = grad_J;
    cudaError_t e = launch_energy_grad(a, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? PANO_OK : cuda_fail(e, "energy launch");
}

pano_status pano_stage_pyr_down_adjoint(const float* gdst, int h, int w, int dst_pitch, float* gsrc, int src_pitch,
                                        void* cuda_stream) {
    if (!gdst || !gsrc || ((uintptr_t)gdst) % 4 || ((uintptr_t)gsrc) % 4)
        return fail(PANO_ERR_INVALID_ARG, "gdst or gsrc NULL or misaligned");
    if (h < 1 || w < 1 || src_pitch < w || dst_pitch < (w + 1) / 2)
        return fail(PANO_ERR_INVALID_ARG, "bad size or pitch");
    cudaError_t e = launch_pyr_down_adjoint(gdst, h, w, dst_pitch, gsrc, src_pitch, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? PANO_OK : cuda_fail(e, "REDUCE adjoint launch");
}

}  // extern "C"
