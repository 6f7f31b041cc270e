// flow_static.cu -- pano_flow_pair_static: the bidirectional flow of
// pano_flow_pair for callers that must not allocate device memory.
//
// Who needs it: a host program that owns the whole GPU through its own memory
// pool (a serving process that reserves all of HBM at start-up and forbids
// any other allocation), or a loop with a per-frame deadline, where
// cudaMalloc / cudaFree would add their latency and their device-wide
// synchronisation to the frame. Such callers can pass their own input and
// output buffers but cannot let the library create a context, because
// pano_flow_create allocates the pyramids and coarse flows with cudaMalloc.
//
// This entry point keeps that scratch in one fixed file-scope device array
// of PANO_STATIC_SCRATCH_BYTES instead. Every GPU that loads the library
// holds the array until the process exits. The kernels are the ones
// pano_flow_pair launches; only where their scratch lives differs.
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "ctx.h"
#include "pano_flow.h"

using namespace pano;

// The shared scratch. All calls, on every stream, use this one array.
static __device__ __align__(256) unsigned char g_static_scratch[PANO_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    bool done = false;
    unsigned char* scratch = nullptr;  // device address of g_static_scratch
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

// Once per device, with that device current: the device address of the
// scratch array (host code cannot use the symbol itself). The kernels'
// shared-memory limits are set by ensure_lk_ready, as for a context.
pano_status setup_current_device(DeviceSetup** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(PANO_ERR_UNSUPPORTED, "device index %d", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup& s = g_setup[dev];
    if (!s.done) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        s.scratch = static_cast<unsigned char*>(p);
        s.done = true;
    }
    *out = &s;
    return PANO_OK;
}

// Bytes of scratch a strip of h x w pixels needs: both luma pyramids and the
// coarse-level flows of both directions, laid out as the entry point carves them.
size_t static_scratch_bytes(int h, int w, int levels) {
    if (h < 1 || w < 1 || levels < 1 || levels > kMaxLevels) return 0;
    size_t total = 0;
    int lh = h, lw = w;
    for (int l = 0; l < levels; ++l) {
        total += 2 * align_up((size_t)align_up(lw, 32) * lh * sizeof(float), 256);      // both pyramids
        if (l > 0) total += 2 * align_up((size_t)align_up(lw, 16) * lh * 8, 256);      // both flows
        lh = (lh + 1) / 2;
        lw = (lw + 1) / 2;
    }
    return total;
}

}  // namespace

extern "C" {

pano_status pano_flow_pair_static(const pano_flow_params* p, const pano_image* L, const pano_image* R,
                                  float* flow_LtoR, float* flow_RtoL, void* cuda_stream) {
    // the argument checks of pano_flow_pair, except that there is no
    // context: its maximum sizes are replaced by the size of the scratch
    pano_status st;
    if ((st = check_params(p)) != PANO_OK) return st;
    if (p->pyr_dtype != PANO_F32)
        return fail(PANO_ERR_UNSUPPORTED, "pyramid dtype %d: this entry point keeps float32 pyramids", p->pyr_dtype);
    if ((st = check_image(L, "L")) != PANO_OK) return st;
    if ((st = check_image(R, "R")) != PANO_OK) return st;
    if ((st = check_same(L, R, "L", "R")) != PANO_OK) return st;
    if ((st = check_flow(flow_LtoR, "flow_LtoR")) != PANO_OK) return st;
    if ((st = check_flow(flow_RtoL, "flow_RtoL")) != PANO_OK) return st;
    const size_t fbytes = (size_t)L->h * L->w * 2 * sizeof(float);
    if (overlaps(flow_LtoR, fbytes, flow_RtoL, fbytes)) return fail(PANO_ERR_INVALID_ARG, "the two flows overlap");
    const size_t need = static_scratch_bytes(L->h, L->w, p->levels);
    if (need > (size_t)PANO_STATIC_SCRATCH_BYTES)
        return fail(PANO_ERR_INVALID_ARG,
                    "strip %dx%d with %d levels needs %zu bytes of scratch; the fixed scratch holds %zu", L->h,
                    L->w, p->levels, need, (size_t)PANO_STATIC_SCRATCH_BYTES);
    int max_smem = 0;
    if ((st = ensure_lk_ready(&max_smem)) != PANO_OK) return st;
    DeviceSetup* ds = nullptr;
    if ((st = setup_current_device(&ds)) != PANO_OK) return st;
    int tw = 0, th = 0;
    if (!pick_tile(p->iters, p->radius, max_smem, &tw, &th))
        return fail(PANO_ERR_UNSUPPORTED, "iters * radius = %d needs more shared memory than the device has",
                    p->iters * p->radius);
    NvtxRange range("pano_flow_pair_static");

    // Carve the fixed scratch exactly as static_scratch_bytes counts it.
    const int nlev = p->levels;
    int hs[kMaxLevels], ws[kMaxLevels], lp[kMaxLevels], fp[kMaxLevels];
    float* pyr[2][kMaxLevels] = {};
    float* flw[2][kMaxLevels] = {};
    unsigned char* cur = ds->scratch;
    for (int l = 0; l < nlev; ++l) {
        hs[l] = l == 0 ? L->h : (hs[l - 1] + 1) / 2;
        ws[l] = l == 0 ? L->w : (ws[l - 1] + 1) / 2;
        lp[l] = (int)align_up(ws[l], 32);
        fp[l] = (int)align_up(ws[l], 16);
        for (int s = 0; s < 2; ++s) {
            pyr[s][l] = reinterpret_cast<float*>(cur);
            cur += align_up((size_t)lp[l] * hs[l] * sizeof(float), 256);
        }
        if (l > 0)
            for (int d = 0; d < 2; ++d) {
                flw[d][l] = reinterpret_cast<float*>(cur);
                cur += align_up((size_t)fp[l] * hs[l] * 8, 256);
            }
    }
    // Nothing in the scratch has to start at zero: every level and every
    // coarse flow is written in full by this call before it is read.
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const pano_image* img[2] = {L, R};
    const float* plane[2][kMaxLevels];
    int ppitch[2][kMaxLevels];
    LumaArgs la;
    memset(&la, 0, sizeof(la));
    la.pyr = kPyrF32;
    for (int si = 0; si < 2; ++si) {
        for (int l = 0; l < nlev; ++l) {
            plane[si][l] = pyr[si][l];
            ppitch[si][l] = lp[l];
        }
        if (img[si]->dtype == PANO_F32 && img[si]->c == 1) {
            // a one-channel float strip is its own luma
            plane[si][0] = static_cast<const float*>(img[si]->data);
            ppitch[si][0] = (int)(img[si]->pitch_bytes / sizeof(float));
        } else {
            la.in[la.count] = desc(img[si]);
            la.out[la.count] = pyr[si][0];
            la.out_pitch[la.count] = lp[0];
            la.count++;
        }
    }
    cudaError_t e;
    int first = 1;  // first level left to REDUCE
    if (la.count == 2 && nlev >= 2) {
        // level 0 and level 1 of both strips in one launch (as pano_flow_pair)
        LumaReduceArgs lr;
        memset(&lr, 0, sizeof(lr));
        for (int i = 0; i < 2; ++i) {
            lr.in[i] = la.in[i];
            lr.l0[i] = la.out[i];
            lr.l0_pitch[i] = la.out_pitch[i];
            lr.l1[i] = pyr[i][1];
            lr.l1_pitch[i] = lp[1];
        }
        lr.count = 2;
        lr.pyr = kPyrF32;
        if ((e = launch_luma_reduce(lr, s)) != cudaSuccess) return cuda_fail(e, "luma launch");
        first = 2;
    } else if (la.count > 0 && (e = launch_luma(la, s)) != cudaSuccess) {
        return cuda_fail(e, "luma launch");
    }
    {
        // the other levels (the same launch sequence as pano_flow_pair)
        PyrSet ps;
        memset(&ps, 0, sizeof(ps));
        for (int si = 0; si < 2; ++si) {
            for (int l = 0; l < nlev; ++l) {
                ps.plane[si][l] = l == 0 ? (const void*)plane[si][0] : (const void*)pyr[si][l];
                ps.pitch[si][l] = l == 0 ? ppitch[si][0] : lp[l];
            }
            ps.h0[si] = hs[0];
            ps.w0[si] = ws[0];
        }
        ps.count = 2;
        ps.nlev = nlev;
        ps.pyr = kPyrF32;
        int kernels = 0;
        if ((e = launch_pyramid_rest(ps, first, nullptr, s, &kernels)) != cudaSuccess)
            return cuda_fail(e, "pyramid launch");
    }
    if ((e = debug_check(s)) != cudaSuccess) return cuda_fail(e, "pyramid (PANO_DEBUG=sync)");
    float* out[2] = {flow_LtoR, flow_RtoL};
    for (int l = nlev - 1; l >= 0; --l) {
        LkArgs ka;
        memset(&ka, 0, sizeof(ka));
        for (int d = 0; d < 2; ++d) {
            ka.dir[d].T = plane[d][l];
            ka.dir[d].pitchT = ppitch[d][l];
            ka.dir[d].J = plane[1 - d][l];
            ka.dir[d].pitchJ = ppitch[1 - d][l];
            ka.dir[d].uin = l == nlev - 1 ? nullptr : flw[d][l + 1];
            ka.dir[d].uin_pitch = l == nlev - 1 ? 0 : fp[l + 1];
            ka.dir[d].uout = l == 0 ? out[d] : flw[d][l];
            ka.dir[d].uout_pitch = l == 0 ? ws[0] : fp[l];
        }
        ka.h = hs[l];
        ka.w = ws[l];
        ka.in_h = l == nlev - 1 ? 0 : hs[l + 1];
        ka.in_w = l == nlev - 1 ? 0 : ws[l + 1];
        ka.mode = l == nlev - 1 ? 0 : 1;
        ka.iters = p->iters;
        ka.radius = p->radius;
        ka.lambda = p->lambda;
        ka.pyr = kPyrF32;
        lk_level_tile(ka.w, ka.h, tw, th, &ka.tile_w, &ka.tile_h);  // as pano_flow_pair
        if ((e = launch_lk_level(ka, 2, s)) != cudaSuccess) return cuda_fail(e, "LK launch");
        if ((e = debug_check(s)) != cudaSuccess) return cuda_fail(e, "LK level (PANO_DEBUG=sync)");
    }
    return PANO_OK;
}

}  // extern "C"
