// ctx.h -- internal: the flow context of the C ABI and the steps of
// pano_flow_pair that the multi-pair rig reuses. Not a public header.
#pragma once

#include "common.cuh"
#include "pano_flow.h"

namespace pano {

// Launch tracing of one context: events around selected launches.
struct Trace {
    unsigned mask;
    int cap, n;
    cudaEvent_t* ev;        // 2 * cap events: start, stop per record
    pano_trace_record* rec;
};

}  // namespace pano

struct pano_flow_ctx {
    pano_flow_params p;
    int max_h, max_w, max_c;
    int device;
    int nlev;
    int lev_h[pano::kMaxLevels], lev_w[pano::kMaxLevels];  // level sizes at the maximum strip size
    int lev_pitch[pano::kMaxLevels];                 // elements
    int flow_pitch[pano::kMaxLevels];                // float2 elements
    void* pyr[2][pano::kMaxLevels];                  // luma pyramids of L and R (pyr_dtype elements)
    float* flw[2][pano::kMaxLevels];                 // flows of levels >= 1, per direction
    void* buf;
    size_t buf_bytes;
    int tile_w, tile_h;
    unsigned long long launches;
    pano::Trace tr;
};

namespace pano {

// Plane pointers and pitches of every pyramid level of both strips of one
// call (level 0 of a one-channel float strip is the strip itself).
struct PairPlanes {
    const void* plane[2][kMaxLevels];  // PyrType of the context
    int pitch[2][kMaxLevels];
    int hs[kMaxLevels], ws[kMaxLevels];
    LumaArgs luma;  // level-0 conversions needed (count may be 0)
};

void pair_planes(const pano_flow_ctx* c, const pano_image* L, const pano_image* R, PairPlanes* pp);
// luma + REDUCE launches of one pair; returns the first launch error
cudaError_t launch_pair_pyramid(pano_flow_ctx* c, const PairPlanes& pp, cudaStream_t s);
// arguments of LK level l of one pair (both directions)
void pair_lk_args(const pano_flow_ctx* c, const PairPlanes& pp, int l, float* flow_LtoR, float* flow_RtoL,
                  LkArgs* ka);
pano_status check_pair_call(const pano_flow_ctx* c, const pano_image* L, const pano_image* R, const float* lr,
                            const float* rl);

// Argument checks and error reporting shared by the C entry points: each
// failing check stores its message for pano_last_error and returns the
// status.
pano_status fail(pano_status st, const char* fmt, ...);
pano_status cuda_fail(cudaError_t e, const char* what);
pano_status check_image(const pano_image* im, const char* name);
pano_status check_same(const pano_image* a, const pano_image* b, const char* na, const char* nb);
pano_status check_flow(const void* f, const char* name);
pano_status check_params(const pano_flow_params* p);
bool overlaps(const void* a, size_t na, const void* b, size_t nb);
int elem_size(int dtype);           // bytes of one element of a pano_dtype
int pyr_type(int pyr_dtype);        // PyrType of a pano_dtype
size_t align_up(size_t v, size_t a);
ImageDesc desc(const pano_image* im);
// largest tile of the LK tile kernel that fits max_smem bytes
bool pick_tile(int iters, int radius, int max_smem, int* tw, int* th);
// sets the kernels' shared-memory limits once per device; returns the limit
pano_status ensure_lk_ready(int* max_smem_out);

// The pyramid levels below level 1 (or 0): one REDUCE launch per level for
// levels 1 and 2, then launches of up to four levels each. plane/pitch give
// every level of every plane (level 0 of a plane may be the strip itself);
// h0/w0 the level-0 sizes. Launches are traced in *tr (if not null) and
// added to *kernels.
struct PyrSet {
    const void* plane[kMaxPlanes][kMaxLevels];
    int pitch[kMaxPlanes][kMaxLevels];
    int h0[kMaxPlanes], w0[kMaxPlanes];
    int count, nlev, pyr;
};
cudaError_t launch_pyramid_rest(const PyrSet& ps, int first, Trace* tr, cudaStream_t s, int* kernels);

// PANO_DEBUG: a comma-separated list read from the environment at each call.
//   sync        synchronise the stream after every stage of a call (outside
//               stream capture) and report the first failing stage
//   fail_alloc  make the device allocation of the next create calls fail
//               (the host-side failure path, without a GPU fault)
constexpr unsigned kDebugSync = 1u, kDebugFailAlloc = 2u;
unsigned debug_flags();
// cudaMalloc, or the simulated failure of PANO_DEBUG=fail_alloc
cudaError_t device_alloc(void** p, size_t bytes);
// with PANO_DEBUG=sync: the error of the work enqueued so far on s
cudaError_t debug_check(cudaStream_t s);

// An NVTX range around a host-side call (shown by profilers; free otherwise).
struct NvtxRange {
    explicit NvtxRange(const char* name);
    ~NvtxRange();
};

void trace_free(Trace& t);
pano_status trace_enable(Trace& t, unsigned kind_mask, int capacity);
pano_status trace_read(Trace& t, pano_trace_record* out, int max_records, int* n_out);
int trace_begin(Trace& t, unsigned kind, int level, cudaStream_t s);  // slot or -1
void trace_end(Trace& t, int slot, cudaStream_t s);

}  // namespace pano
