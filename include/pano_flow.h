/*
 * pano_flow.h -- C ABI of the GB300 (sm_103a) asymmetric bidirectional
 * optical-flow blend of two overlap strips.
 *
 * Method: Meng & Liu, "High-quality Panorama Stitching based on Asymmetric
 * Bidirectional Optical Flow", Section III-C. Two already-aligned overlap
 * strips OverlappedL / OverlappedR (Section III-C, the Area3 crop of images L
 * and R) are blended into F through
 *   - a Gaussian pyramid of each strip's luma,
 *   - dense pyramidal Lucas-Kanade flow in both directions, FlowLtoR and
 *     FlowRtoL (Section III-C-1),
 *   - the global blending coefficient Blend, Eq. (1) (Section III-C-2),
 *   - the flow warp and asymmetric softmax blend of Code 1 (Section III-C-3).
 *
 * Conventions shared by every call
 *   Memory      All image and flow pointers are CUDA device memory owned by
 *               the caller; the library never frees them. A context owns its
 *               own scratch (pyramids and coarse-level flows), allocated once
 *               by pano_flow_create and freed by pano_flow_destroy.
 *   Streams     Every call only enqueues work on `cuda_stream` (a
 *               cudaStream_t; NULL = the legacy default stream) and returns;
 *               outputs are valid once that stream reaches them. No call
 *               synchronises, allocates or frees device memory after
 *               pano_flow_create, so a sequence of calls can be captured in a
 *               CUDA graph. Use one context per stream; a context is not
 *               thread-safe. Call with the context's device current.
 *   Errors      Arguments are checked on the host before anything is
 *               enqueued; a call that fails its checks enqueues nothing and
 *               writes no output. CUDA errors map to PANO_ERR_CUDA. Nothing
 *               throws or exits across this boundary. pano_last_error()
 *               returns a message for the last failing call on the calling
 *               thread.
 *   Images      pano_image describes a row-major (h, w, c) image with
 *               interleaved channels: sample (y, x, k) is at
 *               data + y * pitch_bytes + (x * c + k) * element_size.
 *               PANO_U8 samples are read as value / 255; PANO_F32 samples are
 *               taken as they are (intended range [0, 1]).
 *   Flows       A flow field is (h, w, 2) float32, contiguous (row pitch
 *               w * 2 floats), 8-byte aligned: element [y][x][0] is the
 *               column offset, [y][x][1] the row offset, in pixels.
 *               FlowAtoB lives on A's grid and satisfies
 *               A(p) ~ B(p + FlowAtoB(p)) (Section III-C-1: the flow of
 *               OverlappedR relative to OverlappedL is FlowRtoL).
 *   Borders     Every sampler clamps to the edge of the strip.
 */
#ifndef PANO_FLOW_H
#define PANO_FLOW_H

#include <stddef.h>

#if defined(__GNUC__)
#define PANO_API __attribute__((visibility("default")))
#else
#define PANO_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pano_status {
    PANO_OK = 0,
    PANO_ERR_INVALID_ARG = 1,  /* null pointer, bad size, pitch or alignment */
    PANO_ERR_UNSUPPORTED = 2,  /* valid request this build does not implement */
    PANO_ERR_OOM = 3,          /* device allocation failed (create only) */
    PANO_ERR_CUDA = 4,         /* a CUDA call or launch failed */
    PANO_ERR_TIMEOUT = 5       /* reserved: a bounded device wait gave up */
} pano_status;

typedef enum pano_dtype {
    PANO_U8 = 0,
    PANO_F32 = 1,
    PANO_BF16 = 2,   /* pyramid storage only (pano_flow_params.pyr_dtype) */
    PANO_F16 = 3     /* pyramid storage only (pano_flow_params.pyr_dtype) */
} pano_dtype;

typedef struct pano_image {
    void* data;          /* device pointer, aligned to the element size */
    int h, w, c;         /* rows, columns, channels (1 or 3) */
    size_t pitch_bytes;  /* bytes between rows, >= w * c * element size */
    int dtype;           /* a pano_dtype */
} pano_image;

/* Method parameters. The paper publishes none of them (Section III-C-1
 * leaves the Lucas-Kanade parameters open; Section III-C-3 names
 * kSoftmaxSharpness and kFlowMagCoef without values). */
typedef struct pano_flow_params {
    int levels;           /* pyramid levels, 1..12 (default 4) */
    int iters;            /* Lucas-Kanade steps per level, 0..16 (default 5) */
    int radius;           /* window radius r, window (2r+1)^2, 1..3 (default 2) */
    float lambda;         /* damping towards the current flow, >= 0 (default 1e-2) */
    float soft_sharpness; /* kSoftmaxSharpness of Code 1 (default 10) */
    float flow_mag_coef;  /* kFlowMagCoef of Code 1 (default 20) */
    int pyr_dtype;        /* storage of the pyramid levels, luma included: PANO_F32 (default),
                             PANO_BF16 or PANO_F16 (rounded to nearest even when stored; all
                             arithmetic stays FP32). Not a choice the paper makes */
} pano_flow_params;

typedef struct pano_flow_ctx pano_flow_ctx;

/* Fill *p with the defaults listed above. */
PANO_API void pano_flow_params_default(pano_flow_params* p);

/* Create a context for strips of at most max_h x max_w pixels and max_c
 * channels on the current device, and allocate its scratch:
 * two pyramids of pyr_dtype levels (~ 2 * e * (4/3) * max_h * max_w bytes, e = 4
 * for PANO_F32 and 2 for the 16-bit types) and
 * the coarse-level flows of both directions (~ 2 * 8 * (1/3) * max_h * max_w
 * bytes). *out receives the context; on failure *out is NULL.
 * Errors: INVALID_ARG (null p/out, parameters out of range, sizes < 1),
 * UNSUPPORTED (sizes beyond 32-bit offsets), OOM, CUDA. */
PANO_API pano_status pano_flow_create(const pano_flow_params* p, int max_h, int max_w, int max_c,
                             pano_flow_ctx** out);

/* Asymmetric bidirectional optical flow of a strip pair (Section III-C-1):
 * FlowLtoR with L as template and R as target, FlowRtoL with the roles
 * exchanged, each by pyramidal Lucas-Kanade over the luma of the strips
 * (BT.601 for 3 channels). L and R must have the same h, w, c and dtype
 * (PANO_U8 or PANO_F32, c = 1 or 3, within the context's maxima).
 * flow_LtoR and flow_RtoL receive (h, w, 2) float32 fields as described
 * under "Flows"; they must not overlap each other or the inputs.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
PANO_API pano_status pano_flow_pair(pano_flow_ctx* ctx, const pano_image* L, const pano_image* R,
                           float* flow_LtoR, float* flow_RtoL, void* cuda_stream);

/* Code 1 (Section III-C-3), Area3 branch, for every pixel p of the strips:
 *   BlendL = 1 - Blend(p), BlendR = Blend(p)
 *   ColorL = L(p + (1 - BlendL) FlowRtoL(p)),  ColorR = R(p + (1 - BlendR) FlowLtoR(p))
 *   FlowL  = 1 + kFlowMagCoef |FlowRtoL(p)| / w,  FlowR = 1 + kFlowMagCoef |FlowLtoR(p)| / w
 *   F(p)   = softmax-weighted sum of ColorL and ColorR with exponents
 *            kSoftmaxSharpness * BlendL * FlowL and kSoftmaxSharpness * BlendR * FlowR,
 * per channel, with bilinear clamp-to-edge sampling.
 * blend: (h, w) float32 contiguous array of Blend values (Eq. 1), or NULL
 * for the Eq. (1) value of a full-height strip with Area1 on its left and
 * Area2 on its right, Blend(x) = (x + 1) / (w + 1).
 * F: same h, w, c and dtype as L. PANO_U8 output is round-half-even of
 * 255 * F clamped to [0, 255]; PANO_F32 output is F.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
PANO_API pano_status pano_blend_pair(pano_flow_ctx* ctx, const pano_image* L, const pano_image* R,
                            const float* flow_LtoR, const float* flow_RtoL, const float* blend,
                            pano_image* F, void* cuda_stream);

/* Code 1 (Section III-C-3) on a whole canvas, every branch, for every pixel p:
 *   label(p) == 1 (Area1): F(p) = L(p);   label(p) == 2 (Area2): F(p) = R(p);
 *   label(p) == 3 (Area3): the blend of pano_blend_pair at p, with L and R
 *                          the canvas images (samples clamp at the canvas
 *                          border, not at the overlap's);
 *   any other label:       F(p) = 0.
 * L, R, F: canvas images (device data), same h, w, c (1 or 3) and dtype
 *   (PANO_U8 or PANO_F32); values of L and R outside their own areas are
 *   read only where an Area3 sample lands there.
 * label: h x w bytes, row pitch label_pitch bytes (the label canvas of
 *   pano_blend_coeff). blend: h x w float32 Blend values of Eq. (1), row
 *   pitch blend_pitch floats (e.g. from pano_blend_coeff).
 * flow_LtoR, flow_RtoL: (flow_h, flow_w, 2) float32 contiguous, the flows of
 *   the overlap crop whose pixel (0, 0) is canvas pixel (flow_y0, flow_x0),
 *   as pano_flow_pair gives them for that crop of L and R. FlowMag divides by
 *   flow_w, the overlap width. An Area3 pixel outside the crop uses zero flow.
 * params: only soft_sharpness and flow_mag_coef are read.
 * F must not overlap any input. No allocation; asynchronous on cuda_stream.
 * Errors: INVALID_ARG (NULL or misaligned pointers, sizes that differ, a crop
 * outside the canvas, overlapping F), UNSUPPORTED (16-bit or >3-channel
 * images), CUDA. */
PANO_API pano_status pano_compose_pair(const pano_flow_params* params, const pano_image* L,
                                       const pano_image* R, const unsigned char* label, size_t label_pitch,
                                       const float* blend, int blend_pitch, const float* flow_LtoR,
                                       const float* flow_RtoL, int flow_y0, int flow_x0, int flow_h,
                                       int flow_w, pano_image* F, void* cuda_stream);

/* Free the context and its scratch. NULL is accepted. Work already enqueued
 * that uses the context must have completed. */
PANO_API pano_status pano_flow_destroy(pano_flow_ctx* ctx);

/* Message describing the last failing call on the calling thread ("" if
 * none). The pointer stays valid until the next call on this thread. */
PANO_API const char* pano_last_error(const pano_flow_ctx* ctx);

/* ----------------------------------------------------------------------
 * Global blending coefficient of Eq. (1) (Section III-C-2) for overlaps of
 * any shape. label is an h x w canvas of bytes (row pitch label_pitch):
 * 1 = Area1 (covered by L only), 2 = Area2 (R only), 3 = Area3 (the
 * overlap), any other value = neither. blend receives h x w float32 values
 * (row pitch blend_pitch elements):
 *   Blend = 0 in Area1, 1 in Area2, 0.5 in neither, and in Area3
 *   Lmin / (Lmin + Rmin), Lmin / Rmin the Euclidean distances between pixel
 *   centres to the nearest Area1 / Area2 pixel.
 * With no Area1 pixel on the canvas Area3 gets 1, with no Area2 pixel 0,
 * with neither 0.5 (the limits of Eq. 1). The distances are exact (integer
 * distance transform); the ratio is rounded in FP32. The Blend array of a
 * strip can be passed to pano_blend_pair.
 * scratch: device memory of at least pano_blend_coeff_scratch_bytes(h, w)
 * bytes (8 * h * w), 4-byte aligned; label, blend and scratch must not
 * overlap. Sides up to 65535; the width is limited further by shared memory
 * (4 bytes per column and 5 KB per row: 56000 columns on a GB300).
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA.
 * ---------------------------------------------------------------------- */
PANO_API size_t pano_blend_coeff_scratch_bytes(int h, int w);
PANO_API pano_status pano_blend_coeff(const unsigned char* label, int h, int w, size_t label_pitch, float* blend,
                                      int blend_pitch, void* scratch, size_t scratch_bytes, void* cuda_stream);

/* ----------------------------------------------------------------------
 * Differentiable refinement. Not a step of the paper: a build extension
 * that refines a flow by gradient steps on the energy
 *   E(u) = sum_p (J(p + u(p)) - T(p))^2
 *        + alpha sum_p sum_c [(u_c(p + e_x) - u_c(p))^2 [x < w-1] + (u_c(p + e_y) - u_c(p))^2 [y < h-1]]
 * i.e. the data term of the flow step plus the smoothness term of the
 * Horn-Schunck half of the reference the paper cites for LK ([20]). J is
 * sampled with the bilinear clamp-to-edge sampler of the flow path.
 * ---------------------------------------------------------------------- */

/* E and its gradients for template T and target J (h x w float32, row pitch
 * `pitch` floats) and flow u ((h, w, 2) float32 contiguous).
 * energy: device pointer to one double that receives E (reduced in FP64), or
 * NULL. grad_u ((h, w, 2)), grad_T ((h, w)) and grad_J ((h, w)), all float32
 * contiguous, receive dE/du, dE/dT and dE/dJ; any may be NULL. dE/dJ is
 * accumulated with atomic additions, so its last bits vary between runs.
 * Errors: INVALID_ARG, CUDA. */
PANO_API pano_status pano_energy_grad(const float* T, const float* J, int h, int w, int pitch, const float* u,
                                      float alpha, double* energy, float* grad_u, float* grad_T, float* grad_J,
                                      void* cuda_stream);

/* Transpose of pano_stage_pyr_down: given the gradient gdst of the
 * ceil(h/2) x ceil(w/2) output (row pitch dst_pitch), writes the gradient
 * gsrc of the h x w input (row pitch src_pitch). Errors: INVALID_ARG, CUDA. */
PANO_API pano_status pano_stage_pyr_down_adjoint(const float* gdst, int h, int w, int dst_pitch, float* gsrc,
                                                 int src_pitch, void* cuda_stream);

/* ----------------------------------------------------------------------
 * Flow without any device allocation. (The paper has no counterpart: this is
 * a deployment variant of pano_flow_pair.)
 *
 * pano_flow_create allocates its scratch with cudaMalloc. Some callers cannot
 * allow that: a process that owns all of the GPU's memory through its own
 * pool and forbids other allocations, or a frame loop with a deadline, where
 * cudaMalloc / cudaFree would add latency and device-wide synchronisation.
 * pano_flow_pair_static computes exactly what pano_flow_pair computes (same
 * kernels, same results) without a context: its scratch is one fixed array
 * of PANO_STATIC_SCRATCH_BYTES bytes inside the library, which every GPU that
 * loads the library holds until the process exits. The call never allocates
 * or frees device memory.
 *
 *   Size limit  The scratch holds both luma pyramids and the coarse-level
 *               flows of both directions, about 16 * h * w bytes (4 levels
 *               or more): strips up to about one megapixel (e.g. 1024 x 1024)
 *               fit. Larger strips are rejected with PANO_ERR_INVALID_ARG and
 *               a message giving the bytes needed; nothing is enqueued.
 *   Set-up      The first call on each device, with that device current,
 *               looks up the array's device address (cudaGetSymbolAddress)
 *               and sets the kernel's shared-memory limit. Make that first
 *               call before any stream capture on the device.
 *   Sharing     All calls, on every stream and thread, use the same array,
 *               and it keeps whatever the last call wrote. Nothing in it
 *               needs to start at zero: each call writes every byte it reads.
 *               Calls whose work overlaps on the GPU race on the array:
 *               order them on one stream (or with events).
 * Arguments, flows and errors are those of pano_flow_pair; `params` replaces
 * the context and must keep float32 pyramids (pyr_dtype PANO_F32; UNSUPPORTED
 * otherwise).
 * ---------------------------------------------------------------------- */
#define PANO_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)

PANO_API pano_status pano_flow_pair_static(const pano_flow_params* params, const pano_image* L,
                                           const pano_image* R, float* flow_LtoR, float* flow_RtoL,
                                           void* cuda_stream);

/* ----------------------------------------------------------------------
 * Tracing. When enabled, every launch of a kernel kind selected by
 * kind_mask that a context call enqueues is bracketed by two CUDA events on
 * that call's stream, so its device time can be read back. Events are
 * created by pano_trace_enable (not by the traced calls); at most `capacity`
 * launches are recorded until the next pano_trace_read.
 * ---------------------------------------------------------------------- */
#define PANO_TRACE_LUMA     0x1u   /* level-0 luma */
#define PANO_TRACE_PYR_DOWN 0x2u   /* pyramid REDUCE */
#define PANO_TRACE_LK       0x4u   /* one Lucas-Kanade level, both directions */
#define PANO_TRACE_BLEND    0x8u   /* Code 1 blend */
#define PANO_TRACE_LUMA_REDUCE 0x10u  /* level 0 (luma) and level 1 (its REDUCE) in one launch */
#define PANO_TRACE_PYR_TAIL 0x20u  /* several REDUCE steps (levels 3 and below) in one launch */

typedef struct pano_trace_record {
    int kind;     /* one PANO_TRACE_* bit */
    int level;    /* pyramid level (LK, REDUCE destination), else 0 */
    float ms;     /* device time between the two events */
} pano_trace_record;

/* Enable tracing of the kinds in kind_mask with room for `capacity`
 * launches; capacity 0 (or kind_mask 0) disables it and frees the events.
 * Errors: INVALID_ARG, OOM, CUDA. */
PANO_API pano_status pano_trace_enable(pano_flow_ctx* ctx, unsigned kind_mask, int capacity);

/* Wait for the recorded events, copy up to max_records records (launch
 * order) to out, store their number in *n_out, and start a new recording.
 * Errors: INVALID_ARG, CUDA. */
PANO_API pano_status pano_trace_read(pano_flow_ctx* ctx, pano_trace_record* out, int max_records,
                                     int* n_out);

/* Number of kernel launches this context has enqueued since creation. */
PANO_API unsigned long long pano_flow_launches(const pano_flow_ctx* ctx);

/* ----------------------------------------------------------------------
 * Stage entry points. Each runs one step of the path above on caller
 * buffers with the same kernels pano_flow_pair / pano_blend_pair use, so
 * each step can be checked and reused on its own. Float planes are
 * row-major float32 with the given row pitch in elements.
 * ---------------------------------------------------------------------- */

/* Level 0 of the pyramid: unit-scaled luma Y (h x w) of an image (BT.601
 * for c = 3, the sample itself for c = 1). Y pitch >= w. */
PANO_API pano_status pano_stage_luma(const pano_image* in, float* Y, int y_pitch, void* cuda_stream);

/* Level 0 and level 1 of the pyramid in one launch, as pano_flow_pair forms
 * them: Y as pano_stage_luma writes it (h x w) and Y1 its REDUCE as
 * pano_stage_pyr_down writes it (ceil(h/2) x ceil(w/2)), bit for bit.
 * Pitches in floats. */
PANO_API pano_status pano_stage_luma_pyr(const pano_image* in, float* Y, int y_pitch, float* Y1, int y1_pitch,
                                         void* cuda_stream);

/* Levels 1 .. nlev-1 of the pyramid of Y (h x w, row pitch `pitch` floats)
 * with the launch sequence pano_flow_pair uses (one-level REDUCE launches
 * for levels 1 and 2, several levels per launch after that): levels[l - 1]
 * receives level l, ceil(h / 2^l) x ceil(w / 2^l), row pitch pitches[l - 1]
 * floats. The same values as nlev - 1 pano_stage_pyr_down calls, bit for
 * bit. nlev in 2..12. */
PANO_API pano_status pano_stage_pyramid(const float* Y, int h, int w, int pitch, float* const* levels,
                                        const int* pitches, int nlev, void* cuda_stream);

/* One pyramid REDUCE step (Section III-C-1, "LK pyramid"): [1 4 6 4 1]/16
 * along y then x, replicate border, keep even rows and columns.
 * src h x w -> dst ceil(h/2) x ceil(w/2). */
PANO_API pano_status pano_stage_pyr_down(const float* src, int h, int w, int src_pitch, float* dst,
                                int dst_pitch, void* cuda_stream);

/* `iters` Lucas-Kanade steps at one level (Section III-C-1) on template T
 * and target J (both h x w, same pitch), each step as described for
 * pano_flow_pair: every pixel solves
 *   (G(p) + lambda I) v = sum_{q in W(p)} grad T(q) (grad T(q) . u(q) - It(q)) + lambda u(p),
 *   It(q) = J(q + u(q)) - T(q),  G(p) = sum_{q in W(p)} grad T grad T^T,
 * over the (2r+1)^2 box W(p) clipped to the image, then sets u(p) = v.
 * Starting flow: flow_in == NULL -> zero; upsample == 0 -> flow_in is an
 * (h, w, 2) field used as is; upsample == 1 -> flow_in is the (in_h, in_w, 2)
 * field of the next coarser level, and the start is 2 * flow_in sampled
 * bilinearly at (x/2, y/2) (coarse-to-fine propagation).
 * flow_out: (h, w, 2); it must not overlap flow_in. iters = 0 writes the
 * starting flow. */
PANO_API pano_status pano_stage_lk(const float* T, const float* J, int h, int w, int pitch,
                          const float* flow_in, int in_h, int in_w, int upsample,
                          float* flow_out, int iters, int radius, float lambda,
                          void* cuda_stream);

/* Kernel of one LK level (pano_stage_lk_kernel, and per level in the rig of
 * pano_rig.h). Both kernels compute the same equations with the same order
 * of FP32 operations; results differ only in rounding, because each tile or
 * segment measures its flows against its own reference flow. */
#define PANO_LK_AUTO   0  /* the kernel pano_flow_pair runs for a level of this size: streamed
                             for levels of at least 50000 pixels (1 <= iters <= 5), tiled
                             below (16 x 8 tiles below 16000 pixels) */
#define PANO_LK_STREAM 1  /* streamed row chunks down column bands (1 <= iters <= 5) */
#define PANO_LK_TILE   2  /* output tiles with a halo of iters * radius pixels */

/* pano_stage_lk with the kernel chosen by the caller (a PANO_LK_* value);
 * pano_stage_lk itself runs PANO_LK_STREAM when 1 <= iters <= 5, else
 * PANO_LK_TILE. Errors as pano_stage_lk; INVALID_ARG for an unknown kernel,
 * UNSUPPORTED for PANO_LK_STREAM outside 1 <= iters <= 5. */
PANO_API pano_status pano_stage_lk_kernel(const float* T, const float* J, int h, int w, int pitch,
                                          const float* flow_in, int in_h, int in_w, int upsample,
                                          float* flow_out, int iters, int radius, float lambda,
                                          int kernel, void* cuda_stream);

/* Bilinear flow warp, dst(p) = src(p + scale * flow(p)), per channel,
 * clamp-to-edge; Code 1 evaluates it with scale = Blend for L and FlowRtoL
 * and scale = 1 - Blend for R and FlowLtoR. dst: same h, w, c as src,
 * dtype PANO_F32, unit-scaled values. */
PANO_API pano_status pano_stage_warp(const pano_image* src, const float* flow, float scale,
                            pano_image* dst, void* cuda_stream);

/* ----------------------------------------------------------------------
 * Index checks (debug build only). The `check` variant of the library
 * (build.build(variant="check"), compiled with -DPANO_BOUNDS_CHECK) checks
 * before the access every shared-memory and global index of the two LK
 * kernels and of the pyramid kernels, the image gathers of the blends,
 * the compose and the warp, every index of the distance transform of
 * Eq. (1) and of the energy and adjoint kernels. An index outside its
 * array is counted, the first one recorded, and the access clamped into
 * the array, so nothing traps.
 * pano_debug_bounds copies the record into out[4] = {count, site, index,
 * bound} and clears it; call it after the work has completed (synchronise
 * first). In the normal build it writes zeros and returns UNSUPPORTED.
 * Errors: INVALID_ARG (out NULL), UNSUPPORTED, CUDA. */
PANO_API pano_status pano_debug_bounds(unsigned* out);

#ifdef __cplusplus
}
#endif

#endif /* PANO_FLOW_H */
