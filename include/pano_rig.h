/* pano_rig.h -- every overlap pair of a 360-degree camera rig in one call.
 *
 * A panorama of Section III is stitched pair by pair: each adjacent pair of
 * camera images shares an overlap strip (Area3 of Code 1), whose flows in
 * both directions (Section III-C-1) and blend (Code 1 with Eq. 1) are those
 * of pano_flow_pair and pano_blend_pair. A rig object runs the same path for
 * all pairs of a rig at once and places every blended strip in one
 * panorama canvas (the last step of Code 1, which writes Area3 into the
 * output beside the copied Area1 and Area2):
 *
 *   luma of all strips          one launch
 *   REDUCE of all strips        one launch per level
 *   LK, both directions, every  per level, one persistent launch of the
 *   pair                        streamed kernel over the (pair, direction,
 *                               band, segment) work list and/or one tiled
 *                               grid per tile shape over those pairs
 *   blend into the canvas       one launch
 *
 * The whole sequence can be captured once in a CUDA graph and replayed. The
 * streamed segment height and the tile shape of each level come from the
 * rig's autotuner (pano_rig_autotune) or from pano_rig_set_tuning. The halo
 * of a tile or segment is fixed by the method (iters * radius pixels per
 * side: step k at p reads the flows of step k - 1 on the window of p); the
 * tuning sets the area over which that halo is paid.
 *
 * Results: with the default tuning (PANO_LK_AUTO everywhere) the flows of
 * pair k equal bit for bit those pano_flow_pair computes for the same strips
 * and parameters. Other tunings change only the FP32 rounding of the flows
 * (each tile or segment measures its flows against its own reference flow).
 *
 * Errors, streams and ownership follow pano_flow.h; pano_last_error(NULL)
 * gives the message of the last failing call on the calling thread.
 */
#ifndef PANO_RIG_H
#define PANO_RIG_H

#include "pano_flow.h"

#ifdef __cplusplus
extern "C" {
#endif

#define PANO_RIG_MAX_PAIRS 8

/* Geometry of a rig. Strip k (both its L and its R image) is h x w[k] with
 * c channels of `dtype`. Its blended strip lands on canvas rows
 * canvas_y0 .. canvas_y0 + h - 1 and columns (canvas_x0[k] + x) mod
 * canvas_w, x = 0 .. w[k] - 1 (the canvas is an equirectangular panorama,
 * so spans wrap around its seam). Where the spans of several pairs cover a
 * canvas column, the pair with the highest index writes it; canvas pixels
 * outside every span are left as they are (the caller's Area1/Area2
 * content). */
typedef struct pano_rig_desc {
    int n_pairs;                        /* 1..PANO_RIG_MAX_PAIRS */
    int h;                              /* strip height, shared by all pairs */
    int w[PANO_RIG_MAX_PAIRS];          /* strip (overlap) widths, 1..canvas_w */
    int c;                              /* channels, 1 or 3 */
    int dtype;                          /* PANO_U8 or PANO_F32 */
    int canvas_h, canvas_w;             /* canvas size; canvas_y0 + h <= canvas_h */
    int canvas_y0;                      /* canvas row of strip row 0, >= 0 */
    int canvas_x0[PANO_RIG_MAX_PAIRS];  /* canvas column of strip column 0, in [0, canvas_w) */
} pano_rig_desc;

typedef struct pano_rig_tuning {
    int kernel;          /* a PANO_LK_* value (pano_flow.h) */
    int seg_rows;        /* streamed kernel: rows per segment, 0 = automatic (about 256,
                            rounded to whole waves of the GPU) */
    int tile_w, tile_h;  /* tiled kernel: output tile; both 0 = the default tile */
    float ms;            /* device time of the level measured by pano_rig_autotune, else 0 */
} pano_rig_tuning;

typedef struct pano_rig pano_rig;

/* Create a rig for the geometry *d on the current device: the pyramids of
 * all 2 * n_pairs strips, the coarse-level flows, the level-0 flows of
 * every pair (used when a call passes no flow buffers) and a private
 * capture stream. Every level starts with PANO_LK_AUTO tuning.
 * Errors: INVALID_ARG (null argument, parameters or geometry out of range),
 * UNSUPPORTED (sizes beyond 32-bit offsets), OOM, CUDA. Pyramids are stored as
 * p->pyr_dtype (see pano_flow_params). */
PANO_API pano_status pano_rig_create(const pano_flow_params* p, const pano_rig_desc* d, pano_rig** out);

/* Flows of every pair and, if canvas != NULL, their blends placed on the
 * canvas, enqueued on cuda_stream.
 *   L, R        arrays of n_pairs image descriptors (device data, geometry
 *               of the rig); pair k is (L[k], R[k]).
 *   flow_LtoR,  arrays of n_pairs device pointers to (h, w[k], 2) float32
 *   flow_RtoL   fields (see pano_flow_pair), or NULL arrays to keep the
 *               flows in the rig (pano_rig_flows).
 *   canvas      canvas_h x canvas_w image with the rig's c and dtype, or
 *               NULL to compute flows only. It must not overlap any input.
 *   use_graph   0: enqueue the kernels directly. 1: replay a CUDA graph of
 *               the same sequence. The rig keeps up to 4 graphs, one per
 *               distinct set of pointers, pitches and tuning (e.g. the two
 *               buffer sets of a double-buffered pipeline); a call with a
 *               new set captures a graph in place of the least recently
 *               used one. Tracing records only calls with use_graph = 0.
 * The device that was current at pano_rig_create must be current.
 * Errors: INVALID_ARG, CUDA. */
PANO_API pano_status pano_rig_run(pano_rig* rig, const pano_image* L, const pano_image* R,
                                  float* const* flow_LtoR, float* const* flow_RtoL, pano_image* canvas,
                                  int use_graph, void* cuda_stream);

/* Autotune the LK kernel of every level on the strips L, R (flows kept in
 * the rig): after one full run, each level is timed with CUDA events, `reps`
 * launches per candidate after one warm-up launch, over PANO_LK_AUTO, the
 * streamed kernel with segment heights {auto, 64, 96, 128, 192, 256, 384}
 * and the tiled kernel with every tile of {32x8, 32x16, 16x16, 64x8, 64x16,
 * 32x32} that fits the device's shared memory; the fastest (median) becomes
 * the level's tuning. Synchronises cuda_stream. Errors: INVALID_ARG, CUDA. */
PANO_API pano_status pano_rig_autotune(pano_rig* rig, const pano_image* L, const pano_image* R, int reps,
                                       void* cuda_stream);

/* Read or set the tuning of one level (0 = finest). set checks the kernel
 * value, that a streamed level has 1 <= iters <= 5 and that a tile fits
 * the device's shared memory. Errors: INVALID_ARG, UNSUPPORTED. */
PANO_API pano_status pano_rig_get_tuning(const pano_rig* rig, int level, pano_rig_tuning* out);
PANO_API pano_status pano_rig_set_tuning(pano_rig* rig, int level, const pano_rig_tuning* t);

/* Device pointers of the rig's own level-0 flows of pair k (valid until
 * pano_rig_destroy). Errors: INVALID_ARG. */
PANO_API pano_status pano_rig_flows(const pano_rig* rig, int k, float** flow_LtoR, float** flow_RtoL);

/* Tracing of pano_rig_run calls with use_graph = 0, as pano_trace_enable
 * and pano_trace_read for a flow context (PANO_TRACE_* kinds; an LK level
 * split over both kernel kinds gives two records). */
PANO_API pano_status pano_rig_trace_enable(pano_rig* rig, unsigned kind_mask, int capacity);
PANO_API pano_status pano_rig_trace_read(pano_rig* rig, pano_trace_record* out, int max_records, int* n_out);

/* Kernel launches the rig has enqueued since creation (a graph replay
 * counts the kernels of the graph), and the number of graphs captured. */
PANO_API unsigned long long pano_rig_launches(const pano_rig* rig);
PANO_API int pano_rig_graph_captures(const pano_rig* rig);

/* Free the rig, its buffers, graph and stream. NULL is accepted. Work
 * already enqueued that uses the rig must have completed. */
PANO_API pano_status pano_rig_destroy(pano_rig* rig);

#ifdef __cplusplus
}
#endif

#endif /* PANO_RIG_H */
