/*
 * gr.h -- C ABI of libgr, exact graph-layout readability metrics on one GPU.
 *
 * The five metrics are those of "Scalable Readability Evaluation for Graph
 * Layouts: 2D Geometric Distributed Algorithms" (arXiv 2411.09809), Sec. 2.1:
 *   node occlusion N_c          (Algorithm 1)
 *   minimum angle M_a           (Algorithm 2)
 *   edge length variation M_l   (Algorithm 3)
 *   edge crossings E_c          (Algorithm 4)
 *   edge crossing angle E_ca    (Algorithm 5)
 * All of them are computed exactly (counts are exact integers; float metrics
 * carry only rounding error), unlike the paper's approximate "enhanced"
 * algorithms of Sec. 3.2.
 *
 * Conventions shared by every entry point
 *   - Coordinates: int32 pairs [V][2] in [0, 65536) (GR_COORD_I32).
 *   - Edges: int32 pairs [E][2] of vertex ids in [0, V); no self-loops.
 *     Duplicate edges are allowed (they share endpoints, so never cross).
 *   - Pointers to inputs may be device or host memory (pinned or pageable);
 *     the library looks the kind up and copies host inputs to the device on
 *     the layout's stream.  The library never keeps a caller pointer after a
 *     call returns: it copies what it needs into memory it owns.
 *   - Every call returns a gr_status; on error the outputs are left
 *     untouched and gr_last_error() describes the failure (thread-local).
 *   - Calls on one gr_layout must not run concurrently from several host
 *     threads.  Work is issued on the layout's stream (gr_stream_t is the
 *     same type as cudaStream_t; NULL selects the legacy default stream).
 *
 * Degenerate cases, where the paper is silent (the library's fixed reading):
 *   - two edges that share a vertex id never cross;
 *   - a zero-length edge (distinct ids, equal coordinates) takes part in no
 *     crossing and no angle; it has length 0 for M_l;
 *   - a collinear pair whose extents meet is counted once in
 *     collinear_overlaps and is not part of E_c or E_ca;
 *   - E_c counts proper crossings plus touching pairs (an endpoint of one
 *     edge on the other edge), as Algorithm 4's "<= 0" predicate does;
 *   - the crossing angle a_c is the acute angle between the two lines;
 *   - E_ca = 1 when E_c = 0; M_a = 1 when no vertex has two non-zero-length
 *     incident edges; M_l = 0 when |E| <= 1 or the mean length is 0.
 */
#ifndef GR_H
#define GR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gr_stream_t; /* identical to cudaStream_t */
typedef struct gr_layout gr_layout;

typedef enum {
    GR_OK = 0,
    GR_EINVAL = 1,   /* bad argument, vertex id out of range or self-loop */
    GR_ERANGE = 2,   /* coordinate outside [0, 65536) */
    GR_ENOMEM = 3,   /* device allocation failed */
    GR_ECUDA = 4,    /* a CUDA call failed (message in gr_last_error) */
    GR_ETIMEOUT = 5, /* a bounded device-side wait gave up */
    GR_ENOTSUP = 6   /* feature not supported for this input */
} gr_status;

typedef enum { GR_COORD_I32 = 0, GR_COORD_F32 = 1 } gr_coord_type;

/* Metric selection bits for gr_evaluate. */
enum {
    GR_METRIC_OCCLUSION = 1u,
    GR_METRIC_MIN_ANGLE = 2u,
    GR_METRIC_EDGE_LENGTH = 4u,
    GR_METRIC_CROSSINGS = 8u, /* E_c and E_ca together */
    GR_METRIC_ALL = 15u
};

/* Which pair kernel computes crossings. */
typedef enum {
    GR_PATH_AUTO = 0,     /* density heuristic picks */
    GR_PATH_GRID = 1,     /* uniform grid + per-cell pair kernel */
    GR_PATH_ALLPAIRS = 2, /* tiled brute force over all edge pairs */
    GR_PATH_DELTA = 3     /* (results only) updated from the previous evaluation by gr_move_vertices */
} gr_path;

/* Where the grid path tests pairs of two long segments (segments spanning
 * more than two cell lines): a grid cannot prune those, so by default the
 * cost model may send them to all-pairs tiles over the list of long
 * segments instead.  Either choice gives the same exact counts. */
typedef enum {
    GR_LONG_AUTO = 0,      /* cost model picks */
    GR_LONG_ALLPAIRS = 1,  /* all-pairs tiles over the long segments */
    GR_LONG_GRID = 2       /* in the grid cells with every other pair */
} gr_long_pairs;

typedef struct {
    int32_t crossing_path;  /* gr_path; 0 = auto */
    int32_t cell_log2;      /* crossing grid cell side 2^k, k in [6, 16]; 0 = auto */
    int32_t occlusion_path; /* gr_path for occlusion; 0 = auto */
    int32_t profile;        /* non-zero: enable phase timing at creation */
    int32_t long_pairs;     /* gr_long_pairs; 0 = auto */
} gr_options;

typedef struct {
    double ideal_rad;    /* ideal crossing angle in (0, pi/2]; <= 0 selects 70 deg */
    int64_t occlusion_d; /* occlusion diameter d = 2r >= 0 (pairs with distance < d) */
} gr_params;

typedef struct {
    int64_t crossings;          /* E_c = proper + touching */
    int64_t proper;             /* the two segments cross at interior points */
    int64_t touching;           /* an endpoint lies on the other segment */
    int64_t collinear_overlaps; /* collinear pairs whose extents meet (not in E_c) */
    int64_t zero_length_edges;  /* edges with equal endpoint coordinates */
    int64_t pairs_tested;       /* candidate pairs the pair kernel evaluated */
} gr_crossing_counts;

typedef struct {
    gr_crossing_counts c;
    double angle_dev_sum; /* sum over the E_c pairs of |ideal - a_c|, radians */
    double ideal_rad;     /* the ideal angle used */
    double E_ca;          /* 1 - angle_dev_sum / (ideal * E_c); 1 if E_c = 0 */
} gr_crossing_angle_result;

typedef struct {
    double M_a;                 /* 1 - sum_d / n_vertices_counted; 1 if none */
    double sum_d;               /* sum of d_v over counted vertices */
    int64_t n_vertices_counted; /* vertices with >= 2 non-zero-length edges */
} gr_min_angle_result;

typedef struct {
    uint32_t metrics;       /* the metric bits that were evaluated */
    int32_t crossing_path;  /* gr_path taken for crossings (1 grid, 2 all-pairs) */
    int32_t cell_log2;      /* grid cell side used for crossings (0 if all-pairs) */
    int32_t occlusion_path; /* gr_path taken for occlusion */
    gr_crossing_angle_result crossing;
    int64_t occlusion_pairs; /* N_c */
    int64_t occlusion_d;
    gr_min_angle_result min_angle;
    double M_l;
    int64_t grid_records;   /* (edge, cell) records binned by the grid path */
} gr_result;

/* Creates a layout from V vertex coordinates and E edges (Sec. 2.1 inputs;
 * Algorithms 1-5 take the vertex table D_pos and the edge table D_e).
 * `xy` is [V][2] of `coord_type` (int32, or FP32: see below), `edges` is [E][2]
 * int32, device or host memory.  Validates the input on the device and
 * synchronises the stream: GR_EINVAL for a vertex id outside [0, V) or a
 * self-loop, GR_ERANGE for a coordinate outside [0, 65536).  `opt` may be
 * NULL.  The layout owns device memory sized for V and E until destroyed.
 * V >= 0, E >= 0, both < 2^31. */
gr_status gr_layout_create(gr_layout **out, const void *xy, gr_coord_type coord_type,
                           int64_t V, const int32_t *edges, int64_t E,
                           const gr_options *opt, gr_stream_t stream);

/* Replaces the coordinates (and, when `edges` is not NULL, the edge list) of
 * an existing layout, keeping V and E.  Stream-ordered, no synchronisation:
 * validation errors are reported by the next gr_evaluate. */
gr_status gr_layout_update(gr_layout *layout, const void *xy, const int32_t *edges);

gr_status gr_layout_destroy(gr_layout *layout);

/* Evaluates the metrics selected by `metrics` (GR_METRIC_* bits) and writes
 * them to the host struct `out`.  `params` may be NULL (ideal 70 deg, d 0).
 * Synchronises the layout's stream.  GR_EINVAL for d < 0 or an ideal angle
 * above pi/2, and for invalid input left by gr_layout_update. */
gr_status gr_evaluate(gr_layout *layout, uint32_t metrics, const gr_params *params,
                      gr_result *out);

/* gr_evaluate without any host synchronisation: the evaluation is ordered
 * after the work already queued on `stream` (NULL: the layout's stream), and
 * the gr_result is written to `d_result`, DEVICE memory owned by the caller,
 * before anything queued on `stream` afterwards runs.  The call can itself be
 * captured into the caller's CUDA graph (it replays the layout's own graph
 * of this configuration) once a gr_evaluate of the layout with the same
 * metrics and parameters has planned it and sized its buffers; before that,
 * and whenever the layout's plan changes, the call synchronises once to plan.
 * A result whose `metrics` field is 0 reports a failed evaluation (invalid
 * input, or inputs that outgrew the planned buffers): call gr_evaluate for
 * the error.  Incremental moves after an asynchronous evaluation start with
 * a full evaluation.  GR_COORD_I32 layouts only. */
gr_status gr_evaluate_async(gr_layout *layout, uint32_t metrics, const gr_params *params, gr_result *d_result,
                            gr_stream_t stream);

/* Node occlusion N_c (Sec. 2.1, Algorithm 1): unordered vertex pairs whose
 * distance is < d, d = 2r.  Strict inequality; d = 0 gives 0. */
gr_status gr_node_occlusion(gr_layout *layout, int64_t d, int64_t *out_pairs);

/* Minimum angle M_a (Sec. 2.1, Algorithm 2), averaged over the vertices with
 * at least two non-zero-length incident edges. */
gr_status gr_min_angle(gr_layout *layout, gr_min_angle_result *out);

/* Edge length variation M_l (Sec. 2.1, Algorithm 3), every edge counted once. */
gr_status gr_edge_length_variation(gr_layout *layout, double *out_M_l);

/* Edge crossings E_c and their classes (Sec. 2.1, Algorithm 4). */
gr_status gr_edge_crossings(gr_layout *layout, gr_crossing_counts *out);

/* Edge crossing angle E_ca (Sec. 2.1, Algorithm 5) with ideal angle
 * `ideal_rad` in (0, pi/2]; <= 0 selects 70 deg = 7 pi / 18. */
gr_status gr_crossing_angle(gr_layout *layout, double ideal_rad, gr_crossing_angle_result *out);

/* The paper's approximate crossing count and crossing angle (Sec. 3.2.2 and
 * Sec. 3.2.3 with Eq. 1), for comparison with the exact metrics.  The plane
 * is cut by the lines x = s * strip_width (GR_STRIP_VERTICAL) or
 * y = s * strip_width (GR_STRIP_HORIZONTAL); two segments that both cross
 * both lines of a strip count as crossing when their order along the lines
 * reverses strictly from one line to the other (y at a line compared as the
 * exact key floor(y * 2^30)).  Pairs whose crossing lies in a strip that
 * one of them does not span are missed, so the count never exceeds E_c.
 * angle_dev_sum and E_ca are Algorithm 5's sum and metric over the counted
 * pairs.  GR_STRIP_BOTH runs both orientations and reports the one with the
 * larger count.  strip_width in [1, 65535], ideal_rad in (0, pi/2] (<= 0:
 * 70 deg).  GR_COORD_I32 layouts only (GR_ENOTSUP otherwise); synchronises;
 * result on the host. */
enum { GR_STRIP_VERTICAL = 0, GR_STRIP_HORIZONTAL = 1, GR_STRIP_BOTH = 2 };
typedef struct {
    int64_t crossings;     /* pairs counted (the E_c estimate) */
    int64_t records;       /* (segment, strip) records of the reported orientation */
    int64_t strips;        /* strips of width strip_width covering [0, 65536) */
    double angle_dev_sum;  /* sum of |ideal - a_c| over the counted pairs, radians */
    double ideal_rad;
    double E_ca;           /* 1 - angle_dev_sum / (ideal_rad * crossings); 1 when crossings = 0 */
    int32_t orientation;   /* the orientation reported */
    int32_t strip_width;
} gr_strip_result;
gr_status gr_strip_crossings(gr_layout *layout, int32_t strip_width, int32_t orientation, double ideal_rad,
                             gr_strip_result *out);

/* Per-edge crossing data (the per-segment quantity of Sec. 3.2.3 / Eq. 1,
 * computed exactly): for every edge e, the number of proper crossings,
 * touching pairs and collinear overlaps it takes part in, and the sum of
 * |ideal - a_c| over its E_c partners.  `d_counts` is DEVICE memory
 * int64 [E][3], `d_dev` DEVICE memory double [E]; both caller-owned and
 * overwritten.  Edges are indexed as passed to gr_layout_create. */
gr_status gr_crossings_per_edge(gr_layout *layout, double ideal_rad, int64_t *d_counts,
                                double *d_dev);

/* ------------------------------------------------- incremental moves
 * gr_move_vertices moves the n vertices ids[i] (distinct, in [0, V)) to
 * xy_new[i] (int32 [n][2] in [0, 65536); ids and xy_new in host or device
 * memory) and evaluates the metrics of the moved layout, as gr_evaluate
 * would.  When the previous evaluation of this layout (gr_evaluate or
 * gr_move_vertices, with no gr_layout_update since) covered the crossings
 * and occlusion requested here with the same ideal angle and d, those counts
 * and the crossing-angle sum are updated instead of recomputed: only the
 * pairs of an edge with a moved endpoint (crossings, Algorithms 4 and 5) and
 * of a moved vertex (occlusion, Algorithm 1) are classified, before and after
 * the move, so the work is proportional to (affected edges) x E + n x V; the
 * result equals a full evaluation exactly (the same predicates and integer
 * angle terms).  Minimum angle and edge length variation are recomputed.
 * The result's crossing_path and occlusion_path are then GR_PATH_DELTA and
 * pairs_tested counts the pairs this call tested.  Otherwise the moves are
 * applied and a full evaluation runs.  GR_EINVAL for an id outside [0, V) or
 * given twice, GR_ERANGE for a coordinate outside [0, 65536); the layout is
 * unchanged then.  GR_COORD_I32 layouts only (GR_ENOTSUP otherwise).
 * Synchronises. */
gr_status gr_move_vertices(gr_layout *layout, int64_t n, const int32_t *ids, const int32_t *xy_new,
                           uint32_t metric_mask, const gr_params *params, gr_result *out);

/* ------------------------------------------------- differentiable form
 * Layouts created with GR_COORD_F32 take FP32 coordinates [V][2] (any finite
 * values; GR_ERANGE otherwise).  Their crossing set is decided exactly on the
 * FP32 inputs (orientation signs through an FP32 error-bound filter, an FP64
 * one and exact expansion arithmetic, after Shewchuk 1997); gr_evaluate
 * supports the crossing, edge length and minimum angle metrics on them
 * (occlusion: GR_ENOTSUP).
 *
 * gr_diff_forward evaluates E_ca (ideal `ideal_rad`, <= 0 for 70 deg), M_l
 * and M_a (Sec. 2.1, Algorithms 2, 3, 5) into out3 = {E_ca, M_l, M_a} (host or
 * device memory), keeps what the gradient needs (for every segment the
 * signed count of its crossing pairs' angle terms, for every vertex its
 * smallest gap) and synchronises the host (it reads back the status).
 * gr_diff_backward then writes to d_grad_xy ([V][2] FP32, DEVICE memory,
 * overwritten) the gradient of
 *   gout3[0] * E_ca + gout3[1] * M_l + gout3[2] * M_a
 * with respect to the coordinates, with that crossing set and those gaps held
 * fixed (the metrics are piecewise smooth; the gradient is the one of the
 * current piece).  The paper defines the metrics only; the gradient is this
 * library's addition (layout optimisation is the application the paper names).
 *
 * Streams: both calls are ordered after the work already queued on `stream`
 * (NULL: the layout's own stream), and later work on `stream` sees their
 * outputs.  gr_diff_forward returns GR_ENOTSUP while `stream` is being
 * captured into a CUDA graph.  gr_diff_backward with `gout3` in device memory
 * does not synchronise the host (host memory: it does, after copying gout3);
 * while `stream` is being captured it adds its kernels to the caller's graph
 * (gout3 must then be device memory), and each replay of that graph computes
 * the gradient of the last gr_diff_forward that completed before the replay
 * (the counts and gaps are read from the layout at replay time).  Replays,
 * backward calls and forwards of one layout share its scratch buffers, so
 * they must not overlap on the GPU.  GR_ENOTSUP also when the layout's own
 * stream is being captured while `stream` names another one. */
gr_status gr_diff_forward(gr_layout *layout, double ideal_rad, float *out3, gr_stream_t stream);
gr_status gr_diff_backward(gr_layout *layout, const float *gout3, float *d_grad_xy, gr_stream_t stream);

/* ------------------------------------------------------------- batches
 * Many independent layouts evaluated together (the batched form of the five
 * metrics): layouts are packed one after another.  `v_off` and `e_off` are
 * int64 [n_layouts + 1] prefix offsets (host or device memory): layout l owns
 * vertices [v_off[l], v_off[l+1]) of `xy` ([V][2] int32, V = v_off[n]) and
 * edges [e_off[l], e_off[l+1]) of `edges` ([E][2] int32), whose vertex ids
 * are local to the layout (0 <= id < v_off[l+1] - v_off[l]).  Results are
 * per layout, exactly those of gr_evaluate on each layout alone, except that
 * crossings always take the grid path (pairs_tested counts grid candidates).
 *
 * gr_batch_create validates (GR_EINVAL / GR_ERANGE as gr_layout_create),
 * plans one crossing grid per layout (cell size from a cost model on the
 * layout's segment count and length, shifted by an offset) and picks the
 * tile height of the pair kernel's work items (16 or 32 segments: two items
 * per warp or one), both by an autotuner that times the crossing pipeline of
 * each choice (opt->cell_log2 < 0 fixes the offset instead; the environment
 * variable GR_BATCH_TILE = 16 or 32 fixes the tile height; the tuned pair is
 * cached in the file named by GR_TUNE_CACHE when it is set), and
 * synchronises.  gr_batch_evaluate runs
 * the evaluation as one CUDA graph on the batch's stream (captured on the
 * first call and again when the metrics, ideal angle or d change), writes
 * gr_result [n_layouts] to `out` (host or device memory) and synchronises.
 * gr_batch_update replaces coordinates (and edges if not NULL), same sizes. */
typedef struct gr_batch gr_batch;

gr_status gr_batch_create(gr_batch **out, int64_t n_layouts, const int64_t *v_off, const int64_t *e_off,
                          const void *xy, gr_coord_type coord_type, const int32_t *edges,
                          const gr_options *opt, gr_stream_t stream);
gr_status gr_batch_update(gr_batch *batch, const void *xy, const int32_t *edges);
gr_status gr_batch_evaluate(gr_batch *batch, uint32_t metrics, const gr_params *params, gr_result *out);
gr_status gr_batch_destroy(gr_batch *batch);
/* The plan gr_batch_create settled on: the cell-size offset added to every
 * layout's cost-model choice and the tile height (16 or 32) of the pair
 * kernel's work items. */
gr_status gr_batch_tuning(const gr_batch *batch, int32_t *cell_offset, int32_t *tile);
/* gr_batch_evaluate without any host synchronisation: ordered after the work
 * queued on `stream` (NULL: the batch's stream), results written to
 * `d_results` (DEVICE memory, [n_layouts] gr_result) before anything queued
 * on `stream` afterwards runs; capturable into the caller's CUDA graph once a
 * gr_batch_evaluate with the same metrics and parameters has run.  Results
 * whose `metrics` field is 0 report a failed evaluation (gr_batch_evaluate
 * gives the error). */
gr_status gr_batch_evaluate_async(gr_batch *batch, uint32_t metrics, const gr_params *params, gr_result *d_results,
                                  gr_stream_t stream);

/* ------------------------------------------------------------- tracing
 * Phase timing: when enabled on a layout, every gr_layout_update,
 * gr_evaluate, gr_diff_forward and gr_diff_backward records CUDA events
 * around its phases on the layout's stream;
 * gr_profile_read returns the accumulated device time and call count of each
 * phase (optionally resetting them).  Events cost a few microseconds per
 * phase, so leave profiling off when not reading it. */
typedef enum {
    GR_PHASE_GATHER = 0,     /* input copies, validation, gather (a1) */
    GR_PHASE_EDGE_LENGTH,    /* a10 */
    GR_PHASE_MIN_ANGLE,      /* a9 */
    GR_PHASE_OCCL_BIN,       /* a8 binning: count, scan, stencil work */
    GR_PHASE_OCCL_PAIRS,     /* a8 scatter + pair kernel, or all-pairs tiles */
    GR_PHASE_CROSS_BIN,      /* a2-a3: DDA count, cell offsets, work items */
    GR_PHASE_CROSS_SCATTER,  /* a4: records sorted by cell */
    GR_PHASE_CROSS_PAIRS,    /* a6 per-cell pair kernel, or a7 all-pairs tiles */
    GR_PHASE_FINALIZE,       /* a11 and the result copy */
    GR_PHASE_DIFF_BACKWARD,  /* gr_diff_backward: the three adjoint kernels */
    GR_PHASE_STRIP_SORT,     /* gr_strip_crossings: records emitted and sorted by (l, r) in each strip */
    GR_PHASE_STRIP_COUNT,    /* gr_strip_crossings: merge by r, inverted pairs and their angle terms */
    GR_NUM_PHASES
} gr_phase;

typedef struct {
    double ms[16];     /* accumulated device milliseconds per gr_phase */
    int64_t calls[16]; /* number of times each phase ran */
} gr_profile;

gr_status gr_profile_enable(gr_layout *layout, int enable);
gr_status gr_profile_read(gr_layout *layout, gr_profile *out, int reset);

/* Bytes this layout has copied host->device and device->host since it was
 * created (inputs given in host memory, result and status read-backs). */
gr_status gr_io_bytes(gr_layout *layout, int64_t *h2d, int64_t *d2h);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all layouts, all threads). */
int64_t gr_kernel_launches(void);

/* ------------------------------------------------------- parts of a layout
 * The pair work of one layout in n_parts disjoint shares, for evaluating one
 * large layout on several GPUs (one part per rank) -- the spatial
 * partitioning by which Sec. 3.2.1-3.2.2 split the plane across machines,
 * made exact: every pair is counted in one cell (the owner of its
 * intersection point) and every cell's pairs are enumerated by work items,
 * so a split of the work items (the all-pairs tiles, the occlusion points)
 * splits the tallies with nothing counted twice.  Binning, minimum angle and
 * edge length variation are repeated by every part (they are O(|E|)).
 *
 * gr_evaluate_part evaluates part `part` (0 <= part < n_parts) of a
 * GR_COORD_I32 layout with the metrics and parameters of gr_evaluate and
 * writes its tallies to *out (host memory); it synchronises.  Summing the
 * gr_partial of all parts field by field (an integer all-reduce: every field
 * is an exact integer, and the values only part 0 reports are zero in the
 * others) and passing the sum to gr_combine_parts gives the gr_result of
 * gr_evaluate on the whole layout, bit for bit.  gr_combine_parts is host
 * arithmetic only (no GPU needed).  Errors: GR_EINVAL for a bad part or
 * NULL, GR_ENOTSUP for FP32 layouts, else as gr_evaluate. */
typedef struct {
    /* summed over the parts (each pair and each vertex pair counts in one part) */
    int64_t proper, touching, collinear_overlaps, occlusion_pairs;
    int64_t dev_hi32, dev_lo32; /* sum of |ideal - a_c| in units of pi / 2^32: dev_hi32 * 2^32 + dev_lo32 */
    /* part 0's values, zero in every other part */
    int64_t metrics, crossing_path, cell_log2, occlusion_path;
    int64_t zero_length_edges, pairs_tested, n_vertices_counted, grid_records;
    int64_t min_angle_sum_d_bits, M_a_bits, M_l_bits; /* IEEE-754 bit patterns of part 0's doubles */
} gr_partial;

gr_status gr_evaluate_part(gr_layout *layout, uint32_t metric_mask, const gr_params *params, int32_t part,
                           int32_t n_parts, gr_partial *out);
gr_status gr_combine_parts(const gr_partial *sum, const gr_params *params, gr_result *out);

/* ------------------------------------------------- no device allocation
 * Edge crossings and crossing angle of one layout of at most
 * GR_NOALLOC_MAX_EDGES edges, computed without allocating anything: for
 * callers that cannot call cudaMalloc -- a process whose device memory is
 * already committed to its own pool allocator under a fixed budget, or a
 * latency-critical caller that cannot afford cudaMalloc / cudaFree, which may
 * block or synchronise the device.  The paper has no counterpart; the
 * results equal gr_crossing_angle's on the same layout.
 *
 * `d_xy` [V][2] and `d_edges` [E][2] are DEVICE memory (int32, as for
 * gr_layout_create); `out` is device or host memory.  Work runs on `stream`
 * and the call synchronises it.  Scratch is a fixed array of about 1 MiB in
 * the library's device image, held by every GPU that loads the library
 * until the process exits.  Every call looks up the array's device address
 * (cudaGetSymbolAddress) with its device current; the first call on a device
 * is the set-up that also loads the library's module there, so make that
 * first call before any stream capture on the device.  Every call reuses the
 * same array: calls whose GPU work overlaps (other streams or host threads)
 * race and must be serialised by the caller.  GR_EINVAL for E above the
 * limit, for host-memory inputs, bad ids or self-loops; GR_ERANGE for
 * coordinates outside [0, 65536). */
#define GR_NOALLOC_MAX_EDGES 32768
gr_status gr_crossing_angle_noalloc(const int32_t *d_xy, int64_t V, const int32_t *d_edges, int64_t E,
                                    double ideal_rad, gr_crossing_angle_result *out, gr_stream_t stream);

/* Message of the last failed call on this host thread ("" if none). */
const char *gr_last_error(void);

/* Library version string. */
const char *gr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GR_H */
