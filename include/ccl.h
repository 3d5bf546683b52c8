/*
 * ccl.h - C ABI of the GB300 (sm_103a) library for run-based black-and-white
 * connected component analysis: foreground and background labelling, the
 * adjacency (inclusion) tree, per-component features and hole filling, as
 * defined by Lemaitre & Lacassagne, "A new run-based Connected Component
 * Labeling for efficiently analyzing and processing holes".
 *
 * Problem statement (the paper, Section 1 and Section 3 opening): assign a
 * number to every connected component of a binary image, foreground AND
 * background, compute the tree of which component surrounds which, compute
 * features on the fly, and fill holes by editing the tree and the
 * equivalence table rather than the pixels.
 *
 * Conventions shared by every call
 *   - Images are uint8, row-major [h][pitch] in device memory; a pixel is
 *     foreground when its byte is nonzero (the paper's algorithms take 0/1
 *     pixels). Bytes at x >= w are never interpreted.
 *   - Foreground components use 8-adjacency and background components
 *     4-adjacency (Algorithm 2); ccl_set_connectivity selects the
 *     complementary pair (Section 3.2: the 8-adjacency switch of Algorithm 2
 *     taken for the other colour).
 *   - Node 0 is the exterior: the background component made of every
 *     background pixel connected to the image border (Section 3.1 defines
 *     surrounding through paths to the exterior of the image). It exists even
 *     when it has no pixel.
 *   - Every other component is a node numbered 1.. in raster order of its
 *     first pixel (row-major). This is a dense renumbering of the paper's
 *     final roots (Algorithm 3), which are the labels of each component's
 *     top-most run. Results are therefore unique and compared bit for bit.
 *   - tree_parent[n] is the node that is adjacent to n and surrounds it
 *     (Section 3.1); it is the node of the pixel directly above n's first
 *     pixel, or 0 when that pixel is on row 0. tree_parent[0] = -1.
 *   - Features (Section 3.2, last paragraph) are int64, structure of arrays:
 *     features[f * capacity + n] for f = CCL_F_*: area S, inclusive bounding
 *     box, Sx = sum of x, Sy = sum of y, x = column and y = row, 0-based. A
 *     node without pixels (the exterior of an all-foreground image) has
 *     S = Sx = Sy = 0, xmin = ymin = INT64_MAX, xmax = ymax = -1.
 *   - Buffers are owned by the caller. A context owns only its scratch.
 *   - Every call enqueues its work on the given CUDA stream and returns
 *     without waiting, except ccl_get_counts. Argument errors return at once
 *     with nothing enqueued. Errors found on the device (node capacity
 *     exceeded, an iteration limit reached) are OR'd into counts[3] and the
 *     context's status, which ccl_get_counts returns.
 *   - There is no CPU fallback: without a usable sm_103a device, calls
 *     return CCL_ERR_CUDA.
 *   - A context is not thread-safe; calls on one context must come from one
 *     host thread at a time and, when they use different streams, the caller
 *     orders them (each analyze reuses the same scratch).
 */
#ifndef CCL_GB300_H
#define CCL_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t is a pointer to this opaque type; 0 is the legacy default stream. */
typedef struct CUstream_st *ccl_stream_t;

typedef struct ccl_ctx ccl_ctx;

typedef enum {
    CCL_OK = 0,
    CCL_ERR_ARG = 1,        /* bad size, null required pointer, bad enum */
    CCL_ERR_ALIGN = 2,      /* image pointer or pitch not 16-byte aligned */
    CCL_ERR_CAPACITY = 4,   /* more nodes than the output buffers hold, or a
                               batch larger than the context was created for */
    CCL_ERR_OOM = 8,        /* device allocation failed at create time */
    CCL_ERR_CUDA = 16,      /* a CUDA call failed / no usable device */
    CCL_ERR_ITER_LIMIT = 32,/* a bounded device loop gave up (never expected) */
    CCL_ERR_STATE = 64      /* call out of order (fill before analyze) */
} ccl_status;

enum {
    CCL_F_AREA = 0,
    CCL_F_XMIN = 1,
    CCL_F_YMIN = 2,
    CCL_F_XMAX = 3,
    CCL_F_YMAX = 4,
    CCL_F_SX = 5,
    CCL_F_SY = 6,
    CCL_F_COUNT = 7
};

enum {
    CCL_CONN_8FG_4BG = 0,  /* Algorithm 2 as printed: c8 = parity of the run */
    CCL_CONN_4FG_8BG = 1   /* the complementary pair: c8 = parity xor 1 */
};

/* Upper bound on the number of nodes of a w x h image:
 * ceil(h/2)*ceil(w/2) foreground components (one per 2x2 block at most)
 * + ceil(w*h/2) background components (a checkerboard) + 1 (the exterior).
 * Returns -1 for w <= 0 or h <= 0. */
int64_t ccl_node_capacity(int32_t w, int32_t h);

/* Create a context for images of exactly w x h pixels with row pitch `pitch`
 * bytes. Requirements: 1 <= w, 1 <= h, w*h < 2^31, pitch >= w,
 * pitch % 16 == 0 (else CCL_ERR_ALIGN). Allocates all device scratch now
 * (about 8 bytes per pixel); later calls allocate nothing. *out is set to
 * NULL on failure. */
ccl_status ccl_create(ccl_ctx **out, int32_t w, int32_t h, int32_t pitch);

/* Select the adjacency pair for later analyses of this context
 * (CCL_CONN_8FG_4BG, the default, or CCL_CONN_4FG_8BG). */
ccl_status ccl_set_connectivity(ccl_ctx *ctx, int32_t conn);

/* Analyse one image (Algorithms 1-4: segments, B&W unification, transitive
 * closure with the adjacency table, features, relabelling).
 *   d_img          [h][pitch] uint8, 16-byte aligned, nonzero = foreground
 *   d_fg_labels    [h][w] int32 out: node id of foreground pixels, -1 for
 *                  background pixels; NULL skips the label images
 *   d_bg_labels    [h][w] int32 out: node id of background pixels, -1 for
 *                  foreground pixels; must be NULL exactly when d_fg_labels is
 *   d_tree_parent  [cap] int32 out, cap = ccl_node_capacity(w, h)
 *   d_features     [CCL_F_COUNT][cap] int64 out
 *   d_counts       [4] int32 out: {n_nodes, n_foreground_nodes,
 *                  n_background_nodes (node 0 included), status bits}
 * Entries >= n_nodes of the node arrays are left untouched. The context
 * remembers d_tree_parent, d_features and d_counts for ccl_fill_holes; they
 * must stay valid until then. */
ccl_status ccl_analyze(ccl_ctx *ctx, const uint8_t *d_img, int32_t *d_fg_labels,
                       int32_t *d_bg_labels, int32_t *d_tree_parent, int64_t *d_features,
                       int32_t *d_counts, ccl_stream_t stream);

/* Hole filling on the node tables of the last ccl_analyze (Algorithm 3,
 * hole-filling branch), extended with an area threshold: a hole (background
 * node other than 0) whose own area is <= area_threshold is absorbed by its
 * parent, and so are the foreground children of an absorbed hole; deeper
 * holes are judged on their own area. area_threshold < 0 fills nothing;
 * INT64_MAX fills every hole, as Algorithm 3 does. No pixel is touched.
 *   d_fill_map          [cap] int32 out: surviving node of every node
 *   d_filled_features   [CCL_F_COUNT][cap] int64 out: merged features of
 *                       survivors; absorbed nodes get the empty features
 *   d_filled_parent     [cap] int32 out: map[parent] for survivors, -1 for
 *                       node 0 and for absorbed nodes
 * Returns CCL_ERR_STATE if no analyze was enqueued on this context. */
ccl_status ccl_fill_holes(ccl_ctx *ctx, int64_t area_threshold, int32_t *d_fill_map,
                          int64_t *d_filled_features, int32_t *d_filled_parent,
                          ccl_stream_t stream);

/* Area filter on either colour, the connected operator of which hole filling
 * is one case (Algorithm 3, hole-filling branch; Section 5 names filtering
 * components on their features as the general form):
 *   CCL_TARGET_HOLES    background nodes other than 0 with area <= T are
 *                       absorbed by their parent (exactly ccl_fill_holes);
 *   CCL_TARGET_OBJECTS  foreground nodes with area <= T are absorbed by their
 *                       parent background node (small objects removed).
 * The children of an absorbed node (other colour) are absorbed with it.
 * Outputs and rules otherwise as for ccl_fill_holes. */
enum { CCL_TARGET_HOLES = 0, CCL_TARGET_OBJECTS = 1 };
ccl_status ccl_filter_components(ccl_ctx *ctx, int32_t target, int64_t area_threshold, int32_t *d_map,
                                 int64_t *d_features, int32_t *d_parent, ccl_stream_t stream);

/* Label images after the last fill / filter of this context (Algorithm 4
 * applied to the filtered equivalence table): every pixel of node n takes
 * map[n], in d_fg_out when that survivor is foreground and in d_bg_out
 * otherwise (-1 in the other image). Reads the label images of the last
 * ccl_analyze; the outputs may be those same buffers (in place).
 * CCL_ERR_STATE if the last analyze wrote no label images or no fill ran. */
ccl_status ccl_relabel_filtered(ccl_ctx *ctx, int32_t *d_fg_out, int32_t *d_bg_out, ccl_stream_t stream);

/* Wait for the stream of the last call and read that call's counts (any
 * pointer may be NULL). Returns the OR of the device status bits of the last
 * analyze / fill (CCL_OK when clean). */
ccl_status ccl_get_counts(ccl_ctx *ctx, int32_t *n_nodes, int32_t *n_fg, int32_t *n_bg);

/* Euler number of the last analysed image (waits like ccl_get_counts): the
 * number of foreground components minus the number of holes, n_fg - (n_bg - 1)
 * (the paper lists it among the computed features, Sections 1 and 4). */
ccl_status ccl_get_euler(ccl_ctx *ctx, int64_t *euler);

/* ---------------------------------------------------------------- batches */

/* One image of a batch. All pointers are device pointers owned by the
 * caller; fg_labels/bg_labels may both be NULL; fill_map, filled_features
 * and filled_parent are used only by ccl_fill_holes_batched (NULL = skip
 * that image). capacity is the row stride of features / filled_features and
 * the length of tree_parent, fill_map and filled_parent; a capacity smaller
 * than ccl_node_capacity(w, h) is allowed and reported through
 * counts[3] |= CCL_ERR_CAPACITY when exceeded. */
typedef struct {
    const uint8_t *img;
    int32_t w, h, pitch;
    int32_t *fg_labels, *bg_labels;
    int32_t *tree_parent;
    int64_t *features;
    int32_t *counts;
    int64_t capacity;
    int32_t *fill_map;
    int64_t *filled_features;
    int32_t *filled_parent;
} ccl_image_desc;

/* Create a context for batches of up to max_images images whose pixel counts
 * sum to at most max_total_pixels and whose sides are at most max_side. */
ccl_status ccl_create_batched(ccl_ctx **out, int32_t max_images, int64_t max_total_pixels,
                              int32_t max_side);

/* Analyse n images at once: each phase of the method runs as one launch over
 * the tiles of all images (a persistent grid that draws tiles from a device
 * work counter). host_descs is copied before the call returns. When the
 * shape of the batch (sizes, pitches, label on/off) repeats, the launch
 * sequence is replayed from a cached CUDA graph. */
ccl_status ccl_analyze_batched(ccl_ctx *ctx, const ccl_image_desc *host_descs, int32_t n,
                               ccl_stream_t stream);

/* ccl_analyze_batched for frames that are still in host memory; the paper
 * has no counterpart: this is the ingest of a serving loop, which receives
 * frames from decoders or the network in host buffers. host_frames[i] holds
 * image i's h rows of w bytes, host_pitches[i] bytes apart (>= w); each is
 * copied asynchronously on the stream into host_descs[i].img (a device
 * buffer of the caller, rows host_descs[i].pitch bytes apart; one linear
 * copy when the two pitches are equal, else a 2-D copy) before the
 * analysis, which then runs as in ccl_analyze_batched. Frames in
 * page-locked memory (allocated pinned, or registered with cudaHostRegister)
 * are read by the copy engine directly, so they must stay unchanged until
 * the stream has passed the copy; other host memory is staged by the CUDA
 * driver. A null pointer, a non-positive size or a host pitch below w:
 * CCL_ERR_ARG, with nothing enqueued. */
ccl_status ccl_analyze_batched_from_host(ccl_ctx *ctx, const ccl_image_desc *host_descs,
                                         const uint8_t *const *host_frames, const int64_t *host_pitches,
                                         int32_t n, ccl_stream_t stream);

/* Hole filling for every image of the last batch that has fill buffers. */
ccl_status ccl_fill_holes_batched(ccl_ctx *ctx, int64_t area_threshold, ccl_stream_t stream);

/* Area filter (ccl_filter_components) for every image of the last batch
 * that has fill buffers. */
ccl_status ccl_filter_components_batched(ccl_ctx *ctx, int32_t target, int64_t area_threshold,
                                         ccl_stream_t stream);

/* ccl_relabel_filtered for the images of the last batch: host arrays of n
 * device pointers (n = the batch's image count), entry i for image i; a
 * NULL pair skips the image. An image needs label images and fill buffers
 * in its descriptor (CCL_ERR_STATE otherwise). */
ccl_status ccl_relabel_filtered_batched(ccl_ctx *ctx, int32_t *const *d_fg_out, int32_t *const *d_bg_out,
                                        ccl_stream_t stream);

/* Tile height for later analyses of this context: 32 rows (default) or 16.
 * Results are identical; the speed differs with the image (ccl.autotune
 * picks one per size class by timing the choices). */
ccl_status ccl_set_tile_rows(ccl_ctx *ctx, int32_t rows);

/* Tile width for later analyses of this context: 1024 columns (default, one
 * 32-pixel word per thread of a tile row's warp) or 512. Narrower tiles give
 * small or narrow images more tiles to spread over the SMs; wider tiles have
 * fewer tile edges to merge. Results are identical; ccl.autotune times the
 * choices. Other values: CCL_ERR_ARG. */
ccl_status ccl_set_tile_cols(ccl_ctx *ctx, int32_t cols);

/* Merge schedule for later analyses of this context: the number of work
 * items that share one 32-pixel word of a boundary between two bands of
 * tiles in the cross-tile merge (the unification of Algorithm 2 across tile
 * edges): 1, 2, 4 (default) or 8, each item taking 32 / items_per_word of
 * the word's columns. More items spread a dense boundary's unions over more
 * threads; fewer have less overhead on sparse boundaries. Results are
 * identical; ccl.autotune times the choices. Other values: CCL_ERR_ARG. */
ccl_status ccl_set_merge_split(ccl_ctx *ctx, int32_t items_per_word);

/* Enable (1) or disable (0) the CUDA-graph cache of ccl_analyze_batched and
 * ccl_analyze. */
ccl_status ccl_set_graph_cache(ccl_ctx *ctx, int32_t enable);

/* ------------------------------------------------------- instrumentation */

/* Phases of one analysis and of one hole filling, in launch order. */
enum {
    CCL_PHASE_PROLOGUE = 0,  /* per-image counters and the exterior node */
    CCL_PHASE_LABEL = 1,     /* runs and in-tile union-find (Algorithms 1, 2) */
    CCL_PHASE_MERGE = 2,     /* cross-tile and exterior links (Algorithm 2) */
    CCL_PHASE_RESOLVE = 3,   /* final roots of tile-border parts (Algorithm 3) */
    CCL_PHASE_SCAN = 4,      /* raster-order node numbering */
    CCL_PHASE_CANON = 5,     /* node ids of multi-tile components */
    CCL_PHASE_WRITE = 6,     /* labels, features, tree (Algorithms 3, 4) */
    CCL_PHASE_FILL_MAP = 7,  /* hole filling: survivors (Algorithm 3) */
    CCL_PHASE_FILL_MERGE = 8,/* hole filling: feature merge */
    CCL_PHASE_COUNT = 9
};

/* Record CUDA events between the phases of the next max_calls analyse / fill
 * calls (0 turns recording off). While recording, calls launch their
 * kernels directly instead of replaying a graph. */
ccl_status ccl_enable_phase_timing(ccl_ctx *ctx, int32_t max_calls);

/* Wait for the recorded calls and return, per phase, the summed device time
 * in milliseconds and the number of timed launches of that phase
 * (arrays of CCL_PHASE_COUNT). Clears the records. */
ccl_status ccl_read_phase_timing(ccl_ctx *ctx, double *total_ms, int64_t *count);

/* Number of kernels this context has enqueued since it was created
 * (graph replays count the kernels they contain). */
ccl_status ccl_get_launch_count(ccl_ctx *ctx, int64_t *launches);

/* ------------------------------------------------ allocation-free variant */

/* ccl_analyze_static has no counterpart in the paper. It runs the same
 * single-image analysis as ccl_create + ccl_analyze, but takes its scratch
 * from a fixed array that the library keeps on every GPU that loads it
 * (CCL_STATIC_SCRATCH_BYTES, held until the process exits) and allocates
 * nothing. It is meant for callers that cannot call cudaMalloc: code whose
 * device memory is owned entirely by another allocator, and latency-critical
 * loops that must not allocate after start-up because cudaMalloc / cudaFree
 * can synchronise the device and take unbounded time.
 *
 * Limits: w * h <= CCL_STATIC_MAX_PIXELS and w, h <= CCL_STATIC_MAX_SIDE;
 * larger images return CCL_ERR_CAPACITY with nothing enqueued. Other
 * arguments are as for ccl_analyze (8-foreground / 4-background adjacency),
 * with capacity = length of d_tree_parent and row stride of d_features
 * (ccl_node_capacity(w, h) always suffices; fewer slots are allowed and
 * reported through d_counts[3] |= CCL_ERR_CAPACITY when exceeded).
 *
 * The first call on a device (with that device current) looks up the
 * array's device address and sets kernel attributes; make that first call
 * before any stream capture. All calls share one array per device: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be ordered by the caller. Each call clears the counters it needs; the
 * array keeps the last call's tables otherwise. */
#define CCL_STATIC_MAX_PIXELS (1 << 20)
#define CCL_STATIC_MAX_SIDE 4096
#define CCL_STATIC_SCRATCH_BYTES (12 << 20)
ccl_status ccl_analyze_static(const uint8_t *d_img, int32_t w, int32_t h, int32_t pitch,
                              int32_t *d_fg_labels, int32_t *d_bg_labels, int32_t *d_tree_parent,
                              int64_t *d_features, int64_t capacity, int32_t *d_counts,
                              ccl_stream_t stream);

const char *ccl_status_string(ccl_status status);

/* Free the context and its scratch (waits for its pending work). */
void ccl_destroy(ccl_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* CCL_GB300_H */
