/*
 * CPU oracle for black-and-white connected component analysis.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do. It shares no code, header, table or helper with the
 * CUDA library.
 *
 * It computes, by plain breadth-first flood fill, the result that the paper
 * (Lemaitre & Lacassagne, "A new run-based Connected Component Labeling for
 * efficiently analyzing and processing holes") defines:
 *   - components of foreground (nonzero) pixels with 8-adjacency and of
 *     background pixels with 4-adjacency (Section 3.2, Algorithm 2 and the
 *     remark on the complementary adjacency; the complementary pair
 *     4-foreground / 8-background is selected by conn = 1);
 *   - the exterior of the image as background component 0: every background
 *     pixel connected to the image border (Section 3.1: surrounding is
 *     defined by the paths to the exterior of the image);
 *   - the adjacency (inclusion) tree, parent[C] = the component that is both
 *     adjacent to C and surrounds C (Section 3.1), read at the pixel directly
 *     above the raster-first pixel of C (Section 3.1, "initial adjacency": a
 *     new label records the label next to its top-most pixel);
 *   - per component features: bounding box and first moments S, Sx, Sy
 *     (Section 3.2, last paragraph);
 *   - hole filling (Algorithm 3, the hole-filling branch), extended with an
 *     area threshold.
 *
 * Canonical numbering: the exterior is node 0; every other component gets
 * 1 + its rank in raster order of its first pixel. This is a dense
 * renumbering of the paper's final roots, which are the labels of each
 * component's top-most (raster-first) run.
 *
 * Feature layout: structure of arrays, feat[f * cap + n] for f in
 * {AREA, XMIN, YMIN, XMAX, YMAX, SX, SY}. Coordinates are 0-based column x
 * and row y; the box is inclusive. A component with no pixel (the exterior
 * of an all-foreground image) has area = Sx = Sy = 0, xmin = ymin =
 * INT64_MAX and xmax = ymax = -1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_AREA = 0, OR_XMIN, OR_YMIN, OR_XMAX, OR_YMAX, OR_SX, OR_SY, OR_NF };

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_CAPACITY = 3, OR_ERR_OOM = 4 };

/* Flood the component of (x0, y0) with the given label. Pixels of the same
 * colour as the seed join through 4-adjacency, and also through the four
 * diagonals when eight is nonzero. */
static void flood(const uint8_t *img, int32_t w, int32_t h, int32_t pitch,
                  int32_t *node, int32_t *queue, int32_t x0, int32_t y0,
                  int32_t label, int eight)
{
    const int colour = img[(int64_t)y0 * pitch + x0] != 0;
    int64_t head = 0, tail = 0;
    node[(int64_t)y0 * w + x0] = label;
    queue[tail++] = y0 * w + x0;
    while (head < tail) {
        const int32_t p = queue[head++];
        const int32_t y = p / w, x = p % w;
        for (int dy = -1; dy <= 1; ++dy) {
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0) continue;
                if (!eight && dx != 0 && dy != 0) continue;
                const int32_t nx = x + dx, ny = y + dy;
                if (nx < 0 || ny < 0 || nx >= w || ny >= h) continue;
                if ((img[(int64_t)ny * pitch + nx] != 0) != colour) continue;
                if (node[(int64_t)ny * w + nx] != -1) continue;
                node[(int64_t)ny * w + nx] = label;
                queue[tail++] = ny * w + nx;
            }
        }
    }
}

/*
 * Label one image.
 *   img      [h][pitch] bytes, nonzero = foreground; bytes at x >= w ignored
 *   conn     0: 8-foreground / 4-background; 1: 4-foreground / 8-background
 *   node     out [h][w] node id of every pixel (may be NULL)
 *   fg, bg   out [h][w] node id for pixels of that colour, -1 otherwise
 *            (either may be NULL)
 *   parent   out [cap] tree parent, parent[0] = -1
 *   feat     out [OR_NF][cap]
 *   node_fg  out [cap] 1 for foreground nodes, 0 for background (may be NULL)
 *   counts   out [4] = {N, foreground nodes, background nodes incl. node 0, 0}
 * Returns OR_ERR_CAPACITY (counts still filled) when N > cap.
 */
int oracle_analyze(const uint8_t *img, int32_t w, int32_t h, int32_t pitch,
                   int32_t conn, int32_t *node_out, int32_t *fg, int32_t *bg,
                   int32_t *parent, int64_t *feat, int64_t cap,
                   uint8_t *node_fg, int32_t *counts)
{
    if (w <= 0 || h <= 0 || pitch < w || cap < 1 || (conn != 0 && conn != 1))
        return OR_ERR_ARG;
    const int64_t npx = (int64_t)w * h;
    if (npx > INT32_MAX - 2) return OR_ERR_ARG;
    const int fg_eight = (conn == 0), bg_eight = (conn == 1);

    int32_t *node = node_out ? node_out : (int32_t *)malloc(sizeof(int32_t) * npx);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * npx);
    int32_t *first = (int32_t *)malloc(sizeof(int32_t) * (npx + 1));
    if (!node || !queue || !first) {
        if (!node_out) free(node);
        free(queue);
        free(first);
        return OR_ERR_OOM;
    }
    for (int64_t i = 0; i < npx; ++i) node[i] = -1;

    /* Exterior: background pixels reachable from any border background pixel. */
    for (int32_t y = 0; y < h; ++y) {
        for (int32_t x = 0; x < w; ++x) {
            const int border = (x == 0 || y == 0 || x == w - 1 || y == h - 1);
            if (!border) continue;
            if (img[(int64_t)y * pitch + x] != 0) continue;
            if (node[(int64_t)y * w + x] != -1) continue;
            flood(img, w, h, pitch, node, queue, x, y, 0, bg_eight);
        }
    }
    first[0] = -1;

    /* Every other component, numbered in raster order of its first pixel. */
    int32_t next = 1;
    for (int32_t y = 0; y < h; ++y) {
        for (int32_t x = 0; x < w; ++x) {
            if (node[(int64_t)y * w + x] != -1) continue;
            const int isfg = img[(int64_t)y * pitch + x] != 0;
            first[next] = y * w + x;
            flood(img, w, h, pitch, node, queue, x, y, next,
                  isfg ? fg_eight : bg_eight);
            ++next;
        }
    }
    const int32_t n_nodes = next;

    /* Colour of every node, from its first pixel; node 0 is background. */
    int32_t n_fg = 0;
    for (int32_t n = 1; n < n_nodes; ++n) {
        const int32_t p = first[n];
        const int isfg = img[(int64_t)(p / w) * pitch + (p % w)] != 0;
        n_fg += isfg;
        if (node_fg && n < cap) node_fg[n] = (uint8_t)isfg;
    }
    if (node_fg) node_fg[0] = 0;

    if (counts) {
        counts[0] = n_nodes;
        counts[1] = n_fg;
        counts[2] = n_nodes - n_fg;
        counts[3] = 0;
    }

    const int64_t nstore = n_nodes < cap ? n_nodes : cap;
    if (feat) {
        for (int64_t n = 0; n < nstore; ++n) {
            feat[OR_AREA * cap + n] = 0;
            feat[OR_SX * cap + n] = 0;
            feat[OR_SY * cap + n] = 0;
            feat[OR_XMIN * cap + n] = INT64_MAX;
            feat[OR_YMIN * cap + n] = INT64_MAX;
            feat[OR_XMAX * cap + n] = -1;
            feat[OR_YMAX * cap + n] = -1;
        }
        for (int32_t y = 0; y < h; ++y) {
            for (int32_t x = 0; x < w; ++x) {
                const int32_t n = node[(int64_t)y * w + x];
                if (n >= cap) continue;
                feat[OR_AREA * cap + n] += 1;
                feat[OR_SX * cap + n] += x;
                feat[OR_SY * cap + n] += y;
                if (x < feat[OR_XMIN * cap + n]) feat[OR_XMIN * cap + n] = x;
                if (y < feat[OR_YMIN * cap + n]) feat[OR_YMIN * cap + n] = y;
                if (x > feat[OR_XMAX * cap + n]) feat[OR_XMAX * cap + n] = x;
                if (y > feat[OR_YMAX * cap + n]) feat[OR_YMAX * cap + n] = y;
            }
        }
    }

    if (parent) {
        parent[0] = -1;
        for (int64_t n = 1; n < nstore; ++n) {
            const int32_t p = first[n];
            const int32_t y = p / w, x = p % w;
            parent[n] = (y == 0) ? 0 : node[(int64_t)(y - 1) * w + x];
        }
    }

    for (int32_t y = 0; y < h; ++y) {
        for (int32_t x = 0; x < w; ++x) {
            const int64_t i = (int64_t)y * w + x;
            const int isfg = img[(int64_t)y * pitch + x] != 0;
            if (fg) fg[i] = isfg ? node[i] : -1;
            if (bg) bg[i] = isfg ? -1 : node[i];
        }
    }

    if (!node_out) free(node);
    free(queue);
    free(first);
    return n_nodes > cap ? OR_ERR_CAPACITY : OR_OK;
}

/*
 * Component filtering by area, the connected operator the paper applies to
 * holes (Algorithm 3, hole-filling branch: a root whose surrounding
 * component is not the exterior is made equivalent to it) and names for
 * other features (Section 5). target_fg = 0 fills holes: a background
 * component other than the exterior is absorbed by its parent when its own
 * area is at most T. target_fg = 1 removes small objects the same way: a
 * foreground component with area at most T is absorbed by its parent
 * background component. Either way the children of an absorbed component
 * (of the other colour) are absorbed with it. Nodes are visited in
 * increasing order, so a parent is settled before its children
 * (parent[n] < n).
 *   target(n) = colour(n) == target_fg, n != 0 and area[n] <= T  (T < 0: none)
 *   map[n]    = map[parent[n]] if target(n), or if colour(n) != target_fg,
 *               n != 0 and target(parent[n]); otherwise n.
 * Survivors (map[s] == s) get the merge (sum / min / max) of the features of
 * all nodes mapped to them; absorbed nodes get the empty-component features.
 * filled_parent[s] = map[parent[s]] for survivors (-1 for node 0), and -1 for
 * absorbed nodes. The tree passed in is not modified.
 */
int oracle_filter(int32_t n_nodes, const int32_t *parent, const int64_t *feat,
                  int64_t cap, const uint8_t *node_fg, int32_t target_fg, int64_t T,
                  int32_t *map, int64_t *ffeat, int64_t fcap, int32_t *fparent)
{
    if (n_nodes < 1 || n_nodes > cap || n_nodes > fcap) return OR_ERR_ARG;
    if (target_fg != 0 && target_fg != 1) return OR_ERR_ARG;
    uint8_t *hole = (uint8_t *)malloc((size_t)n_nodes);
    if (!hole) return OR_ERR_OOM;
    for (int32_t n = 0; n < n_nodes; ++n) {
        const int is_target_colour = (node_fg[n] != 0) == (target_fg != 0);
        hole[n] = (uint8_t)(T >= 0 && n != 0 && is_target_colour &&
                            feat[OR_AREA * cap + n] <= T);
        if (hole[n] || (n != 0 && !is_target_colour && hole[parent[n]]))
            map[n] = map[parent[n]];
        else
            map[n] = n;
    }
    for (int32_t n = 0; n < n_nodes; ++n) {
        ffeat[OR_AREA * fcap + n] = 0;
        ffeat[OR_SX * fcap + n] = 0;
        ffeat[OR_SY * fcap + n] = 0;
        ffeat[OR_XMIN * fcap + n] = INT64_MAX;
        ffeat[OR_YMIN * fcap + n] = INT64_MAX;
        ffeat[OR_XMAX * fcap + n] = -1;
        ffeat[OR_YMAX * fcap + n] = -1;
    }
    for (int32_t n = 0; n < n_nodes; ++n) {
        const int32_t s = map[n];
        ffeat[OR_AREA * fcap + s] += feat[OR_AREA * cap + n];
        ffeat[OR_SX * fcap + s] += feat[OR_SX * cap + n];
        ffeat[OR_SY * fcap + s] += feat[OR_SY * cap + n];
        if (feat[OR_XMIN * cap + n] < ffeat[OR_XMIN * fcap + s])
            ffeat[OR_XMIN * fcap + s] = feat[OR_XMIN * cap + n];
        if (feat[OR_YMIN * cap + n] < ffeat[OR_YMIN * fcap + s])
            ffeat[OR_YMIN * fcap + s] = feat[OR_YMIN * cap + n];
        if (feat[OR_XMAX * cap + n] > ffeat[OR_XMAX * fcap + s])
            ffeat[OR_XMAX * fcap + s] = feat[OR_XMAX * cap + n];
        if (feat[OR_YMAX * cap + n] > ffeat[OR_YMAX * fcap + s])
            ffeat[OR_YMAX * fcap + s] = feat[OR_YMAX * cap + n];
    }
    for (int32_t n = 0; n < n_nodes; ++n) {
        if (map[n] != n)
            fparent[n] = -1;
        else
            fparent[n] = parent[n] < 0 ? -1 : map[parent[n]];
    }
    free(hole);
    return OR_OK;
}

/* Hole filling: the filter with background as the target colour. */
int oracle_fill(int32_t n_nodes, const int32_t *parent, const int64_t *feat,
                int64_t cap, const uint8_t *node_fg, int64_t T, int32_t *map,
                int64_t *ffeat, int64_t fcap, int32_t *fparent)
{
    return oracle_filter(n_nodes, parent, feat, cap, node_fg, 0, T, map, ffeat,
                         fcap, fparent);
}
