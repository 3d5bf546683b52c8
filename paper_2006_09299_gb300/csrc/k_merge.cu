// Phase 2: join tile-local components across tile edges, settle every
// component's final root, and number the components.
//
//   k_merge    the cross-tile part of Algorithm 2's unification: pairs of
//              edge cells of neighbouring tiles are linked with the same
//              overlap rules as inside a tile, and background cells on the
//              image border are linked to the exterior (the epilog of
//              Algorithm 2, extended to all four borders).
//   k_resolve  the transitive closure of Algorithm 3 on the border roots:
//              each points straight at its final root, the component's
//              raster-first local root; final roots that are not the
//              exterior mark their first pixel in the node bit plane.
//   k_scan_*   exclusive scan of node counts per tile row, in raster order:
//              node id = 1 + number of node first-pixels before this one.
//   k_canon    node ids of the border-root components, their count, and the
//              initial feature records that the write phase accumulates into.
#include "ccl_dev.cuh"

namespace ccl {

__device__ __forceinline__ int image_of_item(const Batch &B, int64_t item, int kind) {
    int lo = 0, hi = B.n_img - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const ImgDesc &m = B.desc[mid];
        const int64_t v = kind == 0 ? m.hitem0 : (kind == 1 ? m.vitem0 : m.pitem0);
        if (v <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

enum { TOP, BOTTOM, LEFT, RIGHT };

// Union-find slot of the border root that owns edge cell `pos` (a column for
// TOP / BOTTOM, a row for LEFT / RIGHT) of tile lt.
__device__ __forceinline__ uint32_t edge_slot(const Batch &B, const ImgDesc &d, int lt, int side, int pos) {
    const TileHdr &h = B.s.thdr[d.tile0 + lt];
    const int64_t eb = h.b;
    const int tw = h.tw;
    const int off = side == TOP ? pos : side == BOTTOM ? tw + pos : side == LEFT ? 2 * tw + pos : 2 * tw + h.th + pos;
    return (uint32_t)(B.n_img + eb) + B.s.edges[eb + off];
}

__device__ __forceinline__ uint32_t plane_word(const Batch &B, const ImgDesc &d, int y, int j) {
    return B.s.fgbits[(d.seg0 + (int64_t)y * d.TX) * B.wpr + j];
}

__device__ __forceinline__ bool pixel_fg(const Batch &B, const ImgDesc &d, int y, int x) {
    return (plane_word(B, d, y, x >> 5) >> (x & 31)) & 1u;
}

// Run starts of a row word, with a forced start at every tile column start
// (runs never cross a tile's left edge; wpr words per tile row).
__device__ __forceinline__ uint32_t starts(uint32_t c, uint32_t cl, int j, int wpr, uint32_t vm) {
    const uint32_t prev = (c << 1) | (cl >> 31);
    return ((c ^ prev) | ((j & (wpr - 1)) == 0 ? 1u : 0u)) & vm;
}

template <int CONN>
__device__ void merge_rows(const Batch &B, const ImgDesc &d, int64_t item, bool *ok) {
    const int64_t words = (int64_t)d.TX * B.wpr;
    const int lt = B.log_tw, tm = B.tw - 1;
    const int hs = B.hsplit;
    const int part = (int)(item % hs);   // columns [part, part + 1) x 32 / hsplit of the word
    item /= hs;
    const int bb = (int)(item / words);        // boundary between band bb and bb+1
    const int j = (int)(item - (int64_t)bb * words);
    const int span = 32 / hs;
    const uint32_t range = span == 32 ? FULL : (((1u << span) - 1u) << (span * part));
    const int x = 32 * j;
    if (x >= d.w) return;
    const int yu = (bb + 1) * B.th - 1, yd = yu + 1;
    const int vcnt = min(d.w - x, 32);
    const uint32_t vm = vcnt >= 32 ? FULL : ((1u << vcnt) - 1u);
    const uint32_t cu = plane_word(B, d, yu, j), cd = plane_word(B, d, yd, j);
    const uint32_t cul = j ? plane_word(B, d, yu, j - 1) : 0u, cdl = j ? plane_word(B, d, yd, j - 1) : 0u;
    const uint32_t cur = (j + 1) < words ? plane_word(B, d, yu, j + 1) : 0u;
    const uint32_t cdr = (j + 1) < words ? plane_word(B, d, yd, j + 1) : 0u;
    const uint32_t eu = starts(cu, cul, j, B.wpr, vm), ed = starts(cd, cdl, j, B.wpr, vm);
    const uint32_t vml = FULL;   // the word to the left is always fully valid
    const uint32_t vmr = (x + 32 < d.w) ? (d.w - x - 32 >= 32 ? FULL : ((1u << (d.w - x - 32)) - 1u)) : 0u;
    const uint32_t ad = CONN ? (~cd & vm) : cd, au = CONN ? (~cu & vm) : cu;
    const uint32_t bd = CONN ? cd : (~cd & vm), bu = CONN ? cu : (~cu & vm);
    const uint32_t adl = CONN ? (~cdl & vml) : cdl, aul = CONN ? (~cul & vml) : cul;
    const uint32_t adr = CONN ? (~cdr & vmr) : cdr, aur = CONN ? (~cur & vmr) : cur;
    const uint32_t ad_prev = (ad << 1) | (j ? adl >> 31 : 0u), ad_next = (ad >> 1) | (adr << 31);
    const uint32_t au_prev = (au << 1) | (j ? aul >> 31 : 0u), au_next = (au >> 1) | (aur << 31);
    const uint32_t va = ad & au & ((ed & ad) | (eu & au)) & range;
    const uint32_t vb = bd & bu & ((ed & bd) | (eu & bu)) & range;
    const uint32_t d1 = ad & ~au & au_next & ~ad_next & range;
    const uint32_t d2 = ad & ~au & au_prev & ~ad_prev & range;
    const int ltu = bb * d.TX, ltd = (bb + 1) * d.TX;   // first tile of each band
    uint32_t m = va | vb;
    while (m) {
        const int xx = x + __ffs(m) - 1;
        m &= m - 1;
        global_union(B.s.gp, edge_slot(B, d, ltd + (xx >> lt), TOP, xx & tm),
                     edge_slot(B, d, ltu + (xx >> lt), BOTTOM, xx & tm), ok);
    }
    m = d1;
    while (m) {
        const int xx = x + __ffs(m) - 1;
        m &= m - 1;
        const int xu = xx + 1;
        global_union(B.s.gp, edge_slot(B, d, ltd + (xx >> lt), TOP, xx & tm),
                     edge_slot(B, d, ltu + (xu >> lt), BOTTOM, xu & tm), ok);
    }
    m = d2;
    while (m) {
        const int xx = x + __ffs(m) - 1;
        m &= m - 1;
        const int xu = xx - 1;
        global_union(B.s.gp, edge_slot(B, d, ltd + (xx >> lt), TOP, xx & tm),
                     edge_slot(B, d, ltu + (xu >> lt), BOTTOM, xu & tm), ok);
    }
}

template <int CONN>
__device__ void merge_cols(const Batch &B, const ImgDesc &d, int64_t item, bool *ok) {
    const int vb = (int)(item / d.h);          // boundary between tile columns vb and vb+1
    const int y = (int)(item - (int64_t)vb * d.h);
    const int x0 = (vb + 1) * B.tw;
    const int ty = y / B.th, r = y - ty * B.th;
    const int th = min(B.th, d.h - ty * B.th);
    const int ltl = ty * d.TX + vb, ltr = ltl + 1;
    const bool cl = pixel_fg(B, d, y, x0 - 1), cr = pixel_fg(B, d, y, x0);
    if (cl == cr) {
        bool redundant = false;
        if (r > 0) redundant = pixel_fg(B, d, y - 1, x0 - 1) == cl && pixel_fg(B, d, y - 1, x0) == cl;
        if (!redundant)
            global_union(B.s.gp, edge_slot(B, d, ltl, RIGHT, r), edge_slot(B, d, ltr, LEFT, r), ok);
    }
    if (r + 1 < th) {
        const bool dl = pixel_fg(B, d, y + 1, x0 - 1), dr = pixel_fg(B, d, y + 1, x0);
        const bool al = CONN ? !cl : cl, ar = CONN ? !cr : cr;
        const bool bl = CONN ? !dl : dl, br = CONN ? !dr : dr;
        if (al && br && !ar && !bl)   // (y, x0-1) - (y+1, x0)
            global_union(B.s.gp, edge_slot(B, d, ltl, RIGHT, r), edge_slot(B, d, ltr, LEFT, r + 1), ok);
        if (ar && bl && !al && !br)   // (y, x0) - (y+1, x0-1)
            global_union(B.s.gp, edge_slot(B, d, ltr, LEFT, r), edge_slot(B, d, ltl, RIGHT, r + 1), ok);
    }
}

// Background cells on the image border belong to the exterior.
__device__ void merge_perimeter(const Batch &B, const ImgDesc &d, int img, int64_t item, bool *ok) {
    const int64_t words = (int64_t)d.TX * B.wpr;
    const uint32_t ext = (uint32_t)img;
    if (item < 2 * words) {
        const bool bottom = item >= words;
        const int j = (int)(bottom ? item - words : item);
        const int x = 32 * j;
        if (x >= d.w) return;
        const int y = bottom ? d.h - 1 : 0;
        const int vcnt = min(d.w - x, 32);
        const uint32_t vm = vcnt >= 32 ? FULL : ((1u << vcnt) - 1u);
        const uint32_t c = plane_word(B, d, y, j);
        const uint32_t cl = j ? plane_word(B, d, y, j - 1) : FULL;
        const uint32_t bg = ~c & vm, bgl = ~cl;
        const uint32_t bprev = (bg << 1) | (bgl >> 31);
        const uint32_t st = (bg & ~bprev) | ((j & (B.wpr - 1)) == 0 ? (bg & 1u) : 0u);
        const int lt0 = bottom ? (d.TY - 1) * d.TX : 0;
        uint32_t m = st;
        while (m) {
            const int xx = x + __ffs(m) - 1;
            m &= m - 1;
            global_union(B.s.gp, edge_slot(B, d, lt0 + (xx >> B.log_tw), bottom ? BOTTOM : TOP, xx & (B.tw - 1)),
                         ext, ok);
        }
        return;
    }
    const bool right = item >= 2 * words + d.h;
    const int y = (int)(item - 2 * words - (right ? d.h : 0));
    const int x = right ? d.w - 1 : 0;
    if (pixel_fg(B, d, y, x)) return;
    const int ty = y / B.th, r = y - ty * B.th;
    if (r > 0 && !pixel_fg(B, d, y - 1, x)) return;   // same run of border cells, already linked
    const int lt = ty * d.TX + (right ? d.TX - 1 : 0);
    global_union(B.s.gp, edge_slot(B, d, lt, right ? RIGHT : LEFT, r), ext, ok);
}

template <int CONN>
__global__ void k_merge(Batch B) {
    pdl_trigger();
    pdl_wait();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool ok = true;
    int img = -1;
    if (g < B.n_hitems) {
        img = image_of_item(B, g, 0);
        const ImgDesc &d = B.desc[img];
        merge_rows<CONN>(B, d, g - d.hitem0, &ok);
    } else if (g < B.n_hitems + B.n_vitems) {
        const int64_t it = g - B.n_hitems;
        img = image_of_item(B, it, 1);
        const ImgDesc &d = B.desc[img];
        merge_cols<CONN>(B, d, it - d.vitem0, &ok);
    } else if (g < B.n_hitems + B.n_vitems + B.n_pitems) {
        const int64_t it = g - B.n_hitems - B.n_vitems;
        img = image_of_item(B, it, 2);
        const ImgDesc &d = B.desc[img];
        merge_perimeter(B, d, img, it - d.pitem0, &ok);
    }
    if (!ok) set_status(B, B.desc[img], ST_ITER);
}

// A group of g warps per tile (tiles strided over the groups of the grid;
// g = 1 when the tiles outnumber the resident warps, up to a whole CTA when
// there are few), one thread per border root: settle the final root of each
// border root. (The finds walk chains in L2, so the more of them run side by
// side the better.)
__global__ void __launch_bounds__(NTHREADS) k_resolve(Batch B, int g) {
    pdl_trigger();
    pdl_wait();
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (NTHREADS / 32) + (threadIdx.x >> 5);   // global warp
    const int groups = gridDim.x * (NTHREADS / 32) / g, gt = (gw % g) * 32 + lane;
    for (int t = gw / g; t < B.n_tiles; t += groups) {
        const TileHdr &h = B.s.thdr[t];
        const int img = h.img;
        const ImgDesc &d = B.desc[img];
        const int nb = B.s.tstat[t].z;
        const uint32_t slot0 = (uint32_t)(B.n_img + h.b);
        bool ok = true;
        int nfg = 0;
        for (int kb = gt; kb < nb; kb += 32 * g) {
            const uint32_t slot = slot0 + kb;
            const uint32_t root = global_find(B.s.gp, slot, &ok);
            if (root != slot) {
                B.s.gp[slot] = ld_volatile_u64(B.s.gp + root);
            } else {
                const int64_t key = (int64_t)(B.s.gp[slot] >> 32) - 1;
                const int y = (int)(key / h.w), x = (int)(key - (int64_t)y * h.w);
                atomicOr(&B.s.nodebits[(h.seg0 + (int64_t)y * h.TX) * B.wpr + (x >> 5)], 1u << (x & 31));
                nfg += (B.s.binfo[slot] >> 16) & 1;
            }
        }
        nfg = warp_sum(nfg);
        if (lane == 0 && nfg) atomicAdd(&B.s.img_cnt[4 * img + 1], nfg);
        if (!ok) set_status(B, d, ST_ITER);
    }
}

// Node count of every segment (one tile row: wpr words of the node plane).
__global__ void __launch_bounds__(SCAN_B) k_scan_count(Batch B) {
    pdl_trigger();
    pdl_wait();
    __shared__ int sPart[SCAN_B / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
    int c = 0;
    if (s < B.n_segs) {
        // one segment per thread: its words in independent vector loads
        const uint4 *w4 = reinterpret_cast<const uint4 *>(B.s.nodebits + s * B.wpr);
        const int nq = B.wpr / 4;
        uint4 v[WPR_MAX / 4];
#pragma unroll
        for (int q = 0; q < WPR_MAX / 4; ++q) v[q] = q < nq ? w4[q] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int q = 0; q < WPR_MAX / 4; ++q) c += __popc(v[q].x) + __popc(v[q].y) + __popc(v[q].z) + __popc(v[q].w);
        B.s.seg_cnt[s] = c;
    }
    const int wsum = warp_sum(c);
    if (lane == 0) sPart[warp] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int k = 0; k < SCAN_B / 32; ++k) tot += sPart[k];
        B.s.blk_sum[blockIdx.x] = tot;
    }
}

// Exclusive scan of the block sums, one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan_blocks(Batch B, int nblk) {
    pdl_trigger();
    pdl_wait();
    __shared__ int sW[32];
    __shared__ int sCarry;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) sCarry = 0;
    __syncthreads();
    for (int base = 0; base < nblk; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < nblk ? B.s.blk_sum[i] : 0;
        int wt;
        const int ex = warp_excl_sum(v, &wt);
        if (lane == 0) sW[warp] = wt;
        __syncthreads();
        int wpre = 0, btot = 0;
        for (int k = 0; k < 32; ++k) {
            const int s = sW[k];
            if (k < warp) wpre += s;
            btot += s;
        }
        const int carry = sCarry;
        if (i < nblk) B.s.blk_sum[i] = carry + wpre + ex;
        __syncthreads();
        if (threadIdx.x == 0) sCarry = carry + btot;
        __syncthreads();
    }
}

// Segment bases: block base + exclusive scan inside the block.
__global__ void __launch_bounds__(SCAN_B) k_scan_apply(Batch B) {
    pdl_trigger();
    pdl_wait();
    __shared__ int sW[SCAN_B / 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * SCAN_B + threadIdx.x;
    const int v = s < B.n_segs ? B.s.seg_cnt[s] : 0;
    int wt;
    const int ex = warp_excl_sum(v, &wt);
    if (lane == 0) sW[warp] = wt;
    __syncthreads();
    int wbase = 0;
    for (int k = 0; k < warp; ++k) wbase += sW[k];
    const int base = B.s.blk_sum[blockIdx.x];
    if (s < B.n_segs) B.s.seg_base[s] = base + wbase + ex;
    if (s == B.n_segs - 1) B.s.seg_base[B.n_segs] = base + wbase + ex + v;
}

// Node id of the component whose first pixel has raster index key: 1 + the
// nodes of the segments before, + the first-pixel bits before it in its
// segment (the segment's words read with independent vector loads).
__device__ __forceinline__ int node_id_of_key(const Batch &B, const ImgDesc &d, int64_t key) {
    const int y = (int)(key / d.w), x = (int)(key - (int64_t)y * d.w);
    const int64_t s = d.seg0 + (int64_t)y * d.TX + (x >> B.log_tw);
    int id = 1 + B.s.seg_base[s] - B.s.seg_base[d.seg0];
    const uint32_t *w = B.s.nodebits + s * B.wpr;
    const int l = (x & (B.tw - 1)) >> 5;
    const uint4 *w4 = reinterpret_cast<const uint4 *>(w);
#pragma unroll
    for (int q = 0; q < WPR_MAX / 4; ++q) {
        if (4 * q < l) {
            const uint4 v = w4[q];
            id += __popc(v.x) + (4 * q + 1 < l ? __popc(v.y) : 0) + (4 * q + 2 < l ? __popc(v.z) : 0) +
                  (4 * q + 3 < l ? __popc(v.w) : 0);
        }
    }
    return id + __popc(w[l] & mask_lt(x & 31));
}

__global__ void __launch_bounds__(NTHREADS) k_canon(Batch B, int g) {
    pdl_trigger();
    pdl_wait();
    // image totals
    for (int i = blockIdx.x * NTHREADS + threadIdx.x; i < B.n_img; i += gridDim.x * NTHREADS) {
        const ImgDesc &d = B.desc[i];
        const int n = 1 + B.s.seg_base[d.seg0 + (int64_t)d.h * d.TX] - B.s.seg_base[d.seg0];
        const int nfg = B.s.img_cnt[4 * i + 1];
        d.counts[0] = n;
        d.counts[1] = nfg;
        d.counts[2] = n - nfg;
        if (n > d.cap) set_status(B, d, ST_CAPACITY);
    }
    // a group of g warps per tile (as in k_resolve), one thread per border
    // root: node ids and initial records of the final roots
    const int gw = blockIdx.x * (NTHREADS / 32) + (threadIdx.x >> 5);
    const int groups = gridDim.x * (NTHREADS / 32) / g, gt = (gw % g) * 32 + (threadIdx.x & 31);
    for (int t = gw / g; t < B.n_tiles; t += groups) {
        const TileHdr &h = B.s.thdr[t];
        const ImgDesc &d = B.desc[h.img];
        const int nb = B.s.tstat[t].z;
        const uint32_t slot0 = (uint32_t)(B.n_img + h.b);
        for (int kb = gt; kb < nb; kb += 32 * g) {
            const uint32_t slot = slot0 + kb;
            const unsigned long long v = B.s.gp[slot];
            if ((uint32_t)v != slot) continue;
            const int64_t key = (int64_t)(v >> 32) - 1;
            const int id = node_id_of_key(B, d, key);
            B.s.canon[slot] = id;
            if (id < d.cap) {
                const int64_t cap = d.cap;
                d.feat[0 * cap + id] = 0;
                d.feat[1 * cap + id] = INT64_MAX;
                d.feat[2 * cap + id] = key / d.w;
                d.feat[3 * cap + id] = -1;
                d.feat[4 * cap + id] = -1;
                d.feat[5 * cap + id] = 0;
                d.feat[6 * cap + id] = 0;
                if (id < d.ncap) B.s.node_fg[d.node0 + id] = (uint8_t)((B.s.binfo[slot] >> 16) & 1);
            }
        }
    }
}

void launch_merge(const Batch &B, cudaStream_t st) {
    const int64_t n = B.n_hitems + B.n_vitems + B.n_pitems;
    if (n == 0) return;
    const int grid = (int)((n + 255) / 256);
    if (B.conn == 0)
        launch_dep(k_merge<0>, grid, 256, 0, st, B);
    else
        launch_dep(k_merge<1>, grid, 256, 0, st, B);
}

// Warps per tile for the border-root kernels: the resident warps shared out
// over the tiles, a power of two from 1 to a CTA's 8.
static int border_group(const Batch &B, const LaunchCfg &c) {
    const int64_t warps = (int64_t)8 * c.sms * (NTHREADS / 32);
    int g = 1;
    while (g < NTHREADS / 32 && (int64_t)B.n_tiles * g * 2 <= warps) g *= 2;
    return g;
}

static int border_grid(const Batch &B, const LaunchCfg &c, int g) {
    const int64_t blocks = ((int64_t)B.n_tiles * g + NTHREADS / 32 - 1) / (NTHREADS / 32);
    return (int)max((int64_t)1, min(blocks, (int64_t)8 * c.sms));
}

void launch_resolve(const Batch &B, const LaunchCfg &c, cudaStream_t st) {
    const int g = border_group(B, c);
    launch_dep(k_resolve, border_grid(B, c, g), NTHREADS, 0, st, B, g);
}

void launch_scan(const Batch &B, cudaStream_t st) {
    const int nblk = (int)((B.n_segs + SCAN_B - 1) / SCAN_B);
    launch_dep(k_scan_count, nblk, SCAN_B, 0, st, B);
    launch_dep(k_scan_blocks, 1, 1024, 0, st, B, nblk);
    launch_dep(k_scan_apply, nblk, SCAN_B, 0, st, B);
}

void launch_canon(const Batch &B, const LaunchCfg &c, cudaStream_t st) {
    const int g = border_group(B, c);
    launch_dep(k_canon, border_grid(B, c, g), NTHREADS, 0, st, B, g);
}

}  // namespace ccl
