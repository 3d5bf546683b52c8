// Phase 1 of the analysis: per-tile run extraction and run unification.
//
// The paper's steps 1a and 1b (Algorithms 1 and 2) scan one row at a time and
// grow one equivalence table for the whole image. Here every tile of 32 rows
// x 1024 columns (or 16 rows, or 512 columns) is handled by one CTA, all rows
// at once:
//   - the tile's rows are loaded into registers one tile ahead (32 bytes per
//     thread, one thread per 32-pixel word) and packed into a
//     1-bit-per-pixel plane;
//   - run starts come from an XOR of each word with itself shifted by one
//     pixel (Algorithm 1's edge detection x0 xor x1), 32 pixels at a time; a
//     scan of the per-word counts numbers the runs in raster order (the run
//     ordinal), and every run is entered in a run list (its first pixel and
//     colour);
//   - every later step takes one thread per run (a balanced share of the
//     tile's runs per thread, whatever the run count of each word): the
//     overlap test of Algorithm 2 becomes a range of run ordinals in the row
//     above, found from two bit counts (an 8-adjacent colour's window is
//     widened by one pixel on each side, the c8 of Algorithm 2), and the
//     runs of that range with the same colour (every other run: colours
//     alternate along a row) are united;
//   - each union is a union by minimum run ordinal in a shared-memory parent
//     table, so the root of a tile-local component is its raster-first run,
//     as the paper's root is its smallest (top-most) label.
// Results kept for the later phases: every run's root ordinal (with its
// first pixel and colour), one record per local root, the roots of the tile's edge cells (for the cross-tile
// merge) and the first-pixel bits of components that stay inside the tile.
#include "ccl_dev.cuh"

namespace ccl {

// rootinfo layout: bits 0-15 local pixel index of the root's first pixel
// (row * tile width + column), bit 16 foreground, bit 17 touches a tile edge,
// bits 18-29 border ordinal of the root within the tile, bit 30 the
// component has a single run in the tile.
constexpr int RI_FG = 16, RI_BORDER = 17, RI_KB = 18, RI_SINGLE = 30;

__global__ void k_prologue(Batch B) {
    pdl_trigger();
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *B.s.status = 0;
        for (int k = 0; k < 8; ++k) B.s.work[k] = 0;
    }
    if (i < B.n_tiles) {
        // per tile: its image, and where its rows start for the row loads
        const int img = image_of_tile(B, i);
        const ImgDesc &d = B.desc[img];
        const TileGeo g = tile_geo(d, i - d.tile0, B.th, B.tw);
        const uint64_t src = (uint64_t)(d.img + (int64_t)g.y0 * d.pitch + g.x0);
        B.s.tstat[i] = make_int4(0, 0, 0, img);
        B.s.tsrc[i] = make_int4((int)(uint32_t)src, (int)(uint32_t)(src >> 32), d.pitch,
                                g.th | (((g.tw + 15) & ~15) << 8));
        TileHdr h;
        h.px = g.px;
        h.b = g.b;
        h.b_above = g.ty > 0 ? tile_geo(d, i - d.tile0 - d.TX, B.th, B.tw).b : 0;
        h.seg0 = d.seg0;
        h.img = img;
        h.tx = g.tx;
        h.y0 = g.y0;
        h.x0 = g.x0;
        h.th = g.th;
        h.tw = g.tw;
        h.TX = d.TX;
        h.w = d.w;
        B.s.thdr[i] = h;
    }
    if (i >= B.n_img) return;
    const ImgDesc &d = B.desc[i];
    for (int k = 0; k < 4; ++k) {
        d.counts[k] = 0;
        B.s.img_cnt[4 * i + k] = 0;
    }
    // the exterior: node 0, its own root in the device-wide union-find
    B.s.gp[i] = (unsigned long long)i;
    B.s.canon[i] = 0;
    const int64_t cap = d.cap;
    d.feat[0 * cap] = 0;
    d.feat[1 * cap] = INT64_MAX;
    d.feat[2 * cap] = INT64_MAX;
    d.feat[3 * cap] = -1;
    d.feat[4 * cap] = -1;
    d.feat[5 * cap] = 0;
    d.feat[6 * cap] = 0;
    d.parent[0] = -1;
    B.s.node_fg[d.node0] = 0;
}

// After the root ordinals are known, par[root] holds them: ordinal (bits
// 0-14), border ordinal (bits 15-26) and this tag (a run ordinal never has it).
constexpr uint32_t PAR_TAG = 0x80000000u, PAR_ORD = 0x7FFFu;

// 16-byte asynchronous copy global -> shared (both 16-byte aligned); the
// issuing thread waits for all of its copies with cp_async_wait_all.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// ------------------------------------------- run-ordinal union-find (shared)
// Parents are run ordinals; a root is its own parent and every link points
// to a smaller ordinal, so a native shared atomicMin both links and resolves
// races: the union by minimum of Algorithm 2 on the tile's label space.

__device__ __forceinline__ uint32_t ld_par(const uint32_t *par, uint32_t a) {
    return *(volatile const uint32_t *)(par + a);
}

// Find with path halving: every other node on the way up is pointed at its
// grandparent, one of its ancestors whatever unions run at the same time.
__device__ __forceinline__ uint32_t run_find_halving(uint32_t *par, uint32_t a, bool *ok) {
    for (int it = 0; it < LOCAL_FIND_LIMIT; ++it) {
        const uint32_t p = ld_par(par, a);
        if (p == a) return a;
        const uint32_t g = ld_par(par, p);
        if (g == p) return p;
        *(volatile uint32_t *)(par + a) = g;
        a = g;
    }
    *ok = false;
    return a;
}

// Plain find (no writes), for the closure once every union is done.
__device__ __forceinline__ uint32_t run_find(const uint32_t *par, uint32_t a, bool *ok) {
    for (int it = 0; it < LOCAL_FIND_LIMIT; ++it) {
        const uint32_t p = ld_par(par, a);
        if (p == a) return a;
        a = p;
    }
    *ok = false;
    return a;
}

// Returns the root the two sets were joined under (an ancestor of both a
// and b), where the caller's next union with a may start its find.
__device__ __forceinline__ uint32_t run_union(uint32_t *par, uint32_t a, uint32_t b, bool *ok) {
    for (int it = 0; it < LOCAL_UNION_LIMIT; ++it) {
        a = run_find_halving(par, a, ok);
        b = run_find_halving(par, b, ok);
        if (a == b || !*ok) return a;
        if (a < b) { const uint32_t t = a; a = b; b = t; }
        const uint32_t old = atomicMin(par + a, b);
        if (old == a) return b;
        a = old;
    }
    *ok = false;
    return a;
}

// Tile geometry of the labeller: TH rows x TW columns (WPR = TW / 32 words
// per row; a warp holds 32 / WPR rows), one thread per 32-pixel word (NT
// threads), up to NPX runs.
template <int TH, int TW> struct LabelCfg {
    static constexpr int WPR = TW / 32;
    static constexpr int LOG_TW = TW == 1024 ? 10 : 9;
    static constexpr int NT = TH * WPR;       // threads = words of a tile
    static constexpr int NW = NT / 32;        // warps
    static constexpr int NPX = TH * TW;       // pixels = most runs
    static constexpr int KMAX = NPX / NT;     // rounds of the per-run loops (32)
    static_assert(TW == 512 || TW == 1024, "tile widths");
};

template <int TH, int TW>
constexpr size_t label_smem() {
    using C = LabelCfg<TH, TW>;
    return (size_t)C::NPX * 4            // par
           + (size_t)C::NPX * 2          // run list
           + (size_t)C::NPX / 8          // border flags per run
           + 3 * (size_t)C::NT * 4       // colour, run-start and node-bit planes
           + ((size_t)C::NT + 8) * 2     // run ordinal of each word's first run
           + 2 * (size_t)C::KMAX * C::NW * 4;  // multi-run roots and root counts per (round, warp)
}

// End column (exclusive) of run i of row r: the next run's start on the same
// row, else the tile width.
template <int TW, uint32_t LMASK = 0xFFFFu>
__device__ __forceinline__ int run_end(const uint16_t *list, int i, int n, int r, int tw) {
    constexpr int LOG_TW = TW == 1024 ? 10 : 9;
    if (i + 1 < n) {
        const int pn = (int)((list[i + 1] & LMASK) >> 1);
        if ((pn >> LOG_TW) == r) return pn & (TW - 1);
    }
    return tw;
}

// Ordinal of the run covering column x of row r (the word holds a run start
// at or before x, or the run started in an earlier word of the row).
template <int WPR>
__device__ __forceinline__ int ord_at(const uint16_t *sOrd, const uint32_t *sE, int r, int x) {
    const int wi = r * WPR + (x >> 5);
    return (int)sOrd[wi] + __popc(sE[wi] & mask_le(x & 31)) - 1;
}

// Same-colour runs of row rr that touch run [s, e) of colour c (rr = the row
// above or below): the ordinal range [*jf, *jl], every other ordinal. An
// 8-adjacent colour's window is widened by one pixel on each side.
template <int CONN, int WPR>
__device__ __forceinline__ void touching(const uint16_t *sOrd, const uint32_t *sE, const uint32_t *sC, int rr,
                                         int s, int e, uint32_t c, int tw, int *jf, int *jl) {
    const int adj8 = CONN ? (int)(c ^ 1u) : (int)c;
    const int xa = max(s - adj8, 0), xb = min(e - 1 + adj8, tw - 1);
    const int wa = rr * WPR + (xa >> 5), wb = rr * WPR + (xb >> 5);
    const uint32_t ea = sE[wa];
    const int ba = (int)sOrd[wa];
    const int oa = ba + __popc(ea & mask_le(xa & 31)) - 1;
    int ob;
    if (wb == wa) {
        ob = ba + __popc(ea & mask_le(xb & 31)) - 1;
    } else {
        ob = ord_at<WPR>(sOrd, sE, rr, xb);
    }
    const uint32_t ca = (sC[wa] >> (xa & 31)) & 1u;
    *jf = oa + (int)(ca != c);
    *jl = ob;
}

// One CTA per tile at a time, one thread per 32-pixel word. The image rows
// of the next tile are loaded into registers while the CTA works on the
// current one: thread 0 claims tiles from the work counter two ahead and
// fetches the header of the next tile into shared memory.
//
// Root ordinals: the roots of components with more than one run come first
// (in raster order of their first pixel), then the single-run roots; the
// feature pass keeps on-chip records for the former only. Border ordinals
// (roots touching a tile edge) are handed out in any order.
template <int CONN, int TH, int TW>
__global__ void __launch_bounds__(LabelCfg<TH, TW>::NT, 1024 / LabelCfg<TH, TW>::NT) k_label(Batch B) {
    using C = LabelCfg<TH, TW>;
    constexpr int NT = C::NT, NW = C::NW, NPX = C::NPX, KMAX = C::KMAX, WPR = C::WPR, LOG_TW = C::LOG_TW;
    // tiles of at most 16384 pixels leave bit 15 of a run-list entry free: it
    // marks a run that a same-colour run of the row below touches
    constexpr bool BELOW = NPX <= 16384;
    constexpr uint32_t LMASK = BELOW ? 0x7FFFu : 0xFFFFu;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *par = (uint32_t *)smem;                         // [NPX]
    uint16_t *list = (uint16_t *)(par + NPX);                 // [NPX] pixel index << 1 | colour
    uint32_t *sBrd = (uint32_t *)(list + NPX);                // [NPX / 32] root touches a tile edge
    uint32_t *sC = sBrd + NPX / 32;                           // [TH][WPR] colour bits
    uint32_t *sE = sC + NT;                                   // [TH][WPR] run starts
    uint32_t *sNB = sE + NT;                                  // [TH][WPR] first pixels of internal nodes
    uint32_t *sCnt = sNB + NT;                                // [KMAX][NW] multi | single << 16
    uint32_t *sMul = sCnt + KMAX * NW;                        // [KMAX][NW] multi-run roots (ballot)
    uint16_t *sOrd = (uint16_t *)(sMul + KMAX * NW);          // [NT + 1] first run ordinal of each word
    __shared__ int sT[2], sWarpTot[32], sNb, sFg, sOk;
    __shared__ TileHdr sHdr[2];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r_w = tid / WPR, l_w = tid % WPR;   // this thread's word: row, word in row
    pdl_wait();   // the prologue's headers and counters are visible

    // the rows of a tile: 32 bytes of row r_w at column 32 l_w (16-byte loads
    // that stay inside the row's bytes rounded up to 16, hence its pitch)
    uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
    auto load_rows = [&](int4 rec) {
        const uint8_t *src = (const uint8_t *)(((uint64_t)(uint32_t)rec.y << 32) | (uint32_t)rec.x);
        const int rows = rec.w & 0xFF, bytes = rec.w >> 8;
        v0 = v1 = make_uint4(0, 0, 0, 0);
        if (r_w < rows) {
            const uint4 *p = (const uint4 *)(src + (int64_t)r_w * rec.z + 32 * l_w);
            if (32 * l_w < bytes) v0 = __ldcs(p);
            if (32 * l_w + 16 < bytes) v1 = __ldcs(p + 1);
        }
    };
    if (tid == 0) {
        const int t0 = atomicAdd(&B.s.work[0], 1);
        sT[0] = t0;
        sT[1] = atomicAdd(&B.s.work[0], 1);
        if (t0 < B.n_tiles) sHdr[0] = B.s.thdr[t0];   // later headers: cp.async one tile ahead
        sOk = 1;
        sFg = 0;
        sNb = 0;
    }
    for (int i = tid; i < NPX / 32; i += NT) sBrd[i] = 0u;
    sNB[tid] = 0u;
    __syncthreads();
    if (sT[0] < B.n_tiles) load_rows(B.s.tsrc[sT[0]]);

    for (int q = 0;; q ^= 1) {
        const int t = sT[q];
        if (t >= B.n_tiles) break;
        const int tn = sT[q ^ 1];   // the next tile (claimed one tile ago)
        const TileHdr &h = sHdr[q];
        // thread 0 claims the tile after next and copies the next tile's
        // header into the other slot (nobody reads it during this tile); both
        // are waited for at the end of the tile
        int claim = 0;
        if (tid == 0) {
            claim = atomicAdd(&B.s.work[0], 1);
            if (tn < B.n_tiles)
                for (int k = 0; k < (int)(sizeof(TileHdr) / 16); ++k)
                    cp_async16((char *)&sHdr[q ^ 1] + 16 * k, (const char *)(B.s.thdr + tn) + 16 * k);
        }
        const int img = h.img, y0 = h.y0, x0 = h.x0, th = h.th, tw = h.tw;
        const ImgDesc &d = B.desc[img];
        const int64_t rowwords = (int64_t)h.TX * WPR;
        const int64_t plane0 = (h.seg0 + (int64_t)y0 * h.TX + h.tx) * WPR;  // word (y0, tile col)
        int4 rec_next = make_int4(0, 0, 0, 0);
        if (tn < B.n_tiles) rec_next = B.s.tsrc[tn];   // used for the row loads below
        bool ok = true;

        // ---- the rows: pack bits, find run starts, number the runs
        uint32_t word = 0, e = 0;
        {
            const int vcnt = min(max(tw - 32 * l_w, 0), 32);
            const uint32_t vm = r_w < th ? (vcnt >= 32 ? FULL : ((1u << vcnt) - 1u)) : 0u;
            word = (nz16(v0) | (nz16(v1) << 16)) & vm;
            if (r_w < th) B.s.fgbits[plane0 + r_w * rowwords + l_w] = word;
            sC[tid] = word;
            // runs never cross a tile's left edge (a warp holds whole rows)
            const uint32_t left = __shfl_up_sync(FULL, word, 1);
            const uint32_t prev = (word << 1) | (l_w ? (left >> 31) : 0u);
            e = ((word ^ prev) | (l_w == 0 ? 1u : 0u)) & vm;
            sE[tid] = e;
        }
        int tot;
        const int wex = warp_excl_sum(__popc(e), &tot);
        if (lane == 0) sWarpTot[warp] = tot;
        __syncthreads();
        int n;   // runs of the tile
        {
            int wb, wt;
            const int pre = warp_excl_sum(lane < NW ? sWarpTot[lane] : 0, &wt);
            wb = __shfl_sync(FULL, pre, warp);
            n = wt;
            const int o0 = wb + wex;
            sOrd[tid] = (uint16_t)o0;
            if (tid == 0) sOrd[NT] = (uint16_t)n;
            // run list and parents: every run its own root
            uint32_t m = e;
            int o = o0;
            const int base = r_w * TW + 32 * l_w;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                list[o] = (uint16_t)(((base + b) << 1) | ((word >> b) & 1u));
                par[o] = (uint32_t)o;
                ++o;
            }
        }
        __syncthreads();

        // ---- contacts of every run with the row above (Algorithm 2). All
        // runs are united at the same time: the union by minimum with
        // atomicMin stays correct under concurrent unions, and the paper's
        // row-by-row order only matters for the provisional labels, not for
        // the classes.
        for (int i = tid; i < n; i += NT) {
            const uint32_t v = list[i] & LMASK;
            const int pix = (int)(v >> 1), r = pix >> LOG_TW, s = pix & (TW - 1);
            if (r == 0) continue;
            const int e_ = run_end<TW, LMASK>(list, i, n, r, tw);
            int jf, jl;
            touching<CONN, WPR>(sOrd, sE, sC, r - 1, s, e_, v & 1u, tw, &jf, &jl);
            uint32_t ra = (uint32_t)i;   // an ancestor of run i: where the next union's find starts
            for (int j = jf; j <= jl; j += 2) {
                // run j has a same-colour contact below (read by the closure)
                if (BELOW) atomicOr((uint32_t *)list + (j >> 1), 1u << (15 + 16 * (j & 1)));
                ra = run_union(par, ra, (uint32_t)j, &ok);
            }
        }
        // the rows of the next tile: their loads complete during the rest of
        // this tile
        if (tn < B.n_tiles) load_rows(rec_next);
        __syncthreads();

        // ---- closure: every run points at its root (Algorithm 3, in-tile);
        // roots touching a tile edge are marked; each root is classified (a
        // root is its component's raster-first run, so nothing above touches
        // it: the component has more runs exactly when the root's run touches
        // a same-colour run of the row below, which the unions above flagged
        // in the run list, or a touching range tells on the widest tiles) and
        // counted per (round, warp)
        int k = 0;
        for (int i0 = 0; i0 < n; i0 += NT, ++k) {
            const int i = i0 + tid;
            bool is_root = false, multi = false;
            if (i < n) {
                const uint32_t vr = list[i], v = vr & LMASK;
                const int pix = (int)(v >> 1), r = pix >> LOG_TW, s = pix & (TW - 1);
                const int e_ = run_end<TW, LMASK>(list, i, n, r, tw);
                const uint32_t p = ld_par(par, (uint32_t)i);
                const uint32_t root = p == (uint32_t)i ? p : run_find(par, p, &ok);
                if (root != p) par[i] = root;
                is_root = root == (uint32_t)i;
                if (r == 0 || r == th - 1 || s == 0 || e_ == tw) atomicOr(&sBrd[root >> 5], 1u << (root & 31));
                if (BELOW) {
                    multi = (vr >> 15) & 1u;
                } else if (is_root && r + 1 < th) {
                    int jf, jl;
                    touching<CONN, WPR>(sOrd, sE, sC, r + 1, s, e_, v & 1u, tw, &jf, &jl);
                    multi = jf <= jl;
                }
            }
            const uint32_t bm = __ballot_sync(FULL, is_root && multi), bs = __ballot_sync(FULL, is_root && !multi);
            if (lane == 0) {
                sCnt[k * NW + warp] = (uint32_t)__popc(bm) | ((uint32_t)__popc(bs) << 16);
                sMul[k * NW + warp] = bm;
            }
        }
        __syncthreads();

        // ---- root ordinals: exclusive scan of the counts in raster order
        // (round-major, then warp), multi-run roots and single-run roots
        const int nk = k;   // rounds of this tile
        uint32_t cnt_ex, cnt_tot;
        {
            const uint32_t cv = tid < nk * NW ? sCnt[tid] : 0u;
            uint32_t wt;
            const uint32_t ex = warp_excl_sum_u32(cv, &wt);
            if (lane == 0) sWarpTot[warp] = (int)wt;
            __syncthreads();
            uint32_t bt;
            const uint32_t wpre = warp_excl_sum_u32(lane < NW ? (uint32_t)sWarpTot[lane] : 0u, &bt);
            cnt_ex = __shfl_sync(FULL, wpre, warp) + ex;
            cnt_tot = bt;
            if (tid < nk * NW) sCnt[tid] = cnt_ex;
        }
        __syncthreads();
        const int n_multi = (int)(cnt_tot & 0xFFFFu), n_single = (int)(cnt_tot >> 16);

        // ---- per root: record, border slot, ordinal into par[root]
        uint32_t *rr = B.s.run_root + h.px;
        uint32_t *ri = B.s.rootinfo + h.px;
        const uint32_t slot0 = (uint32_t)(B.n_img + h.b);
        int nfg = 0;
        k = 0;
        for (int i0 = 0; i0 < n; i0 += NT, ++k) {
            const int i = i0 + tid;
            bool is_root = false, border = false;
            if (i < n) {
                is_root = ld_par(par, (uint32_t)i) == (uint32_t)i;
                border = is_root && ((sBrd[i >> 5] >> (i & 31)) & 1u);
            }
            const uint32_t bm = sMul[k * NW + warp];
            const bool multi = (bm >> lane) & 1u;
            const uint32_t bs = __ballot_sync(FULL, is_root && !multi);
            const uint32_t bb = __ballot_sync(FULL, border);
            int kb0 = 0;
            if (lane == 0 && bb) kb0 = atomicAdd(&sNb, __popc(bb));
            kb0 = __shfl_sync(FULL, kb0, 0);
            if (is_root) {
                const uint32_t base = sCnt[k * NW + warp];
                const uint32_t lt = mask_lt(lane);
                const int kk = multi ? (int)(base & 0xFFFFu) + __popc(bm & lt)
                                     : n_multi + (int)(base >> 16) + __popc(bs & lt);
                const uint32_t v = list[i] & LMASK;
                const int pix = (int)(v >> 1);
                const uint32_t fg = v & 1u;
                uint32_t info = (uint32_t)pix | (fg << RI_FG) | (multi ? 0u : (1u << RI_SINGLE));
                uint32_t pv = PAR_TAG | (uint32_t)kk;
                if (border) {
                    const int kb = kb0 + __popc(bb & lt);
                    const uint32_t slot = slot0 + kb;
                    const int r = pix >> LOG_TW, s = pix & (TW - 1);
                    const int64_t key = (int64_t)(y0 + r) * h.w + x0 + s;
                    B.s.gp[slot] = ((unsigned long long)(key + 1) << 32) | slot;
                    B.s.binfo[slot] = (uint32_t)kk | (fg << 16);
                    info |= (1u << RI_BORDER) | ((uint32_t)kb << RI_KB);
                    pv |= (uint32_t)kb << 15;
                } else {
                    nfg += (int)fg;
                    atomicOr(&sNB[pix >> 5], 1u << (pix & 31));
                }
                ri[kk] = info;
                par[i] = pv;
            }
        }
        __syncthreads();

        // ---- per run: root ordinal and the run's list entry; per edge cell:
        // border ordinal of its root; first pixels of the internal nodes
        for (int i = tid; i < n; i += NT) {
            uint32_t v = ld_par(par, (uint32_t)i);
            if (!(v & PAR_TAG)) v = ld_par(par, v);
            rr[i] = ((v & PAR_ORD) << 16) | (list[i] & LMASK);
        }
        // (cell i of the loop is also its offset: top, bottom, left, right)
        uint16_t *eg = B.s.edges + h.b;
        const int nedge = 2 * tw + 2 * th;
        for (int i = tid; i < nedge; i += NT) {
            int r, c;
            if (i < tw) { r = 0; c = i; }
            else if (i < 2 * tw) { r = th - 1; c = i - tw; }
            else if (i < 2 * tw + th) { r = i - 2 * tw; c = 0; }
            else { r = i - 2 * tw - th; c = tw - 1; }
            uint32_t v = ld_par(par, (uint32_t)ord_at<WPR>(sOrd, sE, r, c));
            if (!(v & PAR_TAG)) v = ld_par(par, v);
            eg[i] = (uint16_t)((v >> 15) & 0xFFFu);
        }
        if (r_w < th) B.s.nodebits[plane0 + r_w * rowwords + l_w] = sNB[tid];
        sNB[tid] = 0u;
        for (int i = tid; i < (n + 31) / 32; i += NT) sBrd[i] = 0u;
        nfg = warp_sum(nfg);
        if (lane == 0 && nfg) atomicAdd(&sFg, nfg);
        if (!ok) atomicAnd(&sOk, 0);
        if (tid == 0) {
            cp_async_wait_all();   // the next header has landed
            sT[q] = claim;         // read as the next-but-one tile after this barrier
        }
        __syncthreads();
        if (tid == 0) {
            B.s.tstat[t] = make_int4(n, n_multi | (n_single << 16), sNb, img);
            if (sFg) atomicAdd(&B.s.img_cnt[4 * img + 1], sFg);
            if (!sOk) set_status(B, d, ST_ITER);
            sFg = 0;
            sOk = 1;
            sNb = 0;
        }
    }
    pdl_trigger();   // no tile left: the next kernel may be scheduled
}

void launch_prologue(const Batch &B, cudaStream_t st) {
    const int n = B.n_img > B.n_tiles ? B.n_img : B.n_tiles;
    k_prologue<<<(n + 255) / 256, 256, 0, st>>>(B);
}

template <int CONN, int TH, int TW>
static void launch_label_shape(const Batch &B, const LaunchCfg &c, cudaStream_t st) {
    using C = LabelCfg<TH, TW>;
    const int grid = min(B.n_tiles, (1024 / C::NT) * c.sms);
    launch_dep(k_label<CONN, TH, TW>, grid, C::NT, label_smem<TH, TW>(), st, B);
}

template <int CONN>
static void launch_label_conn(const Batch &B, const LaunchCfg &c, cudaStream_t st) {
    if (B.tw == 1024) {
        if (B.th == 32) launch_label_shape<CONN, 32, 1024>(B, c, st);
        else launch_label_shape<CONN, 16, 1024>(B, c, st);
    } else {
        if (B.th == 32) launch_label_shape<CONN, 32, 512>(B, c, st);
        else launch_label_shape<CONN, 16, 512>(B, c, st);
    }
}

void launch_label(const Batch &B, const LaunchCfg &c, cudaStream_t st) {
    if (B.conn == 0) launch_label_conn<0>(B, c, st);
    else launch_label_conn<1>(B, c, st);
}

template <typename K>
static cudaError_t configure_smem(K kernel, size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

template <int CONN>
static cudaError_t configure_label_conn() {
    cudaError_t e = configure_smem(k_label<CONN, 32, 1024>, label_smem<32, 1024>());
    if (e == cudaSuccess) e = configure_smem(k_label<CONN, 16, 1024>, label_smem<16, 1024>());
    if (e == cudaSuccess) e = configure_smem(k_label<CONN, 32, 512>, label_smem<32, 512>());
    if (e == cudaSuccess) e = configure_smem(k_label<CONN, 16, 512>, label_smem<16, 512>());
    return e;
}

cudaError_t configure_label() {
    cudaError_t e = configure_label_conn<0>();
    if (e == cudaSuccess) e = configure_label_conn<1>();
    return e;
}

}  // namespace ccl
