// Phase 3: per tile, write the two label images, the features and the tree.
//
// This is the paper's relabelling (Algorithm 4: every run's pixels receive
// the final label of the run) fused with the feature merge and the
// adjacency-to-root step of Algorithm 3:
//   - each run's record from phase 1 (its root ordinal, first pixel and
//     colour) gives the run's node id, through a per-tile table of the
//     roots' node ids;
//   - features (ComputeFeatures of Algorithm 2: S, Sx, Sy and the box) are
//     accumulated per local root in shared memory, one thread per run; the
//     runs of one root on one row that sit two runs apart (a component
//     crossing the row many times) are summed first with a warp scan, so
//     such a component costs one shared update per warp and row; components
//     that stay inside the tile are then written with plain
//     stores, and border components are merged into their node with atomics,
//     first combined per tile in a small hash table; a root with a single
//     run in the tile takes its features from that run;
//   - the tree parent of a node whose first pixel lies in this tile is the
//     node of the pixel directly above that first pixel (the initial
//     adjacency of Algorithm 2, kept for the root by Algorithm 3), set in
//     the per-root loop by the local root that starts at that pixel;
//   - the label rows are written 4 pixels per lane, so that each warp
//     stores 512 contiguous bytes per instruction.
#include "ccl_dev.cuh"

namespace ccl {

// Launch shape per tile shape (TH rows x TW columns, WPR = TW / 32 words per
// row): NT threads, each holding two 32-pixel words of the tile (word t and
// word t + NT, so a warp holds 32 / WPR rows in each half of the tile),
// several CTAs per SM so that one streams its label rows while another
// computes. Root ordinals of a
// tile put the roots of components with several runs first, then the
// single-run roots. Multi-run roots below MAXR accumulate their features in
// on-chip records (more spill to global atomics); node ids of the first
// MAXID roots are kept on chip (the rest are computed when needed);
// 2^HASH_BITS entries combine the feature contributions of border roots.
template <int TH, int TW> struct WriteCfg;
template <> struct WriteCfg<32, 1024> {
    static constexpr int NT = 512, MAXR = 2048, MAXID = 8192, HASH_BITS = 9, CTAS = 2;
};
template <> struct WriteCfg<16, 1024> {
    static constexpr int NT = 256, MAXR = 768, MAXID = 2560, HASH_BITS = 8, CTAS = 5;
};
template <> struct WriteCfg<32, 512> {
    static constexpr int NT = 256, MAXR = 768, MAXID = 2560, HASH_BITS = 8, CTAS = 5;
};
template <> struct WriteCfg<16, 512> {
    static constexpr int NT = 128, MAXR = 320, MAXID = 1280, HASH_BITS = 7, CTAS = 10;
};

template <int TH, int TW>
constexpr size_t write_smem() {
    using C = WriteCfg<TH, TW>;
    constexpr size_t NWD = (size_t)TH * (TW / 32);
    return (size_t)C::MAXR * 6 * 4                // records
           + (size_t)C::MAXID * 4                 // node id per root
           + 3 * NWD * 4                          // colour, run-start and node-bit planes
           + (size_t)7 * 4 * (1 << C::HASH_BITS)  // border combining table
           + (NWD + 8) * 2                        // first run ordinal of each word
           + NWD * 2;                             // node bits before each word in its row
}

// Per-tile combining table for the features of border roots, which the
// cross-tile merge may have joined to the same node: every entry of one tile
// belongs to the tile's image, so the key is the node id and the sums are
// tile-relative and fit 32 bits (area <= 2^15, sum of x - x0 < 2^24, sum of
// y - y0 < 2^20); rows is a mask of the tile rows the contributions cover.
template <int BITS> struct TileHash {
    static constexpr int N = 1 << BITS;
    static constexpr uint32_t EMPTY = 0xFFFFFFFFu;
    uint32_t *key, *area, *sx, *sy, *xmin, *xmax, *rows;
    __device__ __forceinline__ explicit TileHash(uint32_t *mem) {
        key = mem;
        area = key + N;
        sx = area + N;
        sy = sx + N;
        xmin = sy + N;
        xmax = xmin + N;
        rows = xmax + N;
    }
    __device__ __forceinline__ void reset(int e) const {
        key[e] = EMPTY;
        area[e] = 0u;
        sx[e] = 0u;
        sy[e] = 0u;
        xmin[e] = EMPTY;
        xmax[e] = 0u;
        rows[e] = 0u;
    }
    // false when the probes found no free entry (the caller adds to the
    // global record directly)
    __device__ __forceinline__ bool push(uint32_t id, uint32_t a, uint32_t lsx, uint32_t lsy, uint32_t lx0,
                                         uint32_t lx1, uint32_t rmask) const {
        const uint32_t h = (id * 2654435761u) >> (32 - BITS);
        for (int probe = 0; probe < 16; ++probe) {
            const int e = (int)((h + probe) & (N - 1));
            const uint32_t prev = atomicCAS(key + e, EMPTY, id);
            if (prev == EMPTY || prev == id) {
                atomicAdd(area + e, a);
                atomicAdd(sx + e, lsx);
                atomicAdd(sy + e, lsy);
                atomicMin(xmin + e, lx0);
                atomicMax(xmax + e, lx1);
                atomicOr(rows + e, rmask);
                return true;
            }
        }
        return false;
    }
};

// A contribution to a node record. Apart from the exterior (node 0), a
// record written with atomics already holds its exact ymin: a border node's
// record starts at its first pixel's row (node ids pass), a spilled record
// at its root's row, and no pixel of a component lies above its first
// pixel. So six reductions instead of seven.
__device__ __forceinline__ void feat_add(int64_t *base, int64_t cap, int id, unsigned long long area,
                                         unsigned long long sx, unsigned long long sy, long long xmin, long long ymin,
                                         long long xmax, long long ymax) {
    red_add_u64(base + 0 * cap + id, area);
    red_min_s64(base + 1 * cap + id, xmin);
    if (id == 0) red_min_s64(base + 2 * cap + id, ymin);
    red_max_s64(base + 3 * cap + id, xmax);
    red_max_s64(base + 4 * cap + id, ymax);
    red_add_u64(base + 5 * cap + id, sx);
    red_add_u64(base + 6 * cap + id, sy);
}

// 16-byte label store that does not allocate in L1, which stays free for
// the run and root records the tile's loops read.
__device__ __forceinline__ void st_na_v4(int32_t *p, int a, int b, int c, int e) {
    asm volatile("st.global.L1::no_allocate.v4.s32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(a), "r"(b), "r"(c), "r"(e));
}

__device__ __forceinline__ void cp_async16_w(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all_w() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Run record fields (see Scratch::run_root).
__device__ __forceinline__ int rec_root(uint32_t v) { return (int)(v >> 16); }
__device__ __forceinline__ int rec_pix(uint32_t v) { return (int)((v >> 1) & 0x7FFFu); }

// Exclusive prefix sum over segments of W consecutive lanes (one tile row);
// *total receives the segment's sum.
template <int W>
__device__ __forceinline__ int seg_excl_sum(int v, int *total) {
    const int l = threadIdx.x & (W - 1);
    int x = v;
#pragma unroll
    for (int o = 1; o < W; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o, W);
        if (l >= o) x += y;
    }
    *total = __shfl_sync(FULL, x, W - 1, W);
    return x - v;
}

// The bit-plane words of one tile held by one thread (two words), loaded
// one tile ahead.
struct PlaneRegs {
    uint32_t c[2], nb[2];
    int seg[2], seg_first;
};

// One CTA per tile at a time. Thread 0 claims tiles three ahead and copies
// the headers and counts of the tile after next into shared memory; the bit
// planes of the next tile are loaded into registers while the CTA works on
// the current one.
template <int TH, int TW>
__global__ void __launch_bounds__(WriteCfg<TH, TW>::NT, WriteCfg<TH, TW>::CTAS) k_write(Batch B) {
    using C = WriteCfg<TH, TW>;
    constexpr int WPR = TW / 32, LOG_TW = TW == 1024 ? 10 : 9;
    constexpr int NT = C::NT, NWD = TH * WPR, MAXR = C::MAXR, MAXID = C::MAXID;
    constexpr int HN = 1 << C::HASH_BITS;
    static_assert(NWD == 2 * NT, "two words per thread");
    extern __shared__ __align__(16) unsigned char smem[];
    // feature records of the multi-run roots, structure of arrays (tile-local x, y)
    uint32_t *sArea = (uint32_t *)smem;
    uint32_t *sSx = sArea + MAXR;
    uint32_t *sSy = sSx + MAXR;
    uint32_t *sX0 = sSy + MAXR;
    uint32_t *sX1 = sX0 + MAXR;
    uint32_t *sRows = sX1 + MAXR;                      // bit r: a run on row r
    int32_t *sId = (int32_t *)(sRows + MAXR);          // node id per root ordinal
    uint32_t *sC = (uint32_t *)(sId + MAXID);          // [TH][WPR] colour bits
    uint32_t *sE = sC + NWD;                           // [TH][WPR] run starts
    uint32_t *sNB = sE + NWD;                          // [TH][WPR] first pixels of nodes
    uint32_t *hmem = sNB + NWD;                        // combining table
    uint16_t *sOrd = (uint16_t *)(hmem + 7 * HN);      // [NWD + 8] first run ordinal of each word
    uint16_t *sNBPre = sOrd + NWD + 8;                 // [NWD] node bits before the word in its row
    __shared__ int sT[3], sRowTot[TH], sRowSeg[TH], sCap;
    __shared__ TileHdr sHdr[3];
    __shared__ int4 sSt[3];
    const TileHash<C::HASH_BITS> H(hmem);

    const int tid = threadIdx.x, lane = tid & 31;
    const int l = tid % WPR;   // this thread's word within its rows (word tid and word tid + NT)
    pdl_wait();   // node ids, merged roots and counters are visible

    auto load_planes = [&](const TileHdr &h, PlaneRegs &p) {
        const int64_t rowwords = (int64_t)h.TX * WPR;
        const int64_t plane0 = (h.seg0 + (int64_t)h.y0 * h.TX + h.tx) * WPR;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int r = (tid + j * NT) / WPR;
            p.c[j] = p.nb[j] = 0u;
            p.seg[j] = 0;
            if (r < h.th) {
                p.c[j] = B.s.fgbits[plane0 + r * rowwords + l];
                p.nb[j] = B.s.nodebits[plane0 + r * rowwords + l];
                if (l == 0) p.seg[j] = B.s.seg_base[h.seg0 + (int64_t)(h.y0 + r) * h.TX + h.tx];
            }
        }
        p.seg_first = l == 0 ? B.s.seg_base[h.seg0] : 0;
    };

    int nc = 0;   // thread 0: the tile claimed for two iterations on
    if (tid == 0) {
        const int t0 = atomicAdd(&B.s.work[3], 1);
        const int t1 = atomicAdd(&B.s.work[3], 1);
        sT[0] = t0;
        sT[1] = t1;
        if (t0 < B.n_tiles) {
            sHdr[0] = B.s.thdr[t0];
            sSt[0] = B.s.tstat[t0];
        }
        if (t1 < B.n_tiles) {
            sHdr[1] = B.s.thdr[t1];
            sSt[1] = B.s.tstat[t1];
        }
        nc = atomicAdd(&B.s.work[3], 1);
        sCap = 0;
    }
    for (int e = tid; e < HN; e += NT) H.reset(e);
    __syncthreads();
    PlaneRegs pr;
    if (sT[0] < B.n_tiles) load_planes(sHdr[0], pr);

    for (int slot = 0;;) {
        const int s1 = slot == 2 ? 0 : slot + 1, s2 = s1 == 2 ? 0 : s1 + 1;
        const int t = sT[slot];
        if (t >= B.n_tiles) break;
        const int tn = sT[s1];
        // thread 0: the header and counts of the tile after next (claimed one
        // iteration ago) into the free slot, and the next claim; both are
        // waited for before the tile's last barrier
        int cur_claim = 0;
        if (tid == 0) {
            cur_claim = nc;
            if (nc < B.n_tiles) {
                for (int k = 0; k < (int)(sizeof(TileHdr) / 16); ++k)
                    cp_async16_w((char *)&sHdr[s2] + 16 * k, (const char *)(B.s.thdr + nc) + 16 * k);
                cp_async16_w(&sSt[s2], B.s.tstat + nc);
            }
            nc = atomicAdd(&B.s.work[3], 1);
        }
        const TileHdr &h = sHdr[slot];
        const int4 st = sSt[slot];
        const int img = h.img;
        const ImgDesc &d = B.desc[img];
        const int y0 = h.y0, x0 = h.x0, th = h.th, tw = h.tw;
        const int64_t cap = d.cap;
        const int n_img = B.n_img;
        const int n_multi = st.y & 0xFFFF, n_roots = n_multi + (int)((uint32_t)st.y >> 16);
        const uint32_t *rr = B.s.run_root + h.px;
        const uint32_t *ri = B.s.rootinfo + h.px;
        const uint32_t slot0 = (uint32_t)(n_img + h.b);
        bool over = false;

        // ---- bit planes of the tile: colour, run starts, node first-pixels
        int rex[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int word = tid + j * NT, r = word / WPR;
            const uint32_t c = pr.c[j];
            const int vcnt = min(max(tw - 32 * l, 0), 32);
            const uint32_t vr = r < th ? (vcnt >= 32 ? FULL : ((1u << vcnt) - 1u)) : 0u;
            const uint32_t left = __shfl_up_sync(FULL, c, 1);
            const uint32_t prev = (c << 1) | (l ? (left >> 31) : 0u);
            const uint32_t e = ((c ^ prev) | (l == 0 ? 1u : 0u)) & vr;
            sC[word] = c;
            sE[word] = e;
            sNB[word] = pr.nb[j];
            int ntot, rtot;
            sNBPre[word] = (uint16_t)seg_excl_sum<WPR>(__popc(pr.nb[j]), &ntot);
            rex[j] = seg_excl_sum<WPR>(__popc(e), &rtot);
            if (l == 0) {
                sRowTot[r] = rtot;
                sRowSeg[r] = r < th ? pr.seg[j] - pr.seg_first : 0;
            }
        }
        __syncthreads();
        // the planes of the next tile (its header landed one tile ago)
        if (tn < B.n_tiles) load_planes(sHdr[s1], pr);
        int n;   // runs of the tile
        {
            int wt;
            const int ex = warp_excl_sum(lane < TH ? sRowTot[lane] : 0, &wt);
            n = wt;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int r = (tid + j * NT) / WPR;
                sOrd[tid + j * NT] = (uint16_t)(__shfl_sync(FULL, ex, r) + rex[j]);
            }
            if (tid == 0) sOrd[NWD] = (uint16_t)n;
        }
        for (int k = tid; k < min(n_multi, MAXR); k += NT) {
            sArea[k] = 0u;
            sSx[k] = 0u;
            sSy[k] = 0u;
            sX0[k] = 0xFFFFu;
            sX1[k] = 0u;
            sRows[k] = 0u;
        }

        // node id of a local root (rootinfo: its first pixel, border flag and
        // border ordinal)
        auto root_id = [&](uint32_t info) -> int {
            const int idx = info & 0xFFFF;
            if (!((info >> 17) & 1u)) {
                const int r = idx >> LOG_TW, c = idx & (TW - 1), wi = r * WPR + (c >> 5);
                return 1 + sRowSeg[r] + (int)sNBPre[wi] + __popc(sNB[wi] & mask_lt(c & 31));
            }
            const uint32_t root = (uint32_t)B.s.gp[slot0 + ((info >> 18) & 0xFFFu)];
            return root < (uint32_t)n_img ? 0 : B.s.canon[root];
        };
        auto id_of = [&](int k) -> int { return k < MAXID ? sId[k] : root_id(ri[k]); };
        // ordinal of the run covering column x of row r
        auto ord_at = [&](int r, int x) -> int {
            const int wi = r * WPR + (x >> 5);
            return (int)sOrd[wi] + __popc(sE[wi] & mask_le(x & 31)) - 1;
        };

        // ---- node ids of the roots; global records of spilled multi-run roots
        // records loaded two iterations ahead, a border root's union-find
        // entry one iteration ahead (from the record that has arrived)
        auto gp_of = [&](uint32_t info) -> uint32_t {
            return (info >> 17) & 1u ? (uint32_t)B.s.gp[slot0 + ((info >> 18) & 0xFFFu)] : 0u;
        };
        uint32_t info_a = tid < n_roots ? ri[tid] : 0u;
        uint32_t info_b = tid + NT < n_roots ? ri[tid + NT] : 0u;
        uint32_t gp_a = gp_of(info_a);
        for (int k = tid; k < n_roots; k += NT) {
            const uint32_t info = info_a, groot = gp_a;
            info_a = info_b;
            gp_a = k + NT < n_roots ? gp_of(info_a) : 0u;
            info_b = k + 2 * NT < n_roots ? ri[k + 2 * NT] : 0u;
            const int id = !((info >> 17) & 1u) ? root_id(info) : (groot < (uint32_t)n_img ? 0 : B.s.canon[groot]);
            if (k < MAXID) sId[k] = id;
            if (k < n_multi && k >= MAXR && !((info >> 17) & 1u) && id < cap) {
                d.feat[0 * cap + id] = 0;
                d.feat[1 * cap + id] = INT64_MAX;
                d.feat[2 * cap + id] = y0 + ((info & 0xFFFF) >> LOG_TW);
                d.feat[3 * cap + id] = -1;
                d.feat[4 * cap + id] = -1;
                d.feat[5 * cap + id] = 0;
                d.feat[6 * cap + id] = 0;
            }
        }
        __syncthreads();

        // ---- label rows (each warp its two rows, 4 pixels per lane per step)
        if (B.labels && d.fg != nullptr) {
#pragma unroll 1
            for (int j = 0; j < 2; ++j) {
                const int r = (tid + j * NT) / WPR;
                if (r >= th) break;
                int32_t *fgrow = d.fg + (int64_t)(y0 + r) * h.w + x0;
                int32_t *bgrow = d.bg + (int64_t)(y0 + r) * h.w + x0;
                constexpr int G = TW / (4 * WPR), GB = 4;   // groups per lane, groups per batch
#pragma unroll 1
                for (int g0 = 0; g0 < G; g0 += GB) {
                    int q0[GB];
                    uint32_t v0[GB];
#pragma unroll
                    for (int u = 0; u < GB; ++u) {
                        const int x = 4 * WPR * (g0 + u) + 4 * l;
                        q0[u] = x < tw ? ord_at(r, x) : -1;
                        v0[u] = q0[u] >= 0 ? rr[q0[u]] : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < GB; ++u) {
                        if (q0[u] < 0) continue;
                        const int x = 4 * WPR * (g0 + u) + 4 * l;
                        const int wi = r * WPR + (x >> 5), b = x & 31;
                        const uint32_t ew = sE[wi], cw = sC[wi];
                        // run starts inside the group (usually none: one lookup)
                        const uint32_t s3 = (ew >> (b + 1)) & 7u, c4 = (cw >> b) & 15u;
                        int id[4];
                        id[0] = id_of(rec_root(v0[u]));
                        if (s3 == 0u) {
                            id[1] = id[2] = id[3] = id[0];
                        } else {
                            const int q1 = q0[u] + (int)(s3 & 1u), q2 = q1 + (int)((s3 >> 1) & 1u),
                                      q3 = q2 + (int)(s3 >> 2);
                            id[1] = id_of(rec_root(rr[q1]));
                            id[2] = id_of(rec_root(rr[q2]));
                            id[3] = id_of(rec_root(rr[q3]));
                        }
                        int fv[4], bv[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const bool isfg = (c4 >> i) & 1u;
                            fv[i] = isfg ? id[i] : -1;
                            bv[i] = isfg ? -1 : id[i];
                        }
                        if (d.vec) {
                            st_na_v4(fgrow + x, fv[0], fv[1], fv[2], fv[3]);
                            st_na_v4(bgrow + x, bv[0], bv[1], bv[2], bv[3]);
                        } else {
#pragma unroll
                            for (int i = 0; i < 4; ++i) {
                                if (x + i < tw) {
                                    fgrow[x + i] = fv[i];
                                    bgrow[x + i] = bv[i];
                                }
                            }
                        }
                    }
                }
            }
        }

        // ---- run features of the multi-run roots (one thread per run, 32
        // consecutive runs per warp). Along a row the runs alternate colours,
        // so the runs of one component crossing the row many times sit two
        // lanes apart: a segmented scan along such stride-2 chains of equal
        // (root, row) sums them, and only the chain's last lane updates the
        // shared record.
        // records loaded one iteration ahead (the last lane also the record
        // after its run's)
        uint32_t v_nx = tid < n ? rr[tid] : 0xFFFFFFFFu;
        uint32_t vl_nx = lane == 31 && tid + 1 < n ? rr[tid + 1] : 0xFFFFFFFFu;
        for (int i0 = 0; i0 < n; i0 += NT) {
            const int i = i0 + tid;
            const uint32_t v = v_nx, vl = vl_nx;
            if (i + NT < n) v_nx = rr[i + NT];
            if (lane == 31 && i + NT + 1 < n) vl_nx = rr[i + NT + 1];
            // the next run's start: the next lane's record
            uint32_t vn = __shfl_down_sync(FULL, v, 1);
            if (lane == 31) vn = vl;
            const int k = rec_root(v), pix = rec_pix(v), r = pix >> LOG_TW, s = pix & (TW - 1);
            const bool multi = i < n && k < n_multi;
            int en = tw;
            if (i + 1 < n) {
                const int pn = rec_pix(vn);
                if ((pn >> LOG_TW) == r) en = pn & (TW - 1);
            }
            uint32_t len = 0, sx = 0;
            uint32_t key = 0xFFFFFFFFu;   // (root, row) of a multi-run root on chip
            if (multi) {
                len = (uint32_t)(en - s);
                sx = (uint32_t)((s + en - 1) * (en - s) / 2);
                if (k < MAXR) {
                    key = ((uint32_t)k << 5) | (uint32_t)r;
                } else {
                    const int id = id_of(k);
                    if (id < cap)
                        feat_add(d.feat, cap, id, len, sx + (unsigned long long)x0 * len,
                                 (unsigned long long)(y0 + r) * len, x0 + s, y0 + r, x0 + en - 1, y0 + r);
                }
            }
            const uint32_t kprev = __shfl_up_sync(FULL, key, 2);
            const bool cont = lane >= 2 && key != 0xFFFFFFFFu && kprev == key;
            int xs0 = s;
            bool cont_next = false;
            if (__any_sync(FULL, cont)) {   // some run continues a chain
                int head = cont ? 0 : lane;   // lane of this chain's first run
#pragma unroll
                for (int dd = 2; dd < 32; dd <<= 1) {
                    const int hu = __shfl_up_sync(FULL, head, dd);
                    if (lane >= dd) head = max(head, hu);   // even offsets: the same parity
                }
#pragma unroll
                for (int dd = 2; dd < 32; dd <<= 1) {
                    const uint32_t tl = __shfl_up_sync(FULL, len, dd), ts = __shfl_up_sync(FULL, sx, dd);
                    if (lane - dd >= head) {
                        len += tl;
                        sx += ts;
                    }
                }
                xs0 = __shfl_sync(FULL, s, head);
                cont_next = __shfl_down_sync(FULL, (int)cont, 2) != 0;
            }
            if (key != 0xFFFFFFFFu && !(lane < 30 && cont_next)) {
                const int kk = (int)(key >> 5);
                // results unused: reductions, the lane does not wait
                atomicAdd(&sArea[kk], len);
                atomicAdd(&sSx[kk], sx);
                atomicAdd(&sSy[kk], (uint32_t)r * len);
                atomicMin(&sX0[kk], (uint32_t)xs0);
                atomicMax(&sX1[kk], (uint32_t)(en - 1));
                atomicOr(&sRows[kk], 1u << r);
            }
        }

        __syncthreads();

        // ---- per local root: the tree and the features. A node's first
        // pixel is the first pixel of the local root of its component in
        // the tile that holds it (the node bit there); that root sets the
        // node's parent = the node of the pixel directly above (the initial
        // adjacency of Algorithm 2, kept for the root by Algorithm 3), from
        // the row above or, on the tile's top row, the tile above (or the
        // exterior on the image's top row). Features: the records of
        // multi-run roots; the run itself for a single-run root.
        // (root records two iterations ahead; the record of the run above a
        // node's first pixel one iteration ahead)
        auto above_rec = [&](uint32_t info) -> uint32_t {
            const int idx = info & 0xFFFF, r = idx >> LOG_TW, c = idx & (TW - 1);
            const bool first = (sNB[r * WPR + (c >> 5)] >> (c & 31)) & 1u;
            return first && r > 0 ? rr[ord_at(r - 1, c)] : 0u;
        };
        uint32_t fin_a = tid < n_roots ? ri[tid] : 0u;
        uint32_t fin_b = tid + NT < n_roots ? ri[tid + NT] : 0u;
        uint32_t up_a = tid < n_roots ? above_rec(fin_a) : 0u;
        for (int k = tid; k < n_roots; k += NT) {
            const uint32_t info = fin_a, up = up_a;
            fin_a = fin_b;
            if (k + NT < n_roots) up_a = above_rec(fin_a);
            if (k + 2 * NT < n_roots) fin_b = ri[k + 2 * NT];
            const int idx = info & 0xFFFF, r = idx >> LOG_TW, c = idx & (TW - 1);
            const bool isb = (info >> 17) & 1u;
            const int id = id_of(k);
            if ((sNB[r * WPR + (c >> 5)] >> (c & 31)) & 1u) {
                int p = 0;
                if (r > 0) {
                    p = id_of(rec_root(up));
                } else if (y0 > 0) {
                    // the bottom edge cell of the tile above, same column
                    const uint32_t s2b = (uint32_t)(n_img + h.b_above) + B.s.edges[h.b_above + tw + c];
                    const uint32_t root = (uint32_t)B.s.gp[s2b];
                    p = root < (uint32_t)n_img ? 0 : B.s.canon[root];
                }
                if (id < cap) {
                    d.parent[id] = p;
                    if (id < d.ncap) B.s.node_fg[d.node0 + id] = (uint8_t)((info >> 16) & 1u);
                } else {
                    over = true;
                }
            }
            if (k < n_multi && k >= MAXR) continue;   // accumulated in global memory
            if (id >= cap) continue;
            uint32_t la, lsx, lsy, lx0, lx1, rmask;
            if (k < n_multi) {
                la = sArea[k];
                lsx = sSx[k];
                lsy = sSy[k];
                lx0 = sX0[k];
                lx1 = sX1[k];
                rmask = sRows[k];
            } else {
                // the run starting at (r, c) ends where the next run of the
                // row starts: the next run-start bit of the row (none beyond
                // the tile's width), else the row's end
                int wc = c >> 5;
                uint32_t m = sE[r * WPR + wc] & ~mask_le(c & 31);
                while (m == 0u && ++wc < WPR) m = sE[r * WPR + wc];
                const int ce = m ? 32 * wc + __ffs(m) - 1 : tw;
                la = (uint32_t)(ce - c);
                lsx = (uint32_t)((c + ce - 1) * (ce - c) / 2);
                lsy = (uint32_t)r * la;
                lx0 = (uint32_t)c;
                lx1 = (uint32_t)(ce - 1);
                rmask = 1u << r;
            }
            if (isb && H.push((uint32_t)id, la, lsx, lsy, lx0, lx1, rmask)) continue;
            const long long area = la;
            const long long sxg = (long long)lsx + area * x0, syg = (long long)lsy + area * y0;
            const int xmin = x0 + (int)lx0, xmax = x0 + (int)lx1;
            const int ymin = y0 + __ffs(rmask) - 1, ymax = y0 + 31 - __clz(rmask);
            if (!isb) {
                d.feat[0 * cap + id] = area;
                d.feat[1 * cap + id] = xmin;
                d.feat[2 * cap + id] = ymin;
                d.feat[3 * cap + id] = xmax;
                d.feat[4 * cap + id] = ymax;
                d.feat[5 * cap + id] = sxg;
                d.feat[6 * cap + id] = syg;
            } else {
                feat_add(d.feat, cap, id, (unsigned long long)area, (unsigned long long)sxg, (unsigned long long)syg,
                         xmin, ymin, xmax, ymax);
            }
        }
        if (over) atomicOr(&sCap, 1);
        if (tid == 0) {
            cp_async_wait_all_w();   // the header and counts of the tile after next
            sT[s2] = cur_claim;
        }
        __syncthreads();
        // the combining table: flush into the node records, then clear
        for (int e2 = tid; e2 < HN; e2 += NT) {
            const uint32_t id = H.key[e2];
            if (id != H.EMPTY) {
                const unsigned long long a = H.area[e2];
                const uint32_t rm = H.rows[e2];
                feat_add(d.feat, cap, (int)id, a, H.sx[e2] + a * (unsigned long long)x0,
                         H.sy[e2] + a * (unsigned long long)y0, x0 + (int)H.xmin[e2], y0 + __ffs(rm) - 1,
                         x0 + (int)H.xmax[e2], y0 + 31 - __clz(rm));
                H.reset(e2);
            }
        }
        if (tid == 0) {
            if (sCap) set_status(B, d, ST_CAPACITY);
            sCap = 0;
        }
        slot = s1;
    }
    pdl_trigger();   // no tile left: the next kernel may be scheduled
}

template <int TH, int TW>
static void launch_write_shape(const Batch &B, const LaunchCfg &c, cudaStream_t st) {
    using C = WriteCfg<TH, TW>;
    launch_dep(k_write<TH, TW>, min(B.n_tiles, C::CTAS * c.sms), C::NT, write_smem<TH, TW>(), st, B);
}

void launch_write(const Batch &B, const LaunchCfg &c, cudaStream_t st) {
    if (B.tw == 1024) {
        if (B.th == 32) launch_write_shape<32, 1024>(B, c, st);
        else launch_write_shape<16, 1024>(B, c, st);
    } else {
        if (B.th == 32) launch_write_shape<32, 512>(B, c, st);
        else launch_write_shape<16, 512>(B, c, st);
    }
}

template <int TH, int TW>
static cudaError_t configure_write_shape() {
    cudaError_t e = cudaFuncSetAttribute(k_write<TH, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)write_smem<TH, TW>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_write<TH, TW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

cudaError_t configure_write() {
    cudaError_t e = configure_write_shape<32, 1024>();
    if (e == cudaSuccess) e = configure_write_shape<16, 1024>();
    if (e == cudaSuccess) e = configure_write_shape<32, 512>();
    if (e == cudaSuccess) e = configure_write_shape<16, 512>();
    return e;
}

}  // namespace ccl
