// Phase 1 of the analysis: per-tile run extraction and run unification.
//
// The paper's steps 1a and 1b (Algorithms 1 and 2) scan one row at a time and
// grow one equivalence table for the whole image. Here every tile of 32 rows
// x 1024 columns (or 16 rows) is handled by one CTA, all rows at once:
//   - the tile's rows arrive by bulk copies (cp.async.bulk) into shared
//     memory, issued while the CTA works on the previous tile, and are packed
//     into a 1-bit-per-pixel plane, one 32-bit word per lane (1024 columns =
//     one warp, one warp per row);
//   - run starts come from an XOR of each word with itself shifted by one
//     pixel (Algorithm 1's edge detection x0 xor x1), 32 pixels at a time;
//   - the overlap tests of Algorithm 2 become word masks between a row and
//     the row above: an 8-adjacent colour links runs that overlap or touch
//     diagonally (the window widened by c8 = 1 on each side), the 4-adjacent
//     colour links runs that overlap;
//   - each link is a union by minimum run-start index in a shared-memory
//     parent table, so the root of a tile-local component is its
//     raster-first run, as the paper's root is its smallest (top-most) label.
// Results kept for the later phases: every run's root ordinal, one record
// per local root, the roots of the tile's edge cells (for the cross-tile
// merge) and the first-pixel bits of components that stay inside the tile.
#include "ccl_dev.cuh"

namespace ccl {

// rootinfo layout: bits 0-15 local pixel index of the root's first pixel
// (row * 1024 + column), bit 16 foreground, bit 17 touches a tile edge,
// bits 18-29 border ordinal of the root within the tile, bit 30 the
// component has a single run in the tile.
constexpr int RI_FG = 16, RI_BORDER = 17, RI_KB = 18, RI_SINGLE = 30;

__global__ void k_prologue(Batch B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *B.s.status = 0;
        for (int k = 0; k < 8; ++k) B.s.work[k] = 0;
    }
    if (i < B.n_tiles) {
        // per tile: its image, and where its rows start for the bulk copies
        const int img = image_of_tile(B, i);
        const ImgDesc &d = B.desc[img];
        const TileGeo g = tile_geo(d, i - d.tile0, B.th);
        const uint64_t src = (uint64_t)(d.img + (int64_t)g.y0 * d.pitch + g.x0);
        B.s.tstat[i] = make_int4(0, 0, 0, img);
        B.s.tsrc[i] = make_int4((int)(uint32_t)src, (int)(uint32_t)(src >> 32), d.pitch,
                                g.th | (((g.tw + 15) & ~15) << 8));
        TileHdr h;
        h.px = g.px;
        h.b = g.b;
        h.b_above = g.ty > 0 ? tile_geo(d, i - d.tile0 - d.TX, B.th).b : 0;
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

// Valid-pixel mask of word l of a tile row tw pixels wide (0 outside).
__device__ __forceinline__ uint32_t valid_mask(int tw, int l) {
    if (l < 0 || l >= WPR) return 0u;
    const int n = min(max(tw - 32 * l, 0), 32);
    return n >= 32 ? FULL : ((1u << n) - 1u);
}

// Run start (tile-local column) of the run holding column x of row r.
__device__ __forceinline__ int run_start_col(const uint32_t (*sE)[WPR], const uint16_t (*sRS)[WPR],
                                             int r, int x) {
    const int l = x >> 5;
    const uint32_t m = sE[r][l] & mask_le(x & 31);
    return m ? (l << 5) + 31 - __clz(m) : (int)sRS[r][l];
}

// Contacts between row r and row r - 1 whose column lies in word l (32
// pixels), as bit masks over the word's pixels of row r. Each pair of
// touching runs is marked once:
//   mv  vertical overlaps of either colour (8-adjacent: at the first column
//       of the overlap, where one of the two runs starts; 4-adjacent: the
//       same), the pixel above is the partner;
//   m1  diagonal-only contacts of the 8-adjacent colour, up-right: the
//       partner is the pixel above and to the right (Algorithm 2 widens the
//       8-adjacent run's window by one pixel on each side);
//   m2  the same, up-left (a pixel can have both diagonal contacts).
template <int CONN>
__device__ __forceinline__ void contact_masks(const uint32_t (*sC)[WPR], const uint32_t (*sE)[WPR], int r, int l,
                                              int tw, uint32_t *mv, uint32_t *m1, uint32_t *m2) {
    const uint32_t vm = valid_mask(tw, l), vml = valid_mask(tw, l - 1), vmr = valid_mask(tw, l + 1);
    const uint32_t cc = sC[r][l], cu = sC[r - 1][l];
    const uint32_t ec = sE[r][l], eu = sE[r - 1][l];
    const uint32_t ccl = l ? sC[r][l - 1] : 0u, cul = l ? sC[r - 1][l - 1] : 0u;
    const uint32_t ccr = l < WPR - 1 ? sC[r][l + 1] : 0u, cur = l < WPR - 1 ? sC[r - 1][l + 1] : 0u;
    const uint32_t ac = CONN ? (~cc & vm) : cc;   // the 8-adjacent colour
    const uint32_t au = CONN ? (~cu & vm) : cu;
    const uint32_t bc = CONN ? cc : (~cc & vm);   // the 4-adjacent colour
    const uint32_t bu = CONN ? cu : (~cu & vm);
    const uint32_t acl = l ? (CONN ? (~ccl & vml) : ccl) : 0u, aul = l ? (CONN ? (~cul & vml) : cul) : 0u;
    const uint32_t acr = CONN ? (~ccr & vmr) : ccr, aur = CONN ? (~cur & vmr) : cur;
    const uint32_t ac_prev = (ac << 1) | (acl >> 31);   // bit x: pixel x-1
    const uint32_t ac_next = (ac >> 1) | (acr << 31);   // bit x: pixel x+1
    const uint32_t au_prev = (au << 1) | (aul >> 31);
    const uint32_t au_next = (au >> 1) | (aur << 31);
    const uint32_t va = ac & au & ((ec & ac) | (eu & au));
    const uint32_t vb = bc & bu & ((ec & bc) | (eu & bu));
    *mv = va | vb;
    *m1 = ac & ~au & au_next & ~ac_next;   // (r,x)-(r-1,x+1)
    *m2 = ac & ~au & au_prev & ~ac_prev;   // (r,x)-(r-1,x-1)
}

// Union the runs of each contact in word l of boundary r (row r with row
// r - 1); the union by minimum of Algorithm 2. The run starts of the lane's
// own word in both rows are kept in registers; only a diagonal partner in a
// neighbouring word is looked up in shared memory.
__device__ __forceinline__ void unite_contacts(uint32_t *par, const uint32_t (*sE)[WPR], const uint16_t (*sRS)[WPR],
                                               int r, int l, uint32_t mv, uint32_t m1, uint32_t m2, bool *ok) {
    const uint32_t ec = sE[r][l], eu = sE[r - 1][l];
    const int rowc = r * TW, rowu = (r - 1) * TW;
    const int cover_c = rowc + sRS[r][l], cover_u = rowu + sRS[r - 1][l];   // runs covering bit 0
    const int word_c = rowc + 32 * l + 31, word_u = rowu + 32 * l + 31;
    // run start (tile-local index) of the run holding bit b of word l
    auto start_c = [&](int b) {
        const uint32_t m = ec & mask_le(b);
        return m ? word_c - __clz(m) : cover_c;
    };
    auto start_u = [&](int b) {
        const uint32_t m = eu & mask_le(b);
        return m ? word_u - __clz(m) : cover_u;
    };
    uint32_t m = mv | m1;   // disjoint sets of pixels
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int bu = b + (int)((m1 >> b) & 1u);   // partner bit in the row above
        const int u = bu < 32 ? start_u(bu) : rowu + run_start_col(sE, sRS, r - 1, 32 * l + 32);
        local_union(par, start_c(b), u, ok);
    }
    m = m2;   // partner up-left
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int u = b > 0 ? start_u(b - 1) : rowu + run_start_col(sE, sRS, r - 1, 32 * l - 1);
        local_union(par, start_c(b), u, ok);
    }
}

// After the root ordinals are known, par[root] holds them: ordinal (bits
// 0-14), border ordinal (bits 15-26) and this tag (a run index never has it).
constexpr uint32_t PAR_TAG = 0x80000000u;

// One CTA per tile at a time, one warp per tile row. The image rows of the
// next tile are fetched by bulk copies into a staging buffer while the CTA
// works on the current one: the last warp claims tiles from the work counter
// one tile ahead, loads the claimed tile's copy record during the tile
// before, and issues the copies (one row per lane) as soon as the staging
// buffer has been read.
//
// Root ordinals: the roots of components with more than one run come first
// (in raster order of their first pixel), then the single-run roots; the
// feature pass keeps on-chip records for the former only.
template <int CONN, int TH>
__global__ void __launch_bounds__(TH * 32, TH == 32 ? 1 : 2) k_label(Batch B) {
    constexpr int LABEL_THREADS = TH * 32;   // one row per warp
    constexpr int LABEL_WARPS = TH;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *par = (uint32_t *)smem;                                    // 4 B per tile pixel
    uint32_t(*sC)[WPR] = (uint32_t(*)[WPR])(smem + TH * TW * 4);         // colour bits
    uint32_t(*sE)[WPR] = sC + TH;                                        // run starts
    uint32_t(*sR)[WPR] = sE + TH;                                        // local roots
    uint32_t(*sB)[WPR] = sR + TH;                                        // border roots
    uint32_t(*sMul)[WPR] = sB + TH;                                      // roots of several runs
    uint32_t(*sMV)[WPR] = sMul + TH;                                     // contact masks per boundary
    uint32_t(*sM1)[WPR] = sMV + TH;
    uint32_t(*sM2)[WPR] = sM1 + TH;
    uint16_t(*sRS)[WPR] = (uint16_t(*)[WPR])(sM2 + TH);                  // run covering bit 0
    uint16_t(*sRunPre)[WPR] = sRS + TH;                                  // prefix within row
    uint16_t(*sMPre)[WPR] = sRunPre + TH;                                // multi-run roots
    uint16_t(*sSPre)[WPR] = sMPre + TH;                                  // single-run roots
    uint16_t(*sBPre)[WPR] = sSPre + TH;                                  // border roots
    uint8_t *stage = (uint8_t *)(sBPre + TH);                            // TH image rows
    // per row: runs | run-root slots << 16, multi-run roots | single-run
    // roots << 16, border roots (each warp scans them for its row's prefix)
    __shared__ uint32_t sRowTot[3][TH];
    __shared__ bool sRounds[TH];
    __shared__ int sNext, sFg[2], sOk[2], sAbort;
    __shared__ __align__(8) uint64_t sBar;
    __shared__ TileHdr sHdr[2];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool issuer = warp == LABEL_WARPS - 1;   // the whole last warp stages tiles
    // issuer warp: copy the rows (lane r: row r) and the header (lane 0) of
    // tile tn, whose copy record is rec, into the staging buffer and header
    // slot `slot`
    auto stage_tile = [&](int tn, int slot, int4 rec) {
        const uint8_t *src = (const uint8_t *)(((uint64_t)(uint32_t)rec.y << 32) | (uint32_t)rec.x);
        const int rows = rec.w & 0xFF, bytes = rec.w >> 8;
        if (lane == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&sBar, (uint32_t)(rows * bytes + sizeof(TileHdr)));
            bulk_g2s(&sHdr[slot], B.s.thdr + tn, (uint32_t)sizeof(TileHdr), &sBar);
        }
        __syncwarp();
        if (lane < rows) {
            fence_proxy_async_smem();
            bulk_g2s(stage + lane * TW, src + (int64_t)lane * rec.z, (uint32_t)bytes, &sBar);
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(&sBar, 1);
        sAbort = 0;
        sFg[0] = sFg[1] = 0;
        sOk[0] = sOk[1] = 1;
    }
    __syncthreads();
    int claim = 0;        // issuer: the tile claimed for the iteration after next
    int4 rec_next{};      // issuer: its copy record, loaded during the tile before
    if (issuer) {
        int t0 = 0, t1 = 0;
        if (lane == 0) {
            t0 = atomicAdd(&B.s.work[0], 1);
            t1 = atomicAdd(&B.s.work[0], 1);
        }
        t0 = __shfl_sync(FULL, t0, 0);
        t1 = __shfl_sync(FULL, t1, 0);
        if (t0 < B.n_tiles) stage_tile(t0, 0, B.s.tsrc[t0]);
        if (t1 < B.n_tiles) rec_next = B.s.tsrc[t1];
        if (lane == 0) sNext = t0;
        claim = t1;
    }
    __syncthreads();
    uint32_t phase = 0;
    // Per-tile counters alternate between two slots, so that thread 0 can
    // read and reset the slot of one tile while the others start the next:
    // the loop needs no barrier at its top or end.
    for (int q = 0;; q ^= 1) {
        const int t = sNext;   // written before the previous tile's last barrier
        if (t >= B.n_tiles) break;
        const bool staged = mbar_wait(&sBar, phase);
        if (!staged) atomicOr(&sAbort, 1);
        const TileHdr &h = sHdr[phase];
        const int img = h.img, tx = h.tx, y0 = h.y0, x0 = h.x0;
        const int th = staged ? h.th : 0, tw = staged ? h.tw : 0;   // nothing is touched on a failed copy
        const ImgDesc &d = B.desc[img];
        const int64_t rowwords = (int64_t)h.TX * WPR;
        const int64_t plane0 = (h.seg0 + (int64_t)y0 * h.TX + tx) * WPR;  // word (y0, tile col)
        const int vcnt = min(max(tw - 32 * lane, 0), 32);
        const uint32_t vm = vcnt >= 32 ? FULL : ((1u << vcnt) - 1u);
        bool ok = true;

        // ---- the staged rows: pack bits, find run starts (warp = row)
        for (int r = warp; r < TH; r += LABEL_WARPS) {
            uint32_t word = 0;
            if (r < th && vcnt > 0) {
                const uint4 *p = (const uint4 *)(stage + r * TW + 32 * lane);
                uint32_t m = nz16(p[0]);
                if (vcnt > 16) m |= nz16(p[1]) << 16;
                word = m & vm;
            }
            const uint32_t vr = r < th ? vm : 0u;
            sC[r][lane] = word;
            sB[r][lane] = 0;
            if (r < th) B.s.fgbits[plane0 + r * rowwords + lane] = word;
            const uint32_t left = __shfl_up_sync(FULL, word, 1);
            const uint32_t prev = (word << 1) | (lane ? (left >> 31) : 0u);
            const uint32_t e = ((word ^ prev) | (lane == 0 ? 1u : 0u)) & vr;
            sE[r][lane] = e;
            // the run covering bit 0 starts at the last run start of the
            // words before (the highest earlier lane with a start)
            const uint32_t before = __ballot_sync(FULL, e != 0u) & mask_lt(lane);
            const int j = before ? 31 - __clz(before) : 0;
            const uint32_t ej = __shfl_sync(FULL, e, j);
            sRS[r][lane] = (unsigned short)((e & 1u) ? 32 * lane : (before ? 32 * j + 31 - __clz(ej) : 0));
            int tot;
            const int pre = warp_excl_sum(__popc(e), &tot);
            sRunPre[r][lane] = (unsigned short)pre;
            const bool rounds = rr_rounds(tw, tot);
            const int most = (int)__reduce_max_sync(FULL, (unsigned)__popc(e));
            const int slots = rounds ? 32 * most : tot;
            if (lane == 0) {
                sRowTot[0][r] = (uint32_t)tot | ((uint32_t)slots << 16);
                sRounds[r] = rounds;
            }
            uint32_t m = e;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int idx = r * TW + 32 * lane + b;
                par[swz(idx)] = (uint32_t)idx;
            }
        }
        __syncthreads();
        if (sAbort) {
            // a copy did not complete: wait once more, bounded, for the copy
            // in flight, report, and stop
            if (threadIdx.x == 0) {
                mbar_wait(&sBar, phase);
                atomicOr(B.s.status, ST_ITER);
            }
            break;
        }
        phase ^= 1u;
        // the staging buffer and the other header slot are free: fetch the
        // next tile
        if (issuer) {
            const int tn = __shfl_sync(FULL, claim, 0);
            if (tn < B.n_tiles) stage_tile(tn, (int)phase, rec_next);
            if (lane == 0) {
                sNext = tn;
                claim = atomicAdd(&B.s.work[0], 1);
            }
        }

        // ---- contacts of every row with the row above (Algorithm 2)
        // Warp r - 1 takes boundary r (rows r - 1 and r), one word per lane:
        // it computes the boundary's contact masks (kept for the closure
        // below) and unites the runs of each contact. All boundaries are
        // united at the same time: the union by minimum with atomicMin stays
        // correct under concurrent unions, and the paper's row-by-row order
        // only matters for the provisional labels, not for the classes.
        if (warp + 1 < th) {
            const int r = warp + 1;
            uint32_t mv = 0, m1 = 0, m2 = 0;
            if (32 * lane < tw) contact_masks<CONN>(sC, sE, r, lane, tw, &mv, &m1, &m2);
            sMV[r][lane] = mv;
            sM1[r][lane] = m1;
            sM2[r][lane] = m2;
            if (mv | m1 | m2) unite_contacts(par, sE, sRS, r, lane, mv, m1, m2, &ok);
        }
        __syncthreads();

        // ---- closure: every run points at its root (Algorithm 3, in-tile).
        // A root is its component's raster-first run, so nothing above
        // touches it: the component has more runs exactly when the root's
        // run touches the row below, i.e. holds the upper end of one of the
        // contacts of boundary r + 1.
        for (int r = warp; r < TH; r += LABEL_WARPS) {
            uint32_t roots = 0, mul = 0;
            const uint32_t e = r < th ? sE[r][lane] : 0u;
            uint32_t m = e;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int idx = r * TW + 32 * lane + b;
                const int root = local_find(par, idx, &ok);
                par[swz(idx)] = (uint32_t)root;
                if (root == idx) roots |= 1u << b;
            }
            if (roots && r + 1 < th) {
                // upper ends of the contacts of boundary r + 1, word l
                auto upper = [&](int l) -> uint32_t {
                    const uint32_t m1l = l ? sM1[r + 1][l - 1] : 0u, m2r = l < WPR - 1 ? sM2[r + 1][l + 1] : 0u;
                    return sMV[r + 1][l] | (sM1[r + 1][l] << 1) | (m1l >> 31) | (sM2[r + 1][l] >> 1) | (m2r << 31);
                };
                const uint32_t u = upper(lane);
                uint32_t mr = roots;
                while (mr) {
                    const int b = __ffs(mr) - 1;
                    mr &= mr - 1;
                    const uint32_t after = e & ~mask_le(b);   // run starts after b in this word
                    const uint32_t span = (after ? mask_lt(__ffs(after) - 1) : FULL) & ~mask_lt(b);
                    bool hit = (u & span) != 0u;
                    if (!hit && !after) {
                        // a run reaching past the word's end
                        for (int l2 = lane + 1; l2 < WPR; ++l2) {
                            const uint32_t e2 = sE[r][l2];
                            const uint32_t sp = e2 ? mask_lt(__ffs(e2) - 1) : FULL;
                            if (upper(l2) & sp) {
                                hit = true;
                                break;
                            }
                            if (e2) break;
                        }
                    }
                    if (hit) mul |= 1u << b;
                }
            }
            sR[r][lane] = roots;
            sMul[r][lane] = mul;
        }

        // ---- roots of the edge cells are border roots (on the top and
        // bottom rows one cell per run is enough: the one where it starts).
        // This runs alongside the closure: its finds read parents that the
        // closure only ever replaces by the same roots.
        const int nedge = 2 * tw + 2 * th;
        for (int i = threadIdx.x; i < nedge; i += LABEL_THREADS) {
            int r, c;
            if (i < tw) { r = 0; c = i; }
            else if (i < 2 * tw) { r = th - 1; c = i - tw; }
            else if (i < 2 * tw + th) { r = i - 2 * tw; c = 0; }
            else { r = i - 2 * tw - th; c = tw - 1; }
            if (i < 2 * tw && !((sE[r][c >> 5] >> (c & 31)) & 1u)) continue;
            const int root = local_find(par, r * TW + run_start_col(sE, sRS, r, c), &ok);
            atomicOr(&sB[root >> 10][(root >> 5) & 31], 1u << (root & 31));
        }
        __syncthreads();

        // the claim issued above has returned by now: fetch its copy record
        if (issuer) {
            const int tn = __shfl_sync(FULL, claim, 0);
            if (tn < B.n_tiles) rec_next = B.s.tsrc[tn];
        }

        // ---- ordinals of roots and border roots in raster order
        for (int r = warp; r < TH; r += LABEL_WARPS) {
            const uint32_t rm = sR[r][lane], mul = sMul[r][lane];
            int tm, ts, tb;
            const int pm = warp_excl_sum(__popc(rm & mul), &tm);
            const int ps = warp_excl_sum(__popc(rm & ~mul), &ts);
            const int pb = warp_excl_sum(__popc(sB[r][lane]), &tb);
            sMPre[r][lane] = (unsigned short)pm;
            sSPre[r][lane] = (unsigned short)ps;
            sBPre[r][lane] = (unsigned short)pb;
            if (lane == 0) {
                sRowTot[1][r] = (uint32_t)tm | ((uint32_t)ts << 16);
                sRowTot[2][r] = tb;
            }
        }
        __syncthreads();
        // every warp scans the row totals itself (its own row's prefix is all
        // it needs), which saves a barrier
        uint32_t rbase[3], rtot[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint32_t ex = warp_excl_sum_u32(lane < TH ? sRowTot[k][lane] : 0u, &rtot[k]);
            rbase[k] = __shfl_sync(FULL, ex, warp & 31);
        }

        // ---- per root: record, border slot, ordinal into par[root]
        if (threadIdx.x == 0) B.s.tstat[t] = make_int4((int)(rtot[0] & 0xFFFFu), (int)rtot[1], (int)rtot[2], img);
        uint16_t *rr = B.s.run_root + h.px;
        uint32_t *ri = B.s.rootinfo + h.px;
        const uint32_t slot0 = (uint32_t)(B.n_img + h.b);
        const int n_multi = (int)(rtot[1] & 0xFFFFu);
        int nfg = 0;
        for (int r = warp; r < th; r += LABEL_WARPS) {
            const uint32_t rm = sR[r][lane], bm = sB[r][lane], c = sC[r][lane], mul = sMul[r][lane];
            int km = (int)(rbase[1] & 0xFFFFu) + sMPre[r][lane];
            int ks = n_multi + (int)(rbase[1] >> 16) + sSPre[r][lane];
            int kb = (int)rbase[2] + sBPre[r][lane];
            uint32_t m = rm;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int idx = r * TW + 32 * lane + b;
                const uint32_t isb = (bm >> b) & 1u, fg = (c >> b) & 1u, single = ((mul >> b) & 1u) ^ 1u;
                const int k = single ? ks++ : km++;
                ri[k] = (uint32_t)idx | (fg << RI_FG) | (isb << RI_BORDER) | (isb ? ((uint32_t)kb << RI_KB) : 0u) |
                        (single << RI_SINGLE);
                uint32_t v = PAR_TAG | (uint32_t)k;
                if (isb) {
                    const uint32_t slot = slot0 + kb;
                    const int64_t key = (int64_t)(y0 + r) * h.w + x0 + 32 * lane + b;
                    B.s.gp[slot] = ((unsigned long long)(key + 1) << 32) | slot;
                    B.s.binfo[slot] = (uint32_t)k | (fg << 16);
                    v |= (uint32_t)kb << 15;
                    ++kb;
                } else {
                    nfg += (int)fg;
                }
                par[swz(idx)] = v;
            }
            B.s.nodebits[plane0 + r * rowwords + lane] = rm & ~bm;
        }
        __syncthreads();

        // ---- per run: root ordinal; per edge cell: border ordinal of its root
        for (int r = warp; r < th; r += LABEL_WARPS) {
            const bool rounds = sRounds[r];
            const int row_slot = (int)(rbase[0] >> 16), pre = sRunPre[r][lane];
            uint32_t m = sE[r][lane];
            int j = 0;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                uint32_t v = par[swz(r * TW + 32 * lane + b)];
                if (!(v & PAR_TAG)) v = par[swz((int)v)];
                rr[rr_slot(rounds, row_slot, pre, lane, j++)] = (uint16_t)(v & 0x7FFFu);
            }
        }
        // (cell i of the loop is also its offset: top, bottom, left, right)
        uint16_t *eg = B.s.edges + h.b;
        for (int i = threadIdx.x; i < nedge; i += LABEL_THREADS) {
            int r, c;
            if (i < tw) { r = 0; c = i; }
            else if (i < 2 * tw) { r = th - 1; c = i - tw; }
            else if (i < 2 * tw + th) { r = i - 2 * tw; c = 0; }
            else { r = i - 2 * tw - th; c = tw - 1; }
            uint32_t v = par[swz(r * TW + run_start_col(sE, sRS, r, c))];
            if (!(v & PAR_TAG)) v = par[swz((int)v)];
            eg[i] = (uint16_t)((v >> 15) & 0xFFFu);
        }
        nfg = warp_sum(nfg);
        if (lane == 0 && nfg) atomicAdd(&sFg[q], nfg);
        if (!ok) atomicAnd(&sOk[q], 0);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (sFg[q]) atomicAdd(&B.s.img_cnt[4 * img + 1], sFg[q]);
            if (!sOk[q]) set_status(B, d, ST_ITER);
            sFg[q] = 0;   // the slot is next used two tiles on
            sOk[q] = 1;
        }
    }
}

template <int TH>
constexpr size_t label_smem() { return (size_t)TH * TW * 4 + 8 * TH * WPR * 4 + 5 * TH * WPR * 2 + (size_t)TH * TW; }

void launch_prologue(const Batch &B, cudaStream_t st) {
    const int n = B.n_img > B.n_tiles ? B.n_img : B.n_tiles;
    k_prologue<<<(n + 255) / 256, 256, 0, st>>>(B);
}

void launch_label(const Batch &B, const LaunchCfg &c, cudaStream_t st) {
    if (B.th == 32) {
        const int grid = min(B.n_tiles, c.sms);
        if (B.conn == 0)
            k_label<0, 32><<<grid, 1024, label_smem<32>(), st>>>(B);
        else
            k_label<1, 32><<<grid, 1024, label_smem<32>(), st>>>(B);
    } else {
        const int grid = min(B.n_tiles, 2 * c.sms);
        if (B.conn == 0)
            k_label<0, 16><<<grid, 512, label_smem<16>(), st>>>(B);
        else
            k_label<1, 16><<<grid, 512, label_smem<16>(), st>>>(B);
    }
}

template <typename K>
static cudaError_t configure_smem(K kernel, size_t bytes) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

cudaError_t configure_label() {
    cudaError_t e = configure_smem(k_label<0, 32>, label_smem<32>());
    if (e == cudaSuccess) e = configure_smem(k_label<1, 32>, label_smem<32>());
    if (e == cudaSuccess) e = configure_smem(k_label<0, 16>, label_smem<16>());
    if (e == cudaSuccess) e = configure_smem(k_label<1, 16>, label_smem<16>());
    return e;
}

}  // namespace ccl
