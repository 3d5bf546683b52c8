// Phase 1 of the analysis: per-tile run extraction and run unification.
//
// The paper's steps 1a and 1b (Algorithms 1 and 2) scan one row at a time and
// grow one equivalence table for the whole image. Here every tile of 32 rows
// x 1024 columns is handled by one CTA, all rows at once:
//   - the tile is read with 16-byte loads and packed into a 1-bit-per-pixel
//     plane, one 32-bit word per lane (1024 columns = one warp);
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
// bits 18-29 border ordinal of the root within the tile.
constexpr int RI_FG = 16, RI_BORDER = 17, RI_KB = 18;

__global__ void k_prologue(Batch B) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        *B.s.status = 0;
        for (int k = 0; k < 8; ++k) B.s.work[k] = 0;
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

// Union every run of row r with the runs of row r - 1 it touches, for the
// contacts whose column lies in word l (32 pixels) and in bits [lo, hi) of
// that word. Masks mark, once per pair of touching runs, the column where
// the pair is tested:
//   va / vb  vertical overlaps of the 8- / 4-adjacent colour, at the first
//            column of the overlap (where one of the two runs starts);
//   d1 / d2  diagonal-only contacts of the 8-adjacent colour, up-right and
//            up-left (Algorithm 2 widens the 8-adjacent run's window by one
//            pixel on each side).
template <int CONN>
__device__ __forceinline__ void unify_rows(uint32_t *par, const uint32_t (*sC)[WPR],
                                           const uint32_t (*sE)[WPR], const uint16_t (*sRS)[WPR], int r,
                                           int l, int tw, uint32_t range, bool *ok) {
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
    const uint32_t d1 = ac & ~au & au_next & ~ac_next;   // (r,x)-(r-1,x+1)
    const uint32_t d2 = ac & ~au & au_prev & ~ac_prev;   // (r,x)-(r-1,x-1)
    // (a pixel can have both diagonal contacts: d2 gets its own pass)
    uint32_t m = (va | vb | d1) & range;
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int x = 32 * l + b;
        const int xu = ((d1 >> b) & 1u) ? x + 1 : x;
        local_union(par, r * TW + run_start_col(sE, sRS, r, x), (r - 1) * TW + run_start_col(sE, sRS, r - 1, xu), ok);
    }
    m = d2 & range;
    while (m) {
        const int x = 32 * l + __ffs(m) - 1;
        m &= m - 1;
        local_union(par, r * TW + run_start_col(sE, sRS, r, x), (r - 1) * TW + run_start_col(sE, sRS, r - 1, x - 1), ok);
    }
}

// Point every run of row r at its current root.
__device__ __forceinline__ void compress_row(uint32_t *par, const uint32_t (*sE)[WPR], int r, int lane,
                                             bool *ok) {
    uint32_t m = sE[r][lane];
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int idx = r * TW + 32 * lane + b;
        par[swz(idx)] = (uint32_t)local_find(par, idx, ok);
    }
}

template <int CONN, int TH>
__global__ void __launch_bounds__(TH * 16, TH == 32 ? 1 : 2) k_label(Batch B) {
    constexpr int LABEL_THREADS = TH * 16;   // two rows per warp
    constexpr int LABEL_WARPS = TH / 2;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *par = (uint32_t *)smem;                                    // 4 B per tile pixel
    uint32_t(*sC)[WPR] = (uint32_t(*)[WPR])(smem + TH * TW * 4);         // colour bits
    uint32_t(*sE)[WPR] = sC + TH;                                        // run starts
    uint32_t(*sR)[WPR] = sE + TH;                                        // local roots
    uint32_t(*sB)[WPR] = sR + TH;                                        // border roots
    uint16_t(*sRS)[WPR] = (uint16_t(*)[WPR])(sB + TH);                   // run covering bit 0
    uint16_t(*sRunPre)[WPR] = sRS + TH;                                  // prefix within row
    uint16_t(*sRootPre)[WPR] = sRunPre + TH;
    uint16_t(*sBPre)[WPR] = sRootPre + TH;
    __shared__ int sRowTot[3][TH];
    __shared__ int sTot[3];
    __shared__ int sTile, sImg, sFg, sOk;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(&B.s.work[0], 1);
            sTile = t;
            sImg = t < B.n_tiles ? image_of_tile(B, t) : -1;
            sFg = 0;
            sOk = 1;
        }
        __syncthreads();
        const int t = sTile;
        if (t >= B.n_tiles) break;
        const ImgDesc &d = B.desc[sImg];
        const TileGeo g = tile_geo(d, t - d.tile0, TH);
        const int tx = g.tx, y0 = g.y0, x0 = g.x0, th = g.th, tw = g.tw;
        const int64_t rowwords = (int64_t)d.TX * WPR;
        const int64_t plane0 = (d.seg0 + (int64_t)y0 * d.TX + tx) * WPR;  // word (y0, tile col)
        const int vcnt = min(max(tw - 32 * lane, 0), 32);
        const uint32_t vm = vcnt >= 32 ? FULL : ((1u << vcnt) - 1u);
        bool ok = true;

        // ---- read the tile, pack bits, find run starts
        for (int r = warp; r < TH; r += LABEL_WARPS) {
            uint32_t word = 0;
            if (r < th && vcnt > 0) {
                const uint8_t *p = d.img + (int64_t)(y0 + r) * d.pitch + x0 + 32 * lane;
                uint32_t m = nz16(ld_stream16(p));
                if (vcnt > 16) m |= nz16(ld_stream16(p + 16)) << 16;
                word = m & vm;
            }
            const uint32_t vr = r < th ? vm : 0u;
            sC[r][lane] = word;
            if (r < th) B.s.fgbits[plane0 + r * rowwords + lane] = word;
            const uint32_t left = __shfl_up_sync(FULL, word, 1);
            const uint32_t prev = (word << 1) | (lane ? (left >> 31) : 0u);
            const uint32_t e = ((word ^ prev) | (lane == 0 ? 1u : 0u)) & vr;
            sE[r][lane] = e;
            const int last = e ? 32 * lane + 31 - __clz(e) : -1;
            const int incl = warp_incl_max(last);
            int excl = __shfl_up_sync(FULL, incl, 1);
            if (lane == 0) excl = 0;
            sRS[r][lane] = (unsigned short)((e & 1u) ? 32 * lane : max(excl, 0));
            int tot;
            const int pre = warp_excl_sum(__popc(e), &tot);
            sRunPre[r][lane] = (unsigned short)pre;
            if (lane == 0) sRowTot[0][r] = tot;
            uint32_t m = e;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int idx = r * TW + 32 * lane + b;
                par[swz(idx)] = (uint32_t)idx;
            }
        }
        __syncthreads();

        // ---- unify each row with the row above (Algorithm 2)
        // Warp w first unifies its own row pair (2w, 2w + 1) and points row
        // 2w + 1 at the new roots, like one step of the paper's row-by-row
        // scan. Then blocks of 4, 8, 16 and 32 rows are joined across their
        // middle row, one level at a time so that every tree stays a few
        // links deep; each level's contacts are spread over all threads
        // (a word's 32 columns split into 2, 4, 8 or 16 slices).
        if (2 * warp + 1 < th) {
            unify_rows<CONN>(par, sC, sE, sRS, 2 * warp + 1, lane, tw, FULL, &ok);
            __syncwarp();
            compress_row(par, sE, 2 * warp + 1, lane, &ok);
        }
#pragma unroll 1
        for (int bs = 4; bs <= TH; bs *= 2) {
            __syncthreads();
            const int parts = LABEL_THREADS / ((TH / bs) * WPR);   // slices per word
            const int t = threadIdx.x;
            const int j = t / (WPR * parts), l = (t / parts) % WPR, q = t % parts;
            const int r = bs * j + bs / 2;
            const int span = 32 / parts;
            const uint32_t range = (span == 32 ? FULL : (((1u << span) - 1u) << (q * span)));
            if (r < th && 32 * l < tw) unify_rows<CONN>(par, sC, sE, sRS, r, l, tw, range, &ok);
        }
        __syncthreads();

        // ---- closure: every run points at its root (Algorithm 3, in-tile)
        for (int r = warp; r < TH; r += LABEL_WARPS) {
            uint32_t roots = 0;
            uint32_t m = r < th ? sE[r][lane] : 0u;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int idx = r * TW + 32 * lane + b;
                const int root = local_find(par, idx, &ok);
                par[swz(idx)] = (uint32_t)root;
                if (root == idx) roots |= 1u << b;
            }
            sR[r][lane] = roots;
            sB[r][lane] = 0;
        }
        __syncthreads();

        // ---- roots of the edge cells are border roots
        const int nedge = 2 * tw + 2 * th;
        for (int i = threadIdx.x; i < nedge; i += LABEL_THREADS) {
            int r, c;
            if (i < tw) { r = 0; c = i; }
            else if (i < 2 * tw) { r = th - 1; c = i - tw; }
            else if (i < 2 * tw + th) { r = i - 2 * tw; c = 0; }
            else { r = i - 2 * tw - th; c = tw - 1; }
            const int root = par[swz(r * TW + run_start_col(sE, sRS, r, c))];
            atomicOr(&sB[root >> 10][(root >> 5) & 31], 1u << (root & 31));
        }
        __syncthreads();

        // ---- ordinals of roots and border roots in raster order
        for (int r = warp; r < TH; r += LABEL_WARPS) {
            int tr, tb;
            const int pr = warp_excl_sum(__popc(sR[r][lane]), &tr);
            const int pb = warp_excl_sum(__popc(sB[r][lane]), &tb);
            sRootPre[r][lane] = (unsigned short)pr;
            sBPre[r][lane] = (unsigned short)pb;
            if (lane == 0) {
                sRowTot[1][r] = tr;
                sRowTot[2][r] = tb;
            }
        }
        __syncthreads();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                int tot;
                const int ex = warp_excl_sum(lane < TH ? sRowTot[k][lane] : 0, &tot);
                if (lane < TH) sRowTot[k][lane] = ex;
                if (lane == 0) sTot[k] = tot;
            }
        }
        __syncthreads();

        // ---- outputs
        if (threadIdx.x == 0) B.s.tstat[t] = make_int4(sTot[0], sTot[1], sTot[2], 0);
        uint16_t *rr = B.s.run_root + g.px;
        uint32_t *ri = B.s.rootinfo + g.px;
        const uint32_t slot0 = (uint32_t)(B.n_img + g.b);
        int nfg = 0;
        for (int r = warp; r < th; r += LABEL_WARPS) {
            const uint32_t e = sE[r][lane], rm = sR[r][lane], bm = sB[r][lane], c = sC[r][lane];
            int q = sRowTot[0][r] + sRunPre[r][lane];
            uint32_t m = e;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int root = par[swz(r * TW + 32 * lane + b)];
                const int rrow = root >> 10, rl = (root >> 5) & 31;
                const int k = sRowTot[1][rrow] + sRootPre[rrow][rl] +
                              __popc(sR[rrow][rl] & mask_lt(root & 31));
                rr[q++] = (uint16_t)k;
            }
            int k = sRowTot[1][r] + sRootPre[r][lane];
            int kb = sRowTot[2][r] + sBPre[r][lane];
            m = rm;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int idx = r * TW + 32 * lane + b;
                const uint32_t isb = (bm >> b) & 1u, fg = (c >> b) & 1u;
                ri[k] = (uint32_t)idx | (fg << RI_FG) | (isb << RI_BORDER) | (isb ? ((uint32_t)kb << RI_KB) : 0u);
                if (isb) {
                    const uint32_t slot = slot0 + kb;
                    const int64_t key = (int64_t)(y0 + r) * d.w + x0 + 32 * lane + b;
                    B.s.gp[slot] = ((unsigned long long)(key + 1) << 32) | slot;
                    B.s.binfo[slot] = (uint32_t)k | (fg << 16);
                    ++kb;
                } else {
                    nfg += (int)fg;
                }
                ++k;
            }
            B.s.nodebits[plane0 + r * rowwords + lane] = rm & ~bm;
        }
        // edge cells -> border ordinal of their root
        // (cell i of the loop is also its offset: top, bottom, left, right)
        uint16_t *eg = B.s.edges + g.b;
        for (int i = threadIdx.x; i < nedge; i += LABEL_THREADS) {
            int r, c;
            if (i < tw) { r = 0; c = i; }
            else if (i < 2 * tw) { r = th - 1; c = i - tw; }
            else if (i < 2 * tw + th) { r = i - 2 * tw; c = 0; }
            else { r = i - 2 * tw - th; c = tw - 1; }
            const int off = i;
            const int root = par[swz(r * TW + run_start_col(sE, sRS, r, c))];
            const int rrow = root >> 10, rl = (root >> 5) & 31;
            eg[off] = (uint16_t)(sRowTot[2][rrow] + sBPre[rrow][rl] + __popc(sB[rrow][rl] & mask_lt(root & 31)));
        }
        nfg = warp_sum(nfg);
        if (lane == 0 && nfg) atomicAdd(&sFg, nfg);
        if (!ok) atomicAnd(&sOk, 0);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (sFg) atomicAdd(&B.s.img_cnt[4 * sImg + 1], sFg);
            if (!sOk) set_status(B, d, ST_ITER);
        }
        __syncthreads();
    }
}

template <int TH>
constexpr size_t label_smem() { return (size_t)TH * TW * 4 + 4 * TH * WPR * 4 + 4 * TH * WPR * 2; }

void launch_prologue(const Batch &B, cudaStream_t st) {
    k_prologue<<<(B.n_img + 127) / 128, 128, 0, st>>>(B);
}

void launch_label(const Batch &B, const LaunchCfg &c, cudaStream_t st) {
    if (B.th == 32) {
        const int grid = min(B.n_tiles, c.sms);
        if (B.conn == 0)
            k_label<0, 32><<<grid, 512, label_smem<32>(), st>>>(B);
        else
            k_label<1, 32><<<grid, 512, label_smem<32>(), st>>>(B);
    } else {
        const int grid = min(B.n_tiles, 2 * c.sms);
        if (B.conn == 0)
            k_label<0, 16><<<grid, 256, label_smem<16>(), st>>>(B);
        else
            k_label<1, 16><<<grid, 256, label_smem<16>(), st>>>(B);
    }
}

cudaError_t configure_label() {
    cudaError_t e = cudaFuncSetAttribute(k_label<0, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)label_smem<32>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_label<1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)label_smem<32>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_label<0, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)label_smem<16>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_label<1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)label_smem<16>());
    return e;
}

}  // namespace ccl
