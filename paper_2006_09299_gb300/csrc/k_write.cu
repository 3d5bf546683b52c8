// Phase 3: per tile, write the two label images, the features and the tree.
//
// This is the paper's relabelling (Algorithm 4: every run's pixels receive
// the final label of the run) fused with the feature merge and the
// adjacency-to-root step of Algorithm 3:
//   - each run's root ordinal (from phase 1) gives the run's node id;
//   - features (ComputeFeatures of Algorithm 2: S, Sx, Sy and the box) are
//     accumulated per local root in shared memory, run by run; components
//     that stay inside the tile are then written with plain stores, and
//     border components are merged into their node with atomics, first
//     combined per CTA in a small hash table;
//   - the tree parent of a node whose first pixel lies in this tile is the
//     node of the pixel directly above that first pixel (the initial
//     adjacency of Algorithm 2, kept for the root by Algorithm 3);
//   - the label rows are written 4 pixels per lane, so that each warp
//     stores 512 contiguous bytes per instruction.
#include "ccl_dev.cuh"

namespace ccl {


// Root ordinals of a tile put the roots of components with several runs
// first, then the single-run roots. Multi-run roots below MAXR accumulate
// their features in on-chip records (more spill to global atomics); a
// single-run root's features are those of its run, read back from the bit
// planes in the feature pass. Node ids of the first MAXID roots are kept on
// chip. Launch shape per tile height: several CTAs per SM (16 warps in all),
// so that while one waits on its tile's global reads the others stream label
// rows; 16-row tiles have half the pixels and half the records.
template <int TH> struct WriteCfg;
template <> struct WriteCfg<32> { static constexpr int MAXR = 2048, MAXID = 3584, THREADS = 256, CTAS = 2; };
template <> struct WriteCfg<16> { static constexpr int MAXR = 1024, MAXID = 1792, THREADS = 128, CTAS = 4; };

// Per record: S, Sx, Sy, xmin, xmax and the row mask, all updated with
// native 32-bit shared reductions (a packed 64-bit sum was slower).
constexpr int REC_BYTES = 6 * 4;

template <int TH>
constexpr size_t write_smem() {
    constexpr int MAXR = WriteCfg<TH>::MAXR, MAXID = WriteCfg<TH>::MAXID;
    return (size_t)MAXR * REC_BYTES + (size_t)MAXID * 4 + MAXID / 8 + (size_t)(WriteCfg<TH>::THREADS / 32) * TW * 4 +
           3 * TH * WPR * 4 + 2 * TH * WPR * 2;
}

// Features of consecutive runs of one root on one row (tile-local x).
struct RunAcc {
    int k = -1;
    uint32_t len = 0, sx = 0;
    int x0 = 0, x1 = 0;
    __device__ __forceinline__ void start(int kk, int xs, int xe) {
        k = kk;
        len = (uint32_t)(xe - xs);
        sx = (uint32_t)((xs + xe - 1) * (xe - xs) / 2);
        x0 = xs;
        x1 = xe - 1;
    }
    __device__ __forceinline__ void add(int xs, int xe) {
        len += (uint32_t)(xe - xs);
        sx += (uint32_t)((xs + xe - 1) * (xe - xs) / 2);
        x1 = xe - 1;
    }
};

// Segmented inclusive scan over lanes (lane order = x order) of run
// accumulators with equal roots; afterwards only the last lane of each group
// of consecutive lanes with the same root keeps it (the others get k = -1).
__device__ __forceinline__ void warp_combine(RunAcc &a, int lane) {
    const int kprev = __shfl_up_sync(FULL, a.k, 1);
    // nothing to combine unless two consecutive lanes hold the same root
    if (!__any_sync(FULL, lane > 0 && a.k >= 0 && kprev == a.k)) return;
    const bool head = lane == 0 || kprev != a.k;
    int seg = head ? lane : 0;               // lane of this group's first member
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) seg = max(seg, __shfl_up_sync(FULL, seg, d));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t len = __shfl_up_sync(FULL, a.len, d), sx = __shfl_up_sync(FULL, a.sx, d);
        const int x0 = __shfl_up_sync(FULL, a.x0, d);
        if (lane - d >= seg) {
            a.len += len;
            a.sx += sx;
            a.x0 = min(a.x0, x0);
        }
    }
    const int knext = __shfl_down_sync(FULL, a.k, 1);
    if (lane < 31 && knext == a.k) a.k = -1;   // not the group's last lane
}

// Per-tile combining table for the features of border roots, which the
// cross-tile merge may have joined to the same node: every entry of one tile
// belongs to the tile's image, so the key is the node id and the sums are
// tile-relative and fit 32 bits (area <= 2^15, sum of x - x0 < 2^24, sum of
// y - y0 < 2^20); rows is a mask of the tile rows the contributions cover.
// It lives in the run buffers once the label rows are written: 28 bytes per
// entry, 1024 entries for 32-row tiles, 512 for 16-row tiles.
template <int N> struct TileHash {
    static constexpr uint32_t EMPTY = 0xFFFFFFFFu;
    uint32_t *key, *area, *sx, *sy, *xmin, *xmax, *rows;
    __device__ __forceinline__ explicit TileHash(void *mem) {
        key = (uint32_t *)mem;
        area = key + N;
        sx = area + N;
        sy = sx + N;
        xmin = sy + N;
        xmax = xmin + N;
        rows = xmax + N;
    }
    __device__ __forceinline__ void init(int tid, int nthreads) const {
        const uint4 e = make_uint4(EMPTY, EMPTY, EMPTY, EMPTY), z = make_uint4(0u, 0u, 0u, 0u);
        for (int i = tid; i < N / 4; i += nthreads) {
            ((uint4 *)key)[i] = e;
            ((uint4 *)area)[i] = z;
            ((uint4 *)sx)[i] = z;
            ((uint4 *)sy)[i] = z;
            ((uint4 *)xmin)[i] = e;
            ((uint4 *)xmax)[i] = z;
            ((uint4 *)rows)[i] = z;
        }
    }
    // false when the probes found no free entry (the caller adds to the
    // global record directly)
    __device__ __forceinline__ bool push(uint32_t id, uint32_t a, uint32_t lsx, uint32_t lsy, uint32_t lx0,
                                         uint32_t lx1, uint32_t rmask) const {
        constexpr int BITS = N == 1024 ? 10 : 9;
        static_assert(N == 1024 || N == 512, "table sizes");
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
// pixel. So six atomics instead of seven.
__device__ __forceinline__ void feat_add(int64_t *base, int64_t cap, int id, unsigned long long area,
                                         unsigned long long sx, unsigned long long sy, long long xmin, long long ymin,
                                         long long xmax, long long ymax) {
    atomicAdd((unsigned long long *)(base + 0 * cap + id), area);
    atomicMin((long long *)(base + 1 * cap + id), xmin);
    if (id == 0) atomicMin((long long *)(base + 2 * cap + id), ymin);
    atomicMax((long long *)(base + 3 * cap + id), xmax);
    atomicMax((long long *)(base + 4 * cap + id), ymax);
    atomicAdd((unsigned long long *)(base + 5 * cap + id), sx);
    atomicAdd((unsigned long long *)(base + 6 * cap + id), sy);
}

__device__ __forceinline__ void st_cs_v4(int32_t *p, int a, int b, int c, int e) {
    asm volatile("st.global.cs.v4.s32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(a), "r"(b), "r"(c), "r"(e));
}

template <int TH>
__global__ void __launch_bounds__(WriteCfg<TH>::THREADS, WriteCfg<TH>::CTAS) k_write(Batch B) {
    constexpr int MAXR = WriteCfg<TH>::MAXR, MAXID = WriteCfg<TH>::MAXID;
    constexpr int NTHREADS = WriteCfg<TH>::THREADS;
    constexpr int NWARPS = NTHREADS / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    // feature records of the local roots, structure of arrays (tile-local x, y)
    uint32_t *sArea = (uint32_t *)smem;
    uint32_t *sSx = sArea + MAXR;
    uint32_t *sSy = sSx + MAXR;
    uint32_t *sX0 = sSy + MAXR;
    uint32_t *sX1 = sX0 + MAXR;
    uint32_t *sRows = sX1 + MAXR;                                 // bit r: a run on row r
    int32_t *sId = (int32_t *)(sRows + MAXR);                     // node id per local root
    uint32_t *sBrd = (uint32_t *)(sId + MAXID);                   // bit k: root k touches a tile edge
    int32_t *sRid = (int32_t *)(sBrd + MAXID / 32);               // per warp: node id per run of a row
    uint32_t(*sC)[WPR] = (uint32_t(*)[WPR])(sRid + NWARPS * TW);
    uint32_t(*sE)[WPR] = sC + TH;
    uint32_t(*sNB)[WPR] = sE + TH;
    uint16_t(*sRunPre)[WPR] = (uint16_t(*)[WPR])(sNB + TH);
    uint16_t(*sNBPre)[WPR] = sRunPre + TH;
    __shared__ int sRowN[TH], sRowSeg[TH];                 // runs, first node
    __shared__ int sRowBase[TH];                           // run ordinal of the row's first run
    __shared__ int sT[2], sOk[2], sCap[2], sAbort;
    __shared__ TileHdr sHdr[2];
    __shared__ int4 sSt[2];
    __shared__ __align__(8) uint64_t sHBar;

    // the combining table reuses the run buffers once the rows are written
    const TileHash<(TH == 32 ? 1024 : 512)> H(sRid);
    static_assert((TH == 32 ? 1024 : 512) * 7 <= NWARPS * TW, "table fits the run buffers");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // thread 0: bulk-copy the header and counts of tile tn into slot `slot`
    // (tiles are claimed one ahead, so the copy lands during the tile before)
    auto fetch = [&](int tn, int slot) {
        sT[slot] = tn;
        if (tn < B.n_tiles) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&sHBar, (uint32_t)(sizeof(TileHdr) + sizeof(int4)));
            bulk_g2s(&sHdr[slot], B.s.thdr + tn, (uint32_t)sizeof(TileHdr), &sHBar);
            bulk_g2s(&sSt[slot], B.s.tstat + tn, (uint32_t)sizeof(int4), &sHBar);
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(&sHBar, 1);
        sAbort = 0;
        sOk[0] = sOk[1] = 1;
        sCap[0] = sCap[1] = 0;
    }
    __syncthreads();
    int claim = 0;
    if (threadIdx.x == 0) {
        fetch(atomicAdd(&B.s.work[3], 1), 0);
        claim = atomicAdd(&B.s.work[3], 1);
    }
    __syncthreads();
    uint32_t phase = 0;
    // Per-tile flags alternate between two slots, so that thread 0 can read
    // and reset the slot of one tile while the others start the next: the
    // loop needs no barrier at its top or end.
    for (int q = 0;; q ^= 1) {
        const int t = sT[phase];   // written before the previous tile's barriers
        if (t >= B.n_tiles) break;
        if (!mbar_wait(&sHBar, phase)) atomicOr(&sAbort, 1);
        __syncthreads();
        if (sAbort) {
            // the header copy did not complete: wait once more (bounded) and stop
            if (threadIdx.x == 0) {
                mbar_wait(&sHBar, phase);
                atomicOr(B.s.status, ST_ITER);
            }
            break;
        }
        const TileHdr &h = sHdr[phase];
        const int4 st = sSt[phase];
        phase ^= 1u;
        if (threadIdx.x == 0) {
            fetch(claim, (int)phase);
            claim = atomicAdd(&B.s.work[3], 1);
        }
        const int img = h.img;
        const ImgDesc &d = B.desc[img];
        const int tx = h.tx, y0 = h.y0, x0 = h.x0, th = h.th, tw = h.tw;
        const int64_t rowwords = (int64_t)h.TX * WPR;
        const int64_t plane0 = (h.seg0 + (int64_t)y0 * h.TX + tx) * WPR;
        const int64_t cap = d.cap;
        const int n_img = B.n_img;
        const int n_multi = st.y & 0xFFFF, n_roots = n_multi + (int)((uint32_t)st.y >> 16);
        const uint16_t *rr = B.s.run_root + h.px;
        const uint32_t *ri = B.s.rootinfo + h.px;
        const uint32_t slot0 = (uint32_t)(n_img + h.b);
        const int vcnt = min(max(tw - 32 * lane, 0), 32);
        const uint32_t vm = vcnt >= 32 ? FULL : ((1u << vcnt) - 1u);
        bool ok = true, over = false;

        // ---- bit planes of the tile: colour, run starts, node first-pixels
        // (all of this warp's rows are loaded before any is used)
        constexpr int RPW = TH / NWARPS;   // rows per warp
        uint32_t cw[RPW], nbw[RPW];
        int segw[RPW];
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const int r = warp + i * NWARPS;
            cw[i] = nbw[i] = 0u;
            segw[i] = 0;
            if (r < th) {
                cw[i] = B.s.fgbits[plane0 + r * rowwords + lane];
                nbw[i] = B.s.nodebits[plane0 + r * rowwords + lane];
                if (lane == 0) segw[i] = B.s.seg_base[h.seg0 + (int64_t)(y0 + r) * h.TX + tx];
            }
        }
        const int seg_first = lane == 0 ? B.s.seg_base[h.seg0] : 0;
        // node ids of the tile's border roots (their slots are consecutive),
        // fetched while the planes are scanned; the run buffers hold them
        // until the rows reuse that memory
        int32_t *sBid = sRid;
        for (int kb = threadIdx.x; kb < st.z; kb += NTHREADS) {
            const uint32_t root = (uint32_t)B.s.gp[slot0 + kb];
            sBid[kb] = root < (uint32_t)n_img ? 0 : B.s.canon[root];
        }
#pragma unroll
        for (int i = 0; i < RPW; ++i) {
            const int r = warp + i * NWARPS;
            const uint32_t c = cw[i], nb = nbw[i];
            const uint32_t vr = r < th ? vm : 0u;
            const uint32_t left = __shfl_up_sync(FULL, c, 1);
            const uint32_t prev = (c << 1) | (lane ? (left >> 31) : 0u);
            const uint32_t e = ((c ^ prev) | (lane == 0 ? 1u : 0u)) & vr;
            sC[r][lane] = c;
            sE[r][lane] = e;
            sNB[r][lane] = nb;
            int tot;
            sRunPre[r][lane] = (uint16_t)warp_excl_sum(__popc(e), &tot);
            if (lane == 0) sRowN[r] = tot;
            int ntot;
            sNBPre[r][lane] = (uint16_t)warp_excl_sum(__popc(nb), &ntot);
            if (lane == 0) sRowSeg[r] = r < th ? segw[i] - seg_first : 0;
        }
        __syncthreads();
        {
            // every warp scans the run counts itself and keeps the prefixes
            // of its own rows (saves a barrier)
            int tot;
            const int es = warp_excl_sum(lane < TH ? sRowN[lane] : 0, &tot);
            if (lane < TH && lane % NWARPS == warp) sRowBase[lane] = es;
            __syncwarp();
        }

        // node id of a local root; the border roots' ids are in sBid until
        // the rows phase
        auto root_id_early = [&](uint32_t info) -> int {
            const int idx = info & 0xFFFF;
            if (!((info >> 17) & 1u)) {
                const int r = idx >> 10, c = idx & 1023, l = c >> 5;
                return 1 + sRowSeg[r] + sNBPre[r][l] + __popc(sNB[r][l] & mask_lt(c & 31));
            }
            return sBid[(info >> 18) & 0xFFFu];
        };
        auto root_id = [&](uint32_t info) -> int {
            const int idx = info & 0xFFFF;
            if (!((info >> 17) & 1u)) {
                const int r = idx >> 10, c = idx & 1023, l = c >> 5;
                return 1 + sRowSeg[r] + sNBPre[r][l] + __popc(sNB[r][l] & mask_lt(c & 31));
            }
            const uint32_t root = (uint32_t)B.s.gp[slot0 + ((info >> 18) & 0xFFFu)];
            return root < (uint32_t)n_img ? 0 : B.s.canon[root];
        };

        // ---- node ids, edge flags and feature records of the local roots
        uint32_t info_next = warp * 32 + lane < n_roots ? ri[warp * 32 + lane] : 0u;   // one iteration ahead
        for (int k0 = warp * 32; k0 < n_roots; k0 += NTHREADS) {
            const int k = k0 + lane;
            const bool valid = k < n_roots;
            const uint32_t info = info_next;
            if (k + NTHREADS < n_roots) info_next = ri[k + NTHREADS];
            const bool isb = (info >> 17) & 1u;
            const bool multi = k < n_multi;
            const bool spill = valid && multi && k >= MAXR && !isb;
            int id = 0;
            if (valid && (k < MAXID || spill)) id = root_id_early(info);
            if (k0 < MAXID) {
                const uint32_t bal = __ballot_sync(FULL, valid && isb);
                if (lane == 0) sBrd[k0 >> 5] = bal;
                if (valid) sId[k] = id;
            }
            if (valid && multi && k < MAXR) {
                sArea[k] = 0u;
                sSx[k] = 0u;
                sSy[k] = 0u;
                sX0[k] = 0xFFFFu;
                sX1[k] = 0u;
                sRows[k] = 0u;
            } else if (spill && id < cap) {
                d.feat[0 * cap + id] = 0;
                d.feat[1 * cap + id] = INT64_MAX;
                d.feat[2 * cap + id] = y0 + ((info & 0xFFFF) >> 10);
                d.feat[3 * cap + id] = -1;
                d.feat[4 * cap + id] = -1;
                d.feat[5 * cap + id] = 0;
                d.feat[6 * cap + id] = 0;
            }
        }
        __syncthreads();

        // ---- rows: run features, tree parents of the row below, label rows
        const bool labels = B.labels && d.fg != nullptr;
        constexpr int PF = 4;
        int pf[PF];
        int pf_row = -1;
        for (int r = warp; r < th; r += NWARPS) {
            const uint32_t e = sE[r][lane];
            const int row_slot = sRowBase[r], nr = sRowN[r];
            int32_t *rid = sRid + warp * TW;
            // root ordinals of the row's runs (rid: by run index within the
            // row); the first PF rounds were fetched into registers while the
            // warp worked on its previous row
#pragma unroll
            for (int j = 0; j < PF; ++j) {
                const int i = lane + 32 * j;
                if (i < nr) rid[swz(i)] = pf_row == r ? pf[j] : (int)rr[row_slot + i];
            }
            // the rest in groups of 8 loads in flight
            for (int i0 = lane + 32 * PF; i0 < nr; i0 += 8 * 32) {
                int v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = i0 + 32 * u < nr ? (int)rr[row_slot + i0 + 32 * u] : 0;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (i0 + 32 * u < nr) rid[swz(i0 + 32 * u)] = v[u];
            }
            {
                const int rn = r + NWARPS;   // this warp's next row
                if (rn < th) {
                    const int nb = sRowBase[rn], nn = sRowN[rn];
#pragma unroll
                    for (int j = 0; j < PF; ++j) {
                        const int i = lane + 32 * j;
                        pf[j] = i < nn ? (int)rr[nb + i] : 0;
                    }
                    pf_row = rn;
                }
            }
            __syncwarp();
            // each lane walks the runs starting in its word. Along a row the
            // runs alternate colours, so a component crossing the row many
            // times (the percolating one of a dense random image) owns every
            // other run: one register accumulator per run parity sums its
            // runs, and the shared record is updated only when the root changes.
            {
                const int first = e ? 32 * lane + __ffs(e) - 1 : TW;
                const int nxt = min(warp_suffix_min_excl(first, TW), tw);
                int q = sRunPre[r][lane];
                uint32_t m = e;
                RunAcc acc0, acc1;
                auto flush = [&](const RunAcc &a) {
                    // single-run roots (k >= n_multi) need no accumulation:
                    // the feature pass reads their run from the bit planes
                    if (a.k < 0 || a.k >= n_multi) return;
                    if (a.k < MAXR) {
                        // results unused: reductions, the lane does not wait
                        atomicAdd(&sArea[a.k], a.len);
                        atomicAdd(&sSx[a.k], a.sx);
                        atomicAdd(&sSy[a.k], (uint32_t)r * a.len);
                        atomicMin(&sX0[a.k], (uint32_t)a.x0);
                        atomicMax(&sX1[a.k], (uint32_t)a.x1);
                        atomicOr(&sRows[a.k], 1u << r);
                    } else {
                        const int id = root_id(ri[a.k]);
                        if (id < cap)
                            feat_add(d.feat, cap, id, a.len, a.sx + (unsigned long long)x0 * a.len,
                                     (unsigned long long)(y0 + r) * a.len, x0 + a.x0, y0 + r, x0 + a.x1, y0 + r);
                    }
                };
                // one run into the accumulator of its parity (the caller
                // alternates acc0 / acc1 statically)
                auto step = [&](RunAcc &acc) {
                    const int xs = 32 * lane + __ffs(m) - 1;
                    m &= m - 1;
                    const int xe = m ? 32 * lane + __ffs(m) - 1 : nxt;
                    const int k = rid[swz(q)];
                    rid[swz(q)] = k < MAXID ? sId[k] : root_id(ri[k]);
                    if (k == acc.k) {
                        acc.add(xs, xe);
                    } else {
                        flush(acc);
                        acc.start(k, xs, xe);
                    }
                    ++q;
                };
                if ((q & 1) && m) step(acc1);
                while (m) {
                    step(acc0);
                    if (!m) break;
                    step(acc1);
                }
                // the last accumulators of neighbouring lanes often hold the
                // same root (a component crossing the row many times): combine
                // equal roots of consecutive lanes, then the last lane of each
                // group flushes
                warp_combine(acc0, lane);
                warp_combine(acc1, lane);
                flush(acc0);
                flush(acc1);
            }
            __syncwarp();
            // nodes whose first pixel is on row r + 1: parent = node of the
            // pixel above (the initial adjacency of Algorithm 2)
            if (r + 1 < th) {
                const uint32_t nb = sNB[r + 1][lane];
                uint32_t m = nb;
                while (m) {
                    const int b = __ffs(m) - 1;
                    m &= m - 1;
                    const int id = 1 + sRowSeg[r + 1] + sNBPre[r + 1][lane] + __popc(nb & mask_lt(b));
                    const int p = rid[swz(sRunPre[r][lane] + __popc(e & mask_le(b)) - 1)];
                    if (id < cap) {
                        d.parent[id] = p;
                        if (id < d.ncap) B.s.node_fg[d.node0 + id] = (uint8_t)((sC[r + 1][lane] >> b) & 1u);
                    } else {
                        over = true;
                    }
                }
            }
            if (labels) {
                int32_t *fgrow = d.fg + (int64_t)(y0 + r) * h.w + x0;
                int32_t *bgrow = d.bg + (int64_t)(y0 + r) * h.w + x0;
#pragma unroll
                for (int k8 = 0; k8 < TW / 128; ++k8) {
                    const int x = 128 * k8 + 4 * lane;
                    if (x < tw) {
                        const int wl = x >> 5, b = x & 31;
                        const uint32_t ew = sE[r][wl], cw = sC[r][wl];
                        // run index of the group's first pixel, and run starts
                        // inside the group (usually none: one lookup)
                        const int q0 = sRunPre[r][wl] - 1 + __popc(ew & mask_le(b));
                        const uint32_t s3 = (ew >> (b + 1)) & 7u, c4 = (cw >> b) & 15u;
                        int id[4];
                        id[0] = rid[swz(q0)];
                        if (s3 == 0u) {
                            id[1] = id[2] = id[3] = id[0];
                        } else {
                            const int q1 = q0 + (int)(s3 & 1u), q2 = q1 + (int)((s3 >> 1) & 1u),
                                      q3 = q2 + (int)(s3 >> 2);
                            id[1] = rid[swz(q1)];
                            id[2] = rid[swz(q2)];
                            id[3] = rid[swz(q3)];
                        }
                        int fv[4], bv[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const bool isfg = (c4 >> j) & 1u;
                            fv[j] = isfg ? id[j] : -1;
                            bv[j] = isfg ? -1 : id[j];
                        }
                        if (d.vec) {
                            st_cs_v4(fgrow + x, fv[0], fv[1], fv[2], fv[3]);
                            st_cs_v4(bgrow + x, bv[0], bv[1], bv[2], bv[3]);
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                if (x + j < tw) {
                                    fgrow[x + j] = fv[j];
                                    bgrow[x + j] = bv[j];
                                }
                            }
                        }
                    }
                }
            }
            __syncwarp();
        }
        // nodes whose first pixel is on the tile's top row: the pixel above is
        // in the tile above (or outside the image: the exterior)
        if (warp == NWARPS - 1) {
            const uint32_t nb = sNB[0][lane];
            uint32_t m = nb;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1;
                const int c = 32 * lane + b;
                const int id = 1 + sRowSeg[0] + sNBPre[0][lane] + __popc(nb & mask_lt(b));
                int p = 0;
                if (y0 > 0) {
                    // the bottom edge cell of the tile above, same column
                    const uint32_t s2 = (uint32_t)(n_img + h.b_above) + B.s.edges[h.b_above + tw + c];
                    const uint32_t root = (uint32_t)B.s.gp[s2];
                    p = root < (uint32_t)n_img ? 0 : B.s.canon[root];
                }
                if (id < cap) {
                    d.parent[id] = p;
                    if (id < d.ncap) B.s.node_fg[d.node0 + id] = (uint8_t)((sC[0][lane] >> b) & 1u);
                } else {
                    over = true;
                }
            }
        }
        __syncthreads();

        // ---- per local root: features (records of multi-run roots; the
        // run itself for a single-run root)
        H.init(threadIdx.x, NTHREADS);
        __syncthreads();
        uint32_t fin_next = threadIdx.x < n_roots ? ri[threadIdx.x] : 0u;   // one iteration ahead
        for (int k = threadIdx.x; k < n_roots; k += NTHREADS) {
            const uint32_t info = fin_next;
            if (k + NTHREADS < n_roots) fin_next = ri[k + NTHREADS];
            if (k < n_multi && k >= MAXR) continue;   // accumulated in global memory
            const int idx = info & 0xFFFF, r = idx >> 10, c = idx & 1023;
            const bool isb = (info >> 17) & 1u;
            const int id = k < MAXID ? sId[k] : root_id(info);
            if (id >= cap) continue;
            // tile-relative features first
            uint32_t la, lsx, lsy, lx0, lx1, rmask;
            if (k < n_multi) {
                la = sArea[k];
                lsx = sSx[k];
                lsy = sSy[k];
                lx0 = sX0[k];
                lx1 = sX1[k];
                rmask = sRows[k];
            } else {
                // the run starting at (r, c) ends before the next run start
                int l = c >> 5;
                uint32_t m = sE[r][l] & ~mask_le(c & 31);
                while (!m && ++l < WPR) m = sE[r][l];
                const int ce = m ? min(32 * l + __ffs(m) - 1, tw) : tw;
                la = (uint32_t)(ce - c);
                lsx = (uint32_t)((c + ce - 1) * (ce - c) / 2);
                lsy = (uint32_t)r * la;
                lx0 = (uint32_t)c;
                lx1 = (uint32_t)(ce - 1);
                rmask = 1u << r;
            }
            if (isb && H.push((uint32_t)id, la, lsx, lsy, lx0, lx1, rmask)) continue;
            const long long area = la;
            const long long sx = (long long)lsx + area * x0, sy = (long long)lsy + area * y0;
            const int xmin = x0 + (int)lx0, xmax = x0 + (int)lx1;
            const int ymin = y0 + __ffs(rmask) - 1, ymax = y0 + 31 - __clz(rmask);
            if (!isb) {
                d.feat[0 * cap + id] = area;
                d.feat[1 * cap + id] = xmin;
                d.feat[2 * cap + id] = ymin;
                d.feat[3 * cap + id] = xmax;
                d.feat[4 * cap + id] = ymax;
                d.feat[5 * cap + id] = sx;
                d.feat[6 * cap + id] = sy;
            } else {
                feat_add(d.feat, cap, id, (unsigned long long)area, (unsigned long long)sx, (unsigned long long)sy,
                         xmin, ymin, xmax, ymax);
            }
        }
        if (!ok) atomicAnd(&sOk[q], 0);
        if (over) atomicOr(&sCap[q], 1);
        __syncthreads();
        for (int e = threadIdx.x; e < (TH == 32 ? 1024 : 512); e += NTHREADS) {
            const uint32_t id = H.key[e];
            if (id == H.EMPTY) continue;
            const unsigned long long a = H.area[e];
            const uint32_t rm = H.rows[e];
            feat_add(d.feat, cap, (int)id, a, H.sx[e] + a * (unsigned long long)x0, H.sy[e] + a * (unsigned long long)y0,
                     x0 + (int)H.xmin[e], y0 + __ffs(rm) - 1, x0 + (int)H.xmax[e], y0 + 31 - __clz(rm));
        }
        if (threadIdx.x == 0) {
            if (!sOk[q]) set_status(B, d, ST_ITER);
            if (sCap[q]) set_status(B, d, ST_CAPACITY);
            sOk[q] = 1;   // the slot is next used two tiles on
            sCap[q] = 0;
        }
    }
}

void launch_write(const Batch &B, const LaunchCfg &c, cudaStream_t st) {
    if (B.th == 32)
        k_write<32><<<min(B.n_tiles, WriteCfg<32>::CTAS * c.sms), WriteCfg<32>::THREADS, write_smem<32>(), st>>>(B);
    else
        k_write<16><<<min(B.n_tiles, WriteCfg<16>::CTAS * c.sms), WriteCfg<16>::THREADS, write_smem<16>(), st>>>(B);
}

cudaError_t configure_write() {
    cudaError_t e = cudaFuncSetAttribute(k_write<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)write_smem<32>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_write<32>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_write<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)write_smem<16>());
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_write<16>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

}  // namespace ccl
