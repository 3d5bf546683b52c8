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

constexpr uint32_t BOX_INIT = 0x3FFu;   // xmin = 1023, xmax = 0, ymax = 0

constexpr size_t WRITE_SMEM = (size_t)MAXR * 8 + (size_t)MAXR * 4 + (size_t)MAXR * 4 +
                              (size_t)NWARPS * TW * 4 + 3 * TH * WPR * 4 + 2 * TH * WPR * 2;

// Shared-memory box record of a local root: xmin | xmax << 10 | ymax << 20
// (tile-local), updated by a compare-and-swap loop.
__device__ __forceinline__ bool box_update(uint32_t *p, int xs, int xl, int r) {
    uint32_t old = *(volatile uint32_t *)p;
    for (int it = 0; it < (1 << 16); ++it) {
        const uint32_t nx0 = min(old & 1023u, (uint32_t)xs);
        const uint32_t nx1 = max((old >> 10) & 1023u, (uint32_t)xl);
        const uint32_t ny = max(old >> 20, (uint32_t)r);
        const uint32_t nw = nx0 | (nx1 << 10) | (ny << 20);
        if (nw == old) return true;
        const uint32_t prev = atomicCAS(p, old, nw);
        if (prev == old) return true;
        old = prev;
    }
    return false;
}

__device__ __forceinline__ void st_cs_v4(int32_t *p, int a, int b, int c, int e) {
    asm volatile("st.global.cs.v4.s32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(a), "r"(b), "r"(c), "r"(e) : "memory");
}

__global__ void __launch_bounds__(NTHREADS, 2) k_write(Batch B) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *sSum = (unsigned long long *)smem;        // packed S | Sx << 16 | Sy << 41
    uint32_t *sBox = (uint32_t *)(sSum + MAXR);                   // xmin | xmax << 10 | ymax << 20
    int32_t *sId = (int32_t *)(sBox + MAXR);                      // node id per local root
    int32_t *sRid = sId + MAXR;                                   // per warp: node id per run of a row
    uint32_t(*sC)[WPR] = (uint32_t(*)[WPR])(sRid + NWARPS * TW);
    uint32_t(*sE)[WPR] = sC + TH;
    uint32_t(*sNB)[WPR] = sE + TH;
    uint16_t(*sRunPre)[WPR] = (uint16_t(*)[WPR])(sNB + TH);
    uint16_t(*sNBPre)[WPR] = sRunPre + TH;
    __shared__ int sRowRun[TH], sRowSeg[TH];
    __shared__ int sTile, sImg, sOk, sCap;

    // the hash table reuses the run buffers once the rows are written
    const HashTab H = hash_carve(sRid);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        if (threadIdx.x == 0) {
            const int t = atomicAdd(&B.s.work[3], 1);
            sTile = t;
            sImg = t < B.n_tiles ? image_of_tile(B, t) : -1;
            sOk = 1;
            sCap = 0;
        }
        __syncthreads();
        const int t = sTile;
        if (t >= B.n_tiles) break;
        const ImgDesc &d = B.desc[sImg];
        const int lt = t - d.tile0;
        const TileGeo g = tile_geo(d, lt);
        const int tx = g.tx, y0 = g.y0, x0 = g.x0, th = g.th, tw = g.tw;
        const int64_t rowwords = (int64_t)d.TX * WPR;
        const int64_t plane0 = (d.seg0 + (int64_t)y0 * d.TX + tx) * WPR;
        const int64_t cap = d.cap;
        const int n_img = B.n_img;
        const int4 st = B.s.tstat[t];
        const int n_roots = st.y;
        const uint16_t *rr = B.s.run_root + g.px;
        const uint32_t *ri = B.s.rootinfo + g.px;
        const uint32_t slot0 = (uint32_t)(n_img + g.b);
        const int vcnt = min(max(tw - 32 * lane, 0), 32);
        const uint32_t vm = vcnt >= 32 ? FULL : ((1u << vcnt) - 1u);
        bool ok = true;

        // ---- bit planes of the tile: colour, run starts, node first-pixels
        for (int r = warp; r < TH; r += NWARPS) {
            uint32_t c = 0, nb = 0;
            if (r < th) {
                c = B.s.fgbits[plane0 + r * rowwords + lane];
                nb = B.s.nodebits[plane0 + r * rowwords + lane];
            }
            const uint32_t vr = r < th ? vm : 0u;
            const uint32_t left = __shfl_up_sync(FULL, c, 1);
            const uint32_t prev = (c << 1) | (lane ? (left >> 31) : 0u);
            const uint32_t e = ((c ^ prev) | (lane == 0 ? 1u : 0u)) & vr;
            sC[r][lane] = c;
            sE[r][lane] = e;
            sNB[r][lane] = nb;
            int tot;
            sRunPre[r][lane] = (uint16_t)warp_excl_sum(__popc(e), &tot);
            if (lane == 0) sRowRun[r] = tot;
            int ntot;
            sNBPre[r][lane] = (uint16_t)warp_excl_sum(__popc(nb), &ntot);
            if (lane == 0)
                sRowSeg[r] = r < th ? B.s.seg_base[d.seg0 + (int64_t)(y0 + r) * d.TX + tx] - B.s.seg_base[d.seg0] : 0;
        }
        __syncthreads();
        if (warp == 0) {
            int tot;
            sRowRun[lane] = warp_excl_sum(sRowRun[lane], &tot);
        }
        __syncthreads();

        // node id of a local root
        auto root_id = [&](uint32_t info) -> int {
            const int idx = info & 0xFFFF;
            if (!((info >> 17) & 1u)) {
                const int r = idx >> 10, c = idx & 1023, l = c >> 5;
                return 1 + sRowSeg[r] + sNBPre[r][l] + __popc(sNB[r][l] & mask_lt(c & 31));
            }
            const uint32_t root = (uint32_t)B.s.gp[slot0 + (info >> 18)];
            return root < (uint32_t)n_img ? 0 : B.s.canon[root];
        };

        // ---- node ids and feature records of the local roots
        for (int k = threadIdx.x; k < n_roots; k += NTHREADS) {
            const uint32_t info = ri[k];
            const int id = root_id(info);
            if (k < MAXR) {
                sId[k] = id;
                sSum[k] = 0ull;
                sBox[k] = BOX_INIT;
            } else if (!((info >> 17) & 1u) && id < cap) {
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

        // ---- rows: run features, then the label rows
        const bool labels = B.labels && d.fg != nullptr;
        for (int r = warp; r < th; r += NWARPS) {
            const uint32_t e = sE[r][lane];
            const int rowbase = sRowRun[r];
            int q = rowbase + sRunPre[r][lane];
            const int first = e ? 32 * lane + __ffs(e) - 1 : TW;
            const int nxt = min(warp_suffix_min_excl(first, TW), tw);
            int32_t *rid = sRid + warp * TW;
            uint32_t m = e;
            while (m) {
                const int xs = 32 * lane + __ffs(m) - 1;
                m &= m - 1;
                const int xe = m ? 32 * lane + __ffs(m) - 1 : nxt;
                const int k = rr[q];
                const int id = k < MAXR ? sId[k] : root_id(ri[k]);
                rid[q - rowbase] = id;
                ++q;
                const int len = xe - xs;
                const unsigned long long sxl = (unsigned long long)((xs + xe - 1) * len / 2);
                if (k < MAXR) {
                    atomicAdd(&sSum[k], (unsigned long long)len | (sxl << 16) |
                                            ((unsigned long long)(r * len) << 41));
                    ok &= box_update(&sBox[k], xs, xe - 1, r);
                } else if (id < cap) {
                    feat_atomic(d.feat, cap, id, len, sxl + (unsigned long long)x0 * len,
                                (unsigned long long)(y0 + r) * len, x0 + xs, y0 + r, x0 + xe - 1, y0 + r);
                }
            }
            __syncwarp();
            if (labels) {
                int32_t *fgrow = d.fg + (int64_t)(y0 + r) * d.w + x0;
                int32_t *bgrow = d.bg + (int64_t)(y0 + r) * d.w + x0;
#pragma unroll 2
                for (int k8 = 0; k8 < TW / 128; ++k8) {
                    const int x = 128 * k8 + 4 * lane;
                    if (x < tw) {
                        const int wl = x >> 5, b = x & 31;
                        const uint32_t ew = sE[r][wl], cw = sC[r][wl];
                        const int p = sRunPre[r][wl] - 1;
                        int fv[4], bv[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int bit = b + j;
                            const int id = rid[p + __popc(ew & mask_le(bit))];
                            const bool isfg = (cw >> bit) & 1u;
                            fv[j] = isfg ? id : -1;
                            bv[j] = isfg ? -1 : id;
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
        __syncthreads();

        // ---- per local root: features and tree parent
        hash_init(H);
        __syncthreads();
        bool over = false;
        for (int k = threadIdx.x; k < n_roots; k += NTHREADS) {
            const uint32_t info = ri[k];
            const int idx = info & 0xFFFF, r = idx >> 10, c = idx & 1023;
            const bool isb = (info >> 17) & 1u;
            const int id = k < MAXR ? sId[k] : root_id(info);
            bool isnode = !isb;
            if (isb) {
                const uint32_t slot = slot0 + (info >> 18);
                isnode = (uint32_t)B.s.gp[slot] == slot;
            }
            if (k < MAXR) {
                const unsigned long long s = sSum[k];
                const uint32_t bx = sBox[k];
                const long long area = (long long)(s & 0xFFFFull);
                const long long sx = (long long)((s >> 16) & ((1ull << 25) - 1)) + area * x0;
                const long long sy = (long long)((s >> 41) & ((1ull << 20) - 1)) + area * y0;
                const int xmin = x0 + (int)(bx & 1023u), xmax = x0 + (int)((bx >> 10) & 1023u);
                const int ymax = y0 + (int)(bx >> 20), ymin = y0 + r;
                if (!isb) {
                    if (id < cap) {
                        d.feat[0 * cap + id] = area;
                        d.feat[1 * cap + id] = xmin;
                        d.feat[2 * cap + id] = ymin;
                        d.feat[3 * cap + id] = xmax;
                        d.feat[4 * cap + id] = ymax;
                        d.feat[5 * cap + id] = sx;
                        d.feat[6 * cap + id] = sy;
                    }
                } else if (id < cap) {
                    hash_push(H, d.feat, cap, id, area, sx, sy, xmin, ymin, xmax, ymax);
                }
            }
            if (isnode) {
                if (id >= cap) {
                    over = true;
                    continue;
                }
                int p;
                if (y0 + r == 0) {
                    p = 0;
                } else if (r > 0) {
                    const int l = c >> 5;
                    const int q = sRowRun[r - 1] + sRunPre[r - 1][l] + __popc(sE[r - 1][l] & mask_le(c & 31)) - 1;
                    const int kk = rr[q];
                    p = kk < MAXR ? sId[kk] : root_id(ri[kk]);
                } else {
                    const TileGeo ga = tile_geo(d, lt - d.TX);   // the tile above
                    const uint32_t s2 = (uint32_t)(n_img + ga.b) + B.s.edges[ga.b + edge_bottom(ga, c)];
                    const uint32_t root = (uint32_t)B.s.gp[s2];
                    p = root < (uint32_t)n_img ? 0 : B.s.canon[root];
                }
                d.parent[id] = p;
                if (!isb && id < d.ncap) B.s.node_fg[d.node0 + id] = (uint8_t)((info >> 16) & 1u);
            }
        }
        if (!ok) atomicAnd(&sOk, 0);
        if (over) atomicOr(&sCap, 1);
        __syncthreads();
        hash_flush(H, d.feat, cap);
        if (threadIdx.x == 0) {
            if (!sOk) set_status(B, d, ST_ITER);
            if (sCap) set_status(B, d, ST_CAPACITY);
        }
        __syncthreads();
    }
}

void launch_write(const Batch &B, const LaunchCfg &c, cudaStream_t st) {
    k_write<<<min(B.n_tiles, 2 * c.sms), NTHREADS, WRITE_SMEM, st>>>(B);
}

cudaError_t configure_write() {
    return cudaFuncSetAttribute(k_write, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WRITE_SMEM);
}

}  // namespace ccl
