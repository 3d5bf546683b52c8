// Internal device-side definitions of the CUDA path: tile geometry, the
// per-image descriptor, the scratch layout, and the bit and union-find
// primitives shared by the kernels.
//
// Terminology (mapped onto the paper's LSL B&W, Section 3.2):
//   run        a maximal horizontal run of one colour inside a tile row
//              (the paper's segment, Algorithm 1); a run never crosses a
//              tile's left or right edge.
//   local root the run that owns a tile-local component: the component's
//              raster-first run inside the tile. The in-tile union-find links
//              runs by minimum start index, the paper's union "by min"
//              (Algorithm 2) on the tile's own label space.
//   border root a local root whose component touches the tile's edge; only
//              these enter the device-wide union-find, keyed by the raster
//              index of their first pixel so that the final root of every
//              component is its raster-first run (Algorithm 3's final root).
//   node       a component of the whole image; node ids are 1 + the rank of
//              the component's first pixel in raster order, 0 = exterior.
#pragma once
#include <cstdint>
#include <utility>
#include <cuda_runtime.h>

namespace ccl {

constexpr int TW_MAX = 1024;           // tile width in pixels: 1024 (default, 32 words) or
constexpr int TW_MIN = 512;            // 512 (16 words), chosen per context (ccl_set_tile_cols)
constexpr int TH_MAX = 32;             // tile height in rows: 32 (default) or 16,
constexpr int TH_MIN = 16;             // chosen per context (ccl_set_tile_rows)
constexpr int TILE_PX = TH_MAX * TW_MAX;   // 32768: local pixel index fits 15 bits
constexpr int WPR_MAX = TW_MAX / 32;   // most 32-bit words per tile row
constexpr int NTHREADS = 256;          // threads of the write / resolve / canon kernels
constexpr int NWARPS = NTHREADS / 32;
// Horizontal tile-boundary merge items per word of the boundary row: each
// item takes 32 / hsplit of the word's columns, so a dense boundary spreads
// its unions over more threads (a per-context choice, Batch::hsplit).
constexpr int H_SPLIT_DEFAULT = 4;
constexpr int SCAN_B = 256;            // segments per block of the node scan
constexpr unsigned FULL = 0xFFFFFFFFu;

// Loop limits: every retry loop of the union-finds is bounded and reports
// CCL_ERR_ITER_LIMIT instead of spinning forever.
constexpr int LOCAL_FIND_LIMIT = TILE_PX + 8;
constexpr int LOCAL_UNION_LIMIT = 1 << 16;
constexpr int GLOBAL_FIND_LIMIT = 1 << 24;
constexpr int GLOBAL_UNION_LIMIT = 1 << 16;

// Status bits (identical values to ccl_status in include/ccl.h).
constexpr int ST_CAPACITY = 4;
constexpr int ST_ITER = 32;

// Per-image descriptor, built on the host for every analyse call.
struct ImgDesc {
    const uint8_t *img;
    int32_t *fg, *bg;          // label images or null
    int32_t *parent;           // [cap]
    int64_t *feat;             // [7][cap]
    int32_t *counts;           // [4]
    int64_t cap;
    int32_t *fill_map;         // [cap] or null
    int64_t *filled_feat;      // [7][cap]
    int32_t *filled_parent;    // [cap]
    int32_t *fg_out, *bg_out;  // label images rewritten through fill_map (or null)
    int32_t w, h, pitch;
    int32_t TX, TY;            // tiles across and down
    int32_t tile0;             // first flat tile of the image
    int64_t seg0;              // first segment; segment = one tile row (y, tx)
    int64_t node0;             // first per-node colour byte
    int64_t ncap;              // colour bytes reserved for the image
    int64_t hitem0, vitem0, pitem0;  // first border-merge work item of each kind
    int64_t px0;               // first entry of the per-pixel run / root tables
    int64_t b0;                // first entry of the per-edge-cell tables
    int32_t vec;               // label rows 16-byte aligned: vector stores
    int32_t pad_;
};

// Device scratch, carved out of one allocation by the host. A tile's
// run_root region holds one record per run of the tile, in raster order of
// the runs (the run ordinal): root ordinal << 16 | first pixel (row * 1024 +
// column) << 1 | colour.

// Geometry of one tile, written once per analysis by the prologue and
// fetched by the tile kernels with a bulk copy ahead of use.
struct __align__(16) TileHdr {
    int64_t px;                // first entry of the per-pixel tables
    int64_t b;                 // first edge cell
    int64_t b_above;           // first edge cell of the tile above (same column)
    int64_t seg0;              // the image's first segment
    int32_t img, tx, y0, x0, th, tw, TX, w;
};

struct Scratch {
    uint32_t *fgbits;          // [segs*32] foreground bit plane, rows of TX*32 words
    uint32_t *nodebits;        // [segs*32] 1 at the first pixel of every node
    uint32_t *run_root;        // [pixels] per run: root ordinal << 16 | first pixel << 1 | colour
    uint32_t *rootinfo;        // [pixels] per local root, see k_label.cu
    int4 *tstat;               // [tiles] {runs, roots, border roots, image}
    int4 *tsrc;                // [tiles] {first image byte (lo, hi), pitch, rows | copy bytes << 8}
    TileHdr *thdr;             // [tiles]
    uint16_t *edges;           // [edge cells] border ordinal of each edge cell's root
    unsigned long long *gp;    // [n_img + edge cells] device-wide union-find
    uint32_t *binfo;           // [same] root ordinal | colour << 16
    int32_t *canon;            // [same] node id of border roots that are nodes
    int32_t *seg_cnt;          // [segs]
    int32_t *seg_base;         // [segs + 1]
    int32_t *blk_sum;          // [segs / SCAN_B + 1]
    uint8_t *node_fg;          // [sum of ncap] colour of every node
    int32_t *img_cnt;          // [n_img][4]: [1] = foreground nodes
    int32_t *status;           // [1] OR of status bits of the last call
    int32_t *work;             // [8] tile counters of the persistent kernels
};

struct Batch {
    const ImgDesc *desc;
    int32_t th;                // tile height of this call (16 or 32)
    int32_t tw;                // tile width of this call (512 or 1024)
    int32_t wpr;               // tw / 32: words per tile row
    int32_t log_tw;            // log2(tw)
    int32_t n_img;
    int32_t n_tiles;
    int64_t n_segs;
    int64_t n_hitems, n_vitems, n_pitems;
    int32_t conn;
    int32_t labels;
    int32_t hsplit;            // cross-band merge items per boundary word: 1, 2, 4 or 8
    Scratch s;
};

// ------------------------------------------------------------ bit helpers

__device__ __forceinline__ uint32_t mask_le(int b) { return FULL >> (31 - b); }      // bits 0..b
__device__ __forceinline__ uint32_t mask_lt(int b) { return b ? (FULL >> (32 - b)) : 0u; }  // bits 0..b-1

// 4 bytes -> 4 bits, bit j set when byte j is nonzero. The four flag bits
// (7, 15, 23, 31) are gathered by one multiply whose partial products land
// on distinct bit positions, so no carries occur.
__device__ __forceinline__ uint32_t nz4(uint32_t v) {
    uint32_t t = __vcmpne4(v, 0u) & 0x80808080u;
    return (((t >> 7) * 0x00204081u) >> 21) & 0xFu;
}

__device__ __forceinline__ uint32_t nz16(uint4 v) {
    return nz4(v.x) | (nz4(v.y) << 4) | (nz4(v.z) << 8) | (nz4(v.w) << 12);
}

// ------------------------------------- bulk copies into shared memory
// One thread issues cp.async.bulk copies (global -> shared, 16-byte aligned,
// sizes a multiple of 16) that complete on a shared-memory mbarrier; the
// consumers wait on the barrier's phase parity, a bounded number of times.

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Order this thread's earlier generic-proxy accesses of shared memory
// before its later bulk copies into it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

constexpr int MBAR_WAIT_LIMIT = 1 << 20;

// True once the phase with the given parity has completed; false when the
// wait gave up after MBAR_WAIT_LIMIT polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < MBAR_WAIT_LIMIT; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Warp-wide exclusive prefix sum; *total receives the sum over the warp.
__device__ __forceinline__ int warp_excl_sum(int v, int *total) {
    const int lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(FULL, x, 31);
    return x - v;
}

// The same over unsigned values (packed 16-bit fields whose sums stay
// below 2^16 each).
__device__ __forceinline__ uint32_t warp_excl_sum_u32(uint32_t v, uint32_t *total) {
    const int lane = threadIdx.x & 31;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    *total = __shfl_sync(FULL, x, 31);
    return x - v;
}

// Minimum over lanes strictly above this one (big when none).
__device__ __forceinline__ int warp_suffix_min_excl(int v, int none) {
    const int lane = threadIdx.x & 31;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_down_sync(FULL, x, o);
        if (lane + o < 32) x = min(x, y);
    }
    int r = __shfl_down_sync(FULL, x, 1);
    return lane == 31 ? none : r;
}

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ void set_status(const Batch &B, const ImgDesc &d, int bits) {
    atomicOr(B.s.status, bits);
    atomicOr(d.counts + 3, bits);
}

// Geometry of one tile. Per-tile tables are packed without gaps:
//   px  first entry of the tile's run / root tables (th * tw entries: a tile
//       has at most one run and one root per pixel), in raster order of
//       tiles: all bands above hold TH * w pixels, tiles to the left th * TW
//       (TH, TW: the call's tile height and width);
//   b   first entry of the tile's edge-cell tables (2 tw + 2 th entries: top
//       row, bottom row, left column, right column); border roots of the
//       tile occupy device-wide union-find slots n_img + b + ordinal.
struct TileGeo {
    int ty, tx, y0, x0, th, tw;
    int64_t px, b;
};

__device__ __forceinline__ TileGeo tile_geo(const ImgDesc &d, int lt, int TH, int TW) {
    TileGeo g;
    g.ty = lt / d.TX;
    g.tx = lt - g.ty * d.TX;
    g.y0 = g.ty * TH;
    g.x0 = g.tx * TW;
    g.th = min(TH, d.h - g.y0);
    g.tw = min(TW, d.w - g.x0);
    g.px = d.px0 + (int64_t)g.y0 * d.w + (int64_t)g.th * g.x0;
    g.b = d.b0 + (int64_t)g.ty * (2 * (int64_t)d.w + 2 * (int64_t)TH * d.TX) + (int64_t)g.tx * (2 * TW + 2 * g.th);
    return g;
}


// Image owning flat tile t: the last image whose tile0 <= t.
__device__ __forceinline__ int image_of_tile(const Batch &B, int t) {
    int lo = 0, hi = B.n_img - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (B.desc[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// --------------------------------------------- in-tile union-find (shared)
// Parents are 32-bit run-start indices (row * TW + column); a root is its
// own parent and every link points to a smaller index, so a native shared
// atomicMin both links and resolves races: the union by minimum of
// Algorithm 2 on the tile's label space.

// Shared-memory slot of entry i of a per-pixel or per-run table. Entries
// are addressed as row * 1024 + 32 * lane + bit (or lane * runs-per-word +
// j), so the lanes of a warp touch the same bit position of their words at
// the same time; XOR-ing the low five bits with the next five spreads them
// over the 32 banks. The map is a bijection on every block of 1024 entries.
__device__ __forceinline__ int swz(int i) { return i ^ ((i >> 5) & 31); }

__device__ __forceinline__ int local_find(const uint32_t *par, int a, bool *ok) {
    for (int it = 0; it < LOCAL_FIND_LIMIT; ++it) {
        const int p = (int)*(volatile const uint32_t *)(par + swz(a));
        if (p == a) return a;
        a = p;
    }
    *ok = false;
    return a;
}

// Find with path halving: every other node on the way up is pointed at its
// grandparent, which is one of its ancestors whatever unions run at the same
// time (links only ever point at smaller indices of the same class). A later
// phase that needs every run to point straight at its root must therefore
// not run concurrently with this one.
__device__ __forceinline__ int local_find_halving(uint32_t *par, int a, bool *ok) {
    for (int it = 0; it < LOCAL_FIND_LIMIT; ++it) {
        const int p = (int)*(volatile uint32_t *)(par + swz(a));
        if (p == a) return a;
        const int gp = (int)*(volatile uint32_t *)(par + swz(p));
        if (gp == p) return p;
        *(volatile uint32_t *)(par + swz(a)) = (uint32_t)gp;
        a = gp;
    }
    *ok = false;
    return a;
}

__device__ __forceinline__ void local_union(uint32_t *par, int a, int b, bool *ok) {
    for (int it = 0; it < LOCAL_UNION_LIMIT; ++it) {
        a = local_find_halving(par, a, ok);
        b = local_find_halving(par, b, ok);
        if (a == b || !*ok) return;
        if (a < b) { const int t = a; a = b; b = t; }
        const int old = (int)atomicMin(par + swz(a), (uint32_t)b);
        if (old == a) return;
        a = old;
    }
    *ok = false;
}

// ------------------------------------------ device-wide union-find (global)
// gp[slot] = ((key + 1) << 32) | parent_slot, key = raster index of the
// first pixel of the slot's parent (0 for an image's exterior slot). Values
// only decrease, so 64-bit atomicMin links a root under a smaller key, and
// the same atomicMin halves paths safely while other threads link.

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p) {
    return *(volatile const unsigned long long *)p;
}

__device__ __forceinline__ uint32_t global_find(unsigned long long *gp, uint32_t a, bool *ok) {
    for (int it = 0; it < GLOBAL_FIND_LIMIT; ++it) {
        unsigned long long v = ld_volatile_u64(gp + a);
        uint32_t p = (uint32_t)v;
        if (p == a) return a;
        unsigned long long vp = ld_volatile_u64(gp + p);
        uint32_t pp = (uint32_t)vp;
        if (pp != p) atomicMin(gp + a, vp);  // path halving: point a at its grandparent
        a = pp;
    }
    *ok = false;
    return a;
}

__device__ __forceinline__ void global_union(unsigned long long *gp, uint32_t a, uint32_t b, bool *ok) {
    for (int it = 0; it < GLOBAL_UNION_LIMIT; ++it) {
        a = global_find(gp, a, ok);
        b = global_find(gp, b, ok);
        if (a == b || !*ok) return;
        unsigned long long va = ld_volatile_u64(gp + a), vb = ld_volatile_u64(gp + b);
        if ((uint32_t)va != a || (uint32_t)vb != b) continue;  // linked meanwhile: retry
        if (va < vb) {
            uint32_t t = a; a = b; b = t;
            unsigned long long tv = va; va = vb; vb = tv;
        }
        unsigned long long old = atomicMin(gp + a, vb);
        if (old == va) return;
        a = (uint32_t)old;
    }
    *ok = false;
}


// ------------------------------------------- feature merges in global memory
// Features are int64 structure-of-arrays: base[f * cap + id]. Two forms of a
// contribution: global reductions (red: no value returned, the thread does
// not wait for the L2 round trip; the writer's per-tile flushes, spread over
// many records), and atomics (the filter's merge, whose flushes from every
// CTA meet on a few large survivors: measured faster there).

__device__ __forceinline__ void red_add_u64(int64_t *p, unsigned long long v) {
    asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_min_s64(int64_t *p, long long v) {
    asm volatile("red.global.min.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void red_max_s64(int64_t *p, long long v) {
    asm volatile("red.global.max.s64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void feat_atomic(int64_t *base, int64_t cap, int id, unsigned long long area,
                                            unsigned long long sx, unsigned long long sy, long long xmin,
                                            long long ymin, long long xmax, long long ymax) {
    atomicAdd((unsigned long long *)(base + 0 * cap + id), area);
    atomicMin((long long *)(base + 1 * cap + id), xmin);
    atomicMin((long long *)(base + 2 * cap + id), ymin);
    atomicMax((long long *)(base + 3 * cap + id), xmax);
    atomicMax((long long *)(base + 4 * cap + id), ymax);
    atomicAdd((unsigned long long *)(base + 5 * cap + id), sx);
    atomicAdd((unsigned long long *)(base + 6 * cap + id), sy);
}

// A small open-addressing table in shared memory that combines the feature
// contributions a CTA makes to the same node before they reach global
// memory: a component spanning many tiles (or a survivor absorbing many
// holes) would otherwise receive one atomic per contribution on the same
// address. Keys are (image << 32 | node); entries that do not fit go
// straight to global atomics.
constexpr int HT = 256;
constexpr size_t HT_BYTES = (size_t)HT * (4 * 8 + 4 * 4);
constexpr unsigned long long HT_EMPTY = ~0ull;

struct HashTab {
    unsigned long long *key, *area, *sx, *sy;
    int *xmin, *ymin, *xmax, *ymax;
};

__device__ __forceinline__ HashTab hash_carve(void *mem) {
    HashTab H;
    H.key = (unsigned long long *)mem;
    H.area = H.key + HT;
    H.sx = H.area + HT;
    H.sy = H.sx + HT;
    H.xmin = (int *)(H.sy + HT);
    H.ymin = H.xmin + HT;
    H.xmax = H.ymin + HT;
    H.ymax = H.xmax + HT;
    return H;
}

__device__ __forceinline__ void hash_init(const HashTab &H) {
    for (int e = threadIdx.x; e < HT; e += blockDim.x) {
        H.key[e] = HT_EMPTY;
        H.area[e] = 0;
        H.sx[e] = 0;
        H.sy[e] = 0;
        H.xmin[e] = INT32_MAX;
        H.ymin[e] = INT32_MAX;
        H.xmax[e] = -1;
        H.ymax[e] = -1;
    }
}

// Features of one contribution (global coordinates).
struct FeatAcc {
    unsigned long long area, sx, sy;
    int xmin, ymin, xmax, ymax;
};

__device__ __forceinline__ void acc_merge(FeatAcc &a, const FeatAcc &b) {
    a.area += b.area;
    a.sx += b.sx;
    a.sy += b.sy;
    a.xmin = min(a.xmin, b.xmin);
    a.ymin = min(a.ymin, b.ymin);
    a.xmax = max(a.xmax, b.xmax);
    a.ymax = max(a.ymax, b.ymax);
}

// base / cap: the feature table the entry belongs to (used when the table is full).
__device__ __forceinline__ void hash_push(const HashTab &H, int64_t *base, int64_t cap, int img, int id,
                                          const FeatAcc &v) {
    const unsigned long long key = ((unsigned long long)(uint32_t)img << 32) | (uint32_t)id;
    const uint32_t h = ((uint32_t)id * 2654435761u + (uint32_t)img * 40503u) >> 24;
    for (int probe = 0; probe < 8; ++probe) {
        const int e = (h + probe) & (HT - 1);
        const unsigned long long prev = atomicCAS(H.key + e, HT_EMPTY, key);
        if (prev == HT_EMPTY || prev == key) {
            atomicAdd(H.area + e, v.area);
            atomicAdd(H.sx + e, v.sx);
            atomicAdd(H.sy + e, v.sy);
            atomicMin(H.xmin + e, v.xmin);
            atomicMin(H.ymin + e, v.ymin);
            atomicMax(H.xmax + e, v.xmax);
            atomicMax(H.ymax + e, v.ymax);
            return;
        }
    }
    feat_atomic(base, cap, id, v.area, v.sx, v.sy, v.xmin, v.ymin, v.xmax, v.ymax);
}

// Flush every entry into the feature table of its image: the analysed
// features (filled = false) or the filled ones.
__device__ __forceinline__ void hash_flush(const HashTab &H, const ImgDesc *desc, bool filled) {
    for (int e = threadIdx.x; e < HT; e += blockDim.x) {
        const unsigned long long key = H.key[e];
        if (key == HT_EMPTY) continue;
        const ImgDesc &d = desc[key >> 32];
        feat_atomic(filled ? d.filled_feat : d.feat, d.cap, (int)(uint32_t)key, H.area[e], H.sx[e], H.sy[e],
                    H.xmin[e], H.ymin[e], H.xmax[e], H.ymax[e]);
    }
}

// ------------------------------------------------ programmatic launches
// Every kernel after the first of an analysis is launched as a programmatic
// dependent of the kernel before it (launch_dep): its CTAs may be scheduled
// once every CTA of that kernel has allowed it (pdl_trigger), and they wait
// (pdl_wait, first thing in every kernel) until that kernel has completed
// and its memory is visible. The small kernels allow it at their start; the
// persistent tile kernels when a CTA has no tile left, so that the next
// kernel's launch overlaps their tail.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// --------------------------------------------------------- host launchers
struct LaunchCfg {
    int sms;
};

void launch_prologue(const Batch &B, cudaStream_t st);
void launch_label(const Batch &B, const LaunchCfg &c, cudaStream_t st);
void launch_merge(const Batch &B, cudaStream_t st);
void launch_resolve(const Batch &B, const LaunchCfg &c, cudaStream_t st);
void launch_scan(const Batch &B, cudaStream_t st);
void launch_canon(const Batch &B, const LaunchCfg &c, cudaStream_t st);
void launch_write(const Batch &B, const LaunchCfg &c, cudaStream_t st);
void launch_fill(const Batch &B, int64_t area_threshold, int32_t target_fg, const LaunchCfg &c, cudaStream_t st,
                 const cudaEvent_t *ev = nullptr);
void launch_relabel(const Batch &B, const LaunchCfg &c, cudaStream_t st);
cudaError_t configure_label();
cudaError_t configure_write();

}  // namespace ccl
