// Component filtering on the node tables: the paper's hole filling
// (Algorithm 3, hole-filling branch: a root whose surrounding component is
// not the exterior becomes equivalent to it, and its features merge into it;
// no pixel is rescanned) with an area threshold, and its dual for the other
// colour, the feature-based connected operator Section 5 names.
//
// Target colour background (hole filling): a hole (background node other
// than 0) is absorbed when its own area is <= T, and so is every foreground
// child of an absorbed hole. Target colour foreground (object removal): a
// foreground node with area <= T is absorbed by its parent background node,
// with its background children. Every node maps to its nearest
// ancestor-or-self that is not absorbed. T < 0 absorbs nothing; hole filling
// with T = INT64_MAX is exactly the unconditional fill of Algorithm 3.
//
//   k_fill_map    map, survivor features copied, parents of survivors
//   k_fill_merge  features of absorbed nodes merged into their survivor
//   k_relabel     label images rewritten through the map (Algorithm 4 on
//                 the filtered equivalence table)
//
// The node kernels walk one flat index over the nodes of every image of the
// last analysis: image i's nodes start at i + seg_base[first segment of i],
// since the node scan runs across all images in order and each image adds
// its exterior node.
#include "ccl_dev.cuh"

namespace ccl {

constexpr int FILL_WALK_LIMIT = 1 << 24;

struct FillView {
    const int32_t *parent;
    const int64_t *area;
    const uint8_t *fg;
    int64_t T;
    int32_t target;   // colour of the components that can be absorbed
};

__device__ __forceinline__ bool is_target(const FillView &v, int m) {
    return v.T >= 0 && m != 0 && (int)v.fg[m] == v.target && v.area[m] <= v.T;
}

// Every node m > 0 has 0 <= parent[m] < m; a value outside that range is
// reported (CCL_ERR_ITER_LIMIT) and the walk stops instead of reading it.
__device__ __forceinline__ bool absorbed(const FillView &v, int m, bool *ok) {
    if (m == 0) return false;
    if (is_target(v, m)) return true;
    if ((int)v.fg[m] == v.target) return false;
    const int p = v.parent[m];
    if (p < 0 || p >= m) {
        *ok = false;
        return false;
    }
    return is_target(v, p);
}

__device__ __forceinline__ int survivor(const FillView &v, int m, bool *ok) {
    for (int it = 0; it < FILL_WALK_LIMIT; ++it) {
        if (!absorbed(v, m, ok)) return m;
        const int p = v.parent[m];
        if (p < 0 || p >= m) {
            *ok = false;
            return m;
        }
        m = p;
    }
    *ok = false;
    return m;
}

__device__ __forceinline__ int64_t node_base(const Batch &B, int i) {
    return (int64_t)i + B.s.seg_base[B.desc[i].seg0];
}

// Image of flat node index f (cached range [lo, hi) of image img).
struct ImageCursor {
    int img = -1;
    int64_t lo = 0, hi = 0;
    __device__ void seek(const Batch &B, int64_t f) {
        if (f >= lo && f < hi) return;
        int a = 0, b = B.n_img - 1;
        while (a < b) {
            const int mid = (a + b + 1) >> 1;
            if (node_base(B, mid) <= f) a = mid; else b = mid - 1;
        }
        img = a;
        lo = node_base(B, a);
        hi = a + 1 < B.n_img ? node_base(B, a + 1) : (int64_t)B.n_img + B.s.seg_base[B.n_segs];
    }
};

__global__ void __launch_bounds__(256) k_fill_map(Batch B, int64_t T, int32_t target) {
    pdl_trigger();
    pdl_wait();
    const int64_t total = (int64_t)B.n_img + B.s.seg_base[B.n_segs];
    ImageCursor cur;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x) {
        cur.seek(B, f);
        const ImgDesc &d = B.desc[cur.img];
        const int k = (int)(f - cur.lo);
        if (d.fill_map == nullptr || k >= min(d.cap, d.ncap)) continue;
        const FillView v{d.parent, d.feat, B.s.node_fg + d.node0, T, target};
        const int64_t cap = d.cap;
        bool ok = true;
        const int s = survivor(v, k, &ok);
        d.fill_map[k] = s;
        if (s == k) {
#pragma unroll
            for (int q = 0; q < 7; ++q) d.filled_feat[q * cap + k] = d.feat[q * cap + k];
            const int p = d.parent[k];
            d.filled_parent[k] = p < 0 ? -1 : survivor(v, p, &ok);
        } else {
            d.filled_feat[0 * cap + k] = 0;
            d.filled_feat[1 * cap + k] = INT64_MAX;
            d.filled_feat[2 * cap + k] = INT64_MAX;
            d.filled_feat[3 * cap + k] = -1;
            d.filled_feat[4 * cap + k] = -1;
            d.filled_feat[5 * cap + k] = 0;
            d.filled_feat[6 * cap + k] = 0;
            d.filled_parent[k] = -1;
        }
        if (!ok) set_status(B, d, ST_ITER);
    }
}

// Absorbed nodes add their features to their survivor. A warp takes 32
// consecutive node ids at a time (coalesced loads); consecutive absorbed
// nodes usually share their survivor (the holes of one component are
// numbered close together), so a segmented scan in lane order combines each
// group of equal survivors and only the group's last lane pushes, through
// the CTA's hash table, then global atomics.
__global__ void __launch_bounds__(256) k_fill_merge(Batch B) {
    pdl_trigger();
    pdl_wait();
    __shared__ __align__(16) unsigned char hmem[HT_BYTES];
    const HashTab H = hash_carve(hmem);
    hash_init(H);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t total = (int64_t)B.n_img + B.s.seg_base[B.n_segs];
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    ImageCursor cur;
    // lane 31 carries its last group across iterations while the survivor
    // repeats (the holes of one large component, scattered over the image)
    long long ckey = -1;
    int cimg = 0;
    FeatAcc cv{0ull, 0ull, 0ull, INT32_MAX, INT32_MAX, -1, -1};
    auto push = [&](long long k, int im, const FeatAcc &a) {
        const ImgDesc &d = B.desc[im];
        hash_push(H, d.filled_feat, d.cap, im, (int)(uint32_t)k, a);
    };
    auto push_or_carry = [&](long long k, int im, const FeatAcc &a) {
        if (lane != 31) {
            push(k, im, a);
        } else if (k == ckey) {
            acc_merge(cv, a);
        } else {
            if (ckey >= 0) push(ckey, cimg, cv);
            ckey = k;
            cimg = im;
            cv = a;
        }
    };
    for (int64_t base = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < total;
         base += warps * 32) {
        const int64_t f = base + lane;
        long long key = -1;   // (image << 32) | survivor, -1: nothing to add
        FeatAcc v{0ull, 0ull, 0ull, INT32_MAX, INT32_MAX, -1, -1};
        int img = 0;
        if (f < total) {
            cur.seek(B, f);
            img = cur.img;
            const ImgDesc &d = B.desc[img];
            const int k = (int)(f - cur.lo);
            if (d.fill_map != nullptr && k < min(d.cap, d.ncap)) {
                const int s = d.fill_map[k];
                if (s != k) {
                    const int64_t cap = d.cap;
                    key = ((long long)img << 32) | (uint32_t)s;
                    v = FeatAcc{(unsigned long long)d.feat[0 * cap + k], (unsigned long long)d.feat[5 * cap + k],
                                (unsigned long long)d.feat[6 * cap + k], (int)d.feat[1 * cap + k],
                                (int)d.feat[2 * cap + k], (int)d.feat[3 * cap + k], (int)d.feat[4 * cap + k]};
                }
            }
        }
        // segmented inclusive scan over lanes with equal keys (skipped when
        // no lane has anything to add, or no two neighbours share a survivor)
        if (!__any_sync(FULL, key >= 0)) continue;
        const long long kprev = __shfl_up_sync(FULL, key, 1);
        if (!__any_sync(FULL, key >= 0 && lane > 0 && kprev == key)) {
            if (key >= 0) push_or_carry(key, img, v);
            continue;
        }
        int seg = (lane == 0 || kprev != key) ? lane : 0;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) seg = max(seg, __shfl_up_sync(FULL, seg, dd));
        // sums of 32-bit values whose warp total also fits in 32 bits move
        // through 32-bit shuffles (the usual case: small absorbed nodes)
        const unsigned long long lim = 1ull << 27;   // 32 lanes x 2^27 < 2^32
        if (__all_sync(FULL, v.area < lim && v.sx < lim && v.sy < lim)) {
            uint32_t ar = (uint32_t)v.area, sxr = (uint32_t)v.sx, syr = (uint32_t)v.sy;
#pragma unroll
            for (int dd = 1; dd < 32; dd <<= 1) {
                const uint32_t a = __shfl_up_sync(FULL, ar, dd), sx = __shfl_up_sync(FULL, sxr, dd),
                               sy = __shfl_up_sync(FULL, syr, dd);
                const int x0 = __shfl_up_sync(FULL, v.xmin, dd), y0 = __shfl_up_sync(FULL, v.ymin, dd),
                          x1 = __shfl_up_sync(FULL, v.xmax, dd), y1 = __shfl_up_sync(FULL, v.ymax, dd);
                if (lane - dd >= seg) {
                    ar += a;
                    sxr += sx;
                    syr += sy;
                    v.xmin = min(v.xmin, x0);
                    v.ymin = min(v.ymin, y0);
                    v.xmax = max(v.xmax, x1);
                    v.ymax = max(v.ymax, y1);
                }
            }
            v.area = ar;
            v.sx = sxr;
            v.sy = syr;
        } else {
#pragma unroll
            for (int dd = 1; dd < 32; dd <<= 1) {
                const unsigned long long a = __shfl_up_sync(FULL, v.area, dd), sx = __shfl_up_sync(FULL, v.sx, dd),
                                         sy = __shfl_up_sync(FULL, v.sy, dd);
                const int x0 = __shfl_up_sync(FULL, v.xmin, dd), y0 = __shfl_up_sync(FULL, v.ymin, dd),
                          x1 = __shfl_up_sync(FULL, v.xmax, dd), y1 = __shfl_up_sync(FULL, v.ymax, dd);
                if (lane - dd >= seg) {
                    v.area += a;
                    v.sx += sx;
                    v.sy += sy;
                    v.xmin = min(v.xmin, x0);
                    v.ymin = min(v.ymin, y0);
                    v.xmax = max(v.xmax, x1);
                    v.ymax = max(v.ymax, y1);
                }
            }
        }
        const long long knext = __shfl_down_sync(FULL, key, 1);
        if (key >= 0 && (lane == 31 || knext != key)) push_or_carry(key, img, v);
    }
    if (ckey >= 0) push(ckey, cimg, cv);
    __syncthreads();
    hash_flush(H, B.desc, true);
}

// Label images through the map: a pixel of node n takes map[n], in the
// label image of the survivor's colour (-1 in the other). In place is fine
// (each pixel is read before it is written, by the same thread).
__global__ void __launch_bounds__(256) k_relabel(Batch B) {
    pdl_trigger();
    pdl_wait();
    const ImgDesc &d = B.desc[blockIdx.y];
    if (d.fill_map == nullptr || d.fg == nullptr || d.fg_out == nullptr) return;
    const int64_t npx = (int64_t)d.w * d.h;
    const int n = min((int64_t)d.counts[0], min(d.cap, d.ncap));
    const uint8_t *col = B.s.node_fg + d.node0;
    bool ok = true;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npx; i += (int64_t)gridDim.x * blockDim.x) {
        const int f = d.fg[i], g = d.bg[i];
        const int node = f >= 0 ? f : g;
        int s = node, c = 0;
        if (node >= 0 && node < n) s = d.fill_map[node];
        if (s >= 0 && s < n) {
            c = col[s];
        } else {
            ok = false;
            s = -1;
        }
        d.fg_out[i] = c ? s : -1;
        d.bg_out[i] = c ? -1 : s;
    }
    if (!ok) set_status(B, d, ST_CAPACITY);
}

void launch_fill(const Batch &B, int64_t T, int32_t target, const LaunchCfg &c, cudaStream_t st,
                 const cudaEvent_t *ev) {
    const int grid = 8 * c.sms;
    if (ev) cudaEventRecord(ev[0], st);
    k_fill_map<<<grid, 256, 0, st>>>(B, T, target);
    if (ev) cudaEventRecord(ev[1], st);
    // the merge needs 64 registers per thread, so four of its CTAs fit an
    // SM: one resident wave, one table flush per CTA
    launch_dep(k_fill_merge, 4 * c.sms, 256, 0, st, B);
    if (ev) cudaEventRecord(ev[2], st);
}

void launch_relabel(const Batch &B, const LaunchCfg &c, cudaStream_t st) {
    const dim3 grid(max(1, (8 * c.sms + B.n_img - 1) / B.n_img), B.n_img);
    k_relabel<<<grid, 256, 0, st>>>(B);
}

}  // namespace ccl
