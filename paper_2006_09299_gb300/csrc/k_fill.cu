// Hole filling on the node tables (the paper's Algorithm 3, hole-filling
// branch: a root whose surrounding component is not the exterior becomes
// equivalent to it, and its features merge into it; no pixel is rescanned).
//
// Extended with an area threshold T: a hole (background node other than 0)
// is absorbed when its own area is <= T, and so is every foreground child of
// an absorbed hole. Every node maps to its nearest ancestor-or-self that is
// not absorbed. T < 0 absorbs nothing; T = INT64_MAX absorbs every hole and
// reproduces the unconditional fill of Algorithm 3.
//
//   k_fill_map    map, survivor features copied, parents of survivors
//   k_fill_merge  features of absorbed nodes merged into their survivor
#include "ccl_dev.cuh"

namespace ccl {

constexpr int FILL_WALK_LIMIT = 1 << 24;

struct FillView {
    const int32_t *parent;
    const int64_t *area;
    const uint8_t *fg;
    int64_t T;
};

__device__ __forceinline__ bool is_hole(const FillView &v, int m) {
    return v.T >= 0 && m != 0 && !v.fg[m] && v.area[m] <= v.T;
}

// Every node m > 0 has 0 <= parent[m] < m; a value outside that range is
// reported (CCL_ERR_ITER_LIMIT) and the walk stops instead of reading it.
__device__ __forceinline__ bool absorbed(const FillView &v, int m, bool *ok) {
    if (m == 0) return false;
    if (is_hole(v, m)) return true;
    if (!v.fg[m]) return false;
    const int p = v.parent[m];
    if (p < 0 || p >= m) {
        *ok = false;
        return false;
    }
    return is_hole(v, p);
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

__device__ __forceinline__ int fill_nodes(const ImgDesc &d) {
    const int n = d.counts[0];
    return (int)min((int64_t)n, min(d.cap, d.ncap));
}

__global__ void __launch_bounds__(256) k_fill_map(Batch B, int64_t T) {
    const ImgDesc &d = B.desc[blockIdx.y];
    if (d.fill_map == nullptr) return;
    const int n = fill_nodes(d);
    const FillView v{d.parent, d.feat, B.s.node_fg + d.node0, T};
    const int64_t cap = d.cap;
    bool ok = true;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int s = survivor(v, k, &ok);
        d.fill_map[k] = s;
        if (s == k) {
#pragma unroll
            for (int f = 0; f < 7; ++f) d.filled_feat[f * cap + k] = d.feat[f * cap + k];
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
    }
    if (!ok) set_status(B, d, ST_ITER);
}

__global__ void __launch_bounds__(256) k_fill_merge(Batch B) {
    __shared__ __align__(16) unsigned char hmem[HT_BYTES];
    const ImgDesc &d = B.desc[blockIdx.y];
    if (d.fill_map == nullptr) return;
    const int n = fill_nodes(d);
    const int64_t cap = d.cap;
    const HashTab H = hash_carve(hmem);
    hash_init(H);
    __syncthreads();
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int s = d.fill_map[k];
        if (s == k) continue;
        hash_push(H, d.filled_feat, cap, s, (unsigned long long)d.feat[0 * cap + k],
                  (unsigned long long)d.feat[5 * cap + k], (unsigned long long)d.feat[6 * cap + k],
                  (int)d.feat[1 * cap + k], (int)d.feat[2 * cap + k], (int)d.feat[3 * cap + k],
                  (int)d.feat[4 * cap + k]);
    }
    __syncthreads();
    hash_flush(H, d.filled_feat, cap);
}

void launch_fill(const Batch &B, int64_t T, const LaunchCfg &c, cudaStream_t st, const cudaEvent_t *ev) {
    const int bx = max(1, (4 * c.sms + B.n_img - 1) / B.n_img);
    const dim3 grid(bx, B.n_img);
    if (ev) cudaEventRecord(ev[0], st);
    k_fill_map<<<grid, 256, 0, st>>>(B, T);
    if (ev) cudaEventRecord(ev[1], st);
    k_fill_merge<<<grid, 256, 0, st>>>(B);
    if (ev) cudaEventRecord(ev[2], st);
}

}  // namespace ccl
