// ccl_analyze_static: the single-image analysis with its scratch in a
// fixed device array that is part of the library image, for callers that
// cannot allocate device memory.
//
// Who needs it: code whose device memory is owned entirely by another
// allocator (a framework or engine that reserves the GPU's memory pool up
// front and forbids raw cudaMalloc), and latency-critical loops that must
// not call cudaMalloc / cudaFree after start-up, because those calls can
// synchronise the whole device and take unbounded time. ccl_create owns its
// scratch through cudaMalloc; this entry point uses none.
//
// The array g_static_scratch (CCL_STATIC_SCRATCH_BYTES) lives on every GPU
// that loads the library, until the process exits. It holds the same
// tables as a context's scratch, laid out for one image of at most
// CCL_STATIC_MAX_PIXELS pixels with sides of at most CCL_STATIC_MAX_SIDE.
// Every call uses the same array and leaves its tables there; the first
// kernel of each call clears the counters and status words that must start
// at zero, and every other table is fully rewritten before it is read.
// Calls that overlap on the GPU (two streams, or two host threads) race on
// the array: callers must order them.
#include <mutex>

#include "../../include/ccl.h"
#include "ccl_dev.cuh"

using namespace ccl;

// The scratch array (file scope, internal linkage; one per device).
static __device__ __align__(256) unsigned char g_static_scratch[CCL_STATIC_SCRATCH_BYTES];

namespace {

constexpr size_t STATIC_BYTES = (size_t)CCL_STATIC_SCRATCH_BYTES;

constexpr int MAX_DEVICES = 64;
std::mutex g_static_mutex;
void *g_static_ptr[MAX_DEVICES] = {};
int g_static_sms[MAX_DEVICES] = {};

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Copy the descriptor into the array (device code names the array directly).
__global__ void k_static_desc(ImgDesc d, size_t off) {
    *reinterpret_cast<ImgDesc *>(g_static_scratch + off) = d;
}

// One-time set-up of the current device: the array's device address (host
// code cannot use the symbol itself) and the kernels' shared-memory limits.
cudaError_t static_setup(int dev, void **ptr, int *sms) {
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        e = configure_label();
        if (e != cudaSuccess) return e;
        e = configure_write();
        if (e != cudaSuccess) return e;
        g_static_sms[dev] = n;
        g_static_ptr[dev] = p;
    }
    *ptr = g_static_ptr[dev];
    *sms = g_static_sms[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" ccl_status ccl_analyze_static(const uint8_t *d_img, int32_t w, int32_t h, int32_t pitch,
                                         int32_t *d_fg_labels, int32_t *d_bg_labels, int32_t *d_tree_parent,
                                         int64_t *d_features, int64_t capacity, int32_t *d_counts,
                                         ccl_stream_t stream) {
    if (w <= 0 || h <= 0 || pitch < w || capacity < 1) return CCL_ERR_ARG;
    if (!d_img || !d_tree_parent || !d_features || !d_counts) return CCL_ERR_ARG;
    if ((d_fg_labels == nullptr) != (d_bg_labels == nullptr)) return CCL_ERR_ARG;
    if ((int64_t)w * h > CCL_STATIC_MAX_PIXELS || w > CCL_STATIC_MAX_SIDE || h > CCL_STATIC_MAX_SIDE)
        return CCL_ERR_CAPACITY;
    if ((pitch % 16) != 0 || ((uintptr_t)d_img % 16) != 0) return CCL_ERR_ALIGN;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return CCL_ERR_CUDA;
    void *base = nullptr;
    int sms = 0;
    if (static_setup(dev, &base, &sms) != cudaSuccess) return CCL_ERR_CUDA;

    // plan of one image (same geometry as the context path)
    ImgDesc d{};
    d.img = d_img;
    d.fg = d_fg_labels;
    d.bg = d_bg_labels;
    d.parent = d_tree_parent;
    d.feat = d_features;
    d.counts = d_counts;
    d.cap = capacity;
    d.w = w;
    d.h = h;
    d.pitch = pitch;
    d.TX = (w + TW_MAX - 1) / TW_MAX;
    d.TY = (h + TH_MAX - 1) / TH_MAX;
    const int64_t full = ((int64_t)(h + 1) / 2) * ((w + 1) / 2) + ((int64_t)w * h + 1) / 2 + 1;
    d.ncap = capacity < full ? capacity : full;
    d.vec = (w % 4 == 0) && d_fg_labels && ((uintptr_t)d_fg_labels % 16 == 0) && ((uintptr_t)d_bg_labels % 16 == 0);
    const int64_t tiles = (int64_t)d.TX * d.TY, segs = (int64_t)h * d.TX, px = (int64_t)w * h;
    const int64_t edges = 2 * (int64_t)w * d.TY + 2 * (int64_t)h * d.TX;

    // carve the array
    unsigned char *p = (unsigned char *)base;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char *q = p + off;
        off += up256(bytes);
        return q;
    };
    Scratch s;
    const size_t desc_off = off;
    take(sizeof(ImgDesc));
    s.fgbits = (uint32_t *)take(segs * WPR_MAX * 4);
    s.nodebits = (uint32_t *)take(segs * WPR_MAX * 4);
    s.run_root = (uint32_t *)take(px * 4);
    s.rootinfo = (uint32_t *)take(px * 4);
    s.tstat = (int4 *)take(tiles * 16);
    s.tsrc = (int4 *)take(tiles * 16);
    s.thdr = (TileHdr *)take(tiles * sizeof(TileHdr));
    s.edges = (uint16_t *)take(edges * 2);
    s.gp = (unsigned long long *)take((1 + edges) * 8);
    s.binfo = (uint32_t *)take((1 + edges) * 4);
    s.canon = (int32_t *)take((1 + edges) * 4);
    s.seg_cnt = (int32_t *)take(segs * 4);
    s.seg_base = (int32_t *)take((segs + 1) * 4);
    s.blk_sum = (int32_t *)take((segs / SCAN_B + 2) * 4);
    s.node_fg = (uint8_t *)take(d.ncap);
    s.img_cnt = (int32_t *)take(16);
    s.status = (int32_t *)take(16);
    s.work = (int32_t *)take(64);
    if (off > STATIC_BYTES) return CCL_ERR_CAPACITY;

    d.hitem0 = d.vitem0 = d.pitem0 = 0;
    d.tile0 = 0;
    d.seg0 = d.px0 = d.b0 = d.node0 = 0;
    Batch B;
    B.desc = (const ImgDesc *)(p + desc_off);
    B.th = TH_MAX;
    B.tw = TW_MAX;
    B.wpr = WPR_MAX;
    B.log_tw = 10;
    B.n_img = 1;
    B.n_tiles = (int32_t)tiles;
    B.n_segs = segs;
    B.hsplit = H_SPLIT_DEFAULT;
    B.n_hitems = (int64_t)(d.TY - 1) * d.TX * WPR_MAX * B.hsplit;
    B.n_vitems = (int64_t)(d.TX - 1) * h;
    B.n_pitems = 2 * (int64_t)d.TX * WPR_MAX + 2 * (int64_t)h;
    B.conn = CCL_CONN_8FG_4BG;
    B.labels = d_fg_labels != nullptr;
    B.s = s;

    cudaStream_t st = (cudaStream_t)stream;
    const LaunchCfg lc{sms};
    k_static_desc<<<1, 1, 0, st>>>(d, desc_off);
    launch_prologue(B, st);
    launch_label(B, lc, st);
    launch_merge(B, st);
    launch_resolve(B, lc, st);
    launch_scan(B, st);
    launch_canon(B, lc, st);
    launch_write(B, lc, st);
    return cudaGetLastError() == cudaSuccess ? CCL_OK : CCL_ERR_CUDA;
}
