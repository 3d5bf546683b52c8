// Host side of the library: argument checks, the per-call plan of tiles and
// work items, scratch ownership, the launch sequence, and the C ABI declared
// in include/ccl.h.
//
// One analysis = seven stream-ordered phases, each one launch over the tiles
// (or work items) of every image of the call:
//   prologue -> label -> merge -> resolve -> scan -> canon -> write
// Nothing in a call synchronises with the host; errors found on the device
// are OR'd into the status word and into each image's counts[3].
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/ccl.h"
#include "ccl_dev.cuh"

using namespace ccl;

namespace {

constexpr size_t ALIGN = 256;

size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

int64_t formula_capacity(int64_t w, int64_t h) {
    return ((h + 1) / 2) * ((w + 1) / 2) + (w * h + 1) / 2 + 1;
}

// Sizes that a context's scratch must hold.
struct Limits {
    int64_t images = 0, tiles = 0, segs = 0, words = 0, pixels = 0, edges = 0, ncap = 0;
    bool fits(const Limits &o) const {
        return o.images <= images && o.tiles <= tiles && o.segs <= segs && o.words <= words &&
               o.pixels <= pixels && o.edges <= edges && o.ncap <= ncap;
    }
};

struct Plan {
    std::vector<ImgDesc> d;
    int32_t th = TH_MAX;
    int32_t tw = TW_MAX;
    int32_t hsplit = H_SPLIT_DEFAULT;
    Limits need;
    int32_t n_tiles = 0;
    int64_t n_segs = 0, n_h = 0, n_v = 0, n_p = 0;
    bool labels = false;
};

// Shape signature of a batch: equal signatures give equal launch grids.
struct Shape {
    std::vector<int64_t> v;
    bool operator<(const Shape &o) const { return v < o.v; }
};

struct Graph {
    cudaGraphExec_t exec = nullptr;
};

int g_sms = 0;
std::once_flag g_once;
cudaError_t g_init_err = cudaSuccess;

cudaError_t init_device() {
    std::call_once(g_once, [] {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = configure_label();
        if (e == cudaSuccess) e = configure_write();
        g_init_err = e;
    });
    return g_init_err;
}

}  // namespace

struct ccl_ctx {
    bool batched = false;
    int32_t w = 0, h = 0, pitch = 0;    // fixed shape of a single-image context
    int32_t conn = 0;
    int32_t th = TH_MAX;                // tile height (16 or 32)
    int32_t tw = TW_MAX;                // tile width (512 or 1024)
    int32_t hsplit = H_SPLIT_DEFAULT;   // cross-band merge items per boundary word
    Limits cap;
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
    ImgDesc *d_desc = nullptr;          // device copy of the plan
    ImgDesc *h_desc = nullptr;          // pinned staging of the plan, RING slots
    cudaEvent_t ring_ev[8] = {};        // slot k may be rewritten once its copy ran
    int ring_pos = 0;
    Scratch s{};
    Plan last;                          // plan of the last analyse (for fill)
    bool have_last = false;
    cudaStream_t last_stream = nullptr;
    bool graph_cache = true;
    std::map<Shape, Graph> graphs;
    // instrumentation
    int64_t launches = 0;
    std::vector<std::vector<cudaEvent_t>> timing;  // one event set per timed call
    std::vector<int> timing_kind;                  // 0 analyse, 1 fill
    size_t timing_used = 0;
};

// Kernels per analysis (prologue, label, merge, resolve, 3 scan, canon, write)
// and per hole filling (map, merge).
constexpr int ANALYSE_KERNELS = 9;
constexpr int FILL_KERNELS = 2;
constexpr int ANALYSE_PHASES = 7;

constexpr int RING = 8;

static ccl_status from_cuda(cudaError_t e) { return e == cudaSuccess ? CCL_OK : CCL_ERR_CUDA; }

static Limits limits_of_bounds(int64_t images, int64_t pixels, int64_t max_side) {
    Limits L;
    L.images = images;
    L.pixels = pixels;
    // tiles of one image <= (h/TH + 1)(w/TW + 1) <= wh/(TH TW) + h/TH + w/TW + 1,
    // sized for the smallest tile so that every tile shape can run
    L.tiles = pixels / (TH_MIN * TW_MIN) + images * (max_side / TH_MIN + max_side / TW_MIN + 1);
    // tile rows (segments) = h * ceil(w/TW) <= wh/TW + h
    L.segs = pixels / TW_MIN + images * max_side;
    // bit-plane words = h * ceil(w/TW) * TW/32 <= wh/32 + h * TW_MAX/32
    L.words = pixels / 32 + images * max_side * WPR_MAX;
    // edge cells = 2 w TY + 2 h TX <= 2wh/TH + 2w + 2wh/TW + 2h
    L.edges = 2 * pixels / TH_MIN + 2 * pixels / TW_MIN + images * 4 * max_side;
    L.ncap = (3 * pixels) / 4 + images * (max_side / 2 + 3);
    return L;
}

static size_t carve(const Limits &L, Scratch *s, ImgDesc **desc, char *base) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char * {
        char *p = base ? base + off : nullptr;
        off += align_up(bytes);
        return p;
    };
    s->fgbits = (uint32_t *)take(L.words * 4);
    s->nodebits = (uint32_t *)take(L.words * 4);
    s->run_root = (uint32_t *)take(L.pixels * 4);
    s->rootinfo = (uint32_t *)take(L.pixels * 4);
    s->tstat = (int4 *)take(L.tiles * 16);
    s->tsrc = (int4 *)take(L.tiles * 16);
    s->thdr = (TileHdr *)take(L.tiles * sizeof(TileHdr));
    s->edges = (uint16_t *)take(L.edges * 2);
    s->gp = (unsigned long long *)take((L.images + L.edges) * 8);
    s->binfo = (uint32_t *)take((L.images + L.edges) * 4);
    s->canon = (int32_t *)take((L.images + L.edges) * 4);
    s->seg_cnt = (int32_t *)take(L.segs * 4);
    s->seg_base = (int32_t *)take((L.segs + 1) * 4);
    s->blk_sum = (int32_t *)take((L.segs / SCAN_B + 2) * 4);
    s->node_fg = (uint8_t *)take(L.ncap);
    s->img_cnt = (int32_t *)take(L.images * 16);
    s->status = (int32_t *)take(16);
    s->work = (int32_t *)take(64);
    *desc = (ImgDesc *)take(L.images * sizeof(ImgDesc));
    return off;
}

static ccl_status alloc_ctx(ccl_ctx *c, const Limits &L) {
    cudaError_t e = init_device();
    if (e != cudaSuccess) return CCL_ERR_CUDA;
    Scratch tmp;
    ImgDesc *dd;
    const size_t bytes = carve(L, &tmp, &dd, nullptr);
    void *p = nullptr;
    e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CCL_ERR_OOM;
    }
    c->scratch = p;
    c->scratch_bytes = bytes;
    carve(L, &c->s, &c->d_desc, (char *)p);
    c->cap = L;
    e = cudaMallocHost((void **)&c->h_desc, sizeof(ImgDesc) * L.images * RING);
    if (e != cudaSuccess) return CCL_ERR_OOM;
    for (int k = 0; k < RING; ++k) {
        e = cudaEventCreateWithFlags(&c->ring_ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) return CCL_ERR_CUDA;
    }
    return CCL_OK;
}

static ccl_status check_image(const ccl_image_desc &x) {
    if (x.w <= 0 || x.h <= 0 || x.pitch < x.w) return CCL_ERR_ARG;
    if ((int64_t)x.w * x.h >= (int64_t)1 << 31) return CCL_ERR_ARG;
    if (!x.img || !x.tree_parent || !x.features || !x.counts || x.capacity < 1) return CCL_ERR_ARG;
    if ((x.fg_labels == nullptr) != (x.bg_labels == nullptr)) return CCL_ERR_ARG;
    if ((x.pitch % 16) != 0 || ((uintptr_t)x.img % 16) != 0) return CCL_ERR_ALIGN;
    return CCL_OK;
}

static ccl_status build_plan(const ccl_image_desc *in, int n, int32_t th, int32_t tw, int32_t hsplit, Plan *P) {
    P->d.assign(n, ImgDesc{});
    P->th = th;
    P->tw = tw;
    P->hsplit = hsplit;
    const int32_t wpr = tw / 32;
    int64_t tiles = 0, segs = 0, px = 0, edges = 0, ncap = 0, hi = 0, vi = 0, pi = 0;
    bool any_labels = false;
    for (int i = 0; i < n; ++i) {
        const ccl_image_desc &x = in[i];
        ccl_status st = check_image(x);
        if (st != CCL_OK) return st;
        ImgDesc &d = P->d[i];
        d.img = x.img;
        d.fg = x.fg_labels;
        d.bg = x.bg_labels;
        d.parent = x.tree_parent;
        d.feat = x.features;
        d.counts = x.counts;
        d.cap = x.capacity;
        d.fill_map = x.fill_map;
        d.filled_feat = x.filled_features;
        d.filled_parent = x.filled_parent;
        d.w = x.w;
        d.h = x.h;
        d.pitch = x.pitch;
        d.TX = (x.w + tw - 1) / tw;
        d.TY = (x.h + th - 1) / th;
        d.tile0 = (int32_t)tiles;
        d.seg0 = segs;
        d.px0 = px;
        d.b0 = edges;
        d.node0 = ncap;
        d.ncap = std::min<int64_t>(x.capacity, formula_capacity(x.w, x.h));
        d.hitem0 = hi;
        d.vitem0 = vi;
        d.pitem0 = pi;
        d.vec = (x.w % 4 == 0) && x.fg_labels && ((uintptr_t)x.fg_labels % 16 == 0) &&
                ((uintptr_t)x.bg_labels % 16 == 0);
        any_labels |= x.fg_labels != nullptr;
        tiles += (int64_t)d.TX * d.TY;
        segs += (int64_t)x.h * d.TX;
        px += (int64_t)x.w * x.h;
        edges += 2 * (int64_t)x.w * d.TY + 2 * (int64_t)x.h * d.TX;
        ncap += d.ncap;
        hi += (int64_t)(d.TY - 1) * d.TX * wpr * hsplit;
        vi += (int64_t)(d.TX - 1) * x.h;
        pi += 2 * (int64_t)d.TX * wpr + 2 * (int64_t)x.h;
    }
    if (tiles >= INT32_MAX || n + edges >= INT32_MAX) return CCL_ERR_CAPACITY;
    P->n_tiles = (int32_t)tiles;
    P->n_segs = segs;
    P->n_h = hi;
    P->n_v = vi;
    P->n_p = pi;
    P->labels = any_labels;
    P->need.images = n;
    P->need.tiles = tiles;
    P->need.segs = segs;
    P->need.words = segs * wpr;
    P->need.pixels = px;
    P->need.edges = edges;
    P->need.ncap = ncap;
    return CCL_OK;
}

static Batch make_batch(const ccl_ctx *c, const Plan &P) {
    Batch B;
    B.desc = c->d_desc;
    B.th = P.th;
    B.tw = P.tw;
    B.wpr = P.tw / 32;
    B.log_tw = P.tw == 1024 ? 10 : 9;
    B.n_img = (int32_t)P.d.size();
    B.n_tiles = P.n_tiles;
    B.n_segs = P.n_segs;
    B.n_hitems = P.n_h;
    B.n_vitems = P.n_v;
    B.n_pitems = P.n_p;
    B.conn = c->conn;
    B.labels = P.labels ? 1 : 0;
    B.hsplit = P.hsplit;
    B.s = c->s;
    return B;
}

// Enqueue the phases; ev (optional) receives ANALYSE_PHASES + 1 events
// around them.
static void enqueue_analysis(const Batch &B, cudaStream_t st, const cudaEvent_t *ev = nullptr) {
    const LaunchCfg lc{g_sms};
    auto mark = [&](int k) {
        if (ev) cudaEventRecord(ev[k], st);
    };
    mark(0);
    launch_prologue(B, st);
    mark(1);
    launch_label(B, lc, st);
    mark(2);
    launch_merge(B, st);
    mark(3);
    launch_resolve(B, lc, st);
    mark(4);
    launch_scan(B, st);
    mark(5);
    launch_canon(B, lc, st);
    mark(6);
    launch_write(B, lc, st);
    mark(7);
}

// Event set for the next timed call of the given kind, or null.
static const cudaEvent_t *timing_slot(ccl_ctx *c, int kind) {
    if (c->timing_used >= c->timing.size()) return nullptr;
    c->timing_kind[c->timing_used] = kind;
    return c->timing[c->timing_used++].data();
}

static Shape shape_of(const ccl_ctx *c, const Plan &P) {
    Shape s;
    s.v.push_back(c->conn);
    s.v.push_back(P.th);
    s.v.push_back(P.tw);
    s.v.push_back(P.hsplit);
    for (const ImgDesc &d : P.d) {
        s.v.push_back(d.w);
        s.v.push_back(d.h);
        s.v.push_back(d.vec);
        s.v.push_back(d.fg != nullptr);
    }
    return s;
}

// Copy the plan's descriptors to the device through the next pinned staging
// slot, on the stream: the kernels that follow read them from d_desc.
static cudaError_t upload_plan(ccl_ctx *c, const Plan &P, cudaStream_t st) {
    const int k = c->ring_pos;
    c->ring_pos = (c->ring_pos + 1) % RING;
    cudaError_t e = cudaEventSynchronize(c->ring_ev[k]);   // this slot's last copy has run
    if (e != cudaSuccess) return e;
    ImgDesc *h = c->h_desc + (size_t)k * c->cap.images;
    memcpy(h, P.d.data(), sizeof(ImgDesc) * P.d.size());
    e = cudaMemcpyAsync(c->d_desc, h, sizeof(ImgDesc) * P.d.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    return cudaEventRecord(c->ring_ev[k], st);
}

// Upload the plan and enqueue the phases, replaying a cached CUDA graph of
// the kernels when the batch shape has been seen before.
static ccl_status run_plan(ccl_ctx *c, const Plan &P, cudaStream_t st, bool use_graph) {
    if (!c->cap.fits(P.need)) return CCL_ERR_CAPACITY;
    const Batch B = make_batch(c, P);
    cudaError_t e = upload_plan(c, P, st);
    if (e != cudaSuccess) return CCL_ERR_CUDA;
    const cudaEvent_t *ev = timing_slot(c, 0);
    if (ev) use_graph = false;
    if (use_graph) {
        const Shape key = shape_of(c, P);
        auto it = c->graphs.find(key);
        if (it == c->graphs.end()) {
            cudaStream_t cs;
            e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (e != cudaSuccess) return CCL_ERR_CUDA;
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                enqueue_analysis(B, cs);
                e = cudaStreamEndCapture(cs, &g);
            }
            cudaStreamDestroy(cs);
            if (e != cudaSuccess) return CCL_ERR_CUDA;
            Graph G;
            e = cudaGraphInstantiate(&G.exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return CCL_ERR_CUDA;
            it = c->graphs.emplace(key, G).first;
        }
        e = cudaGraphLaunch(it->second.exec, st);
    } else {
        enqueue_analysis(B, st, ev);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return CCL_ERR_CUDA;
    c->launches += ANALYSE_KERNELS;
    c->last = P;
    c->have_last = true;
    c->last_stream = st;
    return CCL_OK;
}

extern "C" {

int64_t ccl_node_capacity(int32_t w, int32_t h) {
    if (w <= 0 || h <= 0) return -1;
    return formula_capacity(w, h);
}

ccl_status ccl_create(ccl_ctx **out, int32_t w, int32_t h, int32_t pitch) {
    if (!out) return CCL_ERR_ARG;
    *out = nullptr;
    if (w <= 0 || h <= 0 || pitch < w || (int64_t)w * h >= ((int64_t)1 << 31)) return CCL_ERR_ARG;
    if (pitch % 16) return CCL_ERR_ALIGN;
    ccl_ctx *c = new ccl_ctx();
    c->w = w;
    c->h = h;
    c->pitch = pitch;
    // sized for the smallest tile (most tiles, segments and edge cells) so
    // that every tile shape can run; the widest tile has the most plane words
    const int64_t TX = (w + TW_MIN - 1) / TW_MIN, TY = (h + TH_MIN - 1) / TH_MIN;
    Limits L;
    L.images = 1;
    L.tiles = TX * TY;
    L.segs = (int64_t)h * TX;
    L.words = (int64_t)h * ((w + TW_MAX - 1) / TW_MAX) * WPR_MAX;
    L.pixels = (int64_t)w * h;
    L.edges = 2 * (int64_t)w * TY + 2 * (int64_t)h * TX;
    L.ncap = formula_capacity(w, h);
    ccl_status st = alloc_ctx(c, L);
    if (st != CCL_OK) {
        ccl_destroy(c);
        return st;
    }
    *out = c;
    return CCL_OK;
}

ccl_status ccl_set_connectivity(ccl_ctx *ctx, int32_t conn) {
    if (!ctx || (conn != CCL_CONN_8FG_4BG && conn != CCL_CONN_4FG_8BG)) return CCL_ERR_ARG;
    ctx->conn = conn;
    return CCL_OK;
}

ccl_status ccl_analyze(ccl_ctx *ctx, const uint8_t *d_img, int32_t *d_fg_labels, int32_t *d_bg_labels,
                       int32_t *d_tree_parent, int64_t *d_features, int32_t *d_counts, ccl_stream_t stream) {
    if (!ctx || ctx->batched) return CCL_ERR_ARG;
    ccl_image_desc x{};
    x.img = d_img;
    x.w = ctx->w;
    x.h = ctx->h;
    x.pitch = ctx->pitch;
    x.fg_labels = d_fg_labels;
    x.bg_labels = d_bg_labels;
    x.tree_parent = d_tree_parent;
    x.features = d_features;
    x.counts = d_counts;
    x.capacity = formula_capacity(ctx->w, ctx->h);
    Plan P;
    ccl_status st = build_plan(&x, 1, ctx->th, ctx->tw, ctx->hsplit, &P);
    if (st != CCL_OK) return st;
    return run_plan(ctx, P, (cudaStream_t)stream, ctx->graph_cache);
}

static ccl_status fill_last(ccl_ctx *ctx, int64_t T, int32_t target, cudaStream_t st) {
    const Plan &P = ctx->last;
    cudaError_t e = upload_plan(ctx, P, st);
    if (e != cudaSuccess) return CCL_ERR_CUDA;
    launch_fill(make_batch(ctx, P), T, target, LaunchCfg{g_sms}, st, timing_slot(ctx, 1));
    e = cudaGetLastError();
    ctx->launches += FILL_KERNELS;
    ctx->last_stream = st;
    return from_cuda(e);
}

ccl_status ccl_filter_components(ccl_ctx *ctx, int32_t target, int64_t area_threshold, int32_t *d_map,
                                 int64_t *d_features, int32_t *d_parent, ccl_stream_t stream) {
    if (!ctx || ctx->batched) return CCL_ERR_ARG;
    if (target != CCL_TARGET_HOLES && target != CCL_TARGET_OBJECTS) return CCL_ERR_ARG;
    if (!d_map || !d_features || !d_parent) return CCL_ERR_ARG;
    if (!ctx->have_last) return CCL_ERR_STATE;
    ImgDesc &d = ctx->last.d[0];
    d.fill_map = d_map;
    d.filled_feat = d_features;
    d.filled_parent = d_parent;
    return fill_last(ctx, area_threshold, target, (cudaStream_t)stream);
}

ccl_status ccl_fill_holes(ccl_ctx *ctx, int64_t area_threshold, int32_t *d_fill_map, int64_t *d_filled_features,
                          int32_t *d_filled_parent, ccl_stream_t stream) {
    return ccl_filter_components(ctx, CCL_TARGET_HOLES, area_threshold, d_fill_map, d_filled_features,
                                 d_filled_parent, stream);
}

ccl_status ccl_relabel_filtered(ccl_ctx *ctx, int32_t *d_fg_out, int32_t *d_bg_out, ccl_stream_t stream) {
    if (!ctx || ctx->batched || !d_fg_out || !d_bg_out) return CCL_ERR_ARG;
    if (!ctx->have_last || !ctx->last.d[0].fill_map || !ctx->last.d[0].fg) return CCL_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    Plan P = ctx->last;
    P.d[0].fg_out = d_fg_out;
    P.d[0].bg_out = d_bg_out;
    cudaError_t e = upload_plan(ctx, P, st);
    if (e != cudaSuccess) return CCL_ERR_CUDA;
    launch_relabel(make_batch(ctx, P), LaunchCfg{g_sms}, st);
    ctx->launches += 1;
    ctx->last_stream = st;
    return from_cuda(cudaGetLastError());
}

ccl_status ccl_relabel_filtered_batched(ccl_ctx *ctx, int32_t *const *d_fg_out, int32_t *const *d_bg_out,
                                        ccl_stream_t stream) {
    if (!ctx || !ctx->batched || !d_fg_out || !d_bg_out) return CCL_ERR_ARG;
    if (!ctx->have_last) return CCL_ERR_STATE;
    Plan P = ctx->last;
    for (size_t i = 0; i < P.d.size(); ++i) {
        ImgDesc &d = P.d[i];
        if ((d_fg_out[i] == nullptr) != (d_bg_out[i] == nullptr)) return CCL_ERR_ARG;
        if (d_fg_out[i] && (!d.fill_map || !d.fg)) return CCL_ERR_STATE;
        d.fg_out = d_fg_out[i];
        d.bg_out = d_bg_out[i];
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = upload_plan(ctx, P, st);
    if (e != cudaSuccess) return CCL_ERR_CUDA;
    launch_relabel(make_batch(ctx, P), LaunchCfg{g_sms}, st);
    ctx->launches += 1;
    ctx->last_stream = st;
    return from_cuda(cudaGetLastError());
}

ccl_status ccl_get_euler(ccl_ctx *ctx, int64_t *euler) {
    if (!ctx || !euler) return CCL_ERR_ARG;
    int32_t n = 0, nf = 0, nb = 0;
    const ccl_status st = ccl_get_counts(ctx, &n, &nf, &nb);
    if (st != CCL_OK && st != CCL_ERR_CAPACITY) return st;
    *euler = (int64_t)nf - ((int64_t)nb - 1);
    return st;
}

ccl_status ccl_get_counts(ccl_ctx *ctx, int32_t *n_nodes, int32_t *n_fg, int32_t *n_bg) {
    if (!ctx) return CCL_ERR_ARG;
    if (!ctx->have_last) return CCL_ERR_STATE;
    cudaError_t e = cudaStreamSynchronize(ctx->last_stream);
    if (e != cudaSuccess) return CCL_ERR_CUDA;
    int32_t cnt[4] = {0, 0, 0, 0};
    e = cudaMemcpy(cnt, ctx->last.d[0].counts, sizeof(cnt), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return CCL_ERR_CUDA;
    int32_t status = 0;
    e = cudaMemcpy(&status, ctx->s.status, sizeof(status), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return CCL_ERR_CUDA;
    if (n_nodes) *n_nodes = cnt[0];
    if (n_fg) *n_fg = cnt[1];
    if (n_bg) *n_bg = cnt[2];
    return (ccl_status)(status | cnt[3]);
}

ccl_status ccl_create_batched(ccl_ctx **out, int32_t max_images, int64_t max_total_pixels, int32_t max_side) {
    if (!out) return CCL_ERR_ARG;
    *out = nullptr;
    if (max_images <= 0 || max_total_pixels <= 0 || max_side <= 0) return CCL_ERR_ARG;
    ccl_ctx *c = new ccl_ctx();
    c->batched = true;
    ccl_status st = alloc_ctx(c, limits_of_bounds(max_images, max_total_pixels, max_side));
    if (st != CCL_OK) {
        ccl_destroy(c);
        return st;
    }
    *out = c;
    return CCL_OK;
}

ccl_status ccl_analyze_batched(ccl_ctx *ctx, const ccl_image_desc *host_descs, int32_t n, ccl_stream_t stream) {
    if (!ctx || !ctx->batched || !host_descs || n <= 0) return CCL_ERR_ARG;
    Plan P;
    ccl_status st = build_plan(host_descs, n, ctx->th, ctx->tw, ctx->hsplit, &P);
    if (st != CCL_OK) return st;
    return run_plan(ctx, P, (cudaStream_t)stream, ctx->graph_cache);
}

ccl_status ccl_analyze_batched_from_host(ccl_ctx *ctx, const ccl_image_desc *host_descs,
                                         const uint8_t *const *host_frames, const int64_t *host_pitches,
                                         int32_t n, ccl_stream_t stream) {
    if (!ctx || !ctx->batched || !host_descs || !host_frames || !host_pitches || n <= 0) return CCL_ERR_ARG;
    for (int32_t i = 0; i < n; ++i) {
        const ccl_image_desc &d = host_descs[i];
        if (!host_frames[i] || !d.img || d.w <= 0 || d.h <= 0 || host_pitches[i] < d.w) return CCL_ERR_ARG;
    }
    // the frames' copies first (the descriptors are checked again by the
    // plan below, before anything is enqueued from here on)
    Plan P;
    ccl_status st = build_plan(host_descs, n, ctx->th, ctx->tw, ctx->hsplit, &P);
    if (st != CCL_OK) return st;
    const cudaStream_t cs = (cudaStream_t)stream;
    for (int32_t i = 0; i < n; ++i) {
        const ccl_image_desc &d = host_descs[i];
        // rows laid out alike on both sides: one linear copy (up to the last
        // row's last pixel); else a 2-D copy of w bytes per row
        const cudaError_t e =
            host_pitches[i] == (int64_t)d.pitch
                ? cudaMemcpyAsync((void *)d.img, host_frames[i], (size_t)(d.h - 1) * (size_t)d.pitch + (size_t)d.w,
                                  cudaMemcpyHostToDevice, cs)
                : cudaMemcpy2DAsync((void *)d.img, (size_t)d.pitch, host_frames[i], (size_t)host_pitches[i],
                                    (size_t)d.w, (size_t)d.h, cudaMemcpyHostToDevice, cs);
        if (e != cudaSuccess) return CCL_ERR_CUDA;
    }
    return run_plan(ctx, P, cs, ctx->graph_cache);
}

ccl_status ccl_filter_components_batched(ccl_ctx *ctx, int32_t target, int64_t area_threshold,
                                         ccl_stream_t stream) {
    if (!ctx || !ctx->batched) return CCL_ERR_ARG;
    if (target != CCL_TARGET_HOLES && target != CCL_TARGET_OBJECTS) return CCL_ERR_ARG;
    if (!ctx->have_last) return CCL_ERR_STATE;
    return fill_last(ctx, area_threshold, target, (cudaStream_t)stream);
}

ccl_status ccl_fill_holes_batched(ccl_ctx *ctx, int64_t area_threshold, ccl_stream_t stream) {
    return ccl_filter_components_batched(ctx, CCL_TARGET_HOLES, area_threshold, stream);
}

ccl_status ccl_set_tile_rows(ccl_ctx *ctx, int32_t rows) {
    if (!ctx || (rows != 16 && rows != 32)) return CCL_ERR_ARG;
    ctx->th = rows;
    return CCL_OK;
}

ccl_status ccl_set_tile_cols(ccl_ctx *ctx, int32_t cols) {
    if (!ctx || (cols != TW_MIN && cols != TW_MAX)) return CCL_ERR_ARG;
    ctx->tw = cols;
    return CCL_OK;
}

ccl_status ccl_set_merge_split(ccl_ctx *ctx, int32_t items_per_word) {
    if (!ctx || (items_per_word != 1 && items_per_word != 2 && items_per_word != 4 && items_per_word != 8))
        return CCL_ERR_ARG;
    ctx->hsplit = items_per_word;
    return CCL_OK;
}

ccl_status ccl_set_graph_cache(ccl_ctx *ctx, int32_t enable) {
    if (!ctx) return CCL_ERR_ARG;
    ctx->graph_cache = enable != 0;
    return CCL_OK;
}

static void free_timing(ccl_ctx *ctx) {
    for (auto &set : ctx->timing)
        for (cudaEvent_t e : set)
            if (e) cudaEventDestroy(e);
    ctx->timing.clear();
    ctx->timing_kind.clear();
    ctx->timing_used = 0;
}

ccl_status ccl_enable_phase_timing(ccl_ctx *ctx, int32_t max_calls) {
    if (!ctx || max_calls < 0) return CCL_ERR_ARG;
    if (ctx->have_last) cudaStreamSynchronize(ctx->last_stream);
    free_timing(ctx);
    ctx->timing.assign(max_calls, std::vector<cudaEvent_t>(ANALYSE_PHASES + 1, nullptr));
    ctx->timing_kind.assign(max_calls, 0);
    for (auto &set : ctx->timing)
        for (cudaEvent_t &e : set)
            if (cudaEventCreate(&e) != cudaSuccess) {
                free_timing(ctx);
                return CCL_ERR_CUDA;
            }
    return CCL_OK;
}

ccl_status ccl_read_phase_timing(ccl_ctx *ctx, double *total_ms, int64_t *count) {
    if (!ctx || !total_ms || !count) return CCL_ERR_ARG;
    for (int k = 0; k < CCL_PHASE_COUNT; ++k) {
        total_ms[k] = 0.0;
        count[k] = 0;
    }
    for (size_t i = 0; i < ctx->timing_used; ++i) {
        const std::vector<cudaEvent_t> &ev = ctx->timing[i];
        if (cudaEventSynchronize(ev[ctx->timing_kind[i] == 0 ? ANALYSE_PHASES : 2]) != cudaSuccess)
            return CCL_ERR_CUDA;
        if (ctx->timing_kind[i] == 0) {
            for (int k = 0; k < ANALYSE_PHASES; ++k) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) != cudaSuccess) return CCL_ERR_CUDA;
                total_ms[k] += ms;
                count[k] += 1;
            }
        } else {
            for (int k = 0; k < 2; ++k) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) != cudaSuccess) return CCL_ERR_CUDA;
                total_ms[CCL_PHASE_FILL_MAP + k] += ms;
                count[CCL_PHASE_FILL_MAP + k] += 1;
            }
        }
    }
    ctx->timing_used = 0;
    return CCL_OK;
}

ccl_status ccl_get_launch_count(ccl_ctx *ctx, int64_t *launches) {
    if (!ctx || !launches) return CCL_ERR_ARG;
    *launches = ctx->launches;
    return CCL_OK;
}

const char *ccl_status_string(ccl_status s) {
    switch ((int)s) {
        case CCL_OK: return "ok";
        case CCL_ERR_ARG: return "invalid argument";
        case CCL_ERR_ALIGN: return "image pointer or pitch not 16-byte aligned";
        case CCL_ERR_CAPACITY: return "capacity exceeded";
        case CCL_ERR_OOM: return "device allocation failed";
        case CCL_ERR_CUDA: return "CUDA error or no usable device";
        case CCL_ERR_ITER_LIMIT: return "device iteration limit reached";
        case CCL_ERR_STATE: return "call out of order";
        default: return "several errors";
    }
}

void ccl_destroy(ccl_ctx *ctx) {
    if (!ctx) return;
    if (ctx->last_stream || ctx->have_last) cudaStreamSynchronize(ctx->last_stream);
    free_timing(ctx);
    for (auto &kv : ctx->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    for (int k = 0; k < RING; ++k)
        if (ctx->ring_ev[k]) cudaEventDestroy(ctx->ring_ev[k]);
    if (ctx->h_desc) cudaFreeHost(ctx->h_desc);
    if (ctx->scratch) cudaFree(ctx->scratch);
    delete ctx;
}

}  // extern "C"
