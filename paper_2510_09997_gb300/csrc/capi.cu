// capi.cu -- extern "C" entry points of libclod (see include/clod.h).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "clod_internal.cuh"

namespace clod {

void launch_frame_setup(const Frame& F, void* ws, const FrameHeader& h, const ViewDev* views, size_t zero_begin,
                        size_t zero_end, int n_sm, cudaStream_t st);
void launch_preprocess(const Frame& F, const clod_scene& S, uint32_t V, uint8_t* mask_out, float* alpha_out,
                       unsigned long long* n_pairs_out, int n_sm, cudaStream_t st, bool select);
cudaError_t launch_bin_sort(const Frame& F, const FrameLayout& L, unsigned long long cap, uint64_t* keys,
                            uint32_t* vals, uint32_t* ranges, cudaStream_t st);
void launch_blend_fwd(const Frame& F, const uint32_t* vals, const uint32_t* ranges, float* image, float* Tout,
                      uint32_t* ncout, unsigned long long* evaluated, int n_sm, cudaStream_t st, bool fast, uint32_t tiles);
cudaError_t bin_sort_setup();
cudaError_t render_setup();
cudaError_t backward_setup();
void launch_backward(const Frame& F, const clod_scene& S, uint32_t V, const uint32_t* vals, const uint32_t* ranges,
                     const float* Tfin, const uint32_t* ncon, const float* dimg, const float* g_alpha_ext,
                     const float* g_alpha_view, void* bwd_ws, float* dmeans, float* dscales, float* dquats, float* dopacity, float* dsh,
                     float* ddecay, int n_sm, cudaStream_t st, bool fast, bool set);
size_t backward_ws_bytes(uint64_t n, uint32_t V);
void launch_l1(const float* img, const float* tgt, int64_t count, float scale, float* loss, float* grad, int n_sm,
               cudaStream_t st);

static thread_local std::string g_err;

clod_status fail(clod_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

clod_status cuda_fail(cudaError_t e, const char* what)
{
    return fail(CLOD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

FrameLayout frame_layout(uint64_t n, uint32_t V, uint32_t TT, uint32_t n_chunks, uint32_t rb_total, uint32_t max_tx,
                         size_t diff_grid_max)
{
    FrameLayout L{};
    L.diff_grid_max = diff_grid_max;
    L.n_chunks = n_chunks;
    L.n_rs_blocks = (uint32_t)((n + RS_ITEMS - 1) / RS_ITEMS);
    L.rb_total = rb_total;
    L.max_tx = max_tx;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    // zero-initialised block first: header, d_max keys, counts, tile counts,
    // the radix passes' digit sums (4 passes of digit totals and of the two
    // levels of group sums, added by the counting kernels' atomics) and the
    // tile scan's look-back words, class counters and ticket
    const int nbk = (int)L.n_rs_blocks;
    L.header = take(sizeof(FrameHeader));
    L.dmax_key = take(sizeof(unsigned long long) * V);
    L.n_surv = take(sizeof(uint32_t) * 2 * V);
    L.tile_count = take(sizeof(uint32_t) * (size_t)TT);
    L.rs_sums = take(sizeof(uint32_t) * 256 * (size_t)V *
                     (4 * (1 + (size_t)rs_groups(nbk, RS_G1) + (size_t)rs_groups(nbk, RS_G2))));
    L.scan = take(sizeof(unsigned long long) * (((size_t)TT + 31) / 32) + sizeof(uint32_t) * 8);
    L.views = take(sizeof(ViewDev) * V);
    L.tile_offset = take(sizeof(uint32_t) * ((size_t)TT + 1));
    L.torder = take(sizeof(uint32_t) * 4 * (size_t)TT);
    const size_t vn = (size_t)V * n;
    L.rec0 = take(sizeof(float4) * vn);
    L.rec1 = take(sizeof(float4) * vn);
    L.rec2 = take(sizeof(float4) * vn);
    L.depth = take(sizeof(float) * vn);
    L.rect = take(sizeof(uint2) * vn);
    L.key0 = take(sizeof(uint32_t) * vn);
    L.val0 = take(sizeof(uint32_t) * vn);
    L.key1 = take(sizeof(uint32_t) * vn);
    L.val1 = take(sizeof(uint32_t) * vn);
    L.srect = take(sizeof(uint2) * vn);
    L.sband = take(sizeof(uint16_t) * vn);
    // per radix block its digit counts (plain stores: no clear needed)
    L.rs_hist = take(sizeof(uint32_t) * 256 * (size_t)V * (size_t)nbk);
    L.scan_cls = take(sizeof(ulonglong2) * 2 * (((size_t)TT + 31) / 32));
    L.cnt = take(sizeof(uint32_t) * (size_t)L.n_chunks * TT);
    L.sel = take(sizeof(SelState) * V);
    L.sel_hist = take(sizeof(uint32_t) * SEL_BINS * (size_t)V);
    L.total = o;
    L.total_tiles = TT;
    L.n_views = V;
    L.n = n;
    return L;
}

Frame frame_ptrs(void* ws, const FrameLayout& L)
{
    char* b = static_cast<char*>(ws);
    Frame F;
    F.hdr = reinterpret_cast<FrameHeader*>(b + L.header);
    F.views = reinterpret_cast<ViewDev*>(b + L.views);
    F.dmax_key = reinterpret_cast<unsigned long long*>(b + L.dmax_key);
    F.n_surv = reinterpret_cast<uint32_t*>(b + L.n_surv);
    F.rec0 = reinterpret_cast<float4*>(b + L.rec0);
    F.rec1 = reinterpret_cast<float4*>(b + L.rec1);
    F.rec2 = reinterpret_cast<float4*>(b + L.rec2);
    F.depth = reinterpret_cast<float*>(b + L.depth);
    F.rect = reinterpret_cast<uint2*>(b + L.rect);
    F.tile_count = reinterpret_cast<uint32_t*>(b + L.tile_count);
    F.tile_offset = reinterpret_cast<uint32_t*>(b + L.tile_offset);
    F.torder = reinterpret_cast<uint32_t*>(b + L.torder);
    F.key0 = reinterpret_cast<uint32_t*>(b + L.key0);
    F.val0 = reinterpret_cast<uint32_t*>(b + L.val0);
    F.key1 = reinterpret_cast<uint32_t*>(b + L.key1);
    F.val1 = reinterpret_cast<uint32_t*>(b + L.val1);
    F.srect = reinterpret_cast<uint2*>(b + L.srect);
    F.sband = reinterpret_cast<uint16_t*>(b + L.sband);
    F.rs_hist = reinterpret_cast<uint32_t*>(b + L.rs_hist);
    F.rs_sums = reinterpret_cast<uint32_t*>(b + L.rs_sums);
    F.scan_st = reinterpret_cast<unsigned long long*>(b + L.scan);
    F.scan_cls = reinterpret_cast<ulonglong2*>(b + L.scan_cls);
    F.scan_ctr = reinterpret_cast<uint32_t*>(b + L.scan + sizeof(unsigned long long) * (((size_t)L.total_tiles + 31) / 32));
    F.cnt = reinterpret_cast<uint32_t*>(b + L.cnt);
    F.sel = reinterpret_cast<SelState*>(b + L.sel);
    F.sel_hist = reinterpret_cast<uint32_t*>(b + L.sel_hist);
    return F;
}

// ---------------------------------------------------------------------------
struct DeviceInfo {
    int n_sm = 0;
    bool ready = false;
};
static std::mutex g_dev_mu;
static DeviceInfo g_dev[64];

clod_status device_ready(int* n_sm)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(CLOD_ERR_CUDA, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DeviceInfo& D = g_dev[dev];
    if (!D.ready) {
        int major = 0, minor = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        if (major != 10 || minor != 3)
            return fail(CLOD_ERR_CUDA, "libclod is built for sm_103a; device %d is sm_%d%d", dev, major, minor);
        e = cudaDeviceGetAttribute(&D.n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        if ((e = bin_sort_setup()) != cudaSuccess) return cuda_fail(e, "bin_sort_setup");
        if ((e = render_setup()) != cudaSuccess) return cuda_fail(e, "render_setup");
        if ((e = backward_setup()) != cudaSuccess) return cuda_fail(e, "backward_setup");
        D.ready = true;
    }
    *n_sm = D.n_sm;
    return CLOD_OK;
}

struct ViewGeom {
    uint32_t TT, n_chunks, rb_total, max_tx;
    size_t diff_max;
};

clod_status check_view(const clod_view& w, int v)
{
    if (w.width < 1 || w.height < 1 || w.width > 16384 || w.height > 16384)
        return fail(CLOD_ERR_ARG, "view %d: size %dx%d outside [1, 16384]", v, w.width, w.height);
    if (!(w.fx > 0.0f) || !(w.fy > 0.0f)) return fail(CLOD_ERR_ARG, "view %d: focal lengths must be > 0", v);
    if (!std::isfinite(w.s_v) || !std::isfinite(w.tau) || !(w.eps >= 0.0f))
        return fail(CLOD_ERR_ARG, "view %d: s_v, tau must be finite and eps >= 0", v);
    if (w.full_width < 0) return fail(CLOD_ERR_ARG, "view %d: full_width < 0", v);
    if (w.full_width > 0) {
        if (w.full_width > 16384 || w.full_height < 1 || w.full_height > 16384)
            return fail(CLOD_ERR_ARG, "view %d: full frame %dx%d outside [1, 16384]", v, w.full_width, w.full_height);
        if (w.region_x < 0 || w.region_y < 0 || w.region_x % TILE || w.region_y % TILE)
            return fail(CLOD_ERR_ARG, "view %d: region origin (%d, %d) must be non-negative multiples of %d", v,
                        w.region_x, w.region_y, TILE);
        if ((int64_t)w.region_x + w.width > w.full_width || (int64_t)w.region_y + w.height > w.full_height)
            return fail(CLOD_ERR_ARG, "view %d: region %dx%d at (%d, %d) leaves the %dx%d frame", v, w.width,
                        w.height, w.region_x, w.region_y, w.full_width, w.full_height);
    }
    return CLOD_OK;
}

void view_record(const clod_view& w, ViewDev& d)
{
    std::memset(&d, 0, sizeof(d));
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) d.R[3 * r + c] = w.viewmat[4 * r + c];
        d.t[r] = w.viewmat[4 * r + 3];
        d.c[r] = w.campos[r];
        d.bg[r] = w.bg[r];
    }
    d.fx = w.fx;
    d.fy = w.fy;
    d.cx = w.cx;
    d.cy = w.cy;
    d.near_z = w.near_z;
    d.s_v = w.s_v;
    d.tau = w.tau;
    d.eps = w.eps;
    d.W = w.width;
    d.H = w.height;
    d.TX = (w.width + TILE - 1) / TILE;
    d.TY = (w.height + TILE - 1) / TILE;
    if (w.full_width > 0) {
        d.ox = w.region_x;
        d.oy = w.region_y;
        d.FW = w.full_width;
        d.FH = w.full_height;
    } else {
        d.FW = w.width;
        d.FH = w.height;
    }
    d.flags = w.flags;
    d.budget = w.budget;
}

static clod_status check_views(const clod_view* views, int32_t V, uint64_t n, ViewGeom* G)
{
    if (!views) return fail(CLOD_ERR_ARG, "views is NULL");
    if (V < 1 || V > MAX_VIEWS) return fail(CLOD_ERR_ARG, "n_views = %d outside [1, %d]", V, MAX_VIEWS);
    uint64_t tt = 0, px = 0;
    for (int v = 0; v < V; ++v) {
        const clod_view& w = views[v];
        clod_status s = check_view(w, v);
        if (s) return s;
        tt += (uint64_t)((w.width + TILE - 1) / TILE) * ((w.height + TILE - 1) / TILE);
        px += (uint64_t)w.width * w.height;
    }
    if (tt > 0x0FFFFFFFull) return fail(CLOD_ERR_ARG, "too many tiles (%llu)", (unsigned long long)tt);
    for (int v = 1; v < V; ++v)
        if ((views[v].flags ^ views[0].flags) & CLOD_FAST_EXP)
            return fail(CLOD_ERR_ARG, "views 0 and %d disagree on CLOD_FAST_EXP (one frame, one exponential)", v);
    G->TT = static_cast<uint32_t>(tt);
    uint64_t bands = 0;
    uint32_t mtx = 1;
    size_t dmx = 0;
    for (int v = 0; v < V; ++v) {
        const int TX = (views[v].width + TILE - 1) / TILE, TY = (views[v].height + TILE - 1) / TILE;
        bands += (uint64_t)((TY + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
        mtx = std::max<uint32_t>(mtx, (uint32_t)TX);
        dmx = std::max<size_t>(dmx, (size_t)(TX + 1) * (TY + 1));
    }
    const uint32_t CH = chunk_count(n, tt);
    const uint64_t rb = (uint64_t)CH * bands;
    G->diff_max = dmx;
    if (rb > 0x7FFFFFFFull) return fail(CLOD_ERR_ARG, "frame too large");
    G->n_chunks = CH;
    G->rb_total = (uint32_t)rb;
    G->max_tx = mtx;
    return CLOD_OK;
}

static void make_view_table(const clod_view* views, int32_t V, uint32_t CH, std::vector<ViewDev>& out)
{
    out.resize(V);
    uint32_t tile_base = 0, rb_base = 0;
    uint64_t pix_base = 0;
    for (int v = 0; v < V; ++v) {
        const clod_view& w = views[v];
        ViewDev& d = out[v];
        view_record(w, d);
        d.tile_base = tile_base;
        d.pix_base = pix_base;
        d.rb_base = rb_base;
        tile_base += (uint32_t)(d.TX * d.TY);
        pix_base += (uint64_t)w.width * w.height;
        rb_base += CH * (uint32_t)((d.TY + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
    }
}

static clod_status check_scene(const clod_scene* S)
{
    if (!S) return fail(CLOD_ERR_ARG, "scene is NULL");
    if (S->n < 0 || S->n >= (1ll << 31)) return fail(CLOD_ERR_ARG, "scene n = %lld outside [0, 2^31)", (long long)S->n);
    if (S->sh_degree < 0 || S->sh_degree > 3) return fail(CLOD_ERR_ARG, "sh_degree %d outside [0, 3]", S->sh_degree);
    if (S->n > 0 && (!S->means || !S->scales || !S->quats || !S->opacity || !S->sh || !S->decay))
        return fail(CLOD_ERR_ARG, "scene array pointer is NULL");
    if (reinterpret_cast<uintptr_t>(S->quats) % 16) return fail(CLOD_ERR_ARG, "quats must be 16-byte aligned");
    if (S->sh_degree == 3 && reinterpret_cast<uintptr_t>(S->sh) % 16)
        return fail(CLOD_ERR_ARG, "sh must be 16-byte aligned for degree 3");
    return CLOD_OK;
}

// Host-side cache of the last layout per workspace pointer: lets the later
// pipeline calls size their launches without reading the device header.
struct WsMeta {
    const void* ws;
    FrameLayout L;
};
static std::mutex g_ws_mu;
static std::vector<WsMeta> g_ws;

static void remember(const void* ws, const FrameLayout& L)
{
    std::lock_guard<std::mutex> lk(g_ws_mu);
    for (auto& m : g_ws)
        if (m.ws == ws) {
            m.L = L;
            return;
        }
    if (g_ws.size() > 256) g_ws.erase(g_ws.begin());
    g_ws.push_back({ws, L});
}

static bool recall(const void* ws, FrameLayout* L)
{
    std::lock_guard<std::mutex> lk(g_ws_mu);
    for (auto& m : g_ws)
        if (m.ws == ws) {
            *L = m.L;
            return true;
        }
    return false;
}

}  // namespace clod

using namespace clod;

extern "C" {

const char* clod_last_error(void) { return g_err.c_str(); }

const char* clod_version(void) { return "libclod 0.1 (sm_103a)"; }

clod_status clod_frame_workspace_size(int64_t n, const clod_view* views, int32_t n_views, size_t* bytes,
                                      clod_frame_layout* layout)
{
    if (!bytes) return fail(CLOD_ERR_ARG, "bytes is NULL");
    if (n < 0 || n >= (1ll << 31)) return fail(CLOD_ERR_ARG, "n = %lld outside [0, 2^31)", (long long)n);
    ViewGeom G;
    clod_status s = check_views(views, n_views, (uint64_t)n, &G);
    if (s) return s;
    const uint32_t TT = G.TT;
    const FrameLayout L = frame_layout((uint64_t)n, (uint32_t)n_views, TT, G.n_chunks, G.rb_total, G.max_tx, G.diff_max);
    *bytes = L.total;
    if (layout) {
        layout->total_bytes = L.total;
        layout->views = L.views;
        layout->dmax_key = L.dmax_key;
        layout->n_survivors = L.n_surv;
        layout->rec0 = L.rec0;
        layout->rec1 = L.rec1;
        layout->rec2 = L.rec2;
        layout->depth = L.depth;
        layout->rect = L.rect;
        layout->tile_count = L.tile_count;
        layout->tile_offset = L.tile_offset;
        layout->total_tiles = TT;
        layout->n_views = (uint32_t)n_views;
    }
    return CLOD_OK;
}

clod_status clod_preprocess(const clod_scene* scene, const clod_view* views, int32_t n_views, void* ws,
                            size_t ws_bytes, uint8_t* mask_out, float* alpha_eff_out, uint32_t* counts_out,
                            uint64_t* n_pairs_out, clod_stream stream)
{
    clod_status s = check_scene(scene);
    if (s) return s;
    ViewGeom G;
    if ((s = check_views(views, n_views, (uint64_t)scene->n, &G))) return s;
    const uint32_t TT = G.TT;
    if (!ws) return fail(CLOD_ERR_ARG, "ws is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(CLOD_ERR_ARG, "ws must be 256-byte aligned");
    FrameLayout L = frame_layout((uint64_t)scene->n, (uint32_t)n_views, TT, G.n_chunks, G.rb_total, G.max_tx, G.diff_max);
    L.fast_exp = (views[0].flags & CLOD_FAST_EXP) ? 1u : 0u;
    if (ws_bytes < L.total)
        return fail(CLOD_ERR_CAPACITY, "frame workspace needs %zu bytes, got %zu", L.total, ws_bytes);
    int n_sm = 0;
    if ((s = device_ready(&n_sm))) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Frame F = frame_ptrs(ws, L);
    std::vector<ViewDev> table;
    make_view_table(views, n_views, G.n_chunks, table);
    FrameHeader h{};
    h.n = (uint64_t)scene->n;
    h.n_views = (uint32_t)n_views;
    h.total_tiles = TT;
    h.n_chunks = L.n_chunks;
    h.n_rs_blocks = L.n_rs_blocks;
    h.max_tx = L.max_tx;
    h.rb_total = L.rb_total;
    // header and view table as kernel parameters; the block after the header cleared
    launch_frame_setup(F, ws, h, table.data(), L.dmax_key, L.views, n_sm, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "clod_preprocess set-up");
    bool select = false;
    for (int v = 0; v < n_views; ++v) select = select || views[v].budget > 0;
    launch_preprocess(F, *scene, (uint32_t)n_views, mask_out, alpha_eff_out,
                      reinterpret_cast<unsigned long long*>(n_pairs_out), n_sm, st, select);
    if (counts_out) {
        e = cudaMemcpyAsync(counts_out, F.n_surv, sizeof(uint32_t) * 2 * n_views, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "clod_preprocess counts");
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "clod_preprocess launch");
    remember(ws, L);
    return CLOD_OK;
}

clod_status clod_bin_sort(void* ws, uint64_t pair_capacity, uint64_t* keys_out, uint32_t* vals_out,
                          uint32_t* ranges_out, clod_stream stream)
{
    if (!ws || !ranges_out) return fail(CLOD_ERR_ARG, "NULL argument to clod_bin_sort");
    if (pair_capacity > 0 && !vals_out) return fail(CLOD_ERR_ARG, "vals_out is NULL");
    if (pair_capacity > 0xFFFFFFFFull) return fail(CLOD_ERR_ARG, "pair_capacity above 2^32 - 1");
    FrameLayout L;
    if (!recall(ws, &L)) return fail(CLOD_ERR_ARG, "ws was not prepared by clod_preprocess");
    int n_sm = 0;
    clod_status s = device_ready(&n_sm);
    if (s) return s;
    const Frame F = frame_ptrs(ws, L);
    cudaError_t e = launch_bin_sort(F, L, pair_capacity, keys_out, vals_out, ranges_out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "clod_bin_sort launch");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "clod_bin_sort launch");
    return CLOD_OK;
}

static clod_status render_common(const void* ws, const uint32_t* vals, const uint32_t* ranges, float* image,
                                 float* T_final, uint32_t* n_contrib, unsigned long long* evaluated, clod_stream stream)
{
    if (!ws || !ranges || !image) return fail(CLOD_ERR_ARG, "NULL argument to clod_render_fwd");
    FrameLayout L;
    if (!recall(ws, &L)) return fail(CLOD_ERR_ARG, "ws was not prepared by clod_preprocess");
    int n_sm = 0;
    clod_status s = device_ready(&n_sm);
    if (s) return s;
    const Frame F = frame_ptrs(const_cast<void*>(ws), L);
    launch_blend_fwd(F, vals, ranges, image, T_final, n_contrib, evaluated, n_sm, static_cast<cudaStream_t>(stream),
                     L.fast_exp != 0, L.total_tiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "clod_render_fwd launch");
    return CLOD_OK;
}

clod_status clod_render_fwd(const void* ws, const uint32_t* vals, const uint32_t* ranges, float* image, float* T_final,
                            uint32_t* n_contrib, clod_stream stream)
{
    return render_common(ws, vals, ranges, image, T_final, n_contrib, nullptr, stream);
}

clod_status clod_render_fwd_count(const void* ws, const uint32_t* vals, const uint32_t* ranges, float* image,
                                  float* T_final, uint32_t* n_contrib, unsigned long long* evaluated,
                                  clod_stream stream)
{
    if (!evaluated) return fail(CLOD_ERR_ARG, "evaluated is NULL");
    return render_common(ws, vals, ranges, image, T_final, n_contrib, evaluated, stream);
}

clod_status clod_frame_check(const void* ws, uint64_t pair_capacity, uint64_t* n_pairs, clod_stream stream)
{
    if (!ws) return fail(CLOD_ERR_ARG, "ws is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "clod_frame_check sync");
    FrameHeader h;
    e = cudaMemcpy(&h, ws, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "clod_frame_check read");
    if (n_pairs) *n_pairs = h.n_pairs;
    if (h.status & STATUS_TIMEOUT) return fail(CLOD_ERR_TIMEOUT, "a device wait gave up");
    if ((h.status & STATUS_OVERFLOW) || h.n_pairs > pair_capacity)
        return fail(CLOD_ERR_CAPACITY, "frame needs %llu pairs, capacity %llu", (unsigned long long)h.n_pairs,
                    (unsigned long long)pair_capacity);
    return CLOD_OK;
}

clod_status clod_backward_workspace_size(int64_t n, int32_t n_views, size_t* bytes)
{
    if (!bytes) return fail(CLOD_ERR_ARG, "bytes is NULL");
    if (n < 0 || n >= (1ll << 31)) return fail(CLOD_ERR_ARG, "n = %lld outside [0, 2^31)", (long long)n);
    if (n_views < 1 || n_views > MAX_VIEWS) return fail(CLOD_ERR_ARG, "n_views = %d outside [1, %d]", n_views, MAX_VIEWS);
    *bytes = backward_ws_bytes((uint64_t)n, (uint32_t)n_views);
    return CLOD_OK;
}

static clod_status render_bwd(const clod_scene* scene, const void* ws, const uint32_t* vals, const uint32_t* ranges,
                              const float* T_final, const uint32_t* n_contrib, const float* dL_dimage,
                              const float* dL_dalpha_eff, const float* dL_dalpha_view, void* bwd_ws,
                              size_t bwd_ws_bytes, float* dmeans,
                              float* dscales, float* dquats, float* dopacity, float* dsh, float* ddecay,
                              clod_stream stream, bool set)
{
    clod_status s = check_scene(scene);
    if (s) return s;
    if (!ws || !ranges || !T_final || !n_contrib || !dL_dimage || !bwd_ws)
        return fail(CLOD_ERR_ARG, "NULL argument to clod_render_bwd");
    if (scene->n > 0 && (!dmeans || !dscales || !dquats || !dopacity || !dsh || !ddecay))
        return fail(CLOD_ERR_ARG, "NULL gradient output");
    FrameLayout L;
    if (!recall(ws, &L)) return fail(CLOD_ERR_ARG, "ws was not prepared by clod_preprocess");
    if (L.n != (uint64_t)scene->n) return fail(CLOD_ERR_ARG, "scene has %lld Gaussians, the frame %llu",
                                               (long long)scene->n, (unsigned long long)L.n);
    const size_t need = backward_ws_bytes(L.n, L.n_views);
    if (bwd_ws_bytes < need) return fail(CLOD_ERR_CAPACITY, "backward workspace needs %zu bytes, got %zu", need, bwd_ws_bytes);
    if (reinterpret_cast<uintptr_t>(bwd_ws) % 256) return fail(CLOD_ERR_ARG, "bwd_ws must be 256-byte aligned");
    int n_sm = 0;
    if ((s = device_ready(&n_sm))) return s;
    const Frame F = frame_ptrs(const_cast<void*>(ws), L);
    launch_backward(F, *scene, L.n_views, vals, ranges, T_final, n_contrib, dL_dimage, dL_dalpha_eff, dL_dalpha_view,
                    bwd_ws, dmeans,
                    dscales, dquats, dopacity, dsh, ddecay, n_sm, static_cast<cudaStream_t>(stream), L.fast_exp != 0,
                    set);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "clod_render_bwd launch");
    return CLOD_OK;
}

clod_status clod_render_bwd(const clod_scene* scene, const void* ws, const uint32_t* vals, const uint32_t* ranges,
                            const float* T_final, const uint32_t* n_contrib, const float* dL_dimage,
                            const float* dL_dalpha_eff, const float* dL_dalpha_view, void* bwd_ws,
                            size_t bwd_ws_bytes, float* dmeans,
                            float* dscales, float* dquats, float* dopacity, float* dsh, float* ddecay,
                            clod_stream stream)
{
    return render_bwd(scene, ws, vals, ranges, T_final, n_contrib, dL_dimage, dL_dalpha_eff, dL_dalpha_view, bwd_ws,
                      bwd_ws_bytes, dmeans, dscales, dquats, dopacity, dsh, ddecay, stream, false);
}

clod_status clod_render_bwd_set(const clod_scene* scene, const void* ws, const uint32_t* vals,
                                const uint32_t* ranges, const float* T_final, const uint32_t* n_contrib,
                                const float* dL_dimage, const float* dL_dalpha_eff, const float* dL_dalpha_view,
                                void* bwd_ws, size_t bwd_ws_bytes, float* dmeans,
                                float* dscales, float* dquats, float* dopacity, float* dsh, float* ddecay,
                                clod_stream stream)
{
    return render_bwd(scene, ws, vals, ranges, T_final, n_contrib, dL_dimage, dL_dalpha_eff, dL_dalpha_view, bwd_ws,
                      bwd_ws_bytes, dmeans, dscales, dquats, dopacity, dsh, ddecay, stream, true);
}

clod_status clod_l1_loss(const float* image, const float* target, int64_t count, float scale, float* loss,
                         float* dL_dimage, clod_stream stream)
{
    if (!image || !target || count < 1) return fail(CLOD_ERR_ARG, "bad argument to clod_l1_loss");
    int n_sm = 0;
    clod_status s = device_ready(&n_sm);
    if (s) return s;
    launch_l1(image, target, count, scale, loss, dL_dimage, n_sm, static_cast<cudaStream_t>(stream));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "clod_l1_loss launch");
    return CLOD_OK;
}

}  // extern "C"
