// server.cu -- continuous-batching render server over a resident scene.
//
// Requests (a view and a caller device buffer for its image) enter a queue.
// A worker thread admits them, in arrival order, into batches of at most
// max_views_per_batch views and max_pixels_per_batch pixels, and launches each
// batch on a free slot: every slot owns a stream, a frame workspace sized for
// the largest admissible batch, a pair buffer and pinned staging for the view
// table and the status read-back.  Batches on different slots overlap on the
// device; requests that arrive while batches run are admitted as soon as a
// slot frees.  One batch is one launch sequence over all its views: the
// scene is read once for the batch (preprocessing loops over the views), the
// sort and the blend run over every view's tiles in one grid each, and the
// blend writes straight into each request's buffer.
//
// With use_graphs, each slot captures its launch sequence once, sized for the
// largest batch; the kernels take the batch's actual sizes from the frame
// header uploaded by the graph's first node, so the one graph replays for
// every batch shape.  A batch whose pairs exceed the slot's capacity is
// split: its requests are re-run alone by a second thread with a stream,
// workspace and pair buffer of its own (the buffer grows, stream-ordered, to
// the largest pair count met), so the re-runs overlap the batches that the
// worker keeps admitting.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "clod_internal.cuh"

namespace clod {

void launch_preprocess(const Frame& F, const clod_scene& S, uint32_t V, uint8_t* mask_out, float* alpha_out,
                       unsigned long long* n_pairs_out, int n_sm, cudaStream_t st, bool select);
cudaError_t launch_bin_sort(const Frame& F, const FrameLayout& L, unsigned long long cap, uint64_t* keys,
                            uint32_t* vals, uint32_t* ranges, cudaStream_t st);
void launch_blend_fwd(const Frame& F, const uint32_t* vals, const uint32_t* ranges, float* image, float* Tout,
                      uint32_t* ncout, unsigned long long* evaluated, int n_sm, cudaStream_t st, bool fast, uint32_t tiles);
clod_status fail(clod_status s, const char* fmt, ...);
clod_status cuda_fail(cudaError_t e, const char* what);
clod_status device_ready(int* n_sm);

static double now_us()
{
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}


struct Request {
    clod_view view;
    float* out = nullptr;
    double t_submit = 0, t_launch = 0, t_done = 0;
    int32_t status = CLOD_OK;
    int32_t batch = 0;
    uint32_t rendered = 0;
    uint64_t pairs = 0;
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    void* ws = nullptr;
    FrameLayout L{};
    uint32_t* vals = nullptr;
    uint32_t* ranges = nullptr;
    ViewDev* h_views = nullptr;      // pinned staging
    FrameHeader* h_hdr_up = nullptr; // pinned staging
    FrameHeader* h_hdr_down = nullptr;
    uint32_t* h_counts = nullptr;    // pinned: per view sum M, rendered
    cudaGraphExec_t graph = nullptr;      // batches without a primitive budget
    cudaGraphExec_t graph_sel = nullptr;  // batches with one (adds the budget select)
    bool busy = false;
    std::vector<uint64_t> tickets;
};

}  // namespace clod

using namespace clod;

struct clod_server {
    clod_scene scene{};
    clod_server_cfg cfg{};
    // re-runs of requests whose batch overflowed its pair capacity
    std::deque<uint64_t> solo_q;
    std::condition_variable cv_solo;
    std::thread solo_worker;
    clod::Slot solo;                 // its stream, workspace (one view of the largest size), staging
    uint32_t* solo_vals = nullptr;   // pair buffer, grown with cudaMallocAsync on the solo stream
    uint64_t solo_cap = 0;
    int device = 0;
    int n_sm = 0;
    uint32_t max_tiles = 0, max_rb = 0, max_tx = 0;
    uint32_t ch = 1;        // rank chunks per view of the largest batch (the slots' layouts)
    uint32_t solo_ch = 1;   // the same for the solo lane's one view of the largest size
    size_t max_diff = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false;
    uint64_t next_ticket = 1;
    clod_status fatal = CLOD_OK;
};

namespace clod {

// The batch's rank chunks per view: chunk_count for its own views, within
// what the slot's layout and captured grids hold (the per (chunk, tile)
// counts, the emission blocks and the counting blocks).
static uint32_t batch_chunks(clod_server* S, const std::vector<const Request*>& batch, const FrameLayout& L)
{
    uint64_t tiles = 0, bands = 0;
    for (const Request* r : batch) {
        const uint64_t TX = (r->view.width + TILE - 1) / TILE, TY = (r->view.height + TILE - 1) / TILE;
        tiles += TX * TY;
        bands += (TY + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;
    }
    uint64_t c = chunk_count((uint64_t)S->scene.n, tiles);
    c = std::min<uint64_t>(c, (uint64_t)L.n_chunks * L.total_tiles / std::max<uint64_t>(1, tiles));
    c = std::min<uint64_t>(c, (uint64_t)L.rb_total / std::max<uint64_t>(1, bands));
    c = std::min<uint64_t>(c, (uint64_t)L.n_chunks * L.n_views / std::max<uint64_t>(1, batch.size()));
    return (uint32_t)std::max<uint64_t>(1, c);
}

static void fill_views(clod_server* S, const std::vector<const Request*>& batch, Slot& sl, FrameHeader& h)
{
    const uint32_t CH = batch_chunks(S, batch, sl.L);
    uint32_t tile_base = 0, rb_base = 0, mtx = 1;
    for (size_t v = 0; v < batch.size(); ++v) {
        const clod_view& w = batch[v]->view;
        ViewDev& d = sl.h_views[v];
        view_record(w, d);
        d.tile_base = tile_base;
        d.rb_base = rb_base;
        d.out_img = batch[v]->out;
        tile_base += (uint32_t)(d.TX * d.TY);
        rb_base += CH * (uint32_t)((d.TY + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
        mtx = std::max<uint32_t>(mtx, (uint32_t)d.TX);
    }
    std::memset(&h, 0, sizeof(h));
    h.n = (uint64_t)S->scene.n;
    h.n_views = (uint32_t)batch.size();
    h.total_tiles = tile_base;
    h.n_chunks = CH;
    h.n_rs_blocks = (uint32_t)(((uint64_t)S->scene.n + RS_ITEMS - 1) / RS_ITEMS);
    h.max_tx = S->max_tx;   // shared-memory layout of the emission blocks: fixed per slot
    h.rb_total = rb_base;
}

// The launch sequence of one batch on a slot (captured once when graphs are on).
static void enqueue_batch(clod_server* S, Slot& sl, cudaStream_t st, bool select)
{
    const Frame F = frame_ptrs(sl.ws, sl.L);
    const int V = (int)S->cfg.max_views_per_batch;
    cudaMemsetAsync(sl.ws, 0, sl.L.views, st);
    cudaMemcpyAsync(F.hdr, sl.h_hdr_up, sizeof(FrameHeader), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(F.views, sl.h_views, sizeof(ViewDev) * V, cudaMemcpyHostToDevice, st);
    launch_preprocess(F, S->scene, (uint32_t)V, nullptr, nullptr, nullptr, S->n_sm, st, select);
    launch_bin_sort(F, sl.L, S->cfg.pair_capacity, nullptr, sl.vals, sl.ranges, st);
    launch_blend_fwd(F, sl.vals, sl.ranges, nullptr, nullptr, nullptr, nullptr, S->n_sm, st, S->cfg.fast_exp != 0,
                     sl.L.total_tiles);
    cudaMemcpyAsync(sl.h_hdr_down, F.hdr, sizeof(FrameHeader), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(sl.h_counts, F.n_surv, sizeof(uint32_t) * 2 * V, cudaMemcpyDeviceToHost, st);
}

static clod_status slot_init(clod_server* S, Slot& sl)
{
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(e, "server slot stream");
    const uint32_t V = (uint32_t)S->cfg.max_views_per_batch;
    sl.L = frame_layout((uint64_t)S->scene.n, V, S->max_tiles, S->ch, S->max_rb, S->max_tx, S->max_diff);
    if ((e = cudaMalloc(&sl.ws, sl.L.total)) != cudaSuccess) return cuda_fail(e, "server workspace");
    if ((e = cudaMalloc(&sl.vals, sizeof(uint32_t) * std::max<uint64_t>(1, S->cfg.pair_capacity))) != cudaSuccess)
        return cuda_fail(e, "server pair buffer");
    if ((e = cudaMalloc(&sl.ranges, sizeof(uint32_t) * 2 * (size_t)S->max_tiles)) != cudaSuccess)
        return cuda_fail(e, "server ranges");
    if ((e = cudaMallocHost(&sl.h_views, sizeof(ViewDev) * V)) != cudaSuccess) return cuda_fail(e, "pinned views");
    if ((e = cudaMallocHost(&sl.h_hdr_up, sizeof(FrameHeader))) != cudaSuccess) return cuda_fail(e, "pinned header");
    if ((e = cudaMallocHost(&sl.h_hdr_down, sizeof(FrameHeader))) != cudaSuccess) return cuda_fail(e, "pinned header");
    if ((e = cudaMallocHost(&sl.h_counts, sizeof(uint32_t) * 2 * V)) != cudaSuccess) return cuda_fail(e, "pinned counts");
    std::memset(sl.h_views, 0, sizeof(ViewDev) * V);
    if (S->cfg.use_graphs) {
        // capture the slot's launch sequences once; sizes come from the header at run time
        for (int sel = 0; sel < 2; ++sel) {
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(sl.stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(e, "begin capture");
            enqueue_batch(S, sl, sl.stream, sel != 0);
            e = cudaStreamEndCapture(sl.stream, &g);
            if (e != cudaSuccess) return cuda_fail(e, "end capture");
            e = cudaGraphInstantiate(sel ? &sl.graph_sel : &sl.graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        }
    }
    return CLOD_OK;
}

// The solo lane: a stream, a workspace for one view of the largest size,
// ranges for its tiles and pinned staging; its pair buffer is allocated on
// first use.
static clod_status solo_init(clod_server* S)
{
    Slot& sl = S->solo;
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "server solo stream");
    const uint32_t TX = S->max_tx, TY = (uint32_t)((S->cfg.max_height + TILE - 1) / TILE);
    const uint32_t rb = S->solo_ch * ((TY + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
    sl.L = frame_layout((uint64_t)S->scene.n, 1, TX * TY, S->solo_ch, rb, TX, S->max_diff);
    if ((e = cudaMalloc(&sl.ws, sl.L.total)) != cudaSuccess) return cuda_fail(e, "server solo workspace");
    if ((e = cudaMalloc(&sl.ranges, sizeof(uint32_t) * 2 * (size_t)TX * TY)) != cudaSuccess)
        return cuda_fail(e, "server solo ranges");
    if ((e = cudaMallocHost(&sl.h_views, sizeof(ViewDev))) != cudaSuccess) return cuda_fail(e, "pinned views");
    if ((e = cudaMallocHost(&sl.h_hdr_down, sizeof(FrameHeader))) != cudaSuccess) return cuda_fail(e, "pinned header");
    if ((e = cudaMallocHost(&sl.h_counts, sizeof(uint32_t) * 2)) != cudaSuccess) return cuda_fail(e, "pinned counts");
    std::memset(sl.h_views, 0, sizeof(ViewDev));
    return CLOD_OK;
}

static void slot_free(Slot& sl)
{
    if (sl.graph) cudaGraphExecDestroy(sl.graph);
    if (sl.graph_sel) cudaGraphExecDestroy(sl.graph_sel);
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    cudaFree(sl.ws);
    cudaFree(sl.vals);
    cudaFree(sl.ranges);
    cudaFreeHost(sl.h_views);
    cudaFreeHost(sl.h_hdr_up);
    cudaFreeHost(sl.h_hdr_down);
    cudaFreeHost(sl.h_counts);
    if (sl.ev) cudaEventDestroy(sl.ev);
    if (sl.stream) cudaStreamDestroy(sl.stream);
}

// Renders one request alone on the solo lane (overflow path): its pair
// count is read back after preprocessing, the lane's pair buffer grows
// (stream-ordered: no device-wide synchronisation) when it is too small, then
// sort and blend.  Runs on the solo thread; other slots keep running.
static clod_status render_alone(clod_server* S, Request& r)
{
    Slot& sl = S->solo;
    const clod_view& w = r.view;
    const int TX = (w.width + TILE - 1) / TILE, TY = (w.height + TILE - 1) / TILE;
    std::vector<const Request*> one{&r};
    FrameHeader h;
    fill_views(S, one, sl, h);     // chunks within the solo layout's
    const uint32_t CH = h.n_chunks;
    const uint32_t rb = CH * (uint32_t)((TY + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
    const FrameLayout L = frame_layout((uint64_t)S->scene.n, 1, (uint32_t)(TX * TY), CH, rb, (uint32_t)TX,
                                       (size_t)(TX + 1) * (TY + 1));
    h.max_tx = (uint32_t)TX;
    const Frame F = frame_ptrs(sl.ws, L);   // the lane's workspace holds one view of the largest size
    cudaStream_t st = sl.stream;
    cudaMemsetAsync(sl.ws, 0, L.views, st);
    cudaMemcpyAsync(F.hdr, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(F.views, sl.h_views, sizeof(ViewDev), cudaMemcpyHostToDevice, st);
    launch_preprocess(F, S->scene, 1, nullptr, nullptr, nullptr, S->n_sm, st, one[0]->view.budget > 0);
    cudaMemcpyAsync(sl.h_hdr_down, F.hdr, sizeof(FrameHeader), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "render_alone");
    const unsigned long long K = sl.h_hdr_down->n_pairs;
    if (K > 0xFFFFFFFFull) return CLOD_ERR_CAPACITY;
    if (K > S->solo_cap) {
        const uint64_t cap = std::min<uint64_t>(0xFFFFFFFFull, K + K / 4 + 1024);
        if (S->solo_vals) cudaFreeAsync(S->solo_vals, st);
        S->solo_vals = nullptr;
        S->solo_cap = 0;
        if ((e = cudaMallocAsync(reinterpret_cast<void**>(&S->solo_vals), sizeof(uint32_t) * cap, st)) != cudaSuccess)
            return cuda_fail(e, "render_alone pairs");
        S->solo_cap = cap;
    }
    launch_bin_sort(F, L, S->solo_cap, nullptr, S->solo_vals, sl.ranges, st);
    launch_blend_fwd(F, S->solo_vals, sl.ranges, nullptr, nullptr, nullptr, nullptr, S->n_sm, st, S->cfg.fast_exp != 0,
                     L.total_tiles);
    cudaMemcpyAsync(sl.h_hdr_down, F.hdr, sizeof(FrameHeader), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(sl.h_counts, F.n_surv, sizeof(uint32_t) * 2, cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "render_alone");
    r.pairs = sl.h_hdr_down->n_pairs;
    r.rendered = sl.h_counts[1];
    if (sl.h_hdr_down->status & STATUS_OVERFLOW) return CLOD_ERR_CAPACITY;
    return CLOD_OK;
}

// The solo thread: re-runs, in arrival order, the requests of overflowed batches.
static void solo_main(clod_server* S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        if (S->solo_q.empty()) {
            S->cv_solo.wait(lk);
            continue;
        }
        const uint64_t tk = S->solo_q.front();
        S->solo_q.pop_front();
        Request copy = S->reqs[tk];
        copy.t_launch = now_us();
        copy.batch = 1;
        lk.unlock();
        const clod_status st = render_alone(S, copy);
        lk.lock();
        Request& r = S->reqs[tk];
        r.t_launch = copy.t_launch;
        r.batch = 1;
        r.pairs = copy.pairs;
        r.rendered = copy.rendered;
        r.status = st;
        r.done = true;
        r.t_done = now_us();
        S->cv_done.notify_all();
    }
}

static void worker_main(clod_server* S)
{
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool progress = false;
        // 1. completions
        for (Slot& sl : S->slots) {
            if (!sl.busy) continue;
            if (cudaEventQuery(sl.ev) != cudaSuccess) continue;
            const double t = now_us();
            const bool overflow = (sl.h_hdr_down->status & STATUS_OVERFLOW) != 0;
            for (size_t k = 0; k < sl.tickets.size(); ++k) {
                Request& r = S->reqs[sl.tickets[k]];
                if (overflow) continue;     // re-run on the solo lane below
                r.done = true;
                r.t_done = t;
                r.status = CLOD_OK;
                r.pairs = sl.h_hdr_down->n_pairs;
                r.rendered = sl.h_counts[2 * k + 1];
            }
            if (overflow) {   // re-run each request alone on the solo lane, in arrival order
                for (uint64_t tk : sl.tickets) S->solo_q.push_back(tk);
                S->cv_solo.notify_one();
            }
            sl.tickets.clear();
            sl.busy = false;
            progress = true;
        }
        if (progress) S->cv_done.notify_all();
        // 2. admissions into free slots
        for (Slot& sl : S->slots) {
            if (sl.busy || S->pending.empty()) continue;
            Request& first = S->reqs[S->pending.front()];
            if (S->cfg.batch_window_us > 0 && (int)S->pending.size() < S->cfg.max_views_per_batch &&
                now_us() - first.t_submit < S->cfg.batch_window_us)
                continue;   // wait a little for more requests to share the launch
            std::vector<const Request*> batch;
            uint64_t pixels = 0;
            while (!S->pending.empty() && (int)batch.size() < S->cfg.max_views_per_batch) {
                Request& r = S->reqs[S->pending.front()];
                const uint64_t p = (uint64_t)r.view.width * r.view.height;
                if (!batch.empty() && pixels + p > S->cfg.max_pixels_per_batch) break;
                pixels += p;
                batch.push_back(&r);
                sl.tickets.push_back(S->pending.front());
                S->pending.pop_front();
            }
            FrameHeader h;
            fill_views(S, batch, sl, h);
            *sl.h_hdr_up = h;
            const double t = now_us();
            for (const Request* r : batch) {
                Request* rw = const_cast<Request*>(r);
                rw->t_launch = t;
                rw->batch = (int32_t)batch.size();
            }
            bool select = false;
            for (const Request* r : batch) select = select || r->view.budget > 0;
            cudaError_t e;
            if (sl.graph) e = cudaGraphLaunch(select ? sl.graph_sel : sl.graph, sl.stream);
            else {
                enqueue_batch(S, sl, sl.stream, select);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.stream);
            if (e != cudaSuccess) {
                for (uint64_t tk : sl.tickets) {
                    Request& r = S->reqs[tk];
                    r.status = CLOD_ERR_CUDA;
                    r.done = true;
                    r.t_done = now_us();
                }
                sl.tickets.clear();
                S->fatal = CLOD_ERR_CUDA;
                S->cv_done.notify_all();
                continue;
            }
            sl.busy = true;
            progress = true;
        }
        if (!progress) {
            bool any_busy = false;
            for (Slot& sl : S->slots) any_busy |= sl.busy;
            // poll the device while batches run; sleep on the queue otherwise
            S->cv_work.wait_for(lk, std::chrono::microseconds(any_busy ? 20 : 500));
        }
    }
}

}  // namespace clod

extern "C" {

clod_status clod_server_create(const clod_scene* scene, const clod_server_cfg* cfg, clod_server** out)
{
    if (!scene || !cfg || !out) return fail(CLOD_ERR_ARG, "NULL argument to clod_server_create");
    if (scene->n < 0 || scene->n >= (1ll << 31) || scene->sh_degree < 0 || scene->sh_degree > 3)
        return fail(CLOD_ERR_ARG, "bad scene");
    if (scene->n > 0 && (!scene->means || !scene->scales || !scene->quats || !scene->opacity || !scene->sh || !scene->decay))
        return fail(CLOD_ERR_ARG, "scene array pointer is NULL");
    if (cfg->max_views_per_batch < 1 || cfg->max_views_per_batch > MAX_VIEWS || cfg->n_slots < 1 || cfg->n_slots > 16 ||
        cfg->queue_capacity < 1 || cfg->max_width < 1 || cfg->max_height < 1 || cfg->max_width > 16384 ||
        cfg->max_height > 16384 || cfg->max_pixels_per_batch < (uint64_t)cfg->max_width * cfg->max_height ||
        cfg->pair_capacity < 1 || cfg->pair_capacity > 0xFFFFFFFFull)
        return fail(CLOD_ERR_ARG, "bad server configuration");
    int n_sm = 0;
    clod_status s = device_ready(&n_sm);
    if (s) return s;
    clod_server* S = new clod_server();
    S->scene = *scene;
    S->cfg = *cfg;
    S->n_sm = n_sm;
    cudaGetDevice(&S->device);
    // bounds of the largest admissible batch
    const uint64_t TXm = (cfg->max_width + TILE - 1) / TILE, TYm = (cfg->max_height + TILE - 1) / TILE;
    const uint64_t B = (uint64_t)cfg->max_views_per_batch;
    const uint64_t tiles_by_px = cfg->max_pixels_per_batch / (TILE * TILE) + B * (TXm + TYm + 1);
    S->max_tiles = (uint32_t)std::min<uint64_t>(B * TXm * TYm, tiles_by_px);
    // every batch takes the chunk count of the largest (B views of the largest size)
    S->ch = chunk_count((uint64_t)scene->n, S->max_tiles);
    S->max_rb = (uint32_t)(B * S->ch * ((TYm + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK));
    S->solo_ch = chunk_count((uint64_t)scene->n, TXm * TYm);
    S->max_tx = (uint32_t)TXm;
    S->max_diff = (size_t)(TXm + 1) * (TYm + 1);
    S->slots.resize(cfg->n_slots);
    for (Slot& sl : S->slots) {
        if ((s = slot_init(S, sl)) != CLOD_OK) {
            for (Slot& q : S->slots) slot_free(q);
            delete S;
            return s;
        }
    }
    if ((s = solo_init(S)) != CLOD_OK) {
        for (Slot& q : S->slots) slot_free(q);
        slot_free(S->solo);
        delete S;
        return s;
    }
    S->worker = std::thread(worker_main, S);
    S->solo_worker = std::thread(solo_main, S);
    *out = S;
    return CLOD_OK;
}

clod_status clod_serve_submit(clod_server* S, const clod_view* view, float* image_out, uint64_t* ticket)
{
    if (!S || !view || !image_out || !ticket) return fail(CLOD_ERR_ARG, "NULL argument to clod_serve_submit");
    const clod_view& w = *view;
    if (w.width < 1 || w.height < 1 || w.width > S->cfg.max_width || w.height > S->cfg.max_height)
        return fail(CLOD_ERR_ARG, "view %dx%d outside the server's %dx%d", w.width, w.height, S->cfg.max_width,
                    S->cfg.max_height);
    if (clod_status s = check_view(w, 0)) return s;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal) return fail(S->fatal, "server stopped after a CUDA error");
    if ((int)S->pending.size() >= S->cfg.queue_capacity) return fail(CLOD_ERR_QUEUE_FULL, "queue full");
    const uint64_t t = S->next_ticket++;
    Request& r = S->reqs[t];
    r.view = w;
    r.out = image_out;
    r.t_submit = now_us();
    S->pending.push_back(t);
    *ticket = t;
    S->cv_work.notify_one();
    return CLOD_OK;
}

static void fill_stats(const Request& r, clod_req_stats* st)
{
    if (!st) return;
    st->status = r.status;
    st->batch_size = r.batch;
    st->submit_us = r.t_submit;
    st->launch_us = r.t_launch;
    st->done_us = r.t_done;
    st->n_rendered = r.rendered;
    st->reserved = 0;
    st->n_pairs = r.pairs;
}

clod_status clod_serve_poll(clod_server* S, uint64_t ticket, int32_t* done, clod_req_stats* stats)
{
    if (!S || !done) return fail(CLOD_ERR_ARG, "NULL argument to clod_serve_poll");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(CLOD_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    *done = it->second.done ? 1 : 0;
    if (!it->second.done) return CLOD_ERR_NOT_READY;
    fill_stats(it->second, stats);
    const clod_status st = it->second.status;
    S->reqs.erase(it);
    return st == CLOD_OK ? CLOD_OK : fail(st, "request failed");
}

clod_status clod_serve_wait(clod_server* S, uint64_t ticket, int64_t timeout_us, clod_req_stats* stats)
{
    if (!S) return fail(CLOD_ERR_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return fail(CLOD_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
    while (!S->reqs[ticket].done) {
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !S->reqs[ticket].done)
            return fail(CLOD_ERR_TIMEOUT, "request %llu not finished after %lld us", (unsigned long long)ticket,
                        (long long)timeout_us);
    }
    Request r = S->reqs[ticket];
    S->reqs.erase(ticket);
    fill_stats(r, stats);
    return r.status == CLOD_OK ? CLOD_OK : fail(r.status, "request failed");
}

clod_status clod_server_destroy(clod_server* S)
{
    if (!S) return fail(CLOD_ERR_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->cv_solo.notify_all();
    if (S->worker.joinable()) S->worker.join();
    if (S->solo_worker.joinable()) S->solo_worker.join();
    for (Slot& sl : S->slots) slot_free(sl);
    if (S->solo_vals) {
        cudaFreeAsync(S->solo_vals, S->solo.stream);
        cudaStreamSynchronize(S->solo.stream);
    }
    slot_free(S->solo);
    delete S;
    return CLOD_OK;
}

}  // extern "C"
