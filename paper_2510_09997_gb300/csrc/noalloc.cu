// noalloc.cu -- clod_render_noalloc: a forward render that allocates no
// device memory.
//
// Some callers cannot call cudaMalloc: code running where the CUDA caching
// allocator of a host framework owns the device memory, real-time loops that
// must not allocate after start-up, or plug-ins handed only raw input and
// output pointers.  For them this entry point renders one view with all of its
// scratch -- the frame workspace, the sorted pair list and the tile ranges --
// in one file-scope __device__ array of fixed size, which every GPU that loads
// the library holds until the process exits.
//
// Limits: at most NA_MAX_GAUSSIANS Gaussians, NA_MAX_SIDE pixels per side and
// NA_MAX_PAIRS (view, tile, Gaussian) pairs.  Calls share the array, so calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race; serialise them.  A call is synchronous: it waits for the
// frame on its stream and reads the frame header back to report overflow, so
// it cannot run inside a stream capture.  The first call on a device also
// looks up the array's device address (with that device current).
#include <algorithm>
#include <cstring>
#include <mutex>

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

constexpr int64_t NA_MAX_GAUSSIANS = 65536;
constexpr int NA_MAX_SIDE = 1024;
constexpr uint64_t NA_MAX_PAIRS = 1ull << 21;
constexpr size_t NA_FRAME_BYTES = size_t(8) << 20;
constexpr int NA_MAX_TILES = (NA_MAX_SIDE / TILE) * (NA_MAX_SIDE / TILE);
constexpr size_t NA_VALS_OFFSET = NA_FRAME_BYTES;
constexpr size_t NA_RANGES_OFFSET = NA_VALS_OFFSET + NA_MAX_PAIRS * sizeof(uint32_t);
constexpr size_t NA_BYTES = NA_RANGES_OFFSET + size_t(NA_MAX_TILES) * 2 * sizeof(uint32_t);

// The scratch array.  In host code its name is only a host-side stand-in:
// kernels get the device address looked up below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

static std::mutex g_na_mu;
static void* g_na_ptr[64];

static clod_status noalloc_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(CLOD_ERR_CUDA, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        // the largest admissible frame (NA_MAX_GAUSSIANS, NA_MAX_SIDE^2 pixels)
        // must fit the frame part of the array; checked once, so that a
        // change of the workspace layout cannot silently shrink the limits
        const uint32_t ch = (uint32_t)std::min<int64_t>((NA_MAX_GAUSSIANS + 1023) / 1024, MAX_CHUNKS);
        const int side = NA_MAX_SIDE / TILE;
        const FrameLayout big = frame_layout(NA_MAX_GAUSSIANS, 1, (uint32_t)NA_MAX_TILES, ch,
                                             ch * (uint32_t)((side + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK),
                                             (uint32_t)side, (size_t)(side + 1) * (side + 1));
        if (big.total > NA_FRAME_BYTES)
            return fail(CLOD_ERR_CUDA, "clod_render_noalloc: the largest frame needs %zu bytes, the array holds %zu",
                        big.total, NA_FRAME_BYTES);
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return CLOD_OK;
}

}  // namespace clod

using namespace clod;

extern "C" clod_status clod_render_noalloc(const clod_scene* scene, const clod_view* view, float* image,
                                           float* T_final, uint32_t* n_contrib, clod_stream stream)
{
    if (!scene || !view || !image) return fail(CLOD_ERR_ARG, "NULL argument to clod_render_noalloc");
    if (scene->n < 0 || scene->n > NA_MAX_GAUSSIANS)
        return fail(CLOD_ERR_ARG, "clod_render_noalloc takes at most %lld Gaussians, got %lld",
                    (long long)NA_MAX_GAUSSIANS, (long long)scene->n);
    if (scene->sh_degree < 0 || scene->sh_degree > 3) return fail(CLOD_ERR_ARG, "sh_degree %d outside [0, 3]", scene->sh_degree);
    if (scene->n > 0 && (!scene->means || !scene->scales || !scene->quats || !scene->opacity || !scene->sh || !scene->decay))
        return fail(CLOD_ERR_ARG, "scene array pointer is NULL");
    if (reinterpret_cast<uintptr_t>(scene->quats) % 16 || (scene->sh_degree == 3 && reinterpret_cast<uintptr_t>(scene->sh) % 16))
        return fail(CLOD_ERR_ARG, "quats (and sh at degree 3) must be 16-byte aligned");
    const clod_view& w = *view;
    if (w.width < 1 || w.height < 1 || w.width > NA_MAX_SIDE || w.height > NA_MAX_SIDE)
        return fail(CLOD_ERR_ARG, "clod_render_noalloc takes views up to %dx%d, got %dx%d", NA_MAX_SIDE, NA_MAX_SIDE,
                    w.width, w.height);
    if (clod_status sv = check_view(w, 0)) return sv;

    int n_sm = 0;
    clod_status s = device_ready(&n_sm);
    if (s) return s;
    void* base = nullptr;
    if ((s = noalloc_scratch(&base))) return s;

    const uint64_t n = (uint64_t)scene->n;
    const int TX = (w.width + TILE - 1) / TILE, TY = (w.height + TILE - 1) / TILE;
    const uint32_t bands = (uint32_t)((TY + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK);
    const uint32_t CH = chunk_count(n, (uint64_t)TX * TY);
    const uint32_t rb_total = CH * bands;
    const FrameLayout L = frame_layout(n, 1, (uint32_t)(TX * TY), CH, rb_total, (uint32_t)TX,
                                       (size_t)(TX + 1) * (TY + 1));
    if (L.total > NA_FRAME_BYTES) return fail(CLOD_ERR_CAPACITY, "frame needs %zu bytes of scratch, %zu available",
                                              L.total, NA_FRAME_BYTES);
    char* b = static_cast<char*>(base);
    const Frame F = frame_ptrs(b, L);
    uint32_t* vals = reinterpret_cast<uint32_t*>(b + NA_VALS_OFFSET);
    uint32_t* ranges = reinterpret_cast<uint32_t*>(b + NA_RANGES_OFFSET);

    ViewDev vd;
    view_record(w, vd);
    FrameHeader h;
    std::memset(&h, 0, sizeof(h));
    h.n = n;
    h.n_views = 1;
    h.total_tiles = (uint32_t)(TX * TY);
    h.n_chunks = L.n_chunks;
    h.n_rs_blocks = L.n_rs_blocks;
    h.max_tx = L.max_tx;
    h.rb_total = L.rb_total;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the array keeps the previous call's contents: clear what accumulates
    cudaError_t e = cudaMemsetAsync(b, 0, L.views, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(F.hdr, &h, sizeof(h), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(F.views, &vd, sizeof(vd), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "clod_render_noalloc upload");
    launch_preprocess(F, *scene, 1, nullptr, nullptr, nullptr, n_sm, st, w.budget > 0);
    if ((e = launch_bin_sort(F, L, NA_MAX_PAIRS, nullptr, vals, ranges, st)) != cudaSuccess)
        return cuda_fail(e, "clod_render_noalloc sort launch");
    launch_blend_fwd(F, vals, ranges, image, T_final, n_contrib, nullptr, n_sm, st, (view->flags & CLOD_FAST_EXP) != 0,
                     (uint32_t)(TX * TY));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "clod_render_noalloc launch");
    // the pair count is data dependent: wait for the frame and report overflow
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "clod_render_noalloc sync");
    FrameHeader out;
    if ((e = cudaMemcpy(&out, F.hdr, sizeof(out), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "clod_render_noalloc status");
    if ((out.status & STATUS_OVERFLOW) || out.n_pairs > NA_MAX_PAIRS)
        return fail(CLOD_ERR_CAPACITY, "frame has %llu pairs, clod_render_noalloc holds at most %llu; nothing written",
                    (unsigned long long)out.n_pairs, (unsigned long long)NA_MAX_PAIRS);
    return CLOD_OK;
}
