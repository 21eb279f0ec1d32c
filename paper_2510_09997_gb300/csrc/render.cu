// render.cu -- front-to-back alpha blending of every tile (Sec. 3.1, Eq. 1).
//
// Persistent blocks of 256 threads (one 16x16 tile, one pixel per thread)
// take tiles from an atomic queue.  For its tile a block walks the sorted
// list in batches of 256: each thread gathers one Gaussian's record
// (u, v, -A/2, -B | -C/2, alpha'', r, g | b) into shared memory, then every
// thread blends the batch for its pixel in list order.  The block stops as
// soon as all its pixels are saturated (__syncthreads_count).  This is plain
// FP32/ALU work with one exponential per evaluated pair: no tensor cores.
#include <algorithm>

#include "clod_internal.cuh"

namespace clod {

template <bool COUNT>
__global__ void __launch_bounds__(BLOCK_PIX) k_blend_fwd(Frame F, const uint32_t* __restrict__ vals,
                                                         const uint32_t* __restrict__ ranges,
                                                         float* __restrict__ image, float* __restrict__ Tout,
                                                         uint32_t* __restrict__ ncout,
                                                         unsigned long long* __restrict__ evaluated)
{
    __shared__ float4 s0[BLOCK_PIX];
    __shared__ float4 s1[BLOCK_PIX];
    __shared__ float s2[BLOCK_PIX];
    __shared__ uint32_t s_tile;
    __shared__ int s_view;
    const FrameHeader* hdr = F.hdr;
    if (hdr->status & STATUS_OVERFLOW) return;
    const uint32_t TT = hdr->total_tiles;
    const uint32_t V = hdr->n_views;
    const int64_t n = static_cast<int64_t>(hdr->n);
    unsigned long long evals = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t t = atomicAdd(&F.hdr->work[0], 1u);
            s_tile = t;
            int v = 0;
            if (t < TT)
                for (uint32_t u = 0; u < V; ++u) {
                    const ViewDev& W = F.views[u];
                    if (t >= W.tile_base && t < W.tile_base + (uint32_t)(W.TX * W.TY)) {
                        v = (int)u;
                        break;
                    }
                }
            s_view = v;
        }
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= TT) break;
        const ViewDev& W = F.views[s_view];
        const uint32_t local = t - W.tile_base;
        const int tx = (int)(local % (uint32_t)W.TX), ty = (int)(local / (uint32_t)W.TX);
        const int px = tx * TILE + (int)(threadIdx.x & 15), py = ty * TILE + (int)(threadIdx.x >> 4);
        const bool inside = px < W.W && py < W.H;
        const float fpx = __fadd_rn(static_cast<float>(px), 0.5f);
        const float fpy = __fadd_rn(static_cast<float>(py), 0.5f);
        const uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
        const int64_t vn = (int64_t)s_view * n;
        float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
        uint32_t last = 0;
        bool done = !inside;
        for (uint32_t b = start; b < end; b += BLOCK_PIX) {
            if (__syncthreads_count(done) == BLOCK_PIX) break;
            const uint32_t j = b + threadIdx.x;
            if (j < end) {
                const int64_t g = vn + vals[j];
                s0[threadIdx.x] = F.rec0[g];
                s1[threadIdx.x] = F.rec1[g];
                s2[threadIdx.x] = F.rec2[g];
            }
            __syncthreads();
            const int cnt = (int)min((uint32_t)BLOCK_PIX, end - b);
            if (!done) {
                for (int k = 0; k < cnt; ++k) {
                    const float4 a = s0[k];
                    const float4 c = s1[k];
                    if (COUNT) ++evals;
                    const float al = blend_alpha(__fsub_rn(a.x, fpx), __fsub_rn(a.y, fpy), a.z, a.w, c.x, c.y);
                    if (al < 0.0f) continue;
                    const float tt = __fmul_rn(T, __fsub_rn(1.0f, al));
                    if (tt < 1e-4f) {
                        done = true;
                        break;
                    }
                    const float w = __fmul_rn(al, T);
                    C0 = __fmaf_rn(c.z, w, C0);
                    C1 = __fmaf_rn(c.w, w, C1);
                    C2 = __fmaf_rn(s2[k], w, C2);
                    T = tt;
                    last = b - start + (uint32_t)k + 1u;
                }
            }
        }
        if (inside) {
            const size_t plane = (size_t)W.W * W.H;
            const size_t p = (size_t)py * W.W + px;
            float* img = image + 3 * W.pix_base;
            img[p] = __fmaf_rn(T, W.bg[0], C0);
            img[plane + p] = __fmaf_rn(T, W.bg[1], C1);
            img[2 * plane + p] = __fmaf_rn(T, W.bg[2], C2);
            if (Tout) Tout[W.pix_base + p] = T;
            if (ncout) ncout[W.pix_base + p] = last;
        }
        __syncthreads();
    }
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
        if ((threadIdx.x & 31) == 0 && evals) atomicAdd(evaluated, evals);
    }
}

static int g_blend_blocks_per_sm = 0;

cudaError_t render_setup()
{
    int b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_blend_fwd<false>, BLOCK_PIX, 0);
    if (e != cudaSuccess) return e;
    g_blend_blocks_per_sm = b > 0 ? b : 1;
    return cudaSuccess;
}

void launch_blend_fwd(const Frame& F, const uint32_t* vals, const uint32_t* ranges, float* image, float* Tout,
                      uint32_t* ncout, unsigned long long* evaluated, int n_sm, cudaStream_t st)
{
    const int blocks = n_sm * std::max(1, g_blend_blocks_per_sm);
    cudaMemsetAsync(&F.hdr->work[0], 0, sizeof(uint32_t), st);
    if (evaluated)
        k_blend_fwd<true><<<blocks, BLOCK_PIX, 0, st>>>(F, vals, ranges, image, Tout, ncout, evaluated);
    else
        k_blend_fwd<false><<<blocks, BLOCK_PIX, 0, st>>>(F, vals, ranges, image, Tout, ncout, nullptr);
}

}  // namespace clod
