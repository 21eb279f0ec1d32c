// render.cu -- front-to-back alpha blending of every tile (Sec. 3.1, Eq. 1).
//
// Persistent blocks of 256 threads (one 16x16 tile, one pixel per thread;
// each warp an 8x4 patch) take tiles from an atomic queue.  For its tile a
// block walks the sorted list in batches of 256: each thread gathers one
// Gaussian's record (u, v, -A/2, -B | -C/2, alpha'', r, g | b) into shared
// memory and derives a box that holds every pixel the Gaussian can reach with
// opacity >= 1/255; then every thread blends the batch for its pixel in list
// order.  A warp whose patch misses a Gaussian's box skips it as a whole --
// every one of its pixels would skip it anyway, so no result changes.  The
// block stops once all its pixels are saturated (__syncthreads_count).
// Plain FP32/ALU work with one exponential per evaluated pair: no tensor
// cores.
#include <algorithm>

#include "clod_internal.cuh"

namespace clod {

// Box around (u, v) holding every pixel centre where the blend's opacity can
// reach 1/255: there power >= P* = max(-5.6, -ln(255 alpha'')), i.e. the
// ellipse d^T Q d <= 2|P*| (Q the conic), whose half-extents are
// sqrt(2|P*| Sigma_xx), sqrt(2|P*| Sigma_yy) with Sigma = Q^-1.  Widened by
// 0.1% (+0.01 px) so FP32 rounding of the power can never put a reached pixel
// outside, and by the half-size of the 8x4 patch (3.5, 1.5), so the warp test
// is |u - patch centre| > extent.  alpha'' < 1/255 reaches no pixel.  For a
// conic so elongated that A C - B^2 loses more than 0.1% of A C to
// cancellation the box is not trusted: such a Gaussian is never skipped.
__device__ __forceinline__ float4 reach_box(float4 a, float4 c, float b)
{
    const float A = -2.0f * a.z, B = -a.w, C = -2.0f * c.x;
    const float det = A * C - B * B;
    const float a255 = 255.0f * c.y;
    if (!(a255 >= 1.0f)) return make_float4(b, -1.0f, -1.0f, 0.0f);
    if (!(det > 1e-3f * (A * C)) || !(A > 0.0f) || !(C > 0.0f))
        return make_float4(b, __int_as_float(0x7f800000), __int_as_float(0x7f800000), 0.0f);
    const float P = fminf(5.6f, logf(a255));
    const float r2 = 2.0f * P * 1.001f + 1e-3f;
    const float xe = sqrtf(r2 * (C / det)) * 1.001f + 0.01f;
    const float ye = sqrtf(r2 * (A / det)) * 1.001f + 0.01f;
    return make_float4(b, xe + 3.5f, ye + 1.5f, 0.0f);
}

template <bool COUNT>
__global__ void __launch_bounds__(BLOCK_PIX) k_blend_fwd(Frame F, const uint32_t* __restrict__ vals,
                                                         const uint32_t* __restrict__ ranges,
                                                         float* __restrict__ image, float* __restrict__ Tout,
                                                         uint32_t* __restrict__ ncout,
                                                         unsigned long long* __restrict__ evaluated)
{
    __shared__ float4 s0[BLOCK_PIX];
    __shared__ float4 s1[BLOCK_PIX];
    __shared__ float4 s2[BLOCK_PIX];   // b, half-extents of the reach box (+ patch half-size)
    __shared__ uint32_t s_tile;
    __shared__ int s_view;
    const FrameHeader* hdr = F.hdr;
    if (hdr->status & STATUS_OVERFLOW) return;
    // 8x4 patch of this warp inside the tile, lane -> pixel
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ox = (wid & 1) * 8 + (lane & 7), oy = (wid >> 1) * 4 + (lane >> 3);
    const float pcx = (float)((wid & 1) * 8) + 4.0f, pcy = (float)((wid >> 1) * 4) + 2.0f;
    const uint32_t TT = hdr->total_tiles;
    const uint32_t V = hdr->n_views;
    const int64_t n = static_cast<int64_t>(hdr->n);
    unsigned long long evals = 0, n_exp = 0, n_con = 0;
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
        const int px = tx * TILE + ox, py = ty * TILE + oy;
        const bool inside = px < W.W && py < W.H;
        const float fpx = __fadd_rn(static_cast<float>(px), 0.5f);
        const float fpy = __fadd_rn(static_cast<float>(py), 0.5f);
        const float wcx = (float)(tx * TILE) + pcx, wcy = (float)(ty * TILE) + pcy;
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
                const float4 a = F.rec0[g];
                const float4 c = F.rec1[g];
                s0[threadIdx.x] = a;
                s1[threadIdx.x] = c;
                s2[threadIdx.x] = reach_box(a, c, F.rec2[g]);
            }
            __syncthreads();
            const int cnt = (int)min((uint32_t)BLOCK_PIX, end - b);
            if (!done) {
                for (int k = 0; k < cnt; ++k) {
                    const float4 a = s0[k];
                    if (COUNT) ++evals;
                    else {
                        const float4 q = s2[k];
                        if (fabsf(a.x - wcx) > q.y || fabsf(a.y - wcy) > q.z) continue;   // warp-uniform
                    }
                    const float4 c = s1[k];
                    const float ddx = __fsub_rn(a.x, fpx), ddy = __fsub_rn(a.y, fpy);
                    if (COUNT) {
                        const float pw = __fmaf_rn(ddx, __fmaf_rn(a.z, ddx, __fmul_rn(a.w, ddy)),
                                                   __fmul_rn(__fmul_rn(c.x, ddy), ddy));
                        if (!(pw > 0.0f || pw < -5.6f)) ++n_exp;
                    }
                    const float al = blend_alpha(ddx, ddy, a.z, a.w, c.x, c.y);
                    if (al < 0.0f) continue;
                    const float tt = __fmul_rn(T, __fsub_rn(1.0f, al));
                    if (tt < 1e-4f) {
                        done = true;
                        break;
                    }
                    const float w = __fmul_rn(al, T);
                    C0 = __fmaf_rn(c.z, w, C0);
                    C1 = __fmaf_rn(c.w, w, C1);
                    C2 = __fmaf_rn(s2[k].x, w, C2);
                    T = tt;
                    last = b - start + (uint32_t)k + 1u;
                    if (COUNT) ++n_con;
                }
            }
        }
        if (inside) {
            const size_t plane = (size_t)W.W * W.H;
            const size_t p = (size_t)py * W.W + px;
            float* img = W.out_img ? W.out_img : image + 3 * W.pix_base;
            img[p] = __fmaf_rn(T, W.bg[0], C0);
            img[plane + p] = __fmaf_rn(T, W.bg[1], C1);
            img[2 * plane + p] = __fmaf_rn(T, W.bg[2], C2);
            if (W.out_T) W.out_T[p] = T;
            else if (Tout) Tout[W.pix_base + p] = T;
            if (W.out_nc) W.out_nc[p] = last;
            else if (ncout) ncout[W.pix_base + p] = last;
        }
        __syncthreads();
    }
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) {
            evals += __shfl_xor_sync(0xffffffffu, evals, o);
            n_exp += __shfl_xor_sync(0xffffffffu, n_exp, o);
            n_con += __shfl_xor_sync(0xffffffffu, n_con, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(evaluated, evals);
            atomicAdd(evaluated + 1, n_exp);
            atomicAdd(evaluated + 2, n_con);
        }
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
