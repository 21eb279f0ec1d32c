// render.cu -- front-to-back alpha blending of every tile (Sec. 3.1, Eq. 1).
//
// Persistent blocks of 128 threads; each warp takes (16x16 tile, quarter)
// items from an atomic queue over the work order the tile scan wrote (longer
// lists first), owns that 8x8 patch (two vertically adjacent pixels per
// thread) and walks the tile's sorted list on its own, 32 entries at a time: every
// lane gathers one record (u, v, -A/2, -B | -C/2, alpha'', r, g | b, reach
// half-extents, power floor) and tests the box that holds every pixel the
// Gaussian can reach with opacity >= 1/255 (computed once per Gaussian by the
// preprocessing); the warp blends, in list order, only the entries whose box
// meets its patch -- every pixel of the patch would skip the others anyway, so
// no result changes.  Per pixel, a power below the Gaussian's floor (opacity
// < 1/255 for certain) skips the exponential, and the per-pixel updates run
// under predicates rather than branches (the kernel is issue bound).  A warp
// stops once its 64 pixels are saturated.  The exponential is the
// reproducible software one, or with CLOD_FAST_EXP the special-function unit's.
// Plain FP32/ALU work with one exponential per evaluated pair: no tensor
// cores.
#include <algorithm>

#include "clod_internal.cuh"

namespace clod {

// Blend of one pixel against one staged Gaussian (the decision arithmetic of
// the spec).  Updates T, colour, contributor position; sets done on the stop.
struct Px {
    float T, C0, C1, C2;
    uint32_t last;
    bool done;
};

template <bool COUNT>
__device__ __forceinline__ void blend_one(Px& q, float fpx, float fpy, const float4& a, const float4& c, float cb,
                                          uint32_t pos, unsigned long long& n_exp, unsigned long long& n_con)
{
    const float ddx = __fsub_rn(a.x, fpx), ddy = __fsub_rn(a.y, fpy);
    if (COUNT) {
        const float pw = __fmaf_rn(ddx, __fmaf_rn(a.z, ddx, __fmul_rn(a.w, ddy)), __fmul_rn(__fmul_rn(c.x, ddy), ddy));
        if (pw <= 0.0f && pw >= -5.6f) ++n_exp;
    }
    const float al = blend_alpha(ddx, ddy, a.z, a.w, c.x, c.y);
    if (al < 0.0f) return;
    // contributor or stop, without a second branch: a stopping pixel adds
    // 0 * colour (exact: C + 0 = C) and keeps T and last
    const float tt = __fmul_rn(q.T, __fsub_rn(1.0f, al));
    const bool con = !(tt < 1e-4f);
    const float w = con ? __fmul_rn(al, q.T) : 0.0f;
    q.C0 = __fmaf_rn(c.z, w, q.C0);
    q.C1 = __fmaf_rn(c.w, w, q.C1);
    q.C2 = __fmaf_rn(cb, w, q.C2);
    q.T = con ? tt : q.T;
    q.last = con ? pos : q.last;
    q.done = !con;
    if (COUNT && con) ++n_con;
}

// The contributor/stop update of one pixel whose opacity al passed the skip
// tests (ok): same results as blend_one.  A stopping pixel keeps C, T and
// last (blend_one adds 0 * colour, which leaves the non-negative sums as they
// are).
__device__ __forceinline__ void blend_finish(Px& q, bool ok, float al, const float4& c, float cb, uint32_t pos)
{
    const float tt = __fmul_rn(q.T, __fsub_rn(1.0f, al));
    const bool con = ok && !(tt < 1e-4f);
    if (con) {
        const float w = __fmul_rn(al, q.T);
        q.C0 = __fmaf_rn(c.z, w, q.C0);
        q.C1 = __fmaf_rn(c.w, w, q.C1);
        q.C2 = __fmaf_rn(cb, w, q.C2);
        q.T = tt;
        q.last = pos;
    }
    q.done = q.done || (ok && !con);
}

// Both pixels of a thread against one Gaussian: the two powers, then (if
// either lies in [pf, 0], pf >= -5.6 the Gaussian's power floor) the two
// exponentials side by side, so that their dependency chains interleave.
// Below pf the opacity is < 1/255 (skipped either way): every pixel's result
// is that of blend_one (FAST: with the exponential of CLOD_FAST_EXP).
template <bool FAST>
__device__ __forceinline__ void blend_pair(Px& q0, Px& q1, bool t0, bool t1, float fpx, float fpy0, float fpy1,
                                           const float4& a, const float4& c, float cb, float pf, uint32_t pos)
{
    const float ddx = __fsub_rn(a.x, fpx);
    const float dy0 = __fsub_rn(a.y, fpy0), dy1 = __fsub_rn(a.y, fpy1);
    const float p0 = __fmaf_rn(ddx, __fmaf_rn(a.z, ddx, __fmul_rn(a.w, dy0)), __fmul_rn(__fmul_rn(c.x, dy0), dy0));
    const float p1 = __fmaf_rn(ddx, __fmaf_rn(a.z, ddx, __fmul_rn(a.w, dy1)), __fmul_rn(__fmul_rn(c.x, dy1), dy1));
    const bool r0 = t0 && p0 <= 0.0f && p0 >= pf;
    const bool r1 = t1 && p1 <= 0.0f && p1 >= pf;
    // skipped by the whole warp when no pixel of its patch is in range (a
    // warp-uniform branch); a pixel out of range evaluates its exponential too
    // (its result is dropped: ok below is false)
    if (!__any_sync(0xffffffffu, r0 || r1)) return;
    // (with the hardware exponential a second exponential is cheaper than
    // the vote that would avoid it)
    if (FAST || __any_sync(0xffffffffu, r0 && r1)) {
        const float g0 = blend_exp<FAST>(p0), g1 = blend_exp<FAST>(p1);
        const float a0 = fminf(0.99f, __fmul_rn(c.y, g0)), a1 = fminf(0.99f, __fmul_rn(c.y, g1));
        blend_finish(q0, r0 && !(a0 < (1.0f / 255.0f)), a0, c, cb, pos);
        blend_finish(q1, r1 && !(a1 < (1.0f / 255.0f)), a1, c, cb, pos);
    } else {
        // no lane has both pixels in range: one exponential per lane, for the
        // pixel that is (the same value either pixel would get)
        const float g = blend_exp<FAST>(r0 ? p0 : p1);
        const float al = fminf(0.99f, __fmul_rn(c.y, g));
        const bool ok = !(al < (1.0f / 255.0f));
        blend_finish(q0, r0 && ok, al, c, cb, pos);
        blend_finish(q1, r1 && ok, al, c, cb, pos);
    }
}

__device__ __forceinline__ void store_px(const ViewDev& W, const Px& q, int px, int py, float* image, float* Tout,
                                         uint32_t* ncout)
{
    if (px >= W.W || py >= W.H) return;
    const size_t plane = (size_t)W.W * W.H;
    const size_t p = (size_t)py * W.W + px;
    float* img = W.out_img ? W.out_img : image + 3 * W.pix_base;
    img[p] = __fmaf_rn(q.T, W.bg[0], q.C0);
    img[plane + p] = __fmaf_rn(q.T, W.bg[1], q.C1);
    img[2 * plane + p] = __fmaf_rn(q.T, W.bg[2], q.C2);
    if (W.out_T) W.out_T[p] = q.T;
    else if (Tout) Tout[W.pix_base + p] = q.T;
    if (W.out_nc) W.out_nc[p] = q.last;
    else if (ncout) ncout[W.pix_base + p] = q.last;
}

constexpr int BLEND_THREADS = 128;   // 4 warps per 16x16 tile, 8x8 pixels per warp, 2 per thread
constexpr int BLEND_BLOCKS_PER_SM_MAX = 5;        // resident blocks per SM for small frames
constexpr uint32_t BLEND_SMALL_TILES = 16384;      // tiles of a frame below which that holds

// Each warp takes (tile, 8x8 quarter) work items from an atomic queue and
// walks the tile's list on its own, 32 entries at a time: every lane gathers
// one record and tests its reach box against the warp's patch; the ballot of
// hits is then blended in list order from per-warp shared slots.  A warp
// leaves its patch when all 64 pixels are saturated and takes the next item;
// nothing waits for the other warps of the block.  COUNT: the counting
// variant (every pair visited, software exponential); FAST: the exponential
// of CLOD_FAST_EXP.  Registers for nine blocks per SM (the grid launches at
// most BLEND_BLOCKS_PER_SM_MAX): left to itself, ptxas fits the kernel in 48
// registers with a 4-byte spill inside the list walk, which measured 20 %
// slower over the orbit sweep than 55 registers without one.
template <bool COUNT, bool FAST>
__global__ void __launch_bounds__(BLEND_THREADS, 9) k_blend_fwd(Frame F, const uint32_t* __restrict__ vals,
                                                             const uint32_t* __restrict__ ranges,
                                                             float* __restrict__ image, float* __restrict__ Tout,
                                                             uint32_t* __restrict__ ncout,
                                                             unsigned long long* __restrict__ evaluated)
{
    pdl_wait();
    __shared__ float4 s0[4][32];
    __shared__ float4 s1[4][32];
    __shared__ float4 s2[4][32];
    const FrameHeader* hdr = F.hdr;
    if (hdr->status & STATUS_OVERFLOW) return;
    const uint32_t TT = hdr->total_tiles;
    const uint32_t V = hdr->n_views;
    const int64_t n = static_cast<int64_t>(hdr->n);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned long long evals = 0, n_exp = 0, n_con = 0;
    for (;;) {
        // work item = (tile, quarter): this warp's 8x8 patch of a tile
        uint32_t unit = 0;
        if (lane == 0) unit = atomicAdd(&F.hdr->work[0], 1u);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if ((unit >> 2) >= TT) break;
        const uint32_t t = work_tile(F, unit >> 2, TT);     // longest tile lists first
        const int qd = (int)(unit & 3u);
        int view = 0;
        for (uint32_t u = 1; u < V; ++u)
            if (t >= F.views[u].tile_base) view = (int)u;
        const ViewDev& W = F.views[view];
        const int ox = (qd & 1) * 8 + (lane & 7), oy = (qd >> 1) * 8 + (lane >> 3) * 2;
        const float pcx = (float)((qd & 1) * 8) + 4.0f, pcy = (float)((qd >> 1) * 8) + 4.0f;
        const uint32_t local = t - W.tile_base;
        const int tx = (int)(local % (uint32_t)W.TX), ty = (int)(local / (uint32_t)W.TX);
        const int px = tx * TILE + ox, py0 = ty * TILE + oy, py1 = py0 + 1;
        // pixel centres in full-frame coordinates (a region view is offset by ox, oy)
        const float fpx = __fadd_rn(static_cast<float>(px + W.ox), 0.5f);
        const float fpy0 = __fadd_rn(static_cast<float>(py0 + W.oy), 0.5f);
        const float fpy1 = __fadd_rn(static_cast<float>(py1 + W.oy), 0.5f);
        const float wcx = (float)(tx * TILE + W.ox) + pcx, wcy = (float)(ty * TILE + W.oy) + pcy;
        const uint32_t start = ranges[2 * t], end = ranges[2 * t + 1];
        const int64_t vn = (int64_t)view * n;
        Px q0{1.0f, 0.0f, 0.0f, 0.0f, 0u, !(px < W.W && py0 < W.H)};
        Px q1{1.0f, 0.0f, 0.0f, 0.0f, 0u, !(px < W.W && py1 < W.H)};
        for (uint32_t b = start; b < end; b += 32) {
            if (__all_sync(0xffffffffu, q0.done && q1.done)) break;
            const uint32_t j = b + lane;
            bool hit = false;
            if (j < end) {
                const int64_t g = vn + vals[j];
                const float4 a = F.rec0[g];
                const float4 c = F.rec1[g];
                const float4 e = F.rec2[g];
                s0[wid][lane] = a;
                s1[wid][lane] = c;
                s2[wid][lane] = e;
                // the reach box (stored by the preprocessing) against the warp's 8x8 patch
                if (COUNT) hit = true;
                else hit = !(fabsf(a.x - wcx) > e.y + 3.5f || fabsf(a.y - wcy) > e.z + 3.5f);
            }
            unsigned m = __ballot_sync(0xffffffffu, hit);
            __syncwarp();
            const uint32_t pos0 = b - start + 1u;     // list position (1-based) of entry 0 of the batch
            while (m) {
                const int k = __ffs(m) - 1;
                m &= m - 1;
                const float4 a = s0[wid][k];
                const float4 c = s1[wid][k];
                const float4 e = s2[wid][k];
                const uint32_t pos = pos0 + (uint32_t)k;
                if (COUNT) {
                    if (!q0.done) {
                        ++evals;
                        blend_one<COUNT>(q0, fpx, fpy0, a, c, e.x, pos, n_exp, n_con);
                    }
                    if (!q1.done) {
                        ++evals;
                        blend_one<COUNT>(q1, fpx, fpy1, a, c, e.x, pos, n_exp, n_con);
                    }
                } else {
                    // per pixel, the power floor e.w decides (no box test: the
                    // warp's box test above already passed, and a pixel outside
                    // the reach box has a power below the floor)
                    blend_pair<FAST>(q0, q1, !q0.done, !q1.done, fpx, fpy0, fpy1, a, c, e.x, e.w, pos);
                }
            }
            __syncwarp();
        }
        store_px(W, q0, px, py0, image, Tout, ncout);
        store_px(W, q1, px, py1, image, Tout, ncout);
    }
    // the last warp out resets the tile queue for the next call on this frame
    if (lane == 0) {
        const uint32_t total = gridDim.x * (blockDim.x >> 5);
        if (atomicAdd(&F.hdr->work[3], 1u) == total - 1) {
            F.hdr->work[0] = 0u;
            F.hdr->work[3] = 0u;
        }
    }
    if (COUNT) {
        for (int o = 16; o > 0; o >>= 1) {
            evals += __shfl_xor_sync(0xffffffffu, evals, o);
            n_exp += __shfl_xor_sync(0xffffffffu, n_exp, o);
            n_con += __shfl_xor_sync(0xffffffffu, n_con, o);
        }
        if (lane == 0) {
            atomicAdd(evaluated, evals);
            atomicAdd(evaluated + 1, n_exp);
            atomicAdd(evaluated + 2, n_con);
        }
    }
}

static int g_blend_blocks_per_sm[2] = {0, 0};

cudaError_t render_setup()
{
    int b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_blend_fwd<false, false>, BLEND_THREADS, 0);
    if (e != cudaSuccess) return e;
    g_blend_blocks_per_sm[0] = b > 0 ? b : 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_blend_fwd<false, true>, BLEND_THREADS, 0);
    if (e != cudaSuccess) return e;
    g_blend_blocks_per_sm[1] = b > 0 ? b : 1;
    return cudaSuccess;
}

void launch_blend_fwd(const Frame& F, const uint32_t* vals, const uint32_t* ranges, float* image, float* Tout,
                      uint32_t* ncout, unsigned long long* evaluated, int n_sm, cudaStream_t st, bool fast,
                      uint32_t tiles)
{
    // A frame of fewer than BLEND_SMALL_TILES tiles (one 1080p view) takes at
    // most five resident blocks per SM: the issue-bound blend keeps most of
    // its rate with 20 warps per SM, and the register file it leaves free
    // lets other streams' latency-bound kernels (the preprocessing and sort
    // of frames in flight) run beside it.  Eight 1080p frames in flight over
    // the orbit sweep: 4195 frames/s at nine blocks per SM (its occupancy
    // limit), 4371 at five, 4459 at four; one frame at a time 2094 / 2082 /
    // 2049 (five blocks with the registers of five, 69 instead of 56: 4228 in
    // flight).  Larger frames (training batches, 4K views, eight 4K views)
    // fill the GPU alone and keep every resident block: eight 4K views' blend
    // took 4.85 ms at nine blocks per SM, 5.05 at five.
    const int occ = std::max(1, g_blend_blocks_per_sm[fast ? 1 : 0]);
    const int blocks = n_sm * (tiles < BLEND_SMALL_TILES ? std::min(BLEND_BLOCKS_PER_SM_MAX, occ) : occ);
    if (evaluated)
        launch(k_blend_fwd<true, false>, blocks, BLEND_THREADS, 0, st, F, vals, ranges, image, Tout, ncout, evaluated);
    else if (fast)
        launch(k_blend_fwd<false, true>, blocks, BLEND_THREADS, 0, st, F, vals, ranges, image, Tout, ncout, nullptr);
    else
        launch(k_blend_fwd<false, false>, blocks, BLEND_THREADS, 0, st, F, vals, ranges, image, Tout, ncout, nullptr);
}

}  // namespace clod
