// backward.cu -- hand-written reverse pass of the rasterizer.
//
//   k_blend_bwd      per tile, per pixel, the contributors in reverse order:
//                    T before each one is recovered as T_after / (1 - a);
//                    with the suffix S = sum_{k>j} c_k a_k T_k + T_final bg,
//                    dC/da_j = c_j T_j - S / (1 - a_j) (Eq. 1 differentiated).
//                    The skip decisions are re-taken with the forward's FP32
//                    sequence, so exactly the forward's contributors are
//                    visited.  Per-Gaussian 2D gradients (u, v, A, B, C,
//                    alpha'', r, g, b) are warp-reduced and added with 9
//                    scalar atomics into a per-(view, Gaussian) buffer.
//   k_preprocess_bwd per Gaussian, over the views: chain rule through the
//                    conic (inverse 2D covariance), the EWA Jacobian, the
//                    projection, Sigma = R S S^T R^T, the SH colour and the
//                    attenuated opacity of Eq. 2 (alpha, sigma_d, and mu via
//                    d and d_max); accumulates into the parameter gradients.
//   k_dmax_bwd       the d_max term: d_max = d_{j*} passes the summed
//                    dL/d d_max to mu_{j*}.
#include <algorithm>

#include "clod_internal.cuh"

namespace clod {

struct BwdLayout {
    size_t g2d, dmax_grad, total;
};

BwdLayout bwd_layout(uint64_t n, uint32_t V)
{
    BwdLayout L{};
    size_t o = 0;
    L.g2d = o;
    o += ((size_t)V * n * 3 * sizeof(float4) + 255) & ~size_t(255);
    L.dmax_grad = o;
    o += ((size_t)V * sizeof(float) + 255) & ~size_t(255);
    L.total = o;
    return L;
}

__device__ __forceinline__ float warp_sum(float x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Sum of the 9 values v[0..8] over the 32 lanes of a warp: total 8 by a
// full butterfly (returned in t8 on every lane), totals 0..7 scattered by
// halving exchanges over lane bits 4, 3, 2 and full sums over bits 1, 0:
// afterwards lane l holds the total of value l >> 2.
__device__ __forceinline__ float warp_reduce9(float (&v)[16], float& t8)
{
    const int lane = threadIdx.x & 31;
    float x = v[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    t8 = x;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool hi = lane & 16;
        const float keep = hi ? v[4 + i] : v[i], give = hi ? v[i] : v[4 + i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool hi = lane & 8;
        const float keep = hi ? v[2 + i] : v[i], give = hi ? v[i] : v[2 + i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
    {
        const bool hi = lane & 4;
        const float keep = hi ? v[1] : v[0], give = hi ? v[0] : v[1];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, give, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

struct BPx {
    float T, d0, d1, d2, S0, S1, S2;
    uint32_t last;
    float fy;
};

// Reverse blend of one pixel against one staged Gaussian at list position
// pos (1-based), split in two: the forward's decision arithmetic (explicit
// round-to-nearest intrinsics, never fused: same power, same exponential,
// same skip) in bwd_pair, the gradients in bwd_tail, which adds the pixel's
// 9 gradients into g.
// The gradient part for a pixel whose power is in range (r) and whose
// exponential is G.
__device__ __forceinline__ bool bwd_tail(BPx& q, bool r, float G, float dx, float dy, const float4& a,
                                         const float4& c, float cb, float (&g)[16])
{
    // without branches: a pixel that skips (ok false) adds zeros and keeps its
    // state, which leaves every sum as it was (they are never -0)
    const float raw = __fmul_rn(c.y, G);
    const float al = fminf(0.99f, raw);     // <= 0.99 for any G, so 1 - al >= 0.01
    const bool ok = r && !(al < (1.0f / 255.0f));
    const float iom = __fdividef(1.0f, 1.0f - al);   // fast reciprocal
    const float Tb = q.T * iom;
    const float w = ok ? al * Tb : 0.0f;
    g[6] += w * q.d0;
    g[7] += w * q.d1;
    g[8] += w * q.d2;
    const float dal = q.d0 * (c.z * Tb - q.S0 * iom) + q.d1 * (c.w * Tb - q.S1 * iom) + q.d2 * (cb * Tb - q.S2 * iom);
    q.S0 += c.z * w;
    q.S1 += c.w * w;
    q.S2 += cb * w;
    q.T = ok ? Tb : q.T;
    // alpha = alpha'' G below the 0.99 clamp: gradients through it
    const bool lin = ok && !(raw > 0.99f);
    g[5] += lin ? dal * G : 0.0f;
    const float gp = lin ? dal * al : 0.0f;
    g[0] += gp * (2.0f * a.z * dx + a.w * dy);
    g[1] += gp * (a.w * dx + 2.0f * c.x * dy);
    g[2] += gp * (-0.5f * dx * dx);
    g[3] += gp * (-dx * dy);
    g[4] += gp * (-0.5f * dy * dy);
    return ok;
}

// Both pixels of a thread against one Gaussian (only if not past their last
// contributor), the two exponentials side by side.  Powers below the
// Gaussian's floor pf (>= -5.6) give opacity < 1/255, skipped as in the
// forward pass (FAST: with the exponential of CLOD_FAST_EXP, as the forward).
template <bool FAST>
__device__ __forceinline__ bool bwd_pair(BPx& q0, BPx& q1, bool t0, bool t1, float fpx, const float4& a,
                                         const float4& c, float cb, float pf, uint32_t pos, float (&g)[16])
{
    t0 = t0 && pos <= q0.last;
    t1 = t1 && pos <= q1.last;
    const float dx = __fsub_rn(a.x, fpx);
    const float dy0 = __fsub_rn(a.y, q0.fy), dy1 = __fsub_rn(a.y, q1.fy);
    const float p0 = __fmaf_rn(dx, __fmaf_rn(a.z, dx, __fmul_rn(a.w, dy0)), __fmul_rn(__fmul_rn(c.x, dy0), dy0));
    const float p1 = __fmaf_rn(dx, __fmaf_rn(a.z, dx, __fmul_rn(a.w, dy1)), __fmul_rn(__fmul_rn(c.x, dy1), dy1));
    const bool r0 = t0 && p0 <= 0.0f && p0 >= pf;
    const bool r1 = t1 && p1 <= 0.0f && p1 >= pf;
    // skipped by the whole warp when no pixel is in range (warp-uniform); a
    // pixel out of range evaluates its exponential too (bwd_tail drops it)
    if (!__any_sync(0xffffffffu, r0 || r1)) return false;
    // (with the hardware exponential a second exponential is cheaper than
    // the vote that would avoid it)
    if (FAST || __any_sync(0xffffffffu, r0 && r1)) {
        const float G0 = blend_exp<FAST>(p0), G1 = blend_exp<FAST>(p1);
        bool any = bwd_tail(q0, r0, G0, dx, dy0, a, c, cb, g);
        any |= bwd_tail(q1, r1, G1, dx, dy1, a, c, cb, g);
        return any;
    }
    // no lane has both pixels in range: one exponential and one gradient tail
    // per lane, on the pixel that is in range (the other pixel's tail would
    // add zeros and keep its state); selects, no branches
    const bool s1 = !r0;
    BPx q;
    q.T = s1 ? q1.T : q0.T;
    q.d0 = s1 ? q1.d0 : q0.d0;
    q.d1 = s1 ? q1.d1 : q0.d1;
    q.d2 = s1 ? q1.d2 : q0.d2;
    q.S0 = s1 ? q1.S0 : q0.S0;
    q.S1 = s1 ? q1.S1 : q0.S1;
    q.S2 = s1 ? q1.S2 : q0.S2;
    const float G = blend_exp<FAST>(s1 ? p1 : p0);
    const bool any = bwd_tail(q, r0 || r1, G, dx, s1 ? dy1 : dy0, a, c, cb, g);
    q0.T = s1 ? q0.T : q.T;
    q0.S0 = s1 ? q0.S0 : q.S0;
    q0.S1 = s1 ? q0.S1 : q.S1;
    q0.S2 = s1 ? q0.S2 : q.S2;
    q1.T = s1 ? q.T : q1.T;
    q1.S0 = s1 ? q.S0 : q1.S0;
    q1.S1 = s1 ? q.S1 : q1.S1;
    q1.S2 = s1 ? q.S2 : q1.S2;
    return any;
}

constexpr int BWD_THREADS = 128;   // 4 warps per tile, 8x8 pixels per warp, 2 per thread

template <bool FAST>
__global__ void __launch_bounds__(BWD_THREADS, 6) k_blend_bwd(Frame F, const uint32_t* __restrict__ vals,
                                                           const uint32_t* __restrict__ ranges,
                                                           const float* __restrict__ Tfin,
                                                           const uint32_t* __restrict__ ncon,
                                                           const float* __restrict__ dimg, float* __restrict__ g2d)
{
    pdl_wait();
    __shared__ float4 s0[4][32];
    __shared__ float4 s1[4][32];
    __shared__ float4 s2[4][32];
    __shared__ int64_t sg[4][32];
    const FrameHeader* hdr = F.hdr;
    if (hdr->status & STATUS_OVERFLOW) return;
    const uint32_t TT = hdr->total_tiles;
    const uint32_t V = hdr->n_views;
    const int64_t n = static_cast<int64_t>(hdr->n);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        // work item = (tile, quarter): this warp's 8x8 patch of a tile
        uint32_t unit = 0;
        if (lane == 0) unit = atomicAdd(&F.hdr->work[1], 1u);
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
        const int px = tx * TILE + ox;
        const float fpx = __fadd_rn(static_cast<float>(px + W.ox), 0.5f);
        const float wcx = (float)(tx * TILE + W.ox) + pcx, wcy = (float)(ty * TILE + W.oy) + pcy;
        const uint32_t start = ranges[2 * t];
        const int64_t vn = (int64_t)view * n;
        BPx q[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int py = ty * TILE + oy + r;
            q[r].fy = __fadd_rn(static_cast<float>(py + W.oy), 0.5f);
            q[r].T = 1.0f;
            q[r].d0 = q[r].d1 = q[r].d2 = q[r].S0 = q[r].S1 = q[r].S2 = 0.0f;
            q[r].last = 0;
            if (px < W.W && py < W.H) {
                const size_t plane = (size_t)W.W * W.H, p = (size_t)py * W.W + px;
                q[r].T = Tfin[W.pix_base + p];
                q[r].last = ncon[W.pix_base + p];
                const float* di = dimg + 3 * W.pix_base;
                q[r].d0 = di[p];
                q[r].d1 = di[plane + p];
                q[r].d2 = di[2 * plane + p];
                q[r].S0 = q[r].T * W.bg[0];
                q[r].S1 = q[r].T * W.bg[1];
                q[r].S2 = q[r].T * W.bg[2];
            }
        }
        // walk from this warp's last contributor back to the start
        uint32_t m = max(q[0].last, q[1].last);
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        for (uint32_t hi = m; hi > 0;) {
            const uint32_t lo = hi > 32 ? hi - 32 : 0;     // positions [lo, hi), 0-based
            const uint32_t j = lo + lane;
            bool hit = false;
            if (j < hi) {
                const int64_t g = vn + vals[start + j];
                const float4 a = F.rec0[g];
                const float4 c = F.rec1[g];
                s0[wid][lane] = a;
                s1[wid][lane] = c;
                const float4 e = F.rec2[g];
                s2[wid][lane] = e;
                sg[wid][lane] = g;
                hit = !(fabsf(a.x - wcx) > e.y + 3.5f || fabsf(a.y - wcy) > e.z + 3.5f);
            }
            unsigned bm = __ballot_sync(0xffffffffu, hit);
            __syncwarp();
            while (bm) {
                const int k = 31 - __clz(bm);         // highest position first
                bm &= ~(1u << k);
                const float4 a = s0[wid][k];
                const float4 c = s1[wid][k];
                const float4 e = s2[wid][k];
                const uint32_t pos = lo + (uint32_t)k + 1u;
                float g[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) g[i] = 0.0f;
                // per pixel, the power floor e.w decides, as in the forward pass
                const bool any = bwd_pair<FAST>(q[0], q[1], true, true, fpx, a, c, e.x, e.w, pos, g);
                if (__any_sync(0xffffffffu, any)) {
                    float t8;
                    const float tot = warp_reduce9(g, t8);
                    if (!(lane & 3)) atomicAdd(g2d + 12 * sg[wid][k] + (lane >> 2), tot);
                    else if (lane == 1) atomicAdd(g2d + 12 * sg[wid][k] + 8, t8);
                }
            }
            __syncwarp();
            hi = lo;
        }
    }
}

// Real SH basis function k (colour-model signs) at unit direction (x, y, z)
// and its partial derivatives; xx, yy, zz are the squares.
__device__ __forceinline__ void sh_term(int k, float x, float y, float z, float xx, float yy, float zz, float& b,
                                        float& bx, float& by, float& bz)
{
    const float C1 = CLOD_SH_C1;
    bx = by = bz = 0.f;
    switch (k) {
    case 0: b = CLOD_SH_C0; break;
    case 1: b = -C1 * y; by = -C1; break;
    case 2: b = C1 * z; bz = C1; break;
    case 3: b = -C1 * x; bx = -C1; break;
    case 4: b = CLOD_SH_C2_0 * x * y; bx = CLOD_SH_C2_0 * y; by = CLOD_SH_C2_0 * x; break;
    case 5: b = CLOD_SH_C2_1 * y * z; by = CLOD_SH_C2_1 * z; bz = CLOD_SH_C2_1 * y; break;
    case 6:
        b = CLOD_SH_C2_2 * (2.f * zz - xx - yy);
        bx = -2.f * CLOD_SH_C2_2 * x; by = -2.f * CLOD_SH_C2_2 * y; bz = 4.f * CLOD_SH_C2_2 * z;
        break;
    case 7: b = CLOD_SH_C2_3 * x * z; bx = CLOD_SH_C2_3 * z; bz = CLOD_SH_C2_3 * x; break;
    case 8: b = CLOD_SH_C2_4 * (xx - yy); bx = 2.f * CLOD_SH_C2_4 * x; by = -2.f * CLOD_SH_C2_4 * y; break;
    case 9:
        b = CLOD_SH_C3_0 * y * (3.f * xx - yy);
        bx = 6.f * CLOD_SH_C3_0 * x * y; by = CLOD_SH_C3_0 * (3.f * xx - 3.f * yy);
        break;
    case 10:
        b = CLOD_SH_C3_1 * x * y * z;
        bx = CLOD_SH_C3_1 * y * z; by = CLOD_SH_C3_1 * x * z; bz = CLOD_SH_C3_1 * x * y;
        break;
    case 11:
        b = CLOD_SH_C3_2 * y * (4.f * zz - xx - yy);
        bx = -2.f * CLOD_SH_C3_2 * x * y; by = CLOD_SH_C3_2 * (4.f * zz - xx - 3.f * yy);
        bz = 8.f * CLOD_SH_C3_2 * y * z;
        break;
    case 12:
        b = CLOD_SH_C3_3 * z * (2.f * zz - 3.f * xx - 3.f * yy);
        bx = -6.f * CLOD_SH_C3_3 * x * z; by = -6.f * CLOD_SH_C3_3 * y * z;
        bz = CLOD_SH_C3_3 * (6.f * zz - 3.f * xx - 3.f * yy);
        break;
    case 13:
        b = CLOD_SH_C3_4 * x * (4.f * zz - xx - yy);
        bx = CLOD_SH_C3_4 * (4.f * zz - 3.f * xx - yy); by = -2.f * CLOD_SH_C3_4 * x * y;
        bz = 8.f * CLOD_SH_C3_4 * x * z;
        break;
    case 14:
        b = CLOD_SH_C3_5 * z * (xx - yy);
        bx = 2.f * CLOD_SH_C3_5 * x * z; by = -2.f * CLOD_SH_C3_5 * y * z; bz = CLOD_SH_C3_5 * (xx - yy);
        break;
    default:
        b = CLOD_SH_C3_6 * x * (xx - 3.f * yy);
        bx = CLOD_SH_C3_6 * (3.f * xx - 3.f * yy); by = -6.f * CLOD_SH_C3_6 * x * y;
        break;
    }
}

// dst = x (SET) or dst += x.
template <bool SET>
__device__ __forceinline__ void put(float& dst, float x)
{
    if (SET) dst = x;
    else dst += x;
}

// Rotation matrix (row-major) of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void rotation(float qw, float qx, float qy, float qz, float (&r)[9])
{
    r[0] = 1.f - 2.f * (qy * qy + qz * qz);
    r[1] = 2.f * (qx * qy - qw * qz);
    r[2] = 2.f * (qx * qz + qw * qy);
    r[3] = 2.f * (qx * qy + qw * qz);
    r[4] = 1.f - 2.f * (qx * qx + qz * qz);
    r[5] = 2.f * (qy * qz - qw * qx);
    r[6] = 2.f * (qx * qz - qw * qy);
    r[7] = 2.f * (qy * qz + qw * qx);
    r[8] = 1.f - 2.f * (qx * qx + qy * qy);
}

// Index of entry (a, b) of a symmetric 3x3 matrix stored as its upper
// triangle: 00 01 02 11 12 22.
__host__ __device__ constexpr int sym3(int a, int b)
{
    return a <= b ? (a == 0 ? b : (a == 1 ? 2 + b : 5)) : (b == 0 ? a : (b == 1 ? 2 + a : 5));
}

struct ParamGrads {
    float* dmeans;
    float* dscales;
    float* dquats;
    float* dopacity;
    float* dsh;
    float* ddecay;
};

// SET: the parameter gradients are overwritten (every element written,
// zeros where the Gaussian survives in no view) instead of accumulated.
template <int DEG, bool SET>
__global__ void __launch_bounds__(128, 5) k_preprocess_bwd(Frame F, clod_scene S, const float4* __restrict__ g2d,
                                                        const float* __restrict__ g_alpha_ext,
                                                        const float* __restrict__ g_alpha_view,
                                                        float* __restrict__ dmax_grad, ParamGrads P)
{
    pdl_wait();
    __shared__ ViewDev sv[MAX_VIEWS];
    __shared__ float sdmax[MAX_VIEWS];
    __shared__ float sdmg[MAX_VIEWS];
    __shared__ float sgav[MAX_VIEWS];
    // each thread's SH gradient summed over the views, element-major (no bank
    // conflicts); added to the gradient buffer once per Gaussian
    __shared__ float s_dsh[48][129];     // padded: the warps' row-wise read-out is conflict free
    const uint32_t V = F.hdr->n_views;
    {
        const int words = static_cast<int>(V * sizeof(ViewDev) / 4);
        const int* src = reinterpret_cast<const int*>(F.views);
        int* dst = reinterpret_cast<int*>(sv);
        for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
        for (uint32_t v = threadIdx.x; v < V; v += blockDim.x) {
            sdmax[v] = decode_dmax(F.dmax_key[v]);
            sdmg[v] = 0.f;
            sgav[v] = g_alpha_view ? g_alpha_view[v] : 0.f;
        }
    }
    __syncthreads();
    const int64_t n = S.n;
    constexpr int K = (DEG + 1) * (DEG + 1);
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const bool active = i < n;
        float gm0 = 0.f, gm1 = 0.f, gm2 = 0.f, gop = 0.f, gdec = 0.f;
        // Sigma (upper triangle, sym3 order) from the first surviving view
        // on, and the sum over the views of dL/dSigma + its transpose: the
        // chain through M = R(q) diag(s) is linear in it, so it runs once
        // per Gaussian after the views
        bool geo = false;
        float Sg[6], gSy[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) Sg[k] = gSy[k] = 0.f;
        float mx = 0.f, my = 0.f, mz = 0.f, alpha = 0.f, sigma = 0.f;
        bool sh_any = false;
        if (active) {
            mx = S.means[3 * i];
            my = S.means[3 * i + 1];
            mz = S.means[3 * i + 2];
            alpha = S.opacity[i];
            sigma = S.decay[i];
        }
        for (uint32_t v = 0; v < V; ++v) {
            if (!active) break;
            const ViewDev& W = sv[v];
            const int64_t o = (int64_t)v * n + i;
            const uint2 rc = F.rect[o];
            const bool surv = (rc.y & 0xFFFFu) > (rc.x & 0xFFFFu);
            float g_a2 = (g_alpha_ext ? g_alpha_ext[o] : 0.f) + sgav[v];
            float e0, e1, e2;
            const float d = cam_dist(W, mx, my, mz, e0, e1, e2);
            if (surv) {
                const float4 G0 = g2d[3 * o], G1 = g2d[3 * o + 1];
                const float Gb = g2d[3 * o + 2].x;
                const float g_u = G0.x, g_v = G0.y, g_A = G0.z, g_B = G0.w, g_C = G1.x;
                g_a2 += G1.y;
                const float g_col[3] = {G1.z, G1.w, Gb};
                // the forward's clamped colours: max(SH + 0.5, 0) > 0 is the
                // forward's own decision of whether the clamp was inactive
                const float4 R1 = F.rec1[o];
                const float col[3] = {R1.z, R1.w, F.rec2[o].x};
                // ---- colour (SH) -------------------------------------------------
                const float inv_d = 1.0f / d;
                const float dx = e0 * inv_d, dy = e1 * inv_d, dz = e2 * inv_d;
                const float* shp = S.sh + (size_t)i * K * 3;
                // gradient reaching each channel's SH sum (0 where the clamp held)
                const float gc0 = col[0] > 0.0f ? g_col[0] : 0.0f;
                const float gc1 = col[1] > 0.0f ? g_col[1] : 0.0f;
                const float gc2 = col[2] > 0.0f ? g_col[2] : 0.0f;
                float gdx = 0.f, gdy = 0.f, gdz = 0.f;
                if (gc0 != 0.0f || gc1 != 0.0f || gc2 != 0.0f) {
                    if (!sh_any) {
#pragma unroll
                        for (int j = 0; j < 3 * K; ++j) s_dsh[j][threadIdx.x] = 0.0f;
                        sh_any = true;
                    }
                    const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
                    // one basis function and its direction derivatives at a
                    // time (k is a compile-time constant after unrolling)
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        float bk, bxk, byk, bzk;
                        sh_term(k, dx, dy, dz, xx, yy, zz, bk, bxk, byk, bzk);
                        const float s = __ldg(shp + 3 * k) * gc0 + __ldg(shp + 3 * k + 1) * gc1 +
                                        __ldg(shp + 3 * k + 2) * gc2;
                        gdx += bxk * s;
                        gdy += byk * s;
                        gdz += bzk * s;
                        s_dsh[3 * k][threadIdx.x] += bk * gc0;
                        s_dsh[3 * k + 1][threadIdx.x] += bk * gc1;
                        s_dsh[3 * k + 2][threadIdx.x] += bk * gc2;
                    }
                }
                // direction = e / |e|
                const float dotg = gdx * dx + gdy * dy + gdz * dz;
                gm0 += (gdx - dx * dotg) * inv_d;
                gm1 += (gdy - dy * dotg) * inv_d;
                gm2 += (gdz - dz * dotg) * inv_d;

                // ---- Sigma = M M^T, M = R(q) diag(s): the same for every view,
                // formed at the Gaussian's first surviving view ------------------
                if (!geo) {
                    const float4 q = reinterpret_cast<const float4*>(S.quats)[i];
                    const float qn = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
                    float r[9], Mm[9];
                    rotation(q.x / qn, q.y / qn, q.z / qn, q.w / qn, r);
                    const float sc[3] = {S.scales[3 * i], S.scales[3 * i + 1], S.scales[3 * i + 2]};
                    for (int a_ = 0; a_ < 3; ++a_)
                        for (int b_ = 0; b_ < 3; ++b_) Mm[3 * a_ + b_] = r[3 * a_ + b_] * sc[b_];
                    for (int a_ = 0; a_ < 3; ++a_)
                        for (int b_ = a_; b_ < 3; ++b_)
                            Sg[sym3(a_, b_)] = Mm[3 * a_] * Mm[3 * b_] + Mm[3 * a_ + 1] * Mm[3 * b_ + 1] +
                                               Mm[3 * a_ + 2] * Mm[3 * b_ + 2];
                    geo = true;
                }
                // ---- forward recomputation of the projection --------------------
                float tx, ty, tz;
                cam_point(W, mx, my, mz, tx, ty, tz);
                const float limx = 1.3f * (0.5f * (float)W.FW / W.fx), limy = 1.3f * (0.5f * (float)W.FH / W.fy);
                const float txz = tx / tz, tyz = ty / tz;
                const bool clx = txz < -limx || txz > limx, cly = tyz < -limy || tyz > limy;
                const float txc = fminf(limx, fmaxf(-limx, txz)) * tz;
                const float tyc = fminf(limy, fmaxf(-limy, tyz)) * tz;
                const float itz = 1.0f / tz, itz2 = itz * itz;
                const float j00 = W.fx * itz, j02 = -W.fx * txc * itz2;
                const float j11 = W.fy * itz, j12 = -W.fy * tyc * itz2;
                float T0[3], T1[3];
                for (int k = 0; k < 3; ++k) {
                    T0[k] = j00 * W.R[k] + j02 * W.R[6 + k];
                    T1[k] = j11 * W.R[3 + k] + j12 * W.R[6 + k];
                }
                float ST0[3], ST1[3];  // Sigma T0^T, Sigma T1^T
                for (int k = 0; k < 3; ++k) {
                    ST0[k] = Sg[sym3(k, 0)] * T0[0] + Sg[sym3(k, 1)] * T0[1] + Sg[sym3(k, 2)] * T0[2];
                    ST1[k] = Sg[sym3(k, 0)] * T1[0] + Sg[sym3(k, 1)] * T1[1] + Sg[sym3(k, 2)] * T1[2];
                }
                const float ca = T0[0] * ST0[0] + T0[1] * ST0[1] + T0[2] * ST0[2] + 0.3f;
                const float cb = T0[0] * ST1[0] + T0[1] * ST1[1] + T0[2] * ST1[2];
                const float cc = T1[0] * ST1[0] + T1[1] * ST1[1] + T1[2] * ST1[2] + 0.3f;
                const float det = ca * cc - cb * cb;
                const float id = 1.0f / det, id2 = id * id;
                // ---- conic -> 2D covariance --------------------------------------
                const float g_ca = g_A * (-cc * cc * id2) + g_B * (cb * cc * id2) + g_C * (id - ca * cc * id2);
                const float g_cb = g_A * (2.f * cb * cc * id2) + g_B * (-id - 2.f * cb * cb * id2) + g_C * (2.f * ca * cb * id2);
                const float g_cc = g_A * (id - ca * cc * id2) + g_B * (ca * cb * id2) + g_C * (-ca * ca * id2);
                // ---- 2D covariance -> Sigma (summed over the views as the
                // symmetric dL/dSigma + its transpose) and T ----------------------
                for (int k = 0; k < 3; ++k)
                    for (int l = k; l < 3; ++l)
                        gSy[sym3(k, l)] += 2.f * g_ca * T0[k] * T0[l] + g_cb * (T0[k] * T1[l] + T1[k] * T0[l]) +
                                           2.f * g_cc * T1[k] * T1[l];
                float gT0[3], gT1[3];
                for (int k = 0; k < 3; ++k) {
                    gT0[k] = 2.f * g_ca * ST0[k] + g_cb * ST1[k];
                    gT1[k] = 2.f * g_cc * ST1[k] + g_cb * ST0[k];
                }
                // ---- T = J W -> J -> camera point -----------------------------------
                float gj00 = 0.f, gj02 = 0.f, gj11 = 0.f, gj12 = 0.f;
                for (int k = 0; k < 3; ++k) {
                    gj00 += gT0[k] * W.R[k];
                    gj02 += gT0[k] * W.R[6 + k];
                    gj11 += gT1[k] * W.R[3 + k];
                    gj12 += gT1[k] * W.R[6 + k];
                }
                float gtx = 0.f, gty = 0.f, gtz = 0.f;
                gtz += gj00 * (-W.fx * itz2) + gj11 * (-W.fy * itz2);
                if (clx) gtz += gj02 * (W.fx * (txc * itz) * itz2);          // j02 = -fx L / tz
                else {
                    gtx += gj02 * (-W.fx * itz2);
                    gtz += gj02 * (2.f * W.fx * tx * itz2 * itz);
                }
                if (cly) gtz += gj12 * (W.fy * (tyc * itz) * itz2);
                else {
                    gty += gj12 * (-W.fy * itz2);
                    gtz += gj12 * (2.f * W.fy * ty * itz2 * itz);
                }
                // mean2d
                gtx += g_u * W.fx * itz;
                gty += g_v * W.fy * itz;
                gtz += -(g_u * W.fx * tx + g_v * W.fy * ty) * itz2;
                gm0 += W.R[0] * gtx + W.R[3] * gty + W.R[6] * gtz;
                gm1 += W.R[1] * gtx + W.R[4] * gty + W.R[7] * gtz;
                gm2 += W.R[2] * gtx + W.R[5] * gty + W.R[8] * gtz;
            }
            // ---- attenuated opacity (Eq. 2) ----------------------------------------
            if (g_a2 != 0.0f) {
                if (W.flags & CLOD_LOD_OFF) {
                    gop += g_a2;
                } else {
                    const float dmax = sdmax[v];
                    const bool norm = !(W.flags & CLOD_NO_NORMALIZE);
                    const float dn = norm ? (dmax > 0.f ? d / dmax : 0.f) : d;
                    const float sr = sigma > 0.f ? sigma : 0.f;
                    const float D = 2.f * sr * sr + W.eps;
                    const float q = dn * W.s_v;
                    const float x = q * q / D;
                    const float E = exp_spec(-x);
                    const float a2 = alpha * E;
                    gop += g_a2 * E;
                    if (sigma > 0.f) gdec += g_a2 * a2 * x * 4.f * sr / D;
                    const float gdn = g_a2 * a2 * (-2.f * dn * W.s_v * W.s_v / D);
                    float gd = 0.f;
                    if (!norm) gd = gdn;
                    else if (dmax > 0.f) {
                        gd = gdn / dmax;
                        atomicAdd_block(&sdmg[v], -gdn * d / (dmax * dmax));
                    }
                    if (d > 0.f) {
                        gm0 += gd * e0 / d;
                        gm1 += gd * e1 / d;
                        gm2 += gd * e2 / d;
                    }
                }
            }
        }
        if (SET) {
            // the warp's 32 SH gradient rows are contiguous: written by the
            // whole warp, element by element in address order, each element
            // read from its Gaussian's column of s_dsh (zero for a Gaussian
            // whose colour got no gradient)
            constexpr int R = 3 * K;
            const unsigned has = __ballot_sync(0xffffffffu, sh_any);
            const int lane = threadIdx.x & 31, col0 = threadIdx.x & ~31;
            const int64_t i0 = i - lane;
            const int cnt = (int)min((int64_t)32, n - i0);
            __syncwarp();
            float* dst = P.dsh + (size_t)max((int64_t)0, i0) * R;
            for (int e = lane; e < cnt * R; e += 32) {
                const int t = e / R, j = e - t * R;
                dst[e] = ((has >> t) & 1u) ? s_dsh[j][col0 + t] : 0.0f;
            }
            __syncwarp();     // before a lane reuses its column for the next Gaussian
        } else if (sh_any) {
            // added row by row (measured faster than the warp's read-modify-
            // write of whole rows)
            float* dshp = P.dsh + (size_t)i * K * 3;
#pragma unroll
            for (int j = 0; j < 3 * K; ++j) dshp[j] += s_dsh[j][threadIdx.x];
        }
        if (SET && active && !geo) {
            P.dscales[3 * i] = P.dscales[3 * i + 1] = P.dscales[3 * i + 2] = 0.0f;
            P.dquats[4 * i] = P.dquats[4 * i + 1] = P.dquats[4 * i + 2] = P.dquats[4 * i + 3] = 0.0f;
        }
        if (geo) {
            // ---- Sigma = M M^T, M = R(q) diag(s), with the views' summed
            // dL/dSigma + transpose: dM = G M, dR = dM diag(s), ds, dq ----------
            const float4 q = reinterpret_cast<const float4*>(S.quats)[i];
            const float qn = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
            const float qw = q.x / qn, qx = q.y / qn, qy = q.z / qn, qz = q.w / qn;
            float r[9];
            rotation(qw, qx, qy, qz, r);
            const float sc[3] = {S.scales[3 * i], S.scales[3 * i + 1], S.scales[3 * i + 2]};
            float gM[9];
            for (int a_ = 0; a_ < 3; ++a_)
                for (int b_ = 0; b_ < 3; ++b_) {
                    float acc = 0.f;
                    for (int k = 0; k < 3; ++k) acc += gSy[sym3(a_, k)] * (r[3 * k + b_] * sc[b_]);
                    gM[3 * a_ + b_] = acc;
                }
            float gR[9];
            for (int a_ = 0; a_ < 3; ++a_)
                for (int b_ = 0; b_ < 3; ++b_) gR[3 * a_ + b_] = gM[3 * a_ + b_] * sc[b_];
            put<SET>(P.dscales[3 * i], gM[0] * r[0] + gM[3] * r[3] + gM[6] * r[6]);
            put<SET>(P.dscales[3 * i + 1], gM[1] * r[1] + gM[4] * r[4] + gM[7] * r[7]);
            put<SET>(P.dscales[3 * i + 2], gM[2] * r[2] + gM[5] * r[5] + gM[8] * r[8]);
            const float gw = 2.f * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
            const float gx = 2.f * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2.f * qx * gR[4] - qw * gR[5] + qz * gR[6] +
                                    qw * gR[7] - 2.f * qx * gR[8]);
            const float gy = 2.f * (-2.f * qy * gR[0] + qx * gR[1] + qw * gR[2] + qx * gR[3] + qz * gR[5] - qw * gR[6] +
                                    qz * gR[7] - 2.f * qy * gR[8]);
            const float gz = 2.f * (-2.f * qz * gR[0] - qw * gR[1] + qx * gR[2] + qw * gR[3] - 2.f * qz * gR[4] +
                                    qy * gR[5] + qx * gR[6] + qy * gR[7]);
            const float dot = gw * qw + gx * qx + gy * qy + gz * qz;
            put<SET>(P.dquats[4 * i], (gw - qw * dot) / qn);
            put<SET>(P.dquats[4 * i + 1], (gx - qx * dot) / qn);
            put<SET>(P.dquats[4 * i + 2], (gy - qy * dot) / qn);
            put<SET>(P.dquats[4 * i + 3], (gz - qz * dot) / qn);
        }
        if (active) {
            put<SET>(P.dmeans[3 * i], gm0);
            put<SET>(P.dmeans[3 * i + 1], gm1);
            put<SET>(P.dmeans[3 * i + 2], gm2);
            put<SET>(P.dopacity[i], gop);
            put<SET>(P.ddecay[i], gdec);
        }
    }
    __syncthreads();
    for (uint32_t v = threadIdx.x; v < V; v += blockDim.x)
        if (sdmg[v] != 0.f) atomicAdd(&dmax_grad[v], sdmg[v]);
}

// d_max = d_{j*}: dL/dmu_{j*} += (dL/d d_max) (mu_{j*} - c) / d_{j*}.
__global__ void k_dmax_bwd(Frame F, clod_scene S, const float* __restrict__ dmax_grad, float* __restrict__ dmeans)
{
    pdl_wait();
    const uint32_t V = F.hdr->n_views;
    for (uint32_t v = threadIdx.x; v < V; v += blockDim.x) {
        const unsigned long long key = F.dmax_key[v];
        const float g = dmax_grad[v];
        if (!key || g == 0.f) continue;
        const uint32_t j = 0xFFFFFFFFu - static_cast<uint32_t>(key & 0xFFFFFFFFull);
        const ViewDev& W = F.views[v];
        float e0, e1, e2;
        const float d = cam_dist(W, S.means[3 * j], S.means[3 * j + 1], S.means[3 * j + 2], e0, e1, e2);
        if (d > 0.f) {
            atomicAdd(&dmeans[3 * j], g * e0 / d);
            atomicAdd(&dmeans[3 * j + 1], g * e1 / d);
            atomicAdd(&dmeans[3 * j + 2], g * e2 / d);
        }
    }
}

// L1 loss: loss += scale * sum |img - target| / count; grad = scale * sign(img - target) / count.
__global__ void k_l1_loss(const float* __restrict__ img, const float* __restrict__ tgt, int64_t count, float scale,
                          float* __restrict__ loss, float* __restrict__ grad)
{
    pdl_wait();
    float acc = 0.f;
    const float w = scale / static_cast<float>(count);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
        const float dlt = img[k] - tgt[k];
        acc += fabsf(dlt);
        if (grad) grad[k] = dlt > 0.f ? w : (dlt < 0.f ? -w : 0.f);
    }
    acc = warp_sum(acc);
    __shared__ float ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float a = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.f;
        a = warp_sum(a);
        if (threadIdx.x == 0 && loss) atomicAdd(loss, a * w);
    }
}

static int g_bwd_blocks_per_sm = 0;
static int g_pbwd_blocks_per_sm = 0;

cudaError_t backward_setup()
{
    int b = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_blend_bwd<false>, BWD_THREADS, 0);
    if (e != cudaSuccess) return e;
    g_bwd_blocks_per_sm = b > 0 ? b : 1;
    // the degree-3 kernel uses the most registers: its residency bounds the others'
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_preprocess_bwd<3, false>, 128, 0);
    if (e != cudaSuccess) return e;
    g_pbwd_blocks_per_sm = b > 0 ? b : 1;
    return cudaSuccess;
}

void launch_backward(const Frame& F, const clod_scene& S, uint32_t V, const uint32_t* vals, const uint32_t* ranges,
                     const float* Tfin, const uint32_t* ncon, const float* dimg, const float* g_alpha_ext,
                     const float* g_alpha_view, void* bwd_ws, float* dmeans, float* dscales, float* dquats, float* dopacity, float* dsh,
                     float* ddecay, int n_sm, cudaStream_t st, bool fast, bool set)
{
    const BwdLayout L = bwd_layout((uint64_t)S.n, V);
    char* b = static_cast<char*>(bwd_ws);
    float4* g2d = reinterpret_cast<float4*>(b + L.g2d);
    float* dmg = reinterpret_cast<float*>(b + L.dmax_grad);
    cudaMemsetAsync(bwd_ws, 0, L.total, st);
    cudaMemsetAsync(&F.hdr->work[1], 0, sizeof(uint32_t), st);
    if (fast)
        launch(k_blend_bwd<true>, n_sm * std::max(1, g_bwd_blocks_per_sm), BWD_THREADS, 0, st, F, vals, ranges, Tfin,
               ncon, dimg, reinterpret_cast<float*>(g2d));
    else
        launch(k_blend_bwd<false>, n_sm * std::max(1, g_bwd_blocks_per_sm), BWD_THREADS, 0, st, F, vals, ranges, Tfin,
               ncon, dimg, reinterpret_cast<float*>(g2d));
    ParamGrads P{dmeans, dscales, dquats, dopacity, dsh, ddecay};
    // one resident wave (the loop strides over the rest): each block walks many
    // Gaussians, so the uneven ends of its warps' walks weigh little
    int blocks = static_cast<int>(std::min<int64_t>((S.n + 127) / 128, (int64_t)n_sm * std::max(1, g_pbwd_blocks_per_sm)));
    if (blocks < 1) blocks = 1;
    if (S.n > 0) {
        if (set) {
            switch (S.sh_degree) {
            case 0: launch(k_preprocess_bwd<0, true>, blocks, 128, 0, st, F, S, g2d, g_alpha_ext, g_alpha_view, dmg, P); break;
            case 1: launch(k_preprocess_bwd<1, true>, blocks, 128, 0, st, F, S, g2d, g_alpha_ext, g_alpha_view, dmg, P); break;
            case 2: launch(k_preprocess_bwd<2, true>, blocks, 128, 0, st, F, S, g2d, g_alpha_ext, g_alpha_view, dmg, P); break;
            default: launch(k_preprocess_bwd<3, true>, blocks, 128, 0, st, F, S, g2d, g_alpha_ext, g_alpha_view, dmg, P); break;
            }
        } else {
            switch (S.sh_degree) {
            case 0: launch(k_preprocess_bwd<0, false>, blocks, 128, 0, st, F, S, g2d, g_alpha_ext, g_alpha_view, dmg, P); break;
            case 1: launch(k_preprocess_bwd<1, false>, blocks, 128, 0, st, F, S, g2d, g_alpha_ext, g_alpha_view, dmg, P); break;
            case 2: launch(k_preprocess_bwd<2, false>, blocks, 128, 0, st, F, S, g2d, g_alpha_ext, g_alpha_view, dmg, P); break;
            default: launch(k_preprocess_bwd<3, false>, blocks, 128, 0, st, F, S, g2d, g_alpha_ext, g_alpha_view, dmg, P); break;
            }
        }
    }
    launch(k_dmax_bwd, 1, 64, 0, st, F, S, dmg, dmeans);
}

size_t backward_ws_bytes(uint64_t n, uint32_t V) { return bwd_layout(n, V).total; }

void launch_l1(const float* img, const float* tgt, int64_t count, float scale, float* loss, float* grad, int n_sm,
               cudaStream_t st)
{
    int blocks = static_cast<int>(std::min<int64_t>((count + 255) / 256, (int64_t)n_sm * 4));
    if (blocks < 1) blocks = 1;
    launch(k_l1_loss, blocks, 256, 0, st, img, tgt, count, scale, loss, grad);
}

}  // namespace clod
