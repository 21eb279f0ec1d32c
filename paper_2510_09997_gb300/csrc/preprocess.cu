// preprocess.cu -- per-Gaussian stage of the CLoD-GS rasterizer.
//
//   k_dist_max   d_i = |mu_i - c| and the max of d over the view frustum
//                (Sec. 3.2), with the lowest index among ties.
//   k_preprocess attenuated opacity alpha'' (Eq. 2) and the mask
//                M_i = alpha'' > tau s_v (Sec. 3.2); for survivors the EWA
//                projection, conic, 3-sigma radius, tile rectangle, depth and
//                SH colour (Sec. 3.1); the depth key of every (view,
//                Gaussian) for the depth-rank sort (all ones when culled)
//                and K, the sum of the tiles touched.
//
// Layout: scene arrays are read structure-of-arrays, one Gaussian per thread,
// consecutive Gaussians in consecutive threads (coalesced 12/16-byte rows);
// SH rows (up to 192 B) are read only for survivors.  Outputs are
// view-major [v * n + i].
#include <algorithm>

#include "clod_internal.cuh"

namespace clod {

__device__ __forceinline__ void load_views(ViewDev* sv, const ViewDev* views, uint32_t V)
{
    const int words = static_cast<int>(V * sizeof(ViewDev) / 4);
    const int* src = reinterpret_cast<const int*>(views);
    int* dst = reinterpret_cast<int*>(sv);
    for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long x)
{
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y > x ? y : x;
    }
    return x;
}

// Pass A.  Key = (bits(d) << 32) | (0xFFFFFFFF - i): the max key carries the
// max distance (d >= 0, so its bits order like the value) and, among equal
// distances, the lowest index.  0 means "no Gaussian in the frustum".
__global__ void __launch_bounds__(256) k_dist_max(Frame F, const float* __restrict__ means, int64_t n)
{
    pdl_wait();
    const uint32_t V = F.hdr->n_views;
    __shared__ ViewDev sv[MAX_VIEWS];
    __shared__ unsigned long long wmax[8];
    load_views(sv, F.views, V);
    __syncthreads();
    for (uint32_t v = 0; v < V; ++v) {
        const ViewDev& W = sv[v];
        unsigned long long best = 0ull;
        // DM Gaussians per thread and round, their loads issued together
        constexpr int DM = 4;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += DM * stride) {
            float x[DM], y[DM], z[DM];
#pragma unroll
            for (int u = 0; u < DM; ++u) {
                const int64_t i = i0 + u * stride;
                x[u] = y[u] = z[u] = 0.0f;
                if (i < n) {
                    x[u] = means[3 * i];
                    y[u] = means[3 * i + 1];
                    z[u] = means[3 * i + 2];
                }
            }
#pragma unroll
            for (int u = 0; u < DM; ++u) {
                const int64_t i = i0 + u * stride;
                float tx, ty, tz, e0, e1, e2;
                cam_point(W, x[u], y[u], z[u], tx, ty, tz);
                const float d = cam_dist(W, x[u], y[u], z[u], e0, e1, e2);
                if (i < n && in_frustum(W, tx, ty, tz)) {
                    const unsigned long long key =
                        (static_cast<unsigned long long>(__float_as_uint(d)) << 32) |
                        static_cast<unsigned long long>(0xFFFFFFFFu - static_cast<uint32_t>(i));
                    best = key > best ? key : best;
                }
            }
        }
        best = warp_max_u64(best);
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = best;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned long long b = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0ull;
            b = warp_max_u64(b);
            if (threadIdx.x == 0 && b) atomicMax(&F.dmax_key[v], b);
        }
        __syncthreads();
    }
}

// Pass A for 2..MV views: each thread reads the centres of DM Gaussians
// once and tests them against every view in turn (one view's camera in
// registers at a time); its per-view maxima live in its own column of
// shared memory.  The same keys and maxima as k_dist_max.
template <int MV>
__global__ void __launch_bounds__(256) k_dist_max_views(Frame F, const float* __restrict__ means, int64_t n)
{
    pdl_wait();
    const uint32_t V = F.hdr->n_views;
    __shared__ ViewDev sv[MV];
    __shared__ unsigned long long s_best[MV][256];
    load_views(sv, F.views, V);
    for (uint32_t v = 0; v < V; ++v) s_best[v][threadIdx.x] = 0ull;
    __syncthreads();
    constexpr int DM = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < n; i0 += DM * stride) {
        float x[DM], y[DM], z[DM];
#pragma unroll
        for (int u = 0; u < DM; ++u) {
            const int64_t i = i0 + u * stride;
            x[u] = y[u] = z[u] = 0.0f;
            if (i < n) {
                x[u] = means[3 * i];
                y[u] = means[3 * i + 1];
                z[u] = means[3 * i + 2];
            }
        }
#pragma unroll 1
        for (uint32_t v = 0; v < V; ++v) {
            const ViewDev& W = sv[v];
            unsigned long long best = s_best[v][threadIdx.x];
#pragma unroll
            for (int u = 0; u < DM; ++u) {
                const int64_t i = i0 + u * stride;
                float tx, ty, tz, e0, e1, e2;
                cam_point(W, x[u], y[u], z[u], tx, ty, tz);
                const float d = cam_dist(W, x[u], y[u], z[u], e0, e1, e2);
                if (i < n && in_frustum(W, tx, ty, tz)) {
                    const unsigned long long key =
                        (static_cast<unsigned long long>(__float_as_uint(d)) << 32) |
                        static_cast<unsigned long long>(0xFFFFFFFFu - static_cast<uint32_t>(i));
                    best = key > best ? key : best;
                }
            }
            s_best[v][threadIdx.x] = best;
        }
    }
    __syncthreads();
    // per view: warp maxima, then one warp over the block's eight
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (uint32_t v = (uint32_t)w; v < V; v += blockDim.x >> 5) {
        unsigned long long b = 0ull;
        for (int t = lane; t < (int)blockDim.x; t += 32) b = s_best[v][t] > b ? s_best[v][t] : b;
        b = warp_max_u64(b);
        if (lane == 0 && b) atomicMax(&F.dmax_key[v], b);
    }
}

// Pass B (DEG: the scene's SH degree, so the basis stays in registers).
template <int DEG>
__global__ void __launch_bounds__(256, 4) k_preprocess(Frame F, clod_scene S, uint8_t* __restrict__ mask_out,
                                                    float* __restrict__ alpha_out,
                                                    unsigned long long* __restrict__ n_pairs_out)
{
    pdl_wait();
    const uint32_t V = F.hdr->n_views;
    __shared__ ViewDev sv[MAX_VIEWS];
    __shared__ float sdmax[MAX_VIEWS];
    __shared__ unsigned long long sT[MAX_VIEWS];
    __shared__ uint32_t cnt_mask[MAX_VIEWS], cnt_surv[MAX_VIEWS];
    __shared__ unsigned long long s_pairs;
    load_views(sv, F.views, V);
    for (uint32_t v = threadIdx.x; v < V; v += blockDim.x) {
        sdmax[v] = decode_dmax(F.dmax_key[v]);
        sT[v] = F.sel[v].T;
        cnt_mask[v] = 0;
        cnt_surv[v] = 0;
    }
    if (threadIdx.x == 0) s_pairs = 0ull;
    __syncthreads();
    unsigned long long my_pairs = 0ull;
    const int64_t n = S.n;
    constexpr int K = (DEG + 1) * (DEG + 1);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // the next Gaussian's centre, opacity and decay are loaded one iteration
    // ahead, so that their latency overlaps the current Gaussian's work
    float nmx = 0.f, nmy = 0.f, nmz = 0.f, nalpha = 0.f, nsigma = 0.f;
    {
        const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        if (i < n) {
            nmx = S.means[3 * i];
            nmy = S.means[3 * i + 1];
            nmz = S.means[3 * i + 2];
            nalpha = S.opacity[i];
            nsigma = S.decay[i];
        }
    }
    // block-uniform trip count: every lane reaches the ballots below
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool active = i < n;
        const float mx = nmx, my = nmy, mz = nmz, alpha = nalpha, sigma = nsigma;
        if (i + stride < n) {
            const int64_t j = i + stride;
            nmx = S.means[3 * j];
            nmy = S.means[3 * j + 1];
            nmz = S.means[3 * j + 2];
            nalpha = S.opacity[j];
            nsigma = S.decay[j];
        }
        for (uint32_t v = 0; v < V; ++v) {
            const ViewDev& W = sv[v];
            const int64_t o = (int64_t)v * n + i;
            float e0, e1, e2;
            const float d = cam_dist(W, mx, my, mz, e0, e1, e2);
            const float a2 = attenuated_opacity(W, alpha, sigma, d, sdmax[v]);
            bool M;
            if (W.budget) M = active && budget_key(a2, static_cast<uint32_t>(i)) >= sT[v];   // top-budget by alpha''
            else M = active && ((W.flags & CLOD_LOD_OFF) ? true : (a2 > __fmul_rn(W.s_v, W.tau)));
            if (active && alpha_out) alpha_out[o] = a2;
            if (active && mask_out) mask_out[o] = M ? 1 : 0;
            uint2 rect = make_uint2(0u, 0u);
            bool surv = false;
            uint32_t dkey = 0xFFFFFFFFu;
            if (M) {
                // rotation and scales in one round trip, before they are needed
                const float4 q = reinterpret_cast<const float4*>(S.quats)[i];
                const float s0 = S.scales[3 * i], s1 = S.scales[3 * i + 1], s2 = S.scales[3 * i + 2];
                float tx, ty, tz;
                cam_point(W, mx, my, mz, tx, ty, tz);
                float u = 0.f, vv = 0.f;
                if (tz > W.near_z) project(W, tx, ty, tz, u, vv);
                const bool ok0 = (tz > W.near_z) && isfinite(u) && isfinite(vv);
                // the SH row is fetched into L2 now, while the covariance is
                // computed, for a centre within a frame-sized margin of the
                // frame (a likely survivor); the loads below then hit L2
                if (ok0 && fabsf(u - 0.5f * W.FW) < 1.5f * W.FW && fabsf(vv - 0.5f * W.FH) < 1.5f * W.FH) {
                    const char* row = reinterpret_cast<const char*>(S.sh + (size_t)i * K * 3);
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(row));
                    if (K * 12 > 64) asm volatile("prefetch.global.L2 [%0];" ::"l"(row + 128));
                }
                // 3D covariance Sigma = R S S^T R^T
                float qw = 0.f, qx = 0.f, qy = 0.f, qz = 0.f;
                bool ok1 = false;
                if (ok0) {
                    const float n2 = __fmaf_rn(q.x, q.x, __fmaf_rn(q.y, q.y, __fmaf_rn(q.z, q.z, __fmul_rn(q.w, q.w))));
                    ok1 = n2 > 0.0f;
                    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
                    qw = __fmul_rn(q.x, inv);
                    qx = __fmul_rn(q.y, inv);
                    qy = __fmul_rn(q.z, inv);
                    qz = __fmul_rn(q.w, inv);
                }
                if (ok1) {
                    const float xx = __fmul_rn(qx, qx), yy = __fmul_rn(qy, qy), zz = __fmul_rn(qz, qz);
                    const float xy = __fmul_rn(qx, qy), xz = __fmul_rn(qx, qz), yz = __fmul_rn(qy, qz);
                    const float wx = __fmul_rn(qw, qx), wy = __fmul_rn(qw, qy), wz = __fmul_rn(qw, qz);
                    float r[9];
                    r[0] = __fmaf_rn(-2.0f, __fadd_rn(yy, zz), 1.0f);
                    r[1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
                    r[2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
                    r[3] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
                    r[4] = __fmaf_rn(-2.0f, __fadd_rn(xx, zz), 1.0f);
                    r[5] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
                    r[6] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
                    r[7] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
                    r[8] = __fmaf_rn(-2.0f, __fadd_rn(xx, yy), 1.0f);
                    float Mm[9];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        Mm[3 * a] = __fmul_rn(r[3 * a], s0);
                        Mm[3 * a + 1] = __fmul_rn(r[3 * a + 1], s1);
                        Mm[3 * a + 2] = __fmul_rn(r[3 * a + 2], s2);
                    }
                    float Sg[9];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = a; b < 3; ++b) {
                            const float val = __fmaf_rn(Mm[3 * a], Mm[3 * b],
                                                        __fmaf_rn(Mm[3 * a + 1], Mm[3 * b + 1],
                                                                  __fmul_rn(Mm[3 * a + 2], Mm[3 * b + 2])));
                            Sg[3 * a + b] = val;
                            Sg[3 * b + a] = val;
                        }
                    // EWA: cov2D = J W Sigma W^T J^T + 0.3 I
                    const float Wf = static_cast<float>(W.FW), Hf = static_cast<float>(W.FH);
                    const float limx = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, Wf), W.fx));
                    const float limy = __fmul_rn(1.3f, __fdiv_rn(__fmul_rn(0.5f, Hf), W.fy));
                    const float txc = __fmul_rn(fminf(limx, fmaxf(-limx, __fdiv_rn(tx, tz))), tz);
                    const float tyc = __fmul_rn(fminf(limy, fmaxf(-limy, __fdiv_rn(ty, tz))), tz);
                    const float tz2 = __fmul_rn(tz, tz);
                    const float j00 = __fdiv_rn(W.fx, tz), j02 = __fdiv_rn(-__fmul_rn(W.fx, txc), tz2);
                    const float j11 = __fdiv_rn(W.fy, tz), j12 = __fdiv_rn(-__fmul_rn(W.fy, tyc), tz2);
                    float T0[3], T1[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        T0[k] = __fmaf_rn(j00, W.R[k], __fmul_rn(j02, W.R[6 + k]));
                        T1[k] = __fmaf_rn(j11, W.R[3 + k], __fmul_rn(j12, W.R[6 + k]));
                    }
                    float U0[3], U1[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        U0[k] = __fmaf_rn(T0[0], Sg[k], __fmaf_rn(T0[1], Sg[3 + k], __fmul_rn(T0[2], Sg[6 + k])));
                        U1[k] = __fmaf_rn(T1[0], Sg[k], __fmaf_rn(T1[1], Sg[3 + k], __fmul_rn(T1[2], Sg[6 + k])));
                    }
                    const float ca = __fadd_rn(__fmaf_rn(U0[0], T0[0], __fmaf_rn(U0[1], T0[1], __fmul_rn(U0[2], T0[2]))), 0.3f);
                    const float cb = __fmaf_rn(U0[0], T1[0], __fmaf_rn(U0[1], T1[1], __fmul_rn(U0[2], T1[2])));
                    const float cc = __fadd_rn(__fmaf_rn(U1[0], T1[0], __fmaf_rn(U1[1], T1[1], __fmul_rn(U1[2], T1[2]))), 0.3f);
                    const float det = __fmaf_rn(ca, cc, -__fmul_rn(cb, cb));
                    if (det > 0.0f) {
                        const float idet = __fdiv_rn(1.0f, det);
                        const float A = __fmul_rn(cc, idet), B = __fmul_rn(-cb, idet), C = __fmul_rn(ca, idet);
                        // 3-sigma radius and tile rectangle
                        const float mid = __fmul_rn(0.5f, __fadd_rn(ca, cc));
                        const float disc = fmaxf(0.1f, __fmaf_rn(mid, mid, -det));
                        const float lam = __fadd_rn(mid, __fsqrt_rn(disc));
                        const float rad = ceilf(__fmul_rn(3.0f, __fsqrt_rn(lam)));
                        const float fx0 = floorf(__fmul_rn(__fsub_rn(u, rad), 0.0625f));
                        const float fx1 = floorf(__fmul_rn(__fadd_rn(u, rad), 0.0625f));
                        const float fy0 = floorf(__fmul_rn(__fsub_rn(vv, rad), 0.0625f));
                        const float fy1 = floorf(__fmul_rn(__fadd_rn(vv, rad), 0.0625f));
                        // tile rectangle in the full frame, then within this view's window
                        const int FTX = (W.FW + TILE - 1) / TILE, FTY = (W.FH + TILE - 1) / TILE;
                        const float TXm = static_cast<float>(FTX) - 1.0f, TYm = static_cast<float>(FTY) - 1.0f;
                        const int wx = W.ox / TILE, wy = W.oy / TILE;
                        int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
                        if (!(fx1 < 0.0f || fx0 > TXm || fy1 < 0.0f || fy0 > TYm)) {
                            x0 = max(fx0 < 0.0f ? 0 : static_cast<int>(fx0), wx) - wx;
                            x1 = min(fx1 > TXm ? FTX : static_cast<int>(fx1) + 1, wx + W.TX) - wx;
                            y0 = max(fy0 < 0.0f ? 0 : static_cast<int>(fy0), wy) - wy;
                            y1 = min(fy1 > TYm ? FTY : static_cast<int>(fy1) + 1, wy + W.TY) - wy;
                        }
                        if (x0 < x1 && y0 < y1) {
                            // colour from SH at direction (mu - c) / d
                            const float dx = __fdiv_rn(e0, d), dy = __fdiv_rn(e1, d), dz = __fdiv_rn(e2, d);
                            float bsh[16];
                            sh_basis(dx, dy, dz, DEG, bsh);
                            const float* shp = S.sh + (size_t)i * K * 3;
                            float c0 = __fmul_rn(bsh[0], shp[0]);
                            float c1 = __fmul_rn(bsh[0], shp[1]);
                            float c2 = __fmul_rn(bsh[0], shp[2]);
                            if (DEG == 3) {
                                const float4* s4 = reinterpret_cast<const float4*>(shp);
                                float sh_r[48];
#pragma unroll
                                for (int k = 0; k < 12; ++k) {
                                    const float4 w4 = s4[k];
                                    sh_r[4 * k] = w4.x;
                                    sh_r[4 * k + 1] = w4.y;
                                    sh_r[4 * k + 2] = w4.z;
                                    sh_r[4 * k + 3] = w4.w;
                                }
#pragma unroll
                                for (int k = 1; k < 16; ++k) {
                                    c0 = __fmaf_rn(bsh[k], sh_r[3 * k], c0);
                                    c1 = __fmaf_rn(bsh[k], sh_r[3 * k + 1], c1);
                                    c2 = __fmaf_rn(bsh[k], sh_r[3 * k + 2], c2);
                                }
                            } else {
#pragma unroll
                                for (int k = 1; k < K; ++k) {
                                    c0 = __fmaf_rn(bsh[k], shp[3 * k], c0);
                                    c1 = __fmaf_rn(bsh[k], shp[3 * k + 1], c1);
                                    c2 = __fmaf_rn(bsh[k], shp[3 * k + 2], c2);
                                }
                            }
                            c0 = fmaxf(__fadd_rn(c0, 0.5f), 0.0f);
                            c1 = fmaxf(__fadd_rn(c1, 0.5f), 0.0f);
                            c2 = fmaxf(__fadd_rn(c2, 0.5f), 0.0f);
                            const float nA = __fmul_rn(-0.5f, A), nC = __fmul_rn(-0.5f, C);
                            const float2 ext = reach_half_extents(nA, -B, nC, a2);
                            F.rec0[o] = make_float4(u, vv, nA, -B);
                            F.rec1[o] = make_float4(nC, a2, c0, c1);
                            F.rec2[o] = make_float4(c2, ext.x, ext.y, power_floor(a2));
                            F.depth[o] = tz;
                            dkey = __float_as_uint(tz);
                            rect = make_uint2(static_cast<uint32_t>(x0) | (static_cast<uint32_t>(y0) << 16),
                                              static_cast<uint32_t>(x1) | (static_cast<uint32_t>(y1) << 16));
                            surv = true;
                            my_pairs += (unsigned long long)((x1 - x0) * (y1 - y0));
                        }
                    }
                }
            }
            if (active) {
                F.rect[o] = rect;
                F.key0[o] = dkey;
            }
            // per-view counts: warp-aggregated, then one shared atomic per warp
            const unsigned bm = __ballot_sync(0xffffffffu, M);
            const unsigned bs = __ballot_sync(0xffffffffu, surv);
            if ((threadIdx.x & 31) == 0) {
                if (bm) atomicAdd_block(&cnt_mask[v], __popc(bm));
                if (bs) atomicAdd_block(&cnt_surv[v], __popc(bs));
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) my_pairs += __shfl_xor_sync(0xffffffffu, my_pairs, o);
    if ((threadIdx.x & 31) == 0 && my_pairs) atomicAdd(&s_pairs, my_pairs);
    __syncthreads();
    for (uint32_t v = threadIdx.x; v < V; v += blockDim.x) {
        if (cnt_mask[v]) atomicAdd(&F.n_surv[2 * v], cnt_mask[v]);
        if (cnt_surv[v]) atomicAdd(&F.n_surv[2 * v + 1], cnt_surv[v]);
    }
    if (threadIdx.x == 0 && s_pairs) atomicAdd(&F.hdr->n_pairs, s_pairs);
    if (n_pairs_out) {
        // the last block to finish copies K out (work[2] counts finished blocks)
        __shared__ bool last;
        __threadfence();
        if (threadIdx.x == 0) last = atomicAdd(&F.hdr->work[2], 1u) == gridDim.x - 1;
        __syncthreads();
        if (last && threadIdx.x == 0) {
            __threadfence();
            *n_pairs_out = atomicAdd(&F.hdr->n_pairs, 0ull);
        }
    }
}

// Frame set-up in one launch: the header and the view table arrive as the
// kernel's parameters (no host-to-device copies), and the zero-initialised
// block after the header ([zero_begin, zero_end) bytes of the workspace:
// d_max keys, counts, tile counts) is cleared.
template <int MAXV>
struct SetupArgs {
    FrameHeader h;
    ViewDev views[MAXV];
};

template <int MAXV>
__global__ void __launch_bounds__(256) k_frame_setup(const SetupArgs<MAXV> a, Frame F, char* base, size_t zero_begin,
                                                     size_t zero_end)
{
    pdl_wait();
    uint32_t* z = reinterpret_cast<uint32_t*>(base + zero_begin);
    const size_t words = (zero_end - zero_begin) / 4;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < words; k += (size_t)gridDim.x * blockDim.x)
        z[k] = 0u;
    if (blockIdx.x == 0) {
        if (threadIdx.x == 0) *F.hdr = a.h;
        const int vw = static_cast<int>(a.h.n_views * sizeof(ViewDev) / 4);
        const int* src = reinterpret_cast<const int*>(a.views);
        int* dst = reinterpret_cast<int*>(F.views);
        for (int k = threadIdx.x; k < vw; k += blockDim.x) dst[k] = src[k];
    }
}

template <int MAXV>
static void setup_launch(const Frame& F, void* ws, const FrameHeader& h, const ViewDev* views, size_t zero_begin,
                         size_t zero_end, int n_sm, cudaStream_t st)
{
    SetupArgs<MAXV> a;
    a.h = h;
    for (uint32_t v = 0; v < h.n_views; ++v) a.views[v] = views[v];
    const size_t words = (zero_end - zero_begin) / 4;
    const int blocks = static_cast<int>(std::max<size_t>(1, std::min<size_t>((words + 255) / 256, (size_t)n_sm * 2)));
    launch(k_frame_setup<MAXV>, blocks, 256, 0, st, a, F, static_cast<char*>(ws), zero_begin, zero_end);
}

void launch_frame_setup(const Frame& F, void* ws, const FrameHeader& h, const ViewDev* views, size_t zero_begin,
                        size_t zero_end, int n_sm, cudaStream_t st)
{
    if (h.n_views <= 1) setup_launch<1>(F, ws, h, views, zero_begin, zero_end, n_sm, st);
    else if (h.n_views <= 8) setup_launch<8>(F, ws, h, views, zero_begin, zero_end, n_sm, st);
    else setup_launch<MAX_VIEWS>(F, ws, h, views, zero_begin, zero_end, n_sm, st);
}

void launch_budget_select(const Frame& F, const clod_scene& S, uint32_t V, int n_sm, cudaStream_t st);

// select: run the primitive-budget select (needed when a view has budget > 0).
void launch_preprocess(const Frame& F, const clod_scene& S, uint32_t V, uint8_t* mask_out, float* alpha_out,
                       unsigned long long* n_pairs_out, int n_sm, cudaStream_t st, bool select)
{
    const int64_t n = S.n;
    // one resident wave of each kernel (the loops stride over the rest)
    int blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, (int64_t)n_sm * 4));
    if (blocks < 1) blocks = 1;
    const int dm_blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, (int64_t)n_sm * 4)));
    if (n > 0) {
        if (V == 1) launch(k_dist_max, dm_blocks, 256, 0, st, F, S.means, n);
        else if (V <= 4) launch(k_dist_max_views<4>, dm_blocks, 256, 0, st, F, S.means, n);
        else if (V <= 8) launch(k_dist_max_views<8>, dm_blocks, 256, 0, st, F, S.means, n);
        else launch(k_dist_max, dm_blocks, 256, 0, st, F, S.means, n);
    }
    if (n > 0 && select) launch_budget_select(F, S, V, n_sm, st);
    if (n > 0) {
        switch (S.sh_degree) {
        case 0: launch(k_preprocess<0>, blocks, 256, 0, st, F, S, mask_out, alpha_out, n_pairs_out); break;
        case 1: launch(k_preprocess<1>, blocks, 256, 0, st, F, S, mask_out, alpha_out, n_pairs_out); break;
        case 2: launch(k_preprocess<2>, blocks, 256, 0, st, F, S, mask_out, alpha_out, n_pairs_out); break;
        default: launch(k_preprocess<3>, blocks, 256, 0, st, F, S, mask_out, alpha_out, n_pairs_out); break;
        }
    }
    if (n_pairs_out && n <= 0)   // otherwise k_preprocess's last block writes it
        cudaMemcpyAsync(n_pairs_out, &F.hdr->n_pairs, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st);
}

}  // namespace clod
