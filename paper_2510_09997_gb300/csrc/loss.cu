// loss.cu -- the rendering loss of the training objective (Sec. 3.3):
// L_render = (1 - lambda) L1 + lambda (1 - SSIM), SSIM with an 11x11 Gaussian
// window (sigma 1.5, zero outside the image), C1 = 0.01^2, C2 = 0.03^2,
// averaged over pixels and channels.
//
//   k_ssim_fwd  per 16x16 tile and channel: the tile plus a 5-pixel halo of
//               x and y in shared memory, separable blurs of x, y, x^2, y^2,
//               xy, the SSIM map S, the L1 term; the loss is block-reduced;
//               the three maps the gradient needs are stored:
//                 M1 = dS/dmu_x - 2 mu_x dS/ds_xx - mu_y dS/ds_xy,
//                 M2 = dS/ds_xx, M3 = dS/ds_xy;
//   k_ssim_bwd  per tile: blurs of M1, M2, M3 (the window is symmetric) and
//               dSSIM/dx = (w * M1 + 2 x (w * M2) + y (w * M3)) / N.
//   k_l1_term   lambda = 0: the L1 term alone (no maps).
// The gradient is scaled by the caller's factor of this term in its total.
#include <algorithm>
#include <cmath>

#include "clod_internal.cuh"

namespace clod {

clod_status fail(clod_status s, const char* fmt, ...);
clod_status cuda_fail(cudaError_t e, const char* what);
clod_status device_ready(int* n_sm);

constexpr int SS_T = 16;
constexpr int SS_R = 5;
constexpr int SS_H = SS_T + 2 * SS_R;   // 26
constexpr float SS_C1 = 1e-4f;
constexpr float SS_C2 = 9e-4f;

__constant__ float c_win[2 * SS_R + 1];

__device__ __forceinline__ float ld0(const float* p, int x, int y, int W, int H)
{
    return (x >= 0 && x < W && y >= 0 && y < H) ? p[(size_t)y * W + x] : 0.0f;
}

__device__ __forceinline__ float block_sum(float v)
{
    __shared__ float ws[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) ws[w] = v;
    __syncthreads();
    float t = 0.0f;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;   // valid in thread 0
}

__global__ void __launch_bounds__(SS_T * SS_T) k_ssim_fwd(const float* __restrict__ img, const float* __restrict__ tgt,
                                                          int W, int H, float lam, float inv_n, float* __restrict__ loss,
                                                          float* __restrict__ maps)
{
    pdl_wait();
    __shared__ float sx[SS_H][SS_H], sy[SS_H][SS_H];
    __shared__ float hb[5][SS_H][SS_T];
    const int c = blockIdx.z;
    const size_t plane = (size_t)W * H;
    const float* X = img + c * plane;
    const float* Y = tgt + c * plane;
    const int x0 = blockIdx.x * SS_T - SS_R, y0 = blockIdx.y * SS_T - SS_R;
    for (int k = threadIdx.x; k < SS_H * SS_H; k += blockDim.x) {
        const int i = k / SS_H, j = k % SS_H;
        sx[i][j] = ld0(X, x0 + j, y0 + i, W, H);
        sy[i][j] = ld0(Y, x0 + j, y0 + i, W, H);
    }
    __syncthreads();
    // horizontal pass: rows of the halo, columns of the tile
    for (int k = threadIdx.x; k < SS_H * SS_T; k += blockDim.x) {
        const int i = k / SS_T, j = k % SS_T;
        float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
        for (int t = 0; t <= 2 * SS_R; ++t) {
            const float w = c_win[t], xv = sx[i][j + t], yv = sy[i][j + t];
            a += w * xv;
            b += w * yv;
            aa += w * xv * xv;
            bb += w * yv * yv;
            ab += w * xv * yv;
        }
        hb[0][i][j] = a;
        hb[1][i][j] = b;
        hb[2][i][j] = aa;
        hb[3][i][j] = bb;
        hb[4][i][j] = ab;
    }
    __syncthreads();
    const int tx = threadIdx.x % SS_T, ty = threadIdx.x / SS_T;
    const int px = blockIdx.x * SS_T + tx, py = blockIdx.y * SS_T + ty;
    float acc = 0.0f;
    if (px < W && py < H) {
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t <= 2 * SS_R; ++t) {
            const float w = c_win[t];
#pragma unroll
            for (int q = 0; q < 5; ++q) m[q] += w * hb[q][ty + t][tx];
        }
        const float mx = m[0], my = m[1];
        const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
        const float A1 = 2.f * mx * my + SS_C1, A2 = 2.f * sxy + SS_C2;
        const float B1 = mx * mx + my * my + SS_C1, B2 = sxx + syy + SS_C2;
        const float S = (A1 * A2) / (B1 * B2);
        const float xv = sx[ty + SS_R][tx + SS_R], yv = sy[ty + SS_R][tx + SS_R];
        acc = (1.0f - lam) * fabsf(xv - yv) - lam * S;
        if (maps) {
            const float dmx = (2.f * my * A2) / (B1 * B2) - S * (2.f * mx) / B1;
            const float dsxx = -S / B2;
            const float dsxy = (2.f * A1) / (B1 * B2);
            const size_t p = (size_t)py * W + px;
            maps[(3 * c + 0) * plane + p] = dmx - 2.f * mx * dsxx - my * dsxy;
            maps[(3 * c + 1) * plane + p] = dsxx;
            maps[(3 * c + 2) * plane + p] = dsxy;
        }
    }
    const float tot = block_sum(acc);
    if (threadIdx.x == 0 && loss) {
        const bool first = blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
        atomicAdd(loss, tot * inv_n + (first ? lam : 0.0f));   // lambda (1 - SSIM): the constant once
    }
}

__global__ void __launch_bounds__(SS_T * SS_T) k_ssim_bwd(const float* __restrict__ img, const float* __restrict__ tgt,
                                                          int W, int H, float lam, float ginv_n,
                                                          const float* __restrict__ maps, float* __restrict__ grad)
{
    pdl_wait();
    __shared__ float sm[3][SS_H][SS_H];
    __shared__ float hb[3][SS_H][SS_T];
    const int c = blockIdx.z;
    const size_t plane = (size_t)W * H;
    const int x0 = blockIdx.x * SS_T - SS_R, y0 = blockIdx.y * SS_T - SS_R;
    for (int k = threadIdx.x; k < SS_H * SS_H; k += blockDim.x) {
        const int i = k / SS_H, j = k % SS_H;
#pragma unroll
        for (int q = 0; q < 3; ++q) sm[q][i][j] = ld0(maps + (3 * c + q) * plane, x0 + j, y0 + i, W, H);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < SS_H * SS_T; k += blockDim.x) {
        const int i = k / SS_T, j = k % SS_T;
        float a[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t <= 2 * SS_R; ++t) {
            const float w = c_win[t];
#pragma unroll
            for (int q = 0; q < 3; ++q) a[q] += w * sm[q][i][j + t];
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) hb[q][i][j] = a[q];
    }
    __syncthreads();
    const int tx = threadIdx.x % SS_T, ty = threadIdx.x / SS_T;
    const int px = blockIdx.x * SS_T + tx, py = blockIdx.y * SS_T + ty;
    if (px >= W || py >= H) return;
    float b[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int t = 0; t <= 2 * SS_R; ++t) {
        const float w = c_win[t];
#pragma unroll
        for (int q = 0; q < 3; ++q) b[q] += w * hb[q][ty + t][tx];
    }
    const size_t p = c * plane + (size_t)py * W + px;
    const float xv = img[p], yv = tgt[p];
    const float dssim = b[0] + 2.f * xv * b[1] + yv * b[2];
    const float dl1 = xv > yv ? 1.f : (xv < yv ? -1.f : 0.f);
    grad[p] = ginv_n * ((1.0f - lam) * dl1 - lam * dssim);
}

// w = 0: L1 alone.  loss += mean |x - y|; grad = grad_scale sign(x - y) / count.
__global__ void __launch_bounds__(256) k_l1_term(const float* __restrict__ img, const float* __restrict__ tgt,
                                                 int64_t count, float inv_n, float ginv_n, float* __restrict__ loss,
                                                 float* __restrict__ grad)
{
    pdl_wait();
    float acc = 0.0f;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x) {
        const float d = img[k] - tgt[k];
        acc += fabsf(d);
        if (grad) grad[k] = d > 0.0f ? ginv_n : (d < 0.0f ? -ginv_n : 0.0f);
    }
    const float tot = block_sum(acc);
    if (threadIdx.x == 0 && loss) atomicAdd(loss, tot * inv_n);
}

static bool g_win_ready[64];

static clod_status window_ready()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && g_win_ready[dev]) return CLOD_OK;
    float w[2 * SS_R + 1];
    double s = 0.0, g[2 * SS_R + 1];
    for (int k = 0; k <= 2 * SS_R; ++k) {
        const double x = k - SS_R;
        g[k] = std::exp(-x * x / (2.0 * 1.5 * 1.5));
        s += g[k];
    }
    for (int k = 0; k <= 2 * SS_R; ++k) w[k] = (float)(g[k] / s);
    cudaError_t e = cudaMemcpyToSymbol(c_win, w, sizeof(w));
    if (e != cudaSuccess) return cuda_fail(e, "ssim window");
    if (dev >= 0 && dev < 64) g_win_ready[dev] = true;
    return CLOD_OK;
}

}  // namespace clod

using namespace clod;

extern "C" {

clod_status clod_render_loss_workspace_size(int32_t channels, int32_t height, int32_t width, size_t* bytes)
{
    if (!bytes || channels < 1 || height < 1 || width < 1) return fail(CLOD_ERR_ARG, "bad argument");
    *bytes = sizeof(float) * 3 * (size_t)channels * height * width;
    return CLOD_OK;
}

clod_status clod_render_loss(const float* image, const float* target, int32_t channels, int32_t height, int32_t width,
                             float dssim_weight, float grad_scale, void* ws, size_t ws_bytes, float* loss,
                             float* dL_dimage, clod_stream stream)
{
    if (!image || !target || channels < 1 || height < 1 || width < 1)
        return fail(CLOD_ERR_ARG, "bad argument to clod_render_loss");
    if (!(dssim_weight >= 0.0f && dssim_weight <= 1.0f)) return fail(CLOD_ERR_ARG, "dssim_weight outside [0, 1]");
    size_t need = 0;
    clod_status s = clod_render_loss_workspace_size(channels, height, width, &need);
    if (s) return s;
    if (!std::isfinite(grad_scale)) return fail(CLOD_ERR_ARG, "grad_scale must be finite");
    int n_sm = 0;
    if ((s = device_ready(&n_sm))) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t count = (int64_t)channels * height * width;
    const float inv_n = 1.0f / (float)count;
    if (dssim_weight == 0.0f) {
        const int blocks = static_cast<int>(std::min<int64_t>((count + 255) / 256, (int64_t)n_sm * 4));
        launch(k_l1_term, blocks, 256, 0, st, image, target, count, inv_n, grad_scale * inv_n, loss, dL_dimage);
    } else {
        if (dL_dimage && (!ws || ws_bytes < need))
            return fail(CLOD_ERR_CAPACITY, "render-loss workspace needs %zu bytes, got %zu", need, ws_bytes);
        if ((s = window_ready())) return s;
        const dim3 grid((width + SS_T - 1) / SS_T, (height + SS_T - 1) / SS_T, channels);
        float* maps = dL_dimage ? static_cast<float*>(ws) : nullptr;
        launch(k_ssim_fwd, grid, SS_T * SS_T, 0, st, image, target, width, height, dssim_weight, inv_n, loss, maps);
        if (dL_dimage)
            launch(k_ssim_bwd, grid, SS_T * SS_T, 0, st, image, target, width, height, dssim_weight,
                   grad_scale * inv_n, maps, dL_dimage);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "clod_render_loss launch");
    return CLOD_OK;
}

}  // extern "C"
