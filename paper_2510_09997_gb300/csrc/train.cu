// train.cu -- the training step around the rasterizer (Sec. 3.3).
//
//   k_lreg   per view: eta_actual = sum M_i / N (the mask counts the
//            preprocessing wrote), L_reg = (s_v - 1)^2 ReLU(eta_actual -
//            s_v^-1.5)^2 (Eq. 3-4), the total L_total = sum_v w_v (L_render_v
//            + lambda L_reg_v) (Eq. 5 with w_v = w_s / V), and the
//            straight-through gradient dL/dalpha''_i = w_v lambda 2 (s_v -
//            1)^2 ReLU(.) / N, one scalar per view (dM_i/dalpha''_i := 1).
//   k_adam   one Adam step over the six parameter groups, fused with the
//            activations: the rasterizer's gradients are taken back to the
//            raw parameters (scales = exp(log-scales), opacity =
//            sigmoid(logit)), the moments and raw values are updated, the
//            activated scales and opacities are rewritten from the new raw
//            values and the gradients are cleared for the next step.
#include <algorithm>
#include <cmath>

#include "clod_internal.cuh"

namespace clod {

clod_status fail(clod_status s, const char* fmt, ...);
clod_status cuda_fail(cudaError_t e, const char* what);
clod_status device_ready(int* n_sm);

struct LregArgs {
    float s_v[MAX_VIEWS];
    float w[MAX_VIEWS];
};

__global__ void k_lreg(const uint32_t* __restrict__ counts, double inv_n, float lam, int V, LregArgs a,
                       const float* __restrict__ lrender, float* __restrict__ dalpha, float* __restrict__ total,
                       float* __restrict__ lreg_out)
{
    pdl_wait();
    __shared__ float part[MAX_VIEWS];
    const int v = threadIdx.x;
    float t = 0.0f;
    if (v < V) {
        const float s = a.s_v[v];
        const float eta_a = static_cast<float>(static_cast<double>(counts[2 * v]) * inv_n);
        const float eta_t = powf(s, -1.5f);
        const float relu = fmaxf(eta_a - eta_t, 0.0f);
        const float s1 = (s - 1.0f) * (s - 1.0f);
        const float lreg = s1 * relu * relu;
        if (lreg_out) lreg_out[v] = lreg;
        if (dalpha) dalpha[v] = a.w[v] * lam * 2.0f * s1 * relu * static_cast<float>(inv_n);
        t = a.w[v] * ((lrender ? lrender[v] : 0.0f) + lam * lreg);
    }
    if (v < MAX_VIEWS) part[v] = t;
    __syncthreads();
    if (v == 0 && total) {
        float sum = 0.0f;
        for (int k = 0; k < V; ++k) sum += part[k];
        *total = sum;
    }
}

struct AdamArgs {
    float* p[6];            // raw parameters
    float* g[6];            // gradients with respect to the activated parameters
    float* act[6];          // activated copies (scales, opacity), else null
    int64_t cnt[6];         // elements per group
    int64_t off[7];         // element offsets of the groups in m, v (multiples of 4)
    float step_size[6];     // lr / (1 - beta1^t)
    float b1, b2, inv_bc2_sqrt, eps;
};

// One element of the update (the activation chain rule for the log-scale
// and logit groups, the moments, the bias-corrected step); returns the new
// raw value.
__device__ __forceinline__ float adam_one(const AdamArgs& A, int gi, float ss, bool act, float p, float g, float a,
                                          float& m, float& v)
{
    if (act) g = gi == 1 ? g * a : g * a * (1.0f - a);   // d exp = exp; d sigmoid = a (1 - a)
    m = A.b1 * m + (1.0f - A.b1) * g;
    v = A.b2 * v + (1.0f - A.b2) * g * g;
    const float denom = sqrtf(v) * A.inv_bc2_sqrt + A.eps;
    return p - ss * (m / denom);
}

__device__ __forceinline__ float activate(int gi, float p)
{
    return gi == 1 ? expf(p) : 1.0f / (1.0f + expf(-p));
}

// Group by group, four elements per vector access (the groups' moments start
// at multiples of four elements), two vectors per thread and round with every
// load issued before any store; a scalar tail finishes each group.
// ZERO: clear the gradients after the update.
template <bool ZERO>
__global__ void __launch_bounds__(256, 3) k_adam(AdamArgs A, float* __restrict__ m, float* __restrict__ v)
{
    pdl_wait();
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int gi = 0; gi < 6; ++gi) {
        const int64_t cnt = A.cnt[gi];
        float* __restrict__ P = A.p[gi];
        float* __restrict__ G = A.g[gi];
        float* __restrict__ Act = A.act[gi];
        float* __restrict__ M = m + A.off[gi];
        float* __restrict__ Vv = v + A.off[gi];
        const float ss = A.step_size[gi];
        const bool act = Act != nullptr;
        const int64_t n4 = cnt / 4;
        for (int64_t j0 = tid; j0 < n4; j0 += 2 * stride) {
            float4 p4[2], g4[2], m4[2], v4[2], a4[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int64_t j = j0 + u * stride;
                if (j < n4) {
                    p4[u] = reinterpret_cast<const float4*>(P)[j];
                    g4[u] = reinterpret_cast<const float4*>(G)[j];
                    m4[u] = reinterpret_cast<const float4*>(M)[j];
                    v4[u] = reinterpret_cast<const float4*>(Vv)[j];
                    a4[u] = act ? reinterpret_cast<const float4*>(Act)[j] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int64_t j = j0 + u * stride;
                if (j < n4) {
                    float4 pn;
                    pn.x = adam_one(A, gi, ss, act, p4[u].x, g4[u].x, a4[u].x, m4[u].x, v4[u].x);
                    pn.y = adam_one(A, gi, ss, act, p4[u].y, g4[u].y, a4[u].y, m4[u].y, v4[u].y);
                    pn.z = adam_one(A, gi, ss, act, p4[u].z, g4[u].z, a4[u].z, m4[u].z, v4[u].z);
                    pn.w = adam_one(A, gi, ss, act, p4[u].w, g4[u].w, a4[u].w, m4[u].w, v4[u].w);
                    reinterpret_cast<float4*>(M)[j] = m4[u];
                    reinterpret_cast<float4*>(Vv)[j] = v4[u];
                    reinterpret_cast<float4*>(P)[j] = pn;
                    if (ZERO) reinterpret_cast<float4*>(G)[j] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (act)
                        reinterpret_cast<float4*>(Act)[j] =
                            make_float4(activate(gi, pn.x), activate(gi, pn.y), activate(gi, pn.z), activate(gi, pn.w));
                }
            }
        }
        for (int64_t j = 4 * n4 + tid; j < cnt; j += stride) {
            float mm = M[j], vv = Vv[j];
            const float pn = adam_one(A, gi, ss, act, P[j], G[j], act ? Act[j] : 0.0f, mm, vv);
            M[j] = mm;
            Vv[j] = vv;
            P[j] = pn;
            if (ZERO) G[j] = 0.0f;
            if (act) Act[j] = activate(gi, pn);
        }
    }
}

}  // namespace clod

using namespace clod;

// Element counts of the six groups and their offsets in the moment arrays,
// each group starting at a multiple of 4 elements.
static void adam_groups(int64_t n, int32_t deg, int64_t* cnt, int64_t* off)
{
    const int64_t K = (int64_t)(deg + 1) * (deg + 1);
    const int64_t c[6] = {3 * n, 3 * n, 4 * n, n, 3 * K * n, n};
    off[0] = 0;
    for (int k = 0; k < 6; ++k) {
        cnt[k] = c[k];
        off[k + 1] = off[k] + (c[k] + 3) / 4 * 4;
    }
}

extern "C" {

clod_status clod_adam_state_size(int64_t n, int32_t sh_degree, int64_t* elements)
{
    if (!elements || n < 0 || sh_degree < 0 || sh_degree > 3) return fail(CLOD_ERR_ARG, "bad argument to clod_adam_state_size");
    int64_t cnt[6], off[7];
    adam_groups(n, sh_degree, cnt, off);
    *elements = off[6];
    return CLOD_OK;
}

clod_status clod_step_weights(const float* s_v, int32_t n_views, float s_max, float* weight)
{
    if (!s_v || !weight || n_views < 1 || n_views > MAX_VIEWS) return fail(CLOD_ERR_ARG, "bad argument to clod_step_weights");
    if (!(s_max > 0.0f) || !std::isfinite(s_max)) return fail(CLOD_ERR_ARG, "s_max must be > 0 and finite");
    for (int v = 0; v < n_views; ++v) {
        if (!(s_v[v] > 0.0f) || !std::isfinite(s_v[v])) return fail(CLOD_ERR_ARG, "view %d: s_v must be > 0", v);
        const double r = 1.0 - 0.5 * (double)s_v[v] / (double)s_max;     // Eq. 5
        weight[v] = (float)(r * r / (double)n_views);
    }
    return CLOD_OK;
}

clod_status clod_lreg_grad(const uint32_t* counts, int64_t n, int32_t n_views, const float* s_v, const float* weight,
                           float lambda_reg, const float* lrender, float* dL_dalpha_view, float* total, float* lreg_out,
                           clod_stream stream)
{
    if (!counts || n < 1 || n_views < 1 || n_views > MAX_VIEWS || !s_v || !weight)
        return fail(CLOD_ERR_ARG, "bad argument to clod_lreg_grad");
    LregArgs a{};
    for (int v = 0; v < n_views; ++v) {
        if (!(s_v[v] > 0.0f) || !std::isfinite(s_v[v])) return fail(CLOD_ERR_ARG, "view %d: s_v must be > 0", v);
        a.s_v[v] = s_v[v];
        a.w[v] = weight[v];
    }
    int n_sm = 0;
    clod_status s = device_ready(&n_sm);
    if (s) return s;
    launch(k_lreg, 1, MAX_VIEWS, 0, static_cast<cudaStream_t>(stream), counts, 1.0 / (double)n, lambda_reg, n_views, a,
           lrender, dL_dalpha_view, total, lreg_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "clod_lreg_grad launch");
    return CLOD_OK;
}

clod_status clod_adam_step(const clod_adam_cfg* cfg, int64_t n, int32_t sh_degree, float* const* raw,
                           float* const* grads, float* scales, float* opacity, float* m, float* v, clod_stream stream)
{
    if (!cfg || !raw || !grads || !scales || !opacity || !m || !v || n < 0 || sh_degree < 0 || sh_degree > 3)
        return fail(CLOD_ERR_ARG, "bad argument to clod_adam_step");
    if (cfg->step < 1) return fail(CLOD_ERR_ARG, "Adam step counts from 1");
    if (n == 0) return CLOD_OK;
    AdamArgs A{};
    adam_groups(n, sh_degree, A.cnt, A.off);
    for (int k = 0; k < 6; ++k) {
        if (!raw[k] || !grads[k]) return fail(CLOD_ERR_ARG, "parameter group %d is NULL", k);
        A.p[k] = raw[k];
        A.g[k] = grads[k];
        A.act[k] = nullptr;
    }
    A.act[1] = scales;
    A.act[3] = opacity;
    for (int k = 0; k < 6; ++k)
        if (reinterpret_cast<uintptr_t>(A.p[k]) % 16 || reinterpret_cast<uintptr_t>(A.g[k]) % 16 ||
            reinterpret_cast<uintptr_t>(A.act[k]) % 16)
            return fail(CLOD_ERR_ARG, "parameter group %d: raw, gradient and activated arrays must be 16-byte aligned", k);
    if (reinterpret_cast<uintptr_t>(m) % 16 || reinterpret_cast<uintptr_t>(v) % 16)
        return fail(CLOD_ERR_ARG, "moments must be 16-byte aligned");
    const double bc1 = 1.0 - std::pow((double)cfg->beta1, (double)cfg->step);
    const double bc2 = 1.0 - std::pow((double)cfg->beta2, (double)cfg->step);
    for (int k = 0; k < 6; ++k) A.step_size[k] = (float)(cfg->lr[k] / bc1);
    A.b1 = cfg->beta1;
    A.b2 = cfg->beta2;
    A.inv_bc2_sqrt = (float)(1.0 / std::sqrt(bc2));
    A.eps = cfg->eps;
    int n_sm = 0;
    clod_status s = device_ready(&n_sm);
    if (s) return s;
    const int64_t E = A.off[6];
    // one resident wave (78 registers: 3 blocks of 256 per SM)
    const int blocks = static_cast<int>(std::min<int64_t>((E + 255) / 256, (int64_t)n_sm * 3));
    if (cfg->keep_grads) launch(k_adam<false>, blocks, 256, 0, static_cast<cudaStream_t>(stream), A, m, v);
    else launch(k_adam<true>, blocks, 256, 0, static_cast<cudaStream_t>(stream), A, m, v);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "clod_adam_step launch");
    return CLOD_OK;
}

}  // extern "C"
