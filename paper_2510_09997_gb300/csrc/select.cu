// select.cu -- the primitive budget (Sec. 4.2: models are compared at equal
// Gaussian counts by applying the attenuation of Eq. 2 and keeping the
// primitives of highest attenuated opacity).
//
// For every view with budget B > 0 the mask becomes M_i = key_i >= T, where
// key_i = (bits(alpha''_i) << 32) | (2^32 - 1 - i) and T is the B-th largest
// key: the B Gaussians of highest alpha'', equal alpha'' in index order.  The
// keys are distinct, so exactly min(B, n) are kept.  T is found by a radix
// select, most significant digit first (11, 11, 10, 11, 11, 10 bits): each
// pass counts, among the keys that share the digits fixed so far, how many
// carry each value of the next digit, and fixes the digit at which the
// count from the top reaches the number still to select.  A view stops as
// soon as every key under its prefix is selected.
//
//   k_sel_init   per view: state, cleared counts
//   k_sel_count  one pass of digit counts (the first also writes alpha'',
//                recomputed exactly as k_preprocess does, into the depth
//                array, which is free until k_preprocess)
//   k_sel_pick   per view: suffix sums of the counts, the digit, the state
#include <algorithm>

#include "clod_internal.cuh"

namespace clod {

__constant__ int c_sel_shift[SEL_PASSES] = {53, 42, 32, 21, 10, 0};
__constant__ int c_sel_bits[SEL_PASSES] = {11, 11, 10, 11, 11, 10};

__global__ void __launch_bounds__(256) k_sel_init(Frame F)
{
    pdl_wait();
    const uint32_t v = blockIdx.x;
    if (v >= F.hdr->n_views) return;
    const ViewDev& W = F.views[v];
    uint32_t* h = F.sel_hist + (size_t)v * SEL_BINS;
    for (int k = threadIdx.x; k < SEL_BINS; k += blockDim.x) h[k] = 0u;
    if (threadIdx.x == 0) {
        const uint64_t n = F.hdr->n;
        SelState s{};
        s.remaining = W.budget;
        // no budget, or a budget of all n: nothing to select (T = 0 keeps everything)
        s.done = (W.budget == 0u || (uint64_t)W.budget >= n) ? 1u : 0u;
        F.sel[v] = s;
    }
}

__global__ void __launch_bounds__(256) k_sel_count(Frame F, clod_scene S, int pass)
{
    pdl_wait();
    __shared__ uint32_t h[SEL_BINS];
    __shared__ ViewDev W;
    __shared__ SelState st;
    __shared__ float dmax;
    const uint32_t V = F.hdr->n_views;
    const int64_t n = S.n;
    const int shift = c_sel_shift[pass], bits = c_sel_bits[pass];
    for (uint32_t v = 0; v < V; ++v) {
        __syncthreads();
        if (threadIdx.x == 0) {
            W = F.views[v];
            st = F.sel[v];
            dmax = decode_dmax(F.dmax_key[v]);
        }
        for (int k = threadIdx.x; k < SEL_BINS; k += blockDim.x) h[k] = 0u;
        __syncthreads();
        if (st.done) continue;
        const unsigned long long prefix = st.prefix;
        const int hi = shift + bits;   // bits above this digit: the prefix
        float* a2v = F.depth + (size_t)v * n;
        for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)gridDim.x * blockDim.x) {
            float a2;
            if (pass == 0) {
                float e0, e1, e2;
                const float d = cam_dist(W, S.means[3 * i], S.means[3 * i + 1], S.means[3 * i + 2], e0, e1, e2);
                a2 = attenuated_opacity(W, S.opacity[i], S.decay[i], d, dmax);
                a2v[i] = a2;
            } else {
                a2 = a2v[i];
            }
            const unsigned long long key = budget_key(a2, static_cast<uint32_t>(i));
            if (hi >= 64 || (key >> hi) == prefix)
                atomicAdd_block(&h[(uint32_t)(key >> shift) & ((1u << bits) - 1u)], 1u);
        }
        __syncthreads();
        uint32_t* g = F.sel_hist + (size_t)v * SEL_BINS;
        for (int k = threadIdx.x; k < (1 << bits); k += blockDim.x)
            if (h[k]) atomicAdd(&g[k], h[k]);
    }
}

// One block of 1024 threads per view; thread t owns bins 2047 - 2t and
// 2046 - 2t (descending), so an exclusive scan over threads gives the count
// of keys above each bin.
__global__ void __launch_bounds__(1024) k_sel_pick(Frame F, int pass)
{
    pdl_wait();
    __shared__ uint32_t wsum[32];
    __shared__ int found;
    const uint32_t v = blockIdx.x;
    if (v >= F.hdr->n_views) return;
    SelState* sp = F.sel + v;
    const SelState s0 = *sp;   // read by every thread before any write below
    if (s0.done) return;
    const int shift = c_sel_shift[pass], bits = c_sel_bits[pass];
    const int nb = 1 << bits;
    uint32_t* g = F.sel_hist + (size_t)v * SEL_BINS;
    const int t = threadIdx.x;
    const int dA = nb - 1 - 2 * t, dB = nb - 2 - 2 * t;
    const uint32_t hA = dA >= 0 ? g[dA] : 0u, hB = dB >= 0 ? g[dB] : 0u;
    if (t == 0) found = 0;
    __syncthreads();
    if (dA >= 0) g[dA] = 0u;    // cleared for the next pass
    if (dB >= 0) g[dB] = 0u;
    // exclusive scan of hA + hB over threads
    const uint32_t mine = hA + hB;
    const int lane = t & 31, w = t >> 5;
    uint32_t x = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint32_t above = x - mine;
    for (int k = 0; k < w; ++k) above += wsum[k];
    const uint32_t rem = s0.remaining;
    int digit = -1;
    uint32_t cnt_above = 0, cnt_at = 0;
    if (dA >= 0 && above < rem && above + hA >= rem) {
        digit = dA;
        cnt_above = above;
        cnt_at = hA;
    } else if (dB >= 0 && above + hA < rem && above + hA + hB >= rem) {
        digit = dB;
        cnt_above = above + hA;
        cnt_at = hB;
    }
    if (digit >= 0) {
        found = 1;
        SelState s = s0;
        s.prefix = (s.prefix << bits) | (unsigned long long)digit;
        s.remaining = rem - cnt_above;
        if (cnt_at == s.remaining) {   // every key under the new prefix is selected
            s.T = s.prefix << shift;
            s.done = 1u;
        }
        *sp = s;
    }
    __syncthreads();
    if (t == 0 && !found) {    // fewer candidates than the budget (cannot happen for distinct keys): keep all
        sp->T = 0ull;
        sp->done = 1u;
    }
}

void launch_budget_select(const Frame& F, const clod_scene& S, uint32_t V, int n_sm, cudaStream_t st)
{
    const int64_t n = S.n;
    if (n <= 0) return;
    const int blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, (int64_t)n_sm * 4));
    launch(k_sel_init, V, 256, 0, st, F);
    for (int p = 0; p < SEL_PASSES; ++p) {
        launch(k_sel_count, std::max(blocks, 1), 256, 0, st, F, S, p);
        launch(k_sel_pick, V, 1024, 0, st, F, p);
    }
}

}  // namespace clod
