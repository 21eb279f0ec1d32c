// binsort.cu -- pair emission and the (tile, depth) sort.
//
// The list the blend needs is every (view, tile, Gaussian) pair sorted by the
// 64-bit key ((tile_base(view) + tile) << 32) | bits(depth) -- "sorted by
// depth" (Sec. 3.1) per tile -- with equal keys in Gaussian-index order (the
// stable sort of the index-ordered emission).  It is built as a most-
// significant-digit radix sort whose first digit is the whole global tile id:
//
//   k_scatter       counting-sort scatter: each surviving (view, Gaussian)
//                   writes (bits(depth) << 32 | index) into the bucket of
//                   every tile of its rectangle (bucket offsets = exclusive
//                   scan of the per-tile counts made during preprocessing;
//                   slot by atomic cursor, so order inside a bucket is
//                   arbitrary);
//   k_tile_sort     one block per tile sorts its bucket in shared memory by
//                   the 64-bit (depth, index) value -- a total order, so the
//                   result is unique and equals the stable key sort -- and
//                   writes values, keys and the tile's range;
//   k_tile_sort_big tiles longer than the small kernel's capacity: chunks
//                   sorted in shared memory, then merge-path merges through
//                   a scratch buffer.
//
// HBM traffic per pair: 8 B scattered, 8 B read back, 4 B (values) + 8 B
// (keys, optional) written -- against ~150 B per pair for an LSD radix sort
// over 45-50 key bits.
#include <algorithm>

#include "clod_internal.cuh"

namespace clod {

constexpr int SMALL_CAP = 2048;         // k_tile_sort, 256 threads, 16 KB
constexpr int BIG_THREADS = 1024;
constexpr int BIG_CHUNK = 8192;         // k_tile_sort_big, 64 KB chunks

__global__ void __launch_bounds__(256) k_scatter(Frame F, int64_t n, uint32_t V, unsigned long long* __restrict__ pairs,
                                                 unsigned long long cap)
{
    __shared__ uint32_t s_base[MAX_VIEWS];
    __shared__ int32_t s_tx[MAX_VIEWS];
    const unsigned long long K = F.hdr->n_pairs;
    if (K > cap || (F.hdr->status & STATUS_OVERFLOW)) {
        if (threadIdx.x == 0) atomicOr(&F.hdr->status, STATUS_OVERFLOW);
        return;
    }
    for (uint32_t v = threadIdx.x; v < V; v += blockDim.x) {
        s_base[v] = F.views[v].tile_base;
        s_tx[v] = F.views[v].TX;
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        for (uint32_t v = 0; v < V; ++v) {
            const int64_t o = (int64_t)v * n + i;
            const uint2 r = F.rect[o];
            const uint32_t x0 = r.x & 0xFFFFu, y0 = r.x >> 16, x1 = r.y & 0xFFFFu, y1 = r.y >> 16;
            if (x1 <= x0 || y1 <= y0) continue;
            const unsigned long long val =
                (static_cast<unsigned long long>(__float_as_uint(F.depth[o])) << 32) | static_cast<uint32_t>(i);
            for (uint32_t ty = y0; ty < y1; ++ty)
                for (uint32_t tx = x0; tx < x1; ++tx) {
                    const uint32_t t = s_base[v] + ty * s_tx[v] + tx;
                    const uint32_t pos = atomicAdd(&F.cursor[t], 1u);
                    pairs[pos] = val;
                }
        }
    }
}

// Bitonic sort of s[0, n2) (n2 a power of two) by nthreads threads.
__device__ __forceinline__ void bitonic_sort(unsigned long long* s, int n2)
{
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < (n2 >> 1); t += blockDim.x) {
                const int a = 2 * t - (t & (j - 1));
                const int b = a + j;
                const bool up = (a & k) == 0;
                const unsigned long long x = s[a], y = s[b];
                if ((x > y) == up) {
                    s[a] = y;
                    s[b] = x;
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ void write_sorted(unsigned long long v, uint32_t tile, uint32_t pos,
                                             uint32_t* __restrict__ vals, unsigned long long* __restrict__ keys)
{
    vals[pos] = static_cast<uint32_t>(v);
    if (keys) keys[pos] = (static_cast<unsigned long long>(tile) << 32) | (v >> 32);
}

__global__ void __launch_bounds__(256) k_tile_sort(Frame F, const unsigned long long* __restrict__ pairs,
                                                   unsigned long long cap, uint32_t* __restrict__ vals,
                                                   unsigned long long* __restrict__ keys, uint32_t* __restrict__ ranges)
{
    __shared__ unsigned long long s[SMALL_CAP];
    const uint32_t TT = F.hdr->total_tiles;
    if (F.hdr->status & STATUS_OVERFLOW) return;
    for (uint32_t t = blockIdx.x; t < TT; t += gridDim.x) {
        const uint32_t start = F.tile_offset[t], end = F.tile_offset[t + 1];
        const uint32_t cnt = end - start;
        if (threadIdx.x == 0) {
            ranges[2 * t] = cnt ? start : 0u;
            ranges[2 * t + 1] = cnt ? end : 0u;
        }
        if (cnt == 0) continue;
        if (cnt > SMALL_CAP) {
            if (threadIdx.x == 0) {
                const uint32_t k = atomicAdd(&F.hdr->big_count, 1u);
                F.big_list[k] = t;
            }
            continue;
        }
        int n2 = 1;
        while (n2 < (int)cnt) n2 <<= 1;
        for (int k = threadIdx.x; k < n2; k += blockDim.x) s[k] = k < (int)cnt ? pairs[start + k] : ~0ull;
        __syncthreads();
        if (n2 > 1) bitonic_sort(s, n2);
        for (int k = threadIdx.x; k < (int)cnt; k += blockDim.x) write_sorted(s[k], t, start + k, vals, keys);
        __syncthreads();
    }
}

// Merge-path split: number of elements taken from A among the first k
// outputs of merge(A[0,na), B[0,nb)) (all values distinct).
__device__ __forceinline__ int merge_split(const unsigned long long* A, int na, const unsigned long long* B, int nb,
                                           int k)
{
    int lo = max(0, k - nb), hi = min(k, na);
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (A[m] < B[k - m - 1]) lo = m + 1;
        else hi = m;
    }
    return lo;
}

__global__ void __launch_bounds__(BIG_THREADS) k_tile_sort_big(Frame F, unsigned long long* __restrict__ pairs,
                                                               unsigned long long* __restrict__ scratch,
                                                               uint32_t* __restrict__ vals,
                                                               unsigned long long* __restrict__ keys)
{
    extern __shared__ unsigned long long sb[];
    if (F.hdr->status & STATUS_OVERFLOW) return;
    const uint32_t nb = F.hdr->big_count;
    for (uint32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const uint32_t t = F.big_list[b];
        const uint32_t start = F.tile_offset[t];
        const int len = static_cast<int>(F.tile_offset[t + 1] - start);
        unsigned long long* src = pairs + start;
        unsigned long long* dst = scratch + start;
        // 1. sort chunks of BIG_CHUNK in shared memory, in place
        for (int c0 = 0; c0 < len; c0 += BIG_CHUNK) {
            const int cl = min(BIG_CHUNK, len - c0);
            int n2 = 1;
            while (n2 < cl) n2 <<= 1;
            for (int k = threadIdx.x; k < n2; k += blockDim.x) sb[k] = k < cl ? src[c0 + k] : ~0ull;
            __syncthreads();
            bitonic_sort(sb, n2);
            for (int k = threadIdx.x; k < cl; k += blockDim.x) src[c0 + k] = sb[k];
            __syncthreads();
        }
        // 2. merge runs of width w into the other buffer, w = chunk, 2 chunk, ...
        constexpr int E = 8;   // outputs per thread per step
        for (int w = BIG_CHUNK; w < len; w <<= 1) {
            for (int o0 = threadIdx.x * E; o0 < len; o0 += blockDim.x * E) {
                const int a = (o0 / (2 * w)) * (2 * w);
                const int mid = min(a + w, len), end = min(a + 2 * w, len);
                const int na = mid - a, nbb = end - mid;
                const int k = o0 - a;
                int i = merge_split(src + a, na, src + mid, nbb, k);
                int j = k - i;
                const int cnt = min(E, end - o0);
                for (int e = 0; e < cnt; ++e) {
                    const bool takeA = j >= nbb || (i < na && src[a + i] < src[mid + j]);
                    dst[o0 + e] = takeA ? src[a + i] : src[mid + j];
                    if (takeA) ++i;
                    else ++j;
                }
            }
            __syncthreads();
            unsigned long long* tmp = src;
            src = dst;
            dst = tmp;
        }
        for (int k = threadIdx.x; k < len; k += blockDim.x) write_sorted(src[k], t, start + k, vals, keys);
        __syncthreads();
    }
}

void launch_bin_sort(const Frame& F, int64_t n, uint32_t V, uint32_t total_tiles, unsigned long long* pairs,
                     unsigned long long* scratch, unsigned long long cap, uint64_t* keys, uint32_t* vals,
                     uint32_t* ranges, int n_sm, cudaStream_t st)
{
    int blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, (int64_t)n_sm * 8));
    if (blocks < 1) blocks = 1;
    if (n > 0) k_scatter<<<blocks, 256, 0, st>>>(F, n, V, pairs, cap);
    const int tblocks = static_cast<int>(std::max<uint32_t>(1u, std::min<uint32_t>(total_tiles, 65535u * 4u)));
    k_tile_sort<<<tblocks, 256, 0, st>>>(F, pairs, cap, vals, reinterpret_cast<unsigned long long*>(keys), ranges);
    k_tile_sort_big<<<n_sm, BIG_THREADS, BIG_CHUNK * sizeof(unsigned long long), st>>>(
        F, pairs, scratch, vals, reinterpret_cast<unsigned long long*>(keys));
}

cudaError_t bin_sort_setup()
{
    return cudaFuncSetAttribute(k_tile_sort_big, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                BIG_CHUNK * (int)sizeof(unsigned long long));
}

}  // namespace clod
