// binsort.cu -- pair emission in (tile, depth, index) order.
//
// The list the blend needs is every (view, tile, Gaussian) pair sorted by the
// 64-bit key ((tile_base(view) + tile) << 32) | bits(depth) -- "sorted by
// depth" (Sec. 3.1) per tile -- with equal keys in Gaussian-index order.  It
// is built without sorting the K pairs and without per-pair atomics:
//
//   1. depth-rank sort: a stable LSD radix sort (8-bit digits, four passes)
//      of the survivors' depth bits per view, values = Gaussian index in
//      index order.  Culled Gaussians (keyed all-ones by the preprocessing)
//      are dropped by the first pass, so the later passes move only the
//      survivors.  The last pass also gathers each survivor's tile
//      rectangle into rank order.  Each pass is two launches: per-block
//      digit counts (with per-view digit totals and sums over groups of
//      RS_G1 and RS_G2 blocks, by atomics), then the scatter, where every
//      block adds up its own offsets from the group sums and the counts of
//      the blocks before it in its group (no separate scan).
//   2. the survivors of a view are cut into chunks of consecutive ranks; one
//      warp per (chunk, tile row) walks the chunk's rectangles in rank order
//      and counts, per tile of its row, the pairs the chunk contributes
//      (k_rows<false, false>);
//   3. per tile, an exclusive scan over the chunks, then over the tiles
//      (k_tile_scan: tile offsets, K, ranges, the blends' work order);
//   4. the same walk again (k_rows<true, KEYS>): pair (Gaussian, tile) goes to
//      tile_offset + chunk offset + (number of earlier-ranked Gaussians of the
//      chunk in that tile) -- its final sorted position.
//
// Work is O(n) for the rank sort, O(K) writes for the emission; the only
// atomics add integer counts (order-independent), so the result is
// deterministic and equals the stable sort of the index-ordered emission by
// key.
#include <algorithm>

#include "clod_internal.cuh"

namespace clod {

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Lanes of the warp holding the same value as this lane, for values below
// 2^BITS: one ballot per bit (the same mask as __match_any_sync).
template <int BITS>
__device__ __forceinline__ uint32_t match_bits(uint32_t d)
{
    uint32_t m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bb = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bb : ~bb;
    }
    return m;
}

// ---------------------------------------------------------------------------
// 1. depth-rank sort
// ---------------------------------------------------------------------------
// Keys of the block's items held by this thread: warp w owns items
// [w * PER_WARP, (w + 1) * PER_WARP) of the block, lane l the items
// w * PER_WARP + 32 r + l.  All loads are issued before any is used (one
// round trip).
// 0xFFFFFFFF marks "no item": beyond the block, or culled (the first pass);
// the later passes never hold it, since a survivor's key is the bit pattern
// of a positive depth.
constexpr int RS_PER_WARP = RS_ITEMS / (RS_THREADS / 32);
constexpr int RS_R = RS_PER_WARP / 32;
__device__ __forceinline__ void rs_load_keys(const uint32_t* __restrict__ keys, int64_t base, int cnt,
                                             uint32_t (&kk)[RS_R])
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < RS_R; ++r) {
        const int idx = w * RS_PER_WARP + r * 32 + lane;
        kk[r] = idx < cnt ? keys[base + idx] : 0xFFFFFFFFu;
    }
}

// Items of radix block lb: the first pass reads all n keys of the view (and
// drops the culled), a count known without a load; later passes read the
// view's survivors, n_surv[2 v + 1].
__device__ __forceinline__ int rs_first_count(int64_t n, int lb)
{
    return (int)max((int64_t)0, min((int64_t)RS_ITEMS, n - (int64_t)lb * RS_ITEMS));
}
__device__ __forceinline__ int rs_later_count(const uint32_t* n_surv, int v, int lb)
{
    return (int)max((int64_t)0, min((int64_t)RS_ITEMS, (int64_t)n_surv[2 * v + 1] - (int64_t)lb * RS_ITEMS));
}

// Per-warp digit counts of the held keys, in h[w][digit]; each key's set of
// same-digit lanes is returned in peers[] (the scatter places the keys with it).
__device__ __forceinline__ void rs_warp_counts(const uint32_t (&kk)[RS_R], int shift, uint32_t (*h)[256],
                                               uint32_t (&peers)[RS_R])
{
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = lane; k < 256; k += 32) h[w][k] = 0;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < RS_R; ++r) {
        const bool valid = kk[r] != 0xFFFFFFFFu;
        const uint32_t d = valid ? ((kk[r] >> shift) & 255u) : 256u;
        peers[r] = match_bits<9>(d);     // d <= 256
        if (valid && (__ffs(peers[r]) - 1) == lane) h[w][d] += __popc(peers[r]);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const FrameHeader* __restrict__ hdr,
                                                        const uint32_t* __restrict__ n_surv,
                                                        const uint32_t* __restrict__ keys, int64_t n, int nb, int shift,
                                                        uint32_t* __restrict__ hist, uint32_t* __restrict__ totals,
                                                        uint32_t* __restrict__ sum1, uint32_t* __restrict__ sum2)
{
    pdl_wait();
    __shared__ uint32_t h[RS_THREADS / 32][256];
    const int b = blockIdx.x, v = b / nb, lb = b % nb;
    const int64_t base = (int64_t)v * n + (int64_t)lb * RS_ITEMS;
    // the first pass's keys are loaded before the view check (its count needs
    // no load); a later pass reads its count first, so blocks past the
    // survivors move no data
    uint32_t kk[RS_R];
    int cnt;
    if (shift == 0) {
        cnt = rs_first_count(n, lb);
        rs_load_keys(keys, base, cnt, kk);
        if ((uint32_t)v >= hdr->n_views) return;
    } else {
        if ((uint32_t)v >= hdr->n_views) return;
        cnt = rs_later_count(n_surv, v, lb);
        if (cnt == 0) return;
        rs_load_keys(keys, base, cnt, kk);
    }
    if (cnt == 0) return;     // no items (and none in any later block)
    uint32_t peers[RS_R];
    rs_warp_counts(kk, shift, h, peers);
    __syncthreads();
    uint32_t s = 0;
    for (int w = 0; w < RS_THREADS / 32; ++w) s += h[w][threadIdx.x];
    hist[((size_t)v * nb + lb) * 256 + threadIdx.x] = s;
    if (s) {
        atomicAdd(&totals[v * 256 + threadIdx.x], s);
        atomicAdd(&sum1[((size_t)v * rs_groups(nb, RS_G1) + lb / RS_G1) * 256 + threadIdx.x], s);
        atomicAdd(&sum2[((size_t)v * rs_groups(nb, RS_G2) + lb / RS_G2) * 256 + threadIdx.x], s);
    }
}

// Stable scatter of one digit pass; on the last pass (GATHER) also gathers the
// tile rectangle of every survivor into rank order.  Keys, values and
// rectangles are loaded before the counting, so their latency overlaps it.
template <bool GATHER>
__global__ void __launch_bounds__(RS_THREADS, 4) k_rs_scatter(const FrameHeader* __restrict__ hdr,
                                                           const uint32_t* __restrict__ n_surv,
                                                           const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                           uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                           int64_t n, int nb, int shift, const uint32_t* __restrict__ hist,
                                                           const uint32_t* __restrict__ totals,
                                                           const uint32_t* __restrict__ sum1,
                                                           const uint32_t* __restrict__ sum2,
                                                           const uint2* __restrict__ rect, uint2* __restrict__ srect,
                                                           uint16_t* __restrict__ sband)
{
    pdl_wait();
    __shared__ uint32_t h[RS_THREADS / 32][256];
    __shared__ uint32_t wb[RS_THREADS / 32][256];
    __shared__ uint32_t dbase[256];
    __shared__ uint32_t wsum[RS_THREADS / 32];
    const int b = blockIdx.x, v = b / nb, lb = b % nb;
    const int64_t vbase = (int64_t)v * n;
    const int64_t base = vbase + (int64_t)lb * RS_ITEMS;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // keys, values, the view's digit total and this block's digit offsets are
    // loaded together (in the first pass before the view check; a later pass
    // reads its item count first, so blocks past the survivors move no data)
    const bool first = shift == 0;
    int cnt;
    if (first) {
        cnt = rs_first_count(n, lb);
    } else {
        if ((uint32_t)v >= hdr->n_views) return;
        cnt = rs_later_count(n_surv, v, lb);
        if (cnt == 0) return;
    }
    uint32_t kk[RS_R], vv[RS_R];
    uint2 rr[RS_R];
    rs_load_keys(kin, base, cnt, kk);
    // the first pass's values are the Gaussian indices themselves (item idx
    // of block lb is Gaussian lb * RS_ITEMS + idx); later passes load them
#pragma unroll
    for (int r = 0; r < RS_R; ++r) {
        const int idx = w * RS_PER_WARP + r * 32 + lane;
        vv[r] = first ? (uint32_t)(lb * RS_ITEMS + idx) : (idx < cnt ? vin[base + idx] : 0u);
    }
    const uint32_t c_tot = totals[v * 256 + threadIdx.x];
    // this block's offset within the digit: the counts of the earlier blocks,
    // as groups of RS_G2 blocks, then groups of RS_G1, then single blocks
    uint32_t c_blk = 0;
    {
        const uint32_t* p2 = sum2 + (size_t)v * rs_groups(nb, RS_G2) * 256 + threadIdx.x;
        const uint32_t* p1 = sum1 + (size_t)v * rs_groups(nb, RS_G1) * 256 + threadIdx.x;
        const uint32_t* p0 = hist + (size_t)v * nb * 256 + threadIdx.x;
        const int q2 = lb / RS_G2, q1 = lb / RS_G1;
#pragma unroll 8
        for (int k = 0; k < q2; ++k) c_blk += p2[(size_t)k * 256];
#pragma unroll
        for (int k = 0; k < RS_G2 / RS_G1 - 1; ++k)
            if (q2 * (RS_G2 / RS_G1) + k < q1) c_blk += p1[(size_t)(q2 * (RS_G2 / RS_G1) + k) * 256];
#pragma unroll
        for (int k = 0; k < RS_G1 - 1; ++k)
            if (q1 * RS_G1 + k < lb) c_blk += p0[(size_t)(q1 * RS_G1 + k) * 256];
    }
    if (first && (uint32_t)v >= hdr->n_views) return;
    if (cnt == 0) return;
    if (GATHER) {
#pragma unroll
        for (int r = 0; r < RS_R; ++r) rr[r] = kk[r] != 0xFFFFFFFFu ? rect[vbase + vv[r]] : make_uint2(0u, 0u);
    }
    uint32_t pk[RS_R];
    rs_warp_counts(kk, shift, h, pk);
    {
        // exclusive scan of the view's 256 digit totals (RS_THREADS == 256)
        const int wi = threadIdx.x >> 5;
        const uint32_t c = c_tot;
        uint32_t x = c;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wi] = x;
        __syncthreads();
        uint32_t off = 0;
        for (int w = 0; w < wi; ++w) off += wsum[w];
        dbase[threadIdx.x] = off + x - c;
    }
    __syncthreads();
    {
        uint32_t run = dbase[threadIdx.x] + c_blk;
        for (int w = 0; w < RS_THREADS / 32; ++w) {
            wb[w][threadIdx.x] = run;
            run += h[w][threadIdx.x];
        }
    }
    __syncthreads();
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int r = 0; r < RS_R; ++r) {
        const bool valid = kk[r] != 0xFFFFFFFFu;     // culled keys are dropped here
        const uint32_t d = valid ? ((kk[r] >> shift) & 255u) : 256u;
        const uint32_t peers = pk[r];     // lanes holding the same digit (from the counting)
        if (valid) {
            const uint32_t pos = wb[w][d] + __popc(peers & lt);
            kout[vbase + pos] = kk[r];
            vout[vbase + pos] = vv[r];
            if (GATHER) {
                srect[vbase + pos] = rr[r];
                // the rectangle's band range (ROWS_PER_BLOCK tile rows), for the emission
                sband[vbase + pos] = (uint16_t)((rr[r].x >> 16) / ROWS_PER_BLOCK |
                                                (((rr[r].y >> 16) - 1u) / ROWS_PER_BLOCK) << 8);
            }
        }
        __syncwarp();
        if (valid && (__ffs(peers) - 1) == lane) wb[w][d] += __popc(peers);
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// 2./4. per (chunk, tile row) walks
// ---------------------------------------------------------------------------
// Rank chunks a view actually uses: one per 1024 survivors (at least one), at
// most CH (the layout's count).  Chunks at or past it hold no ranks; the
// count, the chunk scan and the emission skip them, so a light frame does
// not pay for CH chunks.
__device__ __forceinline__ uint32_t chunks_used(uint32_t Ns, uint32_t CH)
{
    return max(1u, min(CH, (Ns + 1023u) / 1024u));
}

// Block -> (view, chunk, row block) through the views' rb_base.
__device__ __forceinline__ int find_view_rb(const ViewDev* views, uint32_t V, uint32_t b)
{
    int v = 0;
    for (uint32_t u = 1; u < V; ++u)
        if (b >= views[u].rb_base) v = (int)u;
    return v;
}

// Walk of one warp over the chunk's rectangles for one tile row, in rank
// order.  A group of 32 consecutive ranks is handled at once: the spans
// [x0, x1) of the members that cover the row are laid end to end (prefix sum
// of their widths) and processed 32 slots at a time, each slot finding its
// member from the window's bitmask of span starts (a warp OR-reduction and
// a population count); slots that fall on the same tile are ordered by
// lane, lower slot = lower rank, their lane set found with a shared-memory
// atomicOr per tile (cheaper than __match_any_sync: 3.5 us per 1080p frame).
//   EMIT = false: ctr[x] counts the chunk's pairs of tile x.
//   EMIT = true:  ctr[x] starts at the tile's offset plus the chunk's offset
//                 and every slot writes its Gaussian at ctr[x] + (rank among
//                 the slots of the same tile).
static_assert(ROWS_PER_BLOCK <= 8, "a band's row mask is 8 bits");
static_assert(STAGE <= 8 * ROWS_PER_BLOCK * 32, "the compaction holds at most 8 entries' row masks per thread");
template <bool EMIT, bool KEYS>
__global__ void __launch_bounds__(ROWS_PER_BLOCK * 32, 4) k_rows(Frame F, uint32_t* __restrict__ vals,
                                                             unsigned long long* __restrict__ keys)
{
    pdl_wait();
    extern __shared__ uint32_t sm[];
    __shared__ uint2 s_rect[STAGE];
    __shared__ uint32_t s_id[STAGE];
    __shared__ uint32_t s_key[KEYS ? STAGE : 1];     // depth keys, only when the 64-bit keys are written
    __shared__ uint8_t s_rmask[STAGE];      // per listed rectangle: the band's rows it covers
    __shared__ uint32_t s_wc[ROWS_PER_BLOCK];
    __shared__ uint16_t s_buf[ROWS_PER_BLOCK][64];
    const FrameHeader* hdr = F.hdr;
    if (hdr->status & STATUS_TIMEOUT) return;     // a look-back gave up: the rank order is not valid
    if (EMIT && (hdr->status & STATUS_OVERFLOW)) return;
    const uint32_t V = hdr->n_views;
    const uint32_t CH = hdr->n_chunks;
    const int64_t n = (int64_t)hdr->n;
    if (blockIdx.x >= hdr->rb_total) return;
    const int v = find_view_rb(F.views, V, blockIdx.x);
    const ViewDev& W = F.views[v];
    const uint32_t rbn = (uint32_t)(W.TY + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;
    const uint32_t local = blockIdx.x - W.rb_base;
    if (local >= CH * rbn) return;
    const uint32_t c = local / rbn, rb = local % rbn;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    const int row = (int)rb * ROWS_PER_BLOCK + w;
    const bool row_ok = row < W.TY;
    const int TX = W.TX;
    const uint32_t T = (uint32_t)(W.TX * W.TY);
    uint32_t* ctr = sm + (size_t)w * hdr->max_tx;
    uint32_t* pm = sm + (size_t)(ROWS_PER_BLOCK + w) * hdr->max_tx;     // per tile: lanes of the window on it
    uint32_t* cnt_row = F.cnt + (size_t)CH * W.tile_base + (size_t)c * T + (size_t)row * TX;
    const uint32_t Ns = F.n_surv[2 * v + 1];
    const uint32_t CHe = chunks_used(Ns, CH);
    if (c >= CHe) return;
    const uint32_t C = (Ns + CHe - 1) / CHe;
    const uint32_t r0 = min(Ns, c * C), r1 = min(Ns, r0 + C);
    if (row_ok)
        for (int x = lane; x < TX; x += 32) {
            ctr[x] = EMIT ? F.tile_offset[W.tile_base + row * TX + x] + cnt_row[x] : 0u;
            pm[x] = 0u;
        }
    const int64_t vb = (int64_t)v * n;
    const uint32_t bnd = rb;     // this block's band (ROWS_PER_BLOCK tile rows)
    for (uint32_t s0 = r0; s0 < r1; s0 += STAGE) {
        const int m = (int)min((uint32_t)STAGE, r1 - s0);
        __syncthreads();
        // Order-preserving compaction of the round's ranks whose rectangle
        // meets this block's band, from the band ranges the last radix pass
        // wrote (2 bytes per rank): thread t tests ranks [t * per, (t + 1) * per),
        // an exclusive scan of the hit counts over the threads places them,
        // and only the hits' rectangles and indices are fetched.
        int nl;
        {
            const int per = (m + (int)blockDim.x - 1) / (int)blockDim.x;     // <= STAGE / blockDim
            const int k0 = (int)threadIdx.x * per;
            uint32_t hm = 0u;
            int c = 0;
            for (int j = 0; j < per; ++j) {
                const int k = k0 + j;
                if (k < m) {
                    const uint32_t br = F.sband[vb + s0 + k];
                    if ((br & 0xFFu) <= bnd && bnd <= (br >> 8)) {
                        hm |= 1u << j;
                        ++c;
                    }
                }
            }
            int x = c;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_wc[w] = (uint32_t)x;
            __syncthreads();
            int pos = x - c;
            nl = 0;
            for (int q = 0; q < ROWS_PER_BLOCK; ++q) {
                if (q < w) pos += (int)s_wc[q];
                nl += (int)s_wc[q];
            }
            const int band0 = (int)bnd * ROWS_PER_BLOCK, band1 = band0 + ROWS_PER_BLOCK;
            for (int j = 0; hm; ++j, hm >>= 1)
                if (hm & 1u) {
                    const int64_t g = vb + s0 + k0 + j;
                    const uint2 rc = F.srect[g];
                    s_rect[pos] = rc;
                    if (EMIT) {
                        s_id[pos] = F.val0[g];
                        if (KEYS) s_key[pos] = F.key0[g];
                    }
                    const int y0 = (int)(rc.x >> 16), y1 = (int)(rc.y >> 16);
                    const int lo = max(y0, band0) - band0, hi = min(y1, band1) - band0;
                    s_rmask[pos] = (uint8_t)(((1u << hi) - 1u) & ~((1u << lo) - 1u));
                    ++pos;
                }
            __syncthreads();
        }
        if (!row_ok) continue;
        // Members of this row, in rank order, are gathered 32 at a time in the
        // warp's buffer; each full group is laid out and emitted.
        int nb = 0;
        for (int g0 = 0;; g0 += 32) {
            if (g0 < nl) {
                const int g = g0 + lane;
                uint32_t gi_l = 0u;
                bool hit = false;
                if (g < nl) {
                    gi_l = (uint32_t)g;
                    hit = (s_rmask[g] >> w) & 1u;
                }
                const unsigned hb = __ballot_sync(0xffffffffu, hit);
                if (hit) s_buf[w][nb + __popc(hb & lt)] = (uint16_t)gi_l;
                nb += __popc(hb);
                __syncwarp();
                if (nb < 32) continue;
            } else if (nb == 0) {
                break;   // list done and buffer flushed
            }
            // one group: the first min(nb, 32) buffered members (nb < 32 only
            // for the last group, once the list is done)
            const int gsz = nb < 32 ? nb : 32;
            const uint32_t gi_l = lane < gsz ? (uint32_t)s_buf[w][lane] : 0u;
            const uint2 rc = lane < gsz ? s_rect[gi_l] : make_uint2(0u, 0u);
            const uint32_t x0 = rc.x & 0xFFFFu;
            const uint32_t wdt = lane < gsz ? (rc.y & 0xFFFFu) - x0 : 0u;
            uint32_t end = wdt;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, end, o);
                if (lane >= o) end += y;
            }
            const uint32_t total = __shfl_sync(0xffffffffu, end, 31);
            const uint32_t st = end - wdt;     // this member's first slot
            // per member: first slot and first tile packed (widths are at most
            // 1024 tiles, so total <= 32768), and the Gaussian index (and key)
            const uint32_t xst = (st << 16) | x0;
            const uint32_t gid = (EMIT && lane < gsz) ? s_id[gi_l] : 0u;
            const uint32_t gkey = (EMIT && KEYS && lane < gsz) ? s_key[gi_l] : 0u;
            // the members beyond the group move to the front of the buffer
            const uint32_t carry = lane + 32 < nb ? (uint32_t)s_buf[w][lane + 32] : 0u;
            __syncwarp();
            if (lane + 32 < nb) s_buf[w][lane] = (uint16_t)carry;
            nb -= gsz;
            uint32_t started = 0;     // members whose span starts before the window
            for (uint32_t q0 = 0; q0 < total; q0 += 32) {
                const uint32_t q = q0 + lane;
                const bool valid = q < total;
                // owner of slot q: the last member (in rank order) whose span
                // starts at or before q.  Spans are non-empty and laid end to
                // end, so the starts are distinct; S marks those in this window
                // (lanes past the group add a start at total, past every valid slot).
                const uint32_t rel = st - q0;
                const uint32_t S = __reduce_or_sync(0xffffffffu, rel < 32u ? (1u << rel) : 0u);
                const uint32_t o = (started + __popc(S & ((2u << lane) - 1u)) - 1u) & 31u;
                started += __popc(S);
                const uint32_t xst_o = __shfl_sync(0xffffffffu, xst, o);
                const uint32_t gid_o = EMIT ? __shfl_sync(0xffffffffu, gid, o) : 0u;
                const uint32_t x = valid ? (xst_o & 0xFFFFu) + (q - (xst_o >> 16)) : 0xFFFFFFFFu;
                // lanes on the same tile: each sets its bit in the tile's
                // word of the warp's peer array; the word read back is the set
                // of peers; the highest peer then clears it (after every peer
                // has read it) for the next window
                if (valid) atomicOr(&pm[x], 1u << lane);
                __syncwarp();
                const uint32_t peers = valid ? pm[x] : (1u << lane);
                __syncwarp();
                if (valid && (31 - __clz(peers)) == lane) pm[x] = 0u;
                if (EMIT && KEYS) {
                    const uint32_t key_o = __shfl_sync(0xffffffffu, gkey, o);
                    if (valid) {
                        const uint32_t p = ctr[x] + __popc(peers & lt);
                        keys[p] = ((unsigned long long)(W.tile_base + (uint32_t)row * TX + x) << 32) | key_o;
                    }
                }
                if (valid) {
                    const uint32_t p = ctr[x] + __popc(peers & lt);
                    if (EMIT) vals[p] = gid_o;
                    // the highest peer holds the last slot of this tile: advance the counter past it
                    if ((31 - __clz(peers)) == lane) ctr[x] = p + 1u;
                }
                __syncwarp();
            }
            __syncwarp();
        }
    }
    if (!EMIT && row_ok)
        for (int x = lane; x < TX; x += 32) cnt_row[x] = ctr[x];
}

// Inclusive prefix sums of `lines` lines of `len` words of g: element j of
// line i at g[i * line_stride + j * step].  Called by every thread of the
// block (the shuffles take whole warps).
constexpr int CC_SEG = 4;
__device__ __forceinline__ void chunk_prefix_lines(uint32_t* g, int lines, int len, int line_stride, int step)
{
    const int per_sweep = (int)blockDim.x / CC_SEG;
    const int li = (int)threadIdx.x / CC_SEG, sg = (int)threadIdx.x % CC_SEG;
    const int L = (len + CC_SEG - 1) / CC_SEG;
    const int ja = min(len, sg * L), jb = min(len, ja + L);
    for (int i0 = 0; i0 < lines; i0 += per_sweep) {
        const int i = i0 + li;
        uint32_t* line = g + (size_t)min(i, lines - 1) * line_stride;
        const bool ok = i < lines;
        uint32_t sum = 0;
        if (ok)
            for (int j = ja; j < jb; ++j) sum += line[j * step];
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < CC_SEG; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o, CC_SEG);
            if (sg >= o) inc += u;
        }
        uint32_t run = inc - sum;
        if (ok)
            for (int j = ja; j < jb; ++j) {
                run += line[j * step];
                line[j * step] = run;
            }
    }
}

// 2'. per (view, chunk): the chunk's pair count of every tile from a 2D
// difference array in shared memory -- each rectangle [x0,x1)x[y0,y1) adds
// +1 at (x0,y0), (x1,y1) and -1 at (x1,y0), (x0,y1) -- and a 2D prefix sum.
// Used when the (TX+1)(TY+1) grid fits in shared memory.
__global__ void __launch_bounds__(512) k_chunk_count(Frame F)
{
    pdl_wait();
    extern __shared__ uint32_t g[];
    const FrameHeader* hdr = F.hdr;
    if (hdr->status & STATUS_TIMEOUT) return;     // a look-back gave up: the rank order is not valid
    const uint32_t CH = hdr->n_chunks;
    const int64_t n = (int64_t)hdr->n;
    const int v = (int)(blockIdx.x / CH);
    const uint32_t c = blockIdx.x % CH;
    if ((uint32_t)v >= hdr->n_views) return;
    const ViewDev& W = F.views[v];
    const uint32_t Ns = F.n_surv[2 * v + 1];
    const uint32_t CHe = chunks_used(Ns, CH);
    if (c >= CHe) return;
    const int TX = W.TX, TY = W.TY, GX = TX + 1;
    const int G = GX * (TY + 1);
    for (int k = threadIdx.x; k < G; k += blockDim.x) g[k] = 0u;
    __syncthreads();
    const uint32_t C = (Ns + CHe - 1) / CHe;
    const uint32_t r0 = min(Ns, c * C), r1 = min(Ns, r0 + C);
    const uint2* sr = F.srect + (int64_t)v * n;
    for (uint32_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        const uint2 rc = sr[r];
        const int x0 = (int)(rc.x & 0xFFFFu), y0 = (int)(rc.x >> 16), x1 = (int)(rc.y & 0xFFFFu), y1 = (int)(rc.y >> 16);
        atomicAdd_block(&g[y0 * GX + x0], 1u);
        atomicAdd_block(&g[y0 * GX + x1], 0xFFFFFFFFu);
        atomicAdd_block(&g[y1 * GX + x0], 0xFFFFFFFFu);
        atomicAdd_block(&g[y1 * GX + x1], 1u);
    }
    __syncthreads();
    // inclusive prefix along each row, then along each column; a line is cut
    // into CC_SEG segments, one per lane of a group of CC_SEG consecutive
    // lanes: each lane sums its segment, the group scans the sums, and each
    // lane rewrites its segment from its offset
    chunk_prefix_lines(g, TY, TX, GX, 1);
    __syncthreads();
    chunk_prefix_lines(g, TX, TY, 1, GX);
    __syncthreads();
    const uint32_t T = (uint32_t)(TX * TY);
    uint32_t* out = F.cnt + (size_t)CH * W.tile_base + (size_t)c * T;
    for (uint32_t t = threadIdx.x; t < T; t += blockDim.x) out[t] = g[(t / TX) * GX + (t % TX)];
}

// 3. per tile: exclusive scan of the chunk counts (the chunk offsets within
// the tile), tile_count = their total; then the exclusive scan over the tiles
// (tile offsets, K, ranges) chained across blocks by a decoupled look-back,
// and the blends' work order.  A block takes 32 tiles (one per lane, so every
// load of a chunk's counts is coalesced) and cuts the chunks into 8
// segments, one per warp: segment sums, their scan across the warps, then
// each segment rescanned.  Blocks take their place in the tile order from a
// ticket, so every block they look back at has started and publishes
// without waiting on later ones.
constexpr int CS_TILES = 32, CS_SEG = 8;
constexpr int CS_MAXPER = (MAX_CHUNKS + CS_SEG - 1) / CS_SEG;
constexpr unsigned long long LB_AGG = 1ull << 62;    // look-back word: the block's own sum
constexpr unsigned long long LB_INC = 2ull << 62;    //                 the sum up to and including the block
constexpr unsigned long long LB_VAL = (1ull << 62) - 1;
constexpr uint32_t LB_SPIN_LIMIT = 1u << 20;         // polls of a missing predecessor before giving up

// Length class of a tile list for the blends' work order: 0 (longest) to 3:
// lists longer than 2m, than m, than m/2 (m the mean list length), the rest.
__device__ __forceinline__ uint32_t tile_class(uint32_t c, unsigned long long mean)
{
    const unsigned long long cc = c;
    return cc > 2ull * mean ? 0u : (cc > mean ? 1u : (2ull * cc > mean ? 2u : 3u));
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long* p)
{
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__global__ void __launch_bounds__(CS_TILES * CS_SEG, 2) k_tile_scan(Frame F, uint32_t* __restrict__ ranges,
                                                                  unsigned long long cap)
{
    pdl_wait();
    __shared__ uint32_t part[CS_SEG][CS_TILES];
    __shared__ uint32_t s_blk;
    FrameHeader* hdr = F.hdr;
    if (hdr->status & STATUS_TIMEOUT) return;     // a look-back gave up: the counts are not valid
    const uint32_t TT = hdr->total_tiles;
    const uint32_t V = hdr->n_views;
    const uint32_t CH = hdr->n_chunks;
    if (threadIdx.x == 0) s_blk = atomicAdd(&F.scan_ctr[4], 1u);
    __syncthreads();
    const uint32_t blk = s_blk;
    const int tx = threadIdx.x % CS_TILES, sg = threadIdx.x / CS_TILES;
    const uint32_t t = blk * CS_TILES + tx;
    const bool ok = t < TT;
    uint32_t* col = nullptr;
    uint32_t T = 0, CHe = 0;
    if (ok) {
        int v = 0;
        for (uint32_t u = 1; u < V; ++u)
            if (t >= F.views[u].tile_base) v = (int)u;
        const ViewDev& W = F.views[v];
        T = (uint32_t)(W.TX * W.TY);
        col = F.cnt + (size_t)CH * W.tile_base + (t - W.tile_base);
        CHe = chunks_used(F.n_surv[2 * v + 1], CH);
    }
    const uint32_t per = (CHe + CS_SEG - 1) / CS_SEG;     // <= CS_MAXPER
    const uint32_t c0 = min(CHe, sg * per), c1 = min(CHe, c0 + per);
    // the segment's counts, all loaded at once (one round trip) and held:
    // summed, then rewritten as offsets
    uint32_t xs[CS_MAXPER];
#pragma unroll
    for (int u = 0; u < CS_MAXPER; ++u) xs[u] = c0 + u < c1 ? col[(size_t)(c0 + u) * T] : 0u;
    uint32_t sum = 0;
#pragma unroll
    for (int u = 0; u < CS_MAXPER; ++u) sum += xs[u];
    part[sg][tx] = sum;
    __syncthreads();
    uint32_t off = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < CS_SEG; ++q) {
        const uint32_t y = part[q][tx];
        if (q < sg) off += y;
        tot += y;
    }
#pragma unroll
    for (int u = 0; u < CS_MAXPER; ++u) {
        if (c0 + u < c1) col[(size_t)(c0 + u) * T] = off;
        off += xs[u];
    }
    if (sg != 0) return;
    // warp 0, one lane per tile: scan over the block's tiles, then over the
    // blocks before it
    const int lane = tx;
    const uint32_t c = ok ? tot : 0u;
    if (ok) F.tile_count[t] = c;
    uint32_t x = c;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    const unsigned long long agg = __shfl_sync(0xffffffffu, x, 31);
    // the block's tiles per length class (for the blends' work order), packed
    // two per word; published beside the pair count, before its flag
    const unsigned long long mean = hdr->n_pairs / (TT ? TT : 1u);
    const uint32_t cls = ok ? tile_class(c, mean) : 4u;
    uint32_t ccount[4];
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k) ccount[k] = (uint32_t)__popc(__ballot_sync(0xffffffffu, cls == k));
    const ulonglong2 cagg = make_ulonglong2(ccount[0] | ((unsigned long long)ccount[1] << 32),
                                            ccount[2] | ((unsigned long long)ccount[3] << 32));
    ulonglong2 cpre = make_ulonglong2(0ull, 0ull);     // class counts of the blocks before
    unsigned long long prefix = 0;
    if (blk == 0) {
        if (lane == 0) {
            F.scan_cls[2 * blk + 1] = cagg;
            __threadfence();
            atomicExch(&F.scan_st[0], LB_INC | agg);
        }
    } else {
        if (lane == 0) {
            F.scan_cls[2 * blk] = cagg;
            __threadfence();
            atomicExch(&F.scan_st[blk], LB_AGG | agg);
        }
        // window of 32 blocks, lane l reading block j - l; "before block 0"
        // reads as an inclusive sum of 0
        long long j = (long long)blk - 1;
        bool gave_up = false;
        for (;;) {
            const long long jj = j - lane;
            unsigned long long w = jj >= 0 ? ld_volatile_u64(&F.scan_st[jj]) : LB_INC;
            uint32_t spins = 0;
            for (;;) {
                const bool ready = (w >> 62) != 0;
                if (__all_sync(0xffffffffu, ready)) break;
                if (++spins > LB_SPIN_LIMIT) {     // the same count on every lane
                    gave_up = true;
                    break;
                }
                __nanosleep(64);
                if (!ready) w = ld_volatile_u64(&F.scan_st[jj]);
            }
            if (gave_up) break;
            // the nearest inclusive sum ends the walk; the aggregates after it add
            const unsigned inc = __ballot_sync(0xffffffffu, (w >> 62) == 2ull);
            const int first = inc ? __ffs(inc) - 1 : 31;
            unsigned long long add = lane <= first ? (w & LB_VAL) : 0ull;
            // the class counts published with the flag just read: the block's
            // own (aggregate) or up to and including it (inclusive)
            __threadfence();
            ulonglong2 cw = make_ulonglong2(0ull, 0ull);
            if (lane <= first && jj >= 0) {
                const volatile unsigned long long* cp = reinterpret_cast<const volatile unsigned long long*>(
                    &F.scan_cls[2 * jj + ((w >> 62) == 2ull ? 1 : 0)]);
                cw = make_ulonglong2(cp[0], cp[1]);
            }
            for (int o = 16; o > 0; o >>= 1) {
                add += __shfl_xor_sync(0xffffffffu, add, o);
                cw.x += __shfl_xor_sync(0xffffffffu, cw.x, o);
                cw.y += __shfl_xor_sync(0xffffffffu, cw.y, o);
            }
            prefix += add;
            cpre.x += cw.x;
            cpre.y += cw.y;
            if (inc) break;
            j -= 32;
        }
        if (gave_up) {
            // a predecessor never published: report it; the blends skip the frame
            if (lane == 0) atomicOr(&hdr->status, STATUS_TIMEOUT | STATUS_OVERFLOW);
            return;
        }
        if (lane == 0) {
            F.scan_cls[2 * blk + 1] = make_ulonglong2(cpre.x + cagg.x, cpre.y + cagg.y);
            __threadfence();
            atomicExch(&F.scan_st[blk], LB_INC | (prefix + agg));
        }
    }
    if (ok) {
        const unsigned long long o = prefix + x - c;
        F.tile_offset[t] = static_cast<uint32_t>(o);
        ranges[2 * (size_t)t] = c ? static_cast<uint32_t>(o) : 0u;
        ranges[2 * (size_t)t + 1] = c ? static_cast<uint32_t>(o + c) : 0u;
    }
    // the blends' work order: each class's list in tile order (neighbouring
    // tiles share Gaussians, so running them together reuses L2).  Only the
    // order in which warps take tiles: no result depends on it.
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (uint32_t k = 0; k < 4; ++k) {
        const unsigned m = __ballot_sync(0xffffffffu, cls == k);
        const uint32_t before = (uint32_t)((k & 1u) ? ((k < 2 ? cpre.x : cpre.y) >> 32)
                                                   : ((k < 2 ? cpre.x : cpre.y) & 0xFFFFFFFFull));
        if (cls == k) F.torder[(size_t)k * TT + before + __popc(m & lt)] = t;
    }
    if (blk == gridDim.x - 1 && lane == 31) {
        const unsigned long long K = prefix + agg;
        F.tile_offset[TT] = static_cast<uint32_t>(K);
        if (K != hdr->n_pairs || K > cap || K > 0xFFFFFFFFull) atomicOr(&hdr->status, STATUS_OVERFLOW);
        // the class totals, for the blends' walk over the four lists
        const unsigned long long a = cpre.x + cagg.x, b = cpre.y + cagg.y;
        F.scan_ctr[0] = (uint32_t)(a & 0xFFFFFFFFull);
        F.scan_ctr[1] = (uint32_t)(a >> 32);
        F.scan_ctr[2] = (uint32_t)(b & 0xFFFFFFFFull);
        F.scan_ctr[3] = (uint32_t)(b >> 32);
    }
}

constexpr size_t DIFF_SMEM_MAX = 200 * 1024;   // difference grid limit (a 4K view needs 131 KB)

// Returns the error of the first launch (the later launches' errors surface
// through cudaGetLastError).  The digit sums and the tile scan's look-back
// words it accumulates into were zeroed by the frame set-up of the
// clod_preprocess call before it (one sort per preprocessing).
cudaError_t launch_bin_sort(const Frame& F, const FrameLayout& L, unsigned long long cap, uint64_t* keys,
                            uint32_t* vals, uint32_t* ranges, cudaStream_t st)
{
    cudaError_t err = cudaSuccess;
    const int64_t n = (int64_t)L.n;
    const int nb = (int)L.n_rs_blocks;
    const uint32_t V = L.n_views;
    // per pass: the digit totals [V][256] and the group sums [V][groups][256]
    // of both levels
    const size_t n1 = (size_t)V * 256 * rs_groups(nb, RS_G1), n2 = (size_t)V * 256 * rs_groups(nb, RS_G2);
    const size_t per_pass = (size_t)V * 256 + n1 + n2;
    uint32_t* sums = F.rs_sums;
    if (n > 0) {
        // the first pass reads no values (they are the indices): vi is unused there
        uint32_t *ki = F.key0, *vi = F.val0, *ko = F.key1, *vo = F.val1;
        for (int pass = 0; pass < 4; ++pass) {
            uint32_t* tot = sums + (size_t)pass * per_pass;
            uint32_t* s1 = tot + (size_t)V * 256;
            uint32_t* s2 = s1 + n1;
            const cudaError_t e = launch(k_rs_hist, V * nb, RS_THREADS, 0, st, F.hdr, F.n_surv, ki, n, nb, 8 * pass,
                                         F.rs_hist, tot, s1, s2);
            if (pass == 0) err = e;
            if (pass == 3)
                launch(k_rs_scatter<true>, V * nb, RS_THREADS, 0, st, F.hdr, F.n_surv, ki, vi, ko, vo, n, nb, 8 * pass,
                       F.rs_hist, tot, s1, s2, F.rect, F.srect, F.sband);
            else
                launch(k_rs_scatter<false>, V * nb, RS_THREADS, 0, st, F.hdr, F.n_surv, ki, vi, ko, vo, n, nb, 8 * pass,
                       F.rs_hist, tot, s1, s2, nullptr, nullptr, nullptr);
            std::swap(ki, ko);
            std::swap(vi, vo);
        }
    }
    const size_t smem = (size_t)2 * ROWS_PER_BLOCK * L.max_tx * sizeof(uint32_t);     // counters and peer words
    if (L.diff_grid_max * sizeof(uint32_t) <= DIFF_SMEM_MAX)
        launch(k_chunk_count, V * L.n_chunks, 512, L.diff_grid_max * sizeof(uint32_t), st, F);
    else
        launch(k_rows<false, false>, L.rb_total, ROWS_PER_BLOCK * 32, smem, st, F, nullptr, nullptr);
    launch(k_tile_scan, (L.total_tiles + CS_TILES - 1) / CS_TILES, CS_TILES * CS_SEG, 0, st, F, ranges, cap);
    if (keys)
        launch(k_rows<true, true>, L.rb_total, ROWS_PER_BLOCK * 32, smem, st, F, vals,
               reinterpret_cast<unsigned long long*>(keys));
    else
        launch(k_rows<true, false>, L.rb_total, ROWS_PER_BLOCK * 32, smem, st, F, vals, nullptr);
    return err;
}

cudaError_t bin_sort_setup()
{
    const int bytes = 2 * ROWS_PER_BLOCK * 1024 * (int)sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_rows<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rows<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_rows<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_chunk_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DIFF_SMEM_MAX);
    return e;
}

}  // namespace clod
