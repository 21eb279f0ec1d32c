// clod_internal.cuh -- device-side records and the fixed FP32 operation
// sequences shared by the libclod kernels.
//
// Every translation unit is compiled with --fmad=false: a*b+c is never fused
// implicitly; every fused multiply-add below is an explicit __fmaf_rn.  Together
// with IEEE division and square root (__fdiv_rn, __fsqrt_rn) this makes each
// quantity that decides an integer outcome a fixed sequence of correctly
// rounded operations.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/clod.h"

namespace clod {

// Programmatic dependent launch.  The library launches its kernels with
// launch() below, which lets the next kernel of the stream be launched while
// this one drains: a dependent launch gap (about 4 us on a 152-SM part for a
// grid of a wave or more) shrinks to about 1.4 us.  Every kernel therefore
// begins with pdl_wait(), before any access to global memory: it returns once
// every earlier kernel of the stream has completed and its writes are visible
// (at once for a launch without the dependency), so no kernel overlaps its
// predecessor's accesses.  No kernel releases its dependents early: blocks
// waiting in pdl_wait would hold SM slots that kernels of other streams (other
// frames in flight) could use.
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... P, typename... A>
inline cudaError_t launch(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

constexpr int TILE = 16;
constexpr int BLOCK_PIX = TILE * TILE;  // 256 threads per tile block
constexpr int MAX_VIEWS = 64;

// Depth-rank sort and emission geometry.
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 2048;          // keys per radix-sort block (8 per thread)
constexpr int RS_G1 = 8, RS_G2 = 64;    // radix-sort blocks per group of the two offset-sum levels
__host__ __device__ inline int rs_groups(int nb, int g) { return (nb + g - 1) / g; }
constexpr int ROWS_PER_BLOCK = 8;       // tile rows per emission block (one warp each)
constexpr int MAX_CHUNKS = 256;         // rank chunks per view
constexpr int STAGE = 2048;             // rectangles staged in shared memory at a time
constexpr uint64_t CHUNK_COUNT_WORDS = 1ull << 24;   // per (chunk, tile) counts aimed at: 64 MB, within L2

// Rank chunks per view of a launch with `tiles` tiles in all: one per 1024
// Gaussians, at most MAX_CHUNKS, and no more than keep the per (chunk, tile)
// counts (chunks x tiles words, written, scanned and read by the emission)
// near CHUNK_COUNT_WORDS -- but at least 32, so that the emission keeps
// enough blocks (a launch of eight 4K views takes 64).
inline uint32_t chunk_count(uint64_t n, uint64_t tiles)
{
    const uint64_t by_n = (n + 1023) / 1024;
    uint64_t by_mem = CHUNK_COUNT_WORDS / (tiles ? tiles : 1);
    if (by_mem < 32) by_mem = 32;
    uint64_t c = by_n < by_mem ? by_n : by_mem;
    if (c < 1) c = 1;
    if (c > (uint64_t)MAX_CHUNKS) c = MAX_CHUNKS;
    return (uint32_t)c;
}

// Frame header at offset 0 of a frame workspace.
struct FrameHeader {
    uint64_t n;             // Gaussians
    uint32_t n_views;
    uint32_t total_tiles;
    unsigned long long n_pairs;  // K = sum of tiles touched over survivors
    uint32_t status;        // STATUS_* bits
    uint32_t n_chunks;      // rank chunks per view
    uint32_t n_rs_blocks;   // radix-sort blocks per view
    uint32_t max_tx;        // widest view, in tiles
    uint32_t rb_total;      // blocks of the emission grids in use
    uint32_t work[4];       // scheduling counters
};
constexpr uint32_t STATUS_OVERFLOW = 1u;
constexpr uint32_t STATUS_TIMEOUT = 2u;

// Device view record (host-built from clod_view).
struct ViewDev {
    float R[9];
    float t[3];
    float fx, fy, cx, cy, near_z;
    float c[3];
    float s_v, tau, eps;
    float bg[3];
    int32_t W, H, TX, TY;   // this view's pixels and tiles (the window of a region view)
    int32_t ox, oy;         // window origin in the full frame, pixels (multiples of 16)
    int32_t FW, FH;         // full frame (W, H for a whole-frame view)
    uint32_t flags;
    uint32_t budget;        // > 0: top-budget mask by alpha''
    uint32_t tile_base;     // global id of this view's first tile
    uint32_t rb_base;       // first block of this view in the emission grids
    uint64_t pix_base;      // first pixel of this view in packed outputs
    float* out_img;         // optional per-view outputs (else packed at pix_base)
    float* out_T;
    uint32_t* out_nc;
};

// Radix select of the primitive budget: per-view state and digit counts.
constexpr int SEL_BINS = 2048;          // 11-bit digits
constexpr int SEL_PASSES = 6;           // 64-bit keys: 11 + 11 + 10 + 11 + 11 + 10 bits
struct SelState {
    unsigned long long T;       // smallest selected key (valid once done)
    unsigned long long prefix;  // high digits fixed so far
    uint32_t remaining;         // selections still to make below the prefix
    uint32_t done;
    uint32_t pad[2];
};

struct FrameLayout {
    size_t header, views, dmax_key, n_surv, rec0, rec1, rec2, depth, rect, tile_count, tile_offset, torder,
        key0, val0, key1, val1, srect, sband, rs_hist, rs_sums, scan, scan_cls, cnt, sel, sel_hist, total;
    uint32_t total_tiles, n_views, n_chunks, n_rs_blocks, rb_total, max_tx;
    uint32_t fast_exp;      // host only: the frame's views carry CLOD_FAST_EXP
    uint64_t n;
    size_t diff_grid_max;   // max over views of (TX + 1) (TY + 1)
};

// Pointers into a frame workspace.
struct Frame {
    FrameHeader* hdr;
    ViewDev* views;
    unsigned long long* dmax_key;
    uint32_t* n_surv;
    float4* rec0;
    float4* rec1;
    float4* rec2;           // (b, reach half-extents x, y, power floor)
    float* depth;
    uint2* rect;
    uint32_t* tile_count;
    uint32_t* tile_offset;
    uint32_t* torder;       // the blends' work order: four class lists of capacity total_tiles
    unsigned long long* scan_st;  // tile scan: per block of 32 tiles, look-back flag and value
    ulonglong2* scan_cls;   // tile scan: per block, its tiles per length class, own and inclusive
    uint32_t* scan_ctr;     // [0..3] tiles per length class, [4] tile-scan block ticket
    uint32_t* key0;         // depth-rank sort ping-pong: keys (depth bits) / values (index)
    uint32_t* val0;
    uint32_t* key1;
    uint32_t* val1;
    uint2* srect;           // tile rectangles in depth-rank order
    uint16_t* sband;        // their emission bands, first | last << 8, in depth-rank order
    uint32_t* rs_hist;      // radix-sort digit counts [view][block][256]
    uint32_t* rs_sums;      // per pass: digit totals [view][256], then the two levels of group sums (zeroed at set-up)
    uint32_t* cnt;          // per (view, chunk, tile) pair counts, then offsets
    SelState* sel;          // primitive-budget select state [view]
    uint32_t* sel_hist;     // its digit counts [view][SEL_BINS]
};

// Tile of the blends' i-th work item.  The tile scan writes the work order
// as four class lists (longest tile lists first), list k at torder + k TT
// holding scan_ctr[k] tiles; together they hold every tile once.
__device__ __forceinline__ uint32_t work_tile(const Frame& F, uint32_t i, uint32_t TT)
{
    uint32_t k = 0;
    while (k < 3) {
        const uint32_t c = F.scan_ctr[k];
        if (i < c) break;
        i -= c;
        ++k;
    }
    return F.torder[(size_t)k * TT + i];
}

// Key of the primitive-budget order: larger key = kept first (alpha''
// descending, then index ascending).  alpha'' >= 0, so its bits order like
// its value.
__device__ __forceinline__ unsigned long long budget_key(float a2, uint32_t i)
{
    return (static_cast<unsigned long long>(__float_as_uint(a2)) << 32) | (0xFFFFFFFFu - i);
}

// ---------------------------------------------------------------------------
// exp_spec: x = k ln2 + r, k = floor(x * L2E) with L2E = 1/ln2 rounded up to
// float (so r >= 0), e^r by a degree-9 Taylor polynomial (Horner), capped at
// 2, scaled by 2^k.  Monotone non-decreasing; 0 below -80 and for NaN.
// ---------------------------------------------------------------------------
// exp_spec for x already known to lie in [-80, 0] (the blends call it after
// their power range test); exp_spec below adds the range handling.
__device__ __forceinline__ float exp_spec_core(float x)
{
    const float L2E = __int_as_float(0x3FB8AA3C);
    const float MAGIC = 12582912.0f;
    const float LN2HI = __int_as_float(0x3F317218);
    const float LN2LO = __int_as_float(0xB102E308);
    float t = __fmaf_rn(x, L2E, MAGIC);
    float kf = __fsub_rn(t, MAGIC);
    // t lies in [MAGIC - 116, MAGIC], where floats are spaced by 1: its bits
    // minus MAGIC's are the same integer as kf (no float-to-int conversion)
    int ki = __float_as_int(t) - 0x4B400000;
    if (__fmaf_rn(x, L2E, -kf) < 0.0f) {
        kf = __fsub_rn(kf, 1.0f);
        ki -= 1;
    }
    float r = __fmaf_rn(kf, -LN2HI, x);
    r = __fmaf_rn(kf, -LN2LO, r);
    float p = __int_as_float(0x3638EF1D);            // 1/9!
    p = __fmaf_rn(p, r, __int_as_float(0x37D00D01)); // 1/8!
    p = __fmaf_rn(p, r, __int_as_float(0x39500D01)); // 1/7!
    p = __fmaf_rn(p, r, __int_as_float(0x3AB60B61)); // 1/6!
    p = __fmaf_rn(p, r, __int_as_float(0x3C088889)); // 1/5!
    p = __fmaf_rn(p, r, __int_as_float(0x3D2AAAAB)); // 1/4!
    p = __fmaf_rn(p, r, __int_as_float(0x3E2AAAAB)); // 1/3!
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    p = fminf(p, 2.0f);
    // p in [1, 2], k >= -116: the scaled value is a normal float
    return __int_as_float(__float_as_int(p) + (ki << 23));
}

__device__ __forceinline__ float exp_spec(float x)
{
    if (!(x >= -80.0f)) return 0.0f;
    if (x > 0.0f) x = 0.0f;
    return exp_spec_core(x);
}

// The blends' exponential when a frame asks for CLOD_FAST_EXP: e^p =
// 2^(p log2 e) on the special-function unit (ex2.approx; one product and one
// MUFU instruction instead of the ~24 of exp_spec_core).  For p in [-5.6, 0]
// its relative error is a few 1e-7 (the rounding of p log2 e and the unit's
// approximation), so opacities follow the real-arithmetic blend within FP32
// rounding, but a decision near a threshold may fall differently from the
// software exponential's: such images are not bit-reproducible by another
// implementation of the FP32 sequence.
__device__ __forceinline__ float exp_fast(float p)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__fmul_rn(p, 1.44269504088896341f)));
    return y;
}

// Exponential of a blend power p in [-5.6, 0]: the software exponential
// (FAST = false, the reproducible decision arithmetic) or exp_fast.
template <bool FAST>
__device__ __forceinline__ float blend_exp(float p)
{
    return FAST ? exp_fast(p) : exp_spec_core(p);
}

// Camera-frame point: t_k = R_k0 x + (R_k1 y + (R_k2 z + t_k)), fused.
__device__ __forceinline__ void cam_point(const ViewDev& V, float x, float y, float z, float& tx, float& ty,
                                          float& tz)
{
    tx = __fmaf_rn(V.R[0], x, __fmaf_rn(V.R[1], y, __fmaf_rn(V.R[2], z, V.t[0])));
    ty = __fmaf_rn(V.R[3], x, __fmaf_rn(V.R[4], y, __fmaf_rn(V.R[5], z, V.t[1])));
    tz = __fmaf_rn(V.R[6], x, __fmaf_rn(V.R[7], y, __fmaf_rn(V.R[8], z, V.t[2])));
}

// Camera distance d = sqrt(e0^2 + e1^2 + e2^2), e = mu - c.
__device__ __forceinline__ float cam_dist(const ViewDev& V, float x, float y, float z, float& e0, float& e1,
                                          float& e2)
{
    e0 = __fsub_rn(x, V.c[0]);
    e1 = __fsub_rn(y, V.c[1]);
    e2 = __fsub_rn(z, V.c[2]);
    return __fsqrt_rn(__fmaf_rn(e0, e0, __fmaf_rn(e1, e1, __fmul_rn(e2, e2))));
}

// Projected centre u = fx (tx/tz) + cx, v likewise.
__device__ __forceinline__ void project(const ViewDev& V, float tx, float ty, float tz, float& u, float& v)
{
    u = __fmaf_rn(V.fx, __fdiv_rn(tx, tz), V.cx);
    v = __fmaf_rn(V.fy, __fdiv_rn(ty, tz), V.cy);
}

// Centre inside the view frustum: t_z > near and (u, v) in [0,W]x[0,H] of the
// full frame.
__device__ __forceinline__ bool in_frustum(const ViewDev& V, float tx, float ty, float tz)
{
    if (!(tz > V.near_z)) return false;
    float u, v;
    project(V, tx, ty, tz, u, v);
    return (u >= 0.0f) && (u <= static_cast<float>(V.FW)) && (v >= 0.0f) && (v <= static_cast<float>(V.FH));
}

// Attenuated opacity of Eq. 2 (dmax = 0 means no Gaussian in the frustum).
__device__ __forceinline__ float attenuated_opacity(const ViewDev& V, float alpha, float sigma, float d,
                                                    float dmax)
{
    if (V.flags & CLOD_LOD_OFF) return alpha;
    float dn;
    if (V.flags & CLOD_NO_NORMALIZE) dn = d;
    else dn = dmax > 0.0f ? __fdiv_rn(d, dmax) : 0.0f;
    float q = __fmul_rn(dn, V.s_v);
    float sr = sigma > 0.0f ? sigma : 0.0f;
    float den = __fmaf_rn(__fadd_rn(sr, sr), sr, V.eps);
    float xx = __fdiv_rn(__fmul_rn(q, q), den);
    return __fmul_rn(alpha, exp_spec(-xx));
}

__device__ __forceinline__ float decode_dmax(unsigned long long key)
{
    return __uint_as_float(static_cast<uint32_t>(key >> 32));
}

// Spherical-harmonic basis constants (real basis, degree <= 3, colour-model signs).
#define CLOD_SH_C0 0.28209479177387814f
#define CLOD_SH_C1 0.4886025119029199f
#define CLOD_SH_C2_0 1.0925484305920792f
#define CLOD_SH_C2_1 (-1.0925484305920792f)
#define CLOD_SH_C2_2 0.31539156525252005f
#define CLOD_SH_C2_3 (-1.0925484305920792f)
#define CLOD_SH_C2_4 0.5462742152960396f
#define CLOD_SH_C3_0 (-0.5900435899266435f)
#define CLOD_SH_C3_1 2.890611442640554f
#define CLOD_SH_C3_2 (-0.4570457994644658f)
#define CLOD_SH_C3_3 0.3731763325901154f
#define CLOD_SH_C3_4 (-0.4570457994644658f)
#define CLOD_SH_C3_5 1.445305721320277f
#define CLOD_SH_C3_6 (-0.5900435899266435f)

// Basis values b[0..(deg+1)^2) at unit direction (x, y, z).
__device__ __forceinline__ void sh_basis(float x, float y, float z, int deg, float* b)
{
    b[0] = CLOD_SH_C0;
    if (deg < 1) return;
    b[1] = __fmul_rn(-CLOD_SH_C1, y);
    b[2] = __fmul_rn(CLOD_SH_C1, z);
    b[3] = __fmul_rn(-CLOD_SH_C1, x);
    if (deg < 2) return;
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float xy = __fmul_rn(x, y), yz = __fmul_rn(y, z), xz = __fmul_rn(x, z);
    b[4] = __fmul_rn(CLOD_SH_C2_0, xy);
    b[5] = __fmul_rn(CLOD_SH_C2_1, yz);
    b[6] = __fmul_rn(CLOD_SH_C2_2, __fsub_rn(__fsub_rn(__fadd_rn(zz, zz), xx), yy));
    b[7] = __fmul_rn(CLOD_SH_C2_3, xz);
    b[8] = __fmul_rn(CLOD_SH_C2_4, __fsub_rn(xx, yy));
    if (deg < 3) return;
    b[9] = __fmul_rn(CLOD_SH_C3_0, __fmul_rn(y, __fsub_rn(__fmul_rn(3.0f, xx), yy)));
    b[10] = __fmul_rn(CLOD_SH_C3_1, __fmul_rn(xy, z));
    b[11] = __fmul_rn(CLOD_SH_C3_2, __fmul_rn(y, __fsub_rn(__fsub_rn(__fmul_rn(4.0f, zz), xx), yy)));
    b[12] = __fmul_rn(CLOD_SH_C3_3,
                      __fmul_rn(z, __fsub_rn(__fsub_rn(__fmul_rn(2.0f, zz), __fmul_rn(3.0f, xx)), __fmul_rn(3.0f, yy))));
    b[13] = __fmul_rn(CLOD_SH_C3_4, __fmul_rn(x, __fsub_rn(__fsub_rn(__fmul_rn(4.0f, zz), xx), yy)));
    b[14] = __fmul_rn(CLOD_SH_C3_5, __fmul_rn(z, __fsub_rn(xx, yy)));
    b[15] = __fmul_rn(CLOD_SH_C3_6, __fmul_rn(x, __fsub_rn(xx, __fmul_rn(3.0f, yy))));
}

// The blend's per-(pixel, Gaussian) opacity, in the decision arithmetic:
// power = dx (-A/2 dx + -B dy) + (-C/2 dy) dy, a = min(0.99, alpha'' exp(power)).
// Returns a < 0 for "skip".  power < -5.6 is skipped without evaluating the
// exponential: exp_spec(-5.6) < 1/255 and exp_spec is monotone, so for such
// powers a < 1/255 for every alpha'' <= 1 and the outcome is the same.
__device__ __forceinline__ float blend_alpha(float dx, float dy, float nA, float nB, float nC, float a2)
{
    const float power = __fmaf_rn(dx, __fmaf_rn(nA, dx, __fmul_rn(nB, dy)), __fmul_rn(__fmul_rn(nC, dy), dy));
    if (!(power <= 0.0f && power >= -5.6f)) return -1.0f;   // also skips a NaN power (exp_spec(NaN) = 0)
    const float a = fminf(0.99f, __fmul_rn(a2, exp_spec_core(power)));   // power in [-5.6, 0]
    return a < (1.0f / 255.0f) ? -1.0f : a;
}

// Host: device record of one view (camera, level of detail, region, budget;
// the packing fields tile_base, rb_base, pix_base and outputs are left 0) and
// its validation.
void view_record(const clod_view& w, ViewDev& d);
clod_status check_view(const clod_view& w, int index);

// Half-extents (x, y) of a box around (u, v) that holds every pixel centre
// where the blend's opacity can reach 1/255, from the stored record values
// nA = -A/2, nB = -B, nC = -C/2 and alpha''.  There power >= P* =
// max(-5.6, -ln(255 alpha'')), i.e. the ellipse d^T Q d <= 2|P*| (Q the
// conic), whose half-extents are sqrt(2|P*| Sigma_xx), sqrt(2|P*| Sigma_yy)
// with Sigma = Q^-1; widened by 0.1% (+0.01 px) so FP32 rounding of the power
// can never put a reached pixel outside.  -inf: reaches no pixel (alpha'' <
// 1/255).  +inf: a conic so elongated that A C - B^2 loses more than 0.1% of
// A C to cancellation is not trusted (never skipped).  Only a cull: no
// decision depends on its rounding.
__device__ __forceinline__ float2 reach_half_extents(float nA, float nB, float nC, float a2)
{
    const float A = -2.0f * nA, B = -nB, C = -2.0f * nC;
    const float det = A * C - B * B;
    const float a255 = 255.0f * a2;
    const float inf = __int_as_float(0x7f800000);
    if (!(a255 >= 1.0f)) return make_float2(-inf, -inf);
    if (!(det > 1e-3f * (A * C)) || !(A > 0.0f) || !(C > 0.0f)) return make_float2(inf, inf);
    const float P = fminf(5.6f, logf(a255));
    const float r2 = 2.0f * P * 1.001f + 1e-3f;
    return make_float2(sqrtf(r2 * (C / det)) * 1.001f + 0.01f, sqrtf(r2 * (A / det)) * 1.001f + 0.01f);
}

// Lowest power at which the blend's opacity can still reach 1/255 (stored
// with the record; the blend skips lower powers without the exponential).
// a = alpha'' exp_spec(power) >= 1/255 needs power >= -ln(255 alpha'') up to
// the relative errors of exp_spec, the product and logf (each a few 1e-7);
// the floor sits 0.1% + 1e-3 below -logf(255 alpha''), so every skipped
// power has a < 1/255 and would be skipped by the exact test as well.  Never
// below -5.6 (the exponential's range); +inf when alpha'' < 1/255 (no power
// reaches 1/255, since exp_spec <= 1 on powers <= 0).  Only a cull.
__device__ __forceinline__ float power_floor(float a2)
{
    const float a255 = 255.0f * a2;
    if (!(a255 >= 1.0f)) return __int_as_float(0x7f800000);
    return fmaxf(-5.6f, -(logf(a255) * 1.001f + 1e-3f));
}

// Frame workspace layout (256-byte aligned arrays).
FrameLayout frame_layout(uint64_t n, uint32_t n_views, uint32_t total_tiles, uint32_t n_chunks, uint32_t rb_total,
                         uint32_t max_tx, size_t diff_grid_max);
Frame frame_ptrs(void* ws, const FrameLayout& L);

}  // namespace clod
