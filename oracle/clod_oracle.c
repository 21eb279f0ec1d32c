/*
 * clod_oracle.c -- CPU oracle for the CLoD-GS rasterizer hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain, single-threaded
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never does.  It shares no code with the CUDA path.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (no contraction: every operation below rounds exactly where written; fmaf()
 * is the C99 correctly rounded fused multiply-add).
 *
 * What it computes, per view (paper section / equation cited at each step):
 *
 *   Stage I  (FP32, op by op, the discrete decisions and the bit-exact values)
 *     camera distance and view-frustum max          -- Sec. 3.2 (d_i, d'_i)
 *     attenuated opacity and the dynamic-threshold
 *     mask                                           -- Sec. 3.2, Eq. 2 and M_i
 *     EWA projection, conic, 3-sigma radius, tile
 *     rectangle, SH colour                           -- Sec. 3.1 (3DGS primitive,
 *                                                       inherited per Sec. 4.1)
 *   Pairs    emission of (view/tile, depth) keys and a stable sort by key,
 *            tile ranges                             -- Sec. 3.1 ("sorted by depth")
 *   Stage II per-pixel front-to-back blending       -- Sec. 3.1, Eq. 1
 *            decisions (skip, stop, contributor count) taken in the FP32
 *            arithmetic below; colour values accumulated in FP64 from an FP64
 *            re-evaluation of Stage I, and also in FP32.
 *
 * exp_spec: the project's own exponential (Cody-Waite reduction, degree-9
 * Taylor polynomial in Horner form, scaling by 2^k; monotone by
 * construction), used wherever an
 * exponential decides an integer outcome, so that both implementations take
 * every decision on identical bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- view record: flat float array ------------------------------------ */
enum {
    OV_R = 0,       /* 9: world->camera rotation, row-major              */
    OV_T = 9,       /* 3: world->camera translation                      */
    OV_FX = 12, OV_FY = 13, OV_CX = 14, OV_CY = 15,
    OV_NEAR = 16,
    OV_C = 17,      /* 3: camera centre (world)                          */
    OV_S = 20,      /* virtual distance scale s_v                        */
    OV_TAU = 21,    /* base opacity threshold tau                        */
    OV_EPS = 22,    /* epsilon of Eq. 2                                  */
    OV_BG = 23,     /* 3: background colour                              */
    OV_W = 26, OV_H = 27,
    OV_FLAGS = 28,  /* bit 0: level of detail off; bit 1: no normalisation */
    OV_BUDGET = 29, /* primitive budget, the bits of a uint32 (0: threshold mask) */
    OV_SIZE = 32
};
#define ORACLE_LOD_OFF 1
#define ORACLE_NO_NORMALIZE 2
#define TILE 16

static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

/* ======================================================================= */
/* exp_spec                                                                */
/* ======================================================================= */
/* Constants: 1/ln 2 rounded UP to float (so the reduced argument below is
 * never negative); 1.5 * 2^23 (adding it rounds to an integer); ln 2 rounded
 * to nearest; ln 2 minus that float, rounded; 1/n! for n = 0..9. */
#define ES_L2E    1.442695140838623046875f          /* 0x3FB8AA3C */
#define ES_MAGIC  12582912.0f                       /* 0x4B400000 */
#define ES_LN2HI  0.693147182464599609375f          /* 0x3F317218 */
#define ES_LN2LO  (-1.904654212125933356583118438720703125e-09f) /* 0xB102E308 */

/* exp_spec(x) for x <= 0 (inputs above 0 are clamped to 0; below -80 or NaN
 * give 0).  Cody-Waite reduction x = k ln 2 + r with k = floor(x * L2E),
 * e^r by the degree-9 Taylor polynomial in Horner form, capped at 2, times
 * 2^k.  Monotone non-decreasing by construction: r >= 0 and non-decreasing in
 * x for fixed k, every Horner step has non-negative operands, the cap keeps
 * the top of each binade at or below the bottom of the next. */
float oracle_exp_spec(float x)
{
    static const float c[10] = {
        1.0f, 1.0f, 0.5f, 0.16666667163372039794921875f,
        0.041666667908430099487304688f, 0.0083333337679505348205566406f,
        0.0013888889225199818611145020f, 0.00019841270113829523324966431f,
        2.4801587642286904156208038330078125e-05f, 2.7557318844628753140568733215332031e-06f };
    if (!(x >= -80.0f)) return 0.0f;            /* also NaN -> 0 */
    if (x > 0.0f) x = 0.0f;
    /* k = floor(x * L2E) of the exact product */
    float t = fmaf(x, ES_L2E, ES_MAGIC);        /* rounds x*L2E to an integer */
    float kf = t - ES_MAGIC;
    if (fmaf(x, ES_L2E, -kf) < 0.0f) kf = kf - 1.0f;
    /* r = x - k ln 2 in two parts, r >= 0 */
    float r = fmaf(kf, -ES_LN2HI, x);
    r = fmaf(kf, -ES_LN2LO, r);
    /* e^r by the Taylor series of degree 9, Horner form */
    float p = c[9];
    for (int n = 8; n >= 0; --n) p = fmaf(p, r, c[n]);
    p = fminf(p, 2.0f);
    /* times 2^k: exact, the result stays a normal number for k >= -116 */
    return ldexpf(p, (int)kf);
}

void oracle_exp_spec_batch(const float* x, float* y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) y[i] = oracle_exp_spec(x[i]);
}

/* Walk every float in [lo, hi] (lo <= hi <= 0) in increasing order and count
 * the places where exp_spec decreases.  Returns the count; *first receives the
 * first offending input (or 0). */
int64_t oracle_exp_spec_monotone_violations(float lo, float hi, float* first)
{
    int64_t bad = 0;
    *first = 0.0f;
    /* negative floats: larger bit pattern = more negative */
    uint32_t ulo = f2u(lo), uhi = f2u(hi);
    float prev = oracle_exp_spec(lo);
    for (uint32_t u = ulo; ; --u) {
        float x = u2f(u);
        float y = oracle_exp_spec(x);
        if (y < prev) { if (!bad) *first = x; ++bad; }
        prev = y;
        if (u == uhi || u == 0x80000000u) break;
    }
    return bad;
}

/* ======================================================================= */
/* Stage I: FP32 per Gaussian, one view                                    */
/* ======================================================================= */
/* Real spherical-harmonic basis constants (degree <= 3), standard
 * normalisation with the Condon-Shortley phase folded into the signs used
 * below (the convention of the 3DGS colour model). */
#define SH_C0 0.28209479177387814f
#define SH_C1 0.4886025119029199f
static const float SH_C2[5] = { 1.0925484305920792f, -1.0925484305920792f, 0.31539156525252005f,
                                -1.0925484305920792f, 0.5462742152960396f };
static const float SH_C3[7] = { -0.5900435899266435f, 2.890611442640554f, -0.4570457994644658f,
                                0.3731763325901154f, -0.4570457994644658f, 1.445305721320277f,
                                -0.5900435899266435f };

/* FP32 basis values b[0..15] for unit direction (x, y, z). */
static void sh_basis_f32(float x, float y, float z, int deg, float* b)
{
    b[0] = SH_C0;
    if (deg < 1) return;
    b[1] = -SH_C1 * y;
    b[2] = SH_C1 * z;
    b[3] = -SH_C1 * x;
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, yz = y * z, xz = x * z;
    b[4] = SH_C2[0] * xy;
    b[5] = SH_C2[1] * yz;
    b[6] = SH_C2[2] * (((zz + zz) - xx) - yy);
    b[7] = SH_C2[3] * xz;
    b[8] = SH_C2[4] * (xx - yy);
    if (deg < 3) return;
    b[9]  = SH_C3[0] * (y * ((3.0f * xx) - yy));
    b[10] = SH_C3[1] * (xy * z);
    b[11] = SH_C3[2] * (y * (((4.0f * zz) - xx) - yy));
    b[12] = SH_C3[3] * (z * (((2.0f * zz) - (3.0f * xx)) - (3.0f * yy)));
    b[13] = SH_C3[4] * (x * (((4.0f * zz) - xx) - yy));
    b[14] = SH_C3[5] * (z * (xx - yy));
    b[15] = SH_C3[6] * (x * (xx - (3.0f * yy)));
}

/* FP64 basis values (same polynomials, double arithmetic). */
static void sh_basis_f64(double x, double y, double z, int deg, double* b)
{
    b[0] = 0.28209479177387814;
    if (deg < 1) return;
    const double c1 = 0.4886025119029199;
    b[1] = -c1 * y; b[2] = c1 * z; b[3] = -c1 * x;
    if (deg < 2) return;
    double xx = x * x, yy = y * y, zz = z * z;
    b[4] = 1.0925484305920792 * x * y;
    b[5] = -1.0925484305920792 * y * z;
    b[6] = 0.31539156525252005 * (2.0 * zz - xx - yy);
    b[7] = -1.0925484305920792 * x * z;
    b[8] = 0.5462742152960396 * (xx - yy);
    if (deg < 3) return;
    b[9]  = -0.5900435899266435 * y * (3.0 * xx - yy);
    b[10] = 2.890611442640554 * x * y * z;
    b[11] = -0.4570457994644658 * y * (4.0 * zz - xx - yy);
    b[12] = 0.3731763325901154 * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    b[13] = -0.4570457994644658 * x * (4.0 * zz - xx - yy);
    b[14] = 1.445305721320277 * z * (xx - yy);
    b[15] = -0.5900435899266435 * x * (xx - 3.0 * yy);
}

void oracle_sh_basis(const double* dirs, int64_t n, int deg, double* out16)
{
    for (int64_t i = 0; i < n; ++i)
        sh_basis_f64(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], deg, out16 + 16 * i);
}

/* Output record per Gaussian (12 floats):
 *   [0] u  [1] v  [2] alpha''  [3] depth t_z
 *   [4] -A/2  [5] -B  [6] -C/2  [7] radius (pixels)
 *   [8] r  [9] g  [10] b  [11] det of the 2D covariance
 * where (A, B, C) is the conic, the inverse 2D covariance [[A, B], [B, C]]. */
#define REC 12

/* Camera-frame position (step S1). */
static void cam_point(const float* V, float x, float y, float z, float* t)
{
    for (int k = 0; k < 3; ++k)
        t[k] = fmaf(V[OV_R + 3 * k], x, fmaf(V[OV_R + 3 * k + 1], y, fmaf(V[OV_R + 3 * k + 2], z, V[OV_T + k])));
}

/* Order of the primitive budget: alpha'' descending, then index ascending. */
static const float* g_sort_alpha;
static int budget_cmp(const void* pa, const void* pb)
{
    const int64_t a = *(const int64_t*)pa, b = *(const int64_t*)pb;
    const float xa = g_sort_alpha[a], xb = g_sort_alpha[b];
    if (xa != xb) return xa > xb ? -1 : 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* Stage I for one view.  Inputs are the activated parameters.
 * Outputs (length n unless noted):
 *   dist      camera distance d_i
 *   in_view   1 if the centre is in the view frustum (t_z > near, projection in
 *             [0,W]x[0,H])
 *   dmax[0]   max of d over in_view (0 if none); argmax[0] lowest index
 *             attaining it (-1 if none)
 *   alpha_eff attenuated opacity alpha'' (Eq. 2)
 *   mask      M_i = alpha'' > tau * s_v (Sec. 3.2), or with a primitive
 *             budget B the B Gaussians of highest alpha'' (Sec. 4.2)
 *   survive   1 if the Gaussian is rasterized: M_i, t_z > near, finite
 *             projection, det > 0, non-empty tile rectangle
 *   rec       REC floats (above) for survivors, zeros otherwise
 *   rect      tile rectangle [x0, y0, x1, y1) for survivors, zeros otherwise
 *   tiles     tiles touched (x1-x0)*(y1-y0), 0 for the culled
 */
void oracle_stage1(int64_t n, int deg, const float* means, const float* scales, const float* quats,
                   const float* opacity, const float* sh, const float* decay, const float* V,
                   float* dist, uint8_t* in_view, float* dmax, int64_t* argmax,
                   float* alpha_eff, uint8_t* mask, uint8_t* survive, float* rec,
                   int32_t* rect, uint32_t* tiles)
{
    const int W = (int)V[OV_W], H = (int)V[OV_H];
    const float Wf = (float)W, Hf = (float)H;
    const int TX = (W + TILE - 1) / TILE, TY = (H + TILE - 1) / TILE;
    const int flags = (int)V[OV_FLAGS];
    const int K = (deg + 1) * (deg + 1);

    /* --- d_i and the view-frustum max (Sec. 3.2) ---------------------- */
    float best = 0.0f;
    int64_t best_i = -1;
    for (int64_t i = 0; i < n; ++i) {
        const float* m = means + 3 * i;
        float t[3];
        cam_point(V, m[0], m[1], m[2], t);
        float e0 = m[0] - V[OV_C], e1 = m[1] - V[OV_C + 1], e2 = m[2] - V[OV_C + 2];
        float d = sqrtf(fmaf(e0, e0, fmaf(e1, e1, e2 * e2)));
        dist[i] = d;
        int iv = 0;
        if (t[2] > V[OV_NEAR]) {
            float u = fmaf(V[OV_FX], t[0] / t[2], V[OV_CX]);
            float v = fmaf(V[OV_FY], t[1] / t[2], V[OV_CY]);
            iv = (u >= 0.0f) && (u <= Wf) && (v >= 0.0f) && (v <= Hf);
        }
        in_view[i] = (uint8_t)iv;
        if (iv && (best_i < 0 || d > best)) { best = d; best_i = i; }
    }
    dmax[0] = best;
    argmax[0] = best_i;

    const float s = V[OV_S];
    const float thr = s * V[OV_TAU];
    const float tanx = (0.5f * Wf) / V[OV_FX];
    const float tany = (0.5f * Hf) / V[OV_FY];
    const float limx = 1.3f * tanx, limy = 1.3f * tany;

    /* --- attenuated opacity, Eq. 2, and the mask M_i ------------------ */
    for (int64_t i = 0; i < n; ++i) {
        float a2;
        int M;
        if (flags & ORACLE_LOD_OFF) {
            a2 = opacity[i];
            M = 1;
        } else {
            float dn;
            if (flags & ORACLE_NO_NORMALIZE) dn = dist[i];
            else dn = best > 0.0f ? dist[i] / best : 0.0f;
            float q = dn * s;
            float sr = decay[i] > 0.0f ? decay[i] : 0.0f;          /* ReLU(sigma_d) */
            float den = fmaf(sr + sr, sr, V[OV_EPS]);               /* 2 sigma^2 + eps */
            float xx = (q * q) / den;
            a2 = opacity[i] * oracle_exp_spec(-xx);
            M = a2 > thr;
        }
        alpha_eff[i] = a2;
        mask[i] = (uint8_t)M;
    }
    /* Primitive budget (Sec. 4.2: primitives of highest attenuated opacity):
     * the mask becomes the first min(budget, n) Gaussians in the order
     * (alpha'' descending, index ascending). */
    uint32_t budget;
    memcpy(&budget, &V[OV_BUDGET], sizeof(budget));
    if (budget > 0 && n > 0) {
        int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
        if (order) {
            for (int64_t i = 0; i < n; ++i) order[i] = i;
            g_sort_alpha = alpha_eff;
            qsort(order, (size_t)n, sizeof(int64_t), budget_cmp);
            for (int64_t i = 0; i < n; ++i) mask[i] = 0;
            for (int64_t r = 0; r < n && r < (int64_t)budget; ++r) mask[order[r]] = 1;
            free(order);
        }
    }

    for (int64_t i = 0; i < n; ++i) {
        float* R = rec + REC * i;
        memset(R, 0, sizeof(float) * REC);
        rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
        tiles[i] = 0;
        survive[i] = 0;
        if (!mask[i]) continue;
        const float a2 = alpha_eff[i];

        const float* m = means + 3 * i;
        float t[3];
        cam_point(V, m[0], m[1], m[2], t);
        const float tx = t[0], ty = t[1], tz = t[2];
        if (!(tz > V[OV_NEAR])) continue;
        const float u = fmaf(V[OV_FX], tx / tz, V[OV_CX]);
        const float v = fmaf(V[OV_FY], ty / tz, V[OV_CY]);
        if (!isfinite(u) || !isfinite(v)) continue;

        /* --- 3D covariance Sigma = R S S^T R^T ------------------------- */
        const float* qq = quats + 4 * i;
        float n2 = fmaf(qq[0], qq[0], fmaf(qq[1], qq[1], fmaf(qq[2], qq[2], qq[3] * qq[3])));
        if (!(n2 > 0.0f)) continue;
        float inv = 1.0f / sqrtf(n2);
        float w = qq[0] * inv, x = qq[1] * inv, y = qq[2] * inv, z = qq[3] * inv;
        float xx = x * x, yy = y * y, zz = z * z;
        float xy = x * y, xz = x * z, yz = y * z;
        float wx = w * x, wy = w * y, wz = w * z;
        float r[9];
        r[0] = fmaf(-2.0f, yy + zz, 1.0f);
        r[1] = 2.0f * (xy - wz);
        r[2] = 2.0f * (xz + wy);
        r[3] = 2.0f * (xy + wz);
        r[4] = fmaf(-2.0f, xx + zz, 1.0f);
        r[5] = 2.0f * (yz - wx);
        r[6] = 2.0f * (xz - wy);
        r[7] = 2.0f * (yz + wx);
        r[8] = fmaf(-2.0f, xx + yy, 1.0f);
        const float* sc = scales + 3 * i;
        float Mm[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Mm[3 * a + b] = r[3 * a + b] * sc[b];
        float S[9];
        for (int a = 0; a < 3; ++a)
            for (int b = a; b < 3; ++b) {
                float v_ = fmaf(Mm[3 * a], Mm[3 * b], fmaf(Mm[3 * a + 1], Mm[3 * b + 1], Mm[3 * a + 2] * Mm[3 * b + 2]));
                S[3 * a + b] = v_;
                S[3 * b + a] = v_;
            }

        /* --- EWA: cov2D = J W Sigma W^T J^T + 0.3 I ------------------- */
        float txc = fminf(limx, fmaxf(-limx, tx / tz)) * tz;
        float tyc = fminf(limy, fmaxf(-limy, ty / tz)) * tz;
        float tz2 = tz * tz;
        float j00 = V[OV_FX] / tz, j02 = -(V[OV_FX] * txc) / tz2;
        float j11 = V[OV_FY] / tz, j12 = -(V[OV_FY] * tyc) / tz2;
        const float* Wv = V + OV_R;
        float T0[3], T1[3];
        for (int k = 0; k < 3; ++k) {
            T0[k] = fmaf(j00, Wv[k], j02 * Wv[6 + k]);
            T1[k] = fmaf(j11, Wv[3 + k], j12 * Wv[6 + k]);
        }
        float U0[3], U1[3];
        for (int k = 0; k < 3; ++k) {
            U0[k] = fmaf(T0[0], S[k], fmaf(T0[1], S[3 + k], T0[2] * S[6 + k]));
            U1[k] = fmaf(T1[0], S[k], fmaf(T1[1], S[3 + k], T1[2] * S[6 + k]));
        }
        float ca = fmaf(U0[0], T0[0], fmaf(U0[1], T0[1], U0[2] * T0[2])) + 0.3f;
        float cb = fmaf(U0[0], T1[0], fmaf(U0[1], T1[1], U0[2] * T1[2]));
        float cc = fmaf(U1[0], T1[0], fmaf(U1[1], T1[1], U1[2] * T1[2])) + 0.3f;

        float det = fmaf(ca, cc, -(cb * cb));
        if (!(det > 0.0f)) continue;
        float idet = 1.0f / det;
        float A = cc * idet, B = -cb * idet, C = ca * idet;

        /* --- 3-sigma radius and tile rectangle ------------------------- */
        float mid = 0.5f * (ca + cc);
        float disc = fmaxf(0.1f, fmaf(mid, mid, -det));
        float lam = mid + sqrtf(disc);
        float rad = ceilf(3.0f * sqrtf(lam));
        float fx0 = floorf((u - rad) * 0.0625f), fx1 = floorf((u + rad) * 0.0625f);
        float fy0 = floorf((v - rad) * 0.0625f), fy1 = floorf((v + rad) * 0.0625f);
        float TXm = (float)TX - 1.0f, TYm = (float)TY - 1.0f;
        if (fx1 < 0.0f || fx0 > TXm || fy1 < 0.0f || fy0 > TYm) continue;
        int x0 = fx0 < 0.0f ? 0 : (int)fx0;
        int x1 = fx1 > TXm ? TX : (int)fx1 + 1;
        int y0 = fy0 < 0.0f ? 0 : (int)fy0;
        int y1 = fy1 > TYm ? TY : (int)fy1 + 1;

        /* --- colour from SH, viewing direction (mu - c)/|mu - c| ------- */
        float e0 = m[0] - V[OV_C], e1 = m[1] - V[OV_C + 1], e2 = m[2] - V[OV_C + 2];
        float d = dist[i];
        float bsh[16];
        sh_basis_f32(e0 / d, e1 / d, e2 / d, deg, bsh);
        float col[3];
        for (int ch = 0; ch < 3; ++ch) {
            float acc = bsh[0] * sh[(size_t)K * 3 * i + ch];
            for (int k = 1; k < K; ++k) acc = fmaf(bsh[k], sh[(size_t)K * 3 * i + 3 * k + ch], acc);
            col[ch] = fmaxf(acc + 0.5f, 0.0f);
        }

        survive[i] = 1;
        R[0] = u; R[1] = v; R[2] = a2; R[3] = tz;
        R[4] = -0.5f * A; R[5] = -B; R[6] = -0.5f * C; R[7] = rad;
        R[8] = col[0]; R[9] = col[1]; R[10] = col[2]; R[11] = det;
        rect[4 * i] = x0; rect[4 * i + 1] = y0; rect[4 * i + 2] = x1; rect[4 * i + 3] = y1;
        tiles[i] = (uint32_t)((x1 - x0) * (y1 - y0));
    }
}

/* ======================================================================= */
/* FP64 re-evaluation of the continuous Stage I values                     */
/* ======================================================================= */
/* Same formulas in double arithmetic, with libm exp, for Gaussians that the
 * FP32 stage kept; the d_max used is d(argmax) recomputed in double.
 * rec64 per Gaussian: u, v, alpha'', A, B, C, r, g, b (9 doubles). */
#define REC64 9
void oracle_stage1_f64(int64_t n, int deg, const float* means, const float* scales, const float* quats,
                       const float* opacity, const float* sh, const float* decay, const float* V,
                       int64_t argmax, const uint8_t* survive, double* rec64)
{
    const double W = V[OV_W], H = V[OV_H];
    const int flags = (int)V[OV_FLAGS];
    const int K = (deg + 1) * (deg + 1);
    double Rv[9], tv[3], c[3];
    for (int k = 0; k < 9; ++k) Rv[k] = V[OV_R + k];
    for (int k = 0; k < 3; ++k) { tv[k] = V[OV_T + k]; c[k] = V[OV_C + k]; }
    const double fx = V[OV_FX], fy = V[OV_FY], cx = V[OV_CX], cy = V[OV_CY];
    double dmax = 0.0;
    if (argmax >= 0) {
        const float* m = means + 3 * argmax;
        double e0 = (double)m[0] - c[0], e1 = (double)m[1] - c[1], e2 = (double)m[2] - c[2];
        dmax = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
    }
    const double limx = 1.3 * (0.5 * W / fx), limy = 1.3 * (0.5 * H / fy);
    for (int64_t i = 0; i < n; ++i) {
        double* o = rec64 + REC64 * i;
        memset(o, 0, sizeof(double) * REC64);
        if (!survive[i]) continue;
        const float* m = means + 3 * i;
        double mu[3] = { m[0], m[1], m[2] };
        double t[3];
        for (int k = 0; k < 3; ++k) t[k] = Rv[3 * k] * mu[0] + Rv[3 * k + 1] * mu[1] + Rv[3 * k + 2] * mu[2] + tv[k];
        double e[3] = { mu[0] - c[0], mu[1] - c[1], mu[2] - c[2] };
        double d = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        double a2 = opacity[i];
        if (!(flags & ORACLE_LOD_OFF)) {
            double dn = (flags & ORACLE_NO_NORMALIZE) ? d : (dmax > 0.0 ? d / dmax : 0.0);
            double sr = decay[i] > 0.0f ? (double)decay[i] : 0.0;
            double q = dn * (double)V[OV_S];
            a2 = (double)opacity[i] * exp(-(q * q) / (2.0 * sr * sr + (double)V[OV_EPS]));
        }
        const float* qq = quats + 4 * i;
        double qn = sqrt((double)qq[0] * qq[0] + (double)qq[1] * qq[1] + (double)qq[2] * qq[2] + (double)qq[3] * qq[3]);
        double w = qq[0] / qn, x = qq[1] / qn, y = qq[2] / qn, z = qq[3] / qn;
        double r[9] = { 1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y) };
        const float* sc = scales + 3 * i;
        double S[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += r[3 * a + k] * r[3 * b + k] * (double)sc[k] * (double)sc[k];
                S[3 * a + b] = acc;
            }
        double txz = t[0] / t[2], tyz = t[1] / t[2];
        double txc = fmin(limx, fmax(-limx, txz)) * t[2];
        double tyc = fmin(limy, fmax(-limy, tyz)) * t[2];
        double J[6] = { fx / t[2], 0.0, -fx * txc / (t[2] * t[2]), 0.0, fy / t[2], -fy * tyc / (t[2] * t[2]) };
        double T[6];
        for (int a = 0; a < 2; ++a)
            for (int k = 0; k < 3; ++k) T[3 * a + k] = J[3 * a] * Rv[k] + J[3 * a + 1] * Rv[3 + k] + J[3 * a + 2] * Rv[6 + k];
        double cov[4];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += T[3 * a + k] * S[3 * k + l] * T[3 * b + l];
                cov[2 * a + b] = acc;
            }
        double ca = cov[0] + 0.3, cb = cov[1], cc = cov[3] + 0.3;
        double det = ca * cc - cb * cb;
        double bsh[16];
        sh_basis_f64(e[0] / d, e[1] / d, e[2] / d, deg, bsh);
        o[0] = fx * txz + cx;
        o[1] = fy * tyz + cy;
        o[2] = a2;
        o[3] = cc / det; o[4] = -cb / det; o[5] = ca / det;
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.0;
            for (int k = 0; k < K; ++k) acc += bsh[k] * (double)sh[(size_t)K * 3 * i + 3 * k + ch];
            acc += 0.5;
            o[6 + ch] = acc > 0.0 ? acc : 0.0;
        }
    }
}

/* ======================================================================= */
/* Pairs: emission, stable sort by key, tile ranges                        */
/* ======================================================================= */
/* For each survivor i in index order and each tile of its rectangle in
 * row-major order, emit key = ((tile_base + ty*TX + tx) << 32) | bits(t_z)
 * and value i.  Returns the number of pairs written (at most cap). */
int64_t oracle_emit_pairs(int64_t n, const float* V, uint32_t tile_base, const uint8_t* survive,
                          const float* rec, const int32_t* rect, uint64_t* keys, uint32_t* vals, int64_t cap)
{
    const int W = (int)V[OV_W];
    const int TX = (W + TILE - 1) / TILE;
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!survive[i]) continue;
        uint64_t dbits = f2u(rec[REC * i + 3]);
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i]; tx < rect[4 * i + 2]; ++tx) {
                if (k < cap) {
                    keys[k] = ((uint64_t)(tile_base + (uint32_t)(ty * TX + tx)) << 32) | dbits;
                    vals[k] = (uint32_t)i;
                }
                ++k;
            }
    }
    return k;
}

/* Stable merge sort of (key, value) by key. */
static void merge_sort(uint64_t* k, uint32_t* v, uint64_t* tk, uint32_t* tv, int64_t n)
{
    if (n < 2) return;
    int64_t h = n / 2;
    merge_sort(k, v, tk, tv, h);
    merge_sort(k + h, v + h, tk, tv, n - h);
    int64_t a = 0, b = h, o = 0;
    while (a < h && b < n) {
        if (k[b] < k[a]) { tk[o] = k[b]; tv[o] = v[b]; ++b; }
        else { tk[o] = k[a]; tv[o] = v[a]; ++a; }
        ++o;
    }
    while (a < h) { tk[o] = k[a]; tv[o] = v[a]; ++a; ++o; }
    while (b < n) { tk[o] = k[b]; tv[o] = v[b]; ++b; ++o; }
    memcpy(k, tk, sizeof(uint64_t) * n);
    memcpy(v, tv, sizeof(uint32_t) * n);
}

int oracle_stable_sort(uint64_t* keys, uint32_t* vals, int64_t n)
{
    uint64_t* tk = (uint64_t*)malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    uint32_t* tv = (uint32_t*)malloc(sizeof(uint32_t) * (n > 0 ? n : 1));
    if (!tk || !tv) { free(tk); free(tv); return -1; }
    merge_sort(keys, vals, tk, tv, n);
    free(tk); free(tv);
    return 0;
}

/* ranges[2t], ranges[2t+1] = first and one-past-last index of sorted keys whose
 * high word is t; [0, 0) for tiles without pairs. */
void oracle_ranges(const uint64_t* keys, int64_t n, int64_t n_tiles, uint32_t* ranges)
{
    memset(ranges, 0, sizeof(uint32_t) * 2 * n_tiles);
    for (int64_t k = 0; k < n; ++k) {
        uint32_t t = (uint32_t)(keys[k] >> 32);
        if (k == 0 || (uint32_t)(keys[k - 1] >> 32) != t) ranges[2 * t] = (uint32_t)k;
        if (k == n - 1 || (uint32_t)(keys[k + 1] >> 32) != t) ranges[2 * t + 1] = (uint32_t)(k + 1);
    }
}

/* ======================================================================= */
/* Stage II: per-pixel blending (Eq. 1)                                    */
/* ======================================================================= */
typedef struct { uint32_t depth; uint32_t id; } cand_t;

static int cand_cmp(const void* a, const void* b)
{
    const cand_t* x = (const cand_t*)a;
    const cand_t* y = (const cand_t*)b;
    if (x->depth != y->depth) return x->depth < y->depth ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

/* Render the given tiles of one view.
 * For each pixel (px, py) of a listed tile, the candidates are every survivor
 * whose tile rectangle contains that tile, taken in ascending (t_z bits,
 * index) order -- "sorted by depth" (Sec. 3.1) with ties broken by index.
 *
 * Per candidate (FP32 decision arithmetic):
 *   dx = u - (px + 0.5), dy = v - (py + 0.5)
 *   power = dx * (-A/2 dx + -B dy) + (-C/2 dy) dy        (fused as written)
 *   skip if power > 0
 *   a = min(0.99, alpha'' * exp_spec(power)); skip if a < 1/255
 *   T' = T (1 - a); stop (excluding this one) if T' < 1e-4
 *   colour += rgb * (a T); T = T'; n_contrib = position + 1
 * Output colour = colour + T * bg.  The FP64 image repeats the accumulation
 * with the FP64 values for exactly the candidates the FP32 decisions kept.
 *
 * img32: 3 x H x W floats, img64: 3 x H x W doubles (may be NULL),
 * T32: H x W, T64: H x W (may be NULL), ncontrib: H x W.
 * If contrib_pix/contrib_gid are given, the (pixel, Gaussian) contributing
 * pairs are appended in blending order up to contrib_cap; the return value is
 * the total number of contributing pairs (or -1 on allocation failure). */
int64_t oracle_render(int64_t n, const float* V, const uint8_t* survive, const float* rec,
                      const int32_t* rect, const double* rec64, const int32_t* tile_list, int64_t n_list,
                      float* img32, double* img64, float* T32, double* T64, uint32_t* ncontrib,
                      int64_t* contrib_pix, int32_t* contrib_gid, int64_t contrib_cap,
                      int64_t* evaluated)
{
    const int W = (int)V[OV_W], H = (int)V[OV_H];
    const int TX = (W + TILE - 1) / TILE;
    const float one255 = 1.0f / 255.0f;
    cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (n > 0 ? n : 1));
    if (!cand) return -1;
    int64_t total = 0, evals = 0;
    for (int64_t li = 0; li < n_list; ++li) {
        const int tile = tile_list[li];
        const int tx = tile % TX, ty = tile / TX;
        int64_t nc = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (!survive[i]) continue;
            const int32_t* r = rect + 4 * i;
            if (tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]) {
                cand[nc].depth = f2u(rec[REC * i + 3]);
                cand[nc].id = (uint32_t)i;
                ++nc;
            }
        }
        qsort(cand, (size_t)nc, sizeof(cand_t), cand_cmp);
        for (int py = ty * TILE; py < ty * TILE + TILE && py < H; ++py)
            for (int px = tx * TILE; px < tx * TILE + TILE && px < W; ++px) {
                const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
                const double dpx = px + 0.5, dpy = py + 0.5;
                float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
                double Td = 1.0, D0 = 0.0, D1 = 0.0, D2 = 0.0;
                uint32_t last = 0;
                for (int64_t j = 0; j < nc; ++j) {
                    const uint32_t g = cand[j].id;
                    const float* R = rec + REC * g;
                    ++evals;
                    float dx = R[0] - fpx, dy = R[1] - fpy;
                    float power = fmaf(dx, fmaf(R[4], dx, R[5] * dy), (R[6] * dy) * dy);
                    if (power > 0.0f) continue;
                    float a = fminf(0.99f, R[2] * oracle_exp_spec(power));
                    if (a < one255) continue;
                    float tt = T * (1.0f - a);
                    if (tt < 1e-4f) break;
                    float wgt = a * T;
                    C0 = fmaf(R[8], wgt, C0);
                    C1 = fmaf(R[9], wgt, C1);
                    C2 = fmaf(R[10], wgt, C2);
                    T = tt;
                    last = (uint32_t)(j + 1);
                    if (rec64) {
                        const double* Q = rec64 + REC64 * g;
                        double ex = Q[0] - dpx, ey = Q[1] - dpy;
                        double pw = -0.5 * (Q[3] * ex * ex + Q[5] * ey * ey) - Q[4] * ex * ey;
                        double ad = Q[2] * exp(pw);
                        if (ad > 0.99) ad = 0.99;
                        double wd = ad * Td;
                        D0 += Q[6] * wd; D1 += Q[7] * wd; D2 += Q[8] * wd;
                        Td *= (1.0 - ad);
                    }
                    if (contrib_pix) {
                        if (total < contrib_cap) {
                            contrib_pix[total] = (int64_t)py * W + px;
                            contrib_gid[total] = (int32_t)g;
                        }
                    }
                    ++total;
                }
                const size_t p = (size_t)py * W + px, plane = (size_t)W * H;
                img32[p] = fmaf(T, V[OV_BG], C0);
                img32[plane + p] = fmaf(T, V[OV_BG + 1], C1);
                img32[2 * plane + p] = fmaf(T, V[OV_BG + 2], C2);
                T32[p] = T;
                ncontrib[p] = last;
                if (img64) {
                    img64[p] = D0 + Td * V[OV_BG];
                    img64[plane + p] = D1 + Td * V[OV_BG + 1];
                    img64[2 * plane + p] = D2 + Td * V[OV_BG + 2];
                }
                if (T64) T64[p] = Td;
            }
    }
    free(cand);
    if (evaluated) *evaluated = evals;
    return total;
}

/* ======================================================================= */
/* Stage II with FP64 decisions (Eq. 1 in real arithmetic)                 */
/* ======================================================================= */
/* Eq. 1 is stated on real numbers, so its three per-pixel decisions -- skip a
 * Gaussian whose power is positive, skip an opacity below 1/255, stop before
 * the transmittance falls below 1e-4 -- are decisions on real values.  This
 * pass takes all three in FP64, on the FP64 records of oracle_stage1_f64,
 * over the same candidates in the same order as oracle_render (Stage I's
 * mask, tile rectangles and depth order: integer outcomes of Stage I).
 *
 * Near a threshold a rasterizer working in finite precision may take either
 * outcome, so a decision whose FP64 quantity lies within a band of its
 * threshold is flagged and both outcomes are followed to the end of the
 * pixel.  The band is the relative tolerance `rel` plus a first-order bound
 * on how far an FP32 evaluation of the same quantity can lie from its FP64
 * value.  With dx = u - x, dy = v - y (pixel centre x, y), the differences
 * du, dv, dA, dB, dC, da2 between the FP32 records (oracle_stage1) and the
 * FP64 records, and U = 2^-24 (FP32 unit roundoff):
 *   power p = -(A dx^2 + C dy^2)/2 - B dx dy
 *     dp = |A dx + B dy| (du + U|dx|) + |C dy + B dx| (dv + U|dy|)
 *        + (dA dx^2 + dC dy^2)/2 + dB |dx dy| + 8 U S,
 *     S = (|A| dx^2 + |C| dy^2)/2 + |B dx dy|
 *   opacity a = min(0.99, alpha'' e^p):  ra = dp + da2/alpha'' + 16 U, the
 *     16 U for the FP32 exponential (a few ulp: a software polynomial or a
 *     hardware base-2 unit after the rounding of p log2 e) and the product
 *   transmittance T' = T (1 - a):  rT' = rT + ra a/(1 - a) + 4 U, with rT = 0
 *     before the first contributor (relative deviations)
 * Flagged when |p| < dp, |a - 1/255| <= (rel + ra)/255 or
 * |T' - 1e-4| <= (rel + rT') 1e-4.  dev scales dp, ra and the 4 U of rT'
 * (1: the bound above; 0: the relative band rel alone).
 *
 * Every pixel yields the outcome of the FP64 decisions (the main path) and
 * one outcome per followed flag, at most max_paths in all (<= 64); flags met
 * once that many paths exist are counted, not followed.
 *
 * Outputs for the listed tiles (3 x H x W / H x W arrays, other pixels
 * untouched): img64, T64, nc64 (main path), n_paths (outcomes followed),
 * n_capped (flags not followed, saturating at 255).  The outcomes beyond the
 * main path are appended to alt_pix (pixel y W + x), alt_val (r, g, b, T) and
 * alt_nc up to alt_cap entries.  Returns the number of such outcomes, or -1
 * on allocation failure. */
typedef struct {
    int64_t j;          /* candidate at which the path resumes */
    int flip;           /* decision inverted at candidate j: 0 none, 1 power, 2 opacity, 3 stop */
    double T, D0, D1, D2, rT;
    uint32_t last;
} path64_t;

#define MAX_PATHS64 64

int64_t oracle_render_f64dec(int64_t n, const float* V, const uint8_t* survive, const float* rec,
                             const int32_t* rect, const double* rec64, const int32_t* tile_list, int64_t n_list,
                             double rel, double dev, int max_paths, double* img64, double* T64, uint32_t* nc64,
                             uint8_t* n_paths, uint8_t* n_capped, int64_t* alt_pix, double* alt_val,
                             uint32_t* alt_nc, int64_t alt_cap)
{
    const int W = (int)V[OV_W], H = (int)V[OV_H];
    const int TX = (W + TILE - 1) / TILE;
    const double U = 5.9604644775390625e-08;    /* 2^-24 */
    const double bg[3] = { V[OV_BG], V[OV_BG + 1], V[OV_BG + 2] };
    if (max_paths < 1) max_paths = 1;
    if (max_paths > MAX_PATHS64) max_paths = MAX_PATHS64;
    cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (n > 0 ? n : 1));
    if (!cand) return -1;
    int64_t n_alt = 0;
    path64_t stack[MAX_PATHS64];
    for (int64_t li = 0; li < n_list; ++li) {
        const int tile = tile_list[li];
        const int tx = tile % TX, ty = tile / TX;
        int64_t nc = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (!survive[i]) continue;
            const int32_t* r = rect + 4 * i;
            if (tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]) {
                cand[nc].depth = f2u(rec[REC * i + 3]);
                cand[nc].id = (uint32_t)i;
                ++nc;
            }
        }
        qsort(cand, (size_t)nc, sizeof(cand_t), cand_cmp);
        for (int py = ty * TILE; py < ty * TILE + TILE && py < H; ++py)
            for (int px = tx * TILE; px < tx * TILE + TILE && px < W; ++px) {
                const double x = px + 0.5, y = py + 0.5;
                const size_t pix = (size_t)py * W + px, plane = (size_t)W * H;
                int created = 1, top = 0, capped = 0, first = 1;
                stack[top++] = (path64_t){ 0, 0, 1.0, 0.0, 0.0, 0.0, 0.0, 0u };
                while (top > 0) {
                    path64_t P = stack[--top];
                    const int64_t j0 = P.j;
                    for (int64_t j = j0; j < nc; ++j) {
                        /* decisions at or before P.flip at the resume point were
                         * branched by the parent path: not flagged again */
                        const int lock = (j == j0) ? P.flip : 0;
                        const uint32_t g = cand[j].id;
                        const double* Q = rec64 + REC64 * g;
                        const float* R = rec + REC * g;
                        const double dx = Q[0] - x, dy = Q[1] - y;
                        const double A = Q[3], B = Q[4], C = Q[5];
                        const double p = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy;
                        const double du = fabs((double)R[0] - Q[0]), dv = fabs((double)R[1] - Q[1]);
                        const double dA = fabs(-2.0 * (double)R[4] - A), dB = fabs(-(double)R[5] - B);
                        const double dC = fabs(-2.0 * (double)R[6] - C);
                        const double S = 0.5 * (fabs(A) * dx * dx + fabs(C) * dy * dy) + fabs(B * dx * dy);
                        const double dp = dev * (fabs(A * dx + B * dy) * (du + U * fabs(dx)) +
                                                 fabs(C * dy + B * dx) * (dv + U * fabs(dy)) +
                                                 0.5 * (dA * dx * dx + dC * dy * dy) + dB * fabs(dx * dy) + 8.0 * U * S);
                        /* decision 1: a positive power is skipped */
                        int skip = p > 0.0;
                        if (lock == 1) skip = !skip;
                        if (fabs(p) < dp && lock < 1) {
                            if (created < max_paths) {
                                stack[top++] = (path64_t){ j, 1, P.T, P.D0, P.D1, P.D2, P.rT, P.last };
                                ++created;
                            } else ++capped;
                        }
                        if (skip) continue;
                        /* decision 2: an opacity below 1/255 is skipped */
                        double a = Q[2] * exp(p);
                        if (a > 0.99) a = 0.99;
                        const double ra = dp + dev * (fabs((double)R[2] - Q[2]) / Q[2] + 16.0 * U);
                        skip = a < 1.0 / 255.0;
                        if (lock == 2) skip = !skip;
                        if (fabs(a - 1.0 / 255.0) <= (rel + ra) / 255.0 && lock < 2) {
                            if (created < max_paths) {
                                stack[top++] = (path64_t){ j, 2, P.T, P.D0, P.D1, P.D2, P.rT, P.last };
                                ++created;
                            } else ++capped;
                        }
                        if (skip) continue;
                        /* decision 3: stop before T' = T (1 - a) falls below 1e-4 */
                        const double tt = P.T * (1.0 - a);
                        const double rT = P.rT + ra * a / (1.0 - a) + dev * 4.0 * U;
                        int stop = tt < 1e-4;
                        if (lock == 3) stop = !stop;
                        if (fabs(tt - 1e-4) <= (rel + rT) * 1e-4 && lock < 3) {
                            if (created < max_paths) {
                                stack[top++] = (path64_t){ j, 3, P.T, P.D0, P.D1, P.D2, P.rT, P.last };
                                ++created;
                            } else ++capped;
                        }
                        if (stop) break;
                        const double wgt = a * P.T;
                        P.D0 += Q[6] * wgt;
                        P.D1 += Q[7] * wgt;
                        P.D2 += Q[8] * wgt;
                        P.T = tt;
                        P.rT = rT;
                        P.last = (uint32_t)(j + 1);
                    }
                    const double o0 = P.D0 + P.T * bg[0], o1 = P.D1 + P.T * bg[1], o2 = P.D2 + P.T * bg[2];
                    if (first) {
                        img64[pix] = o0;
                        img64[plane + pix] = o1;
                        img64[2 * plane + pix] = o2;
                        T64[pix] = P.T;
                        nc64[pix] = P.last;
                        first = 0;
                    } else {
                        if (n_alt < alt_cap) {
                            alt_pix[n_alt] = (int64_t)pix;
                            alt_val[4 * n_alt] = o0;
                            alt_val[4 * n_alt + 1] = o1;
                            alt_val[4 * n_alt + 2] = o2;
                            alt_val[4 * n_alt + 3] = P.T;
                            alt_nc[n_alt] = P.last;
                        }
                        ++n_alt;
                    }
                }
                n_paths[pix] = (uint8_t)created;
                n_capped[pix] = (uint8_t)(capped > 255 ? 255 : capped);
            }
    }
    free(cand);
    return n_alt;
}
