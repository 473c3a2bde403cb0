/*
 * LODGE per-frame render path: plain, slow CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path: it is written from
 * the paper (arXiv 2505.23158) and from the textbook definitions the paper
 * builds on, in the paper's order and notation.
 *
 * Precision: floating point is FP64 (double) everywhere except the
 * "key spec" below, which is evaluated in FP32 with every operation rounded
 * (this file must be compiled with -ffp-contract=off and without
 * -ffast-math).  The key spec decides only integer outcomes - which
 * Gaussians are culled, which tiles a Gaussian is binned to, and the depth
 * bits used as the sort key - so that both implementations can be compared
 * exactly on them.  Every value that reaches a pixel is FP64.
 *
 * Passages followed:
 *   Sec. 3 "Preliminaries: 3DGS"      Eq. 1 alpha, 16x16 tiles, sort by depth,
 *                                     alpha blending (EWA splatting of the
 *                                     3DGS renderer the paper builds on).
 *   Sec. 3 "LOD representation"       Eq. 2 active set at a centre c with
 *                                     d_0 = 0, d_L = inf.
 *   Sec. 3 "Building LOD"             Eq. 3 3D smoothing filter (applied at
 *                                     render time as a per-level variance).
 *   Sec. 3 "Chunk-based rendering"    per-chunk active set at the chunk centre,
 *                                     thresholds offset by the chunk radius
 *                                     (distance to the nearest other centre).
 *   Sec. 3 "Opacity blending"         Eq. 4 two nearest chunks, union of their
 *                                     active sets, opacity of the symmetric
 *                                     difference scaled by t.
 * Readings where the paper is silent are listed in the design notes and at
 * each function below.
 *
 * Parity status: every function here is pinned by the CPU test suite
 * (closed forms, brute force, invariants, textbook reductions).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TILE 16
#define ORC_ALPHA_MAX 0.99
#define ORC_ALPHA_MIN (1.0 / 255.0)
#define ORC_T_MIN 1e-4
#define ORC_DILATION 0.3

/* ---------------------------------------------------------------------- */
/* data structures (oracle-private; the Python wrapper marshals into them) */
/* ---------------------------------------------------------------------- */
typedef struct {
    float R[9];          /* world -> camera rotation, row-major */
    float t[3];          /* world -> camera translation */
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear;
    float pad_;
    double center[3];    /* camera position in world coordinates */
} orc_camera;

typedef struct {
    int64_t n_total;
    int32_t num_levels;
    int32_t sh_degree;
    const int64_t* level_off;   /* num_levels + 1 offsets into the arrays */
    const float* filter_var;    /* per level: variance of the 3D filter */
    const float* means;         /* n_total x 3 */
    const float* scales;        /* n_total x 3, activated (std dev) */
    const float* quats;         /* n_total x 4, unit (w, x, y, z) */
    const float* opac;          /* n_total, activated opacity */
    const float* sh;            /* n_total x 16 x 3 */
    int32_t filter2d;           /* 1: opacity-compensated 2D filter (Mip-Splatting) */
} orc_scene;

int orc_version(void) { return 1; }

/* ---------------------------------------------------------------------- */
/* activation (3DGS convention; the paper leaves it implicit in Sec. 3)     */
/* scale = exp(log_scale), opacity = sigmoid(logit), unit quaternion.      */
/* Evaluated in FP64 and rounded once to FP32.                             */
/* ---------------------------------------------------------------------- */
void orc_activate(int64_t n, const float* log_scales, const float* quats,
                  const float* logits, float* scales_out, float* quats_out,
                  float* opac_out)
{
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 3; ++k)
            scales_out[3 * i + k] = (float)exp((double)log_scales[3 * i + k]);
        double w = quats[4 * i + 0], x = quats[4 * i + 1];
        double y = quats[4 * i + 2], z = quats[4 * i + 3];
        double nrm = sqrt(((w * w + x * x) + y * y) + z * z);
        quats_out[4 * i + 0] = (float)(w / nrm);
        quats_out[4 * i + 1] = (float)(x / nrm);
        quats_out[4 * i + 2] = (float)(y / nrm);
        quats_out[4 * i + 3] = (float)(z / nrm);
        opac_out[i] = (float)(1.0 / (1.0 + exp(-(double)logits[i])));
    }
}

/* ---------------------------------------------------------------------- */
/* Eq. 4 support: chunk radius and the two nearest chunk centres           */
/* ---------------------------------------------------------------------- */
static double dist2_3(const double* a, const double* b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return (dx * dx + dy * dy) + dz * dz;
}

/* Chunk radius r_k = distance to the nearest other chunk centre (the
 * full distance, not half: Sec. 3 "Chunk-based rendering").  K = 1 gives 0. */
void orc_chunk_radius(int32_t K, const double* centers, double* r)
{
    for (int32_t k = 0; k < K; ++k) {
        double best = INFINITY;
        for (int32_t j = 0; j < K; ++j) {
            if (j == k) continue;
            double d = sqrt(dist2_3(centers + 3 * k, centers + 3 * j));
            if (d < best) best = d;
        }
        r[k] = (K > 1) ? best : 0.0;
    }
}

/* Two nearest centres to c (ties to the lower index) and the Eq. 4 weights:
 *   t_A = clamp((c - m_B).(m_A - m_B) / |m_A - m_B|^2, 0, 1)  (Gaussians of A only)
 *   t_B = clamp((c - m_A).(m_B - m_A) / |m_A - m_B|^2, 0, 1)  (Gaussians of B only)
 * K = 1: B = -1 and both weights 1. */
void orc_chunk_pick(int32_t K, const double* centers, const double* c,
                    int32_t* A, int32_t* B, double* tA, double* tB)
{
    int32_t a = -1, b = -1;
    double da = INFINITY, db = INFINITY;
    for (int32_t k = 0; k < K; ++k) {
        double d = dist2_3(c, centers + 3 * k);
        if (d < da) { b = a; db = da; a = k; da = d; }
        else if (d < db) { b = k; db = d; }
    }
    *A = a; *B = b;
    if (b < 0) { *tA = 1.0; *tB = 1.0; return; }
    const double* mA = centers + 3 * a;
    const double* mB = centers + 3 * b;
    double ab[3] = { mA[0] - mB[0], mA[1] - mB[1], mA[2] - mB[2] };
    double n2 = (ab[0] * ab[0] + ab[1] * ab[1]) + ab[2] * ab[2];
    double cB[3] = { c[0] - mB[0], c[1] - mB[1], c[2] - mB[2] };
    double cA[3] = { c[0] - mA[0], c[1] - mA[1], c[2] - mA[2] };
    double ta = ((cB[0] * ab[0] + cB[1] * ab[1]) + cB[2] * ab[2]) / n2;
    double tb = ((cA[0] * -ab[0] + cA[1] * -ab[1]) + cA[2] * -ab[2]) / n2;
    *tA = fmin(1.0, fmax(0.0, ta));
    *tB = fmin(1.0, fmax(0.0, tb));
}

/* Unclamped t_A + t_B, exposed so that the identity t_A + t_B = 1 can be
 * tested independently of clamping. */
double orc_chunk_tsum_unclamped(const double* mA, const double* mB, const double* c)
{
    double ab[3] = { mA[0] - mB[0], mA[1] - mB[1], mA[2] - mB[2] };
    double n2 = (ab[0] * ab[0] + ab[1] * ab[1]) + ab[2] * ab[2];
    double ta = ((c[0] - mB[0]) * ab[0] + (c[1] - mB[1]) * ab[1] + (c[2] - mB[2]) * ab[2]) / n2;
    double tb = ((c[0] - mA[0]) * -ab[0] + (c[1] - mA[1]) * -ab[1] + (c[2] - mA[2]) * -ab[2]) / n2;
    return ta + tb;
}

/* ---------------------------------------------------------------------- */
/* Eq. 2: active Gaussians at centre c                                       */
/*   union over l of { g in G(l) : d_l <= |mu - c| < d_{l+1} },             */
/*   d_0 = 0, d_L = inf.  (Sec. 3 prints "L > l > 0" for the level range;  */
/*   read as 0 <= l < L, consistent with the union bounds in Eq. 2.)        */
/* The comparison that decides membership is the pinned FP32 test:         */
/*   c rounded once to FP32; D = (dx*dx + dy*dy) + dz*dz in FP32;           */
/*   thr_l = (float)(d_l * d_l) with d_l in FP64; member iff                 */
/*   thr_l <= D && D < thr_{l+1}.  The FP64 test is also evaluated and the  */
/*   number of Gaussians on which the two disagree is reported.            */
/* d_inner holds d_1 .. d_{L-1}.                                            */
/* ---------------------------------------------------------------------- */
int64_t orc_lod_select(const orc_scene* sc, const double* c, const double* d_inner,
                       uint8_t* mask, int64_t* n_disagree)
{
    int L = sc->num_levels;
    float c32[3] = { (float)c[0], (float)c[1], (float)c[2] };
    int64_t count = 0, dis = 0;
    for (int l = 0; l < L; ++l) {
        double lo = (l == 0) ? 0.0 : d_inner[l - 1];
        double hi = (l == L - 1) ? INFINITY : d_inner[l];
        float thr_lo = (float)(lo * lo);
        float thr_hi = (l == L - 1) ? INFINITY : (float)(hi * hi);
        for (int64_t g = sc->level_off[l]; g < sc->level_off[l + 1]; ++g) {
            const float* m = sc->means + 3 * g;
            float dx = m[0] - c32[0], dy = m[1] - c32[1], dz = m[2] - c32[2];
            float D = (dx * dx + dy * dy) + dz * dz;
            int in32 = (thr_lo <= D) && (D < thr_hi);
            double ex = (double)m[0] - c[0], ey = (double)m[1] - c[1], ez = (double)m[2] - c[2];
            double d64 = sqrt(ex * ex + ey * ey + ez * ez);
            int in64 = (lo <= d64) && (d64 < hi);
            mask[g] = (uint8_t)in32;
            count += in32;
            dis += (in32 != in64);
        }
    }
    if (n_disagree) *n_disagree = dis;
    return count;
}

/* Per-chunk active set: Eq. 2 at the chunk centre m_k with every inner
 * threshold offset by the chunk radius, d'_l = d_l + r_k (Sec. 3 "Chunk-based
 * rendering"; the sign of the offset is not printed - read as "+" so that a
 * camera within r_k of the centre sees level l no closer than d_l). */
int64_t orc_chunk_select(const orc_scene* sc, int32_t K, const double* centers,
                         const double* d_inner, int32_t k, uint8_t* mask,
                         int64_t* n_disagree)
{
    double* r = (double*)malloc(sizeof(double) * (size_t)K);
    orc_chunk_radius(K, centers, r);
    int L = sc->num_levels;
    double dd[64];
    for (int l = 0; l + 1 < L && l < 64; ++l) dd[l] = d_inner[l] + r[k];
    int64_t n = orc_lod_select(sc, centers + 3 * k, dd, mask, n_disagree);
    free(r);
    return n;
}

/* Union of two gid-ascending active sets with the Eq. 4 multipliers:
 * in both -> 1, A only -> t_A, B only -> t_B.  Output in gid order.
 * Returns the union size. */
int64_t orc_chunk_union(int64_t na, const int64_t* a, int64_t nb, const int64_t* b,
                        double tA, double tB, int64_t* out, float* mult)
{
    int64_t i = 0, j = 0, n = 0;
    while (i < na || j < nb) {
        if (j >= nb || (i < na && a[i] < b[j])) { out[n] = a[i++]; mult[n++] = (float)tA; }
        else if (i >= na || b[j] < a[i]) { out[n] = b[j++]; mult[n++] = (float)tB; }
        else { out[n] = a[i]; mult[n++] = 1.0f; ++i; ++j; }
    }
    return n;
}

/* ---------------------------------------------------------------------- */
/* key spec (FP32, every operation rounded, no fused multiply-add)          */
/* ---------------------------------------------------------------------- */
static int level_of(const orc_scene* sc, int64_t g)
{
    int l = 0;
    while (l + 1 < sc->num_levels && g >= sc->level_off[l + 1]) ++l;
    return l;
}

static float u32_as_f32(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t f32_as_u32(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* Extent threshold for a final opacity o (FP32): Q = 2 ln(255 o_hi) * 1.001
 * where o_hi is the upper end of o's bucket (its FP32 exponent and three
 * leading mantissa bits).  A pixel with alpha = o G >= 1/255 satisfies
 * d^T Sigma'^-1 d <= 2 ln(255 o) <= Q, so the bounding box of that ellipse
 * is conservative for Eq. 1 with the 1/255 skip. */
static float extent_q(float o)
{
    uint32_t top = f32_as_u32(o) >> 20;
    uint32_t b = top - (119u << 3);
    if (top > (127u << 3)) b = 64u;
    double hi = (double)u32_as_f32((b + (119u << 3) + 1u) << 20);
    return (float)(2.0 * log(255.0 * hi) * 1.001);
}

typedef struct {
    float z;          /* camera-space depth (key bits) */
    int32_t rect[4];  /* tile rect tx0, ty0, tx1, ty1 (inclusive) */
    float o32;        /* final opacity in FP32 (decides the extent) */
} orc_key_rec;

/* Camera-relative evaluation point of the key spec.  p = R mu + t equals
 * R (mu - c_hat) + t' for any c_hat, with t' = t + R c_hat.  Taking c_hat =
 * (float)center and forming t' in FP64 keeps mu - c_hat exact (Sterbenz) for
 * Gaussians near the camera, where an FP32 R mu + t would cancel
 * catastrophically in a world hundreds of metres across. */
static void cam_rel(const orc_camera* cam, float chat[3], float tp[3])
{
    for (int i = 0; i < 3; ++i) chat[i] = (float)cam->center[i];
    for (int i = 0; i < 3; ++i)
        tp[i] = (float)((double)cam->t[i] + (((double)cam->R[3 * i] * (double)chat[0]
                        + (double)cam->R[3 * i + 1] * (double)chat[1]) + (double)cam->R[3 * i + 2] * (double)chat[2]));
}

/* Lateral limits of the EWA Jacobian's evaluation point (the 3DGS
 * rasteriser's clamp, kept by the paper's renderer): x/z and y/z are held
 * within 1.3 tan(fov/2) of the axis, tan(fovx/2) = W / (2 fx),
 * tan(fovy/2) = H / (2 fy), formed in FP64 and rounded to FP32.  Without it a
 * Gaussian just past the near plane far off the axis gets a Jacobian that
 * stretches its footprint over the whole image. */
static void lateral_limits(const orc_camera* cam, float* limx, float* limy)
{
    *limx = (float)(1.3 * ((double)cam->width / (2.0 * (double)cam->fx)));
    *limy = (float)(1.3 * ((double)cam->height / (2.0 * (double)cam->fy)));
}

static float cam_depth32(const orc_camera* cam, const float* mu)
{
    float chat[3], tp[3];
    cam_rel(cam, chat, tp);
    const float* R = cam->R;
    float dx = mu[0] - chat[0], dy = mu[1] - chat[1], dz = mu[2] - chat[2];
    return ((R[6] * dx + R[7] * dy) + R[8] * dz) + tp[2];
}

/* Returns 1 if the Gaussian is binned to at least one tile.  Steps:
 *  camera point p = ((R0 d0 + R1 d1) + R2 d2) + t' per row with
 *    d = mu - c_hat (FP32) and c_hat, t' from cam_rel; cull unless z > znear;
 *  per-level 3D filter (Eq. 3, variance v): sigma_k = sqrt(s_k^2 + v) and
 *    opacity compensation ((s0/sigma0)(s1/sigma1))(s2/sigma2), only if v > 0;
 *  final opacity o' = (o * mult) [* comp]; cull if o' < 1/255 (no pixel can
 *    pass the 1/255 skip);
 *  u = x/z, w = y/z; mean' = (fx u + cx, fy w + cy);
 *  EWA Jacobian rows j00 = fx/z, j02 = -(j00 uc), j11 = fy/z, j12 = -(j11 wc),
 *    its evaluation point clamped laterally: uc = min(max(u, -limx), limx),
 *    wc likewise with limy (lateral_limits; the mean keeps u, w);
 *  T = J R; M = rotation of the unit quaternion; A = T M; B = A diag(sigma);
 *  Sigma'_xx = ((B00^2 + B01^2) + B02^2) + 0.3, Sigma'_yy likewise;
 *  r = sqrt(Q Sigma'); pixel range [ceil(m - r - 0.5), floor(m + r - 0.5)]
 *  clipped to the image; cull if empty; tiles = pixel range / 16. */
static int key_spec(const orc_scene* sc, const orc_camera* cam, int64_t g,
                    float mult, orc_key_rec* out)
{
    const float* mu = sc->means + 3 * g;
    const float* R = cam->R;
    float chat[3], tp[3];
    cam_rel(cam, chat, tp);
    float d0 = mu[0] - chat[0], d1 = mu[1] - chat[1], d2 = mu[2] - chat[2];
    float px = ((R[0] * d0 + R[1] * d1) + R[2] * d2) + tp[0];
    float py = ((R[3] * d0 + R[4] * d1) + R[5] * d2) + tp[1];
    float pz = ((R[6] * d0 + R[7] * d1) + R[8] * d2) + tp[2];
    if (!(pz > cam->znear)) return 0;

    const float* s = sc->scales + 3 * g;
    float v = sc->filter_var[level_of(sc, g)];
    float sig[3] = { s[0], s[1], s[2] };
    float o = sc->opac[g] * mult;
    if (v > 0.0f) {
        for (int k = 0; k < 3; ++k) sig[k] = sqrtf(s[k] * s[k] + v);
        float comp = ((s[0] / sig[0]) * (s[1] / sig[1])) * (s[2] / sig[2]);
        o = o * comp;
    }
    /* without the compensated 2D filter the opacity is final here; with it,
     * the opacity cull waits for the compensation below */
    if (!sc->filter2d && !(o >= (float)ORC_ALPHA_MIN)) return 0;

    float u = px / pz, w = py / pz;
    float mx = cam->fx * u + cam->cx;
    float my = cam->fy * w + cam->cy;
    float limx, limy;
    lateral_limits(cam, &limx, &limy);
    float uc = fminf(fmaxf(u, -limx), limx), wc = fminf(fmaxf(w, -limy), limy);
    float j00 = cam->fx / pz, j02 = -(j00 * uc);
    float j11 = cam->fy / pz, j12 = -(j11 * wc);
    float T0[3], T1[3];
    for (int k = 0; k < 3; ++k) {
        T0[k] = j00 * R[k] + j02 * R[6 + k];
        T1[k] = j11 * R[3 + k] + j12 * R[6 + k];
    }
    const float* q = sc->quats + 4 * g;
    float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    float xx = qx * qx, yy = qy * qy, zz = qz * qz;
    float xy = qx * qy, xz = qx * qz, yz = qy * qz;
    float wx = qw * qx, wy = qw * qy, wz = qw * qz;
    float M[3][3];
    M[0][0] = 1.0f - 2.0f * (yy + zz); M[0][1] = 2.0f * (xy - wz); M[0][2] = 2.0f * (xz + wy);
    M[1][0] = 2.0f * (xy + wz); M[1][1] = 1.0f - 2.0f * (xx + zz); M[1][2] = 2.0f * (yz - wx);
    M[2][0] = 2.0f * (xz - wy); M[2][1] = 2.0f * (yz + wx); M[2][2] = 1.0f - 2.0f * (xx + yy);
    float B0[3], B1[3];
    for (int k = 0; k < 3; ++k) {
        float a0 = (T0[0] * M[0][k] + T0[1] * M[1][k]) + T0[2] * M[2][k];
        float a1 = (T1[0] * M[0][k] + T1[1] * M[1][k]) + T1[2] * M[2][k];
        B0[k] = a0 * sig[k];
        B1[k] = a1 * sig[k];
    }
    float aB = (B0[0] * B0[0] + B0[1] * B0[1]) + B0[2] * B0[2];
    float cB = (B1[0] * B1[0] + B1[1] * B1[1]) + B1[2] * B1[2];
    if (sc->filter2d) {
        /* Mip-Splatting's 2D filter: o *= sqrt(det(Sigma2D) / det(Sigma2D + 0.3 I)),
         * det(Sigma2D) = det(B B^T) as the sum of squared 2x2 minors of B
         * (Cauchy-Binet), det(Sigma2D + 0.3 I) = det + 0.3 (aB + cB) + 0.09 */
        float m01 = B0[0] * B1[1] - B0[1] * B1[0];
        float m02 = B0[0] * B1[2] - B0[2] * B1[0];
        float m12 = B0[1] * B1[2] - B0[2] * B1[1];
        float D0 = (m01 * m01 + m02 * m02) + m12 * m12;
        float D1 = (D0 + 0.3f * (aB + cB)) + 0.09f;
        o = o * sqrtf(D0 / D1);
        if (!(o >= (float)ORC_ALPHA_MIN)) return 0;
    }
    float Q = extent_q(o);
    float sxx = aB + 0.3f;
    float syy = cB + 0.3f;
    float rx = sqrtf(Q * sxx), ry = sqrtf(Q * syy);
    float x0 = ceilf((mx - rx) - 0.5f), x1 = floorf((mx + rx) - 0.5f);
    float y0 = ceilf((my - ry) - 0.5f), y1 = floorf((my + ry) - 0.5f);
    float xmax = (float)(cam->width - 1), ymax = (float)(cam->height - 1);
    if (x0 < 0.0f) x0 = 0.0f;
    if (y0 < 0.0f) y0 = 0.0f;
    if (x1 > xmax) x1 = xmax;
    if (y1 > ymax) y1 = ymax;
    if (!(x0 <= x1) || !(y0 <= y1)) return 0;
    out->z = pz;
    out->o32 = o;
    out->rect[0] = (int32_t)x0 / ORC_TILE;
    out->rect[1] = (int32_t)y0 / ORC_TILE;
    out->rect[2] = (int32_t)x1 / ORC_TILE;
    out->rect[3] = (int32_t)y1 / ORC_TILE;
    return 1;
}

/* FP32 key depth of each listed Gaussian (the sort key and near-cull input). */
void orc_depth32(const float* means, const orc_camera* cam, int64_t n, float* z)
{
    for (int64_t i = 0; i < n; ++i) z[i] = cam_depth32(cam, means + 3 * i);
}

/* ---------------------------------------------------------------------- */
/* FP64 projection (EWA splatting, Zwicker et al. as used by 3DGS) and     */
/* view-dependent colour (real spherical harmonics up to degree 3)         */
/* ---------------------------------------------------------------------- */
typedef struct {
    double mx, my;      /* 2D mean mu' (pixel units, pixel i has centre i+0.5) */
    double conic[3];    /* inverse of Sigma': (xx, xy, yy) */
    double cov[3];      /* Sigma' itself (xx, xy, yy) */
    double opacity;     /* o * mult * filter compensation */
    double rgb[3];
} orc_splat;

/* Real orthonormal SH basis up to l = 3, order (l, m = -l..l), for a unit
 * direction (x, y, z).  Constants are the closed-form normalisation of each
 * polynomial (Cartesian form of the real spherical harmonics). */
static void sh_basis(double x, double y, double z, double* Y)
{
    const double PI = 3.14159265358979323846;
    Y[0] = 0.5 * sqrt(1.0 / PI);
    double c1 = sqrt(3.0 / (4.0 * PI));
    Y[1] = c1 * y; Y[2] = c1 * z; Y[3] = c1 * x;
    Y[4] = 0.5 * sqrt(15.0 / PI) * x * y;
    Y[5] = 0.5 * sqrt(15.0 / PI) * y * z;
    Y[6] = 0.25 * sqrt(5.0 / PI) * (3.0 * z * z - 1.0);
    Y[7] = 0.5 * sqrt(15.0 / PI) * x * z;
    Y[8] = 0.25 * sqrt(15.0 / PI) * (x * x - y * y);
    Y[9] = 0.25 * sqrt(35.0 / (2.0 * PI)) * y * (3.0 * x * x - y * y);
    Y[10] = 0.5 * sqrt(105.0 / PI) * x * y * z;
    Y[11] = 0.25 * sqrt(21.0 / (2.0 * PI)) * y * (5.0 * z * z - 1.0);
    Y[12] = 0.25 * sqrt(7.0 / PI) * z * (5.0 * z * z - 3.0);
    Y[13] = 0.25 * sqrt(21.0 / (2.0 * PI)) * x * (5.0 * z * z - 1.0);
    Y[14] = 0.25 * sqrt(105.0 / PI) * z * (x * x - y * y);
    Y[15] = 0.25 * sqrt(35.0 / (2.0 * PI)) * x * (x * x - 3.0 * y * y);
}

void orc_sh_basis(double x, double y, double z, double* Y) { sh_basis(x, y, z, Y); }

static void splat64(const orc_scene* sc, const orc_camera* cam, int64_t g, double mult,
                    orc_splat* o)
{
    double mu[3] = { sc->means[3 * g], sc->means[3 * g + 1], sc->means[3 * g + 2] };
    double R[9], p[3];
    for (int i = 0; i < 9; ++i) R[i] = cam->R[i];
    for (int i = 0; i < 3; ++i)
        p[i] = R[3 * i] * mu[0] + R[3 * i + 1] * mu[1] + R[3 * i + 2] * mu[2] + (double)cam->t[i];
    double fx = cam->fx, fy = cam->fy;
    o->mx = fx * p[0] / p[2] + cam->cx;
    o->my = fy * p[1] / p[2] + cam->cy;
    /* the Jacobian at the laterally clamped point (lateral_limits) */
    float limx32, limy32;
    lateral_limits(cam, &limx32, &limy32);
    double limx = limx32, limy = limy32;
    double uc = fmin(fmax(p[0] / p[2], -limx), limx);
    double wc = fmin(fmax(p[1] / p[2], -limy), limy);
    double J[2][3] = { { fx / p[2], 0.0, -fx * uc / p[2] },
                       { 0.0, fy / p[2], -fy * wc / p[2] } };
    /* world covariance Sigma = Rq diag(s^2 + v) Rq^T (Eq. 3 filter added to
     * the covariance; v = 0 leaves 3DGS's Sigma) */
    double w = sc->quats[4 * g], x = sc->quats[4 * g + 1], y = sc->quats[4 * g + 2], z = sc->quats[4 * g + 3];
    double Rq[3][3] = {
        { 1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y) },
        { 2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x) },
        { 2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y) } };
    double v = sc->filter_var[level_of(sc, g)];
    double s2[3], comp = 1.0;
    for (int k = 0; k < 3; ++k) {
        double s = sc->scales[3 * g + k];
        s2[k] = s * s + v;
        if (v > 0.0) comp *= s / sqrt(s * s + v);
    }
    double S[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += Rq[i][k] * s2[k] * Rq[j][k];
            S[i][j] = acc;
        }
    /* T = J W with W the camera rotation; Sigma' = T Sigma T^T + 0.3 I */
    double T[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            T[i][j] = J[i][0] * R[j] + J[i][1] * R[3 + j] + J[i][2] * R[6 + j];
    double C[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += T[i][a] * S[a][b] * T[j][b];
            C[i][j] = acc;
        }
    double det0 = C[0][0] * C[1][1] - C[0][1] * C[1][0];
    C[0][0] += ORC_DILATION;
    C[1][1] += ORC_DILATION;
    double det = C[0][0] * C[1][1] - C[0][1] * C[1][0];
    /* Mip-Splatting's 2D filter keeps the splat's integral: opacity times
     * sqrt(det(Sigma2D) / det(Sigma2D + 0.3 I)) */
    if (sc->filter2d) comp *= sqrt((det0 > 0.0 ? det0 : 0.0) / det);
    o->cov[0] = C[0][0]; o->cov[1] = C[0][1]; o->cov[2] = C[1][1];
    o->conic[0] = C[1][1] / det;
    o->conic[1] = -C[0][1] / det;
    o->conic[2] = C[0][0] / det;
    o->opacity = (double)sc->opac[g] * mult * comp;
    /* colour: direction from the camera centre to the mean (world space) */
    double d[3] = { mu[0] - cam->center[0], mu[1] - cam->center[1], mu[2] - cam->center[2] };
    double dn = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double Y[16];
    sh_basis(d[0] / dn, d[1] / dn, d[2] / dn, Y);
    int nc = (sc->sh_degree + 1) * (sc->sh_degree + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int k = 0; k < nc; ++k) acc += (double)sc->sh[(g * 16 + k) * 3 + ch] * Y[k];
        acc += 0.5;
        o->rgb[ch] = acc > 0.0 ? acc : 0.0;
    }
}

/* ---------------------------------------------------------------------- */
/* per-pixel compositing (Eq. 1 alpha, front-to-back alpha blending)       */
/* ---------------------------------------------------------------------- */
typedef struct {
    int64_t rec;       /* record (position in the active list) */
    float z;           /* FP32 key depth */
} orc_item;

static int item_cmp(const void* a, const void* b)
{
    const orc_item* x = (const orc_item*)a;
    const orc_item* y = (const orc_item*)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return (x->rec > y->rec) - (x->rec < y->rec);
}

typedef struct {
    double ke_alpha;   /* relative band around 1/255 flagged as knife edge */
    double ke_t;       /* relative band around T = 1e-4 flagged as knife edge */
} orc_knife;

/* Error model of the FP32 renderer being checked, used only to find the
 * decisions of Eq. 1 that FP32 may take the other way (knife edges).
 *   dd:  bound on the error of the pixel offset d = p - mu' in pixels (the
 *        FP32 projected mean and pixel coordinate);
 *   ke0: bound on the relative error of alpha from everything else (the
 *        conic, the exponent, the opacity).
 * A pair's alpha = o' G has relative error at most e = |grad ln G| dd + ke0
 * with |grad ln G| = |Sigma'^-1 d|; alpha clamped at 0.99 with o' G above
 * 0.99 (1 + e) is exact.  T = prod (1 - alpha_j) then has relative error at
 * most E = sum alpha_j / (1 - alpha_j) e_j (first order) plus one rounding
 * per factor.  The alpha < 1/255 skip is a knife edge when
 * |alpha - 1/255| <= e / 255, the T < 1e-4 stop when |T_next - 1e-4| <=
 * E 1e-4. */
typedef struct {
    double dd;
    double ke0;
} orc_fp32_err;

#define ORC_T_ROUND 1.2e-7  /* two FP32 roundings per transmittance factor */
#define ORC_MAX_RUNS 256    /* decision paths enumerated per pixel at most */

/* One pass of the per-pixel loop over a depth-sorted list:
 *   alpha = min(0.99, o' exp(-1/2 d^T Sigma'^-1 d)); skip alpha < 1/255;
 *   T_next = T (1 - alpha); stop (without blending) once T_next < 1e-4;
 *   C += T alpha rgb; T = T_next.  Background is black.
 * Knife-edge decisions are numbered in the order they are met on this pass;
 * those whose bit is set in `flip` are taken the other way.  Returns the
 * number of knife-edge decisions met. */
static int composite_pass(const orc_splat* sp, const orc_item* list, int64_t n,
                          double px, double py, const orc_fp32_err* fe, uint32_t flip,
                          double* rgb, double* Tout, int32_t* ncontrib)
{
    double T = 1.0, E = 0.0, C[3] = { 0, 0, 0 };
    int32_t nc = 0;
    int nk = 0;
    for (int64_t i = 0; i < n; ++i) {
        const orc_splat* s = sp + list[i].rec;
        double dx = px - s->mx, dy = py - s->my;
        double q = s->conic[0] * dx * dx + 2.0 * s->conic[1] * dx * dy + s->conic[2] * dy * dy;
        double G = exp(-0.5 * q);
        double a = s->opacity * G;
        double g0 = s->conic[0] * dx + s->conic[1] * dy;
        double g1 = s->conic[1] * dx + s->conic[2] * dy;
        double e = sqrt(g0 * g0 + g1 * g1) * fe->dd + fe->ke0;
        if (a > ORC_ALPHA_MAX) {
            if (a >= ORC_ALPHA_MAX * (1.0 + e)) e = 0.0;
            a = ORC_ALPHA_MAX;
        }
        int skip = a < ORC_ALPHA_MIN;
        if (fabs(a - ORC_ALPHA_MIN) <= e * ORC_ALPHA_MIN) {
            if (nk < 32 && ((flip >> nk) & 1u)) skip = !skip;
            ++nk;
        }
        if (skip) continue;
        double Tn = T * (1.0 - a);
        double En = E + a / (1.0 - a) * e + ORC_T_ROUND;
        int stop = Tn < ORC_T_MIN;
        if (fabs(Tn - ORC_T_MIN) <= En * ORC_T_MIN) {
            if (nk < 32 && ((flip >> nk) & 1u)) stop = !stop;
            ++nk;
        }
        if (stop) break;
        for (int c = 0; c < 3; ++c) C[c] += T * a * s->rgb[c];
        T = Tn;
        E = En;
        ++nc;
    }
    rgb[0] = C[0]; rgb[1] = C[1]; rgb[2] = C[2];
    *Tout = T;
    *ncontrib = nc;
    return nk;
}

/* Composite one pixel.  rgb/T/ncontrib are the pass that takes every
 * decision as FP64 does.  knife: 0 = no knife-edge decision; 1 = some, and
 * lo/hi (when given) bound, per channel, every result reachable by taking
 * any subset of them the other way (all of which are correct FP32 renders);
 * 2 = more decision paths than ORC_MAX_RUNS, lo/hi incomplete. */
static void composite_pixel(const orc_splat* sp, const orc_item* list, int64_t n,
                            double px, double py, const orc_fp32_err* fe,
                            double* rgb, double* Tout, int32_t* ncontrib, uint8_t* knife,
                            double* lo, double* hi)
{
    int k0 = composite_pass(sp, list, n, px, py, fe, 0u, rgb, Tout, ncontrib);
    *knife = k0 > 0;
    if (lo) for (int c = 0; c < 3; ++c) { lo[c] = rgb[c]; hi[c] = rgb[c]; }
    if (k0 == 0 || !lo) return;
    /* depth-first over flip sets: a path's decisions before its highest
     * flipped one are those of its parent, so children flip later ones */
    uint32_t stack[ORC_MAX_RUNS + 64];
    int sp_top = 0, runs = 1, incomplete = k0 > 32;
    for (int j = 0; j < k0 && j < 32; ++j) stack[sp_top++] = 1u << j;
    while (sp_top > 0) {
        uint32_t m = stack[--sp_top];
        if (runs >= ORC_MAX_RUNS) { incomplete = 1; break; }
        double c3[3], Tt;
        int32_t nct;
        int k = composite_pass(sp, list, n, px, py, fe, m, c3, &Tt, &nct);
        ++runs;
        for (int c = 0; c < 3; ++c) {
            if (c3[c] < lo[c]) lo[c] = c3[c];
            if (c3[c] > hi[c]) hi[c] = c3[c];
        }
        if (k > 32) incomplete = 1;
        int top = 31;
        while (!((m >> top) & 1u)) --top;
        for (int j = top + 1; j < k && j < 32; ++j) {
            if (sp_top >= ORC_MAX_RUNS + 64) { incomplete = 1; break; }
            stack[sp_top++] = m | (1u << j);
        }
    }
    if (incomplete) *knife = 2;
}

/* ---------------------------------------------------------------------- */
/* render                                                                   */
/* ---------------------------------------------------------------------- */
typedef struct {
    int64_t n_visible;     /* Gaussians binned to at least one tile */
    int64_t n_keys;        /* (tile, Gaussian) pairs */
    int64_t n_pairs_eval;  /* (pixel, Gaussian) evaluations performed */
} orc_stats;

/* Render the active list (gids into the scene, per-entry opacity multiplier,
 * NULL = all 1) from one camera.
 *   mode 0 (binned): each tile composites the Gaussians whose tile rect
 *     contains it, ordered by (FP32 depth, record).
 *   mode 1 (brute): each pixel composites every Gaussian in front of the
 *     near plane, ordered by (FP32 depth, record).
 * tiles: optional list of tile ids (ty * tiles_x + tx) to render (NULL =
 * all); pixels of other tiles are left untouched.  Outputs are full-image
 * arrays: rgb H*W*3, T H*W, ncontrib H*W, knife H*W, and (optional, NULL to
 * skip the enumeration) lo, hi H*W*3: composite_pixel's bounds over the
 * FP32-reachable decisions.  err_dd, err_ke0: the FP32 error model
 * (orc_fp32_err). */
int orc_render(const orc_scene* sc, const orc_camera* cam, int64_t n_active,
               const int64_t* gids, const float* mults, int32_t mode,
               const int32_t* tiles, int32_t n_tiles, double err_dd, double err_ke0,
               double* out_rgb, double* out_T, int32_t* out_nc, uint8_t* out_knife,
               double* out_lo, double* out_hi, orc_stats* stats)
{
    const int W = cam->width, H = cam->height;
    const int tx_n = (W + ORC_TILE - 1) / ORC_TILE, ty_n = (H + ORC_TILE - 1) / ORC_TILE;
    orc_fp32_err fe = { err_dd, err_ke0 };
    orc_splat* sp = (orc_splat*)malloc(sizeof(orc_splat) * (size_t)(n_active ? n_active : 1));
    orc_key_rec* kr = (orc_key_rec*)malloc(sizeof(orc_key_rec) * (size_t)(n_active ? n_active : 1));
    uint8_t* vis = (uint8_t*)calloc((size_t)(n_active ? n_active : 1), 1);
    int64_t nvis = 0, nkeys = 0;
    for (int64_t i = 0; i < n_active; ++i) {
        float m = mults ? mults[i] : 1.0f;
        vis[i] = (uint8_t)key_spec(sc, cam, gids[i], m, &kr[i]);
        if (mode == 1) {
            /* brute force keeps every Gaussian in front of the near plane */
            float pz = cam_depth32(cam, sc->means + 3 * gids[i]);
            kr[i].z = pz;
            vis[i] = pz > cam->znear;
        }
        if (vis[i]) {
            splat64(sc, cam, gids[i], (double)m, &sp[i]);
            ++nvis;
            if (mode == 0)
                nkeys += (int64_t)(kr[i].rect[2] - kr[i].rect[0] + 1) * (kr[i].rect[3] - kr[i].rect[1] + 1);
        }
    }
    int32_t ntl = tiles ? n_tiles : tx_n * ty_n;
    int64_t pairs = 0;
    if (mode == 1) {
        orc_item* all = (orc_item*)malloc(sizeof(orc_item) * (size_t)(nvis ? nvis : 1));
        int64_t k = 0;
        for (int64_t i = 0; i < n_active; ++i)
            if (vis[i]) { all[k].rec = i; all[k].z = kr[i].z; ++k; }
        qsort(all, (size_t)nvis, sizeof(orc_item), item_cmp);
        #pragma omp parallel for schedule(dynamic, 1) reduction(+:pairs)
        for (int32_t ti = 0; ti < ntl; ++ti) {
            int32_t tile = tiles ? tiles[ti] : ti;
            int tx = tile % tx_n, ty = tile / tx_n;
            for (int py = ty * ORC_TILE; py < (ty + 1) * ORC_TILE && py < H; ++py)
                for (int px = tx * ORC_TILE; px < (tx + 1) * ORC_TILE && px < W; ++px) {
                    int64_t pix = (int64_t)py * W + px;
                    composite_pixel(sp, all, nvis, px + 0.5, py + 0.5, &fe, out_rgb + 3 * pix,
                                    out_T + pix, out_nc + pix, out_knife + pix,
                                    out_lo ? out_lo + 3 * pix : NULL,
                                    out_hi ? out_hi + 3 * pix : NULL);
                    pairs += nvis;
                }
        }
        free(all);
    } else {
        /* bin: per requested tile, the Gaussians whose tile rect contains it */
        int32_t* slot = (int32_t*)malloc(sizeof(int32_t) * (size_t)tx_n * ty_n);
        for (int32_t t = 0; t < tx_n * ty_n; ++t) slot[t] = -1;
        for (int32_t ti = 0; ti < ntl; ++ti) slot[tiles ? tiles[ti] : ti] = ti;
        int64_t* cnt = (int64_t*)calloc((size_t)ntl + 1, sizeof(int64_t));
        for (int64_t i = 0; i < n_active; ++i) {
            if (!vis[i]) continue;
            for (int ty = kr[i].rect[1]; ty <= kr[i].rect[3]; ++ty)
                for (int tx = kr[i].rect[0]; tx <= kr[i].rect[2]; ++tx) {
                    int32_t s = slot[ty * tx_n + tx];
                    if (s >= 0) cnt[s + 1]++;
                }
        }
        for (int32_t s = 0; s < ntl; ++s) cnt[s + 1] += cnt[s];
        orc_item* lists = (orc_item*)malloc(sizeof(orc_item) * (size_t)(cnt[ntl] ? cnt[ntl] : 1));
        int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ntl ? ntl : 1));
        for (int32_t s = 0; s < ntl; ++s) fill[s] = cnt[s];
        for (int64_t i = 0; i < n_active; ++i) {
            if (!vis[i]) continue;
            for (int ty = kr[i].rect[1]; ty <= kr[i].rect[3]; ++ty)
                for (int tx = kr[i].rect[0]; tx <= kr[i].rect[2]; ++tx) {
                    int32_t s = slot[ty * tx_n + tx];
                    if (s >= 0) { lists[fill[s]].rec = i; lists[fill[s]].z = kr[i].z; fill[s]++; }
                }
        }
        #pragma omp parallel for schedule(dynamic, 1) reduction(+:pairs)
        for (int32_t s = 0; s < ntl; ++s) {
            int32_t tile = tiles ? tiles[s] : s;
            int tx = tile % tx_n, ty = tile / tx_n;
            orc_item* L = lists + cnt[s];
            int64_t n = cnt[s + 1] - cnt[s];
            qsort(L, (size_t)n, sizeof(orc_item), item_cmp);
            for (int py = ty * ORC_TILE; py < (ty + 1) * ORC_TILE && py < H; ++py)
                for (int px = tx * ORC_TILE; px < (tx + 1) * ORC_TILE && px < W; ++px) {
                    int64_t pix = (int64_t)py * W + px;
                    composite_pixel(sp, L, n, px + 0.5, py + 0.5, &fe, out_rgb + 3 * pix,
                                    out_T + pix, out_nc + pix, out_knife + pix,
                                    out_lo ? out_lo + 3 * pix : NULL,
                                    out_hi ? out_hi + 3 * pix : NULL);
                    pairs += n;
                }
        }
        free(slot); free(cnt); free(lists); free(fill);
    }
    if (stats) { stats->n_visible = nvis; stats->n_keys = nkeys; stats->n_pairs_eval = pairs; }
    free(sp); free(kr); free(vis);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* importance score (Sec. 3 "Importance pruning" and "Visibility filtering",  */
/* after RadSplat): the largest blending weight T * alpha a Gaussian          */
/* receives at any pixel of the view, where it is composited.  The pixels,    */
/* order and decisions are those of orc_render's binned mode.                  */
/* ---------------------------------------------------------------------- */
/* One pixel: walk the list as composite_pixel does and raise score[rec] to
 * T * alpha for every composited entry; the flags say whether the pixel has a
 * knife-edge decision (composite_pixel's bands). */
static void importance_pixel(const orc_splat* sp, const orc_item* list, int64_t n, double px,
                             double py, const orc_knife* ke, double* score_all,
                             double* score_clean)
{
    /* first pass: is this pixel a knife edge? */
    double T = 1.0;
    int kf = 0;
    for (int64_t i = 0; i < n; ++i) {
        const orc_splat* s = sp + list[i].rec;
        double dx = px - s->mx, dy = py - s->my;
        double q = s->conic[0] * dx * dx + 2.0 * s->conic[1] * dx * dy + s->conic[2] * dy * dy;
        double a = s->opacity * exp(-0.5 * q);
        if (a > ORC_ALPHA_MAX) a = ORC_ALPHA_MAX;
        if (fabs(a - ORC_ALPHA_MIN) <= ke->ke_alpha * ORC_ALPHA_MIN) kf = 1;
        if (a < ORC_ALPHA_MIN) continue;
        double Tn = T * (1.0 - a);
        if (fabs(Tn - ORC_T_MIN) <= ke->ke_t * ORC_T_MIN) kf = 1;
        if (Tn < ORC_T_MIN) break;
        T = Tn;
    }
    /* second pass: the weights */
    T = 1.0;
    for (int64_t i = 0; i < n; ++i) {
        const orc_splat* s = sp + list[i].rec;
        double dx = px - s->mx, dy = py - s->my;
        double q = s->conic[0] * dx * dx + 2.0 * s->conic[1] * dx * dy + s->conic[2] * dy * dy;
        double a = s->opacity * exp(-0.5 * q);
        if (a > ORC_ALPHA_MAX) a = ORC_ALPHA_MAX;
        if (a < ORC_ALPHA_MIN) continue;
        double Tn = T * (1.0 - a);
        if (Tn < ORC_T_MIN) break;
        double w = T * a;
        int64_t r = list[i].rec;
        if (w > score_all[r]) score_all[r] = w;
        if (!kf && w > score_clean[r]) score_clean[r] = w;
        T = Tn;
    }
}

/* score_all[i]: largest weight of active entry i over all pixels (0 if it is
 * never composited); score_clean[i]: the same over the pixels without a
 * knife-edge decision.  Both are raised, not overwritten, so several views
 * accumulate by calling again. */
int orc_importance(const orc_scene* sc, const orc_camera* cam, int64_t n_active,
                   const int64_t* gids, const float* mults, double ke_alpha, double ke_t,
                   double* score_all, double* score_clean)
{
    const int W = cam->width, H = cam->height;
    const int tx_n = (W + ORC_TILE - 1) / ORC_TILE, ty_n = (H + ORC_TILE - 1) / ORC_TILE;
    const int32_t ntl = tx_n * ty_n;
    orc_knife ke = { ke_alpha, ke_t };
    size_t na = (size_t)(n_active ? n_active : 1);
    orc_splat* sp = (orc_splat*)malloc(sizeof(orc_splat) * na);
    orc_key_rec* kr = (orc_key_rec*)malloc(sizeof(orc_key_rec) * na);
    uint8_t* vis = (uint8_t*)calloc(na, 1);
    for (int64_t i = 0; i < n_active; ++i) {
        float m = mults ? mults[i] : 1.0f;
        vis[i] = (uint8_t)key_spec(sc, cam, gids[i], m, &kr[i]);
        if (vis[i]) splat64(sc, cam, gids[i], (double)m, &sp[i]);
    }
    /* per tile, the entries whose tile rect contains it, by (depth, record) */
    int64_t* cnt = (int64_t*)calloc((size_t)ntl + 1, sizeof(int64_t));
    for (int64_t i = 0; i < n_active; ++i) {
        if (!vis[i]) continue;
        for (int ty = kr[i].rect[1]; ty <= kr[i].rect[3]; ++ty)
            for (int tx = kr[i].rect[0]; tx <= kr[i].rect[2]; ++tx) cnt[ty * tx_n + tx + 1]++;
    }
    for (int32_t t = 0; t < ntl; ++t) cnt[t + 1] += cnt[t];
    orc_item* lists = (orc_item*)malloc(sizeof(orc_item) * (size_t)(cnt[ntl] ? cnt[ntl] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)ntl);
    for (int32_t t = 0; t < ntl; ++t) fill[t] = cnt[t];
    for (int64_t i = 0; i < n_active; ++i) {
        if (!vis[i]) continue;
        for (int ty = kr[i].rect[1]; ty <= kr[i].rect[3]; ++ty)
            for (int tx = kr[i].rect[0]; tx <= kr[i].rect[2]; ++tx) {
                int64_t f = fill[ty * tx_n + tx]++;
                lists[f].rec = i;
                lists[f].z = kr[i].z;
            }
    }
    /* scores per entry are local to this call, then raised into the outputs */
    double* sa = (double*)calloc(na, sizeof(double));
    double* scl = (double*)calloc(na, sizeof(double));
    for (int32_t t = 0; t < ntl; ++t) {
        int tx = t % tx_n, ty = t / tx_n;
        orc_item* L = lists + cnt[t];
        int64_t n = cnt[t + 1] - cnt[t];
        qsort(L, (size_t)n, sizeof(orc_item), item_cmp);
        for (int py = ty * ORC_TILE; py < (ty + 1) * ORC_TILE && py < H; ++py)
            for (int px = tx * ORC_TILE; px < (tx + 1) * ORC_TILE && px < W; ++px)
                importance_pixel(sp, L, n, px + 0.5, py + 0.5, &ke, sa, scl);
    }
    for (int64_t i = 0; i < n_active; ++i) {
        if (sa[i] > score_all[i]) score_all[i] = sa[i];
        if (scl[i] > score_clean[i]) score_clean[i] = scl[i];
    }
    free(sp); free(kr); free(vis); free(cnt); free(lists); free(fill); free(sa); free(scl);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* per-Gaussian projection records and the sorted tile key list             */
/* ---------------------------------------------------------------------- */
/* For each active entry: visible flag, FP32 depth, tile rect, FP32 final
 * opacity, and the FP64 splat (mean', conic, opacity, rgb). */
void orc_project(const orc_scene* sc, const orc_camera* cam, int64_t n_active,
                 const int64_t* gids, const float* mults, uint8_t* visible, float* z,
                 int32_t* rect, float* o32, double* mean2, double* conic, double* cov,
                 double* opac, double* rgb)
{
    for (int64_t i = 0; i < n_active; ++i) {
        float m = mults ? mults[i] : 1.0f;
        orc_key_rec kr;
        int v = key_spec(sc, cam, gids[i], m, &kr);
        visible[i] = (uint8_t)v;
        if (!v) continue;
        z[i] = kr.z;
        o32[i] = kr.o32;
        for (int k = 0; k < 4; ++k) rect[4 * i + k] = kr.rect[k];
        orc_splat s;
        splat64(sc, cam, gids[i], (double)m, &s);
        mean2[2 * i] = s.mx; mean2[2 * i + 1] = s.my;
        for (int k = 0; k < 3; ++k) {
            conic[3 * i + k] = s.conic[k];
            cov[3 * i + k] = s.cov[k];
            rgb[3 * i + k] = s.rgb[k];
        }
        opac[i] = s.opacity;
    }
}

typedef struct { uint64_t key; int64_t rec; } orc_kv;

static int kv_cmp(const void* a, const void* b)
{
    const orc_kv* x = (const orc_kv*)a;
    const orc_kv* y = (const orc_kv*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->rec > y->rec) - (x->rec < y->rec);
}

/* The binned key list: one key per (tile, Gaussian) pair,
 * key = tile_id << 32 | bits(FP32 depth), tile_id = ty * tiles_x + tx,
 * sorted by (key, record).  Depth > znear > 0, so its IEEE bits order like
 * the depth.  Returns the number of keys; writes at most cap of them (keys
 * and the gid of each). */
int64_t orc_keys(const orc_scene* sc, const orc_camera* cam, int64_t n_active,
                 const int64_t* gids, const float* mults, uint64_t* keys_out,
                 int64_t* gid_out, int64_t cap)
{
    const int tx_n = (cam->width + ORC_TILE - 1) / ORC_TILE;
    int64_t n = 0;
    orc_key_rec* kr = (orc_key_rec*)malloc(sizeof(orc_key_rec) * (size_t)(n_active ? n_active : 1));
    uint8_t* vis = (uint8_t*)malloc((size_t)(n_active ? n_active : 1));
    for (int64_t i = 0; i < n_active; ++i) {
        vis[i] = (uint8_t)key_spec(sc, cam, gids[i], mults ? mults[i] : 1.0f, &kr[i]);
        if (vis[i]) n += (int64_t)(kr[i].rect[2] - kr[i].rect[0] + 1) * (kr[i].rect[3] - kr[i].rect[1] + 1);
    }
    if (n <= cap) {
        orc_kv* kv = (orc_kv*)malloc(sizeof(orc_kv) * (size_t)(n ? n : 1));
        int64_t k = 0;
        for (int64_t i = 0; i < n_active; ++i) {
            if (!vis[i]) continue;
            uint64_t zb = f32_as_u32(kr[i].z);
            for (int ty = kr[i].rect[1]; ty <= kr[i].rect[3]; ++ty)
                for (int tx = kr[i].rect[0]; tx <= kr[i].rect[2]; ++tx) {
                    kv[k].key = ((uint64_t)(uint32_t)(ty * tx_n + tx) << 32) | zb;
                    kv[k].rec = i;
                    ++k;
                }
        }
        qsort(kv, (size_t)n, sizeof(orc_kv), kv_cmp);
        for (int64_t j = 0; j < n; ++j) { keys_out[j] = kv[j].key; gid_out[j] = gids[kv[j].rec]; }
        free(kv);
    }
    free(kr); free(vis);
    return n;
}
