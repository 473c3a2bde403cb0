// Adjoint of the frame path for the fine-tuning of a level (Sec. 3 "Building
// LOD representation" and the supplementary optimisation steps: each level
// is fine-tuned with gradients through the renderer).
//
// K8 blend_bwd: per tile and pixel, the Gaussians the pixel blended are
// walked back to front, starting from the stored final transmittance and
// the stored count `last`.  Transmittance before Gaussian i is restored as
// T_i = T_{i+1} / (1 - alpha_i) (no per-pair state is kept), and the colour
// composited behind i, normalised by T_{i+1}, follows
// B_{i-1} = alpha_i c_i + (1 - alpha_i) B_i.  With C = P + T_i alpha_i c_i +
// T_i (1 - alpha_i) B_i:  dC/dc_i = T_i alpha_i,  dC/dalpha_i = T_i (c_i - B_i).
// alpha = min(0.99, 2^(log2 o' - q)) is recomputed with the forward's exact
// FP32 operations, so the skip (alpha < 1/255) and the clamp decide
// identically.
// Per-Gaussian sums are warp-reduced, then added with atomics.
//
// K9 project_bwd: per visible record, the gradients of (mean', U, o', rgb)
// are mapped back through the Cholesky form of the inverse covariance, the
// EWA Jacobian, the quaternion rotation, the Eq. 3 filter, degree-3 SH and
// the activations to the raw parameters, and added (+=) to the caller's
// gradient arrays (each Gaussian has at most one record per frame).
#include "common.cuh"

namespace lodge {

namespace {

constexpr int kBatch = 256;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kHalfLog2e = 0.7213475204444817f;


__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256)
blend_bwd_kernel(int32_t width, int32_t height, int32_t tiles_x, const uint2* __restrict__ ranges,
                 const uint32_t* __restrict__ tile_val, uint32_t vmask, uint32_t n_keys, uint32_t n_rec,
                 const float4* __restrict__ rec_a, const float4* __restrict__ rec_b,
                 const float* __restrict__ rec_c, const float* __restrict__ T_final,
                 const uint32_t* __restrict__ last, const float* __restrict__ dL_drgb,
                 double* __restrict__ grec) {
    __shared__ float4 sa[kBatch];
    __shared__ float4 sb[kBatch];
    __shared__ float sc[kBatch];
    __shared__ uint32_t sr[kBatch];
    __shared__ uint32_t s_max;
    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int x = tx * kTile + (warp & 1) * 8 + (lane & 7);
    const int y = ty * kTile + (warp >> 1) * 4 + (lane >> 3);
    const bool inside = x < width && y < height;
    const float pxf = (float)x + 0.5f, pyf = (float)y + 0.5f;
    uint2 rg = ranges[tile];
    if (rg.y > n_keys || rg.x > rg.y) rg = make_uint2(0, 0);
    const uint32_t n = rg.y - rg.x;
    const int64_t pix = (int64_t)y * width + x;
    float T = 1.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
    uint32_t L = 0;
    if (inside) {
        T = T_final[pix];
        L = min(last[pix], n);
        g0 = dL_drgb[3 * pix];
        g1 = dL_drgb[3 * pix + 1];
        g2 = dL_drgb[3 * pix + 2];
    }
    if (tid == 0) s_max = 0;
    __syncthreads();
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, L);
    if (lane == 0) atomicMax(&s_max, wmax);
    __syncthreads();
    const uint32_t maxL = s_max;
    float B0 = 0.f, B1 = 0.f, B2 = 0.f;
    const int nb = (int)((maxL + kBatch - 1) / kBatch);
    for (int b = nb - 1; b >= 0; --b) {
        __syncthreads();
        const uint32_t idx = (uint32_t)b * kBatch + tid;
        if (idx < maxL) {
            const uint32_t j = min(tile_val[rg.x + idx] & vmask, n_rec - 1u);
            sr[tid] = j;
            sa[tid] = rec_a[j];
            sb[tid] = rec_b[j];
            sc[tid] = rec_c[j];
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBatch, maxL - (uint32_t)b * kBatch);
        for (int k = cnt - 1; k >= 0; --k) {
            const uint32_t i = (uint32_t)b * kBatch + k;
            float d_mx = 0.f, d_my = 0.f, d_u00 = 0.f, d_u01 = 0.f, d_u11 = 0.f, d_o = 0.f;
            float d_r = 0.f, d_g = 0.f, d_b = 0.f;
            bool contrib = false;
            if (i < L) {
                const float4 a = sa[k];
                const float4 bb = sb[k];
                const float dx = pxf - a.x, dy = pyf - a.y;
                // the forward's t, w and alpha (same operations), raw = o' 2^-q
                float t, wq;
                pixel_tw(a, bb, dx, y, t, wq);
                const float raw = ex2_approx(fmaf(-t, t, fmaf(-wq, wq, bb.y)));
                const float alpha = fminf(0.99f, raw);
                if (alpha >= (1.0f / 255.0f)) {
                    contrib = true;
                    const float cr = bb.z, cg = bb.w, cb = sc[k];
                    const float Ti = T / (1.f - alpha);
                    const float wgt = Ti * alpha;
                    d_r = wgt * g0;
                    d_g = wgt * g1;
                    d_b = wgt * g2;
                    const float dA = Ti * ((cr - B0) * g0 + (cg - B1) * g1 + (cb - B2) * g2);
                    B0 = alpha * cr + (1.f - alpha) * B0;
                    B1 = alpha * cg + (1.f - alpha) * B1;
                    B2 = alpha * cb + (1.f - alpha) * B2;
                    T = Ti;
                    if (raw < 0.99f) {
                        const float G = ex2_approx(-fmaf(t, t, wq * wq));   // 2^-q = d alpha / d o'
                        d_o = dA * G;
                        const float dq = -kLn2 * raw * dA;
                        const float dt = 2.f * t * dq, dw = 2.f * wq * dq;
                        d_u00 = dt * dx;
                        d_u01 = dt * dy;
                        d_u11 = dw * dy;
                        d_mx = -(dt * a.z);
                        d_my = -(dt * a.w + dw * bb.x);
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                d_mx = warp_sum(d_mx); d_my = warp_sum(d_my);
                d_u00 = warp_sum(d_u00); d_u01 = warp_sum(d_u01); d_u11 = warp_sum(d_u11);
                d_o = warp_sum(d_o);
                d_r = warp_sum(d_r); d_g = warp_sum(d_g); d_b = warp_sum(d_b);
                // the per-record sums run over every pixel the record covers,
                // often with terms of both signs: accumulate the warp partials
                // in FP64 so their number does not grow the rounding error
                if (lane == 0) {
                    const uint32_t r = sr[k];
                    double* g = grec + r;
                    atomicAdd(g + 0 * (size_t)n_rec, (double)d_mx);
                    atomicAdd(g + 1 * (size_t)n_rec, (double)d_my);
                    atomicAdd(g + 2 * (size_t)n_rec, (double)d_u00);
                    atomicAdd(g + 3 * (size_t)n_rec, (double)d_u01);
                    atomicAdd(g + 4 * (size_t)n_rec, (double)d_u11);
                    atomicAdd(g + 5 * (size_t)n_rec, (double)d_o);
                    atomicAdd(g + 6 * (size_t)n_rec, (double)d_r);
                    atomicAdd(g + 7 * (size_t)n_rec, (double)d_g);
                    atomicAdd(g + 8 * (size_t)n_rec, (double)d_b);
                }
            }
        }
    }
}

constexpr float kY0 = 0.28209479177387814f;
constexpr float kC1 = 0.4886025119029199f;
constexpr float kC2a = 1.0925484305920792f;
constexpr float kC2b = 0.31539156525252005f;
constexpr float kC2c = 0.5462742152960396f;
constexpr float kC3a = 0.5900435899266435f;
constexpr float kC3b = 2.890611442640554f;
constexpr float kC3c = 0.4570457994644658f;
constexpr float kC3d = 0.3731763325901154f;
constexpr float kC3e = 1.445305721320277f;

// basis values and gradients (d Y / d dir) of the real SH up to degree 3
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, float* Y, float* Gx,
                                              float* Gy, float* Gz) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = kY0; Gx[0] = 0.f; Gy[0] = 0.f; Gz[0] = 0.f;
    Y[1] = kC1 * y; Gx[1] = 0.f; Gy[1] = kC1; Gz[1] = 0.f;
    Y[2] = kC1 * z; Gx[2] = 0.f; Gy[2] = 0.f; Gz[2] = kC1;
    Y[3] = kC1 * x; Gx[3] = kC1; Gy[3] = 0.f; Gz[3] = 0.f;
    Y[4] = kC2a * x * y; Gx[4] = kC2a * y; Gy[4] = kC2a * x; Gz[4] = 0.f;
    Y[5] = kC2a * y * z; Gx[5] = 0.f; Gy[5] = kC2a * z; Gz[5] = kC2a * y;
    Y[6] = kC2b * (3.f * zz - 1.f); Gx[6] = 0.f; Gy[6] = 0.f; Gz[6] = 6.f * kC2b * z;
    Y[7] = kC2a * x * z; Gx[7] = kC2a * z; Gy[7] = 0.f; Gz[7] = kC2a * x;
    Y[8] = kC2c * (xx - yy); Gx[8] = 2.f * kC2c * x; Gy[8] = -2.f * kC2c * y; Gz[8] = 0.f;
    Y[9] = kC3a * y * (3.f * xx - yy); Gx[9] = 6.f * kC3a * x * y; Gy[9] = kC3a * (3.f * xx - 3.f * yy); Gz[9] = 0.f;
    Y[10] = kC3b * x * y * z; Gx[10] = kC3b * y * z; Gy[10] = kC3b * x * z; Gz[10] = kC3b * x * y;
    Y[11] = kC3c * y * (5.f * zz - 1.f); Gx[11] = 0.f; Gy[11] = kC3c * (5.f * zz - 1.f); Gz[11] = 10.f * kC3c * y * z;
    Y[12] = kC3d * z * (5.f * zz - 3.f); Gx[12] = 0.f; Gy[12] = 0.f; Gz[12] = kC3d * (15.f * zz - 3.f);
    Y[13] = kC3c * x * (5.f * zz - 1.f); Gx[13] = kC3c * (5.f * zz - 1.f); Gy[13] = 0.f; Gz[13] = 10.f * kC3c * x * z;
    Y[14] = kC3e * z * (xx - yy); Gx[14] = 2.f * kC3e * x * z; Gy[14] = -2.f * kC3e * y * z; Gz[14] = kC3e * (xx - yy);
    Y[15] = kC3a * x * (xx - 3.f * yy); Gx[15] = kC3a * (3.f * xx - 3.f * yy); Gy[15] = -6.f * kC3a * x * y; Gz[15] = 0.f;
}

struct BwdParams {
    DevCamera cam;
    int64_t n_rec;
    const uint32_t* rec_gid;
    const double* grec;          // 9 x n_rec
    const float* means;          // N x 3 raw
    const float4* act_so;        // (s0, s1, s2, o) activated
    const float4* act_q;         // unit quaternion
    const float* sh;             // N x 48
    int32_t sh_degree;
    BwdLevels lv;
    float* g_means;
    float* g_log_scales;
    float* g_quats;
    const float* quats;          // N x 4 raw (for the normalisation adjoint)
    float* g_logits;
    float* g_sh;
};

__global__ void __launch_bounds__(128) project_bwd_kernel(BwdParams P) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= P.n_rec) return;
    const uint32_t gid = P.rec_gid[r];
    // only the trained level's Gaussians receive gradients (the other
    // levels of an LOD frame are fixed)
    if ((int64_t)gid < P.lv.train_lo || (int64_t)gid >= P.lv.train_hi) return;
    const size_t g = (size_t)((int64_t)gid - P.lv.train_lo);   // into the trained level's arrays
    const size_t nr = (size_t)P.n_rec;
    const float gmx = (float)P.grec[r], gmy = (float)P.grec[nr + r];
    const float gu00 = (float)P.grec[2 * nr + r], gu01 = (float)P.grec[3 * nr + r],
                gu11 = (float)P.grec[4 * nr + r];
    const float gop = (float)P.grec[5 * nr + r];
    const float grgb[3] = {(float)P.grec[6 * nr + r], (float)P.grec[7 * nr + r],
                           (float)P.grec[8 * nr + r]};
    const DevCamera& cam = P.cam;
    const float* R = cam.R;

    // ---- forward recomputation (same formulas as the projection)
    const float mu0 = P.means[3 * g], mu1 = P.means[3 * g + 1], mu2 = P.means[3 * g + 2];
    const float e0 = mu0 - cam.chat[0], e1 = mu1 - cam.chat[1], e2 = mu2 - cam.chat[2];
    const float px = R[0] * e0 + R[1] * e1 + R[2] * e2 + cam.tp[0];
    const float py = R[3] * e0 + R[4] * e1 + R[5] * e2 + cam.tp[1];
    const float pz = R[6] * e0 + R[7] * e1 + R[8] * e2 + cam.tp[2];
    const float4 so = P.act_so[gid];
    const float4 qn = P.act_q[gid];
    int lvl = 0;
    while (lvl + 1 < P.lv.num_levels && (int64_t)gid >= P.lv.level_off[lvl + 1]) ++lvl;
    const float v = P.lv.filter_var[lvl];
    float s[3] = {so.x, so.y, so.z}, sig[3] = {so.x, so.y, so.z};
    float comp = 1.f;
    if (v > 0.f) {
        for (int k = 0; k < 3; ++k) { sig[k] = sqrtf(s[k] * s[k] + v); comp *= s[k] / sig[k]; }
    }
    const float iz = 1.f / pz;
    // Jacobian at the laterally clamped point uc = clamp(px / pz), wc likewise;
    // the clamp passes the derivative only inside the limits (closed range)
    const float ux = px * iz, uy = py * iz;
    const bool inx = fabsf(ux) <= cam.limx, iny = fabsf(uy) <= cam.limy;
    const float uc = fminf(fmaxf(ux, -cam.limx), cam.limx);
    const float wc = fminf(fmaxf(uy, -cam.limy), cam.limy);
    const float j00 = cam.fx * iz, j02 = -cam.fx * uc * iz;
    const float j11 = cam.fy * iz, j12 = -cam.fy * wc * iz;
    float T0[3], T1[3];
    for (int k = 0; k < 3; ++k) {
        T0[k] = j00 * R[k] + j02 * R[6 + k];
        T1[k] = j11 * R[3 + k] + j12 * R[6 + k];
    }
    const float qw = qn.x, qx = qn.y, qy = qn.z, qz = qn.w;
    float M[3][3];
    M[0][0] = 1.f - 2.f * (qy * qy + qz * qz); M[0][1] = 2.f * (qx * qy - qw * qz); M[0][2] = 2.f * (qx * qz + qw * qy);
    M[1][0] = 2.f * (qx * qy + qw * qz); M[1][1] = 1.f - 2.f * (qx * qx + qz * qz); M[1][2] = 2.f * (qy * qz - qw * qx);
    M[2][0] = 2.f * (qx * qz - qw * qy); M[2][1] = 2.f * (qy * qz + qw * qx); M[2][2] = 1.f - 2.f * (qx * qx + qy * qy);
    float A0[3], A1[3], B0[3], B1[3];
    for (int k = 0; k < 3; ++k) {
        A0[k] = T0[0] * M[0][k] + T0[1] * M[1][k] + T0[2] * M[2][k];
        A1[k] = T1[0] * M[0][k] + T1[1] * M[1][k] + T1[2] * M[2][k];
        B0[k] = A0[k] * sig[k];
        B1[k] = A1[k] * sig[k];
    }
    const float a = B0[0] * B0[0] + B0[1] * B0[1] + B0[2] * B0[2] + 0.3f;
    const float c = B1[0] * B1[0] + B1[1] * B1[1] + B1[2] * B1[2] + 0.3f;
    const float b = B0[0] * B1[0] + B0[1] * B1[1] + B0[2] * B1[2];
    const float m01 = fmaf(B0[0], B1[1], -B0[1] * B1[0]);
    const float m02 = fmaf(B0[0], B1[2], -B0[2] * B1[0]);
    const float m12 = fmaf(B0[1], B1[2], -B0[2] * B1[1]);
    const float D = m01 * m01 + m02 * m02 + m12 * m12 + 0.3f * (a + c - 0.6f) + 0.09f;
    const float rD = 1.f / sqrtf(D);
    const float u11 = sqrtf(kHalfLog2e / c);
    const float u00 = u11 * c * rD;
    const float u01 = -u11 * b * rD;

    // ---- U -> (a, b, c) of Sigma'
    const float iD = 1.f / D, ic = 1.f / c;
    const float du00_da = -0.5f * u00 * c * iD;
    const float du00_db = u00 * b * iD;
    const float du00_dc = u00 * (0.5f * ic - 0.5f * a * iD);
    const float du01_da = -0.5f * u01 * c * iD;
    const float du01_db = -sqrtf(kHalfLog2e) * a * sqrtf(c) * iD * rD;
    const float du01_dc = u01 * (-0.5f * ic - 0.5f * a * iD);
    const float du11_dc = -0.5f * u11 * ic;
    const float ga = gu00 * du00_da + gu01 * du01_da;
    const float gb = gu00 * du00_db + gu01 * du01_db;
    const float gc = gu00 * du00_dc + gu01 * du01_dc + gu11 * du11_dc;
    // ---- Sigma' = B B^T + 0.3 I,  B = T M diag(sigma)
    float gsig[3], gT0[3] = {0, 0, 0}, gT1[3] = {0, 0, 0}, gM[3][3];
    for (int k = 0; k < 3; ++k) {
        const float gB0 = 2.f * B0[k] * ga + B1[k] * gb;
        const float gB1 = 2.f * B1[k] * gc + B0[k] * gb;
        gsig[k] = A0[k] * gB0 + A1[k] * gB1;
        const float gA0 = sig[k] * gB0, gA1 = sig[k] * gB1;
        for (int j = 0; j < 3; ++j) {
            gT0[j] += gA0 * M[j][k];
            gT1[j] += gA1 * M[j][k];
            gM[j][k] = T0[j] * gA0 + T1[j] * gA1;
        }
    }
    // ---- T = J R
    float gj00 = 0.f, gj02 = 0.f, gj11 = 0.f, gj12 = 0.f;
    for (int k = 0; k < 3; ++k) {
        gj00 += gT0[k] * R[k];
        gj02 += gT0[k] * R[6 + k];
        gj11 += gT1[k] * R[3 + k];
        gj12 += gT1[k] * R[6 + k];
    }
    // j02 = -fx uc / pz: d/dpx = -fx iz duc/dpx, d/dpz = fx uc iz^2 - fx iz duc/dpz
    // with duc/dpx = iz, duc/dpz = -px iz^2 inside the limits and 0 outside
    const float dux_dpx = inx ? iz : 0.f, dux_dpz = inx ? -px * iz * iz : 0.f;
    const float duy_dpy = iny ? iz : 0.f, duy_dpz = iny ? -py * iz * iz : 0.f;
    float gpx = gj02 * (-cam.fx * iz * dux_dpx) + gmx * cam.fx * iz;
    float gpy = gj12 * (-cam.fy * iz * duy_dpy) + gmy * cam.fy * iz;
    float gpz = gj00 * (-cam.fx * iz * iz) + gj02 * (cam.fx * uc * iz * iz - cam.fx * iz * dux_dpz) +
                gj11 * (-cam.fy * iz * iz) + gj12 * (cam.fy * wc * iz * iz - cam.fy * iz * duy_dpz) +
                gmx * (-cam.fx * px * iz * iz) + gmy * (-cam.fy * py * iz * iz);
    float gmu[3];
    for (int k = 0; k < 3; ++k) gmu[k] = R[k] * gpx + R[3 + k] * gpy + R[6 + k] * gpz;

    // ---- colour: rgb = max(0, sum Y_k sh_k + 0.5), Y at the unit direction
    const float ex = e0 - cam.clo[0], ey = e1 - cam.clo[1], ez = e2 - cam.clo[2];
    const float en = sqrtf(ex * ex + ey * ey + ez * ez), ien = 1.f / en;
    const float dx = ex * ien, dy = ey * ien, dz = ez * ien;
    float Y[16], Gx[16], Gy[16], Gz[16];
    sh_basis_grad(dx, dy, dz, Y, Gx, Gy, Gz);
    const int nk = (P.sh_degree + 1) * (P.sh_degree + 1);
    const float* shg = P.sh + (size_t)g * 48;
    float graw[3];
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.5f;
        for (int k = 0; k < nk; ++k) acc = fmaf(Y[k], shg[3 * k + ch], acc);
        graw[ch] = acc > 0.f ? grgb[ch] : 0.f;
    }
    float gdir[3] = {0.f, 0.f, 0.f};
    if (P.g_sh) {
        float* gs = P.g_sh + (size_t)g * 48;
        for (int k = 0; k < nk; ++k)
            for (int ch = 0; ch < 3; ++ch) gs[3 * k + ch] += Y[k] * graw[ch];
    }
    for (int k = 1; k < nk; ++k) {
        const float w = shg[3 * k] * graw[0] + shg[3 * k + 1] * graw[1] + shg[3 * k + 2] * graw[2];
        gdir[0] += w * Gx[k];
        gdir[1] += w * Gy[k];
        gdir[2] += w * Gz[k];
    }
    const float dd = dx * gdir[0] + dy * gdir[1] + dz * gdir[2];
    gmu[0] += (gdir[0] - dx * dd) * ien;
    gmu[1] += (gdir[1] - dy * dd) * ien;
    gmu[2] += (gdir[2] - dz * dd) * ien;
    if (P.g_means)
        for (int k = 0; k < 3; ++k) P.g_means[3 * g + k] += gmu[k];

    // ---- quaternion: M(q_hat), q_hat = q / |q|
    if (P.g_quats) {
        const float gw = 2.f * (-qz * gM[0][1] + qy * gM[0][2] + qz * gM[1][0] - qx * gM[1][2] - qy * gM[2][0] + qx * gM[2][1]);
        const float gx = 2.f * (qy * gM[0][1] + qz * gM[0][2] + qy * gM[1][0] - 2.f * qx * gM[1][1] - qw * gM[1][2] + qz * gM[2][0] + qw * gM[2][1] - 2.f * qx * gM[2][2]);
        const float gy = 2.f * (-2.f * qy * gM[0][0] + qx * gM[0][1] + qw * gM[0][2] + qx * gM[1][0] + qz * gM[1][2] - qw * gM[2][0] + qz * gM[2][1] - 2.f * qy * gM[2][2]);
        const float gz = 2.f * (-2.f * qz * gM[0][0] - qw * gM[0][1] + qx * gM[0][2] + qw * gM[1][0] - 2.f * qz * gM[1][1] + qy * gM[1][2] + qx * gM[2][0] + qy * gM[2][1]);
        const float* qr = P.quats + 4 * (size_t)g;
        const float qnorm = sqrtf(qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3]);
        const float dot = qw * gw + qx * gx + qy * gy + qz * gz;
        const float iq = 1.f / qnorm;
        P.g_quats[4 * g + 0] += (gw - qw * dot) * iq;
        P.g_quats[4 * g + 1] += (gx - qx * dot) * iq;
        P.g_quats[4 * g + 2] += (gy - qy * dot) * iq;
        P.g_quats[4 * g + 3] += (gz - qz * dot) * iq;
    }
    // ---- opacity o' = o * comp (params path: no chunk multiplier)
    const float o = so.w;
    if (P.g_logits) P.g_logits[g] += gop * comp * o * (1.f - o);
    // ---- scales: sigma = sqrt(s^2 + v), comp = prod s / sigma; s = exp(log s)
    if (P.g_log_scales) {
        for (int k = 0; k < 3; ++k) {
            float gs = gsig[k];
            if (v > 0.f) {
                gs = gs * s[k] / sig[k] + gop * o * comp * v / (s[k] * sig[k] * sig[k]);
            }
            P.g_log_scales[3 * g + k] += gs * s[k];
        }
    }
}

}  // namespace

void launch_blend_bwd(const DevCamera& cam, const uint2* ranges, const uint32_t* tile_val,
                      uint32_t vmask, int64_t n_keys, const float4* rec_a, const float4* rec_b, const float* rec_c,
                      int64_t n_rec, const float* T_final, const uint32_t* last,
                      const float* dL_drgb, double* grec, cudaStream_t s) {
    int ntiles = cam.tiles_x * cam.tiles_y;
    if (ntiles == 0 || n_rec == 0) return;
    blend_bwd_kernel<<<ntiles, 256, 0, s>>>(cam.width, cam.height, cam.tiles_x, ranges, tile_val,
                                            vmask, (uint32_t)n_keys, (uint32_t)n_rec, rec_a, rec_b, rec_c,
                                            T_final, last, dL_drgb, grec);
}

void launch_project_bwd(const DevCamera& cam, int64_t n_rec, const uint32_t* rec_gid,
                        const double* grec, const float* means, const float4* act_so,
                        const float4* act_q, const float* quats, const float* sh, int sh_degree,
                        const BwdLevels& lv, float* g_means, float* g_log_scales, float* g_quats,
                        float* g_logits, float* g_sh, cudaStream_t s) {
    if (n_rec == 0) return;
    BwdParams P;
    P.cam = cam;
    P.n_rec = n_rec;
    P.rec_gid = rec_gid;
    P.grec = grec;
    P.means = means;
    P.act_so = act_so;
    P.act_q = act_q;
    P.quats = quats;
    P.sh = sh;
    P.sh_degree = sh_degree;
    P.lv = lv;
    P.g_means = g_means;
    P.g_log_scales = g_log_scales;
    P.g_quats = g_quats;
    P.g_logits = g_logits;
    P.g_sh = g_sh;
    project_bwd_kernel<<<(unsigned)((n_rec + 127) / 128), 128, 0, s>>>(P);
}

}  // namespace lodge
