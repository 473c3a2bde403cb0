// K3: projection of the active Gaussians (EWA splatting with the per-level
// Eq. 3 filter and the Eq. 4 opacity multiplier), degree-3 SH colour, tile
// rect and visibility compaction in one pass (decoupled look-back), so the
// records come out dense and in gid order.
//
// The integer outcomes (near cull, opacity cull, tile rect) and the depth
// sort key are computed by the "key spec": FP32 with every operation
// rounded (__fmul_rn / __fadd_rn / __fdiv_rn / __fsqrt_rn, no contraction),
// in a fixed order, so they are reproducible bit for bit.  Everything that
// only reaches pixels (the inverse covariance, colour) uses ordinary FP32.
#include "common.cuh"

namespace lodge {

namespace {

__constant__ float c_qtable[65];

struct ProjParams {
    DevScene sc;
    DevCamera cam;
    const uint32_t* list;   // active list (gid | flags) or null = dense level 0
    int64_t n_active;
    int64_t n_pad;          // plane stride of the SH planes
    float tA, tB;
    ProjectOut o;
    ProjSources src;        // block sources (kBlocks only)
};

__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }

// opacity-aware extent: bucket = FP32 exponent and 3 leading mantissa bits
__device__ __forceinline__ float extent_q(float o) {
    uint32_t top = __float_as_uint(o) >> 20;
    uint32_t b = top - (119u << 3);
    if (top > (127u << 3)) b = 64u;
    return c_qtable[b];
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
constexpr float kHalfLog2e = 0.7213475204444817f;  // (1/2) log2(e)

__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
    Y[0] = kY0;
    Y[1] = kC1 * y; Y[2] = kC1 * z; Y[3] = kC1 * x;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kC2a * x * y; Y[5] = kC2a * y * z; Y[6] = kC2b * (3.f * zz - 1.f);
    Y[7] = kC2a * x * z; Y[8] = kC2c * (xx - yy);
    Y[9] = kC3a * y * (3.f * xx - yy);
    Y[10] = kC3b * x * y * z;
    Y[11] = kC3c * y * (5.f * zz - 1.f);
    Y[12] = kC3d * z * (5.f * zz - 3.f);
    Y[13] = kC3c * x * (5.f * zz - 1.f);
    Y[14] = kC3e * z * (xx - yy);
    Y[15] = kC3a * x * (xx - 3.f * yy);
}

// Key spec of one Gaussian: camera-relative point, near cull, Eq. 3 filter
// and opacity, opacity-aware extent and the AABB tile rect, every operation
// rounded in a fixed order.  Returns false when the Gaussian yields no key;
// the outputs other than d0..d2 are then unset.
struct KeySplat {
    float d0, d1, d2;          // mean - chat
    float z, mx, my, op;       // depth, projected mean, opacity after Eq. 3 and Eq. 4
    float B0[3], B1[3];        // rows of J W R(q) diag(sigma)
    uint32_t px0, py0, px1, py1;   // pixel range (inclusive), clipped to the image
    uint32_t rx0, ry0, rx1, ry1;   // the same in tiles
};

// kPre: so_pre / q_pre already hold this Gaussian's (scale, opacity) and
// quaternion (loaded together with its mean); otherwise they are loaded here
// once the near cull has passed.
template <bool kPre = false>
__device__ __forceinline__ bool key_splat(const DevScene& sc, const DevCamera& cam, float mxw,
                                          float myw, float mzw, const float4* __restrict__ sso,
                                          const float4* __restrict__ sq, int64_t idx, uint32_t g,
                                          float mult, KeySplat& k, float4 so_pre = float4{},
                                          float4 q_pre = float4{}) {
    const float* R = cam.R;
    k.d0 = fs(mxw, cam.chat[0]);
    k.d1 = fs(myw, cam.chat[1]);
    k.d2 = fs(mzw, cam.chat[2]);
    const float d0 = k.d0, d1 = k.d1, d2 = k.d2;
    float px = fa(fa(fa(fm(R[0], d0), fm(R[1], d1)), fm(R[2], d2)), cam.tp[0]);
    float py = fa(fa(fa(fm(R[3], d0), fm(R[4], d1)), fm(R[5], d2)), cam.tp[1]);
    float pz = fa(fa(fa(fm(R[6], d0), fm(R[7], d1)), fm(R[8], d2)), cam.tp[2]);
    if (!(pz > cam.znear)) return false;
    const float4 so = kPre ? so_pre : sso[idx];
    int l = 0;
    while (l + 1 < sc.num_levels && (int64_t)g >= sc.level_off[l + 1]) ++l;
    const float v = sc.filter_var[l];
    float sig0 = so.x, sig1 = so.y, sig2 = so.z;
    float op = fm(so.w, mult);
    if (v > 0.f) {
        sig0 = __fsqrt_rn(fa(fm(so.x, so.x), v));
        sig1 = __fsqrt_rn(fa(fm(so.y, so.y), v));
        sig2 = __fsqrt_rn(fa(fm(so.z, so.z), v));
        float comp = fm(fm(__fdiv_rn(so.x, sig0), __fdiv_rn(so.y, sig1)), __fdiv_rn(so.z, sig2));
        op = fm(op, comp);
    }
    // without the compensated 2D filter the opacity is final here; with it,
    // the opacity cull waits for the compensation below
    if (!sc.filter2d && !(op >= (float)(1.0 / 255.0))) return false;
    const float4 q = kPre ? q_pre : sq[idx];
    float u = __fdiv_rn(px, pz), w = __fdiv_rn(py, pz);
    float mx = fa(fm(cam.fx, u), cam.cx);
    float my = fa(fm(cam.fy, w), cam.cy);
    // the Jacobian at x/z, y/z clamped laterally to (limx, limy); the mean
    // keeps the unclamped point
    const float uc = fminf(fmaxf(u, -cam.limx), cam.limx);
    const float wc = fminf(fmaxf(w, -cam.limy), cam.limy);
    float j00 = __fdiv_rn(cam.fx, pz), j02 = -fm(j00, uc);
    float j11 = __fdiv_rn(cam.fy, pz), j12 = -fm(j11, wc);
    float T0[3], T1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        T0[c] = fa(fm(j00, R[c]), fm(j02, R[6 + c]));
        T1[c] = fa(fm(j11, R[3 + c]), fm(j12, R[6 + c]));
    }
    float qw = q.x, qx = q.y, qy = q.z, qz = q.w;
    float xx = fm(qx, qx), yy = fm(qy, qy), zz = fm(qz, qz);
    float xy = fm(qx, qy), xz = fm(qx, qz), yz = fm(qy, qz);
    float wx = fm(qw, qx), wy = fm(qw, qy), wz = fm(qw, qz);
    float M[3][3];
    M[0][0] = fs(1.f, fm(2.f, fa(yy, zz))); M[0][1] = fm(2.f, fs(xy, wz)); M[0][2] = fm(2.f, fa(xz, wy));
    M[1][0] = fm(2.f, fa(xy, wz)); M[1][1] = fs(1.f, fm(2.f, fa(xx, zz))); M[1][2] = fm(2.f, fs(yz, wx));
    M[2][0] = fm(2.f, fs(xz, wy)); M[2][1] = fm(2.f, fa(yz, wx)); M[2][2] = fs(1.f, fm(2.f, fa(xx, yy)));
    const float sig[3] = {sig0, sig1, sig2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float a0 = fa(fa(fm(T0[0], M[0][c]), fm(T0[1], M[1][c])), fm(T0[2], M[2][c]));
        float a1 = fa(fa(fm(T1[0], M[0][c]), fm(T1[1], M[1][c])), fm(T1[2], M[2][c]));
        k.B0[c] = fm(a0, sig[c]);
        k.B1[c] = fm(a1, sig[c]);
    }
    const float aB = fa(fa(fm(k.B0[0], k.B0[0]), fm(k.B0[1], k.B0[1])), fm(k.B0[2], k.B0[2]));
    const float cB = fa(fa(fm(k.B1[0], k.B1[0]), fm(k.B1[1], k.B1[1])), fm(k.B1[2], k.B1[2]));
    if (sc.filter2d) {
        // Mip-Splatting's 2D filter: o' *= sqrt(det Sigma2D / det(Sigma2D + 0.3 I)),
        // det Sigma2D = sum of squared 2x2 minors of B (Cauchy-Binet)
        const float m01 = fs(fm(k.B0[0], k.B1[1]), fm(k.B0[1], k.B1[0]));
        const float m02 = fs(fm(k.B0[0], k.B1[2]), fm(k.B0[2], k.B1[0]));
        const float m12 = fs(fm(k.B0[1], k.B1[2]), fm(k.B0[2], k.B1[1]));
        const float D0 = fa(fa(fm(m01, m01), fm(m02, m02)), fm(m12, m12));
        const float D1 = fa(fa(D0, fm(0.3f, fa(aB, cB))), 0.09f);
        op = fm(op, __fsqrt_rn(__fdiv_rn(D0, D1)));
        if (!(op >= (float)(1.0 / 255.0))) return false;
    }
    const float Q = extent_q(op);
    float sxx = fa(aB, 0.3f);
    float syy = fa(cB, 0.3f);
    float rx = __fsqrt_rn(fm(Q, sxx)), ry = __fsqrt_rn(fm(Q, syy));
    float x0 = ceilf(fs(fs(mx, rx), 0.5f)), x1 = floorf(fs(fa(mx, rx), 0.5f));
    float y0 = ceilf(fs(fs(my, ry), 0.5f)), y1 = floorf(fs(fa(my, ry), 0.5f));
    const float xmax = (float)(cam.width - 1), ymax = (float)(cam.height - 1);
    if (x0 < 0.f) x0 = 0.f;
    if (y0 < 0.f) y0 = 0.f;
    if (x1 > xmax) x1 = xmax;
    if (y1 > ymax) y1 = ymax;
    if (!(x0 <= x1 && y0 <= y1)) return false;
    k.z = pz; k.mx = mx; k.my = my; k.op = op;
    k.px0 = (uint32_t)(int)x0; k.py0 = (uint32_t)(int)y0;
    k.px1 = (uint32_t)(int)x1; k.py1 = (uint32_t)(int)y1;
    k.rx0 = k.px0 / kTile; k.ry0 = k.py0 / kTile;
    k.rx1 = k.px1 / kTile; k.ry1 = k.py1 / kTile;
    return true;
}

// six CTAs per SM (at most 42 registers): the kernel is bound by the
// latency of its dependent gathers, so resident warps matter more than the
// few spilled words
template <bool kBlocks>
__global__ void __launch_bounds__(kProjThreads, 6)
project_kernel(ProjParams P, uint32_t* __restrict__ status, uint32_t* __restrict__ tile_counter,
               uint32_t* __restrict__ err) {
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ uint32_t s_scan[33];
    __shared__ unsigned long long s_keys, s_bkeys;
    __shared__ uint32_t s_dh[4][256];   // depth-key digit counts (the depth sort's histogram)
    if (threadIdx.x == 0) { s_tile = atomicAdd(tile_counter, 1u); s_keys = 0ull; s_bkeys = 0ull; }
    if (P.o.depth_hist)
        for (int j = threadIdx.x; j < 4 * 256; j += kProjThreads) (&s_dh[0][0])[j] = 0;
    __syncthreads();
    const uint32_t tile = s_tile;
    const uint32_t ntiles = (uint32_t)((P.n_active + kProjThreads - 1) / kProjThreads);
    const int64_t i = (int64_t)tile * kProjThreads + threadIdx.x;
    const DevScene& sc = P.sc;
    const DevCamera& cam = P.cam;

    bool vis = false;
    uint32_t g = 0, idx = 0;
    float z = 0.f, mxp = 0.f, myp = 0.f, o = 0.f;
    float B0[3], B1[3];
    float d0 = 0.f, d1 = 0.f, d2 = 0.f;
    uint32_t rx0 = 0, ry0 = 0, rx1 = 0, ry1 = 0, pr0 = 0, pr1 = 0;
    // attribute source of this entry: the scene store (indexed by gid) or a
    // chunk block (indexed by position in the block)
    const float* smx = sc.mx;
    const float* smy = sc.my;
    const float* smz = sc.mz;
    const float4* sso = sc.scale_op;
    const float4* sq = sc.quat;
    const float4* ssh = sc.sh;
    int64_t npad = P.n_pad;
    if (i < P.n_active) {
        uint32_t e = P.list ? P.list[i] : (uint32_t)i;
        idx = e & kGidMask;
        float mult = 1.f;
        if ((e & kFlagA) && !(e & kFlagB)) mult = P.tA;
        else if ((e & kFlagB) && !(e & kFlagA)) mult = P.tB;
        if (kBlocks) {
            const bool fa = (e & kFlagA) != 0;
            const int64_t nb = fa ? P.src.n_a : P.src.n_b;
            if ((int64_t)idx >= nb) { atomicOr(err, kErrBadIndex); idx = 0; mult = 0.f; }
            smx = fa ? P.src.a.mx : P.src.b.mx;
            smy = fa ? P.src.a.my : P.src.b.my;
            smz = fa ? P.src.a.mz : P.src.b.mz;
            sso = fa ? P.src.a.scale_op : P.src.b.scale_op;
            sq = fa ? P.src.a.quat : P.src.b.quat;
            ssh = fa ? P.src.a.sh : P.src.b.sh;
            npad = fa ? P.src.npad_a : P.src.npad_b;
            g = (fa ? P.src.gid_a : P.src.gid_b)[idx];
        } else {
            if ((int64_t)idx >= sc.n_total) { atomicOr(err, kErrBadIndex); idx = 0; mult = 0.f; }
            g = idx;
        }
        // the mean, (scale, opacity) and quaternion are loaded together, so
        // that one memory latency, not three in a row, precedes the key spec
        const float mxw = smx[idx], myw = smy[idx], mzw = smz[idx];
        const float4 so = sso[idx], qq = sq[idx];
        KeySplat ks;
        vis = key_splat<true>(sc, cam, mxw, myw, mzw, sso, sq, idx, g, mult, ks, so, qq);
        d0 = ks.d0; d1 = ks.d1; d2 = ks.d2;
        if (vis) {
            // start the SH planes' way into L2 now: the block scan and the
            // conic come before they are read
            const int npl = (3 * (sc.sh_degree + 1) * (sc.sh_degree + 1) + 3) / 4;
            for (int j = 0; j < npl; ++j)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(ssh + (int64_t)j * npad + idx));
        }
        if (vis) {
            z = ks.z; mxp = ks.mx; myp = ks.my; o = ks.op;
#pragma unroll
            for (int k = 0; k < 3; ++k) { B0[k] = ks.B0[k]; B1[k] = ks.B1[k]; }
            rx0 = ks.rx0; ry0 = ks.ry0; rx1 = ks.rx1; ry1 = ks.ry1;
            pr0 = ks.px0 | (ks.py0 << 16);
            pr1 = ks.px1 | (ks.py1 << 16);
        }
    }

    // ---- compaction of visible records (gid order preserved).  The CTA's
    // count is published as soon as it is known and the look-back comes
    // after the attribute work below, so successors rarely wait on it and
    // this CTA's own look-back finds its predecessors' counts in place.
    uint32_t total;
    uint32_t excl = block_exclusive_scan(vis ? 1u : 0u, s_scan, &total);
    if (threadIdx.x == 0) st_volatile(status + tile, (tile == 0 ? kStInc : kStAgg) | total);
    uint32_t nk = vis ? (rx1 - rx0 + 1) * (ry1 - ry0 + 1) : 0u;
    {
        uint32_t wsum = nk;
        for (int off = 16; off > 0; off >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
        if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(&s_keys, (unsigned long long)wsum);
    }
    if (P.o.depth_hist) {
        // the CTA's Gaussians are neighbours in the store, so their depths
        // share the high digits: lanes with the same digit add their count
        // with one shared atomic instead of contending for the word
        const uint32_t zb = __float_as_uint(z);
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const uint32_t d = vis ? (zb >> (8 * p)) & 0xffu : 0x100u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            if (vis && lane == __ffs(peers) - 1) atomicAdd(&s_dh[p][d], (uint32_t)__popc(peers));
        }
    }
    const int bl = P.o.bin_log2;
    if (bl > 0) {   // keys of the coarse bins (squares of 2^bl tiles)
        uint32_t wsum = vis ? ((rx1 >> bl) - (rx0 >> bl) + 1) * ((ry1 >> bl) - (ry0 >> bl) + 1) : 0u;
        for (int off = 16; off > 0; off >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
        if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(&s_bkeys, (unsigned long long)wsum);
    }

    float u00 = 0.f, u01 = 0.f, u11 = 0.f;
    float rgb[3] = {0.5f, 0.5f, 0.5f};
    if (vis) {
        // ---- inverse 2D covariance in Cholesky form, with (1/2) log2(e)
        // folded in: alpha = o' * 2^-((u00 dx + u01 dy)^2 + (u11 dy)^2).  The
        // determinant uses the Cauchy-Binet sum of squared 2x2 minors, which
        // has no cancellation (Sigma' = B B^T + 0.3 I).
        const float aB = B0[0] * B0[0] + B0[1] * B0[1] + B0[2] * B0[2];
        const float cB = B1[0] * B1[0] + B1[1] * B1[1] + B1[2] * B1[2];
        const float bB = B0[0] * B1[0] + B0[1] * B1[1] + B0[2] * B1[2];
        const float m01 = fmaf(B0[0], B1[1], -B0[1] * B1[0]);
        const float m02 = fmaf(B0[0], B1[2], -B0[2] * B1[0]);
        const float m12 = fmaf(B0[1], B1[2], -B0[2] * B1[1]);
        const float D = m01 * m01 + m02 * m02 + m12 * m12 + 0.3f * (aB + cB) + 0.09f;
        const float c = cB + 0.3f;
        const float rD = 1.0f / sqrtf(D);
        u11 = sqrtf(kHalfLog2e / c);
        u00 = u11 * c * rD;
        u01 = -u11 * bB * rD;

        // ---- colour: real SH up to degree 3 at the unit direction camera -> mean
        float dx = d0 - cam.clo[0], dy = d1 - cam.clo[1], dz = d2 - cam.clo[2];
        float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
        float Y[16];
        sh_basis(dx * inv, dy * inv, dz * inv, Y);
        const int nf = 3 * (sc.sh_degree + 1) * (sc.sh_degree + 1);
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            if (4 * j >= nf) break;
            float4 v4 = __ldcs(ssh + (int64_t)j * npad + idx);
            float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int idx = 4 * j + cc;
                if (idx < nf) rgb[idx % 3] = fmaf(Y[idx / 3], vv[cc], rgb[idx % 3]);
            }
        }
    }

    if (threadIdx.x < 32) {
        uint32_t prefix = 0;
        if (tile != 0) {
            prefix = warp_lookback(status, tile, err);
            if (threadIdx.x == 0) st_volatile(status + tile, kStInc | (prefix + total));
        }
        if (threadIdx.x == 0) {
            s_prefix = prefix;
            if (tile == ntiles - 1) P.o.counts[0] = prefix + total;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_keys)
        atomicAdd(reinterpret_cast<unsigned long long*>(P.o.counts + 2), s_keys);
    if (threadIdx.x == 0 && s_bkeys)
        atomicAdd(reinterpret_cast<unsigned long long*>(P.o.counts + 4), s_bkeys);
    if (P.o.depth_hist && total) {
        for (int j = threadIdx.x; j < 4 * 256; j += kProjThreads) {
            const uint32_t c = (&s_dh[0][0])[j];
            if (c) atomicAdd(P.o.depth_hist + j, c);
        }
    }
    if (!vis) return;
    const uint32_t pos = s_prefix + excl;
    P.o.rec_a[pos] = make_float4(mxp, myp, u00, u01);
    // log2 of the opacity: compositing forms alpha as 2^(log2 o' - q)
    P.o.rec_b[pos] = make_float4(u11, log2f(o), fmaxf(rgb[0], 0.f), fmaxf(rgb[1], 0.f));
    P.o.rec_c[pos] = fmaxf(rgb[2], 0.f);
    P.o.rec_rect[pos] = make_uint2(pr0, pr1);   // pixel range
    P.o.rec_gid[pos] = g;
    P.o.depth_key[pos] = __float_as_uint(z);
    P.o.depth_val[pos] = pos;
}


// K10: tile-key counts of the greedy depth-threshold search (Sec. 3,
// "Selecting depth thresholds") for one view, for every candidate value of
// the threshold d_l at once.  With d_1 .. d_{l-1} fixed and levels above l
// unused, a level-(l-1) Gaussian is active for candidate x iff
// lo_{l-1} <= D < x^2 and a level-l Gaussian iff x^2 <= D (Eq. 2, D the
// pinned FP32 squared distance).  With m = #{k : thr_k <= D} (thr ascending)
// the first is active for candidates k >= m, the second for k < m, so each
// Gaussian adds its key count to one bucket and the per-candidate totals are
// prefix sums over buckets (done by the caller):
//   acc[0]          keys of levels < l-1 inside their fixed bands
//   acc[1 + m]      level l-1, active for candidates k >= m  (0 <= m < K)
//   acc[K + 1 + m]  level l, active for candidates k < m     (1 <= m <= K)
__global__ void __launch_bounds__(256)
threshold_cost_kernel(DevScene sc, DevCamera cam, int64_t n, int32_t lvl, ThreshBands b,
                      const float* __restrict__ thr, int32_t K, unsigned long long* __restrict__ acc) {
    extern __shared__ unsigned long long s_acc[];
    float* s_thr = reinterpret_cast<float*>(s_acc + (2 * K + 2));
    for (int i = threadIdx.x; i < 2 * K + 2; i += blockDim.x) s_acc[i] = 0ull;
    for (int i = threadIdx.x; i < K; i += blockDim.x) s_thr[i] = thr[i];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int j = 0;
        while (j + 1 < sc.num_levels && i >= sc.level_off[j + 1]) ++j;
        const float mxw = sc.mx[i], myw = sc.my[i], mzw = sc.mz[i];
        const float dx = __fsub_rn(mxw, b.c[0]);
        const float dy = __fsub_rn(myw, b.c[1]);
        const float dz = __fsub_rn(mzw, b.c[2]);
        const float D = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
        int slot;
        if (j < lvl - 1) {
            if (!(b.lo[j] <= D && D < b.hi[j])) continue;
            slot = 0;
        } else {
            if (j == lvl - 1 && !(b.lo[j] <= D)) continue;
            int lo = 0, hi = K;   // m = number of thresholds <= D
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (s_thr[mid] <= D) lo = mid + 1; else hi = mid;
            }
            const int m = lo;
            if (j == lvl - 1) {
                if (m == K) continue;
                slot = 1 + m;
            } else {
                if (m == 0) continue;
                slot = K + 1 + m;
            }
        }
        KeySplat ks;
        if (!key_splat(sc, cam, mxw, myw, mzw, sc.scale_op, sc.quat, i, (uint32_t)i, 1.f, ks)) continue;
        const unsigned long long tc =
            (unsigned long long)(ks.rx1 - ks.rx0 + 1) * (unsigned long long)(ks.ry1 - ks.ry0 + 1);
        atomicAdd(&s_acc[slot], tc);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * K + 2; i += blockDim.x)
        if (s_acc[i]) atomicAdd(acc + i, s_acc[i]);
}
}  // namespace

cudaError_t upload_qtable(const float* q65) {
    return cudaMemcpyToSymbol(c_qtable, q65, sizeof(float) * 65);
}

void launch_project(const DevScene& sc, const DevCamera& cam, const uint32_t* list,
                    int64_t n_active, float tA, float tB, const ProjectOut& o, uint32_t* status,
                    uint32_t* tile_counter, uint32_t* err, cudaStream_t s,
                    const ProjSources* src) {
    ProjParams P;
    P.sc = sc;
    P.cam = cam;
    P.list = list;
    P.n_active = n_active;
    P.n_pad = (sc.n_total + 63) / 64 * 64;
    P.tA = tA;
    P.tB = tB;
    P.o = o;
    if (src) P.src = *src;
    int64_t ntiles = (n_active + kProjThreads - 1) / kProjThreads;
    if (ntiles == 0) return;
    if (src)
        project_kernel<true><<<(unsigned)ntiles, kProjThreads, 0, s>>>(P, status, tile_counter, err);
    else
        project_kernel<false><<<(unsigned)ntiles, kProjThreads, 0, s>>>(P, status, tile_counter, err);
}

size_t threshold_cost_smem(int K) { return sizeof(unsigned long long) * (2 * K + 2) + sizeof(float) * K; }

void launch_threshold_cost(const DevScene& sc, const DevCamera& cam, int64_t n, int lvl,
                           const ThreshBands& b, const float* d_thr, int K, unsigned long long* acc,
                           cudaStream_t s) {
    if (n <= 0) return;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)device_sms() * 4);
    threshold_cost_kernel<<<grid, 256, threshold_cost_smem(K), s>>>(sc, cam, n, lvl, b, d_thr, K, acc);
}

}  // namespace lodge
