// Backward pass of the GES render for the joint optimisation stage (Sec. 4.2):
// gradients of L = sum(dL/dC * C) with respect to Gaussian position, rotation,
// scale, opacity and SH coefficients, and surfel SH coefficients (surfel
// geometry is fixed in that stage and gets none).
//
// Gaussians, gather form without atomics, in three launches: k_gbwd_rec sets
// every Gaussian up with the forward's device function (so the alpha and
// depth-test decisions are bit-identical) and keeps its record and what the
// chain rule needs; k_gbwd_sweep has each warp sweep its 32 Gaussians' pixel
// bboxes one Gaussian at a time, one pixel per lane (rows read coalesced),
// against per-pixel terms k_pixgrad prepared, and reduce the nine per-lane
// partial sums in a fixed order; k_gbwd_chain runs the chain rule per
// Gaussian.  (Sweeping each footprint in its own lane was measured slower:
// scattered rows, long dependent loops.)
// Surfels, scatter form: one thread per pixel adds its term to the winning
// surfel's sums in 64-bit fixed point (exact, so the order of the atomics
// does not matter), then one thread per surfel runs the SH chain.  Every sum
// has a fixed value, so the result is deterministic.
//
// Per (Gaussian i, pixel) that passes the clamp and the depth test, with
// k = 1/(1+W_G) (Eq. 5; 1/W_G in the Gaussians-only mode) and g = dL/dC:
//   dL/dc_i += alpha k g,  dL/dalpha = k g.(c_i - C),
//   alpha = sigma e^(-q/2):  dalpha/dsigma = e^(-q/2),  dalpha/dq = -alpha/2,
// then q -> (projected centre, conic) -> Sigma2 -> (Sigma3 -> s, r) and
// (Jacobian, centre -> p), and c_i -> SH and p through the view direction.
// Surfel s: dL/dc_s = sum over pixels won by s of k g, then SH.
//
// 2D Gaussians of 2D-GES (Sec. 6.4, Eq. 17-18) take the same three launches
// with their own per-pixel term and chain rule.  At a pixel whose ray d meets
// the splat plane at depth z = (N.t)/(N.d), X = z d - t = f1 a U + f2 b V
// (t the camera-space centre, U, V, N the frame, f_k = s_k S_k the filtered
// scales), alpha = sigma' exp(-(a^2 + b^2)/2), sigma' = sigma/(S1 S2).  With
// rho' = dL/d(a^2 + b^2) = -alpha dL/dalpha / 2, every hit gradient is a
// linear combination of seven moments, so the sweep sums those and the
// chain kernel combines them (U.d/N.d = (a f1 + U.t)/(N.t), likewise V):
//   sum rho' {a, b, a^2, ab, b^2, a r2, b r2},  r2 = a^2 + b^2,
// kept in units of the support radius r (a = r a_n), with dc and
// sum dL/dalpha alpha.  From the hit they pass through S1, S2 (functions of
// the Jacobian J = Jp(t) [s1 U, s2 V]) to t, U, V and s, then to position and
// rotation.
#include "ges_internal.cuh"

namespace ges {

namespace {

struct GLoop {
    float px, py, pxl, pyl, la, lb, lc, sigma, key, r, g, b;
    int x0, y0, x1, y1;
};

// Per pixel, what every Gaussian term there needs: P = (k g, k g.C) with
// k = 1/(1+W_G) (Eq. 5; 1/W_G in the Gaussians-only mode) and g = dL/dC.
// Pixels with W_G = 0 get zeros: no Gaussian contributes there.
__global__ void __launch_bounds__(256) k_pixgrad(int64_t HW, bool gmode, const float *__restrict__ dL,
                                                const float *__restrict__ rgb, const float *__restrict__ aux,
                                                float4 *__restrict__ P)
{
    const int64_t pix = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (pix >= HW) return;
    const float W = __ldg(aux + pix);
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (W > 0.f) {
        const float kk = gmode ? 1.f / W : 1.f / (1.f + W);
        const float g0 = __ldg(dL + pix), g1 = __ldg(dL + HW + pix), g2 = __ldg(dL + 2 * HW + pix);
        const float C0 = __ldg(rgb + pix), C1 = __ldg(rgb + HW + pix), C2 = __ldg(rgb + 2 * HW + pix);
        p = make_float4(kk * g0, kk * g1, kk * g2, kk * (g0 * C0 + g1 * C1 + g2 * C2));
    }
    P[pix] = p;
}

// One pixel of one Gaussian: add its 2D-level gradients to acc (dc(3),
// dsigma, dpx, dpy, dia, dib, dic).  Same alpha and depth test as the forward.
__device__ __forceinline__ void gauss_pixel(const GLoop &s, int x, int y, const CamParams &C, const OptParams &O,
                                            const float4 *__restrict__ P, const float *__restrict__ depth,
                                            float *acc)
{
    const int64_t pix = (int64_t)y * C.W + x;
    GaussRec g;
    g.px = s.px; g.py = s.py; g.pxl = s.pxl; g.pyl = s.pyl;
    g.la = s.la; g.lb = s.lb; g.lc = s.lc; g.sigma = s.sigma;
    float e;
    const float a = gauss_alpha(g, x + 0.5f, y + 0.5f, e);
    if (!(a >= O.alpha_min) || !(s.key < __ldg(depth + pix))) return;
    const float4 p = __ldg(P + pix);
    acc[0] += a * p.x;
    acc[1] += a * p.y;
    acc[2] += a * p.z;
    // dL/dalpha = k g.(c_i - C)
    const float dLda = fmaf(s.r, p.x, fmaf(s.g, p.y, s.b * p.z)) - p.w;
    acc[3] += dLda * e;
    const float dLdq = -0.5f * dLda * a;
    const float dx = (x + 0.5f - s.px) - s.pxl, dy = (y + 0.5f - s.py) - s.pyl;
    // dq/d(px, py) = -2 Sigma2^-1 (dx, dy), from the Cholesky form (accurate far
    // from the centre): Sigma2^-1 d = (a y0 + b y1, c y1) with the record's
    // factors scaled by kL, hence the 1/kL^2
    const float kL2 = 0.72134752044448170f;   // log2(e) / 2
    const float y0 = s.la * dx, y1 = fmaf(s.lb, dx, s.lc * dy);
    acc[4] += dLdq * -2.f * fmaf(s.la, y0, s.lb * y1) / kL2;
    acc[5] += dLdq * -2.f * (s.lc * y1) / kL2;
    acc[6] += dLdq * dx * dx;
    acc[7] += dLdq * 2.f * dx * dy;
    acc[8] += dLdq * dy * dy;
}

// One pixel of one 2D Gaussian: the forward's alpha, clamp and depth test
// from the disc record (r0..r2: forms of 1/z and of a/(r z), b/(r z) around
// the reference pixel; r3.w = eps; cl: the clamped colour and log2 sigma';
// side.w = log2(alpha_min / sigma')), then acc += dc(3), dL/dalpha alpha and
// the seven moments of rho' (a_n = a/r, b_n = b/r).
__device__ __forceinline__ void gauss2d_pixel(const float4 *q, int x, int y, const CamParams &C, const OptParams &O,
                                              const float4 *__restrict__ P, const float *__restrict__ depth,
                                              float *acc)
{
    const int64_t pix = (int64_t)y * C.W + x;
    const float4 r0 = q[0], r1 = q[1], r2 = q[2], r3 = q[3], cl = q[4], side = q[5];
    const float du = (x + 0.5f) - r0.x, dv = (y + 0.5f) - r0.y;
    const float iz = fmaf(r0.w, du, fmaf(r1.x, dv, r0.z));
    const float A = fmaf(r1.y, du, fmaf(r1.z, dv, r1.w));
    const float Bq = fmaf(r2.x, du, fmaf(r2.y, dv, r2.z));
    const float z = __frcp_rn(iz);
    const float rho = fmaf(A, A, Bq * Bq) * (z * z);
    const float a = ex2_approx(fmaf(side.w, rho, cl.w));
    if (!(iz > 0.f && iz < C.izn && z - r3.w < __ldg(depth + pix))) return;
    if (!(fminf(a * 4294967296.f, kAlpha32Max) >= O.alpha_min * 4294967296.f)) return;
    const float4 p = __ldg(P + pix);
    acc[0] += a * p.x;
    acc[1] += a * p.y;
    acc[2] += a * p.z;
    const float dLda = fmaf(cl.x, p.x, fmaf(cl.y, p.y, cl.z * p.z)) - p.w;
    acc[3] += dLda * a;
    const float rp = -0.5f * dLda * a;
    const float an = A * z, bn = Bq * z, r2n = fmaf(an, an, bn * bn);
    acc[4] += rp * an;
    acc[5] += rp * bn;
    acc[6] += rp * an * an;
    acc[7] += rp * an * bn;
    acc[8] += rp * bn * bn;
    acc[9] += rp * an * r2n;
    acc[10] += rp * bn * r2n;
}

// Gaussian backward in three launches.  k_gbwd_rec sets every Gaussian up
// with the forward's device function and stores its raster record (an empty
// bbox when it is not drawn).  k_gbwd_sweep: one thread per Gaussian, the
// warp sweeps its 32 Gaussians' pixel bboxes one Gaussian at a time (one
// pixel per lane, rows read coalesced) and reduces the per-lane partial sums
// with a fixed butterfly into the owning lane, which stores its 9 sums; this
// latency-bound loop runs light on registers, at full occupancy.
// k_gbwd_chain runs the chain rule per Gaussian from those sums (set-up
// recomputed).  The summation order is fixed, so the result is deterministic.
// What the chain rule needs of a Gaussian's set-up, kept by k_gbwd_rec as
// kChainWords structure-of-arrays words (word f of Gaussian i at f M + i) so
// that k_gbwd_chain does not set it up again.
constexpr int kChainWords = kBwdChainWords;
static_assert(kChainWords == 40, "chain words");
__device__ __forceinline__ void chain_put(const GaussOut &o, float *w, int64_t M, int64_t i)
{
    float v[kChainWords];
    int f = 0;
    for (int k = 0; k < 9; ++k) v[f++] = o.R[k];
    for (int k = 0; k < 4; ++k) v[f++] = o.qn[k];
    v[f++] = o.qnorm;
    for (int k = 0; k < 3; ++k) v[f++] = o.s[k];
    for (int k = 0; k < 3; ++k) v[f++] = o.se[k];
    v[f++] = o.k3; v[f++] = o.k2; v[f++] = o.sigma0;
    v[f++] = o.tx; v[f++] = o.ty; v[f++] = o.tz;
    v[f++] = o.ia; v[f++] = o.ib; v[f++] = o.ic;
    v[f++] = o.S2b; v[f++] = o.n0; v[f++] = o.n1; v[f++] = o.det0;
    for (int k = 0; k < 3; ++k) v[f++] = o.dir[k];
    v[f++] = o.dist;
    for (int k = 0; k < 3; ++k) v[f++] = o.raw[k];
    for (int k = 0; k < kChainWords; ++k) w[(int64_t)k * M + i] = v[k];
}
__device__ __forceinline__ void chain_get(GaussOut &o, const float *__restrict__ w, int64_t M, int64_t i)
{
    float v[kChainWords];
    for (int k = 0; k < kChainWords; ++k) v[k] = __ldg(w + (int64_t)k * M + i);
    int f = 0;
    for (int k = 0; k < 9; ++k) o.R[k] = v[f++];
    for (int k = 0; k < 4; ++k) o.qn[k] = v[f++];
    o.qnorm = v[f++];
    for (int k = 0; k < 3; ++k) o.s[k] = v[f++];
    for (int k = 0; k < 3; ++k) o.se[k] = v[f++];
    o.k3 = v[f++]; o.k2 = v[f++]; o.sigma0 = v[f++];
    o.tx = v[f++]; o.ty = v[f++]; o.tz = v[f++];
    o.ia = v[f++]; o.ib = v[f++]; o.ic = v[f++];
    o.S2b = v[f++]; o.n0 = v[f++]; o.n1 = v[f++]; o.det0 = v[f++];
    for (int k = 0; k < 3; ++k) o.dir[k] = v[f++];
    o.dist = v[f++];
    for (int k = 0; k < 3; ++k) o.raw[k] = v[f++];
    o.visible = true;
}

__global__ void __launch_bounds__(256) k_gbwd_rec(SceneView S, CamParams C, OptParams O, float4 *__restrict__ rec,
                                                 float *__restrict__ chain)
{
    const int64_t gi = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (gi >= S.M) return;
    GaussOut o;
    o.visible = false;
    if (O.mode != GES_MODE_SURFELS_ONLY) gauss_setup(S, C, O, gi, o);
    float4 *d = rec + 4 * gi;
    if (!o.visible) {
        // empty bbox: x0 = 1 > x1 = 0
        d[3] = make_float4(0.f, __uint_as_float(1u), __uint_as_float(0u), 0.f);
        return;
    }
    d[0] = make_float4(o.rec.px, o.rec.py, o.rec.pxl, o.rec.pyl);
    d[1] = make_float4(o.rec.la, o.rec.lb, o.rec.lc, o.rec.sigma);
    d[2] = make_float4(o.rec.key, o.rec.r, o.rec.g, o.rec.b);
    d[3] = make_float4(0.f, __uint_as_float(o.rec.bb_lo), __uint_as_float(o.rec.bb_hi), 0.f);
    chain_put(o, chain, S.M, gi);
}

// 2D Gaussians: what the chain rule needs, kChainWords2 words per Gaussian
// in the same structure-of-arrays layout.
constexpr int kChainWords2 = 30;
static_assert(kChainWords2 <= kBwdChainWords, "chain words");
__device__ __forceinline__ void chain2_put(const GaussOut &o, float *w, int64_t M, int64_t i)
{
    float v[kChainWords2];
    int f = 0;
    for (int k = 0; k < 9; ++k) v[f++] = o.R[k];
    for (int k = 0; k < 4; ++k) v[f++] = o.qn[k];
    v[f++] = o.qnorm;
    v[f++] = o.s[0]; v[f++] = o.s[1];
    v[f++] = o.S1; v[f++] = o.S2; v[f++] = o.rsup; v[f++] = o.sigma0;
    v[f++] = o.tx; v[f++] = o.ty; v[f++] = o.tz;
    for (int k = 0; k < 3; ++k) v[f++] = o.dir[k];
    v[f++] = o.dist;
    for (int k = 0; k < 3; ++k) v[f++] = o.raw[k];
    for (int k = 0; k < kChainWords2; ++k) w[(int64_t)k * M + i] = v[k];
}

__global__ void __launch_bounds__(256) k_gbwd_rec2(SceneView S, CamParams C, OptParams O, float4 *__restrict__ rec,
                                                  float *__restrict__ chain)
{
    const int64_t gi = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (gi >= S.M) return;
    GaussOut o;
    o.visible = false;
    if (O.mode != GES_MODE_SURFELS_ONLY) gauss2d_setup(S, C, O, gi, o);
    float4 *d = rec + 6 * gi;
    if (!o.visible) {
        d[3] = make_float4(0.f, __uint_as_float(1u), __uint_as_float(0u), 0.f);
        return;
    }
    const SurfelRec &r = o.drec;
    d[0] = make_float4(r.ur, r.vr, r.iz0, r.gu);
    d[1] = make_float4(r.gv, r.au, r.av, r.a0);
    d[2] = make_float4(r.bu, r.bv, r.b0, __int_as_float(r.id));
    d[3] = make_float4(r.izmax, __uint_as_float(r.bb_lo), __uint_as_float(r.bb_hi), r.pad);
    // float colours (the forward record carries them in 2^-16 units)
    d[4] = make_float4(fminf(o.rgb[0], kColourMax), fminf(o.rgb[1], kColourMax), fminf(o.rgb[2], kColourMax),
                       o.aux[0].w);
    d[5] = o.aux[1];
    chain2_put(o, chain, S.M, gi);
}

// kG 3: 4-quarter EWA records, 9 sums; kG 2: 6-quarter disc records (the
// record and its two side words), 11 sums.
template <int kG>
__global__ void __launch_bounds__(256, 4) k_gbwd_sweep(int64_t M, CamParams C, OptParams O,
                                                      const float4 *__restrict__ rec, const float4 *__restrict__ P,
                                                      const float *__restrict__ depth, float *__restrict__ sums)
{
    constexpr int kQ = kG == 2 ? 6 : 4, kNV = kG == 2 ? 11 : 9;
    const int64_t gi = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t g0 = gi - (threadIdx.x & 31);      // the warp's first Gaussian
    const int lane = threadIdx.x & 31;
    bool vis = false;
    if (gi < M) {
        const float4 r3 = __ldg(rec + kQ * gi + 3);
        const unsigned lo = __float_as_uint(r3.y), hi = __float_as_uint(r3.z);
        vis = (lo & 0xffff) <= (hi & 0xffff) && (lo >> 16) <= (hi >> 16);
    }
    if (gi < M && !vis)
        for (int c = 0; c < kNV; ++c) sums[(int64_t)c * M + gi] = 0.f;
    unsigned big = __ballot_sync(0xffffffffu, vis);
    while (big) {
        const int j = __ffs(big) - 1;
        big &= big - 1;
        // Gaussian g0 + j: every lane reads the same record (a broadcast, from L1)
        const float4 *rj = rec + kQ * (g0 + j);
        float4 q[kQ];
#pragma unroll
        for (int k = 0; k < kQ; ++k) q[k] = __ldg(rj + k);
        const unsigned lo = __float_as_uint(q[3].y), hi = __float_as_uint(q[3].z);
        const int x0 = lo & 0xffff, y0 = lo >> 16, x1 = hi & 0xffff, y1 = hi >> 16;
        GLoop t;
        if (kG == 3) {
            t.px = q[0].x; t.py = q[0].y; t.pxl = q[0].z; t.pyl = q[0].w;
            t.la = q[1].x; t.lb = q[1].y; t.lc = q[1].z; t.sigma = q[1].w;
            t.key = q[2].x; t.r = q[2].y; t.g = q[2].z; t.b = q[2].w;
            t.x0 = x0; t.y0 = y0; t.x1 = x1; t.y1 = y1;
        }
        const int w = x1 - x0 + 1, n = w * (y1 - y0 + 1);
        float part[kNV];
#pragma unroll
        for (int c = 0; c < kNV; ++c) part[c] = 0.f;
        // pixel k of the bbox, row-major (no integer division per pixel)
        const float iw = 1.f / (float)w;
        for (int k = lane; k < n; k += 32) {
            const int r = bbox_row(k, w, iw);
            if (kG == 2) gauss2d_pixel(q, x0 + (k - r * w), y0 + r, C, O, P, depth, part);
            else gauss_pixel(t, x0 + (k - r * w), y0 + r, C, O, P, depth, part);
        }
        float *dst = sums + g0 + j;
        warp_reduce_scatter<kNV>(part, lane, [&](int c, float tot) { dst[(int64_t)c * M] = tot; });
    }
}

// Colour -> SH coefficients (stored) and position through the view direction
// (added to gp).
__device__ __forceinline__ void colour_grad(const SceneView &S, int64_t gi, int K, const GaussOut &o,
                                            const float *dc, const ges_grads &G, float *gp)
{
    float Y[16];
    sh_basis(K, o.dir[0], o.dir[1], o.dir[2], Y);
    float gc[3];
    for (int c = 0; c < 3; ++c) gc[c] = o.raw[c] > 0.f ? dc[c] : 0.f;
    float gd[3] = {0.f, 0.f, 0.f};
    switch (K) {
    case 16: sh_weighted_grad<16>(S.g_sh, gi, S.sh_dtype, gc, o.dir, gd); break;
    case 9: sh_weighted_grad<9>(S.g_sh, gi, S.sh_dtype, gc, o.dir, gd); break;
    case 4: sh_weighted_grad<4>(S.g_sh, gi, S.sh_dtype, gc, o.dir, gd); break;
    default: break;   // degree 0: the colour does not depend on the direction
    }
    if (G.g_sh) store_sh_grad(G.g_sh + 3 * K * gi, K, Y, gc, nullptr);
    if (o.dist > 0.f) {
        const float pr = gd[0] * o.dir[0] + gd[1] * o.dir[1] + gd[2] * o.dir[2];
        for (int a = 0; a < 3; ++a) gp[a] -= (gd[a] - pr * o.dir[a]) / o.dist;
    }
}

// dL/dR (GR[a][b] = dL/dR_ab) -> R(qhat) -> qhat -> q (through the
// normalisation), stored as the four floats of g_rot[gi].
__device__ __forceinline__ void rot_grad(const float (*GR)[3], const GaussOut &o, float *g_rot, int64_t gi)
{
    const float w = o.qn[0], qx = o.qn[1], qy = o.qn[2], qz = o.qn[3];
    float gq[4];
    gq[0] = 2.f * (-qz * GR[0][1] + qy * GR[0][2] + qz * GR[1][0] - qx * GR[1][2] - qy * GR[2][0] + qx * GR[2][1]);
    gq[1] = 2.f * (qy * GR[0][1] + qz * GR[0][2] + qy * GR[1][0] - 2.f * qx * GR[1][1] - w * GR[1][2] +
                   qz * GR[2][0] + w * GR[2][1] - 2.f * qx * GR[2][2]);
    gq[2] = 2.f * (-2.f * qy * GR[0][0] + qx * GR[0][1] + w * GR[0][2] + qx * GR[1][0] + qz * GR[1][2] -
                   w * GR[2][0] + qz * GR[2][1] - 2.f * qy * GR[2][2]);
    gq[3] = 2.f * (-2.f * qz * GR[0][0] - w * GR[0][1] + qx * GR[0][2] + w * GR[1][0] - 2.f * qz * GR[1][1] +
                   qy * GR[1][2] + qx * GR[2][0] + qy * GR[2][1]);
    const float pr = gq[0] * w + gq[1] * qx + gq[2] * qy + gq[3] * qz;
    const float4 r4 = make_float4((gq[0] - pr * o.qn[0]) / o.qnorm, (gq[1] - pr * o.qn[1]) / o.qnorm,
                                  (gq[2] - pr * o.qn[2]) / o.qnorm, (gq[3] - pr * o.qn[3]) / o.qnorm);
    if ((reinterpret_cast<uintptr_t>(g_rot) & 15u) == 0) {
        reinterpret_cast<float4 *>(g_rot)[gi] = r4;
    } else {
        g_rot[4 * gi] = r4.x; g_rot[4 * gi + 1] = r4.y;
        g_rot[4 * gi + 2] = r4.z; g_rot[4 * gi + 3] = r4.w;
    }
}

__global__ void __launch_bounds__(256, 3) k_gbwd_chain(SceneView S, CamParams C, OptParams O,
                                                   const float *__restrict__ sums,
                                                   const float *__restrict__ chain, ges_grads G)
{
    const int64_t gi = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (gi >= S.M) return;
    const int K = (S.deg + 1) * (S.deg + 1);
    unsigned bits = 0u;
    for (int c = 0; c < 9; ++c) bits |= __float_as_uint(__ldg(sums + (int64_t)c * S.M + gi)) & 0x7fffffffu;
    const bool any = bits != 0u;
    // every gradient is linear in the nine sums: a Gaussian that passed the
    // cut and the depth test nowhere (not drawn, or hidden) gets zeros; the
    // others read what k_gbwd_rec kept of their set-up (nonzero sums imply
    // it was drawn)
    GaussOut o;
    o.visible = false;
    if (any && O.mode != GES_MODE_SURFELS_ONLY) chain_get(o, chain, S.M, gi);
    if (!o.visible) {
        if (G.g_pos) for (int a = 0; a < 3; ++a) G.g_pos[3 * gi + a] = 0.f;
        if (G.g_rot) for (int a = 0; a < 4; ++a) G.g_rot[4 * gi + a] = 0.f;
        if (G.g_scale) for (int a = 0; a < 3; ++a) G.g_scale[3 * gi + a] = 0.f;
        if (G.g_opac) G.g_opac[gi] = 0.f;
        if (G.g_sh) store_zeros(G.g_sh + 3 * K * gi, 3 * K);
        return;
    }
    float my[9];
    for (int c = 0; c < 9; ++c) my[c] = sums[(int64_t)c * S.M + gi];
    const float *dc = my;
    float gp[3] = {0.f, 0.f, 0.f};
    colour_grad(S, gi, K, o, dc, G, gp);
    // my[3] is dL/dsigma with sigma = sigma0 k3 k2 (the Mip-GES factors, 1 without them)
    if (G.g_opac) G.g_opac[gi] = my[3] * o.k3 * o.k2;
    // conic Q = Sigma2^-1:  dL/dSigma2 = -Q GQ Q with GQ = [[dia, dib/2], [dib/2, dic]]
    const float Q00 = o.ia, Q01 = o.ib, Q11 = o.ic;
    const float G00 = my[6], G01 = 0.5f * my[7], G11 = my[8];
    // M1 = GQ Q
    const float m00 = G00 * Q00 + G01 * Q01, m01 = G00 * Q01 + G01 * Q11;
    const float m10 = G01 * Q00 + G11 * Q01, m11 = G01 * Q01 + G11 * Q11;
    float S00 = -(Q00 * m00 + Q01 * m10), S01 = -(Q00 * m01 + Q01 * m11);
    float S11 = -(Q01 * m01 + Q11 * m11);
    // screen filter k2 = sqrt(det R2 / det Sigma2), Sigma2 = R2 + lowpass I:
    // dk2/dR2 = (k2/2) (R2^-1 - Sigma2^-1), and k2 R2^-1 = adj(R2) / sqrt(det R2 det Sigma2)
    if (O.filter == GES_FILTER_MIP && o.det0 > 0.f) {
        const float h = 0.5f * my[3] * o.sigma0 * o.k3;
        const float det = o.det0 + O.lowpass * (o.n0 + o.n1) + O.lowpass * O.lowpass;
        const float r = h / sqrtf(o.det0 * det), hk = h * o.k2;
        S00 += r * o.n1 - hk * Q00;
        S01 += -r * o.S2b - hk * Q01;
        S11 += r * o.n0 - hk * Q11;
    }
    const float GS2[2][2] = {{S00, S01}, {S01, S11}};
    // rebuild T = J Rc and Sigma3 = (R S)(R S)^T
    const float x = o.tx, y = o.ty, z = o.tz, iz = 1.f / z;
    const float J00 = C.fx * iz, J02 = -C.fx * x * iz * iz, J11 = C.fy * iz, J12 = -C.fy * y * iz * iz;
    float T[2][3], Mm[3][3], S3[3][3];
    for (int b = 0; b < 3; ++b) {
        T[0][b] = J00 * C.R[b] + J02 * C.R[6 + b];
        T[1][b] = J11 * C.R[3 + b] + J12 * C.R[6 + b];
    }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Mm[a][b] = o.R[3 * a + b] * o.se[b];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S3[a][b] = Mm[a][0] * Mm[b][0] + Mm[a][1] * Mm[b][1] + Mm[a][2] * Mm[b][2];
    // dL/dSigma3 = T^T GS2 T ; dL/dT = 2 GS2 T S3
    float GT2[2][3];   // GS2 T
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b) GT2[a][b] = GS2[a][0] * T[0][b] + GS2[a][1] * T[1][b];
    float GS3[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) GS3[a][b] = T[0][a] * GT2[0][b] + T[1][a] * GT2[1][b];
    float GT[2][3];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b)
            GT[a][b] = 2.f * (GT2[a][0] * S3[0][b] + GT2[a][1] * S3[1][b] + GT2[a][2] * S3[2][b]);
    // T = J Rc  ->  dL/dJ = GT Rc^T (only the non-zero entries of J matter)
    float GJ[2][3];
    for (int a = 0; a < 2; ++a)
        for (int k = 0; k < 3; ++k)
            GJ[a][k] = GT[a][0] * C.R[3 * k] + GT[a][1] * C.R[3 * k + 1] + GT[a][2] * C.R[3 * k + 2];
    const float dpx = my[4], dpy = my[5];
    float gt[3];
    gt[0] = GJ[0][2] * (-C.fx * iz * iz) + dpx * C.fx * iz;
    gt[1] = GJ[1][2] * (-C.fy * iz * iz) + dpy * C.fy * iz;
    gt[2] = GJ[0][0] * (-C.fx * iz * iz) + GJ[0][2] * (2.f * C.fx * x * iz * iz * iz) +
            GJ[1][1] * (-C.fy * iz * iz) + GJ[1][2] * (2.f * C.fy * y * iz * iz * iz) +
            dpx * (-C.fx * x * iz * iz) + dpy * (-C.fy * y * iz * iz);
    for (int a = 0; a < 3; ++a) gp[a] += C.R[a] * gt[0] + C.R[3 + a] * gt[1] + C.R[6 + a] * gt[2];
    if (G.g_pos) for (int a = 0; a < 3; ++a) G.g_pos[3 * gi + a] = gp[a];
    // Sigma3 = Mm Mm^T, Mm = R diag(se), se = sqrt(s^2 + v): dL/dMm = 2 GS3 Mm
    float GR[3][3];
    float gsc[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const float gm = 2.f * (GS3[a][0] * Mm[0][b] + GS3[a][1] * Mm[1][b] + GS3[a][2] * Mm[2][b]);
            gsc[b] += gm * o.R[3 * a + b];
            GR[a][b] = gm * o.se[b];
        }
    const float v3 = S.g_filt3 ? __ldg(S.g_filt3 + gi) : 0.f;
    if (v3 != 0.f) {
        // dse/ds = s/se; k3 = prod |s_j|/se_j: dk3/ds_j = k3 v / (s_j se_j^2)
        const float dk3 = my[3] * o.sigma0 * o.k2;
        for (int b = 0; b < 3; ++b) {
            gsc[b] *= o.s[b] / o.se[b];
            if (o.s[b] != 0.f) gsc[b] += dk3 * o.k3 * v3 / (o.s[b] * o.se[b] * o.se[b]);
        }
    }
    if (G.g_scale) for (int b = 0; b < 3; ++b) G.g_scale[3 * gi + b] = gsc[b];
    if (G.g_rot) rot_grad(GR, o, G.g_rot, gi);
}

// 2D Gaussians: the chain rule from the 11 sums of the sweep (dc, dL/dalpha
// alpha, the seven moments of rho') and the kept set-up words.
__global__ void __launch_bounds__(256, 3) k_gbwd_chain2(SceneView S, CamParams C, OptParams O,
                                                    const float *__restrict__ sums,
                                                    const float *__restrict__ chain, ges_grads G)
{
    const int64_t gi = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (gi >= S.M) return;
    const int K = (S.deg + 1) * (S.deg + 1);
    float my[11];
    unsigned bits = 0u;
    for (int c = 0; c < 11; ++c) {
        my[c] = __ldg(sums + (int64_t)c * S.M + gi);
        bits |= __float_as_uint(my[c]) & 0x7fffffffu;
    }
    if (bits == 0u || O.mode == GES_MODE_SURFELS_ONLY) {
        if (G.g_pos) for (int a = 0; a < 3; ++a) G.g_pos[3 * gi + a] = 0.f;
        if (G.g_rot) for (int a = 0; a < 4; ++a) G.g_rot[4 * gi + a] = 0.f;
        if (G.g_scale) for (int a = 0; a < 2; ++a) G.g_scale[2 * gi + a] = 0.f;
        if (G.g_opac) G.g_opac[gi] = 0.f;
        if (G.g_sh) store_zeros(G.g_sh + 3 * K * gi, 3 * K);
        return;
    }
    GaussOut o;
    float v[kChainWords2];
    for (int k = 0; k < kChainWords2; ++k) v[k] = __ldg(chain + (int64_t)k * S.M + gi);
    int f = 0;
    for (int k = 0; k < 9; ++k) o.R[k] = v[f++];
    for (int k = 0; k < 4; ++k) o.qn[k] = v[f++];
    o.qnorm = v[f++];
    const float s0 = v[f++], s1 = v[f++];
    const float S1 = v[f++], S2 = v[f++], r = v[f++], sigma0 = v[f++];
    const float x = v[f++], y = v[f++], z = v[f++];
    for (int k = 0; k < 3; ++k) o.dir[k] = v[f++];
    o.dist = v[f++];
    for (int k = 0; k < 3; ++k) o.raw[k] = v[f++];

    float gp[3] = {0.f, 0.f, 0.f};
    colour_grad(S, gi, K, o, my, G, gp);
    // sigma' = sigma0 / (S1 S2): dalpha/dsigma' = alpha / sigma'
    const float sigp = sigma0 / (S1 * S2);
    const float dsig = my[3] / sigp;
    if (G.g_opac) G.g_opac[gi] = dsig / (S1 * S2);
    // moments in filtered units (a = r a_n)
    const float r2 = r * r, r3 = r2 * r;
    const float Sa = r * my[4], Sb = r * my[5], Saa = r2 * my[6], Sab = r2 * my[7], Sbb = r2 * my[8];
    const float Sar = r3 * my[9], Sbr = r3 * my[10];
    // camera-space frame, as the set-up forms it
    float U[3], V[3], N[3];
    for (int q = 0; q < 3; ++q) {
        U[q] = C.R[3 * q] * o.R[0] + C.R[3 * q + 1] * o.R[3] + C.R[3 * q + 2] * o.R[6];
        V[q] = C.R[3 * q] * o.R[1] + C.R[3 * q + 1] * o.R[4] + C.R[3 * q + 2] * o.R[7];
        N[q] = C.R[3 * q] * o.R[2] + C.R[3 * q + 1] * o.R[5] + C.R[3 * q + 2] * o.R[8];
    }
    const float f1 = s0 * S1, f2 = s1 * S2;
    const float Ut = U[0] * x + U[1] * y + U[2] * z, Vt = V[0] * x + V[1] * y + V[2] * z;
    const float Nt = N[0] * x + N[1] * y + N[2] * z;
    const float cu = Ut / f1, cv = Vt / f2, k2 = 2.f / Nt;
    // sums of w = 2 rho' (a U.d/f1 + b V.d/f2) / N.d, and of w a, w b
    const float Sw = k2 * (Saa + Sbb + cu * Sa + cv * Sb);
    const float Swa = k2 * (Sar + cu * Saa + cv * Sab);
    const float Swb = k2 * (Sbr + cu * Sab + cv * Sbb);
    float gt[3], gU[3], gV[3], gN[3];
    for (int q = 0; q < 3; ++q) {
        gt[q] = N[q] * Sw - U[q] * (2.f * Sa / f1) - V[q] * (2.f * Sb / f2);
        gU[q] = 2.f * (Saa * U[q] + (f2 / f1) * Sab * V[q]);
        gV[q] = 2.f * ((f1 / f2) * Sab * U[q] + Sbb * V[q]);
        gN[q] = -(f1 * Swa * U[q] + f2 * Swb * V[q]);
    }
    const float gf1 = -2.f * Saa / f1, gf2 = -2.f * Sbb / f2;
    // f_k = s_k S_k and sigma' = sigma0 / (S1 S2)
    const float gS1 = gf1 * s0 - dsig * sigp / S1, gS2 = gf2 * s1 - dsig * sigp / S2;
    float gs0 = gf1 * S1, gs1 = gf2 * S2;
    // S1^2 = 1 + lowpass M11/det, S2^2 = 1 + lowpass M00/det with M = J^T J,
    // J = Jp(t) [s1 U, s2 V]; in the ratios p1 = M11/det, p2 = M00/det, m = M01/det
    const float iz = 1.f / z;
    const float j00 = C.fx * iz, j02 = -C.fx * x * iz * iz, j11 = C.fy * iz, j12 = -C.fy * y * iz * iz;
    const float JU0 = j00 * U[0] + j02 * U[2], JU1 = j11 * U[1] + j12 * U[2];
    const float JV0 = j00 * V[0] + j02 * V[2], JV1 = j11 * V[1] + j12 * V[2];
    const float J00 = s0 * JU0, J01 = s1 * JV0, J10 = s0 * JU1, J11 = s1 * JV1;
    const float dJ = J00 * J11 - J01 * J10;
    const float idet = 1.f / (dJ * dJ);
    const float M00 = J00 * J00 + J10 * J10, M11 = J01 * J01 + J11 * J11, M01 = J00 * J01 + J10 * J11;
    const float p1 = M11 * idet, p2 = M00 * idet, m = M01 * idet;
    const float h1 = gS1 * O.lowpass / (2.f * S1), h2 = gS2 * O.lowpass / (2.f * S2);
    const float gM00 = -h1 * p1 * p1 - h2 * m * m;
    const float gM11 = -h1 * m * m - h2 * p2 * p2;
    const float gM01 = 2.f * m * (h1 * p1 + h2 * p2);
    const float gJ00 = 2.f * J00 * gM00 + J01 * gM01, gJ10 = 2.f * J10 * gM00 + J11 * gM01;
    const float gJ01 = J00 * gM01 + 2.f * J01 * gM11, gJ11 = J10 * gM01 + 2.f * J11 * gM11;
    gs0 += gJ00 * JU0 + gJ10 * JU1;
    gs1 += gJ01 * JV0 + gJ11 * JV1;
    gU[0] += s0 * gJ00 * j00; gU[1] += s0 * gJ10 * j11; gU[2] += s0 * (gJ00 * j02 + gJ10 * j12);
    gV[0] += s1 * gJ01 * j00; gV[1] += s1 * gJ11 * j11; gV[2] += s1 * (gJ01 * j02 + gJ11 * j12);
    // Jp(t) -> t: dL/dJp row a = s1 gJ_a0 U + s2 gJ_a1 V (the non-zero entries)
    const float gj00 = s0 * gJ00 * U[0] + s1 * gJ01 * V[0], gj02 = s0 * gJ00 * U[2] + s1 * gJ01 * V[2];
    const float gj11 = s0 * gJ10 * U[1] + s1 * gJ11 * V[1], gj12 = s0 * gJ10 * U[2] + s1 * gJ11 * V[2];
    gt[0] += gj02 * (-C.fx * iz * iz);
    gt[1] += gj12 * (-C.fy * iz * iz);
    gt[2] += gj00 * (-C.fx * iz * iz) + gj02 * (2.f * C.fx * x * iz * iz * iz) + gj11 * (-C.fy * iz * iz) +
             gj12 * (2.f * C.fy * y * iz * iz * iz);
    if (G.g_scale) { G.g_scale[2 * gi] = gs0; G.g_scale[2 * gi + 1] = gs1; }
    // t = Rc p + tc; U, V, N = Rc R e_k: world gradients through Rc^T
    float GR[3][3];
    for (int a = 0; a < 3; ++a) {
        gp[a] += C.R[a] * gt[0] + C.R[3 + a] * gt[1] + C.R[6 + a] * gt[2];
        GR[a][0] = C.R[a] * gU[0] + C.R[3 + a] * gU[1] + C.R[6 + a] * gU[2];
        GR[a][1] = C.R[a] * gV[0] + C.R[3 + a] * gV[1] + C.R[6 + a] * gV[2];
        GR[a][2] = C.R[a] * gN[0] + C.R[3 + a] * gN[1] + C.R[6 + a] * gN[2];
    }
    if (G.g_pos) for (int a = 0; a < 3; ++a) G.g_pos[3 * gi + a] = gp[a];
    if (G.g_rot) rot_grad(GR, o, G.g_rot, gi);
}

// largest |x| (non-negative floats order like their bit patterns)
__global__ void __launch_bounds__(256) k_absmax(const float *__restrict__ x, int64_t n, unsigned *out)
{
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
    for (int d = 16; d >= 1; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}

// Surfel colour gradients, scatter form: dL/dc_s = sum over the samples s won
// of k g / samples (k = 1/(1+W_G), or 1 with surfels only).  One thread per
// pixel adds the term of each distinct winner among its samples to that
// surfel's three sums, in 64-bit fixed point (units of gmax 2^-30, so one
// term stays within 2^30): integer sums are exact, so the result does not
// depend on the order of the atomics.
__global__ void __launch_bounds__(256) k_surfel_scatter(int64_t N, CamParams C, OptParams O,
                                                       const float *__restrict__ dL, const int32_t *__restrict__ sid,
                                                       const float *__restrict__ aux,
                                                       const unsigned *__restrict__ gmax_bits, long long *acc)
{
    const int64_t HW = (int64_t)C.W * C.H;
    const int64_t pix = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (pix >= HW) return;
    const float gmax = __uint_as_float(*gmax_bits);
    if (!(gmax > 0.f)) return;
    const float g[3] = {__ldg(dL + pix), __ldg(dL + HW + pix), __ldg(dL + 2 * HW + pix)};
    if (g[0] == 0.f && g[1] == 0.f && g[2] == 0.f) return;
    const float scale = 1073741824.f / gmax;   // 2^30 / max |dL/dC|
    const bool full = O.mode == GES_MODE_FULL;
    int32_t w[4];
    for (int q = 0; q < O.samples; ++q) w[q] = __ldg(sid + q * HW + pix);
    for (int q = 0; q < O.samples; ++q) {
        const int32_t s = w[q];
        if (s < 0 || (int64_t)s >= N) continue;
        bool seen = false;
        for (int r = 0; r < q; ++r) seen |= w[r] == s;
        if (seen) continue;
        // with 4 samples each won sample carries a quarter of the pixel
        int won = 0;
        for (int r = 0; r < O.samples; ++r) won += w[r] == s;
        const float kk = (full ? 1.f / (1.f + __ldg(aux + pix)) : 1.f) * (float)won / (float)O.samples;
        unsigned long long *a = reinterpret_cast<unsigned long long *>(acc + 3 * (int64_t)s);
        for (int c = 0; c < 3; ++c) {
            const long long v = f2ll_rn(kk * g[c] * scale);   // |v| <= 2^30
            if (v != 0) atomicAdd(a + c, (unsigned long long)v);
        }
    }
}

// Per surfel: the colour sums -> SH coefficients through Eq. 1 (zero where
// the unclamped colour is not positive).  The view direction and the colour
// are recomputed with the forward's functions, so the clamp gate is the
// forward's.  A surfel that won no sample gets zeros.
__global__ void __launch_bounds__(256) k_surfel_sh(SceneView S, CamParams C, const long long *__restrict__ acc,
                                                  const unsigned *__restrict__ gmax_bits, float *__restrict__ g_sh)
{
    const int64_t si = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (si >= S.N) return;
    const int K = (S.deg + 1) * (S.deg + 1);
    float *out = g_sh + (int64_t)3 * K * si;
    const long long a0 = acc[3 * si], a1 = acc[3 * si + 1], a2 = acc[3 * si + 2];
    if (a0 == 0 && a1 == 0 && a2 == 0) {
        store_zeros(out, 3 * K);
        return;
    }
    const float unit = __uint_as_float(*gmax_bits) * 9.31322574615478516e-10f;   // gmax 2^-30
    const float gc[3] = {__ll2float_rn(a0) * unit, __ll2float_rn(a1) * unit, __ll2float_rn(a2) * unit};
    float dir[3], L, Y[16], rgb[3], raw[3];
    view_dir(C, __ldg(S.s_pos + 3 * si), __ldg(S.s_pos + 3 * si + 1), __ldg(S.s_pos + 3 * si + 2), dir, L);
    sh_basis(K, dir[0], dir[1], dir[2], Y);
    sh_colour(S.s_sh, si, K, S.sh_dtype, Y, rgb, raw);
    store_sh_grad(out, K, Y, gc, raw);
}

}  // namespace

cudaError_t launch_absmax(const float *x, int64_t n, unsigned *out, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned), st);
    if (e != cudaSuccess || n <= 0) return e;
    k_absmax<<<152 * 4, 256, 0, st>>>(x, n, out);
    return cudaGetLastError();
}

cudaError_t launch_backward(const SceneView &S, const CamParams &C, const OptParams &O, const float *dL_drgb,
                            const float *out_rgb, const float *out_depth, const int32_t *surfel_id,
                            const float *aux, const ges_grads &G, long long *s_acc, unsigned *gmax,
                            float4 *pixg, float4 *g_rec, float *g_sums, float *g_chain, cudaStream_t st,
                            cudaEvent_t *ev)
{
    if (ev) cudaEventRecord(ev[0], st);
    if (S.M > 0) {
        const int64_t HW = (int64_t)C.W * C.H;
        k_pixgrad<<<(unsigned)((HW + 255) / 256), 256, 0, st>>>(HW, O.mode == GES_MODE_GAUSSIANS_ONLY, dL_drgb,
                                                                out_rgb, aux, pixg);
        const unsigned nb = (unsigned)((S.M + 255) / 256);
        if (S.gdim == 2) {
            k_gbwd_rec2<<<nb, 256, 0, st>>>(S, C, O, g_rec, g_chain);
            k_gbwd_sweep<2><<<nb, 256, 0, st>>>(S.M, C, O, g_rec, pixg, out_depth, g_sums);
            k_gbwd_chain2<<<nb, 256, 0, st>>>(S, C, O, g_sums, g_chain, G);
        } else {
            k_gbwd_rec<<<nb, 256, 0, st>>>(S, C, O, g_rec, g_chain);
            k_gbwd_sweep<3><<<nb, 256, 0, st>>>(S.M, C, O, g_rec, pixg, out_depth, g_sums);
            k_gbwd_chain<<<nb, 256, 0, st>>>(S, C, O, g_sums, g_chain, G);
        }
    }
    if (ev) cudaEventRecord(ev[1], st);
    if (S.N > 0 && G.s_sh) {
        cudaError_t e = cudaMemsetAsync(s_acc, 0, sizeof(long long) * 3 * (size_t)S.N, st);
        if (e != cudaSuccess) return e;
        const int64_t HW = (int64_t)C.W * C.H;
        if ((e = launch_absmax(dL_drgb, 3 * HW, gmax, st)) != cudaSuccess) return e;
        if (O.mode != GES_MODE_GAUSSIANS_ONLY)
            k_surfel_scatter<<<(unsigned)((HW + 255) / 256), 256, 0, st>>>(S.N, C, O, dL_drgb, surfel_id, aux, gmax,
                                                                           s_acc);
        k_surfel_sh<<<(unsigned)((S.N + 255) / 256), 256, 0, st>>>(S, C, s_acc, gmax, G.s_sh);
    }
    if (ev) cudaEventRecord(ev[2], st);
    return cudaGetLastError();
}

}  // namespace ges
