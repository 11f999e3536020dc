// Backward pass of the GES render for the joint optimisation stage (Sec. 4.2):
// gradients of L = sum(dL/dC * C) with respect to Gaussian position, rotation,
// scale, opacity and SH coefficients, and surfel SH coefficients (surfel
// geometry is fixed in that stage and gets none).
//
// Gather form, no atomics: one thread per primitive.  Each thread sets its
// primitive up with the same device function as the forward pass (so the alpha
// and depth-test decisions are bit-identical); then the warp sweeps its 32
// primitives' pixel bboxes one primitive at a time, one pixel per lane (rows
// read coalesced), and reduces the per-lane partial sums with a fixed
// butterfly into the owning lane.  Finally each thread runs the chain rule for
// its own primitive.  The summation order is fixed, so the result is
// deterministic.  (Sweeping each footprint in its own lane was measured slower:
// scattered rows, long dependent loops.)
//
// Per (Gaussian i, pixel) that passes the clamp and the depth test, with
// k = 1/(1+W_G) (Eq. 5; 1/W_G in the Gaussians-only mode) and g = dL/dC:
//   dL/dc_i += alpha k g,  dL/dalpha = k g.(c_i - C),
//   alpha = sigma e^(-q/2):  dalpha/dsigma = e^(-q/2),  dalpha/dq = -alpha/2,
// then q -> (projected centre, conic) -> Sigma2 -> (Sigma3 -> s, r) and
// (Jacobian, centre -> p), and c_i -> SH and p through the view direction.
// Surfel s: dL/dc_s = sum over pixels won by s of k g, then SH.
#include "ges_internal.cuh"

namespace ges {

namespace {

__device__ __forceinline__ float warp_sum(float x)
{
    for (int d = 16; d >= 1; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    return x;
}


struct GLoop {
    float px, py, pxl, pyl, la, lb, lc, sigma, key, r, g, b, ia, ib, ic;
    int x0, y0, x1, y1;
};

// One pixel of one Gaussian: add its 2D-level gradients to acc (dc(3),
// dsigma, dpx, dpy, dia, dib, dic).  Same alpha and depth test as the forward.
__device__ __forceinline__ void gauss_pixel(const GLoop &s, int x, int y, const CamParams &C, const OptParams &O,
                                            bool gmode, const float *__restrict__ dL,
                                            const float *__restrict__ rgb, const float *__restrict__ depth,
                                            const float *__restrict__ aux, float *acc)
{
    const int64_t HW = (int64_t)C.W * C.H, pix = (int64_t)y * C.W + x;
    GaussRec g;
    g.px = s.px; g.py = s.py; g.pxl = s.pxl; g.pyl = s.pyl;
    g.la = s.la; g.lb = s.lb; g.lc = s.lc; g.sigma = s.sigma;
    float e;
    const float a = gauss_alpha(g, x + 0.5f, y + 0.5f, e);
    if (!(a >= O.alpha_min) || !(s.key < __ldg(depth + pix))) return;
    const float W = __ldg(aux + pix);
    const float kk = gmode ? 1.f / W : 1.f / (1.f + W);
    const float g0 = __ldg(dL + pix), g1 = __ldg(dL + HW + pix), g2 = __ldg(dL + 2 * HW + pix);
    const float C0 = __ldg(rgb + pix), C1 = __ldg(rgb + HW + pix), C2 = __ldg(rgb + 2 * HW + pix);
    acc[0] += a * kk * g0;
    acc[1] += a * kk * g1;
    acc[2] += a * kk * g2;
    const float dLda = kk * (g0 * (s.r - C0) + g1 * (s.g - C1) + g2 * (s.b - C2));
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

__device__ __forceinline__ float shfl_f(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ int shfl_i(int v, int src) { return __shfl_sync(0xffffffffu, v, src); }

__global__ void __launch_bounds__(256) k_gauss_bwd(SceneView S, CamParams C, OptParams O,
                                                  const float *__restrict__ dL, const float *__restrict__ rgb,
                                                  const float *__restrict__ depth, const float *__restrict__ aux,
                                                  ges_grads G)
{
    const int64_t gi = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool gmode = O.mode == GES_MODE_GAUSSIANS_ONLY;
    // 1) set-up (the forward's definition), keep only what the sweep needs
    GLoop s;
    bool vis = false;
    if (gi < S.M && O.mode != GES_MODE_SURFELS_ONLY) {
        GaussOut o;
        gauss_setup(S, C, O, gi, o);
        vis = o.visible;
        if (vis) {
            s = GLoop{o.rec.px, o.rec.py, o.rec.pxl, o.rec.pyl, o.rec.la, o.rec.lb, o.rec.lc, o.rec.sigma,
                      o.rec.key, o.rec.r, o.rec.g, o.rec.b, o.ia, o.ib, o.ic, o.x0, o.y0, o.x1, o.y1};
        }
    }
    float acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    // 2) the whole warp sweeps one Gaussian's pixels at a time (rows are read
    //    coalesced), then reduces with a fixed butterfly
    unsigned big = __ballot_sync(0xffffffffu, vis);
    while (big) {
        const int j = __ffs(big) - 1;
        big &= big - 1;
        GLoop t;
        t.px = shfl_f(s.px, j); t.py = shfl_f(s.py, j); t.pxl = shfl_f(s.pxl, j); t.pyl = shfl_f(s.pyl, j);
        t.la = shfl_f(s.la, j); t.lb = shfl_f(s.lb, j); t.lc = shfl_f(s.lc, j); t.sigma = shfl_f(s.sigma, j);
        t.key = shfl_f(s.key, j); t.r = shfl_f(s.r, j); t.g = shfl_f(s.g, j); t.b = shfl_f(s.b, j);
        t.ia = shfl_f(s.ia, j); t.ib = shfl_f(s.ib, j); t.ic = shfl_f(s.ic, j);
        t.x0 = shfl_i(s.x0, j); t.y0 = shfl_i(s.y0, j); t.x1 = shfl_i(s.x1, j); t.y1 = shfl_i(s.y1, j);
        const int w = t.x1 - t.x0 + 1, n = w * (t.y1 - t.y0 + 1);
        float part[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = lane; k < n; k += 32) gauss_pixel(t, t.x0 + k % w, t.y0 + k / w, C, O, gmode, dL, rgb, depth, aux, part);
        for (int c = 0; c < 9; ++c) {
            const float v = warp_sum(part[c]);
            if (lane == j) acc[c] = v;
        }
    }
    if (gi >= S.M) return;
    const int K = (S.deg + 1) * (S.deg + 1);
    // 3) chain rule for this lane's Gaussian (set-up recomputed: fewer live registers in the sweep)
    GaussOut o;
    o.visible = false;
    if (vis) gauss_setup(S, C, O, gi, o);
    if (!o.visible) {
        if (G.g_pos) for (int a = 0; a < 3; ++a) G.g_pos[3 * gi + a] = 0.f;
        if (G.g_rot) for (int a = 0; a < 4; ++a) G.g_rot[4 * gi + a] = 0.f;
        if (G.g_scale) for (int a = 0; a < 3; ++a) G.g_scale[3 * gi + a] = 0.f;
        if (G.g_opac) G.g_opac[gi] = 0.f;
        if (G.g_sh) for (int a = 0; a < 3 * K; ++a) G.g_sh[3 * K * gi + a] = 0.f;
        return;
    }
    const float *my = acc;
    const float *dc = my;
    float gp[3] = {0.f, 0.f, 0.f};
    // colour -> SH coefficients and position (through the view direction)
    {
        float Y[16], dY[16][3];
        sh_basis(K, o.dir[0], o.dir[1], o.dir[2], Y);
        sh_basis_grad(K, o.dir[0], o.dir[1], o.dir[2], dY);
        float gc[3];
        for (int c = 0; c < 3; ++c) gc[c] = o.raw[c] > 0.f ? dc[c] : 0.f;
        float gd[3] = {0.f, 0.f, 0.f};
        for (int k = 0; k < K; ++k) {
            float sh[3];
            for (int c = 0; c < 3; ++c) sh[c] = load_attr(S.g_sh, 3 * K * gi + 3 * k + c, S.sh_dtype);
            if (G.g_sh) for (int c = 0; c < 3; ++c) G.g_sh[3 * K * gi + 3 * k + c] = Y[k] * gc[c];
            const float w = sh[0] * gc[0] + sh[1] * gc[1] + sh[2] * gc[2];
            for (int a = 0; a < 3; ++a) gd[a] += w * dY[k][a];
        }
        if (o.dist > 0.f) {
            const float pr = gd[0] * o.dir[0] + gd[1] * o.dir[1] + gd[2] * o.dir[2];
            for (int a = 0; a < 3; ++a) gp[a] -= (gd[a] - pr * o.dir[a]) / o.dist;
        }
    }
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
    // R(qhat) -> qhat -> q (through the normalisation)
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
    if (G.g_rot)
        for (int a = 0; a < 4; ++a) G.g_rot[4 * gi + a] = (gq[a] - pr * o.qn[a]) / o.qnorm;
}

__global__ void __launch_bounds__(256) k_surfel_bwd(SceneView S, CamParams C, OptParams O,
                                                   const float *__restrict__ dL, const int32_t *__restrict__ sid,
                                                   const float *__restrict__ aux, float *__restrict__ g_sh)
{
    const int64_t si = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int64_t HW = (int64_t)C.W * C.H;
    const bool full = O.mode == GES_MODE_FULL;
    SurfelOut o;
    o.visible = false;
    if (si < S.N && O.mode != GES_MODE_GAUSSIANS_ONLY) surfel_setup(S, C, O, si, o);
    const bool vis = o.visible;
    int x0 = 0, y0 = 0, x1 = -1, y1 = -1;
    if (vis) { x0 = o.x0; y0 = o.y0; x1 = o.x1; y1 = o.y1; }
    float acc[3] = {0.f, 0.f, 0.f};
    // dL/dc_s = sum over the samples s won of k g / samples (k = 1/(1+W_G),
    // or 1 with surfels only); the warp sweeps one surfel's bbox at a time
    unsigned big = __ballot_sync(0xffffffffu, vis);
    while (big) {
        const int j = __ffs(big) - 1;
        big &= big - 1;
        const int bx0 = shfl_i(x0, j), by0 = shfl_i(y0, j), bx1 = shfl_i(x1, j), by1 = shfl_i(y1, j);
        const int32_t want = (int32_t)(si - lane + j);
        const int w = bx1 - bx0 + 1, n = w * (by1 - by0 + 1);
        float part[3] = {0.f, 0.f, 0.f};
        for (int k = lane; k < n; k += 32) {
            const int64_t pix = (int64_t)(by0 + k / w) * C.W + bx0 + k % w;
            // with 4 samples each won sample carries a quarter of the pixel
            int won = 0;
            for (int q = 0; q < O.samples; ++q) won += __ldg(sid + q * HW + pix) == want;
            if (won == 0) continue;
            const float kk = (full ? 1.f / (1.f + __ldg(aux + pix)) : 1.f) * (float)won / (float)O.samples;
            part[0] += kk * __ldg(dL + pix);
            part[1] += kk * __ldg(dL + HW + pix);
            part[2] += kk * __ldg(dL + 2 * HW + pix);
        }
        for (int c = 0; c < 3; ++c) {
            const float v = warp_sum(part[c]);
            if (lane == j) acc[c] = v;
        }
    }
    if (si >= S.N) return;
    const int K = (S.deg + 1) * (S.deg + 1);
    float *out = g_sh + (int64_t)3 * K * si;
    if (!vis) {
        for (int a = 0; a < 3 * K; ++a) out[a] = 0.f;
        return;
    }
    float Y[16];
    sh_basis(K, o.dir[0], o.dir[1], o.dir[2], Y);
    for (int k = 0; k < K; ++k)
        for (int c = 0; c < 3; ++c) out[3 * k + c] = o.raw[c] > 0.f ? Y[k] * acc[c] : 0.f;
}

}  // namespace

cudaError_t launch_backward(const SceneView &S, const CamParams &C, const OptParams &O, const float *dL_drgb,
                            const float *out_rgb, const float *out_depth, const int32_t *surfel_id,
                            const float *aux, const ges_grads &G, unsigned *status, cudaStream_t st,
                            cudaEvent_t *ev)
{
    (void)status;
    if (ev) cudaEventRecord(ev[0], st);
    if (S.M > 0)
        k_gauss_bwd<<<(unsigned)((S.M + 255) / 256), 256, 0, st>>>(S, C, O, dL_drgb, out_rgb, out_depth, aux, G);
    if (ev) cudaEventRecord(ev[1], st);
    if (S.N > 0 && G.s_sh)
        k_surfel_bwd<<<(unsigned)((S.N + 255) / 256), 256, 0, st>>>(S, C, O, dL_drgb, surfel_id, aux, G.s_sh);
    if (ev) cudaEventRecord(ev[2], st);
    return cudaGetLastError();
}

}  // namespace ges
