/*
 * FP64 reference ("oracle") of the Gaussian-enhanced Surfels (GES) render.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline of the benchmark call this code.  It shares nothing with the CUDA
 * path: no headers, no helpers, no constants.  It is deliberately plain: every
 * pixel is evaluated straight from the paper's definitions in double
 * precision, with no blocking, fusion or reordering beyond skipping pixels
 * that lie outside a primitive's conservative screen rectangle (found through
 * 16x16-pixel cell lists kept in ascending primitive index).
 *
 * What it follows:
 *   Sec. 3        surfel = opaque disc in its local XY plane, placed by scale,
 *                 rotation, translation; colour = SH at the direction from the
 *                 surfel centre to the camera (Eq. 1).
 *   Sec. 4.1      opaque extent: G(x,y) >= 1/255, i.e. x^2+y^2 <= 2 ln 255
 *                 (Eq. 6-7 with w_i = 255).
 *   Sec. 3        pass 1: per-pixel z-buffer of surfel fragments -> C_s, D_s.
 *   Sec. 3        pass 2: C_G, W_G accumulated over Gaussians passing the
 *                 depth test d_i < D_s + eps (Eq. 2-3) with the 2D opacity of
 *                 Eq. 4, clamped to zero below 1/255.
 *   Sec. 3        composite C = (C_s W_s + C_G)/(W_s + W_G), W_s = 1 (Eq. 5).
 *   Sec. 5        eps_i = (5/D) sum_j s_ij with D = 3.
 *   Sec. 7 (ablation) "only surfels" C = C_s, "only Gaussians" C = C_G/W_G.
 *   Sec. 4.1, 5   4x supersampling of the surfel pass (a render at twice the
 *                 resolution, downsampled), done as 4x multisampling in the
 *                 OpenGL renderer; the Gaussians are not multisampled.
 *   Sec. 4.2      joint stage: gradients w.r.t. Gaussian p, s, r, sigma, SH
 *                 and surfel SH, surfel geometry fixed.
 * Readings where the paper is silent (camera model, SH basis, low-pass filter,
 * tie-break, pixel centres) are the ones listed in the design notes; the
 * comments at each use restate them.
 *
 * Parity status: every function below is pinned by the CPU tests against
 * closed forms, library routines, invariants, brute force or finite
 * differences; nothing here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n_surfels, n_gaussians;
    int32_t sh_degree;
    const double *s_pos, *s_rot, *s_scale, *s_sh;            /* [N,3] [N,4] [N,2] [N,K,3] */
    const double *g_pos, *g_rot, *g_scale, *g_opac, *g_sh;   /* [M,3] [M,4] [M,3] [M] [M,K,3] */
    const double *g_filt3;   /* [M] Mip-GES 3D filter variance (world units^2), NULL: none */
    int32_t gauss_dim;       /* 3 (or 0): 3D Gaussians, g_scale [M,3];
                                2: 2D Gaussians of 2D-GES (Sec. 6.4), g_scale [M,2] */
} ora_scene;

typedef struct {
    int32_t width, height;
    double fx, fy, cx, cy;
    double w2c[12];      /* row-major [R|t], world -> camera */
    double znear;
    double bg[3];
} ora_camera;

typedef struct {
    int32_t eps_mode;    /* 0: eps_i = eps_factor/3 * (s1+s2+s3); 1: 0; 2: eps_value */
    double eps_value, eps_factor, lowpass, alpha_min, surfel_r2;
    int32_t mode;        /* 0 full, 1 surfels only, 2 Gaussians only */
    /* ambiguity bands (pixels where several results are correct) */
    double tol_depth_rel, tol_disc_rel, tol_graze, tol_alpha, tol_gdepth_rel;
    int32_t samples;     /* 1: the pixel centre; 4: 4x multisampling of the surfel pass (Sec. 5) */
    int32_t filter;      /* 0: fixed EWA dilation Sigma2 + lowpass I (3DGS, basic GES);
                            1: Mip-GES screen filter: the same dilation with the opacity
                               scaled by sqrt(|Sigma2| / |Sigma2 + lowpass I|) (Sec. 6.1) */
    double tol_disc_graze;   /* rim band at a fragment whose ray meets the disc at cosine c:
                                tol_disc_rel (1 + tol_disc_graze / max(|c|, tol_graze)) */
    double tol_centre_rel;   /* translucent blend order: two surfel centres' camera depths
                                closer than this (relative) may be ordered either way */
} ora_opts;

enum { ORA_OK = 0, ORA_BAD_ARG = 1, ORA_BAD_QUAT = 2, ORA_NOMEM = 3 };
enum { AMB_ID = 1, AMB_COLOR = 2 };

/* ------------------------------------------------------------------------ */
/* small linear algebra                                                      */

static double dot3(const double *a, const double *b) { return a[0]*b[0] + a[1]*b[1] + a[2]*b[2]; }

static void matvec3(const double *M /*3x3 rm*/, const double *v, double *out)
{
    for (int i = 0; i < 3; ++i) out[i] = M[3*i]*v[0] + M[3*i+1]*v[1] + M[3*i+2]*v[2];
}

/* rotation matrix of the normalised quaternion (w,x,y,z) */
static int quat_rot(const double *q, double *R, double *qn, double *norm)
{
    double n = sqrt(q[0]*q[0] + q[1]*q[1] + q[2]*q[2] + q[3]*q[3]);
    if (!(n > 0.0) || !isfinite(n)) return 0;
    double w = q[0]/n, x = q[1]/n, y = q[2]/n, z = q[3]/n;
    if (qn) { qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z; }
    if (norm) *norm = n;
    R[0] = 1 - 2*(y*y + z*z); R[1] = 2*(x*y - w*z);     R[2] = 2*(x*z + w*y);
    R[3] = 2*(x*y + w*z);     R[4] = 1 - 2*(x*x + z*z); R[5] = 2*(y*z - w*x);
    R[6] = 2*(x*z - w*y);     R[7] = 2*(y*z + w*x);     R[8] = 1 - 2*(x*x + y*y);
    return 1;
}

static void cam_rot(const ora_camera *c, double *R)
{
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) R[3*i+j] = c->w2c[4*i+j];
}

static void cam_to_camera(const ora_camera *c, const double *pw, double *pc)
{
    for (int i = 0; i < 3; ++i)
        pc[i] = c->w2c[4*i]*pw[0] + c->w2c[4*i+1]*pw[1] + c->w2c[4*i+2]*pw[2] + c->w2c[4*i+3];
}

/* camera centre o = -R^T t */
static void cam_centre(const ora_camera *c, double *o)
{
    for (int j = 0; j < 3; ++j)
        o[j] = -(c->w2c[j]*c->w2c[3] + c->w2c[4+j]*c->w2c[7] + c->w2c[8+j]*c->w2c[11]);
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics, Condon-Shortley phase, index k = l^2 + l + m.   */
/* Y_l^m = sqrt2 K_l^m P_l^|m|(cos t) {cos,sin}(|m| phi), K_l^m from its     */
/* factorial closed form.  On the unit sphere sin^m(t) e^{i m phi} equals    */
/* (x+iy)^m and P_l^m(z) = (-1)^m (1-z^2)^{m/2} d^m P_l/dz^m, so each Y is a  */
/* polynomial in (x,y,z) evaluated here from the explicit Legendre series.   */

static double factd(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; }

/* d^m/dz^m P_l(z), P_l(z) = 2^-l sum_k (-1)^k (2l-2k)!/(k!(l-k)!(l-2k)!) z^(l-2k) */
static double legendre_dm(int l, int m, double z)
{
    double s = 0.0;
    for (int k = 0; 2*k <= l; ++k) {
        int p = l - 2*k;
        if (p < m) continue;
        double c = factd(2*l - 2*k) / (factd(k) * factd(l - k) * factd(p)) / ldexp(1.0, l);
        if (k & 1) c = -c;
        c *= factd(p) / factd(p - m);
        s += c * pow(z, p - m);
    }
    return s;
}

void ora_sh_basis(int deg, const double *d, double *Y, double *dY /* [K][3] or NULL */)
{
    const double x = d[0], y = d[1], z = d[2];
    for (int l = 0; l <= deg; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m, k = l*l + l + m;
            double K = sqrt((2.0*l + 1.0) / (4.0*M_PI) * factd(l - am) / factd(l + am));
            double D = legendre_dm(l, am, z), dD = legendre_dm(l, am + 1, z);
            /* (x+iy)^am and (x+iy)^(am-1) */
            double re = 1.0, im = 0.0, gre = 0.0, gim = 0.0;
            for (int i = 0; i < am; ++i) {
                gre = re; gim = im;
                double nr = re*x - im*y, ni = re*y + im*x;
                re = nr; im = ni;
            }
            double c = (am & 1) ? -M_SQRT2 * K : M_SQRT2 * K;
            if (m == 0) {
                Y[k] = K * D;
                if (dY) { dY[3*k] = 0.0; dY[3*k+1] = 0.0; dY[3*k+2] = K * dD; }
            } else if (m > 0) {
                Y[k] = c * D * re;
                if (dY) { dY[3*k] = c*D*am*gre; dY[3*k+1] = -c*D*am*gim; dY[3*k+2] = c*dD*re; }
            } else {
                Y[k] = c * D * im;
                if (dY) { dY[3*k] = c*D*am*gim; dY[3*k+1] = c*D*am*gre; dY[3*k+2] = c*dD*im; }
            }
        }
    }
}

/* Eq. 1: colour = max(0, 0.5 + sum_k SH_k Y_k(dir)), dir = (o - p)/|o - p|. */
static void sh_colour(int deg, const double *sh, const double *dir, double *rgb, double *raw)
{
    double Y[16];
    int K = (deg + 1) * (deg + 1);
    ora_sh_basis(deg, dir, Y, NULL);
    for (int ch = 0; ch < 3; ++ch) {
        double s = 0.5;
        for (int k = 0; k < K; ++k) s += sh[3*k + ch] * Y[k];
        if (raw) raw[ch] = s;
        rgb[ch] = s > 0.0 ? s : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* per-primitive set-up                                                      */

typedef struct {
    int valid;
    double pc[3], tu[3], tv[3], n[3];   /* camera space */
    double s1, s2;
    double rgb[3], raw[3], dir[3];
    int x0, x1, y0, y1;                 /* conservative pixel rectangle (culled mode) */
} surf_t;

typedef struct {
    int valid;
    double t[3];                        /* camera-space centre */
    double px, py;                      /* projected centre */
    double ca, cb, cc;                  /* conic = inverse of Sigma2 */
    double S2a, S2b, S2c;               /* Sigma2 entries (a b; b c) */
    double sigma, d, eps;               /* sigma: the opacity after the Mip-GES factors */
    double sigma0, k3, k2;              /* stored opacity, 3D and 2D filter factors */
    double se[3];                       /* axis lengths after the 3D filter */
    double R2a, R2b, R2c;               /* projected covariance before the screen filter */
    double rgb[3], raw[3], dir[3], dist;
    double R[9], qn[4], qnorm;
    int x0, x1, y0, y1;
    int dim;                            /* 3 or 2 */
    surf_t geo;                         /* 2D: splat frame, filtered scales (geo.s1, geo.s2) */
    double S1, S2;                      /* 2D: object-space filter factors (Eq. 18) */
    double nrm[3];                      /* geometry normal (camera space, facing the camera) */
} gauss_t;

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Relative width of the disc-rim ambiguity band for a fragment whose ray
   meets the disc plane at cosine nd.  The fragment's in-plane coordinates are
   conditioned like its depth, z = (n.P)/(n.d), by 1/|cos|, so any float32
   evaluation's rim decision is uncertain in a band that widens at grazing
   incidence; below tol_graze the pixel is flagged as grazing anyway. */
static double disc_band(const ora_opts *o, double nd)
{
    return o->tol_disc_rel * (1.0 + o->tol_disc_graze / fmax(fabs(nd), o->tol_graze));
}

/* Conservative pixel rectangle of the disc a^2 + b^2 <= r^2 of a planar frame
   (camera-space centre pc, axes tu, tv, scales s1, s2): the disc lies inside
   the rectangle pc +- r s1 tu +- r s2 tv; clip it to z >= znear, project the
   vertices, pad by one pixel.  Leaves an empty rectangle when nothing is in
   front of the near plane or on screen. */
static void disc_rect(const ora_camera *c, surf_t *sf, double r)
{
    double cor[4][3], poly[8][3];
    const double sg[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    for (int k = 0; k < 4; ++k)
        for (int j = 0; j < 3; ++j)
            cor[k][j] = sf->pc[j] + sg[k][0]*r*sf->s1*sf->tu[j] + sg[k][1]*r*sf->s2*sf->tv[j];
    int np = 0;
    double zc = c->znear;
    for (int k = 0; k < 4; ++k) {
        const double *a = cor[k], *b = cor[(k + 1) & 3];
        int ia = a[2] >= zc, ib = b[2] >= zc;
        if (ia) { memcpy(poly[np++], a, sizeof(double) * 3); }
        if (ia != ib) {
            double tt = (zc - a[2]) / (b[2] - a[2]);
            for (int j = 0; j < 3; ++j) poly[np][j] = a[j] + tt * (b[j] - a[j]);
            poly[np][2] = zc;
            ++np;
        }
    }
    if (np == 0) return;
    double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    for (int k = 0; k < np; ++k) {
        double u = c->fx * poly[k][0] / poly[k][2] + c->cx, w = c->fy * poly[k][1] / poly[k][2] + c->cy;
        umin = fmin(umin, u); umax = fmax(umax, u); vmin = fmin(vmin, w); vmax = fmax(vmax, w);
    }
    if (!(umax >= -1.0 && vmax >= -1.0 && umin <= c->width + 1.0 && vmin <= c->height + 1.0)) return;
    sf->x0 = clampi((int)floor(umin - 0.5) - 1, 0, c->width - 1);
    sf->x1 = clampi((int)ceil(umax - 0.5) + 1, 0, c->width - 1);
    sf->y0 = clampi((int)floor(vmin - 0.5) - 1, 0, c->height - 1);
    sf->y1 = clampi((int)ceil(vmax - 0.5) + 1, 0, c->height - 1);
}

static int surfel_setup(const ora_scene *S, const ora_camera *c, const ora_opts *o,
                        const double *ocam, int64_t i, surf_t *sf)
{
    double R[9], Rc[9];
    memset(sf, 0, sizeof *sf);
    if (!quat_rot(S->s_rot + 4*i, R, NULL, NULL)) return 0;
    cam_rot(c, Rc);
    double tu[3] = {R[0], R[3], R[6]}, tv[3] = {R[1], R[4], R[7]}, n[3] = {R[2], R[5], R[8]};
    const double *p = S->s_pos + 3*i;
    cam_to_camera(c, p, sf->pc);
    matvec3(Rc, tu, sf->tu); matvec3(Rc, tv, sf->tv); matvec3(Rc, n, sf->n);
    sf->s1 = S->s_scale[2*i]; sf->s2 = S->s_scale[2*i + 1];
    double v[3] = {ocam[0] - p[0], ocam[1] - p[1], ocam[2] - p[2]};
    double L = sqrt(dot3(v, v));
    for (int k = 0; k < 3; ++k) sf->dir[k] = L > 0 ? v[k] / L : 0.0;
    sh_colour(S->sh_degree, S->s_sh + (int64_t)3 * (S->sh_degree + 1) * (S->sh_degree + 1) * i,
              sf->dir, sf->rgb, sf->raw);
    sf->valid = (sf->s1 > 0.0 && sf->s2 > 0.0 && isfinite(sf->s1) && isfinite(sf->s2));
    /* conservative rectangle: the disc (slightly enlarged by the ambiguity band)
       lies inside the rectangle pc +- r s1 tu +- r s2 tv; clip that rectangle to
       z >= znear, project its vertices, pad by one pixel. */
    sf->x0 = 1; sf->x1 = 0; sf->y0 = 1; sf->y1 = 0;
    if (!sf->valid) return 1;
    disc_rect(c, sf, sqrt(o->surfel_r2 * (1.0 + 2.0 * o->tol_disc_rel * (1.0 + o->tol_disc_graze / o->tol_graze))));
    return 1;
}

/* Gaussian: Sigma3 = R diag(s^2) R^T, EWA projection with the affine Jacobian at
   the centre, fixed screen low-pass Sigma2 += lowpass I (3DGS's fixed-size EWA
   filter, Sec. 6.1), conic = Sigma2^-1, depth d_i = camera z of the centre.
   Mip-GES (Sec. 6.1, the filters of Mip-Splatting): a 3D filter of variance v
   per Gaussian, Sigma3 + v I = R diag(s^2 + v) R^T, with the opacity scaled
   by sqrt(|Sigma3| / |Sigma3 + v I|) = prod_j s_j / sqrt(s_j^2 + v); and with
   filter = 1 the screen filter scales the opacity by
   sqrt(|Sigma2'| / |Sigma2' + lowpass I|), Sigma2' the projection before it.
   Both factors keep the Gaussian's integral unchanged (the convolution of a
   Gaussian with a normalised Gaussian kernel).  eps_i uses the stored axis
   lengths s. */
/* 2D Gaussian of 2D-GES (Sec. 6.4): a planar splat like a surfel (centre p,
   axes t_u = R e_x, t_v = R e_y, normal R e_z, scales s1, s2) whose opacity is
   sigma exp(-(a^2 + b^2)/2) at the ray-plane hit (a, b in scale units), with
   the planar depth of that hit for the depth test.  The screen-space EWA
   filter of size r = lowpass is back-projected into object space (Eq. 17-18):
   with J the Jacobian of local unit coordinates -> pixels at the centre, the
   filtered covariance I + r J^-1 J^-T is approximated by diag(S1^2, S2^2),
   S_k = sqrt(1 + r ((J^T J)^-1)_kk) (its diagonal), so the scales become
   s_k S_k and the opacity sigma / (S1 S2).  eps_i = (5/2)(s1 + s2) (D = 2).
   The Mip-GES 3D filter does not apply to 2D Gaussians. */
static int gauss2d_setup(const ora_scene *S, const ora_camera *c, const ora_opts *o,
                         const double *ocam, int64_t i, gauss_t *g, const double *Rc)
{
    g->dim = 2;
    const double *p = S->g_pos + 3*i, *s = S->g_scale + 2*i;
    cam_to_camera(c, p, g->t);
    g->sigma0 = S->g_opac[i];
    g->sigma = g->sigma0;
    g->k3 = 1.0; g->k2 = 1.0;
    surf_t *f = &g->geo;
    double tu[3] = {g->R[0], g->R[3], g->R[6]}, tv[3] = {g->R[1], g->R[4], g->R[7]};
    double n[3] = {g->R[2], g->R[5], g->R[8]};
    memcpy(f->pc, g->t, sizeof g->t);
    matvec3(Rc, tu, f->tu); matvec3(Rc, tv, f->tv); matvec3(Rc, n, f->n);
    f->x0 = 1; f->x1 = 0; f->y0 = 1; f->y1 = 0;
    const double fl = dot3(f->n, f->pc) > 0.0 ? -1.0 : 1.0;   /* face the camera */
    for (int k = 0; k < 3; ++k) g->nrm[k] = fl * f->n[k];
    switch (o->eps_mode) {
    case 0: g->eps = o->eps_factor / 2.0 * (s[0] + s[1]); break;
    case 1: g->eps = 0.0; break;
    default: g->eps = o->eps_value; break;
    }
    g->d = g->t[2];
    double v[3] = {ocam[0] - p[0], ocam[1] - p[1], ocam[2] - p[2]};
    g->dist = sqrt(dot3(v, v));
    for (int k = 0; k < 3; ++k) g->dir[k] = g->dist > 0 ? v[k] / g->dist : 0.0;
    sh_colour(S->sh_degree, S->g_sh + (int64_t)3 * (S->sh_degree + 1) * (S->sh_degree + 1) * i,
              g->dir, g->rgb, g->raw);
    if (!(g->t[2] > c->znear) || !(s[0] > 0.0 && s[1] > 0.0) || !isfinite(s[0]) || !isfinite(s[1])) return 1;
    /* J = Jp [s1 t_u, s2 t_v]: local unit coordinates -> pixels, at the centre */
    const double x = g->t[0], y = g->t[1], z = g->t[2];
    const double Jp[6] = {c->fx / z, 0.0, -c->fx * x / (z*z), 0.0, c->fy / z, -c->fy * y / (z*z)};
    double J[4];
    for (int a = 0; a < 2; ++a) {
        J[2*a] = s[0] * (Jp[3*a]*f->tu[0] + Jp[3*a + 1]*f->tu[1] + Jp[3*a + 2]*f->tu[2]);
        J[2*a + 1] = s[1] * (Jp[3*a]*f->tv[0] + Jp[3*a + 1]*f->tv[1] + Jp[3*a + 2]*f->tv[2]);
    }
    const double M00 = J[0]*J[0] + J[2]*J[2], M01 = J[0]*J[1] + J[2]*J[3], M11 = J[1]*J[1] + J[3]*J[3];
    const double det = M00 * M11 - M01 * M01;
    if (!(det > 0.0) || !isfinite(det)) return 1;
    g->S1 = sqrt(1.0 + o->lowpass * M11 / det);
    g->S2 = sqrt(1.0 + o->lowpass * M00 / det);
    f->s1 = s[0] * g->S1;
    f->s2 = s[1] * g->S2;
    f->valid = 1;
    g->sigma = g->sigma0 / (g->S1 * g->S2);
    g->valid = 1;
    /* exact support: alpha >= a  <=>  a'^2 + b'^2 <= 2 ln(sigma/a) in filtered units;
       widened by the alpha ambiguity band so that culled == brute force exactly */
    double amin = o->alpha_min - o->tol_alpha;
    if (!(g->sigma > amin) || amin <= 0.0) return 1;
    disc_rect(c, f, sqrt(2.0 * log(g->sigma / amin)));
    g->x0 = f->x0; g->x1 = f->x1; g->y0 = f->y0; g->y1 = f->y1;
    return 1;
}

static int gauss_setup(const ora_scene *S, const ora_camera *c, const ora_opts *o,
                       const double *ocam, int64_t i, gauss_t *g)
{
    double Rc[9];
    memset(g, 0, sizeof *g);
    g->x0 = 1; g->x1 = 0; g->y0 = 1; g->y1 = 0;
    g->dim = 3;
    if (!quat_rot(S->g_rot + 4*i, g->R, g->qn, &g->qnorm)) return 0;
    cam_rot(c, Rc);
    if (S->gauss_dim == 2) return gauss2d_setup(S, c, o, ocam, i, g, Rc);
    const double *p = S->g_pos + 3*i, *s = S->g_scale + 3*i;
    cam_to_camera(c, p, g->t);
    g->sigma0 = S->g_opac[i];
    g->sigma = g->sigma0;
    g->k3 = 1.0; g->k2 = 1.0;
    {
        const double v = S->g_filt3 ? S->g_filt3[i] : 0.0;
        for (int k = 0; k < 3; ++k) {
            g->se[k] = sqrt(s[k] * s[k] + v);
            g->k3 *= fabs(s[k]) / g->se[k];
        }
        if (v == 0.0) { g->k3 = 1.0; for (int k = 0; k < 3; ++k) g->se[k] = s[k]; }
    }
    switch (o->eps_mode) {
    case 0: g->eps = o->eps_factor / 3.0 * (s[0] + s[1] + s[2]); break;
    case 1: g->eps = 0.0; break;
    default: g->eps = o->eps_value; break;
    }
    g->d = g->t[2];
    {
        /* geometry normal (Sec. 6.4): the axis of the smallest scale, facing the camera */
        int km = 0;
        for (int k = 1; k < 3; ++k)
            if (fabs(s[k]) < fabs(s[km])) km = k;
        double ax[3] = {g->R[km], g->R[3 + km], g->R[6 + km]};
        matvec3(Rc, ax, g->nrm);
        if (dot3(g->nrm, g->t) > 0.0)
            for (int k = 0; k < 3; ++k) g->nrm[k] = -g->nrm[k];
    }
    double v[3] = {ocam[0] - p[0], ocam[1] - p[1], ocam[2] - p[2]};
    g->dist = sqrt(dot3(v, v));
    for (int k = 0; k < 3; ++k) g->dir[k] = g->dist > 0 ? v[k] / g->dist : 0.0;
    sh_colour(S->sh_degree, S->g_sh + (int64_t)3 * (S->sh_degree + 1) * (S->sh_degree + 1) * i,
              g->dir, g->rgb, g->raw);
    if (!(g->t[2] > c->znear)) return 1;
    double S3[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += g->R[3*a + k] * g->se[k] * g->se[k] * g->R[3*b + k];
            S3[3*a + b] = acc;
        }
    double x = g->t[0], y = g->t[1], z = g->t[2];
    double J[6] = {c->fx / z, 0.0, -c->fx * x / (z*z), 0.0, c->fy / z, -c->fy * y / (z*z)};
    double T[6];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 3; ++b)
            T[3*a + b] = J[3*a]*Rc[b] + J[3*a + 1]*Rc[3 + b] + J[3*a + 2]*Rc[6 + b];
    double S2[4];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += T[3*a + k] * S3[3*k + l] * T[3*b + l];
            S2[2*a + b] = acc;
        }
    g->R2a = S2[0]; g->R2b = 0.5 * (S2[1] + S2[2]); g->R2c = S2[3];
    g->S2a = S2[0] + o->lowpass; g->S2b = g->R2b; g->S2c = S2[3] + o->lowpass;
    double det = g->S2a * g->S2c - g->S2b * g->S2b;
    if (!(det > 0.0) || !isfinite(det)) return 1;
    if (o->filter == 1) {
        double det0 = g->R2a * g->R2c - g->R2b * g->R2b;
        g->k2 = det0 > 0.0 ? sqrt(det0 / det) : 0.0;
    }
    g->sigma = g->sigma0 * g->k3 * g->k2;
    g->ca = g->S2c / det; g->cb = -g->S2b / det; g->cc = g->S2a / det;
    g->px = c->fx * x / z + c->cx;
    g->py = c->fy * y / z + c->cy;
    g->valid = 1;
    /* exact support (Eq. 4 with the 1/255 clamp): alpha >= a  <=>  q <= 2 ln(sigma/a);
       widened by the alpha ambiguity band so that culled == brute force exactly. */
    double amin = o->alpha_min - o->tol_alpha;
    if (!(g->sigma > amin) || amin <= 0.0) return 1;
    double Tq = 2.0 * log(g->sigma / amin);
    double hx = sqrt(Tq * g->S2a), hy = sqrt(Tq * g->S2c);
    double umin = g->px - hx, umax = g->px + hx, vmin = g->py - hy, vmax = g->py + hy;
    if (!(umax >= -1.0 && vmax >= -1.0 && umin <= c->width + 1.0 && vmin <= c->height + 1.0)) return 1;
    g->x0 = clampi((int)floor(umin - 0.5) - 1, 0, c->width - 1);
    g->x1 = clampi((int)ceil(umax - 0.5) + 1, 0, c->width - 1);
    g->y0 = clampi((int)floor(vmin - 0.5) - 1, 0, c->height - 1);
    g->y1 = clampi((int)ceil(vmax - 0.5) + 1, 0, c->height - 1);
    return 1;
}

/* ------------------------------------------------------------------------ */
/* per-pixel definitions                                                     */

/* Ray through the pixel centre (i+0.5, j+0.5): d = ((u-cx)/fx, (v-cy)/fy, 1). */
static void pixel_ray(const ora_camera *c, int i, int j, double *d)
{
    d[0] = ((i + 0.5) - c->cx) / c->fx;
    d[1] = ((j + 0.5) - c->cy) / c->fy;
    d[2] = 1.0;
}

/* Sample k of pixel (i,j).  One sample: the centre.  Four samples (4x
   multisampling, Sec. 5, which equals 4x supersampling for opaque single-
   colour surfels): the 2x2 grid (i + 0.25 + 0.5 (k mod 2), j + 0.25 + 0.5 (k div 2)). */
static void sample_ray(const ora_camera *c, int samples, int i, int j, int k, double *d)
{
    double u = i + 0.5, v = j + 0.5;
    if (samples == 4) { u = i + 0.25 + 0.5 * (k & 1); v = j + 0.25 + 0.5 * (k >> 1); }
    d[0] = (u - c->cx) / c->fx;
    d[1] = (v - c->cy) / c->fy;
    d[2] = 1.0;
}

/* Surfel fragment at a pixel: ray-plane hit depth z (camera z), local disc
   coordinates (a,b) of the hit scaled by (s1,s2), rho = a^2 + b^2.
   Returns 0 when the ray is parallel to the plane. */
static int surfel_hit(const surf_t *sf, const double *d, double *z, double *rho, double *ndot)
{
    double den = dot3(sf->n, d);
    if (ndot) *ndot = den / sqrt(dot3(d, d));
    if (den == 0.0) return 0;
    double zz = dot3(sf->n, sf->pc) / den;
    double X[3] = {zz*d[0] - sf->pc[0], zz*d[1] - sf->pc[1], zz*d[2] - sf->pc[2]};
    double a = dot3(X, sf->tu) / sf->s1, b = dot3(X, sf->tv) / sf->s2;
    *z = zz;
    *rho = a*a + b*b;
    return 1;
}

/* Eq. 4 before the clamp at pixel (i, j), and the depth its depth test uses:
   3D, the centre depth d_i; 2D, the planar depth of the ray-splat hit (no hit
   in front of the near plane: alpha 0, depth +inf).  *ndot: for 2D, the
   cosine between the splat normal and the ray (1 for 3D). */
static double gauss_eval(const ora_camera *c, const gauss_t *g, int i, int j, double *depth, double *ndot)
{
    if (g->dim == 2) {
        double d[3], z, rho, nd;
        pixel_ray(c, i, j, d);
        int hit = surfel_hit(&g->geo, d, &z, &rho, &nd);
        if (ndot) *ndot = nd;
        if (!hit || !(z > c->znear)) { *depth = INFINITY; return 0.0; }
        *depth = z;
        return g->sigma * exp(-0.5 * rho);
    }
    if (ndot) *ndot = 1.0;
    *depth = g->d;
    double dx = (i + 0.5) - g->px, dy = (j + 0.5) - g->py;
    double q = g->ca*dx*dx + 2.0*g->cb*dx*dy + g->cc*dy*dy;
    return g->sigma * exp(-0.5 * q);
}

/* ------------------------------------------------------------------------ */
/* candidate lists per 16x16 pixel cell (culled mode), each in ascending
   primitive index; brute force uses every index */

#define ORA_CELL 16
typedef struct { int64_t *off; int64_t *idx; int cx; } rowlists;

static int build_rows(int W, int H, int64_t n, const int *x0, const int *x1, const int *y0, const int *y1,
                      size_t stride, rowlists *rl)
{
    const int cx = (W + ORA_CELL - 1) / ORA_CELL, cy = (H + ORA_CELL - 1) / ORA_CELL;
    const int64_t nc = (int64_t)cx * cy;
    rl->cx = cx;
    rl->off = calloc((size_t)nc + 1, sizeof(int64_t));
    if (!rl->off) return 0;
#define FLD(p, i) (*(const int *)((const char *)(p) + stride * (i)))
    for (int64_t i = 0; i < n; ++i) {
        if (FLD(x0, i) > FLD(x1, i) || FLD(y0, i) > FLD(y1, i)) continue;
        for (int b = FLD(y0, i) / ORA_CELL; b <= FLD(y1, i) / ORA_CELL; ++b)
            for (int a = FLD(x0, i) / ORA_CELL; a <= FLD(x1, i) / ORA_CELL; ++a) rl->off[(int64_t)b * cx + a + 1]++;
    }
    for (int64_t c = 0; c < nc; ++c) rl->off[c + 1] += rl->off[c];
    rl->idx = malloc(sizeof(int64_t) * (size_t)(rl->off[nc] > 0 ? rl->off[nc] : 1));
    int64_t *cur = malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    if (!rl->idx || !cur) { free(cur); return 0; }
    for (int64_t c = 0; c < nc; ++c) cur[c] = rl->off[c];
    for (int64_t i = 0; i < n; ++i) {
        if (FLD(x0, i) > FLD(x1, i) || FLD(y0, i) > FLD(y1, i)) continue;
        for (int b = FLD(y0, i) / ORA_CELL; b <= FLD(y1, i) / ORA_CELL; ++b)
            for (int a = FLD(x0, i) / ORA_CELL; a <= FLD(x1, i) / ORA_CELL; ++a)
                rl->idx[cur[(int64_t)b * cx + a]++] = i;
    }
#undef FLD
    free(cur);
    return 1;
}

static void free_rows(rowlists *rl) { free(rl->off); free(rl->idx); }

/* ------------------------------------------------------------------------ */
/* forward                                                                   */

typedef struct {
    surf_t *sf; gauss_t *gs;
    rowlists rs, rg;
} prep_t;

static void prep_free(prep_t *P)
{
    free(P->sf); free(P->gs);
    free_rows(&P->rs); free_rows(&P->rg);
}

static int prepare(const ora_scene *S, const ora_camera *c, const ora_opts *o, int culled, prep_t *P)
{
    memset(P, 0, sizeof *P);
    double ocam[3];
    cam_centre(c, ocam);
    int64_t N = S->n_surfels, M = S->n_gaussians;
    P->sf = calloc((size_t)(N > 0 ? N : 1), sizeof(surf_t));
    P->gs = calloc((size_t)(M > 0 ? M : 1), sizeof(gauss_t));
    if (!P->sf || !P->gs) return ORA_NOMEM;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(|:bad)
    for (int64_t i = 0; i < N; ++i) bad |= !surfel_setup(S, c, o, ocam, i, &P->sf[i]);
#pragma omp parallel for schedule(static) reduction(|:bad)
    for (int64_t i = 0; i < M; ++i) bad |= !gauss_setup(S, c, o, ocam, i, &P->gs[i]);
    if (bad) return ORA_BAD_QUAT;
    if (culled) {
        if (!build_rows(c->width, c->height, N, &P->sf[0].x0, &P->sf[0].x1, &P->sf[0].y0, &P->sf[0].y1,
                        sizeof(surf_t), &P->rs)) return ORA_NOMEM;
        if (!build_rows(c->width, c->height, M, &P->gs[0].x0, &P->gs[0].x1, &P->gs[0].y0, &P->gs[0].y1,
                        sizeof(gauss_t), &P->rg)) return ORA_NOMEM;
    }
    return ORA_OK;
}

/* Pass 1 at one sample ray: the lexicographic min of (z, index) over surfels
   whose fragment is inside the opaque disc in front of the near plane, and
   the ambiguity flag of that decision. */
static void zbuffer_sample(const ora_scene *S, const ora_camera *c, const ora_opts *o, const prep_t *P, int culled,
                           int i, int j, const double *d, int64_t *best_out, double *z_out, uint8_t *amb)
{
    const double r2 = o->surfel_r2;
    int64_t best = -1, second = -1;
    double z1 = INFINITY, z2 = INFINITY, rho1 = 0.0, nd1 = 1.0, zband = INFINITY;
    int64_t lo = 0, hi = S->n_surfels;
    if (culled) {
        const int64_t cell = (int64_t)(j / ORA_CELL) * P->rs.cx + i / ORA_CELL;
        lo = P->rs.off[cell]; hi = P->rs.off[cell + 1];
    }
    for (int64_t t = lo; t < hi; ++t) {
        int64_t s = culled ? P->rs.idx[t] : t;
        const surf_t *sf = &P->sf[s];
        if (!sf->valid) continue;
        if (culled && (i < sf->x0 || i > sf->x1 || j < sf->y0 || j > sf->y1)) continue;
        double z, rho, nd;
        if (!surfel_hit(sf, d, &z, &rho, &nd)) continue;
        if (!(z > c->znear)) continue;
        if (fabs(rho - r2) <= disc_band(o, nd) * r2) zband = fmin(zband, z);
        if (!(rho <= r2)) continue;
        if (fabs(z - c->znear) <= o->tol_depth_rel * fmax(1.0, c->znear)) *amb |= AMB_ID;
        if (z < z1 || (z == z1 && s < best)) {
            second = best; z2 = z1;
            best = s; z1 = z; rho1 = rho; nd1 = nd;
        } else if (z < z2 || (z == z2 && s < second)) {
            second = s; z2 = z;
        }
    }
    if (second >= 0 && (z2 - z1) <= o->tol_depth_rel * z1) *amb |= AMB_ID;
    if (best >= 0 && fabs(rho1 - r2) <= disc_band(o, nd1) * r2) *amb |= AMB_ID;
    if (best >= 0 && fabs(nd1) < o->tol_graze) *amb |= AMB_ID;
    if (zband < INFINITY && (best < 0 || zband <= z1 * (1.0 + o->tol_depth_rel))) *amb |= AMB_ID;
    *best_out = best;
    *z_out = z1;
}

/* One pixel of both passes.  Writes C, D_s, the surfel id of every sample,
   W_G, the ambiguity bits and the number of Gaussians that contributed.
   With 4 samples the surfel pass is multisampled (Sec. 5): C_s is the mean
   of the samples' colours (bg where a sample hits nothing) and D_s, for the
   Gaussians' depth test, the nearest sample's depth; the Gaussians are
   evaluated at the pixel centre only. */
/* Geometry of one pixel (Sec. 6.4, Eq. 10-12): the surfel normal N_s (of the
   nearest sample's surfel, facing the camera; 0 where none), D_G and N_G. */
typedef struct {
    double Ns[3], DG, NG[3];
    int covered;
} geo_px;

static void shade_pixel(const ora_scene *S, const ora_camera *c, const ora_opts *o, const prep_t *P,
                        int culled, int i, int j, double *C, double *Ds_out, int32_t *id_out,
                        double *wg_out, uint8_t *amb_out, int32_t *nc_out, geo_px *geo)
{
    const int ns = o->samples == 4 ? 4 : 1;
    uint8_t amb = 0;
    double Ds = INFINITY, Cs[3] = {0, 0, 0};
    int64_t nearest = -1;
    for (int k = 0; k < ns; ++k) {
        int64_t best = -1;
        double z = INFINITY;
        if (o->mode != 2) {
            double d[3];
            sample_ray(c, ns, i, j, k, d);
            zbuffer_sample(S, c, o, P, culled, i, j, d, &best, &z, &amb);
        }
        if (best >= 0 && (z < Ds || (z == Ds && best < nearest))) nearest = best;
        if (best >= 0) Ds = fmin(Ds, z);
        for (int ch = 0; ch < 3; ++ch) Cs[ch] += (best >= 0 ? P->sf[best].rgb[ch] : c->bg[ch]) / ns;
        id_out[k] = (int32_t)best;
    }
    if (geo) {
        memset(geo, 0, sizeof *geo);
        geo->covered = nearest >= 0;
        if (nearest >= 0) {
            const surf_t *sf = &P->sf[nearest];
            const double fl = dot3(sf->n, sf->pc) > 0.0 ? -1.0 : 1.0;
            for (int k = 0; k < 3; ++k) geo->Ns[k] = fl * sf->n[k];
        }
    }

    /* pass 2: order-independent accumulation (Eq. 2-4) */
    double CG[3] = {0, 0, 0}, WG = 0.0;
    int32_t nc = 0;
    if (o->mode != 1) {
        int64_t lo = 0, hi = S->n_gaussians;
        if (culled) {
            const int64_t cell = (int64_t)(j / ORA_CELL) * P->rg.cx + i / ORA_CELL;
            lo = P->rg.off[cell]; hi = P->rg.off[cell + 1];
        }
        for (int64_t t = lo; t < hi; ++t) {
            int64_t k = culled ? P->rg.idx[t] : t;
            const gauss_t *g = &P->gs[k];
            if (!g->valid) continue;
            if (culled && (i < g->x0 || i > g->x1 || j < g->y0 || j > g->y1)) continue;
            double gd, nd;
            double a = gauss_eval(c, g, i, j, &gd, &nd);
            double lim = gd - (Ds + g->eps);
            int pass = gd < Ds + g->eps;
            if (fabs(a - o->alpha_min) <= o->tol_alpha && (pass || fabs(lim) <= o->tol_gdepth_rel * fmax(1.0, Ds)))
                amb |= AMB_COLOR;
            if (a >= o->alpha_min - o->tol_alpha && isfinite(Ds) &&
                fabs(lim) <= o->tol_gdepth_rel * fmax(1.0, Ds))
                amb |= AMB_COLOR;
            /* a splat seen edge-on: its hit and planar depth are ill-conditioned */
            if (g->dim == 2 && a >= o->alpha_min - o->tol_alpha && fabs(nd) < o->tol_graze) amb |= AMB_COLOR;
            if (!(a >= o->alpha_min) || !pass) continue;
            for (int ch = 0; ch < 3; ++ch) CG[ch] += a * g->rgb[ch];
            WG += a;
            if (geo) {
                geo->DG += a * gd;
                for (int ch = 0; ch < 3; ++ch) geo->NG[ch] += a * g->nrm[ch];
            }
            ++nc;
        }
    }
    /* Eq. 5 and the two ablation modes */
    for (int ch = 0; ch < 3; ++ch) {
        if (o->mode == 0) C[ch] = (Cs[ch] * 1.0 + CG[ch]) / (1.0 + WG);
        else if (o->mode == 1) C[ch] = Cs[ch];
        else C[ch] = WG > 0.0 ? CG[ch] / WG : c->bg[ch];
    }
    *Ds_out = Ds;
    *wg_out = WG;
    *amb_out = amb;
    *nc_out = nc;
}

static int check_args(const ora_scene *S, const ora_camera *c, const ora_opts *o)
{
    if (!S || !c || !o) return 0;
    if (c->width <= 0 || c->height <= 0) return 0;
    if (S->sh_degree < 0 || S->sh_degree > 3) return 0;
    if (S->n_surfels < 0 || S->n_gaussians < 0) return 0;
    if (!(c->fx > 0 && c->fy > 0 && c->znear > 0)) return 0;
    if (o->samples != 1 && o->samples != 4) return 0;
    if (o->filter != 0 && o->filter != 1) return 0;
    if (S->gauss_dim != 0 && S->gauss_dim != 2 && S->gauss_dim != 3) return 0;
    return 1;
}

int ora_render(const ora_scene *S, const ora_camera *c, const ora_opts *o, int culled, int nthreads,
               double *rgb, double *depth, int32_t *sid, double *wg, uint8_t *amb, int32_t *ncontrib)
{
    if (!check_args(S, c, o)) return ORA_BAD_ARG;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    prep_t P;
    int st = prepare(S, c, o, culled, &P);
    if (st != ORA_OK) { prep_free(&P); return st; }
    const int W = c->width, H = c->height;
    const int64_t HW = (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < H; ++j) {
        for (int i = 0; i < W; ++i) {
            int64_t pix = (int64_t)j * W + i;
            double C[3], Ds, WG;
            int32_t id[4], nc;
            uint8_t a;
            shade_pixel(S, c, o, &P, culled, i, j, C, &Ds, id, &WG, &a, &nc, NULL);
            for (int ch = 0; ch < 3; ++ch) rgb[ch * HW + pix] = C[ch];
            depth[pix] = Ds;
            for (int k = 0; k < (o->samples == 4 ? 4 : 1); ++k) sid[k * HW + pix] = id[k];
            wg[pix] = WG;
            amb[pix] = a;
            if (ncontrib) ncontrib[pix] = nc;
        }
    }
    prep_free(&P);
    return ORA_OK;
}

/* Geometry maps (Sec. 6.4, Eq. 10-12), camera space: N_s [3,H,W], D_G [H,W],
   N_G [3,H,W] and the smoothed maps D_smooth = (W_s D_s + D_G)/(W_s + W_G),
   N_smooth = (W_s N_s + N_G)/(W_s + W_G) with W_s = 1 where a surfel covers
   the pixel and 0 elsewhere (no surfel depth exists there); where both
   weights are 0, D_smooth = +inf and N_smooth = 0.  d_i, n_i: centre depth and
   smallest-scale axis for 3D Gaussians, planar depth and splat normal for 2D
   ones; normals face the camera.  Also writes amb like ora_render. */
int ora_render_geom(const ora_scene *S, const ora_camera *c, const ora_opts *o, int culled, int nthreads,
                    double *ns_out, double *dg_out, double *ng_out, double *dsm_out, double *nsm_out, uint8_t *amb)
{
    if (!check_args(S, c, o)) return ORA_BAD_ARG;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    prep_t P;
    int st = prepare(S, c, o, culled, &P);
    if (st != ORA_OK) { prep_free(&P); return st; }
    const int W = c->width, H = c->height;
    const int64_t HW = (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < H; ++j) {
        for (int i = 0; i < W; ++i) {
            int64_t pix = (int64_t)j * W + i;
            double C[3], Ds, WG;
            int32_t id[4], nc;
            uint8_t a;
            geo_px g;
            shade_pixel(S, c, o, &P, culled, i, j, C, &Ds, id, &WG, &a, &nc, &g);
            const double ws = g.covered ? 1.0 : 0.0, wt = ws + WG;
            dg_out[pix] = g.DG;
            dsm_out[pix] = wt > 0.0 ? ((g.covered ? Ds : 0.0) + g.DG) / wt : INFINITY;
            for (int ch = 0; ch < 3; ++ch) {
                ns_out[ch * HW + pix] = g.Ns[ch];
                ng_out[ch * HW + pix] = g.NG[ch];
                nsm_out[ch * HW + pix] = wt > 0.0 ? (ws * g.Ns[ch] + g.NG[ch]) / wt : 0.0;
            }
            amb[pix] = a;
        }
    }
    prep_free(&P);
    return ORA_OK;
}

/* Work counts: (sample, surfel) fragments inside the opaque disc in front of
   the near plane, and (pixel, Gaussian) pairs with alpha >= alpha_min. */
int ora_count_fragments(const ora_scene *S, const ora_camera *c, const ora_opts *o, int64_t *n_surf,
                        int64_t *n_gauss)
{
    if (!check_args(S, c, o)) return ORA_BAD_ARG;
    prep_t P;
    int st = prepare(S, c, o, 1, &P);
    if (st != ORA_OK) { prep_free(&P); return st; }
    const int W = c->width, H = c->height;
    int64_t ns = 0, ng = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+:ns, ng)
    for (int j = 0; j < H; ++j) {
        for (int i = 0; i < W; ++i) {
            const int64_t cell = (int64_t)(j / ORA_CELL) * P.rs.cx + i / ORA_CELL;
            const int nsamp = o->samples == 4 ? 4 : 1;
            if (o->mode != 2)
                for (int k = 0; k < nsamp; ++k) {
                    double d[3];
                    sample_ray(c, nsamp, i, j, k, d);
                    for (int64_t t = P.rs.off[cell]; t < P.rs.off[cell + 1]; ++t) {
                        const surf_t *sf = &P.sf[P.rs.idx[t]];
                        if (!sf->valid || i < sf->x0 || i > sf->x1 || j < sf->y0 || j > sf->y1) continue;
                        double z, rho;
                        if (surfel_hit(sf, d, &z, &rho, NULL) && z > c->znear && rho <= o->surfel_r2) ++ns;
                    }
                }
            if (o->mode != 1)
                for (int64_t t = P.rg.off[cell]; t < P.rg.off[cell + 1]; ++t) {
                    const gauss_t *g = &P.gs[P.rg.idx[t]];
                    if (!g->valid || i < g->x0 || i > g->x1 || j < g->y0 || j > g->y1) continue;
                    double gd;
                    if (gauss_eval(c, g, i, j, &gd, NULL) >= o->alpha_min) ++ng;
                }
        }
    }
    prep_free(&P);
    *n_surf = ns;
    *n_gauss = ng;
    return ORA_OK;
}

/* Evaluate surfel sid[k] at pixel (px[k], py[k]): hit depth, rho = a^2+b^2 and
   the cosine between the plane normal and the ray.  Returns per entry 1 on a
   hit, 0 if parallel or invalid. */
int ora_surfel_eval(const ora_scene *S, const ora_camera *c, const ora_opts *o, int64_t n,
                    const int32_t *px, const int32_t *py, const int32_t *sid,
                    double *z, double *rho, double *ndot, int32_t *ok)
{
    if (!check_args(S, c, o)) return ORA_BAD_ARG;
    double ocam[3];
    cam_centre(c, ocam);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
        surf_t sf;
        ok[k] = 0; z[k] = NAN; rho[k] = NAN; ndot[k] = NAN;
        if (sid[k] < 0 || sid[k] >= S->n_surfels) continue;
        if (!surfel_setup(S, c, o, ocam, sid[k], &sf) || !sf.valid) continue;
        double d[3];
        pixel_ray(c, px[k], py[k], d);
        ok[k] = surfel_hit(&sf, d, &z[k], &rho[k], &ndot[k]);
    }
    return ORA_OK;
}

/* Is ids[pix] an acceptable z-buffer answer at each pixel (each sample:
   ids and valid are [samples, H, W])?  The exact answer
   is the lexicographic min of (z, index) over surfels whose fragment is inside
   its disc in front of the near plane; where fragments sit within the bands
   (disc rim |rho - r2| <= band r2 with the band of disc_band, depth gap
   <= tol_depth z) several
   answers are correct.  A surfel s is acceptable iff its fragment is inside
   its disc up to the rim band and in front of the near plane up to the depth
   band, and no surfel clearly in front of it (z_t < z_s (1 - tol_depth)) is
   clearly inside its own disc (rho_t < r2 (1 - band)).  -1 is acceptable
   iff no surfel is clearly inside.  Grazing fragments (|cos| < tol_graze)
   count as inside up to the band, like rim fragments. */
int ora_check_ids(const ora_scene *S, const ora_camera *c, const ora_opts *o, const int32_t *ids,
                  uint8_t *valid)
{
    if (!check_args(S, c, o)) return ORA_BAD_ARG;
    prep_t P;
    int st = prepare(S, c, o, 1, &P);
    if (st != ORA_OK) { prep_free(&P); return st; }
    const int W = c->width, H = c->height, nsamp = o->samples == 4 ? 4 : 1;
    const int64_t HW = (int64_t)W * H;
    const double r2 = o->surfel_r2, td = o->tol_depth_rel;
#pragma omp parallel for schedule(dynamic, 1)
    for (int jk = 0; jk < H * nsamp; ++jk) {
        const int j = jk % H, smp = jk / H;
        for (int i = 0; i < W; ++i) {
            const int64_t pix = smp * HW + (int64_t)j * W + i;
            const int32_t s = ids[pix];
            double d[3];
            sample_ray(c, nsamp, i, j, smp, d);
            double zs = INFINITY;
            int ok = 1;
            if (s >= 0) {
                if (s >= S->n_surfels || !P.sf[s].valid) { valid[pix] = 0; continue; }
                double rho, nd;
                if (!surfel_hit(&P.sf[s], d, &zs, &rho, &nd) || !(zs > c->znear * (1.0 - td)) ||
                    !(rho <= r2 * (1.0 + disc_band(o, nd)) || fabs(nd) < o->tol_graze)) { valid[pix] = 0; continue; }
            }
            const int64_t cell = (int64_t)(j / ORA_CELL) * P.rs.cx + i / ORA_CELL;
            for (int64_t t = P.rs.off[cell]; t < P.rs.off[cell + 1] && ok; ++t) {
                const int64_t q = P.rs.idx[t];
                const surf_t *sf = &P.sf[q];
                if (q == s || !sf->valid || i < sf->x0 || i > sf->x1 || j < sf->y0 || j > sf->y1) continue;
                double z, rho, nd;
                if (!surfel_hit(sf, d, &z, &rho, &nd)) continue;
                if (!(z > c->znear * (1.0 + td))) continue;
                if (!(z < zs * (1.0 - td))) continue;
                if (rho < r2 * (1.0 - disc_band(o, nd)) && fabs(nd) >= o->tol_graze) ok = 0;
            }
            valid[pix] = (uint8_t)ok;
        }
    }
    prep_free(&P);
    return ORA_OK;
}

/* Primitives that touch a flagged pixel (flag[pix] != 0): a Gaussian whose
   alpha (before the clamp) reaches alpha_min - tol_alpha there, a surfel whose
   fragment there lies inside its disc band in front of the near plane.  Used to
   leave out of gradient comparisons the primitives whose gradient depends on
   which of several equally correct forward answers was taken. */
int ora_touching(const ora_scene *S, const ora_camera *c, const ora_opts *o, const uint8_t *flag,
                 uint8_t *s_touch, uint8_t *g_touch)
{
    if (!check_args(S, c, o)) return ORA_BAD_ARG;
    prep_t P;
    int st = prepare(S, c, o, 0, &P);
    if (st != ORA_OK) { prep_free(&P); return st; }
    const int W = c->width;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t s = 0; s < S->n_surfels; ++s) {
        const surf_t *sf = &P.sf[s];
        s_touch[s] = 0;
        if (!sf->valid) continue;
        for (int j = sf->y0; j <= sf->y1 && !s_touch[s]; ++j)
            for (int i = sf->x0; i <= sf->x1; ++i) {
                if (!flag[(int64_t)j * W + i]) continue;
                const int nsamp = o->samples == 4 ? 4 : 1;
                for (int k = 0; k < nsamp && !s_touch[s]; ++k) {
                    double d[3], z, rho, nd;
                    sample_ray(c, nsamp, i, j, k, d);
                    if (surfel_hit(sf, d, &z, &rho, &nd) && z > c->znear &&
                        rho <= o->surfel_r2 * (1.0 + disc_band(o, nd))) s_touch[s] = 1;
                }
                if (s_touch[s]) break;
            }
    }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t k = 0; k < S->n_gaussians; ++k) {
        const gauss_t *g = &P.gs[k];
        g_touch[k] = 0;
        if (!g->valid) continue;
        for (int j = g->y0; j <= g->y1 && !g_touch[k]; ++j)
            for (int i = g->x0; i <= g->x1; ++i) {
                double gd;
                if (flag[(int64_t)j * W + i] && gauss_eval(c, g, i, j, &gd, NULL) >= o->alpha_min - o->tol_alpha) {
                    g_touch[k] = 1;
                    break;
                }
            }
    }
    prep_free(&P);
    return ORA_OK;
}

/* Per-primitive quantities for unit pins.
   surfel: out = [valid, rgb(3), pc(3), n(3), x0, x1, y0, y1]                 (14)
   gauss:  out = [valid, px, py, ca, cb, cc, S2a, S2b, S2c, sigma, d, eps,
                  rgb(3), x0, x1, y0, y1, nrm(3), S1, S2, s1', s2']           (26)
           (2D Gaussians: px..S2c are 0; S1, S2 the object-space filter
            factors, s1', s2' the filtered scales) */
int ora_surfel_info(const ora_scene *S, const ora_camera *c, const ora_opts *o, int64_t i, double *out)
{
    if (!check_args(S, c, o) || i < 0 || i >= S->n_surfels) return ORA_BAD_ARG;
    double ocam[3];
    cam_centre(c, ocam);
    surf_t sf;
    if (!surfel_setup(S, c, o, ocam, i, &sf)) return ORA_BAD_QUAT;
    out[0] = sf.valid;
    for (int k = 0; k < 3; ++k) { out[1 + k] = sf.rgb[k]; out[4 + k] = sf.pc[k]; out[7 + k] = sf.n[k]; }
    out[10] = sf.x0; out[11] = sf.x1; out[12] = sf.y0; out[13] = sf.y1;
    return ORA_OK;
}

int ora_gauss_info(const ora_scene *S, const ora_camera *c, const ora_opts *o, int64_t i, double *out)
{
    if (!check_args(S, c, o) || i < 0 || i >= S->n_gaussians) return ORA_BAD_ARG;
    double ocam[3];
    cam_centre(c, ocam);
    gauss_t g;
    if (!gauss_setup(S, c, o, ocam, i, &g)) return ORA_BAD_QUAT;
    double v[] = {g.valid, g.px, g.py, g.ca, g.cb, g.cc, g.S2a, g.S2b, g.S2c, g.sigma, g.d, g.eps,
                  g.rgb[0], g.rgb[1], g.rgb[2], g.x0, g.x1, g.y0, g.y1,
                  g.nrm[0], g.nrm[1], g.nrm[2], g.S1, g.S2, g.geo.s1, g.geo.s2};
    memcpy(out, v, sizeof v);
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* backward: analytic gradients of L = sum_pixels sum_ch dL_drgb * C           */
/* (Sec. 4.2: Gaussians and surfel SH are optimised, surfel geometry fixed).   */
/* The indicator of the depth test and the 1/255 clamp are piecewise constant, */
/* so they pass no gradient; the colour clamp max(0,.) passes gradient only    */
/* where its argument is positive.                                             */

static void sh_backward(int deg, const double *sh, const double *dir, double dist, const double *raw,
                        const double *dLdc, double *g_sh /* [K,3] */, double *g_pos /* or NULL */)
{
    double Y[16], dY[48];
    int K = (deg + 1) * (deg + 1);
    ora_sh_basis(deg, dir, Y, dY);
    double gd[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ++ch) {
        double gc = raw[ch] > 0.0 ? dLdc[ch] : 0.0;
        for (int k = 0; k < K; ++k) {
            g_sh[3*k + ch] = Y[k] * gc;
            for (int a = 0; a < 3; ++a) gd[a] += gc * sh[3*k + ch] * dY[3*k + a];
        }
    }
    if (g_pos && dist > 0.0) {
        /* dir = (o - p)/|o - p|:  d dir / d p = -(I - dir dir^T)/|o - p| */
        double pr = dot3(gd, dir);
        for (int a = 0; a < 3; ++a) g_pos[a] += -(gd[a] - pr * dir[a]) / dist;
    }
}

/* Rotation gradient: columns GR[:,k] = dL/d(R e_k) -> dL/dq through the
   normalised quaternion qhat = q/|q| and R(qhat). */
static void rot_backward(const double *GR, const double *qn, double qnorm, double *g_q)
{
    double w = qn[0], qx = qn[1], qy = qn[2], qz = qn[3];
    double dR[4][9] = {
        {0, -2*qz, 2*qy, 2*qz, 0, -2*qx, -2*qy, 2*qx, 0},
        {0, 2*qy, 2*qz, 2*qy, -4*qx, -2*w, 2*qz, 2*w, -4*qx},
        {-4*qy, 2*qx, 2*w, 2*qx, 0, 2*qz, -2*w, 2*qz, -4*qy},
        {-4*qz, -2*w, 2*qx, 2*w, -4*qz, 2*qy, 2*qx, 2*qy, 0},
    };
    double gqn[4];
    for (int a = 0; a < 4; ++a) {
        double acc = 0.0;
        for (int k = 0; k < 9; ++k) acc += GR[k] * dR[a][k];
        gqn[a] = acc;
    }
    double pr = gqn[0]*w + gqn[1]*qx + gqn[2]*qy + gqn[3]*qz;
    for (int a = 0; a < 4; ++a) g_q[a] = (gqn[a] - pr * qn[a]) / qnorm;
}

/* 2D Gaussian of 2D-GES (Sec. 6.4, Eq. 17-18), one primitive.  At a pixel
   whose ray d meets the splat plane at z = (N.t)/(N.d), X = z d - t,
   a = X.U / f1, b = X.V / f2 (U, V, N the camera-space frame, t the centre,
   f_k = s_k S_k the filtered scales), alpha = sigma0 / (S1 S2) exp(-(a^2 + b^2)/2).
   The per-pixel part gives dL/d(t, U, V, N, f1, f2, sigma); the object-space
   filter S1 = sqrt(1 + r M11/det M), S2 = sqrt(1 + r M00/det M) with M = J^T J,
   J = Jp(t) [s1 U, s2 V], then passes it on to t, U, V and s.  The depth test
   and the clamp are indicators (no gradient), eps_i included. */
static void gauss2d_backward(const ora_scene *S, const ora_camera *c, const ora_opts *o, const gauss_t *g,
                             int64_t gi, const double *dL_drgb, const double *rgb, const double *Ds,
                             const double *WG, const double *Rc, double *gp, double *g_rot, double *g_scale,
                             double *g_opac, double *g_sh)
{
    const int W = c->width;
    const int64_t HW = (int64_t)W * c->height;
    const int K = (S->sh_degree + 1) * (S->sh_degree + 1);
    const surf_t *f = &g->geo;
    double dc[3] = {0, 0, 0}, dsig = 0.0, gt[3] = {0, 0, 0}, gU[3] = {0, 0, 0}, gV[3] = {0, 0, 0};
    double gN[3] = {0, 0, 0}, gf1 = 0.0, gf2 = 0.0;
    for (int j = g->y0; j <= g->y1; ++j)
        for (int i = g->x0; i <= g->x1; ++i) {
            const int64_t pix = (int64_t)j * W + i;
            double d[3];
            pixel_ray(c, i, j, d);
            const double Nd = dot3(f->n, d);
            if (Nd == 0.0) continue;
            const double z = dot3(f->n, f->pc) / Nd;
            if (!(z > c->znear)) continue;
            double X[3];
            for (int q = 0; q < 3; ++q) X[q] = z * d[q] - f->pc[q];
            const double a = dot3(X, f->tu) / f->s1, b = dot3(X, f->tv) / f->s2;
            const double e = exp(-0.5 * (a*a + b*b)), al = g->sigma * e;
            if (!(al >= o->alpha_min) || !(z < Ds[pix] + g->eps)) continue;
            const double k = o->mode == 0 ? 1.0 / (1.0 + WG[pix]) : 1.0 / WG[pix];
            double gdotcC = 0.0;
            for (int ch = 0; ch < 3; ++ch) {
                const double gch = dL_drgb[ch * HW + pix];
                dc[ch] += al * k * gch;
                gdotcC += gch * (g->rgb[ch] - rgb[ch * HW + pix]);
            }
            const double dLda = k * gdotcC;
            dsig += dLda * e;
            const double dLdrho = dLda * al * (-0.5);
            const double dLa = dLdrho * 2.0 * a, dLb = dLdrho * 2.0 * b;
            const double Ud = dot3(f->tu, d), Vd = dot3(f->tv, d);
            /* dz/dt = N/Nd, dz/dN = -X/Nd, dX/dt = d (dz/dt)^T - I */
            for (int q = 0; q < 3; ++q) {
                gt[q] += dLa * ((Ud / Nd) * f->n[q] - f->tu[q]) / f->s1 +
                         dLb * ((Vd / Nd) * f->n[q] - f->tv[q]) / f->s2;
                gU[q] += dLa * X[q] / f->s1;
                gV[q] += dLb * X[q] / f->s2;
                gN[q] += -(dLa * Ud / f->s1 + dLb * Vd / f->s2) * X[q] / Nd;
            }
            gf1 += dLa * (-a / f->s1);
            gf2 += dLb * (-b / f->s2);
        }
    const double *s = S->g_scale + 2*gi;
    /* colour -> SH and position (through the view direction) */
    sh_backward(S->sh_degree, S->g_sh + (int64_t)3*K*gi, g->dir, g->dist, g->raw, dc, g_sh, gp);
    /* sigma = sigma0 / (S1 S2), f_k = s_k S_k */
    *g_opac = dsig / (g->S1 * g->S2);
    const double gS1 = gf1 * s[0] - dsig * g->sigma / g->S1, gS2 = gf2 * s[1] - dsig * g->sigma / g->S2;
    double gs0 = gf1 * g->S1, gs1 = gf2 * g->S2;
    /* rebuild J = Jp [s1 U, s2 V] and M = J^T J */
    const double x = g->t[0], y = g->t[1], z = g->t[2];
    const double Jp[6] = {c->fx / z, 0.0, -c->fx * x / (z*z), 0.0, c->fy / z, -c->fy * y / (z*z)};
    double JU[2], JV[2], J[4];
    for (int a = 0; a < 2; ++a) {
        JU[a] = dot3(Jp + 3*a, f->tu);
        JV[a] = dot3(Jp + 3*a, f->tv);
        J[2*a] = s[0] * JU[a];
        J[2*a + 1] = s[1] * JV[a];
    }
    const double M00 = J[0]*J[0] + J[2]*J[2], M01 = J[0]*J[1] + J[2]*J[3], M11 = J[1]*J[1] + J[3]*J[3];
    const double det = M00 * M11 - M01 * M01, r = o->lowpass, d2 = det * det;
    /* S1^2 = 1 + r M11/det, S2^2 = 1 + r M00/det */
    const double h1 = gS1 * r / (2.0 * g->S1), h2 = gS2 * r / (2.0 * g->S2);
    const double gM00 = h1 * (-M11 * M11 / d2) + h2 * (-M01 * M01 / d2);
    const double gM11 = h1 * (-M01 * M01 / d2) + h2 * (-M00 * M00 / d2);
    const double gM01 = h1 * (2.0 * M11 * M01 / d2) + h2 * (2.0 * M00 * M01 / d2);
    /* M = J^T J */
    double gJ[4];
    gJ[0] = 2.0 * J[0] * gM00 + J[1] * gM01;
    gJ[2] = 2.0 * J[2] * gM00 + J[3] * gM01;
    gJ[1] = J[0] * gM01 + 2.0 * J[1] * gM11;
    gJ[3] = J[2] * gM01 + 2.0 * J[3] * gM11;
    /* J[a][0] = s1 (Jp_a . U), J[a][1] = s2 (Jp_a . V) */
    double gJp[6];
    for (int a = 0; a < 2; ++a) {
        gs0 += gJ[2*a] * JU[a];
        gs1 += gJ[2*a + 1] * JV[a];
        for (int q = 0; q < 3; ++q) {
            gU[q] += s[0] * gJ[2*a] * Jp[3*a + q];
            gV[q] += s[1] * gJ[2*a + 1] * Jp[3*a + q];
            gJp[3*a + q] = s[0] * gJ[2*a] * f->tu[q] + s[1] * gJ[2*a + 1] * f->tv[q];
        }
    }
    g_scale[0] = gs0;
    g_scale[1] = gs1;
    /* Jp(t) -> t */
    gt[0] += gJp[2] * (-c->fx / (z*z));
    gt[1] += gJp[5] * (-c->fy / (z*z));
    gt[2] += gJp[0] * (-c->fx / (z*z)) + gJp[2] * (2.0 * c->fx * x / (z*z*z))
           + gJp[4] * (-c->fy / (z*z)) + gJp[5] * (2.0 * c->fy * y / (z*z*z));
    /* t = Rc p + tc; U, V, N = Rc R e_k:  world gradients through Rc^T */
    double GR[9];
    for (int q = 0; q < 3; ++q) {
        gp[q] += Rc[q]*gt[0] + Rc[3 + q]*gt[1] + Rc[6 + q]*gt[2];
        GR[3*q] = Rc[q]*gU[0] + Rc[3 + q]*gU[1] + Rc[6 + q]*gU[2];
        GR[3*q + 1] = Rc[q]*gV[0] + Rc[3 + q]*gV[1] + Rc[6 + q]*gV[2];
        GR[3*q + 2] = Rc[q]*gN[0] + Rc[3 + q]*gN[1] + Rc[6 + q]*gN[2];
    }
    rot_backward(GR, g->qn, g->qnorm, g_rot);
}

int ora_backward(const ora_scene *S, const ora_camera *c, const ora_opts *o, int nthreads,
                 const double *dL_drgb,
                 double *gg_pos, double *gg_rot, double *gg_scale, double *gg_opac, double *gg_sh,
                 double *gs_sh)
{
    if (!check_args(S, c, o)) return ORA_BAD_ARG;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    const int W = c->width, H = c->height;
    const int64_t HW = (int64_t)W * H, N = S->n_surfels, M = S->n_gaussians;
    const int D = S->gauss_dim == 2 ? 2 : 3;
    const int K = (S->sh_degree + 1) * (S->sh_degree + 1);
    double *rgb = malloc(sizeof(double) * 3 * (size_t)HW), *Ds = malloc(sizeof(double) * (size_t)HW);
    double *WG = malloc(sizeof(double) * (size_t)HW);
    const int nsamp = o->samples == 4 ? 4 : 1;
    int32_t *sid = malloc(sizeof(int32_t) * (size_t)HW * nsamp);
    uint8_t *amb = malloc((size_t)HW);
    double *gcs = calloc((size_t)(N > 0 ? N : 1) * 3, sizeof(double));
    if (!rgb || !Ds || !WG || !sid || !amb || !gcs) {
        free(rgb); free(Ds); free(WG); free(sid); free(amb); free(gcs);
        return ORA_NOMEM;
    }
    int st = ora_render(S, c, o, 1, nthreads, rgb, Ds, sid, WG, amb, NULL);
    if (st != ORA_OK) { free(rgb); free(Ds); free(WG); free(sid); free(amb); free(gcs); return st; }
    prep_t P;
    st = prepare(S, c, o, 1, &P);
    if (st != ORA_OK) { prep_free(&P); free(rgb); free(Ds); free(WG); free(sid); free(amb); free(gcs); return st; }
    double Rc[9];
    cam_rot(c, Rc);

    /* surfel colours: C depends on c_s through C_s at the samples the surfel
       wins, each weighing 1/samples in the resolve */
    if (o->mode != 2) {
        for (int smp = 0; smp < nsamp; ++smp)
            for (int64_t pix = 0; pix < HW; ++pix) {
                int32_t s = sid[smp * HW + pix];
                if (s < 0) continue;
                double k = (o->mode == 0 ? 1.0 / (1.0 + WG[pix]) : 1.0) / nsamp;
                for (int ch = 0; ch < 3; ++ch) gcs[3*s + ch] += k * dL_drgb[ch * HW + pix];
            }
    }
    memset(gs_sh, 0, sizeof(double) * 3 * (size_t)K * (size_t)N);
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) {
        const surf_t *sf = &P.sf[s];
        if (!sf->valid) continue;
        sh_backward(S->sh_degree, S->s_sh + (int64_t)3*K*s, sf->dir, 0.0, sf->raw, gcs + 3*s,
                    gs_sh + (int64_t)3*K*s, NULL);
    }

    memset(gg_pos, 0, sizeof(double) * 3 * (size_t)M);
    memset(gg_rot, 0, sizeof(double) * 4 * (size_t)M);
    memset(gg_scale, 0, sizeof(double) * D * (size_t)M);
    memset(gg_opac, 0, sizeof(double) * (size_t)M);
    memset(gg_sh, 0, sizeof(double) * 3 * (size_t)K * (size_t)M);
    if (o->mode != 1) {
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t gi = 0; gi < M; ++gi) {
            const gauss_t *g = &P.gs[gi];
            if (!g->valid) continue;
            if (g->dim == 2) {
                gauss2d_backward(S, c, o, g, gi, dL_drgb, rgb, Ds, WG, Rc, gg_pos + 3*gi, gg_rot + 4*gi,
                                 gg_scale + 2*gi, gg_opac + gi, gg_sh + (int64_t)3*K*gi);
                continue;
            }
            /* 2D-level gradients summed over the Gaussian's pixels */
            double dc[3] = {0, 0, 0}, dsig = 0, dpx = 0, dpy = 0, dca = 0, dcb = 0, dcc = 0;
            for (int j = g->y0; j <= g->y1; ++j) {
                for (int i = g->x0; i <= g->x1; ++i) {
                    int64_t pix = (int64_t)j * W + i;
                    double dx = (i + 0.5) - g->px, dy = (j + 0.5) - g->py;
                    double q = g->ca*dx*dx + 2.0*g->cb*dx*dy + g->cc*dy*dy;
                    double e = exp(-0.5 * q), a = g->sigma * e;
                    if (!(a >= o->alpha_min) || !(g->d < Ds[pix] + g->eps)) continue;
                    double k = o->mode == 0 ? 1.0 / (1.0 + WG[pix]) : 1.0 / WG[pix];
                    double gdotcC = 0.0;
                    for (int ch = 0; ch < 3; ++ch) {
                        double gch = dL_drgb[ch * HW + pix];
                        dc[ch] += a * k * gch;
                        gdotcC += gch * (g->rgb[ch] - rgb[ch * HW + pix]);
                    }
                    double dLda = k * gdotcC;
                    dsig += dLda * e;
                    double dLdq = dLda * a * (-0.5);
                    /* q = ca dx^2 + 2 cb dx dy + cc dy^2, dx = u - px */
                    dpx += dLdq * (-(2.0*g->ca*dx + 2.0*g->cb*dy));
                    dpy += dLdq * (-(2.0*g->cb*dx + 2.0*g->cc*dy));
                    dca += dLdq * dx * dx;
                    dcb += dLdq * 2.0 * dx * dy;
                    dcc += dLdq * dy * dy;
                }
            }
            const double *s = S->g_scale + 3*gi;
            double *gp = gg_pos + 3*gi;
            /* colour -> SH and position (through the view direction) */
            sh_backward(S->sh_degree, S->g_sh + (int64_t)3*K*gi, g->dir, g->dist, g->raw, dc,
                        gg_sh + (int64_t)3*K*gi, gp);
            /* sigma = sigma0 k3 k2 (Mip-GES factors; both 1 without the filters) */
            gg_opac[gi] = dsig * g->k3 * g->k2;
            const double dk2 = dsig * g->sigma0 * g->k3, dk3 = dsig * g->sigma0 * g->k2;
            /* conic Q = Sigma2^-1 (symmetric), dL/dQ as a symmetric matrix */
            double Q[4] = {g->ca, g->cb, g->cb, g->cc};
            double GQ[4] = {dca, 0.5*dcb, 0.5*dcb, dcc};
            double GS2[4];
            /* dL/dSigma2 = -Q GQ Q */
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    double acc = 0.0;
                    for (int k = 0; k < 2; ++k)
                        for (int l = 0; l < 2; ++l) acc += Q[2*a + k] * GQ[2*k + l] * Q[2*l + b];
                    GS2[2*a + b] = -acc;
                }
            /* screen filter: k2 = sqrt(det R2 / det Sigma2) with Sigma2 = R2 + lowpass I,
               d ln det A / dA = A^-1, so dk2/dR2 = (k2/2) (R2^-1 - Sigma2^-1) */
            if (o->filter == 1 && g->k2 > 0.0) {
                double d0 = g->R2a * g->R2c - g->R2b * g->R2b;
                double I0[4] = {g->R2c / d0, -g->R2b / d0, -g->R2b / d0, g->R2a / d0};
                for (int a = 0; a < 4; ++a) GS2[a] += dk2 * 0.5 * g->k2 * (I0[a] - Q[a]);
            }
            /* rebuild J, T = J Rc, Sigma3 */
            double x = g->t[0], y = g->t[1], z = g->t[2];
            double J[6] = {c->fx / z, 0.0, -c->fx * x / (z*z), 0.0, c->fy / z, -c->fy * y / (z*z)};
            double T[6], S3[9];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 3; ++b)
                    T[3*a + b] = J[3*a]*Rc[b] + J[3*a + 1]*Rc[3 + b] + J[3*a + 2]*Rc[6 + b];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; ++k) acc += g->R[3*a + k] * g->se[k] * g->se[k] * g->R[3*b + k];
                    S3[3*a + b] = acc;
                }
            /* Sigma2 = T S3 T^T (+ lowpass I):  dL/dS3 = T^T GS2 T,  dL/dT = 2 GS2 T S3 */
            double GS3[9], GT[6];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double acc = 0.0;
                    for (int k = 0; k < 2; ++k)
                        for (int l = 0; l < 2; ++l) acc += T[3*k + a] * GS2[2*k + l] * T[3*l + b];
                    GS3[3*a + b] = acc;
                }
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 3; ++b) {
                    double acc = 0.0;
                    for (int k = 0; k < 2; ++k)
                        for (int l = 0; l < 3; ++l) acc += GS2[2*a + k] * T[3*k + l] * S3[3*l + b];
                    GT[3*a + b] = 2.0 * acc;
                }
            /* T = J Rc:  dL/dJ = GT Rc^T */
            double GJ[6];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 3; ++b)
                    GJ[3*a + b] = GT[3*a]*Rc[3*b] + GT[3*a + 1]*Rc[3*b + 1] + GT[3*a + 2]*Rc[3*b + 2];
            /* camera-space centre: through J and the projected centre */
            double gt[3];
            gt[0] = GJ[2] * (-c->fx / (z*z)) + dpx * (c->fx / z);
            gt[1] = GJ[5] * (-c->fy / (z*z)) + dpy * (c->fy / z);
            gt[2] = GJ[0] * (-c->fx / (z*z)) + GJ[2] * (2.0 * c->fx * x / (z*z*z))
                  + GJ[4] * (-c->fy / (z*z)) + GJ[5] * (2.0 * c->fy * y / (z*z*z))
                  + dpx * (-c->fx * x / (z*z)) + dpy * (-c->fy * y / (z*z));
            /* t = Rc p + tc:  dL/dp += Rc^T gt */
            for (int a = 0; a < 3; ++a) gp[a] += Rc[a]*gt[0] + Rc[3 + a]*gt[1] + Rc[6 + a]*gt[2];
            /* S3 = Mm Mm^T with Mm = R diag(se), se = sqrt(s^2 + v):  dL/dMm = 2 GS3 Mm */
            double GM[9];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; ++k) acc += GS3[3*a + k] * g->R[3*k + b] * g->se[b];
                    GM[3*a + b] = 2.0 * acc;
                }
            double GR[9];
            const double v3 = S->g_filt3 ? S->g_filt3[gi] : 0.0;
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int a = 0; a < 3; ++a) { acc += GM[3*a + b] * g->R[3*a + b]; GR[3*a + b] = GM[3*a + b] * g->se[b]; }
                /* dse/ds = s/se;  k3 = prod |s_j|/se_j:  dk3/ds_j = k3 v / (s_j se_j^2) */
                double gs = v3 != 0.0 ? acc * s[b] / g->se[b] : acc;
                if (v3 != 0.0 && s[b] != 0.0) gs += dk3 * g->k3 * v3 / (s[b] * g->se[b] * g->se[b]);
                gg_scale[3*gi + b] = gs;
            }
            rot_backward(GR, g->qn, g->qnorm, gg_rot + 4*gi);
        }
    }
    prep_free(&P);
    free(rgb); free(Ds); free(WG); free(sid); free(amb); free(gcs);
    return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* translucent surfels (Sec. 4.1, Eq. 6-7): the differentiable surfel render  */
/* of the coarse stage.                                                        */
/* alpha_i = min(1, w_i G(a, b)), G = exp(-(a^2 + b^2)/2) at the ray-plane hit */
/* (a, b in scale units), clamped to 0 where min(alpha_i, G) < 1/255.  The     */
/* rasterisation follows 2DGS: front-to-back alpha blending in the order of    */
/* the surfel centres' camera depths (ties: lower index first), stopping once  */
/* the transmittance falls below 1e-4 after a blend; C += T bg at the end.     */
/* With front_first (the w_i >= 30 regime), each pixel blends its frontmost    */
/* covering surfel (least depth at the pixel, ties: lower index) first and the */
/* others in the sorted order.                                                 */

#define ORA_T_STOP 1e-4

typedef struct { int64_t s; double zc, z, a, G, rho; } tcontrib;

static int tcontrib_cmp(const void *pa, const void *pb)
{
    const tcontrib *a = pa, *b = pb;
    if (a->zc < b->zc) return -1;
    if (a->zc > b->zc) return 1;
    return (a->s > b->s) - (a->s < b->s);
}

/* Contributors of pixel (i, j) in blending order; returns their number, or -1
   when out of memory.  *list is grown with realloc.  amb gets AMB_COLOR where
   a decision sits within the bands (cut-off, blend order, front choice, near
   plane, grazing). */
static int64_t tcollect(const ora_scene *S, const ora_camera *c, const ora_opts *o, const prep_t *P, int culled,
                        const double *w, int front_first, int i, int j, tcontrib **list, int64_t *cap,
                        uint8_t *amb)
{
    double d[3];
    pixel_ray(c, i, j, d);
    const double amin = o->alpha_min;
    int64_t n = 0, lo = 0, hi = S->n_surfels;
    if (culled) {
        const int64_t cell = (int64_t)(j / ORA_CELL) * P->rs.cx + i / ORA_CELL;
        lo = P->rs.off[cell]; hi = P->rs.off[cell + 1];
    }
    for (int64_t t = lo; t < hi; ++t) {
        const int64_t s = culled ? P->rs.idx[t] : t;
        const surf_t *sf = &P->sf[s];
        if (!sf->valid) continue;
        if (culled && (i < sf->x0 || i > sf->x1 || j < sf->y0 || j > sf->y1)) continue;
        double z, rho, nd;
        if (!surfel_hit(sf, d, &z, &rho, &nd)) continue;
        if (!(z > c->znear)) continue;
        const double G = exp(-0.5 * rho), a = fmin(1.0, w[s] * G);
        const double m = fmin(a, G);
        if (fabs(m - amin) <= o->tol_alpha) *amb |= AMB_COLOR;
        if (!(m >= amin)) continue;
        if (fabs(nd) < o->tol_graze || fabs(z - c->znear) <= o->tol_depth_rel * fmax(1.0, c->znear)) *amb |= AMB_COLOR;
        if (n == *cap) {
            int64_t nc = *cap ? 2 * *cap : 64;
            tcontrib *nl = realloc(*list, sizeof(tcontrib) * (size_t)nc);
            if (!nl) return -1;
            *list = nl; *cap = nc;
        }
        (*list)[n++] = (tcontrib){s, sf->pc[2], z, a, G, rho};
    }
    qsort(*list, (size_t)n, sizeof(tcontrib), tcontrib_cmp);
    for (int64_t k = 1; k < n; ++k)
        if ((*list)[k].zc - (*list)[k - 1].zc <= o->tol_centre_rel * fabs((*list)[k].zc)) *amb |= AMB_COLOR;
    if (front_first && n > 1) {
        int64_t f = 0;
        for (int64_t k = 1; k < n; ++k)
            if ((*list)[k].z < (*list)[f].z || ((*list)[k].z == (*list)[f].z && (*list)[k].s < (*list)[f].s)) f = k;
        for (int64_t k = 0; k < n; ++k)
            if (k != f && (*list)[k].z - (*list)[f].z <= o->tol_depth_rel * (*list)[f].z) *amb |= AMB_COLOR;
        tcontrib fr = (*list)[f];
        memmove(*list + 1, *list, sizeof(tcontrib) * (size_t)f);
        (*list)[0] = fr;
    }
    return n;
}

int ora_render_translucent(const ora_scene *S, const ora_camera *c, const ora_opts *o, const double *w,
                           int front_first, int culled, int nthreads, double *rgb, double *T_out,
                           int32_t *front, int32_t *nblend, uint8_t *amb)
{
    if (!check_args(S, c, o) || !w) return ORA_BAD_ARG;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    prep_t P;
    int st = prepare(S, c, o, culled, &P);
    if (st != ORA_OK) { prep_free(&P); return st; }
    const int W = c->width, H = c->height;
    const int64_t HW = (int64_t)W * H;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(|:bad)
    for (int j = 0; j < H; ++j) {
        tcontrib *list = NULL;
        int64_t cap = 0;
        for (int i = 0; i < W; ++i) {
            const int64_t pix = (int64_t)j * W + i;
            uint8_t a8 = 0;
            const int64_t n = tcollect(S, c, o, &P, culled, w, front_first, i, j, &list, &cap, &a8);
            if (n < 0) { bad = 1; break; }
            double C[3] = {0, 0, 0}, T = 1.0;
            int32_t nb = 0;
            for (int64_t k = 0; k < n; ++k) {
                const tcontrib *e = &list[k];
                for (int ch = 0; ch < 3; ++ch) C[ch] += P.sf[e->s].rgb[ch] * e->a * T;
                T *= 1.0 - e->a;
                ++nb;
                if (fabs(T - ORA_T_STOP) <= 1e-6 * ORA_T_STOP) a8 |= AMB_COLOR;
                if (T < ORA_T_STOP) break;
            }
            for (int ch = 0; ch < 3; ++ch) rgb[ch * HW + pix] = C[ch] + T * c->bg[ch];
            T_out[pix] = T;
            /* the frontmost contributor (least depth at the pixel); another
               contributor within the depth band of it makes the choice
               ambiguous (either is a correct answer in finite precision) */
            int64_t f = -1;
            double fz = INFINITY;
            for (int64_t k = 0; k < n; ++k)
                if (list[k].z < fz || (list[k].z == fz && list[k].s < f)) { f = list[k].s; fz = list[k].z; }
            for (int64_t k = 0; k < n; ++k)
                if (list[k].s != f && list[k].z - fz <= o->tol_depth_rel * fz) a8 |= AMB_ID;
            front[pix] = (int32_t)f;
            nblend[pix] = nb;
            amb[pix] = a8;
        }
        free(list);
    }
    prep_free(&P);
    return bad ? ORA_NOMEM : ORA_OK;
}

/* Covering score (Sec. 4.1, pruning): the number of pixels at which each
   surfel is the frontmost contributor of the translucent render. */
int ora_covering_counts(const ora_scene *S, const ora_camera *c, const ora_opts *o, const double *w,
                        int64_t *counts)
{
    if (!check_args(S, c, o) || !w) return ORA_BAD_ARG;
    const int64_t HW = (int64_t)c->width * c->height;
    double *rgb = malloc(sizeof(double) * 3 * (size_t)HW), *T = malloc(sizeof(double) * (size_t)HW);
    int32_t *fr = malloc(sizeof(int32_t) * (size_t)HW), *nb = malloc(sizeof(int32_t) * (size_t)HW);
    uint8_t *amb = malloc((size_t)HW);
    int st = ORA_NOMEM;
    if (rgb && T && fr && nb && amb) st = ora_render_translucent(S, c, o, w, 1, 1, 0, rgb, T, fr, nb, amb);
    if (st == ORA_OK) {
        memset(counts, 0, sizeof(int64_t) * (size_t)(S->n_surfels > 0 ? S->n_surfels : 0));
        for (int64_t p = 0; p < HW; ++p)
            if (fr[p] >= 0) ++counts[fr[p]];
    }
    free(rgb); free(T); free(fr); free(nb); free(amb);
    return st;
}

/* Gradients of L = sum(dL_drgb * C) of the translucent render with respect to
   surfel position, rotation (through the normalisation), scales, w and SH.
   With T_i the transmittance before contributor i, S_{i+1} the colour seen
   behind it (S = c a + (1 - a) S, ending in bg): dC/dc_i = a_i T_i,
   dC/da_i = T_i (c_i - S_{i+1}); where w G < 1: da/dw = G, da/drho = -w G / 2,
   rho = a^2 + b^2; the hit coordinate a = ((z d - P).U)/s1 with
   z = (N.P)/(N.d) gives da/dP = ((U.d)/(N.d) N - U)/s1, da/dU = (z d - P)/s1,
   da/dN = (U.d)(P - z d)/((N.d) s1), da/ds1 = -a/s1 (b likewise with V, s2).
   The cut-off, the order and the early stop are piecewise constant. */
int ora_backward_translucent(const ora_scene *S, const ora_camera *c, const ora_opts *o, const double *w,
                             int front_first, int nthreads, const double *dL_drgb, double *gs_pos,
                             double *gs_rot, double *gs_scale, double *gs_w, double *gs_sh)
{
    if (!check_args(S, c, o) || !w) return ORA_BAD_ARG;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    prep_t P;
    int st = prepare(S, c, o, 1, &P);
    if (st != ORA_OK) { prep_free(&P); return st; }
    const int W = c->width, H = c->height;
    const int64_t HW = (int64_t)W * H, N = S->n_surfels;
    const int K = (S->sh_degree + 1) * (S->sh_degree + 1);
    /* per surfel, camera space: gP(3) gU(3) gV(3) gN(3) gs1 gs2 gw gc(3) = 18 */
    double *acc = calloc((size_t)(N > 0 ? N : 1) * 18, sizeof(double));
    if (!acc) { prep_free(&P); return ORA_NOMEM; }
    int bad = 0;
    /* rows are summed serially per row block to keep the result deterministic */
    for (int j = 0; j < H && !bad; ++j) {
        tcontrib *list = NULL;
        int64_t cap = 0;
        for (int i = 0; i < W; ++i) {
            const int64_t pix = (int64_t)j * W + i;
            uint8_t a8 = 0;
            const int64_t n = tcollect(S, c, o, &P, 1, w, front_first, i, j, &list, &cap, &a8);
            if (n < 0) { bad = 1; break; }
            int64_t nb = 0;
            double T = 1.0;
            for (int64_t k = 0; k < n; ++k) {
                T *= 1.0 - list[k].a;
                ++nb;
                if (T < ORA_T_STOP) break;
            }
            const double g[3] = {dL_drgb[pix], dL_drgb[HW + pix], dL_drgb[2 * HW + pix]};
            /* transmittances before each blended contributor */
            double *Tb = malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
            if (!Tb) { bad = 1; break; }
            T = 1.0;
            for (int64_t k = 0; k < nb; ++k) { Tb[k] = T; T *= 1.0 - list[k].a; }
            double Sb[3] = {c->bg[0], c->bg[1], c->bg[2]};
            double d[3];
            pixel_ray(c, i, j, d);
            for (int64_t k = nb - 1; k >= 0; --k) {
                const tcontrib *e = &list[k];
                const surf_t *sf = &P.sf[e->s];
                double *A = acc + 18 * e->s;
                double dLda = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    A[15 + ch] += e->a * Tb[k] * g[ch];
                    dLda += Tb[k] * (sf->rgb[ch] - Sb[ch]) * g[ch];
                }
                for (int ch = 0; ch < 3; ++ch) Sb[ch] = sf->rgb[ch] * e->a + (1.0 - e->a) * Sb[ch];
                if (!(w[e->s] * e->G < 1.0)) continue;        /* alpha clamped at 1: no gradient */
                A[14] += dLda * e->G;
                const double dLdrho = dLda * (-0.5 * w[e->s] * e->G);
                /* local coordinates and their derivatives */
                const double Nd = dot3(sf->n, d), Ud = dot3(sf->tu, d), Vd = dot3(sf->tv, d);
                const double z = e->z;
                double X[3];
                for (int q = 0; q < 3; ++q) X[q] = z * d[q] - sf->pc[q];
                const double a = dot3(X, sf->tu) / sf->s1, b = dot3(X, sf->tv) / sf->s2;
                const double dLa = dLdrho * 2.0 * a, dLb = dLdrho * 2.0 * b;
                for (int q = 0; q < 3; ++q) {
                    A[q] += dLa * ((Ud / Nd) * sf->n[q] - sf->tu[q]) / sf->s1 +
                            dLb * ((Vd / Nd) * sf->n[q] - sf->tv[q]) / sf->s2;
                    A[3 + q] += dLa * X[q] / sf->s1;
                    A[6 + q] += dLb * X[q] / sf->s2;
                    A[9 + q] += dLa * Ud * (-X[q]) / (Nd * sf->s1) + dLb * Vd * (-X[q]) / (Nd * sf->s2);
                }
                A[12] += dLa * (-a / sf->s1);
                A[13] += dLb * (-b / sf->s2);
            }
            free(Tb);
        }
        free(list);
    }
    if (bad) { free(acc); prep_free(&P); return ORA_NOMEM; }
    double Rc[9];
    cam_rot(c, Rc);
    for (int64_t s = 0; s < N; ++s) {
        const double *A = acc + 18 * s;
        double *gp = gs_pos + 3 * s;
        double R[9], qn[4], qnorm;
        for (int q = 0; q < 3; ++q) gp[q] = Rc[q] * A[0] + Rc[3 + q] * A[1] + Rc[6 + q] * A[2];
        for (int q = 0; q < 4; ++q) gs_rot[4 * s + q] = 0.0;
        gs_scale[2 * s] = A[12]; gs_scale[2 * s + 1] = A[13];
        gs_w[s] = A[14];
        memset(gs_sh + (int64_t)3 * K * s, 0, sizeof(double) * 3 * (size_t)K);
        const surf_t *sf = &P.sf[s];
        if (!sf->valid || !quat_rot(S->s_rot + 4 * s, R, qn, &qnorm)) continue;
        /* U = Rc R e_x, V = Rc R e_y, N = Rc R e_z:  dL/dR[:,k] = Rc^T g */
        double GR[9];
        for (int q = 0; q < 3; ++q) {
            GR[3 * q] = Rc[q] * A[3] + Rc[3 + q] * A[4] + Rc[6 + q] * A[5];
            GR[3 * q + 1] = Rc[q] * A[6] + Rc[3 + q] * A[7] + Rc[6 + q] * A[8];
            GR[3 * q + 2] = Rc[q] * A[9] + Rc[3 + q] * A[10] + Rc[6 + q] * A[11];
        }
        double wq = qn[0], qx = qn[1], qy = qn[2], qz = qn[3];
        double dR[4][9] = {
            {0, -2*qz, 2*qy, 2*qz, 0, -2*qx, -2*qy, 2*qx, 0},
            {0, 2*qy, 2*qz, 2*qy, -4*qx, -2*wq, 2*qz, 2*wq, -4*qx},
            {-4*qy, 2*qx, 2*wq, 2*qx, 0, 2*qz, -2*wq, 2*qz, -4*qy},
            {-4*qz, -2*wq, 2*qx, 2*wq, -4*qz, 2*qy, 2*qx, 2*qy, 0},
        };
        double gqn[4];
        for (int a = 0; a < 4; ++a) {
            double acc2 = 0.0;
            for (int k = 0; k < 9; ++k) acc2 += GR[k] * dR[a][k];
            gqn[a] = acc2;
        }
        double pr = gqn[0]*wq + gqn[1]*qx + gqn[2]*qy + gqn[3]*qz;
        for (int a = 0; a < 4; ++a) gs_rot[4 * s + a] = (gqn[a] - pr * qn[a]) / qnorm;
        /* colour -> SH and position (through the view direction) */
        double ocam[3], v[3];
        cam_centre(c, ocam);
        for (int q = 0; q < 3; ++q) v[q] = ocam[q] - S->s_pos[3 * s + q];
        sh_backward(S->sh_degree, S->s_sh + (int64_t)3 * K * s, sf->dir, sqrt(dot3(v, v)), sf->raw, A + 15,
                    gs_sh + (int64_t)3 * K * s, gp);
    }
    free(acc);
    prep_free(&P);
    return ORA_OK;
}

/* Contribution score of each Gaussian (Sec. 4.2, Eq. 9), for pruning:
   s_i = max over the pixels where Gaussian i contributes (clamp and depth
   test passed) of c_max alpha_i / (W_s + W_G), c_max its largest colour
   channel, W_s = 1; 0 where it contributes nowhere. */
int ora_contribution(const ora_scene *S, const ora_camera *c, const ora_opts *o, double *score)
{
    if (!check_args(S, c, o)) return ORA_BAD_ARG;
    const int W = c->width, H = c->height;
    const int64_t HW = (int64_t)W * H, M = S->n_gaussians;
    double *rgb = malloc(sizeof(double) * 3 * (size_t)HW), *Ds = malloc(sizeof(double) * (size_t)HW);
    double *WG = malloc(sizeof(double) * (size_t)HW);
    int32_t *sid = malloc(sizeof(int32_t) * (size_t)HW * (o->samples == 4 ? 4 : 1));
    uint8_t *amb = malloc((size_t)HW);
    if (!rgb || !Ds || !WG || !sid || !amb) { free(rgb); free(Ds); free(WG); free(sid); free(amb); return ORA_NOMEM; }
    int st = ora_render(S, c, o, 1, 0, rgb, Ds, sid, WG, amb, NULL);
    prep_t P;
    if (st == ORA_OK) st = prepare(S, c, o, 1, &P);
    else memset(&P, 0, sizeof P);
    if (st == ORA_OK) {
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t k = 0; k < M; ++k) {
            const gauss_t *g = &P.gs[k];
            double best = 0.0;
            if (g->valid) {
                const double cm = fmax(g->rgb[0], fmax(g->rgb[1], g->rgb[2]));
                for (int j = g->y0; j <= g->y1; ++j)
                    for (int i = g->x0; i <= g->x1; ++i) {
                        const int64_t pix = (int64_t)j * W + i;
                        double gd;
                        const double a = gauss_eval(c, g, i, j, &gd, NULL);
                        if (!(a >= o->alpha_min) || !(gd < Ds[pix] + g->eps)) continue;
                        best = fmax(best, cm * a / (1.0 + WG[pix]));
                    }
            }
            score[k] = best;
        }
    }
    prep_free(&P);
    free(rgb); free(Ds); free(WG); free(sid); free(amb);
    return st;
}

/* Mip-GES 3D filter variance per Gaussian (Sec. 6.1, Mip-Splatting's world-space
   filter): v_i = s3d / nu_i^2 with nu_i the highest sampling rate at which the
   training cameras see the centre, nu = max(fx, fy) / z over the cameras whose
   image rectangle [0,W] x [0,H] contains the projected centre at z > znear.  A
   Gaussian no camera sees gets the largest v among those seen (0 if none is). */
int ora_filter3d(const ora_scene *S, const ora_camera *cams, int n_cams, double s3d, double *out_v)
{
    if (!S || !cams || n_cams <= 0 || !(s3d >= 0.0) || S->n_gaussians < 0) return ORA_BAD_ARG;
    double vmax = 0.0;
    int any = 0;
    for (int64_t i = 0; i < S->n_gaussians; ++i) {
        double nu = 0.0;
        for (int k = 0; k < n_cams; ++k) {
            const ora_camera *c = &cams[k];
            double t[3];
            cam_to_camera(c, S->g_pos + 3*i, t);
            if (!(t[2] > c->znear)) continue;
            double u = c->fx * t[0] / t[2] + c->cx, v = c->fy * t[1] / t[2] + c->cy;
            if (!(u >= 0.0 && u <= c->width && v >= 0.0 && v <= c->height)) continue;
            nu = fmax(nu, fmax(c->fx, c->fy) / t[2]);
        }
        if (nu > 0.0) {
            out_v[i] = s3d / (nu * nu);
            vmax = any ? fmax(vmax, out_v[i]) : out_v[i];
            any = 1;
        } else {
            out_v[i] = -1.0;
        }
    }
    for (int64_t i = 0; i < S->n_gaussians; ++i)
        if (out_v[i] < 0.0) out_v[i] = any ? vmax : 0.0;
    return ORA_OK;
}

int ora_version(void) { return 1; }
