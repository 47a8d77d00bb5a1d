/*
 * pvg_oracle.c -- plain, slow FP64 CPU oracle of the PVG renderer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library; the product
 * (the CUDA path behind include/pvg.h) never calls it and shares no code,
 * header, table or constant with it.
 *
 * What it computes, step by step, and the passage each step follows
 * (Periodic Vibration Gaussian, arXiv 2311.18561):
 *
 *   1. Time evaluation (Sec. 3.2, Eq. 6 and Eq. 7):
 *        mu~(t) = mu + l/(2 pi) sin(2 pi (t - tau)/l) v
 *        o~(t)  = o exp(-(t - tau)^2 / (2 beta^2))
 *   2. View transform p = W mu~ + t_c and the near-plane / opacity culls
 *      (Sec. 3.1: the Gaussians are ordered by camera-space depth).
 *   3. 3D covariance Sigma = R(q) diag(s)^2 R(q)^T (Sec. 3.1, the scaling /
 *      unit-quaternion decomposition) and the EWA projection
 *      Sigma' = J W Sigma W^T J^T (Sec. 3.1, Eq. 2), plus a low-pass
 *      dilation h I (a 3DGS convention the paper inherits; h is an option).
 *   4. Colour c from real spherical harmonics (the colour c of Sec. 3.1;
 *      SH is the 3DGS convention the paper inherits), orthonormal basis with
 *      the Condon-Shortley phase, evaluated at the viewing direction, +0.5,
 *      clamped at 0.
 *   5. Per pixel, front-to-back alpha blending over all surviving Gaussians
 *      ordered by (camera depth, index) (Sec. 3.1, Eq. 3), alpha = o~ G_2D,
 *      with the depth and opacity channels Sec. 3.1 renders beside
 *      colour and the opacity O = sum T alpha of the sky step of Sec. 3.4.  Gates (3DGS conventions, options here): alpha capped
 *      at 0.99, alpha < 1/255 skipped, stop before a Gaussian whose blend
 *      would leave T (1 - alpha) < 1e-4.  Finally C += T bg.
 *   6. Culled mode: identical result, but a Gaussian is only considered for
 *      pixels inside its box |x - u| <= sqrt(Q Sigma'_xx),
 *      |y - v| <= sqrt(Q Sigma'_yy), Q = 2 ln(255 o~); outside that box
 *      o~ G_2D < 1/255, so the skipped evaluations could not have blended.
 *   7. Backward: exact FP64 reverse mode of steps 1-5 (the render function
 *      is differentiable, Sec. 3.1 Eq. 4 and Sec. 3.2 Eq. 8).
 *   8. Extra channels composited with the same weights T_i alpha_i and no
 *      background: the average velocity v_bar = v exp(-rho/2) (Eq. 10; its
 *      rendered map is the velocity map of Sec. 3.4 and Sec. 4), the
 *      staticness rho = beta / l clamped to [0, 2] (the rho map of the
 *      dynamic-element analysis) and a per-Gaussian semantic vector
 *      (semantic rendering, 19 classes in the paper), with their reverse
 *      mode.
 *
 * Parameters are physical values (s > 0, o in (0,1), beta > 0, l > 0);
 * the quaternion (w,x,y,z) need not be normalised and is normalised here.
 * Camera: world->camera 3x4 row-major [R | t] with OpenCV axes, pixel
 * (px, py) sampled at (px + 0.5, py + 0.5).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI (2.0 * M_PI)

/* camera array layout: viewmat[12], fx, fy, cx, cy, width, height, t,
 * z_near, bg0, bg1, bg2, dt (temporal-smoothing shift, 0 = plain render) */
enum { CAM_FX = 12, CAM_FY, CAM_CX, CAM_CY, CAM_W, CAM_H, CAM_T, CAM_ZNEAR, CAM_BG, CAM_DT = CAM_BG + 3,
       CAM_LEN = CAM_DT + 1 };
/* option array layout */
enum { OPT_H = 0, OPT_ACAP, OPT_AMIN, OPT_TSTOP, OPT_FOVCLAMP, OPT_LEN };

typedef struct {
    int valid;
    double delta, theta, sin_t, cos_t, egate; /* time terms */
    double dt, vbar_w;                        /* flow shift and exp(-rho / 2) */
    double mut[3], ot;                        /* mu~(t), o~(t) */
    double p[3];                              /* camera-space mean */
    int clamp_x, clamp_y;                     /* -1, 0, +1 */
    double txc, tyc;                          /* clamped x, y used in J */
    double J[2][3];
    double qn[4], qlen, R[3][3];
    double Sigma[3][3], M[3][3];
    double cov2[3];                           /* A, B, C (with dilation) */
    double det, conic[3];                     /* a, b, c */
    double uv[2], z;
    double dir[3], dist;                      /* unit view direction */
    double rgb_raw[3], rgb[3];
    double rx, ry;                            /* culled-mode box half extents */
} gauss_t;

typedef struct {
    int64_t n;
    int degree;
    const double *mu, *vel, *tau, *beta, *period, *scale, *quat, *opac, *sh;
} scene_t;

/* ------------------------------------------------------------------ */
/* real spherical harmonics, degree <= 3                               */
/* ------------------------------------------------------------------ */
/* Normalisation factors from the textbook expression
 * N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (x sqrt 2 for m != 0),
 * multiplied out for each polynomial below. */
static void sh_consts(double c[16])
{
    c[0] = 0.5 * sqrt(1.0 / M_PI);            /* Y00 */
    c[1] = sqrt(3.0 / (4.0 * M_PI));          /* l = 1 */
    c[2] = 0.5 * sqrt(15.0 / M_PI);           /* xy, yz, xz */
    c[3] = 0.25 * sqrt(5.0 / M_PI);           /* 3z^2 - 1 */
    c[4] = 0.25 * sqrt(15.0 / M_PI);          /* x^2 - y^2 */
    c[5] = 0.25 * sqrt(35.0 / (2.0 * M_PI));  /* y(3x^2-y^2), x(x^2-3y^2) */
    c[6] = 0.5 * sqrt(105.0 / M_PI);          /* xyz */
    c[7] = 0.25 * sqrt(21.0 / (2.0 * M_PI));  /* y(5z^2-1), x(5z^2-1) */
    c[8] = 0.25 * sqrt(7.0 / M_PI);           /* z(5z^2-3) */
    c[9] = 0.25 * sqrt(105.0 / M_PI);         /* z(x^2-y^2) */
}

/* Y[k] for k = l^2 + l + m, m = -l..l, at the unit vector (x, y, z); if dY
 * is given, also the gradient of each polynomial w.r.t. (x, y, z). */
static void sh_basis(int degree, const double d[3], double *Y, double (*dY)[3])
{
    double c[16];
    sh_consts(c);
    const double x = d[0], y = d[1], z = d[2];
    int K = (degree + 1) * (degree + 1);
    for (int k = 0; k < K; k++) {
        Y[k] = 0.0;
        if (dY) dY[k][0] = dY[k][1] = dY[k][2] = 0.0;
    }
#define SETG(k, gx, gy, gz) do { if (dY) { dY[k][0] = (gx); dY[k][1] = (gy); dY[k][2] = (gz); } } while (0)
    Y[0] = c[0];
    if (degree < 1) return;
    Y[1] = -c[1] * y;  SETG(1, 0, -c[1], 0);
    Y[2] = c[1] * z;   SETG(2, 0, 0, c[1]);
    Y[3] = -c[1] * x;  SETG(3, -c[1], 0, 0);
    if (degree < 2) return;
    Y[4] = c[2] * x * y;                       SETG(4, c[2] * y, c[2] * x, 0);
    Y[5] = -c[2] * y * z;                      SETG(5, 0, -c[2] * z, -c[2] * y);
    Y[6] = c[3] * (2 * z * z - x * x - y * y); SETG(6, -2 * c[3] * x, -2 * c[3] * y, 4 * c[3] * z);
    Y[7] = -c[2] * x * z;                      SETG(7, -c[2] * z, 0, -c[2] * x);
    Y[8] = c[4] * (x * x - y * y);             SETG(8, 2 * c[4] * x, -2 * c[4] * y, 0);
    if (degree < 3) return;
    Y[9] = -c[5] * y * (3 * x * x - y * y);
    SETG(9, -c[5] * 6 * x * y, -c[5] * (3 * x * x - 3 * y * y), 0);
    Y[10] = c[6] * x * y * z;
    SETG(10, c[6] * y * z, c[6] * x * z, c[6] * x * y);
    Y[11] = -c[7] * y * (4 * z * z - x * x - y * y);
    SETG(11, -c[7] * (-2 * x * y), -c[7] * (4 * z * z - x * x - 3 * y * y), -c[7] * 8 * y * z);
    Y[12] = c[8] * z * (2 * z * z - 3 * x * x - 3 * y * y);
    SETG(12, c[8] * (-6 * x * z), c[8] * (-6 * y * z), c[8] * (6 * z * z - 3 * x * x - 3 * y * y));
    Y[13] = -c[7] * x * (4 * z * z - x * x - y * y);
    SETG(13, -c[7] * (4 * z * z - 3 * x * x - y * y), -c[7] * (-2 * x * y), -c[7] * 8 * x * z);
    Y[14] = c[9] * z * (x * x - y * y);
    SETG(14, c[9] * 2 * x * z, -c[9] * 2 * y * z, c[9] * (x * x - y * y));
    Y[15] = -c[5] * x * (x * x - 3 * y * y);
    SETG(15, -c[5] * (3 * x * x - 3 * y * y), -c[5] * (-6 * x * y), 0);
#undef SETG
}

/* ------------------------------------------------------------------ */
/* step 1: time evaluation (Eq. 6, Eq. 7)                             */
/* ------------------------------------------------------------------ */
/* With dt != 0 this is the flow-translated state of the temporal
 * smoothing of Sec. 3.4: the point is queried at t - dt and
 * moved by the average velocity v_bar = v exp(-rho / 2), rho = beta / l
 * (Eq. 10), times dt; its opacity is the one at t - dt. */
static void time_eval(const scene_t *S, int64_t i, double t, double dt, gauss_t *g)
{
    const double l = S->period[i], b = S->beta[i];
    g->dt = dt;
    g->delta = (t - dt) - S->tau[i];
    g->theta = TWO_PI * g->delta / l;
    g->sin_t = sin(g->theta);
    g->cos_t = cos(g->theta);
    g->vbar_w = exp(-0.5 * b / l);
    const double amp = l / TWO_PI * g->sin_t + dt * g->vbar_w;
    for (int k = 0; k < 3; k++)
        g->mut[k] = S->mu[3 * i + k] + amp * S->vel[3 * i + k];
    g->egate = exp(-0.5 * g->delta * g->delta / (b * b));
    g->ot = S->opac[i] * g->egate;
}

static void quat_to_rot(const double q[4], double R[3][3])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* steps 1-4 for Gaussian i; g->valid = 0 if culled */
static void preprocess_one(const scene_t *S, int64_t i, const double *cam, const double *opt, gauss_t *g)
{
    memset(g, 0, sizeof(*g));
    time_eval(S, i, cam[CAM_T], cam[CAM_DT], g);
    const double *V = cam; /* row-major 3x4 */
    for (int r = 0; r < 3; r++)
        g->p[r] = V[4 * r + 0] * g->mut[0] + V[4 * r + 1] * g->mut[1] + V[4 * r + 2] * g->mut[2] + V[4 * r + 3];
    g->z = g->p[2];
    if (g->p[2] <= cam[CAM_ZNEAR]) return;
    if (g->ot < opt[OPT_AMIN]) return;

    /* Sigma = R diag(s^2) R^T */
    double qq = 0.0;
    for (int k = 0; k < 4; k++) qq += S->quat[4 * i + k] * S->quat[4 * i + k];
    g->qlen = sqrt(qq);
    for (int k = 0; k < 4; k++) g->qn[k] = S->quat[4 * i + k] / g->qlen;
    quat_to_rot(g->qn, g->R);
    const double *s = &S->scale[3 * i];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += g->R[a][k] * s[k] * s[k] * g->R[b][k];
            g->Sigma[a][b] = acc;
        }
    /* M = W Sigma W^T with W the rotation part of the view matrix */
    double WS[3][3];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += V[4 * a + k] * g->Sigma[k][b];
            WS[a][b] = acc;
        }
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += WS[a][k] * V[4 * b + k];
            g->M[a][b] = acc;
        }
    /* Jacobian of the perspective map at p, with x/z and y/z clamped to the
     * widened frustum */
    const double fx = cam[CAM_FX], fy = cam[CAM_FY];
    const double limx = opt[OPT_FOVCLAMP] * 0.5 * cam[CAM_W] / fx;
    const double limy = opt[OPT_FOVCLAMP] * 0.5 * cam[CAM_H] / fy;
    const double x = g->p[0], y = g->p[1], z = g->p[2];
    double rxz = x / z, ryz = y / z;
    g->clamp_x = rxz < -limx ? -1 : (rxz > limx ? 1 : 0);
    g->clamp_y = ryz < -limy ? -1 : (ryz > limy ? 1 : 0);
    if (g->clamp_x) rxz = g->clamp_x * limx;
    if (g->clamp_y) ryz = g->clamp_y * limy;
    g->txc = rxz * z;
    g->tyc = ryz * z;
    g->J[0][0] = fx / z; g->J[0][1] = 0.0;    g->J[0][2] = -fx * g->txc / (z * z);
    g->J[1][0] = 0.0;    g->J[1][1] = fy / z; g->J[1][2] = -fy * g->tyc / (z * z);
    double JM[2][3];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 3; b++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += g->J[a][k] * g->M[k][b];
            JM[a][b] = acc;
        }
    double C2[2][2];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += JM[a][k] * g->J[b][k];
            C2[a][b] = acc;
        }
    g->cov2[0] = C2[0][0] + opt[OPT_H];
    g->cov2[1] = 0.5 * (C2[0][1] + C2[1][0]);
    g->cov2[2] = C2[1][1] + opt[OPT_H];
    g->det = g->cov2[0] * g->cov2[2] - g->cov2[1] * g->cov2[1];
    if (!(g->det > 0.0)) return;
    g->conic[0] = g->cov2[2] / g->det;
    g->conic[1] = -g->cov2[1] / g->det;
    g->conic[2] = g->cov2[0] / g->det;
    g->uv[0] = fx * x / z + cam[CAM_CX];
    g->uv[1] = fy * y / z + cam[CAM_CY];

    /* colour from SH at the direction camera centre -> mu~ */
    double cc[3]; /* camera centre = -R^T t */
    for (int k = 0; k < 3; k++)
        cc[k] = -(V[0 + k] * V[3] + V[4 + k] * V[7] + V[8 + k] * V[11]);
    double dd[3], dn = 0.0;
    for (int k = 0; k < 3; k++) { dd[k] = g->mut[k] - cc[k]; dn += dd[k] * dd[k]; }
    g->dist = sqrt(dn);
    for (int k = 0; k < 3; k++) g->dir[k] = dd[k] / g->dist;
    double Y[16];
    sh_basis(S->degree, g->dir, Y, NULL);
    const int K = (S->degree + 1) * (S->degree + 1);
    for (int ch = 0; ch < 3; ch++) {
        double acc = 0.0;
        for (int k = 0; k < K; k++) acc += S->sh[(i * K + k) * 3 + ch] * Y[k];
        g->rgb_raw[ch] = acc + 0.5;
        g->rgb[ch] = g->rgb_raw[ch] > 0.0 ? g->rgb_raw[ch] : 0.0;
    }
    /* box of step 6 */
    const double Q = 2.0 * log(g->ot / opt[OPT_AMIN]);
    g->rx = sqrt(Q > 0 ? Q * g->cov2[0] : 0.0);
    g->ry = sqrt(Q > 0 ? Q * g->cov2[2] : 0.0);
    g->valid = 1;
}

static scene_t make_scene(int64_t n, int degree, const double *mu, const double *vel, const double *tau,
                          const double *beta, const double *period, const double *scale,
                          const double *quat, const double *opac, const double *sh)
{
    scene_t S = {n, degree, mu, vel, tau, beta, period, scale, quat, opac, sh};
    return S;
}

/* sort key for the depth order: (z ascending, index ascending) */
typedef struct { double z; int64_t idx; } zkey_t;
static int cmp_zkey(const void *a, const void *b)
{
    const zkey_t *x = (const zkey_t *)a, *y = (const zkey_t *)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* valid Gaussians in depth order; returns count, list in *out (malloc) */
static int64_t depth_order(const gauss_t *G, int64_t n, int64_t **out)
{
    zkey_t *keys = (zkey_t *)malloc(sizeof(zkey_t) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        if (G[i].valid) { keys[m].z = G[i].z; keys[m].idx = i; m++; }
    qsort(keys, (size_t)m, sizeof(zkey_t), cmp_zkey);
    *out = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t j = 0; j < m; j++) (*out)[j] = keys[j].idx;
    free(keys);
    return m;
}

static void preprocess_all(const scene_t *S, const double *cam, const double *opt, gauss_t *G)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < S->n; i++) preprocess_one(S, i, cam, opt, &G[i]);
}

/* alpha of Gaussian g at sample point (sx, sy); also G_2D and the offsets */
static double eval_alpha(const gauss_t *g, double sx, double sy, const double *opt,
                         double *Gout, double *dx, double *dy, int *capped)
{
    *dx = sx - g->uv[0];
    *dy = sy - g->uv[1];
    const double power = -0.5 * (g->conic[0] * *dx * *dx + g->conic[2] * *dy * *dy) - g->conic[1] * *dx * *dy;
    *Gout = exp(power);
    const double a = g->ot * *Gout;
    *capped = a > opt[OPT_ACAP];
    return *capped ? opt[OPT_ACAP] : a;
}

/* ------------------------------------------------------------------ */
/* exported: step 1 alone                                              */
/* ------------------------------------------------------------------ */
int pvgo_time_eval(int64_t n, const double *mu, const double *vel, const double *tau, const double *beta,
                   const double *period, const double *opac, double t, double dt, double *out_mut, double *out_ot)
{
    scene_t S = make_scene(n, 0, mu, vel, tau, beta, period, NULL, NULL, opac, NULL);
    for (int64_t i = 0; i < n; i++) {
        gauss_t g;
        time_eval(&S, i, t, dt, &g);
        for (int k = 0; k < 3; k++) out_mut[3 * i + k] = g.mut[k];
        out_ot[i] = g.ot;
    }
    return 0;
}

/* exported: SH basis values (and gradients) at unit directions */
int pvgo_sh_basis(int degree, int64_t n, const double *dirs, double *out_Y, double *out_dY)
{
    if (degree < 0 || degree > 3) return -1;
    const int K = (degree + 1) * (degree + 1);
    for (int64_t i = 0; i < n; i++) {
        double Y[16], dY[16][3];
        sh_basis(degree, &dirs[3 * i], Y, dY);
        for (int k = 0; k < K; k++) {
            out_Y[i * K + k] = Y[k];
            if (out_dY)
                for (int c = 0; c < 3; c++) out_dY[(i * K + k) * 3 + c] = dY[k][c];
        }
    }
    return 0;
}

/* exported: steps 1-4 per Gaussian.  Outputs (each may be NULL):
 * valid[n] int32, mut[n,3], ot[n], pcam[n,3], uv[n,2], cov2[n,3] (A,B,C),
 * conic[n,3], rgb[n,3], box[n,2] (rx, ry). */
int pvgo_preprocess(int64_t n, int degree, const double *mu, const double *vel, const double *tau,
                    const double *beta, const double *period, const double *scale, const double *quat,
                    const double *opac, const double *sh, const double *cam, const double *opt,
                    int32_t *valid, double *mut, double *ot, double *pcam, double *uv, double *cov2,
                    double *conic, double *rgb, double *box)
{
    if (degree < 0 || degree > 3 || n < 0) return -1;
    scene_t S = make_scene(n, degree, mu, vel, tau, beta, period, scale, quat, opac, sh);
    gauss_t *G = (gauss_t *)malloc(sizeof(gauss_t) * (size_t)(n > 0 ? n : 1));
    preprocess_all(&S, cam, opt, G);
    for (int64_t i = 0; i < n; i++) {
        const gauss_t *g = &G[i];
        if (valid) valid[i] = g->valid;
        for (int k = 0; k < 3; k++) {
            if (mut) mut[3 * i + k] = g->mut[k];
            if (pcam) pcam[3 * i + k] = g->p[k];
            if (cov2) cov2[3 * i + k] = g->cov2[k];
            if (conic) conic[3 * i + k] = g->conic[k];
            if (rgb) rgb[3 * i + k] = g->rgb[k];
        }
        if (ot) ot[i] = g->ot;
        if (uv) { uv[2 * i] = g->uv[0]; uv[2 * i + 1] = g->uv[1]; }
        if (box) { box[2 * i] = g->rx; box[2 * i + 1] = g->ry; }
    }
    free(G);
    return 0;
}

/* ------------------------------------------------------------------ */
/* step 5 / 6: per-pixel compositing                                   */
/* ------------------------------------------------------------------ */
static int near_gate(double v, double thr) { return fabs(v - thr) <= 1e-5 * thr; }

/* ------------------------------------------------------------------ */
/* sky cube map (Sec. 3.4, sky refinement)                             */
/* ------------------------------------------------------------------ */
/* Background C_f = C + (1 - O) f_sky(d): d is the world direction of the
 * pixel's ray (sample point jittered by jitter[2][H][W] pixels if given),
 * f_sky a cube map of 6 faces x res x res RGB texels, faces +X -X +Y -Y +Z
 * -Z, face coordinates of the OpenGL cube-map convention, bilinear
 * filtering inside a face with edge texels clamped. */
typedef struct { const double *tex; int res; const double *jitter; } sky_t;

static void sky_texels(const sky_t *K, const double *cam, int px, int py, int64_t idx[4], double w[4])
{
    const int W = (int)cam[CAM_W], H = (int)cam[CAM_H];
    double sx = px + 0.5, sy = py + 0.5;
    if (K->jitter) {
        sx += K->jitter[(int64_t)py * W + px];
        sy += K->jitter[(int64_t)H * W + (int64_t)py * W + px];
    }
    const double dc[3] = {(sx - cam[CAM_CX]) / cam[CAM_FX], (sy - cam[CAM_CY]) / cam[CAM_FY], 1.0};
    double d[3];
    for (int k = 0; k < 3; k++) d[k] = cam[0 + k] * dc[0] + cam[4 + k] * dc[1] + cam[8 + k] * dc[2];
    const double ax = fabs(d[0]), ay = fabs(d[1]), az = fabs(d[2]);
    int face;
    double sc, tc, ma;
    if (ax >= ay && ax >= az) {
        ma = ax;
        if (d[0] > 0) { face = 0; sc = -d[2]; tc = -d[1]; } else { face = 1; sc = d[2]; tc = -d[1]; }
    } else if (ay >= az) {
        ma = ay;
        if (d[1] > 0) { face = 2; sc = d[0]; tc = d[2]; } else { face = 3; sc = d[0]; tc = -d[2]; }
    } else {
        ma = az;
        if (d[2] > 0) { face = 4; sc = d[0]; tc = -d[1]; } else { face = 5; sc = -d[0]; tc = -d[1]; }
    }
    const double s = 0.5 * (sc / ma + 1.0), t = 0.5 * (tc / ma + 1.0);
    const int R = K->res;
    const double x = s * R - 0.5, y = t * R - 0.5;
    const double x0f = floor(x), y0f = floor(y);
    const double fx = x - x0f, fy = y - y0f;
    int x0 = (int)x0f, y0 = (int)y0f, x1 = x0 + 1, y1 = y0 + 1;
    x0 = x0 < 0 ? 0 : (x0 > R - 1 ? R - 1 : x0);
    x1 = x1 < 0 ? 0 : (x1 > R - 1 ? R - 1 : x1);
    y0 = y0 < 0 ? 0 : (y0 > R - 1 ? R - 1 : y0);
    y1 = y1 < 0 ? 0 : (y1 > R - 1 ? R - 1 : y1);
    const int64_t base = (int64_t)face * R * R;
    idx[0] = base + (int64_t)y0 * R + x0; w[0] = (1 - fx) * (1 - fy);
    idx[1] = base + (int64_t)y0 * R + x1; w[1] = fx * (1 - fy);
    idx[2] = base + (int64_t)y1 * R + x0; w[2] = (1 - fx) * fy;
    idx[3] = base + (int64_t)y1 * R + x1; w[3] = fx * fy;
}

static void sky_value(const sky_t *K, const double *cam, int px, int py, double out[3])
{
    int64_t idx[4];
    double w[4];
    sky_texels(K, cam, px, py, idx, w);
    for (int c = 0; c < 3; c++) {
        out[c] = 0.0;
        for (int k = 0; k < 4; k++) out[c] += w[k] * K->tex[idx[k] * 3 + c];
    }
}

/* ------------------------------------------------------------------ */
/* step 8: extra composited channels                                   */
/* ------------------------------------------------------------------ */
/* Channel order: v_bar (3, world frame) if FEAT_VBAR, rho clamped to
 * [0, 2] (1) if FEAT_RHO, the n_sem semantic values if FEAT_SEM. */
enum { FEAT_VBAR = 1, FEAT_RHO = 2, FEAT_SEM = 4 };
typedef struct { int mask, n_sem, F; const double *sem; } feat_t;

static int feat_count(int mask, int n_sem)
{
    return ((mask & FEAT_VBAR) ? 3 : 0) + ((mask & FEAT_RHO) ? 1 : 0) + ((mask & FEAT_SEM) ? n_sem : 0);
}

static void feat_values(const scene_t *S, int64_t i, const feat_t *Fs, double *f)
{
    int c = 0;
    const double rho = S->beta[i] / S->period[i];
    if (Fs->mask & FEAT_VBAR) {
        const double w = exp(-0.5 * rho);
        for (int k = 0; k < 3; k++) f[c++] = S->vel[3 * i + k] * w;
    }
    if (Fs->mask & FEAT_RHO) f[c++] = rho < 2.0 ? rho : 2.0;
    if (Fs->mask & FEAT_SEM)
        for (int k = 0; k < Fs->n_sem; k++) f[c++] = Fs->sem[i * Fs->n_sem + k];
}

/* adjoint of feat_values for Gaussian i given dL/df */
static void feat_backward(const scene_t *S, int64_t i, const feat_t *Fs, const double *gf, double *dvel,
                          double *dbeta, double *dperiod, double *dsem)
{
    int c = 0;
    const double l = S->period[i], b = S->beta[i], rho = b / l;
    if (Fs->mask & FEAT_VBAR) {
        /* v_bar = v exp(-rho / 2): d/dv = exp(-rho/2), d/drho = -v_bar / 2 */
        const double w = exp(-0.5 * rho);
        double gr = 0.0;
        for (int k = 0; k < 3; k++) {
            dvel[3 * i + k] += gf[c + k] * w;
            gr += gf[c + k] * S->vel[3 * i + k] * w * -0.5;
        }
        dbeta[i] += gr / l;
        dperiod[i] += -gr * b / (l * l);
        c += 3;
    }
    if (Fs->mask & FEAT_RHO) {
        if (rho < 2.0) {
            dbeta[i] += gf[c] / l;
            dperiod[i] += -gf[c] * b / (l * l);
        }
        c += 1;
    }
    if (Fs->mask & FEAT_SEM)
        for (int k = 0; k < Fs->n_sem; k++) dsem[i * Fs->n_sem + k] += gf[c + k];
}

/* per-Gaussian feature table [n, F] (rows of culled Gaussians unused) */
static double *feat_table(const scene_t *S, const gauss_t *G, const feat_t *Fs)
{
    if (Fs->F == 0) return NULL;
    double *FV = (double *)calloc((size_t)(S->n > 0 ? S->n : 1) * (size_t)Fs->F, sizeof(double));
    for (int64_t i = 0; i < S->n; i++)
        if (G[i].valid) feat_values(S, i, Fs, &FV[i * Fs->F]);
    return FV;
}

/* composite one pixel (px, py) over the depth-ordered list.  out receives
 * r, g, b, depth, opacity and the final transmittance; phi (if F > 0) the
 * F composited channels of the feature table FV; if `blend` is non-NULL
 * it receives the blended list (indices, alpha, T, G, offsets) */
typedef struct { int64_t idx; double alpha, T, G, dx, dy; int capped; } blend_t;

static void composite_pixel(const gauss_t *G, const int64_t *order, int64_t m, int culled, int px, int py,
                            const double *cam, const double *opt, const sky_t *sky, const double *FV, int F,
                            double out[6], double *phi, int32_t *nblend, int32_t *flag, blend_t *blend)
{
    const double sx = px + 0.5, sy = py + 0.5;
    double T = 1.0, C[3] = {0, 0, 0}, D = 0.0, O = 0.0, zprev = -1.0;
    int nb = 0, fl = 0;
    for (int c = 0; c < F; c++) phi[c] = 0.0;
    for (int64_t j = 0; j < m; j++) {
        const gauss_t *g = &G[order[j]];
        if (culled && (fabs(sx - g->uv[0]) > g->rx || fabs(sy - g->uv[1]) > g->ry)) continue;
        double Gv, dx, dy;
        int capped;
        const double a = eval_alpha(g, sx, sy, opt, &Gv, &dx, &dy, &capped);
        if (near_gate(g->ot * Gv, opt[OPT_AMIN])) fl = 1;
        if (a < opt[OPT_AMIN]) continue;
        const double Tn = T * (1.0 - a);
        if (near_gate(Tn, opt[OPT_TSTOP])) fl = 1;
        if (Tn < opt[OPT_TSTOP]) break;
        if (nb > 0 && fabs(g->z - zprev) < 1e-6 * fabs(g->z)) fl = 1;
        zprev = g->z;
        if (blend) {
            blend[nb].idx = order[j]; blend[nb].alpha = a; blend[nb].T = T; blend[nb].G = Gv;
            blend[nb].dx = dx; blend[nb].dy = dy; blend[nb].capped = capped;
        }
        const double w = a * T;
        for (int c = 0; c < 3; c++) C[c] += g->rgb[c] * w;
        for (int c = 0; c < F; c++) phi[c] += FV[order[j] * F + c] * w;
        D += g->z * w;
        O += w;
        T = Tn;
        nb++;
    }
    if (sky && sky->tex) {
        double f[3];
        sky_value(sky, cam, px, py, f);
        for (int c = 0; c < 3; c++) out[c] = C[c] + (1.0 - O) * f[c];
    } else {
        for (int c = 0; c < 3; c++) out[c] = C[c] + T * cam[CAM_BG + c];
    }
    out[3] = D;
    out[4] = O;
    out[5] = T;
    if (nblend) *nblend = nb;
    if (flag) *flag = fl;
}

/* exported: render.  mode 0 = brute force over every surviving Gaussian,
 * mode 1 = culled (step 6).  pix = NULL renders the full image in row-major
 * order (P = W H); otherwise P (px, py) int32 pairs.  Outputs per pixel:
 * rgb[P,3], depth[P] (sum T alpha z), alpha[P] (sum T alpha), T[P] (final
 * transmittance), nblend[P], flag[P] (1 if a gate was within 1e-5 relative
 * of its threshold or two blended depths were within 1e-6 relative).
 * feat_mask / n_sem / sem select the extra channels of step 8 (sem: [n,
 * n_sem]); feat receives them [P, F] (NULL if feat_mask = 0). */
int pvgo_render(int64_t n, int degree, const double *mu, const double *vel, const double *tau,
                const double *beta, const double *period, const double *scale, const double *quat,
                const double *opac, const double *sh, const double *cam, const double *opt, int mode,
                int64_t npix, const int32_t *pix, const double *sky_tex, int sky_res, const double *sky_jitter,
                int feat_mask, int n_sem, const double *sem, double *rgb, double *depth, double *alpha,
                double *Tout, int32_t *nblend, int32_t *flag, double *feat)
{
    const sky_t sky = {sky_tex, sky_res, sky_jitter};
    if (degree < 0 || degree > 3 || n < 0) return -1;
    if ((feat_mask & FEAT_SEM) && (n_sem <= 0 || !sem)) return -1;
    const feat_t Fs = {feat_mask, n_sem, feat_count(feat_mask, n_sem), sem};
    if (Fs.F > 0 && !feat) return -1;
    const int W = (int)cam[CAM_W], H = (int)cam[CAM_H];
    if (W <= 0 || H <= 0) return -1;
    scene_t S = make_scene(n, degree, mu, vel, tau, beta, period, scale, quat, opac, sh);
    gauss_t *G = (gauss_t *)malloc(sizeof(gauss_t) * (size_t)(n > 0 ? n : 1));
    preprocess_all(&S, cam, opt, G);
    int64_t *order = NULL;
    const int64_t m = depth_order(G, n, &order);
    double *FV = feat_table(&S, G, &Fs);
    const int64_t P = pix ? npix : (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < P; k++) {
        const int px = pix ? pix[2 * k] : (int)(k % W);
        const int py = pix ? pix[2 * k + 1] : (int)(k / W);
        double out[6];
        int32_t nb, fl;
        composite_pixel(G, order, m, mode == 1, px, py, cam, opt, &sky, FV, Fs.F, out,
                        feat ? &feat[k * Fs.F] : NULL, &nb, &fl, NULL);
        if (rgb) { rgb[3 * k] = out[0]; rgb[3 * k + 1] = out[1]; rgb[3 * k + 2] = out[2]; }
        if (depth) depth[k] = out[3];
        if (alpha) alpha[k] = out[4];
        if (Tout) Tout[k] = out[5];
        if (nblend) nblend[k] = nb;
        if (flag) flag[k] = fl;
    }
    free(FV);
    free(order);
    free(G);
    return 0;
}

/* exported: number of threads a parallel region uses */
int pvgo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* step 7: exact reverse mode                                          */
/* ------------------------------------------------------------------ */
/* per-Gaussian image-space gradient accumulator */
enum { G2_U = 0, G2_V, G2_A, G2_B, G2_C, G2_O, G2_R, G2_G, G2_BL, G2_Z, G2_LEN };

/* growable list of (Gaussian index, `stride` gradient terms: the 10
 * image-space terms, then dL/d(feature) of step 8) */
typedef struct { int64_t len, cap; int stride; int64_t *idx; double *val; } contrib_list_t;

static double *contrib_push(contrib_list_t *L, int64_t idx)
{
    if (L->len == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 1024;
        L->idx = (int64_t *)realloc(L->idx, sizeof(int64_t) * (size_t)L->cap);
        L->val = (double *)realloc(L->val, sizeof(double) * (size_t)L->stride * (size_t)L->cap);
    }
    L->idx[L->len] = idx;
    double *A = &L->val[L->len * L->stride];
    for (int c = 0; c < L->stride; c++) A[c] = 0.0;
    L->len++;
    return A;
}

/* chain rule from the image-space gradients of Gaussian i to its
 * parameters (adjoint of steps 1-4) */
static void backward_one(const scene_t *S, int64_t i, const gauss_t *g, const double *cam, const double *opt,
                         const double *g2, double *dmu, double *dvel, double *dtau, double *dbeta,
                         double *dperiod, double *dscale, double *dquat, double *dopac, double *dsh)
{
    const double *V = cam;
    const double fx = cam[CAM_FX], fy = cam[CAM_FY];
    const int K = (S->degree + 1) * (S->degree + 1);
    double gmut[3] = {0, 0, 0};
    double gp[3] = {0, 0, 0};

    /* colour: rgb = max(0, sum_k sh_k Y_k(dir) + 0.5) */
    {
        double Y[16], dY[16][3];
        sh_basis(S->degree, g->dir, Y, dY);
        double gdir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ch++) {
            if (!(g->rgb_raw[ch] > 0.0)) continue;
            const double gc = g2[G2_R + ch];
            for (int k = 0; k < K; k++) {
                dsh[(i * K + k) * 3 + ch] += gc * Y[k];
                const double coef = S->sh[(i * K + k) * 3 + ch];
                for (int a = 0; a < 3; a++) gdir[a] += gc * coef * dY[k][a];
            }
        }
        /* dir = (mu~ - c)/|mu~ - c| */
        double dot = 0.0;
        for (int a = 0; a < 3; a++) dot += g->dir[a] * gdir[a];
        for (int a = 0; a < 3; a++) gmut[a] += (gdir[a] - g->dir[a] * dot) / g->dist;
    }

    /* conic = inverse of cov2 */
    const double a = g->conic[0], b = g->conic[1], c = g->conic[2];
    const double Qm[2][2] = {{a, b}, {b, c}};
    const double Gh[2][2] = {{g2[G2_A], 0.5 * g2[G2_B]}, {0.5 * g2[G2_B], g2[G2_C]}};
    double QG[2][2], Gs[2][2];
    for (int r = 0; r < 2; r++)
        for (int s = 0; s < 2; s++) QG[r][s] = Qm[r][0] * Gh[0][s] + Qm[r][1] * Gh[1][s];
    for (int r = 0; r < 2; r++)
        for (int s = 0; s < 2; s++) Gs[r][s] = -(QG[r][0] * Qm[0][s] + QG[r][1] * Qm[1][s]);
    /* cov2 = J M J^T + h I: gradients for M (3x3) and J (2x3) */
    double GM[3][3], GJ[2][3];
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) {
            double acc = 0.0;
            for (int u = 0; u < 2; u++)
                for (int w = 0; w < 2; w++) acc += g->J[u][r] * Gs[u][w] * g->J[w][s];
            GM[r][s] = acc;
        }
    for (int r = 0; r < 2; r++)
        for (int s = 0; s < 3; s++) {
            double acc = 0.0;
            for (int u = 0; u < 2; u++)
                for (int k = 0; k < 3; k++) acc += Gs[r][u] * g->J[u][k] * g->M[k][s];
            GJ[r][s] = 2.0 * acc;
        }
    /* M = W Sigma W^T */
    double GS[3][3];
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) {
            double acc = 0.0;
            for (int u = 0; u < 3; u++)
                for (int w = 0; w < 3; w++) acc += V[4 * u + r] * GM[u][w] * V[4 * w + s];
            GS[r][s] = acc;
        }
    /* Sigma = R diag(s^2) R^T */
    const double *sc = &S->scale[3 * i];
    double RtGR[3][3], GR[3][3];
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) {
            double acc = 0.0;
            for (int u = 0; u < 3; u++)
                for (int w = 0; w < 3; w++) acc += g->R[u][r] * GS[u][w] * g->R[w][s];
            RtGR[r][s] = acc;
        }
    for (int k = 0; k < 3; k++) dscale[3 * i + k] += 2.0 * sc[k] * RtGR[k][k];
    for (int r = 0; r < 3; r++)
        for (int s = 0; s < 3; s++) {
            double acc = 0.0;
            for (int u = 0; u < 3; u++) acc += GS[r][u] * g->R[u][s];
            GR[r][s] = 2.0 * acc * sc[s] * sc[s];
        }
    /* R(q^) */
    {
        const double w = g->qn[0], x = g->qn[1], y = g->qn[2], z = g->qn[3];
        const double dRw[3][3] = {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}};
        const double dRx[3][3] = {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}};
        const double dRy[3][3] = {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}};
        const double dRz[3][3] = {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}};
        double gq[4] = {0, 0, 0, 0};
        for (int r = 0; r < 3; r++)
            for (int s = 0; s < 3; s++) {
                gq[0] += GR[r][s] * dRw[r][s];
                gq[1] += GR[r][s] * dRx[r][s];
                gq[2] += GR[r][s] * dRy[r][s];
                gq[3] += GR[r][s] * dRz[r][s];
            }
        double dot = 0.0;
        for (int k = 0; k < 4; k++) dot += g->qn[k] * gq[k];
        for (int k = 0; k < 4; k++) dquat[4 * i + k] += (gq[k] - g->qn[k] * dot) / g->qlen;
    }
    /* J(p) with the frustum clamp */
    {
        const double x = g->p[0], y = g->p[1], z = g->p[2];
        const double limx = opt[OPT_FOVCLAMP] * 0.5 * cam[CAM_W] / fx;
        const double limy = opt[OPT_FOVCLAMP] * 0.5 * cam[CAM_H] / fy;
        gp[2] += GJ[0][0] * (-fx / (z * z)) + GJ[1][1] * (-fy / (z * z));
        if (g->clamp_x == 0) {
            gp[0] += GJ[0][2] * (-fx / (z * z));
            gp[2] += GJ[0][2] * (2.0 * fx * x / (z * z * z));
        } else {
            gp[2] += GJ[0][2] * (fx * g->clamp_x * limx / (z * z));
        }
        if (g->clamp_y == 0) {
            gp[1] += GJ[1][2] * (-fy / (z * z));
            gp[2] += GJ[1][2] * (2.0 * fy * y / (z * z * z));
        } else {
            gp[2] += GJ[1][2] * (fy * g->clamp_y * limy / (z * z));
        }
        /* projected mean */
        gp[0] += g2[G2_U] * fx / z;
        gp[2] += -g2[G2_U] * fx * x / (z * z);
        gp[1] += g2[G2_V] * fy / z;
        gp[2] += -g2[G2_V] * fy * y / (z * z);
        /* depth channel */
        gp[2] += g2[G2_Z];
    }
    /* p = W mu~ + t */
    for (int k = 0; k < 3; k++) gmut[k] += V[0 + k] * gp[0] + V[4 + k] * gp[1] + V[8 + k] * gp[2];

    /* time evaluation adjoint */
    const double l = S->period[i], be = S->beta[i];
    const double gv_dot = gmut[0] * S->vel[3 * i] + gmut[1] * S->vel[3 * i + 1] + gmut[2] * S->vel[3 * i + 2];
    const double amp = l / TWO_PI * g->sin_t + g->dt * g->vbar_w;
    for (int k = 0; k < 3; k++) {
        dmu[3 * i + k] += gmut[k];
        dvel[3 * i + k] += gmut[k] * amp;
    }
    double gtau = -g->cos_t * gv_dot;
    dperiod[i] += gv_dot * (g->sin_t / TWO_PI - g->delta / l * g->cos_t);
    /* flow shift dt v exp(-beta / (2 l)) */
    const double gsh = gv_dot * g->dt * g->vbar_w;
    dbeta[i] += gsh * (-0.5 / l);
    dperiod[i] += gsh * (0.5 * be / (l * l));
    const double go = g2[G2_O];
    dopac[i] += go * g->egate;
    gtau += go * g->ot * g->delta / (be * be);
    dbeta[i] += go * g->ot * g->delta * g->delta / (be * be * be);
    dtau[i] += gtau;
}

/* exported: gradients of L = sum(dL_rgb . rgb) + sum(dL_depth depth) +
 * sum(dL_alpha alpha) (+ sum(dL_feat . feat) for the step-8 channels
 * selected by feat_mask; dsem [n, n_sem] receives the semantic gradient)
 * w.r.t. every parameter (and the sky texels, if a sky
 * map is given: dsky[6 res res 3]), over the full image
 * (pix = NULL, row-major pixels) or over the P listed (px, py) pixels
 * (dL arrays then indexed by list position); mode 0 brute force, 1 culled
 * (same result).  Gradient arrays are overwritten.  If g2d is non-NULL it
 * receives the per-Gaussian image-space gradients [n, 10]:
 * (u, v, conic a, b, c, o~, r, g, b, z). */
int pvgo_render_bwd(int64_t n, int degree, const double *mu, const double *vel, const double *tau,
                    const double *beta, const double *period, const double *scale, const double *quat,
                    const double *opac, const double *sh, const double *cam, const double *opt, int mode,
                    int64_t npix, const int32_t *pix, const double *sky_tex, int sky_res,
                    const double *sky_jitter, int feat_mask, int n_sem, const double *sem,
                    const double *dL_feat, const double *dL_rgb, const double *dL_depth,
                    const double *dL_alpha, double *dmu, double *dvel, double *dtau, double *dbeta,
                    double *dperiod, double *dscale, double *dquat, double *dopac, double *dsh, double *g2d,
                    double *dsky, double *dsem)
{
    const sky_t sky = {sky_tex, sky_res, sky_jitter};
    if (sky_tex && dsky) memset(dsky, 0, sizeof(double) * 18 * (size_t)sky_res * (size_t)sky_res);
    if (degree < 0 || degree > 3 || n < 0) return -1;
    if ((feat_mask & FEAT_SEM) && (n_sem <= 0 || !sem || !dsem)) return -1;
    const feat_t Fs = {feat_mask, n_sem, feat_count(feat_mask, n_sem), sem};
    if (Fs.F > 0 && !dL_feat) return -1;
    const int stride = G2_LEN + Fs.F;
    if (dsem && (feat_mask & FEAT_SEM)) memset(dsem, 0, sizeof(double) * (size_t)n * (size_t)n_sem);
    const int W = (int)cam[CAM_W], H = (int)cam[CAM_H];
    const int K = (degree + 1) * (degree + 1);
    scene_t S = make_scene(n, degree, mu, vel, tau, beta, period, scale, quat, opac, sh);
    gauss_t *G = (gauss_t *)malloc(sizeof(gauss_t) * (size_t)(n > 0 ? n : 1));
    preprocess_all(&S, cam, opt, G);
    int64_t *order = NULL;
    const int64_t m = depth_order(G, n, &order);
    double *FV = feat_table(&S, G, &Fs);
    double *acc = (double *)calloc((size_t)(n > 0 ? n : 1) * (size_t)stride, sizeof(double));
    const int64_t P = pix ? npix : (int64_t)W * H;
    /* pixels are split into fixed contiguous chunks, one per thread; each
     * thread lists its per-(pixel, Gaussian) contributions and the lists are
     * added in chunk order, so the sums do not depend on scheduling */
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    contrib_list_t *lists = (contrib_list_t *)calloc((size_t)nthreads, sizeof(contrib_list_t));
#pragma omp parallel num_threads(nthreads)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        const int64_t k0 = P * tid / nthreads, k1 = P * (tid + 1) / nthreads;
        blend_t *bl = (blend_t *)malloc(sizeof(blend_t) * (size_t)(m > 0 ? m : 1));
        double *phi = (double *)malloc(sizeof(double) * (size_t)(2 * Fs.F + 1));
        double *sF = phi + Fs.F; /* feature suffix sums */
        contrib_list_t *L = &lists[tid];
        L->stride = stride;
        for (int64_t k = k0; k < k1; k++) {
            const int px = pix ? pix[2 * k] : (int)(k % W);
            const int py = pix ? pix[2 * k + 1] : (int)(k / W);
            double out[6];
            int32_t nb;
            composite_pixel(G, order, m, mode == 1, px, py, cam, opt, &sky, FV, Fs.F, out, phi, &nb, NULL, bl);
            const double *gF = Fs.F ? &dL_feat[k * Fs.F] : NULL;
            for (int c = 0; c < Fs.F; c++) sF[c] = 0.0; /* no feature background */
            const double Tfin = out[5];
            const double gC[3] = {dL_rgb[3 * k], dL_rgb[3 * k + 1], dL_rgb[3 * k + 2]};
            const double gD = dL_depth[k];
            double gO = dL_alpha[k];
            /* suffix sums S_j = sum_{m > j} x_m alpha_m T_m (+ bg T_final for colour) */
            double sC[3] = {Tfin * cam[CAM_BG], Tfin * cam[CAM_BG + 1], Tfin * cam[CAM_BG + 2]};
            if (sky.tex) {
                /* colour = C + (1 - O) f: dL/dO gains -gC.f, dL/df = (1 - O) gC,
                 * and no constant background */
                int64_t ti[4];
                double tw[4], f[3] = {0, 0, 0};
                sky_texels(&sky, cam, px, py, ti, tw);
                for (int c = 0; c < 3; c++) {
                    for (int q = 0; q < 4; q++) f[c] += tw[q] * sky.tex[ti[q] * 3 + c];
                    gO -= gC[c] * f[c];
                    sC[c] = 0.0;
                }
                if (dsky) {
                    const double wO = 1.0 - out[4];
#pragma omp critical(pvgo_sky)
                    for (int q = 0; q < 4; q++)
                        for (int c = 0; c < 3; c++) dsky[ti[q] * 3 + c] += tw[q] * wO * gC[c];
                }
            }
            double sD = 0.0, sO = 0.0;
            for (int j = nb - 1; j >= 0; j--) {
                const blend_t *e = &bl[j];
                const gauss_t *g = &G[e->idx];
                double *A = contrib_push(L, e->idx);
                const double w = e->alpha * e->T;
                /* d/dalpha_j of each channel */
                double ga = 0.0;
                for (int c = 0; c < 3; c++) ga += gC[c] * (g->rgb[c] * e->T - sC[c] / (1.0 - e->alpha));
                ga += gD * (g->z * e->T - sD / (1.0 - e->alpha));
                ga += gO * (e->T - sO / (1.0 - e->alpha));
                const double *f = Fs.F ? &FV[e->idx * Fs.F] : NULL;
                for (int c = 0; c < Fs.F; c++) {
                    ga += gF[c] * (f[c] * e->T - sF[c] / (1.0 - e->alpha));
                    A[G2_LEN + c] = gF[c] * w;
                }
                for (int c = 0; c < 3; c++) A[G2_R + c] = gC[c] * w;
                A[G2_Z] = gD * w;
                if (!e->capped) {
                    A[G2_O] = ga * e->G;
                    const double gpow = ga * e->alpha; /* alpha = o~ exp(power) */
                    const double dx = e->dx, dy = e->dy;
                    A[G2_A] = gpow * (-0.5 * dx * dx);
                    A[G2_B] = gpow * (-dx * dy);
                    A[G2_C] = gpow * (-0.5 * dy * dy);
                    A[G2_U] = gpow * (g->conic[0] * dx + g->conic[1] * dy);
                    A[G2_V] = gpow * (g->conic[1] * dx + g->conic[2] * dy);
                }
                for (int c = 0; c < 3; c++) sC[c] += g->rgb[c] * w;
                for (int c = 0; c < Fs.F; c++) sF[c] += f[c] * w;
                sD += g->z * w;
                sO += w;
            }
        }
        free(phi);
        free(bl);
    }
    for (int t = 0; t < nthreads; t++) {
        for (int64_t q = 0; q < lists[t].len; q++) {
            double *A = &acc[lists[t].idx[q] * stride];
            for (int c = 0; c < stride; c++) A[c] += lists[t].val[q * stride + c];
        }
        free(lists[t].idx);
        free(lists[t].val);
    }
    free(lists);
    memset(dmu, 0, sizeof(double) * 3 * (size_t)n);
    memset(dvel, 0, sizeof(double) * 3 * (size_t)n);
    memset(dtau, 0, sizeof(double) * (size_t)n);
    memset(dbeta, 0, sizeof(double) * (size_t)n);
    memset(dperiod, 0, sizeof(double) * (size_t)n);
    memset(dscale, 0, sizeof(double) * 3 * (size_t)n);
    memset(dquat, 0, sizeof(double) * 4 * (size_t)n);
    memset(dopac, 0, sizeof(double) * (size_t)n);
    memset(dsh, 0, sizeof(double) * 3 * (size_t)K * (size_t)n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        if (g2d)
            for (int c = 0; c < G2_LEN; c++) g2d[i * G2_LEN + c] = acc[i * stride + c];
        if (!G[i].valid) continue;
        backward_one(&S, i, &G[i], cam, opt, &acc[i * stride], dmu, dvel, dtau, dbeta, dperiod, dscale, dquat,
                     dopac, dsh);
        if (Fs.F) feat_backward(&S, i, &Fs, &acc[i * stride + G2_LEN], dvel, dbeta, dperiod, dsem);
    }
    free(FV);
    free(acc);
    free(order);
    free(G);
    return 0;
}
