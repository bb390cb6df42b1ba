/*
 * tgs_oracle.c -- plain FP64 CPU oracle for the Trick-GS differentiable rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may load this library. The CUDA product path never calls it, and the two share no code.
 *
 * What it computes (paper sections in brackets):
 *   - Gaussian volume mask with straight-through binarisation, applied to opacity and scale
 *     [Sec. "Pruning with Volume Masking", mask equation].
 *   - Per-band SH masks with straight-through binarisation [Sec. "SH Masking", Eq. sh-masks].
 *   - EWA projection of each 3D Gaussian to a 2D Gaussian G'(x) = exp(-1/2 (x-mu')^T
 *     Sigma'^-1 (x-mu')) [Sec. "Preliminaries", Eq. 1], with the low-pass term Sigma' + sI,
 *     s = 0.3 by default [Sec. "Progressive training by scales of Gaussians"].
 *   - View-dependent colour from SH of degree <= 3 [Sec. "Preliminaries"].
 *   - Front-to-back alpha blending C = sum_i c_i a_i prod_{j<i}(1 - a_j) [Eq. 2].
 *   - The exact (piecewise) gradient of all of the above, computed with the transmittance of
 *     every fragment stored in forward order (no reverse division).
 * Conventions the paper leaves to the original 3DGS rasterizer (pixel frame, 3-sigma box,
 * alpha clamp 0.99, skip below 1/255, stop before T < 1e-4, colour offset 1/2 and clamp at 0,
 * near plane, Jacobian clamp 1.3) are written out where they are used.
 *
 * Everything is double precision. Inputs arrive as the float32 values the GPU receives,
 * promoted to double. Three places use float32 on purpose, because the method's definition
 * fixes them as float32 quantities: the mask thresholds logit(eps) are rounded to float32,
 * and sort keys use the float32 bits of the depth.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_SUPPORT_BOX3 0
#define ORC_SUPPORT_ALPHA 1

/* ------------------------------------------------------------------------------------ */
/* Inputs                                                                               */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    const double *means;          /* [n,3] */
    const double *log_scales;     /* [n,3] */
    const double *quats;          /* [n,4] w,x,y,z (not necessarily unit) */
    const double *opacity_logits; /* [n] */
    const double *sh_dc;          /* [n,3] */
    const double *sh_rest;        /* [n,15,3] or NULL */
    const uint8_t *sh_degree;     /* [n] active degree per Gaussian, or NULL */
    const double *mask_logits;    /* [n] or NULL (no volume mask) */
    const double *sh_mask_logits; /* [n,3] or NULL (no band masks) */
    int64_t deg_max;              /* 0..3 */
} orc_params;

typedef struct {
    double *means, *log_scales, *quats, *opacity_logits, *sh_dc, *sh_rest, *mask_logits,
        *sh_mask_logits; /* same shapes as orc_params; NULL entries are skipped */
} orc_grads;

/* Camera, flat: R[9] row-major world->camera rotation, t[3], campos[3], fx, fy, cx, cy,
   W, H, low-pass s. */
typedef struct {
    double R[3][3], t[3], campos[3], fx, fy, cx, cy, s;
    int W, H;
} cam_t;

/* Settings, flat: tile, support mode, eps_mask, eps_sh, near, bg[3]. */
typedef struct {
    int tile, support;
    double tau_m, tau_sh; /* thresholds on the logits: float32(log(eps / (1 - eps))) */
    double near_z, bg[3];
} cfg_t;

static cam_t read_cam(const double *c) {
    cam_t k;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) k.R[i][j] = c[3 * i + j];
    for (int i = 0; i < 3; i++) k.t[i] = c[9 + i];
    for (int i = 0; i < 3; i++) k.campos[i] = c[12 + i];
    k.fx = c[15];
    k.fy = c[16];
    k.cx = c[17];
    k.cy = c[18];
    k.W = (int)c[19];
    k.H = (int)c[20];
    k.s = c[21];
    return k;
}

static double logit_f32(double eps) {
    /* sigma(m) > eps  <=>  m > log(eps / (1 - eps)); the threshold is fixed as a float32. */
    return (double)(float)log(eps / (1.0 - eps));
}

static cfg_t read_cfg(const double *c) {
    cfg_t k;
    k.tile = (int)c[0];
    k.support = (int)c[1];
    k.tau_m = logit_f32(c[2]);
    k.tau_sh = logit_f32(c[3]);
    k.near_z = c[4];
    k.bg[0] = c[5];
    k.bg[1] = c[6];
    k.bg[2] = c[7];
    return k;
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* ------------------------------------------------------------------------------------ */
/* Real spherical harmonics, degree <= 3                                                */
/* ------------------------------------------------------------------------------------ */
/*
 * Basis Y_k(d), k = l*l + l + m, for a unit direction d = (x, y, z). The sign convention is
 * the one 3DGS uses: starting from the complex SH with the Condon-Shortley phase,
 *   m < 0: sqrt(2) Im Y_l^{|m|},   m = 0: Y_l^0,   m > 0: sqrt(2) Re Y_l^m.
 * Written as homogeneous polynomials so they can be differentiated componentwise.
 * dY[k][c] is the partial derivative of that polynomial with respect to component c.
 */
void orc_sh_eval(double x, double y, double z, double Y[16], double dY[16][3]) {
    const double pi = 3.14159265358979323846;
    const double k0 = 0.5 / sqrt(pi);
    const double k1 = sqrt(3.0 / (4.0 * pi));
    const double k2a = 0.5 * sqrt(15.0 / pi);
    const double k2b = 0.25 * sqrt(5.0 / pi);
    const double k2c = 0.25 * sqrt(15.0 / pi);
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double k3b = 0.5 * sqrt(105.0 / pi);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double k3d = 0.25 * sqrt(7.0 / pi);
    const double k3e = 0.25 * sqrt(105.0 / pi);
    double xx = x * x, yy = y * y, zz = z * z;
    memset(dY, 0, sizeof(double) * 48);
    Y[0] = k0;
    /* l = 1 */
    Y[1] = -k1 * y;
    dY[1][1] = -k1;
    Y[2] = k1 * z;
    dY[2][2] = k1;
    Y[3] = -k1 * x;
    dY[3][0] = -k1;
    /* l = 2 */
    Y[4] = k2a * x * y;
    dY[4][0] = k2a * y;
    dY[4][1] = k2a * x;
    Y[5] = -k2a * y * z;
    dY[5][1] = -k2a * z;
    dY[5][2] = -k2a * y;
    Y[6] = k2b * (2.0 * zz - xx - yy);
    dY[6][0] = -2.0 * k2b * x;
    dY[6][1] = -2.0 * k2b * y;
    dY[6][2] = 4.0 * k2b * z;
    Y[7] = -k2a * x * z;
    dY[7][0] = -k2a * z;
    dY[7][2] = -k2a * x;
    Y[8] = k2c * (xx - yy);
    dY[8][0] = 2.0 * k2c * x;
    dY[8][1] = -2.0 * k2c * y;
    /* l = 3 */
    Y[9] = -k3a * y * (3.0 * xx - yy);
    dY[9][0] = -k3a * 6.0 * x * y;
    dY[9][1] = -k3a * (3.0 * xx - 3.0 * yy);
    Y[10] = k3b * x * y * z;
    dY[10][0] = k3b * y * z;
    dY[10][1] = k3b * x * z;
    dY[10][2] = k3b * x * y;
    Y[11] = -k3c * y * (4.0 * zz - xx - yy);
    dY[11][0] = -k3c * (-2.0 * x * y);
    dY[11][1] = -k3c * (4.0 * zz - xx - 3.0 * yy);
    dY[11][2] = -k3c * 8.0 * y * z;
    Y[12] = k3d * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    dY[12][0] = k3d * (-6.0 * x * z);
    dY[12][1] = k3d * (-6.0 * y * z);
    dY[12][2] = k3d * (6.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[13] = -k3c * x * (4.0 * zz - xx - yy);
    dY[13][0] = -k3c * (4.0 * zz - 3.0 * xx - yy);
    dY[13][1] = -k3c * (-2.0 * x * y);
    dY[13][2] = -k3c * 8.0 * x * z;
    Y[14] = k3e * z * (xx - yy);
    dY[14][0] = k3e * 2.0 * x * z;
    dY[14][1] = -k3e * 2.0 * y * z;
    dY[14][2] = k3e * (xx - yy);
    Y[15] = -k3a * x * (xx - 3.0 * yy);
    dY[15][0] = -k3a * (3.0 * xx - 3.0 * yy);
    dY[15][1] = -k3a * (-6.0 * x * y);
}

/* Batch form for tests: dirs [n,3] (used as given), Y [n,16], dY [n,16,3]. */
void orc_sh_basis(int64_t n, const double *dirs, double *Y, double *dY) {
    for (int64_t i = 0; i < n; i++) {
        double y[16], dy[16][3];
        orc_sh_eval(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], y, dy);
        memcpy(Y + 16 * i, y, sizeof y);
        if (dY) memcpy(dY + 48 * i, dy, sizeof dy);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Small matrix helpers                                                                 */
/* ------------------------------------------------------------------------------------ */

static void mat3_mul(double A[3][3], double B[3][3], double C[3][3]) {
    double T[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            T[i][j] = 0.0;
            for (int k = 0; k < 3; k++) T[i][j] += A[i][k] * B[k][j];
        }
    memcpy(C, T, sizeof T);
}

static void mat3_transpose(double A[3][3], double B[3][3]) {
    double T[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T[i][j] = A[j][i];
    memcpy(B, T, sizeof T);
}

/* Rotation matrix of a unit quaternion (w, x, y, z) and its partial derivatives. */
static void quat_to_rot(const double q[4], double R[3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1.0 - 2.0 * (y * y + z * z);
    R[0][1] = 2.0 * (x * y - w * z);
    R[0][2] = 2.0 * (x * z + w * y);
    R[1][0] = 2.0 * (x * y + w * z);
    R[1][1] = 1.0 - 2.0 * (x * x + z * z);
    R[1][2] = 2.0 * (y * z - w * x);
    R[2][0] = 2.0 * (x * z - w * y);
    R[2][1] = 2.0 * (y * z + w * x);
    R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

static void quat_to_rot_partials(const double q[4], double dR[4][3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    /* d/dw */
    double Dw[3][3] = {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}};
    /* d/dx */
    double Dx[3][3] = {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}};
    /* d/dy */
    double Dy[3][3] = {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}};
    /* d/dz */
    double Dz[3][3] = {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}};
    memcpy(dR[0], Dw, sizeof Dw);
    memcpy(dR[1], Dx, sizeof Dx);
    memcpy(dR[2], Dy, sizeof Dy);
    memcpy(dR[3], Dz, sizeof Dz);
}

/* ------------------------------------------------------------------------------------ */
/* Preprocess: one Gaussian in one view                                                  */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    int visible;
    /* activations */
    double M;                 /* hard volume mask in {0,1} */
    double Msh[4];            /* effective band mask: Msh[0] = 1; bands above the degree = 0 */
    int deg;                  /* active degree of this Gaussian */
    double scale[3], sig_o, opac; /* s = M exp(l), sigma(o), o' = M sigma(o) */
    double qn[4], qnorm;      /* normalised quaternion and the norm of the input */
    double Rq[3][3];          /* rotation of the Gaussian */
    double Sigma[3][3];       /* 3D covariance */
    /* camera */
    double tc[3];             /* view-space mean */
    double u, w;              /* clamped t_x/t_z and t_y/t_z */
    int clamp_x, clamp_y;     /* 1 if the clamp is active */
    double J[2][3];
    double T2[2][3];          /* J * R_view */
    double cov2d[2][2];       /* Sigma' including the low-pass term */
    double det;
    double conic[3];          /* a, b, c of Sigma'^-1 = [[a, b], [b, c]] */
    double mean2d[2];         /* mu' - 1/2: pixel (px, py) samples the Gaussian at (px, py) */
    double lambda1, rcont;    /* largest eigenvalue bound and the continuous radius */
    int radius;
    int rect[4];              /* inclusive pixel rect: x_lo, x_hi, y_lo, y_hi */
    /* colour */
    double dir[3], dist;      /* unit direction from the camera centre, and its length */
    double Y[16], dY[16][3];
    double raw[3], rgb[3];
    int clamped[3];           /* raw < 0: colour channel clamped to 0 */
    /* decision margins, in units of the float32 uncertainty of the decided quantity */
    double m_all, m_edge;
} pre_t;

static int finite3(const double *v) { return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]); }

static int preprocess_one(const orc_params *P, int64_t i, const cam_t *cam, const cfg_t *cfg,
                          pre_t *o) {
    memset(o, 0, sizeof *o);
    o->visible = 0;
    o->m_all = INFINITY;
    o->m_edge = INFINITY;
    const double *mu = P->means + 3 * i;
    const double *ls = P->log_scales + 3 * i;
    const double *q = P->quats + 4 * i;

    /* --- volume mask and activations [mask equation; M applied to opacity and scale] --- */
    o->M = 1.0;
    if (P->mask_logits) o->M = (P->mask_logits[i] > cfg->tau_m) ? 1.0 : 0.0;
    o->deg = (int)P->deg_max;
    if (P->sh_degree && P->sh_degree[i] < o->deg) o->deg = P->sh_degree[i];
    o->Msh[0] = 1.0;
    for (int l = 1; l <= 3; l++) {
        double m = 1.0;
        if (P->sh_mask_logits) m = (P->sh_mask_logits[3 * i + l - 1] > cfg->tau_sh) ? 1.0 : 0.0;
        o->Msh[l] = (l <= o->deg) ? m : 0.0;
    }
    for (int k = 0; k < 3; k++) o->scale[k] = o->M * exp(ls[k]);
    o->sig_o = sigmoid(P->opacity_logits[i]);
    o->opac = o->M * o->sig_o;
    if (o->M == 0.0) return 0; /* masked Gaussian: opacity 0, never blended */

    o->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(o->qnorm > 0.0) || !isfinite(o->qnorm)) return 0;
    for (int k = 0; k < 4; k++) o->qn[k] = q[k] / o->qnorm;
    quat_to_rot(o->qn, o->Rq);

    /* Sigma = R S S^T R^T */
    double RS[3][3], RSt[3][3];
    for (int r = 0; r < 3; r++)
        for (int c = 0; c < 3; c++) RS[r][c] = o->Rq[r][c] * o->scale[c];
    mat3_transpose(RS, RSt);
    mat3_mul(RS, RSt, o->Sigma);

    /* --- view transform and near-plane cull --- */
    for (int r = 0; r < 3; r++)
        o->tc[r] = cam->R[r][0] * mu[0] + cam->R[r][1] * mu[1] + cam->R[r][2] * mu[2] + cam->t[r];
    if (!finite3(o->tc) || !finite3(mu) || !finite3(ls)) return 0;
    if (!(o->tc[2] > cfg->near_z)) return 0;
    o->m_all = fmin(o->m_all, fabs(o->tc[2] - cfg->near_z) / (1e-6 * (fabs(o->tc[2]) + 1.0)));

    /* --- EWA: Sigma' = J W Sigma W^T J^T + s I  [Eq. 1 and the low-pass term] --- */
    double tz = o->tc[2];
    double limx = 1.3 * (0.5 * cam->W / cam->fx);
    double limy = 1.3 * (0.5 * cam->H / cam->fy);
    double ux = o->tc[0] / tz, uy = o->tc[1] / tz;
    o->clamp_x = (ux < -limx || ux > limx);
    o->clamp_y = (uy < -limy || uy > limy);
    o->u = fmin(limx, fmax(-limx, ux));
    o->w = fmin(limy, fmax(-limy, uy));
    o->J[0][0] = cam->fx / tz;
    o->J[0][1] = 0.0;
    o->J[0][2] = -cam->fx * o->u / tz;
    o->J[1][0] = 0.0;
    o->J[1][1] = cam->fy / tz;
    o->J[1][2] = -cam->fy * o->w / tz;
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++)
            o->T2[r][c] = o->J[r][0] * cam->R[0][c] + o->J[r][1] * cam->R[1][c] +
                          o->J[r][2] * cam->R[2][c];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) {
            double acc = 0.0;
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) acc += o->T2[r][a] * o->Sigma[a][b] * o->T2[c][b];
            o->cov2d[r][c] = acc;
        }
    o->cov2d[0][0] += cam->s;
    o->cov2d[1][1] += cam->s;
    o->det = o->cov2d[0][0] * o->cov2d[1][1] - o->cov2d[0][1] * o->cov2d[1][0];
    if (!(o->det > 0.0) || !isfinite(o->det)) return 0;
    o->conic[0] = o->cov2d[1][1] / o->det;
    o->conic[1] = -o->cov2d[0][1] / o->det;
    o->conic[2] = o->cov2d[0][0] / o->det;

    /* --- footprint radius --- */
    double mid = 0.5 * (o->cov2d[0][0] + o->cov2d[1][1]);
    o->lambda1 = mid + sqrt(fmax(0.1, mid * mid - o->det));
    if (cfg->support == ORC_SUPPORT_ALPHA) {
        if (o->opac < 1.0 / 255.0) return 0;
        o->m_all = fmin(o->m_all, fabs(o->opac * 255.0 - 1.0) / 1e-5);
        o->rcont = sqrt(2.0 * o->lambda1 * log(255.0 * o->opac));
    } else {
        o->rcont = 3.0 * sqrt(o->lambda1);
    }
    double rf = ceil(o->rcont);
    if (rf > 1073741824.0) rf = 1073741824.0; /* 2^30: covers any image */
    o->radius = (int)rf;
    if (o->radius <= 0) return 0;
    {
        double dr = fabs(o->rcont - round(o->rcont));
        o->m_edge = fmin(o->m_edge, dr / (1e-6 * (o->rcont + 1.0)));
    }

    /* --- pixel frame: pixel (px, py) is sampled at integer coordinates in mu' - 1/2 --- */
    o->mean2d[0] = cam->fx * o->tc[0] / tz + cam->cx - 0.5;
    o->mean2d[1] = cam->fy * o->tc[1] / tz + cam->cy - 0.5;
    if (!isfinite(o->mean2d[0]) || !isfinite(o->mean2d[1])) return 0;

    /* inclusive pixel rect of the box |p - mu'| <= r, clipped to the image */
    double lo[2], hi[2];
    int lim[2] = {cam->W - 1, cam->H - 1};
    for (int a = 0; a < 2; a++) {
        lo[a] = ceil(o->mean2d[a] - o->radius);
        hi[a] = floor(o->mean2d[a] + o->radius);
        double unc = 1e-6 * (fabs(o->mean2d[a]) + o->radius + 1.0);
        o->m_edge = fmin(o->m_edge, fabs(o->mean2d[a] - o->radius - round(o->mean2d[a] - o->radius)) / unc);
        o->m_edge = fmin(o->m_edge, fabs(o->mean2d[a] + o->radius - round(o->mean2d[a] + o->radius)) / unc);
        if (lo[a] < 0.0) lo[a] = 0.0;
        if (hi[a] > (double)lim[a]) hi[a] = (double)lim[a];
        if (lo[a] > hi[a]) return 0;
    }
    o->rect[0] = (int)lo[0];
    o->rect[1] = (int)hi[0];
    o->rect[2] = (int)lo[1];
    o->rect[3] = (int)hi[1];

    /* --- colour from SH with band masks [Eq. sh-masks], offset 1/2, clamped at 0 --- */
    double dv[3] = {mu[0] - cam->campos[0], mu[1] - cam->campos[1], mu[2] - cam->campos[2]};
    o->dist = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    if (!(o->dist > 0.0)) return 0;
    for (int k = 0; k < 3; k++) o->dir[k] = dv[k] / o->dist;
    orc_sh_eval(o->dir[0], o->dir[1], o->dir[2], o->Y, o->dY);
    for (int ch = 0; ch < 3; ch++) {
        double v = 0.5 + o->Y[0] * P->sh_dc[3 * i + ch];
        for (int k = 1; k < 16; k++) {
            int l = (k < 4) ? 1 : (k < 9) ? 2 : 3;
            if (o->Msh[l] == 0.0 || !P->sh_rest) continue;
            v += o->Msh[l] * o->Y[k] * P->sh_rest[45 * i + 3 * (k - 1) + ch];
        }
        o->raw[ch] = v;
        o->clamped[ch] = (v < 0.0);
        o->rgb[ch] = o->clamped[ch] ? 0.0 : v;
    }
    if (!finite3(o->rgb)) return 0;
    o->visible = 1;
    return 1;
}

/* Per-Gaussian outputs of one view, structure of arrays. */
typedef struct {
    double *mean2d;   /* [n,2] */
    double *depth;    /* [n] view-space z */
    double *conic;    /* [n,3] */
    double *opacity;  /* [n] */
    double *rgb;      /* [n,3] */
    int32_t *radius;  /* [n], 0 = culled */
    int32_t *rect;    /* [n,4] inclusive pixel rect x_lo, x_hi, y_lo, y_hi */
    double *m_all;    /* [n] margin applying to every pixel of the Gaussian (or NULL) */
    double *m_edge;   /* [n] margin applying to the border pixels of the box (or NULL) */
} orc_splats;

/* Forward preprocess of all Gaussians for one view. */
int orc_preprocess(const orc_params *P, const double *camv, const double *cfgv, orc_splats *S) {
    cam_t cam = read_cam(camv);
    cfg_t cfg = read_cfg(cfgv);
    for (int64_t i = 0; i < P->n; i++) {
        pre_t o;
        int vis = preprocess_one(P, i, &cam, &cfg, &o);
        S->radius[i] = vis ? o.radius : 0;
        for (int k = 0; k < 2; k++) S->mean2d[2 * i + k] = vis ? o.mean2d[k] : 0.0;
        S->depth[i] = vis ? o.tc[2] : 0.0;
        for (int k = 0; k < 3; k++) S->conic[3 * i + k] = vis ? o.conic[k] : 0.0;
        S->opacity[i] = vis ? o.opac : 0.0;
        for (int k = 0; k < 3; k++) S->rgb[3 * i + k] = vis ? o.rgb[k] : 0.0;
        for (int k = 0; k < 4; k++) S->rect[4 * i + k] = vis ? o.rect[k] : 0;
        if (S->m_all) S->m_all[i] = vis ? o.m_all : INFINITY;
        if (S->m_edge) S->m_edge[i] = vis ? o.m_edge : INFINITY;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Keys, sort and tile ranges                                                           */
/* ------------------------------------------------------------------------------------ */
/*
 * For every visible Gaussian i (radius > 0), in increasing i, and every tile of its rect in
 * row-major order, emit key = ((tile_offset + tile) << 32) | float32_bits(depth_i) with value
 * value_offset + i. The keys are then stably sorted, i.e. ties keep emission order. Tiles of
 * the rect: [x_lo / B, x_hi / B] x [y_lo / B, y_hi / B] for tile size B.
 */
static uint32_t f32_bits(double d) {
    float f = (float)d;
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/*
 * Tile cull test of the key definition, in float32. g = (mx, my, a, b, c, tau, b / c, b / a)
 * of one splat as the float32 values of its record. A tile is kept when the minimum over the pixel-centre rectangle
 * [x0, x1] x [y0, y1] (the tile clipped to the splat's rect) of
 * Q(p) = (p - m)^T [[a, b], [b, c]] (p - m) is <= tau. When the centre m is outside the
 * rectangle the minimum lies on an edge facing m; on a vertical edge x = xe the minimiser is
 * y = my - (b / c) (xe - mx) clamped to the edge (a convex 1D quadratic), on a horizontal
 * edge x = mx - (b / a) (ye - my) clamped; the two ratios come from the record. Every step is one float32 operation in the order written
 * (the file is compiled without contraction), as the definition states.
 */
static float quad_f32(float a, float b, float c, float dx, float dy) {
    float q1 = (a * dx) * dx;
    float q2 = ((2.0f * b) * dx) * dy;
    float q3 = (c * dy) * dy;
    return (q1 + q2) + q3;
}

static int tile_keep_f32(const float *g, int x0, int x1, int y0, int y1) {
    float mx = g[0], my = g[1], a = g[2], b = g[3], c = g[4], tau = g[5], bc = g[6], ba = g[7];
    float fx0 = (float)x0, fx1 = (float)x1, fy0 = (float)y0, fy1 = (float)y1;
    if (mx >= fx0 && mx <= fx1 && my >= fy0 && my <= fy1) return 0.0f <= tau;
    float q = INFINITY;
    if (mx < fx0 || mx > fx1) {
        float xe = mx < fx0 ? fx0 : fx1;
        float dx = xe - mx;
        float ys = my - bc * dx;
        float dy = fminf(fmaxf(ys, fy0), fy1) - my;
        q = fminf(q, quad_f32(a, b, c, dx, dy));
    }
    if (my < fy0 || my > fy1) {
        float ye = my < fy0 ? fy0 : fy1;
        float dy = ye - my;
        float xs = mx - ba * dy;
        float dx = fminf(fmaxf(xs, fx0), fx1) - mx;
        q = fminf(q, quad_f32(a, b, c, dx, dy));
    }
    return q <= tau;
}

/* Whether tile (tx, ty) of Gaussian i gets a key: always without cull data, else the test. */
static int key_kept(const int32_t *rect, const float *cull, int64_t i, int tile, int tx, int ty) {
    if (!cull) return 1;
    const int32_t *rc = rect + 4 * i;
    int x0 = tx * tile > rc[0] ? tx * tile : rc[0];
    int x1 = tx * tile + tile - 1 < rc[1] ? tx * tile + tile - 1 : rc[1];
    int y0 = ty * tile > rc[2] ? ty * tile : rc[2];
    int y1 = ty * tile + tile - 1 < rc[3] ? ty * tile + tile - 1 : rc[3];
    return tile_keep_f32(cull + 8 * i, x0, x1, y0, y1);
}

/* Rects are expected inside the image; any other rect is rejected (no keys) rather than
   indexed outside the tile grid. */
static int rect_ok(const int32_t *rc, int W, int H) {
    return rc[0] >= 0 && rc[0] <= rc[1] && rc[1] < W && rc[2] >= 0 && rc[2] <= rc[3] && rc[3] < H;
}

int64_t orc_count_keys(int64_t n, const int32_t *radius, const int32_t *rect, const float *cull,
                       int W, int H, int tile) {
    int64_t K = 0;
    for (int64_t i = 0; i < n; i++) {
        if (radius[i] <= 0 || !rect_ok(rect + 4 * i, W, H)) continue;
        for (int ty = rect[4 * i + 2] / tile; ty <= rect[4 * i + 3] / tile; ty++)
            for (int tx = rect[4 * i + 0] / tile; tx <= rect[4 * i + 1] / tile; tx++)
                K += key_kept(rect, cull, i, tile, tx, ty);
    }
    return K;
}

typedef struct {
    uint64_t key;
    uint32_t val;
} kv_t;

static int kv_cmp(const void *a, const void *b) {
    const kv_t *x = (const kv_t *)a, *y = (const kv_t *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->val != y->val) return x->val < y->val ? -1 : 1;
    return 0;
}

/* Emits and stably sorts the keys of one view. ranges [ntiles,2] gets [start, end) per tile
   (relative to the start of this view's keys), empty tiles [0, 0). Returns K. */
int64_t orc_keys(int64_t n, const int32_t *radius, const int32_t *rect, const double *depth,
                 const float *cull, int W, int H, int tile, uint64_t tile_offset,
                 uint32_t value_offset, uint64_t *keys, uint32_t *vals, uint32_t *ranges) {
    int gx = (W + tile - 1) / tile, gy = (H + tile - 1) / tile;
    int64_t K = orc_count_keys(n, radius, rect, cull, W, H, tile);
    kv_t *kv = (kv_t *)malloc(sizeof(kv_t) * (size_t)(K > 0 ? K : 1));
    int64_t e = 0;
    for (int64_t i = 0; i < n; i++) {
        if (radius[i] <= 0 || !rect_ok(rect + 4 * i, W, H)) continue;
        uint32_t db = f32_bits(depth[i]);
        for (int ty = rect[4 * i + 2] / tile; ty <= rect[4 * i + 3] / tile; ty++)
            for (int tx = rect[4 * i + 0] / tile; tx <= rect[4 * i + 1] / tile; tx++) {
                if (!key_kept(rect, cull, i, tile, tx, ty)) continue;
                uint64_t t = tile_offset + (uint64_t)(ty * gx + tx);
                kv[e].key = (t << 32) | db;
                kv[e].val = value_offset + (uint32_t)i;
                e++;
            }
    }
    /* (key, value) order equals a stable sort on key because values were emitted ascending */
    qsort(kv, (size_t)K, sizeof(kv_t), kv_cmp);
    if (ranges) memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)gx * gy);
    for (int64_t k = 0; k < K; k++) {
        if (keys) keys[k] = kv[k].key;
        if (vals) vals[k] = kv[k].val;
        if (ranges) {
            uint64_t t = (kv[k].key >> 32) - tile_offset;
            if (k == 0 || (kv[k - 1].key >> 32) != (kv[k].key >> 32)) ranges[2 * t] = (uint32_t)k;
            ranges[2 * t + 1] = (uint32_t)(k + 1);
        }
    }
    free(kv);
    return K;
}

/* ------------------------------------------------------------------------------------ */
/* Blend [Eq. 2] and its backward                                                       */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    const orc_splats *S;
    int64_t n;
    int W, H, tile, brute, gx, gy;
    double bg[3];
    const uint32_t *vals;    /* tiled: sorted Gaussian ids */
    const uint32_t *ranges;  /* tiled: per-tile [start, end) */
    const uint32_t *order;   /* brute: visible Gaussians sorted by (depth bits, id) */
    int64_t n_order;
    int use_depth_margin;
    const uint8_t *tile_mask; /* NULL, or 1 for every tile to process */
    /* forward outputs */
    double *image, *T_final, *margin;
    int32_t *last, *n_contrib, *n_examined, *n_eval;
    /* backward */
    const double *dL_dimg;
    double *acc; /* [nthreads][n][9] */
    int64_t *hits; /* [nthreads][n]: fragments blended per Gaussian (significance score) */
    int nthreads;
} blend_job;

typedef struct {
    blend_job *job;
    int tid;
} blend_arg;

/* One fragment as seen by one pixel. */
typedef struct {
    uint32_t id;
    double alpha, T, G, x, dx, dy;
} frag_t;

/* Blend a single pixel; if frags != NULL, also records the contributing fragments. */
static int blend_pixel(const blend_job *J, int px, int py, const uint32_t *list, int64_t len,
                       double C[3], double *T_out, int32_t *last, int32_t *ncontrib,
                       int32_t *nexam, int32_t *neval, double *margin, frag_t *frags) {
    const orc_splats *S = J->S;
    double T = 1.0;
    C[0] = C[1] = C[2] = 0.0;
    int nc = 0;
    int32_t lst = 0, ex = 0, ev = 0;
    double mg = INFINITY;
    double prev_depth = NAN;
    for (int64_t k = 0; k < len; k++) {
        uint32_t g = list[k];
        ex = (int32_t)(k + 1);
        const int32_t *rc = S->rect + 4 * (int64_t)g;
        int inside = (px >= rc[0] && px <= rc[1] && py >= rc[2] && py <= rc[3]);
        int near_edge = (px >= rc[0] - 1 && px <= rc[1] + 1 && py >= rc[2] - 1 && py <= rc[3] + 1) &&
                        (px <= rc[0] || px >= rc[1] || py <= rc[2] || py >= rc[3]);
        if (!inside && !(near_edge && margin)) continue;
        double dx = S->mean2d[2 * g] - px, dy = S->mean2d[2 * g + 1] - py;
        const double *cn = S->conic + 3 * g;
        double power = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
        double G = exp(power);
        double x = S->opacity[g] * G;
        if (!inside) {
            /* box edge that could move by one pixel: would this fragment have counted? */
            if (power <= 0.0 && x >= 1.0 / 255.0 && S->m_edge) mg = fmin(mg, S->m_edge[g]);
            continue;
        }
        ev++;  /* the pixel is in the rect: this fragment is evaluated */
        if (power > 0.0) continue;
        double alpha = fmin(0.99, x);
        if (margin) mg = fmin(mg, fabs(x * 255.0 - 1.0) / 1e-5);
        if (alpha < 1.0 / 255.0) continue;
        if (margin) {
            if (S->m_all) mg = fmin(mg, S->m_all[g]);
            if (near_edge && S->m_edge) mg = fmin(mg, S->m_edge[g]);
            if (J->use_depth_margin && !isnan(prev_depth)) {
                double ulp = fabs(S->depth[g]) * 1.1920928955078125e-07;
                mg = fmin(mg, fabs(S->depth[g] - prev_depth) / (8.0 * ulp));
            }
            prev_depth = S->depth[g];
        }
        double Tn = T * (1.0 - alpha);
        if (margin) mg = fmin(mg, fabs(Tn / 1e-4 - 1.0) / 1e-4);
        if (Tn < 1e-4) break;
        for (int ch = 0; ch < 3; ch++) C[ch] += S->rgb[3 * g + ch] * alpha * T;
        if (frags) {
            frags[nc].id = g;
            frags[nc].alpha = alpha;
            frags[nc].T = T;
            frags[nc].G = G;
            frags[nc].x = x;
            frags[nc].dx = dx;
            frags[nc].dy = dy;
        }
        T = Tn;
        lst = (int32_t)(k + 1);
        nc++;
    }
    *T_out = T;
    *last = lst;
    *ncontrib = nc;
    *nexam = ex;
    *neval = ev;
    if (margin) *margin = mg;
    return nc;
}

/* Backward of one pixel, from its fragments stored in forward order. Adds dL/d(mean2d,
   conic, opacity, rgb) of each fragment's Gaussian to acc[id*9 + ...]. */
static void backward_pixel(const blend_job *J, const frag_t *f, int nc, double T_final,
                           const double dLdC[3], double *acc) {
    const orc_splats *S = J->S;
    /* A_i = colour accumulated behind fragment i, P_i = prod_{j>i} (1 - a_j) */
    double A[3] = {0.0, 0.0, 0.0}, Pbehind = 1.0;
    for (int i = nc - 1; i >= 0; i--) {
        const frag_t *fr = f + i;
        const double *c = S->rgb + 3 * fr->id;
        double *g = acc + 9 * (int64_t)fr->id;
        /* dC/dc_i = a_i T_i */
        for (int ch = 0; ch < 3; ch++) g[6 + ch] += fr->alpha * fr->T * dLdC[ch];
        /* dC/da_i = T_i (c_i - A_i) - T_i P_i bg */
        double dLda = 0.0;
        for (int ch = 0; ch < 3; ch++)
            dLda += dLdC[ch] * (fr->T * (c[ch] - A[ch]) - fr->T * Pbehind * J->bg[ch]);
        /* a = min(0.99, o' G): zero derivative where the clamp is active */
        if (fr->x <= 0.99) {
            const double *cn = S->conic + 3 * fr->id;
            double o = S->opacity[fr->id];
            double dLdG = dLda * o;
            double dLdpow = dLdG * fr->G;
            g[5] += dLda * fr->G;
            g[0] += dLdpow * (-cn[0] * fr->dx - cn[1] * fr->dy);
            g[1] += dLdpow * (-cn[2] * fr->dy - cn[1] * fr->dx);
            g[2] += dLdpow * (-0.5 * fr->dx * fr->dx);
            g[3] += dLdpow * (-fr->dx * fr->dy);
            g[4] += dLdpow * (-0.5 * fr->dy * fr->dy);
        }
        /* move one fragment towards the camera */
        for (int ch = 0; ch < 3; ch++) A[ch] = fr->alpha * c[ch] + (1.0 - fr->alpha) * A[ch];
        Pbehind *= (1.0 - fr->alpha);
    }
    (void)T_final;
}

static void *blend_worker(void *p) {
    blend_arg *a = (blend_arg *)p;
    blend_job *J = a->job;
    int ntiles = J->gx * J->gy;
    int64_t maxlen = J->brute ? J->n_order : 0;
    if (!J->brute)
        for (int t = 0; t < ntiles; t++) {
            int64_t l = (int64_t)J->ranges[2 * t + 1] - J->ranges[2 * t];
            if (l > maxlen) maxlen = l;
        }
    frag_t *frags = NULL;
    if (J->dL_dimg || J->hits) frags = (frag_t *)malloc(sizeof(frag_t) * (size_t)(maxlen > 0 ? maxlen : 1));
    double *acc = J->acc ? J->acc + (int64_t)a->tid * J->n * 9 : NULL;
    int64_t *hits = J->hits ? J->hits + (int64_t)a->tid * J->n : NULL;
    for (int t = a->tid; t < ntiles; t += J->nthreads) {
        if (J->tile_mask && !J->tile_mask[t]) continue;
        int tx = t % J->gx, ty = t / J->gx;
        const uint32_t *list;
        int64_t len;
        if (J->brute) {
            list = J->order;
            len = J->n_order;
        } else {
            list = J->vals + J->ranges[2 * t];
            len = (int64_t)J->ranges[2 * t + 1] - J->ranges[2 * t];
        }
        for (int py = ty * J->tile; py < (ty + 1) * J->tile && py < J->H; py++)
            for (int px = tx * J->tile; px < (tx + 1) * J->tile && px < J->W; px++) {
                int64_t pix = (int64_t)py * J->W + px;
                double C[3], T, mg;
                int32_t lst, nc, ex, ev;
                int ncf = blend_pixel(J, px, py, list, len, C, &T, &lst, &nc, &ex, &ev,
                                      J->margin ? &mg : NULL, frags);
                if (J->image)
                    for (int ch = 0; ch < 3; ch++)
                        J->image[(int64_t)ch * J->W * J->H + pix] = C[ch] + T * J->bg[ch];
                if (J->T_final) J->T_final[pix] = T;
                if (J->last) J->last[pix] = lst;
                if (J->n_contrib) J->n_contrib[pix] = nc;
                if (J->n_examined) J->n_examined[pix] = ex;
                if (J->n_eval) J->n_eval[pix] = ev;
                if (J->margin) J->margin[pix] = mg;
                if (hits)
                    for (int f = 0; f < ncf; f++) hits[frags[f].id]++;
                if (J->dL_dimg) {
                    double d[3];
                    for (int ch = 0; ch < 3; ch++)
                        d[ch] = J->dL_dimg[(int64_t)ch * J->W * J->H + pix];
                    backward_pixel(J, frags, ncf, T, d, acc);
                }
            }
    }
    free(frags);
    return NULL;
}

typedef struct {
    uint32_t db, id;
} did_t;

static int did_cmp(const void *a, const void *b) {
    const did_t *x = (const did_t *)a, *y = (const did_t *)b;
    if (x->db != y->db) return x->db < y->db ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

static int run_blend(blend_job *J) {
    uint64_t *keys = NULL;
    uint32_t *vals = NULL, *ranges = NULL, *order = NULL;
    J->gx = (J->W + J->tile - 1) / J->tile;
    J->gy = (J->H + J->tile - 1) / J->tile;
    if (J->vals && J->ranges) {
        /* lists given by the caller (from orc_keys of the same records) */
    } else if (J->brute) {
        did_t *d = (did_t *)malloc(sizeof(did_t) * (size_t)(J->n > 0 ? J->n : 1));
        int64_t m = 0;
        for (int64_t i = 0; i < J->n; i++)
            if (J->S->radius[i] > 0 && rect_ok(J->S->rect + 4 * i, J->W, J->H)) {
                d[m].db = f32_bits(J->S->depth[i]);
                d[m].id = (uint32_t)i;
                m++;
            }
        qsort(d, (size_t)m, sizeof(did_t), did_cmp);
        order = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
        for (int64_t i = 0; i < m; i++) order[i] = d[i].id;
        free(d);
        J->order = order;
        J->n_order = m;
    } else if (J->tile_mask) {
        /* Only the marked tiles: each one's list is the (depth bits, id) order of the visible
           Gaussians whose rect covers it -- the same lists a full key sort gives them. */
        const int ntile = J->gx * J->gy;
        ranges = (uint32_t *)calloc(2 * (size_t)ntile, sizeof(uint32_t));
        int64_t total = 0;
        for (int pass = 0; pass < 2; pass++) {
            if (pass == 1) {
                uint32_t acc = 0;
                for (int t = 0; t < ntile; t++) {
                    uint32_t c = ranges[2 * t + 1];
                    ranges[2 * t] = acc;
                    ranges[2 * t + 1] = acc;  /* becomes the end while filling */
                    acc += c;
                }
                total = acc;
                vals = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(total > 0 ? total : 1));
            }
            for (int64_t i = 0; i < J->n; i++) {
                if (J->S->radius[i] <= 0 || !rect_ok(J->S->rect + 4 * i, J->W, J->H)) continue;
                const int32_t *rc = J->S->rect + 4 * i;
                for (int ty = rc[2] / J->tile; ty <= rc[3] / J->tile; ty++)
                    for (int tx = rc[0] / J->tile; tx <= rc[1] / J->tile; tx++) {
                        int t = ty * J->gx + tx;
                        if (!J->tile_mask[t]) continue;
                        if (pass == 0) ranges[2 * t + 1]++;
                        else vals[ranges[2 * t + 1]++] = (uint32_t)i;
                    }
            }
        }
        for (int t = 0; t < ntile; t++) {
            uint32_t a = ranges[2 * t], b = ranges[2 * t + 1];
            if (b - a < 2) continue;
            did_t *d = (did_t *)malloc(sizeof(did_t) * (b - a));
            for (uint32_t k = a; k < b; k++) {
                d[k - a].db = f32_bits(J->S->depth[vals[k]]);
                d[k - a].id = vals[k];
            }
            qsort(d, b - a, sizeof(did_t), did_cmp);
            for (uint32_t k = a; k < b; k++) vals[k] = d[k - a].id;
            free(d);
        }
        (void)total;
        J->vals = vals;
        J->ranges = ranges;
    } else {
        int64_t K = orc_count_keys(J->n, J->S->radius, J->S->rect, NULL, J->W, J->H, J->tile);
        vals = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(K > 0 ? K : 1));
        ranges = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)J->gx * J->gy);
        orc_keys(J->n, J->S->radius, J->S->rect, J->S->depth, NULL, J->W, J->H, J->tile, 0, 0,
                 NULL, vals, ranges);
        J->vals = vals;
        J->ranges = ranges;
    }
    int nt = J->nthreads < 1 ? 1 : J->nthreads;
    J->nthreads = nt;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nt);
    blend_arg *args = (blend_arg *)malloc(sizeof(blend_arg) * nt);
    for (int i = 0; i < nt; i++) {
        args[i].job = J;
        args[i].tid = i;
        if (nt == 1)
            blend_worker(&args[i]);
        else
            pthread_create(&th[i], NULL, blend_worker, &args[i]);
    }
    if (nt > 1)
        for (int i = 0; i < nt; i++) pthread_join(th[i], NULL);
    free(th);
    free(args);
    free(keys);
    free(vals);
    free(ranges);
    free(order);
    return 0;
}

/* Forward blend of one view. brute = 1 scans all Gaussians per pixel in (depth, id) order
   instead of the tile lists. Any output pointer may be NULL. */
int orc_blend(int64_t n, const orc_splats *S, int W, int H, int tile, const double *bg,
              int brute, int nthreads, int use_depth_margin, const uint8_t *tile_mask,
              const uint32_t *list_vals, const uint32_t *list_ranges,
              double *image, double *T_final, int32_t *last, int32_t *n_contrib,
              int32_t *n_examined, int32_t *n_eval, double *margin) {
    blend_job J;
    memset(&J, 0, sizeof J);
    J.tile_mask = tile_mask;
    J.vals = list_vals;
    J.ranges = list_ranges;
    J.S = S;
    J.n = n;
    J.W = W;
    J.H = H;
    J.tile = tile;
    J.brute = brute;
    for (int c = 0; c < 3; c++) J.bg[c] = bg[c];
    J.nthreads = nthreads;
    J.use_depth_margin = use_depth_margin;
    J.image = image;
    J.T_final = T_final;
    J.last = last;
    J.n_contrib = n_contrib;
    J.n_examined = n_examined;
    J.n_eval = n_eval;
    J.margin = margin;
    return run_blend(&J);
}

/* Backward of the blend of one view: writes dL/d(mean2d[2], conic[3], opacity, rgb[3]) per
   Gaussian into g9 [n,9] (overwritten). */
int orc_blend_backward(int64_t n, const orc_splats *S, int W, int H, int tile, const double *bg,
                       const double *dL_dimg, int nthreads, const uint8_t *tile_mask,
                       const uint32_t *list_vals, const uint32_t *list_ranges, double *g9) {
    blend_job J;
    memset(&J, 0, sizeof J);
    J.tile_mask = tile_mask;
    J.vals = list_vals;
    J.ranges = list_ranges;
    J.S = S;
    J.n = n;
    J.W = W;
    J.H = H;
    J.tile = tile;
    for (int c = 0; c < 3; c++) J.bg[c] = bg[c];
    J.nthreads = nthreads < 1 ? 1 : nthreads;
    J.dL_dimg = dL_dimg;
    J.acc = (double *)calloc((size_t)J.nthreads * (size_t)n * 9, sizeof(double));
    run_blend(&J);
    memset(g9, 0, sizeof(double) * 9 * (size_t)n);
    for (int t = 0; t < J.nthreads; t++)
        for (int64_t i = 0; i < 9 * n; i++) g9[i] += J.acc[(int64_t)t * 9 * n + i];
    free(J.acc);
    return 0;
}

/* Ray hits of Eq. significance-score for one view: per Gaussian, the number of pixels whose
   forward blend (Eq. 2) blends it, i.e. the indicator 1(G(X_j), r_i) summed over the
   view's rays, read as "fragment j contributes to pixel i" (alpha >= 1/255, before the
   pixel's stop). Adds into hits [n]. */
int orc_hits(int64_t n, const orc_splats *S, int W, int H, int tile, int brute, int nthreads,
             const uint8_t *tile_mask, const uint32_t *list_vals, const uint32_t *list_ranges,
             int64_t *hits) {
    blend_job J;
    memset(&J, 0, sizeof J);
    J.tile_mask = tile_mask;
    J.vals = list_vals;
    J.ranges = list_ranges;
    J.S = S;
    J.n = n;
    J.W = W;
    J.H = H;
    J.tile = tile;
    J.brute = brute;
    J.nthreads = nthreads < 1 ? 1 : nthreads;
    J.hits = (int64_t *)calloc((size_t)J.nthreads * (size_t)(n > 0 ? n : 1), sizeof(int64_t));
    run_blend(&J);
    for (int t = 0; t < J.nthreads; t++)
        for (int64_t i = 0; i < n; i++) hits[i] += J.hits[(int64_t)t * n + i];
    free(J.hits);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Backward of the preprocess: chain rule to all inputs, plus densification statistics   */
/* ------------------------------------------------------------------------------------ */
/*
 * g9 [n,9] holds dL/d(mean2d x, y; conic a, b, c; opacity; rgb r, g, b) for this view, with
 * the conic gradient taken with respect to the scalar b of power = -1/2(a dx^2 + c dy^2)
 * - b dx dy. Gradients are ADDED into G (so several views accumulate). Statistics: for every
 * Gaussian visible in this view, stat_accum += |dL/dmean2d|_2 (pixel units), stat_count += 1,
 * stat_maxr = max(stat_maxr, radius).
 */
int orc_preprocess_backward(const orc_params *P, const double *camv, const double *cfgv,
                            const double *g9, orc_grads *G, double *stat_accum,
                            int32_t *stat_count, int32_t *stat_maxr) {
    cam_t cam = read_cam(camv);
    cfg_t cfg = read_cfg(cfgv);
    for (int64_t i = 0; i < P->n; i++) {
        pre_t o;
        if (!preprocess_one(P, i, &cam, &cfg, &o)) continue;
        const double *g = g9 + 9 * i;
        if (stat_accum) stat_accum[i] += sqrt(g[0] * g[0] + g[1] * g[1]);
        if (stat_count) stat_count[i] += 1;
        if (stat_maxr && o.radius > stat_maxr[i]) stat_maxr[i] = o.radius;

        double g_mu[3] = {0, 0, 0};
        double g_M = 0.0;

        /* --- colour --- */
        double g_raw[3];
        for (int ch = 0; ch < 3; ch++) g_raw[ch] = o.clamped[ch] ? 0.0 : g[6 + ch];
        if (G->sh_dc)
            for (int ch = 0; ch < 3; ch++) G->sh_dc[3 * i + ch] += o.Y[0] * g_raw[ch];
        double g_dir[3] = {0, 0, 0};
        double g_band[4] = {0, 0, 0, 0};
        for (int k = 1; k < 16 && P->sh_rest; k++) {
            int l = (k < 4) ? 1 : (k < 9) ? 2 : 3;
            if (l > o.deg) continue;
            for (int ch = 0; ch < 3; ch++) {
                double f = P->sh_rest[45 * i + 3 * (k - 1) + ch];
                /* straight-through band mask: d/dM^l is taken whatever the hard value */
                g_band[l] += o.Y[k] * f * g_raw[ch];
                if (o.Msh[l] == 0.0) continue;
                if (G->sh_rest) G->sh_rest[45 * i + 3 * (k - 1) + ch] += o.Msh[l] * o.Y[k] * g_raw[ch];
                for (int c = 0; c < 3; c++) g_dir[c] += o.Msh[l] * f * o.dY[k][c] * g_raw[ch];
            }
        }
        if (P->sh_mask_logits && G->sh_mask_logits)
            for (int l = 1; l <= 3; l++) {
                if (l > o.deg) continue;
                double s = sigmoid(P->sh_mask_logits[3 * i + l - 1]);
                G->sh_mask_logits[3 * i + l - 1] += g_band[l] * s * (1.0 - s);
            }
        /* unit direction d = v / |v|: dL/dv = (I - d d^T) dL/dd / |v| */
        {
            double dd = g_dir[0] * o.dir[0] + g_dir[1] * o.dir[1] + g_dir[2] * o.dir[2];
            for (int c = 0; c < 3; c++) g_mu[c] += (g_dir[c] - o.dir[c] * dd) / o.dist;
        }

        /* --- opacity o' = M sigma(o) --- */
        if (G->opacity_logits) G->opacity_logits[i] += g[5] * o.M * o.sig_o * (1.0 - o.sig_o);
        g_M += g[5] * o.sig_o;

        /* --- conic = Sigma'^-1: dL/dSigma' = -Q dL/dQ Q with Q symmetric --- */
        double Q[2][2] = {{o.conic[0], o.conic[1]}, {o.conic[1], o.conic[2]}};
        double GQ[2][2] = {{g[2], 0.5 * g[3]}, {0.5 * g[3], g[4]}};
        double tmp[2][2], GS2[2][2];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 2; c++) tmp[r][c] = Q[r][0] * GQ[0][c] + Q[r][1] * GQ[1][c];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 2; c++) GS2[r][c] = -(tmp[r][0] * Q[0][c] + tmp[r][1] * Q[1][c]);

        /* --- Sigma' = T Sigma T^T + sI, T = J W: dL/dSigma = T^T G T, dL/dT = 2 G T Sigma --- */
        double GSig[3][3];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double acc = 0.0;
                for (int r = 0; r < 2; r++)
                    for (int c = 0; c < 2; c++) acc += o.T2[r][a] * GS2[r][c] * o.T2[c][b];
                GSig[a][b] = acc;
            }
        double GT[2][3];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++) {
                double acc = 0.0;
                for (int k = 0; k < 2; k++)
                    for (int m = 0; m < 3; m++) acc += GS2[r][k] * o.T2[k][m] * o.Sigma[m][c];
                GT[r][c] = 2.0 * acc;
            }
        /* T = J R_view: dL/dJ = dL/dT R_view^T */
        double GJ[2][3];
        for (int r = 0; r < 2; r++)
            for (int c = 0; c < 3; c++)
                GJ[r][c] = GT[r][0] * cam.R[c][0] + GT[r][1] * cam.R[c][1] + GT[r][2] * cam.R[c][2];

        /* --- J(t) and mean2d(t) --- */
        double tx = o.tc[0], ty = o.tc[1], tz = o.tc[2];
        double g_t[3] = {0, 0, 0};
        /* J00 = fx / tz, J11 = fy / tz */
        g_t[2] += GJ[0][0] * (-cam.fx / (tz * tz)) + GJ[1][1] * (-cam.fy / (tz * tz));
        /* J02 = -fx u / tz with u = clamp(tx / tz) */
        {
            double du_dtx = o.clamp_x ? 0.0 : 1.0 / tz;
            double du_dtz = o.clamp_x ? 0.0 : -tx / (tz * tz);
            g_t[0] += GJ[0][2] * (-cam.fx / tz) * du_dtx;
            g_t[2] += GJ[0][2] * (cam.fx * o.u / (tz * tz) - cam.fx / tz * du_dtz);
            double dw_dty = o.clamp_y ? 0.0 : 1.0 / tz;
            double dw_dtz = o.clamp_y ? 0.0 : -ty / (tz * tz);
            g_t[1] += GJ[1][2] * (-cam.fy / tz) * dw_dty;
            g_t[2] += GJ[1][2] * (cam.fy * o.w / (tz * tz) - cam.fy / tz * dw_dtz);
        }
        /* mean2d = (fx tx / tz + cx - 1/2, fy ty / tz + cy - 1/2) */
        g_t[0] += g[0] * cam.fx / tz;
        g_t[2] += g[0] * (-cam.fx * tx / (tz * tz));
        g_t[1] += g[1] * cam.fy / tz;
        g_t[2] += g[1] * (-cam.fy * ty / (tz * tz));
        /* t = R_view mu + t_view */
        for (int c = 0; c < 3; c++)
            g_mu[c] += cam.R[0][c] * g_t[0] + cam.R[1][c] * g_t[1] + cam.R[2][c] * g_t[2];

        /* --- Sigma = (R S)(R S)^T: dL/d(RS) = 2 G (RS) --- */
        double RS[3][3], GRS[3][3];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) RS[r][c] = o.Rq[r][c] * o.scale[c];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                double acc = 0.0;
                for (int k = 0; k < 3; k++) acc += (GSig[r][k] + GSig[k][r]) * RS[k][c];
                GRS[r][c] = acc;
            }
        double g_scale[3] = {0, 0, 0}, GR[3][3];
        for (int r = 0; r < 3; r++)
            for (int c = 0; c < 3; c++) {
                g_scale[c] += GRS[r][c] * o.Rq[r][c];
                GR[r][c] = GRS[r][c] * o.scale[c];
            }
        /* s = M exp(l) */
        for (int c = 0; c < 3; c++) {
            if (G->log_scales) G->log_scales[3 * i + c] += g_scale[c] * o.scale[c];
            g_M += g_scale[c] * exp(P->log_scales[3 * i + c]);
        }
        /* R(q_hat), q_hat = q / |q| */
        double dR[4][3][3], g_qn[4] = {0, 0, 0, 0};
        quat_to_rot_partials(o.qn, dR);
        for (int k = 0; k < 4; k++)
            for (int r = 0; r < 3; r++)
                for (int c = 0; c < 3; c++) g_qn[k] += GR[r][c] * dR[k][r][c];
        double qd = 0.0;
        for (int k = 0; k < 4; k++) qd += g_qn[k] * o.qn[k];
        if (G->quats)
            for (int k = 0; k < 4; k++) G->quats[4 * i + k] += (g_qn[k] - o.qn[k] * qd) / o.qnorm;

        if (G->means)
            for (int c = 0; c < 3; c++) G->means[3 * i + c] += g_mu[c];
        /* straight-through volume mask: dL/dm = dL/dM sigma'(m) */
        if (P->mask_logits && G->mask_logits) {
            double s = sigmoid(P->mask_logits[i]);
            G->mask_logits[i] += g_M * s * (1.0 - s);
        }
    }
    return 0;
}

/* Mean-reduced L1 loss of one view and its gradient: loss += scale * sum |img - target|,
   dL/dimg = scale * sign(img - target) with sign(0) = 0. */
double orc_l1(int64_t m, const double *img, const double *target, double scale, double *grad) {
    double s = 0.0;
    for (int64_t i = 0; i < m; i++) {
        double d = img[i] - target[i];
        s += fabs(d);
        if (grad) grad[i] = scale * (d > 0.0 ? 1.0 : (d < 0.0 ? -1.0 : 0.0));
    }
    return s * scale;
}
