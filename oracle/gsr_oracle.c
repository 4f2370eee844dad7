/*
 * gsr_oracle.c -- plain, slow FP64 CPU reference of the differentiable
 * Gaussian rasteriser.  TEST INFRASTRUCTURE ONLY: it is used by tests/,
 * by __graft_entry__.smoke() and by bench.py's cpu_baseline leg, never by
 * the product path.  It shares no code, header or constant with the CUDA
 * library.
 *
 * What it computes (paper Sec. 3.3, Eq. "rendering"):
 *   C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j),   alpha_i = sigma_i G_i,
 * with c_i the colour converted from spherical harmonics and G_i the
 * projected 2-D Gaussian of primitive i (position P, rotation r, scale s,
 * density sigma, SH coefficients), rendered at a keyframe pose (R, t) into
 * colour, depth and opacity, and differentiated by backpropagation with
 * respect to every Gaussian parameter and to the keyframe pose (Sec. 3.3,
 * last paragraph; Supp. Sec. 1.3 "Feedback").
 *
 * Readings where the paper is silent (3DGS conventions it inherits):
 *   - product index: prod_{j<i}(1 - alpha_j) (the printed equation repeats i);
 *   - Sigma = R diag(s^2) R^T, R from the normalised quaternion (w,x,y,z),
 *     s = exp(log_s), sigma = 1/(1+exp(-logit));
 *   - camera frame p = W P + t; Gaussians with p_z <= 0.2 are culled;
 *   - EWA: Sigma' = J W Sigma W^T J^T + 0.3 I, J the pinhole Jacobian at p
 *     with x/z, y/z clamped to +-1.3 * (W/2)/fx, (H/2)/fy; det(Sigma') <= 0
 *     culls; pixel centres sit at integer (x, y); u = fx x/z + cx;
 *   - per pixel: Gaussians with Mahalanobis d^2 <= 9 on Sigma', sorted by
 *     (z, index); alpha = min(0.99, sigma exp(-d^2/2)); alpha < 1/255 is
 *     skipped; if T(1 - alpha) < 1e-4 the walk stops without adding it;
 *   - colour c = max(0, sum_k SH_k Y_k(dir) + 0.5), dir = (P - C)/|P - C|,
 *     C = -W^T t, real SH with the Condon-Shortley phase, order (l, m=-l..l);
 *   - depth D = sum_i w_i z_i (w_i = alpha_i T_i), opacity A = sum_i w_i;
 *   - median depth (the paper renders "median depth" as MonoGS does): the z
 *     of the last contributor whose transmittance in front of it, T_i, is
 *     above 0.5 -- the Gaussian during which the accumulated opacity passes
 *     0.5, or the last contributor if it never does; 0 without contributors.
 *     Its gradient goes to that contributor's z only;
 *   - pose gradient: left perturbation T_cw <- Exp(xi) T_cw, xi = (rho, phi),
 *     taken at xi = 0;
 *   - gradients through the alpha clamp, the colour clamp and a clamped
 *     Jacobian coordinate are zero (exact derivative of the clamped map).
 *
 * Per pixel the oracle also records the smallest relative margin of the
 * threshold decisions it took (cutoff, alpha skip, transmittance stop) and,
 * apart from them, of its depth-order decisions, so that tests can tell
 * FP32-vs-FP64 decision flips from errors.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef struct {
    int N, sh_degree;
    const double *means;          /* [3][N] */
    const double *log_scales;     /* [3][N] */
    const double *quats;          /* [4][N] (w, x, y, z), unnormalised */
    const double *opacity_logits; /* [N] */
    const double *sh;             /* [(deg+1)^2 * 3][N], row k*3 + channel */
} og_gaussians;

typedef struct {
    int H, W;
    double fx, fy, cx, cy;
    double T_cw[12]; /* row-major [W | t], world -> camera */
} og_camera;

#define NEAR_Z 0.2
#define DILATION 0.3
#define CUTOFF_D2 9.0
#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_STOP 1e-4
#define FOV_CLAMP 1.3
#define PI 3.14159265358979323846
#define OG_NOUT 10 /* doubles per pixel written by the render calls */

/* ------------------------------------------------------------------ */
/* Real spherical harmonics up to degree 3 (closed forms on the unit    */
/* sphere, Condon-Shortley phase), and their gradients as polynomials   */
/* in (x, y, z).                                                         */
/* ------------------------------------------------------------------ */
static void sh_basis(int deg, const double d[3], double Y[16], double dY[16][3]) {
    const double x = d[0], y = d[1], z = d[2];
    const double k0 = 0.5 * sqrt(1.0 / PI);
    const double k1 = sqrt(3.0 / (4.0 * PI));
    const double k2a = 0.5 * sqrt(15.0 / PI), k2b = 0.25 * sqrt(5.0 / PI), k2c = 0.25 * sqrt(15.0 / PI);
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * PI)), k3b = 0.5 * sqrt(105.0 / PI);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * PI)), k3d = 0.25 * sqrt(7.0 / PI), k3e = 0.25 * sqrt(105.0 / PI);
    double g[16][3];
    memset(g, 0, sizeof g);
    double v[16] = {0};
    v[0] = k0;
    if (deg >= 1) {
        v[1] = -k1 * y;  g[1][1] = -k1;
        v[2] = k1 * z;   g[2][2] = k1;
        v[3] = -k1 * x;  g[3][0] = -k1;
    }
    if (deg >= 2) {
        v[4] = k2a * x * y;            g[4][0] = k2a * y;  g[4][1] = k2a * x;
        v[5] = -k2a * y * z;           g[5][1] = -k2a * z; g[5][2] = -k2a * y;
        v[6] = k2b * (3 * z * z - 1);  g[6][2] = 6 * k2b * z;
        v[7] = -k2a * x * z;           g[7][0] = -k2a * z; g[7][2] = -k2a * x;
        v[8] = k2c * (x * x - y * y);  g[8][0] = 2 * k2c * x; g[8][1] = -2 * k2c * y;
    }
    if (deg >= 3) {
        v[9] = -k3a * (3 * x * x * y - y * y * y);
        g[9][0] = -6 * k3a * x * y; g[9][1] = -k3a * (3 * x * x - 3 * y * y);
        v[10] = k3b * x * y * z;
        g[10][0] = k3b * y * z; g[10][1] = k3b * x * z; g[10][2] = k3b * x * y;
        v[11] = -k3c * y * (5 * z * z - 1);
        g[11][1] = -k3c * (5 * z * z - 1); g[11][2] = -10 * k3c * y * z;
        v[12] = k3d * (5 * z * z * z - 3 * z);
        g[12][2] = k3d * (15 * z * z - 3);
        v[13] = -k3c * x * (5 * z * z - 1);
        g[13][0] = -k3c * (5 * z * z - 1); g[13][2] = -10 * k3c * x * z;
        v[14] = k3e * z * (x * x - y * y);
        g[14][0] = 2 * k3e * x * z; g[14][1] = -2 * k3e * y * z; g[14][2] = k3e * (x * x - y * y);
        v[15] = -k3a * (x * x * x - 3 * x * y * y);
        g[15][0] = -k3a * (3 * x * x - 3 * y * y); g[15][1] = 6 * k3a * x * y;
    }
    for (int k = 0; k < 16; ++k) {
        Y[k] = v[k];
        if (dY) for (int j = 0; j < 3; ++j) dY[k][j] = g[k][j];
    }
}

/* Rotation matrix of the normalised quaternion (w, x, y, z). */
static void quat_to_rot(const double qu[4], double R[3][3]) {
    const double w = qu[0], x = qu[1], y = qu[2], z = qu[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

/* d R / d q_k for the normalised quaternion, k = w, x, y, z. */
static void quat_rot_grad(const double qu[4], double dR[4][3][3]) {
    const double w = qu[0], x = qu[1], y = qu[2], z = qu[3];
    double Rw[3][3] = {{0, -2 * z, 2 * y}, {2 * z, 0, -2 * x}, {-2 * y, 2 * x, 0}};
    double Rx[3][3] = {{0, 2 * y, 2 * z}, {2 * y, -4 * x, -2 * w}, {2 * z, 2 * w, -4 * x}};
    double Ry[3][3] = {{-4 * y, 2 * x, 2 * w}, {2 * x, 0, 2 * z}, {-2 * w, 2 * z, -4 * y}};
    double Rz[3][3] = {{-4 * z, -2 * w, 2 * x}, {2 * w, -4 * z, 2 * y}, {2 * x, 2 * y, 0}};
    memcpy(dR[0], Rw, sizeof Rw);
    memcpy(dR[1], Rx, sizeof Rx);
    memcpy(dR[2], Ry, sizeof Ry);
    memcpy(dR[3], Rz, sizeof Rz);
}

/* ------------------------------------------------------------------ */
/* Projection of one Gaussian into one view (steps: activation, camera  */
/* transform, EWA projection, SH colour).                               */
/* ------------------------------------------------------------------ */
typedef struct {
    int valid;
    double qu[4], qnorm, R[3][3], s[3], Sigma[3][3];
    double pc[3];
    double J[2][3];
    int clamp_x, clamp_y;
    double T[2][3];       /* J W */
    double cov[3];        /* Sigma' = [[cov0, cov1], [cov1, cov2]], dilated */
    double conic[3];      /* Sigma'^-1 = [[c0, c1], [c1, c2]] */
    double u, v, z;
    double opacity;
    double dvec[3], dist, dir[3], Y[16], dY[16][3];
    double raw[3], rgb[3];
} og_proj;

static void project(const og_gaussians *G, const og_camera *cam, int g, og_proj *P) {
    const int N = G->N;
    memset(P, 0, sizeof *P);
    const double *Tc = cam->T_cw;
    const double Wm[3][3] = {{Tc[0], Tc[1], Tc[2]}, {Tc[4], Tc[5], Tc[6]}, {Tc[8], Tc[9], Tc[10]}};
    const double t[3] = {Tc[3], Tc[7], Tc[11]};
    const double mu[3] = {G->means[g], G->means[N + g], G->means[2 * N + g]};

    /* activation and 3-D covariance */
    double q[4];
    for (int k = 0; k < 4; ++k) q[k] = G->quats[k * N + g];
    P->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) P->qu[k] = q[k] / P->qnorm;
    quat_to_rot(P->qu, P->R);
    for (int k = 0; k < 3; ++k) P->s[k] = exp(G->log_scales[k * N + g]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += P->R[i][k] * P->s[k] * P->s[k] * P->R[j][k];
            P->Sigma[i][j] = acc;
        }
    P->opacity = 1.0 / (1.0 + exp(-G->opacity_logits[g]));

    /* camera transform and near cull */
    for (int i = 0; i < 3; ++i) P->pc[i] = Wm[i][0] * mu[0] + Wm[i][1] * mu[1] + Wm[i][2] * mu[2] + t[i];
    const double x = P->pc[0], y = P->pc[1], z = P->pc[2];
    P->z = z;
    if (!(z > NEAR_Z)) return;

    /* EWA projection */
    const double limx = FOV_CLAMP * 0.5 * cam->W / cam->fx, limy = FOV_CLAMP * 0.5 * cam->H / cam->fy;
    double txz = x / z, tyz = y / z;
    P->clamp_x = (txz < -limx || txz > limx);
    P->clamp_y = (tyz < -limy || tyz > limy);
    if (txz < -limx) txz = -limx;
    if (txz > limx) txz = limx;
    if (tyz < -limy) tyz = -limy;
    if (tyz > limy) tyz = limy;
    const double xc = txz * z, yc = tyz * z;
    P->J[0][0] = cam->fx / z; P->J[0][1] = 0;            P->J[0][2] = -cam->fx * xc / (z * z);
    P->J[1][0] = 0;           P->J[1][1] = cam->fy / z;  P->J[1][2] = -cam->fy * yc / (z * z);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += P->J[i][k] * Wm[k][j];
            P->T[i][j] = acc;
        }
    double C2[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += P->T[i][a] * P->Sigma[a][b] * P->T[j][b];
            C2[i][j] = acc;
        }
    P->cov[0] = C2[0][0] + DILATION;
    P->cov[1] = C2[0][1];
    P->cov[2] = C2[1][1] + DILATION;
    const double det = P->cov[0] * P->cov[2] - P->cov[1] * P->cov[1];
    if (!(det > 0)) return;
    P->conic[0] = P->cov[2] / det;
    P->conic[1] = -P->cov[1] / det;
    P->conic[2] = P->cov[0] / det;
    P->u = cam->fx * x / z + cam->cx;
    P->v = cam->fy * y / z + cam->cy;

    /* SH colour */
    const double Cc[3] = {-(Wm[0][0] * t[0] + Wm[1][0] * t[1] + Wm[2][0] * t[2]),
                          -(Wm[0][1] * t[0] + Wm[1][1] * t[1] + Wm[2][1] * t[2]),
                          -(Wm[0][2] * t[0] + Wm[1][2] * t[1] + Wm[2][2] * t[2])};
    for (int i = 0; i < 3; ++i) P->dvec[i] = mu[i] - Cc[i];
    P->dist = sqrt(P->dvec[0] * P->dvec[0] + P->dvec[1] * P->dvec[1] + P->dvec[2] * P->dvec[2]);
    for (int i = 0; i < 3; ++i) P->dir[i] = P->dvec[i] / P->dist;
    sh_basis(G->sh_degree, P->dir, P->Y, P->dY);
    const int K = (G->sh_degree + 1) * (G->sh_degree + 1);
    for (int c = 0; c < 3; ++c) {
        double acc = 0.5;
        for (int k = 0; k < K; ++k) acc += G->sh[(k * 3 + c) * N + g] * P->Y[k];
        P->raw[c] = acc;
        P->rgb[c] = acc > 0 ? acc : 0;
    }
    P->valid = 1;
}

/* Gradients of one (view, Gaussian) projection: from screen-space grads
 * sg = [du, dv, dconic0, dconic1, dconic2, dopacity, dr, dg, db, dz]
 * to parameter grads (accumulated) and the view's pose twist (accumulated). */
static void project_backward(const og_gaussians *G, const og_camera *cam, int g, const og_proj *P,
                             const double sg[10], double *gm, double *gls, double *gq, double *gl,
                             double *gsh, double pose[6]) {
    const int N = G->N;
    const double *Tc = cam->T_cw;
    const double Wm[3][3] = {{Tc[0], Tc[1], Tc[2]}, {Tc[4], Tc[5], Tc[6]}, {Tc[8], Tc[9], Tc[10]}};
    const double x = P->pc[0], y = P->pc[1], z = P->pc[2];
    double dpc[3] = {0, 0, 0};
    double dmu[3] = {0, 0, 0};

    /* opacity logit */
    gl[g] += sg[5] * P->opacity * (1 - P->opacity);

    /* colour -> SH coefficients and view direction */
    const int K = (G->sh_degree + 1) * (G->sh_degree + 1);
    double ddir[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c) {
        if (!(P->raw[c] > 0)) continue;
        const double dr = sg[6 + c];
        for (int k = 0; k < K; ++k) {
            gsh[(k * 3 + c) * N + g] += dr * P->Y[k];
            const double coef = G->sh[(k * 3 + c) * N + g];
            for (int j = 0; j < 3; ++j) ddir[j] += dr * coef * P->dY[k][j];
        }
    }
    /* dir = dvec/|dvec|: project out the radial part */
    double dd = ddir[0] * P->dir[0] + ddir[1] * P->dir[1] + ddir[2] * P->dir[2];
    double ddvec[3];
    for (int j = 0; j < 3; ++j) ddvec[j] = (ddir[j] - P->dir[j] * dd) / P->dist;
    for (int j = 0; j < 3; ++j) dmu[j] += ddvec[j];
    /* camera centre C = -W^T t moves by -W^T rho under the left perturbation */
    double dC[3] = {-ddvec[0], -ddvec[1], -ddvec[2]};

    /* pixel mean and depth */
    dpc[0] += sg[0] * cam->fx / z;
    dpc[1] += sg[1] * cam->fy / z;
    dpc[2] += -sg[0] * cam->fx * x / (z * z) - sg[1] * cam->fy * y / (z * z);
    dpc[2] += sg[9];

    /* conic -> Sigma' (matrix form; the off-diagonal scalar appears twice) */
    const double Gc[2][2] = {{sg[2], 0.5 * sg[3]}, {0.5 * sg[3], sg[4]}};
    const double Ci[2][2] = {{P->conic[0], P->conic[1]}, {P->conic[1], P->conic[2]}};
    double tmp[2][2], dS2[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) tmp[i][j] = Gc[i][0] * Ci[0][j] + Gc[i][1] * Ci[1][j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) dS2[i][j] = -(Ci[i][0] * tmp[0][j] + Ci[i][1] * tmp[1][j]);

    /* Sigma' = T Sigma T^T (+ dilation): grads of Sigma and T */
    double dSigma[3][3], dT[2][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) acc += P->T[i][a] * dS2[i][j] * P->T[j][b];
            dSigma[a][b] = acc;
        }
    for (int i = 0; i < 2; ++i)
        for (int a = 0; a < 3; ++a) {
            double acc = 0;
            for (int j = 0; j < 2; ++j)
                for (int b = 0; b < 3; ++b) acc += dS2[i][j] * P->T[j][b] * P->Sigma[b][a];
            dT[i][a] = 2 * acc;
        }
    /* T = J W */
    double dJ[2][3], dWcov[3][3];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += dT[i][j] * Wm[k][j];
            dJ[i][k] = acc;
        }
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) dWcov[k][j] = P->J[0][k] * dT[0][j] + P->J[1][k] * dT[1][j];
    /* J(p) with the clamped x/z, y/z */
    const double fx = cam->fx, fy = cam->fy;
    const double limx = FOV_CLAMP * 0.5 * cam->W / fx, limy = FOV_CLAMP * 0.5 * cam->H / fy;
    double txz = x / z, tyz = y / z;
    if (txz < -limx) txz = -limx;
    if (txz > limx) txz = limx;
    if (tyz < -limy) tyz = -limy;
    if (tyz > limy) tyz = limy;
    const double xc = txz * z, yc = tyz * z;
    dpc[2] += dJ[0][0] * (-fx / (z * z)) + dJ[1][1] * (-fy / (z * z));
    if (P->clamp_x) {
        dpc[2] += dJ[0][2] * fx * xc / (z * z * z);
    } else {
        dpc[0] += dJ[0][2] * (-fx / (z * z));
        dpc[2] += dJ[0][2] * 2 * fx * x / (z * z * z);
    }
    if (P->clamp_y) {
        dpc[2] += dJ[1][2] * fy * yc / (z * z * z);
    } else {
        dpc[1] += dJ[1][2] * (-fy / (z * z));
        dpc[2] += dJ[1][2] * 2 * fy * y / (z * z * z);
    }

    /* p = W mu + t */
    for (int j = 0; j < 3; ++j) dmu[j] += Wm[0][j] * dpc[0] + Wm[1][j] * dpc[1] + Wm[2][j] * dpc[2];
    for (int j = 0; j < 3; ++j) gm[j * N + g] += dmu[j];

    /* Sigma = M M^T, M = R diag(s) */
    double M[3][3], dM[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = P->R[i][j] * P->s[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += (dSigma[i][k] + dSigma[k][i]) * M[k][j];
            dM[i][j] = acc;
        }
    double dR[3][3];
    for (int j = 0; j < 3; ++j) {
        double ds = 0;
        for (int i = 0; i < 3; ++i) {
            ds += dM[i][j] * P->R[i][j];
            dR[i][j] = dM[i][j] * P->s[j];
        }
        gls[j * N + g] += ds * P->s[j];
    }
    double dRq[4][3][3], dqu[4];
    quat_rot_grad(P->qu, dRq);
    for (int k = 0; k < 4; ++k) {
        double acc = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) acc += dR[i][j] * dRq[k][i][j];
        dqu[k] = acc;
    }
    double qd = 0;
    for (int k = 0; k < 4; ++k) qd += P->qu[k] * dqu[k];
    for (int k = 0; k < 4; ++k) gq[k * N + g] += (dqu[k] - P->qu[k] * qd) / P->qnorm;

    /* pose twist (rho, phi) of the left perturbation Exp(xi) T_cw:
     *   p' = R(phi) p + rho, W' = R(phi) W, C' = C - W^T rho  */
    for (int i = 0; i < 3; ++i)
        pose[i] += dpc[i] - (Wm[i][0] * dC[0] + Wm[i][1] * dC[1] + Wm[i][2] * dC[2]);
    pose[3] += P->pc[1] * dpc[2] - P->pc[2] * dpc[1];
    pose[4] += P->pc[2] * dpc[0] - P->pc[0] * dpc[2];
    pose[5] += P->pc[0] * dpc[1] - P->pc[1] * dpc[0];
    double A[3][3]; /* dWcov W^T */
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) A[i][k] = dWcov[i][0] * Wm[k][0] + dWcov[i][1] * Wm[k][1] + dWcov[i][2] * Wm[k][2];
    pose[3] += A[2][1] - A[1][2];
    pose[4] += A[0][2] - A[2][0];
    pose[5] += A[1][0] - A[0][1];
}

/* ------------------------------------------------------------------ */
/* Per-pixel compositing.                                               */
/* ------------------------------------------------------------------ */
typedef struct { double z; int g; double d2; } cand_t;

typedef struct {
    int g;
    double alpha, Gexp, T, dx, dy;
    int clamped;
} contrib_t;

static int cand_cmp(const void *a, const void *b) {
    const cand_t *x = a, *y = b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return (x->g > y->g) - (x->g < y->g);
}

static double fmin2(double a, double b) { return a < b ? a : b; }

/* Composites one pixel from its candidate list.  Fills out[0..2] colour,
 * out[3] depth, out[4] opacity (sum of weights), out[5] final transmittance,
 * out[6] threshold margin (cutoff, alpha skip, transmittance stop),
 * out[7] median depth, out[8] the median's decision margin (min over
 * contributors of |T_i / 0.5 - 1|), out[9] depth-order margin (the smallest
 * relative gap between the depths of consecutive candidates up to the one
 * the walk stopped at, and the one after it); returns the number of
 * contributors written. */
typedef struct {
    cand_t *buf;
    contrib_t *con;
    double *psg;
    int cap;
} scratch_t;

static void scratch_reserve(scratch_t *s, int n, int want_bwd) {
    if (n <= s->cap) return;
    int cap = s->cap ? s->cap : 256;
    while (cap < n) cap *= 2;
    s->buf = realloc(s->buf, sizeof(cand_t) * (size_t)cap);
    if (want_bwd) {
        s->con = realloc(s->con, sizeof(contrib_t) * (size_t)cap);
        s->psg = realloc(s->psg, sizeof(double) * 10 * (size_t)cap);
    }
    s->cap = cap;
}

static int pixel_forward(const og_proj *P, const int *cand, int ncand, double px, double py,
                         scratch_t *s, int want_bwd, double out[OG_NOUT], int *ncontrib) {
    int n = 0;
    const double keep_d2 = CUTOFF_D2 * (1 + 1e-3);
    for (int k = 0; k < ncand; ++k) {
        const og_proj *p = &P[cand[k]];
        if (!p->valid) continue;
        const double dx = px - p->u, dy = py - p->v;
        const double d2 = p->conic[0] * dx * dx + 2 * p->conic[1] * dx * dy + p->conic[2] * dy * dy;
        if (d2 <= keep_d2) {
            scratch_reserve(s, n + 1, want_bwd);
            cand_t *buf = s->buf;
            buf[n].z = p->z;
            buf[n].g = cand[k];
            buf[n].d2 = d2;
            ++n;
        }
    }
    cand_t *buf = s->buf;
    contrib_t *con = want_bwd ? s->con : NULL;
    if (n > 0) qsort(buf, n, sizeof(cand_t), cand_cmp);
    double T = 1, C[3] = {0, 0, 0}, D = 0, A = 0, margin = 1e30, Zmed = 0, mmed = 1e30, zmargin = 1e30;
    int nc = 0;
    double prev_z = -1;
    for (int k = 0; k < n; ++k) {
        const og_proj *p = &P[buf[k].g];
        const double d2 = buf[k].d2;
        margin = fmin2(margin, fabs(d2 - CUTOFF_D2) / CUTOFF_D2);
        /* an exact tie is ordered by the index on either side, whatever the
         * precision; only distinct close depths can swap under rounding */
        if (prev_z > 0 && p->z != prev_z) zmargin = fmin2(zmargin, fabs(p->z - prev_z) / p->z);
        prev_z = p->z;
        if (d2 > CUTOFF_D2) continue;
        const double Gexp = exp(-0.5 * d2);
        const double a_raw = p->opacity * Gexp;
        margin = fmin2(margin, fabs(a_raw / ALPHA_MIN - 1));
        if (a_raw < ALPHA_MIN) continue;
        const int clamped = a_raw > ALPHA_MAX;
        const double alpha = clamped ? ALPHA_MAX : a_raw;
        const double Tn = T * (1 - alpha);
        margin = fmin2(margin, fabs(Tn / T_STOP - 1));
        if (Tn < T_STOP) {
            /* the candidate after the stop would have been reached first had
             * the two depths swapped */
            if (k + 1 < n && P[buf[k + 1].g].z != p->z)
                zmargin = fmin2(zmargin, fabs(P[buf[k + 1].g].z - p->z) / P[buf[k + 1].g].z);
            break;
        }
        const double w = alpha * T;
        mmed = fmin2(mmed, fabs(T / 0.5 - 1));
        if (T > 0.5) Zmed = p->z;
        for (int c = 0; c < 3; ++c) C[c] += w * p->rgb[c];
        D += w * p->z;
        A += w;
        if (con) {
            con[nc].g = buf[k].g;
            con[nc].alpha = alpha;
            con[nc].Gexp = Gexp;
            con[nc].T = T;
            con[nc].dx = px - p->u;
            con[nc].dy = py - p->v;
            con[nc].clamped = clamped;
        }
        ++nc;
        T = Tn;
    }
    out[0] = C[0]; out[1] = C[1]; out[2] = C[2];
    out[3] = D; out[4] = A; out[5] = T; out[6] = margin; out[7] = Zmed; out[8] = mmed; out[9] = zmargin;
    *ncontrib = nc;
    return nc;
}

/* Backward of one pixel: writes 10 screen-space grads per contributor.  gM
 * (dL/d median depth) goes to the z of the contributor the median took. */
static void pixel_backward(const og_proj *P, const contrib_t *con, int nc, double T_final,
                           const double gC[3], double gD, double gA, double gM, double *sg /* [nc][10] */) {
    int med = -1;
    for (int i = 0; i < nc; ++i)
        if (con[i].T > 0.5) med = i;
    double BC[3] = {0, 0, 0}, BD = 0;
    for (int i = nc - 1; i >= 0; --i) {
        const og_proj *p = &P[con[i].g];
        const double a = con[i].alpha, Ti = con[i].T;
        double *o = sg + 10 * i;
        for (int c = 0; c < 10; ++c) o[c] = 0;
        for (int c = 0; c < 3; ++c) o[6 + c] = gC[c] * a * Ti;
        o[9] = gD * a * Ti + (i == med ? gM : 0.0);
        double dA = Ti * ((p->rgb[0] - BC[0]) * gC[0] + (p->rgb[1] - BC[1]) * gC[1] +
                          (p->rgb[2] - BC[2]) * gC[2] + (p->z - BD) * gD) +
                    gA * T_final / (1 - a);
        for (int c = 0; c < 3; ++c) BC[c] = BC[c] * (1 - a) + p->rgb[c] * a;
        BD = BD * (1 - a) + p->z * a;
        if (con[i].clamped) continue;
        o[5] = dA * con[i].Gexp;
        const double dd2 = dA * (-0.5 * a);
        const double dx = con[i].dx, dy = con[i].dy;
        o[0] = dd2 * (-2) * (p->conic[0] * dx + p->conic[1] * dy);
        o[1] = dd2 * (-2) * (p->conic[1] * dx + p->conic[2] * dy);
        o[2] = dd2 * dx * dx;
        o[3] = dd2 * 2 * dx * dy;
        o[4] = dd2 * dy * dy;
    }
}

/* ------------------------------------------------------------------ */
/* Candidate gathering: all Gaussians (brute force) or a bucket grid of */
/* 16-pixel cells built from each Gaussian's padded 3-sigma box.        */
/* ------------------------------------------------------------------ */
#define CELL 16
typedef struct {
    int cw, ch;
    int64_t *start; /* [cw*ch + 1] */
    int *items;
} buckets_t;

static void build_buckets(const og_proj *P, int N, const og_camera *cam, buckets_t *B) {
    B->cw = (cam->W + CELL - 1) / CELL;
    B->ch = (cam->H + CELL - 1) / CELL;
    const int ncell = B->cw * B->ch;
    B->start = calloc((size_t)ncell + 1, sizeof(int64_t));
    const double r2 = CUTOFF_D2 * (1 + 2e-3);
    for (int pass = 0; pass < 2; ++pass) {
        int64_t *fill = NULL;
        if (pass == 1) {
            for (int c = 0; c < ncell; ++c) B->start[c + 1] += B->start[c];
            B->items = malloc(sizeof(int) * (size_t)(B->start[ncell] > 0 ? B->start[ncell] : 1));
            fill = calloc((size_t)ncell, sizeof(int64_t));
        }
        for (int g = 0; g < N; ++g) {
            const og_proj *p = &P[g];
            if (!p->valid) continue;
            const double ex = sqrt(r2 * p->cov[0]) + 1, ey = sqrt(r2 * p->cov[2]) + 1;
            double x0 = ceil(p->u - ex), x1 = floor(p->u + ex), y0 = ceil(p->v - ey), y1 = floor(p->v + ey);
            if (x0 < 0) x0 = 0;
            if (y0 < 0) y0 = 0;
            if (x1 > cam->W - 1) x1 = cam->W - 1;
            if (y1 > cam->H - 1) y1 = cam->H - 1;
            if (x0 > x1 || y0 > y1) continue;
            for (int cy = (int)y0 / CELL; cy <= (int)y1 / CELL; ++cy)
                for (int cx = (int)x0 / CELL; cx <= (int)x1 / CELL; ++cx) {
                    const int c = cy * B->cw + cx;
                    if (pass == 0) B->start[c + 1]++;
                    else B->items[B->start[c] + fill[c]++] = g;
                }
        }
        free(fill);
    }
}

/* ------------------------------------------------------------------ */
/* Threaded drivers.                                                    */
/* ------------------------------------------------------------------ */
typedef struct {
    const og_proj *P;
    int N;
    const og_camera *cam;
    const buckets_t *B;    /* NULL = brute force */
    const int *all;        /* 0..N-1 for brute force */
    const int64_t *pix;    /* pixel linear indices (y*W + x) */
    int64_t p0, p1;        /* range of pixels for this worker */
    double *out;           /* [npix][OG_NOUT] */
    int32_t *ncontrib;
    /* backward */
    const double *gC, *gD, *gA, *gM;   /* gM may be NULL */
    double *sg;            /* growable [n][10] */
    int *sg_g;
    int64_t sg_n, sg_cap;
} work_t;

static void *worker(void *arg) {
    work_t *w = arg;
    scratch_t s = {0};
    const int want_bwd = w->gC != NULL;
    scratch_reserve(&s, 256, want_bwd);
    for (int64_t i = w->p0; i < w->p1; ++i) {
        const int64_t lin = w->pix[i];
        const int px = (int)(lin % w->cam->W), py = (int)(lin / w->cam->W);
        const int *cand;
        int ncand;
        if (w->B) {
            const int c = (py / CELL) * w->B->cw + px / CELL;
            cand = w->B->items + w->B->start[c];
            ncand = (int)(w->B->start[c + 1] - w->B->start[c]);
        } else {
            cand = w->all;
            ncand = w->N;
        }
        double o[OG_NOUT];
        int nc = 0;
        pixel_forward(w->P, cand, ncand, (double)px, (double)py, &s, want_bwd, o, &nc);
        if (w->out) memcpy(w->out + OG_NOUT * i, o, sizeof o);
        if (w->ncontrib) w->ncontrib[i] = nc;
        if (w->gC) {
            double *psg = s.psg;
            const contrib_t *con = s.con;
            pixel_backward(w->P, con, nc, o[5], w->gC + 3 * i, w->gD[i], w->gA[i], w->gM ? w->gM[i] : 0.0, psg);
            if (w->sg_n + nc > w->sg_cap) {
                int64_t cap = w->sg_cap ? w->sg_cap : 1024;
                while (cap < w->sg_n + nc) cap *= 2;
                w->sg = realloc(w->sg, sizeof(double) * 10 * (size_t)cap);
                w->sg_g = realloc(w->sg_g, sizeof(int) * (size_t)cap);
                w->sg_cap = cap;
            }
            memcpy(w->sg + 10 * w->sg_n, psg, sizeof(double) * 10 * (size_t)nc);
            for (int k = 0; k < nc; ++k) w->sg_g[w->sg_n + k] = con[k].g;
            w->sg_n += nc;
        }
    }
    free(s.buf);
    free(s.con);
    free(s.psg);
    return NULL;
}

typedef struct {
    const og_gaussians *G;
    const og_camera *cam;
    og_proj *P;
    int g0, g1;
} proj_work_t;

static void *proj_worker(void *arg) {
    proj_work_t *w = arg;
    for (int g = w->g0; g < w->g1; ++g) project(w->G, w->cam, g, &w->P[g]);
    return NULL;
}

static int num_threads(int req) {
    if (req > 0) return req;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

static void project_all(const og_gaussians *G, const og_camera *cam, og_proj *P, int nt) {
    pthread_t th[256];
    proj_work_t w[256];
    if (nt > 256) nt = 256;
    for (int k = 0; k < nt; ++k) {
        w[k].G = G; w[k].cam = cam; w[k].P = P;
        w[k].g0 = (int)((int64_t)G->N * k / nt);
        w[k].g1 = (int)((int64_t)G->N * (k + 1) / nt);
        pthread_create(&th[k], NULL, proj_worker, &w[k]);
    }
    for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
}

/* One view, a list of pixels: forward (and backward when gC != NULL).  For
 * the backward, screen-space grads are summed per Gaussian in pixel order
 * into sgrad [10][N] (zeroed by the caller). */
static int run_view(const og_gaussians *G, const og_camera *cam, const int64_t *pix, int64_t npix,
                    int brute, int nt, double *out, int32_t *ncontrib,
                    const double *gC, const double *gD, const double *gA, const double *gM, double *sgrad,
                    og_proj *P) {
    const int N = G->N;
    project_all(G, cam, P, nt);
    buckets_t B = {0};
    int *all = NULL;
    if (brute) {
        all = malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
        for (int g = 0; g < N; ++g) all[g] = g;
    } else {
        build_buckets(P, N, cam, &B);
    }
    if (nt > 256) nt = 256;
    if (nt > npix) nt = npix > 0 ? (int)npix : 1;
    pthread_t th[256];
    work_t *w = calloc((size_t)nt, sizeof(work_t));
    for (int k = 0; k < nt; ++k) {
        w[k].P = P; w[k].N = N; w[k].cam = cam; w[k].B = brute ? NULL : &B; w[k].all = all;
        w[k].pix = pix; w[k].p0 = npix * k / nt; w[k].p1 = npix * (k + 1) / nt;
        w[k].out = out; w[k].ncontrib = ncontrib;
        w[k].gC = gC; w[k].gD = gD; w[k].gA = gA; w[k].gM = gM;
        pthread_create(&th[k], NULL, worker, &w[k]);
    }
    for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
    if (gC) {
        /* deterministic: workers hold consecutive pixel ranges, summed in order */
        for (int k = 0; k < nt; ++k) {
            for (int64_t i = 0; i < w[k].sg_n; ++i) {
                const int g = w[k].sg_g[i];
                for (int c = 0; c < 10; ++c) sgrad[(size_t)c * N + g] += w[k].sg[10 * i + c];
            }
            free(w[k].sg);
            free(w[k].sg_g);
        }
    }
    free(w);
    free(all);
    free(B.start);
    free(B.items);
    return 0;
}

static int64_t *full_pixels(const og_camera *cam, int64_t *npix) {
    *npix = (int64_t)cam->H * cam->W;
    int64_t *p = malloc(sizeof(int64_t) * (size_t)(*npix > 0 ? *npix : 1));
    for (int64_t i = 0; i < *npix; ++i) p[i] = i;
    return p;
}

/* ------------------------------------------------------------------ */
/* Exported API (ctypes).                                               */
/* ------------------------------------------------------------------ */

/* Per-pixel forward over V views.  pix_off[V+1] and pix (concatenated
 * linear pixel indices y*W+x) select the pixels; pix == NULL renders every
 * pixel of every view in order.  out [P][OG_NOUT]: r, g, b, depth, opacity,
 * T_final, threshold margin, median depth, median margin, depth-order
 * margin.  ncontrib [P]. */
int og_render(const og_gaussians *G, int V, const og_camera *cams, const int64_t *pix_off,
              const int64_t *pix, int brute, int threads, double *out, int32_t *ncontrib) {
    const int nt = num_threads(threads);
    og_proj *P = malloc(sizeof(og_proj) * (size_t)(G->N > 0 ? G->N : 1));
    int64_t base = 0;
    for (int v = 0; v < V; ++v) {
        int64_t np;
        int64_t *own = NULL;
        const int64_t *pv;
        if (pix) {
            np = pix_off[v + 1] - pix_off[v];
            pv = pix + pix_off[v];
        } else {
            own = full_pixels(&cams[v], &np);
            pv = own;
        }
        run_view(G, &cams[v], pv, np, brute, nt, out + OG_NOUT * base, ncontrib + base, NULL, NULL, NULL, NULL, NULL, P);
        base += np;
        free(own);
    }
    free(P);
    return 0;
}

/* Forward + backward.  gC [P][3], gD [P], gA [P] are dL/d(colour, depth,
 * opacity) at the selected pixels, gM [P] dL/d(median depth) or NULL.  Gradients (zeroed here) come back for
 * means [3][N], log_scales [3][N], quats [4][N], opacity_logits [N],
 * sh [K*3][N], pose [V][6] (rho, phi) and, if screen != NULL, the summed
 * screen-space grads [V][10][N] (du, dv, dconic0..2, dopacity, drgb, dz). */
int og_render_backward(const og_gaussians *G, int V, const og_camera *cams, const int64_t *pix_off,
                       const int64_t *pix, int brute, int threads, const double *gC, const double *gD,
                       const double *gA, const double *gM, double *out, int32_t *ncontrib, double *gm, double *gls,
                       double *gq, double *gl, double *gsh, double *pose, double *screen) {
    const int N = G->N;
    const int K = (G->sh_degree + 1) * (G->sh_degree + 1);
    const int nt = num_threads(threads);
    memset(gm, 0, sizeof(double) * 3 * (size_t)N);
    memset(gls, 0, sizeof(double) * 3 * (size_t)N);
    memset(gq, 0, sizeof(double) * 4 * (size_t)N);
    memset(gl, 0, sizeof(double) * (size_t)N);
    memset(gsh, 0, sizeof(double) * 3 * (size_t)K * (size_t)N);
    memset(pose, 0, sizeof(double) * 6 * (size_t)V);
    og_proj *P = malloc(sizeof(og_proj) * (size_t)(N > 0 ? N : 1));
    double *sgrad = malloc(sizeof(double) * 10 * (size_t)(N > 0 ? N : 1));
    int64_t base = 0;
    for (int v = 0; v < V; ++v) {
        int64_t np;
        int64_t *own = NULL;
        const int64_t *pv;
        if (pix) {
            np = pix_off[v + 1] - pix_off[v];
            pv = pix + pix_off[v];
        } else {
            own = full_pixels(&cams[v], &np);
            pv = own;
        }
        memset(sgrad, 0, sizeof(double) * 10 * (size_t)N);
        run_view(G, &cams[v], pv, np, brute, nt, out + OG_NOUT * base, ncontrib + base, gC + 3 * base,
                 gD + base, gA + base, gM ? gM + base : NULL, sgrad, P);
        for (int g = 0; g < N; ++g) {
            if (!P[g].valid) continue;
            double s[10];
            int any = 0;
            for (int c = 0; c < 10; ++c) {
                s[c] = sgrad[(size_t)c * N + g];
                any |= s[c] != 0;
            }
            if (screen)
                for (int c = 0; c < 10; ++c) screen[((size_t)v * 10 + c) * N + g] = s[c];
            if (any) project_backward(G, &cams[v], g, &P[g], s, gm, gls, gq, gl, gsh, pose + 6 * v);
        }
        base += np;
        free(own);
    }
    free(sgrad);
    free(P);
    return 0;
}

/* Projection of every Gaussian into one view, for tests of the intermediate
 * quantities.  out [N][16]: valid, u, v, z, conic0..2, cov0..2, opacity,
 * r, g, b, clamp_x, clamp_y. */
int og_project(const og_gaussians *G, const og_camera *cam, double *out) {
    og_proj P;
    for (int g = 0; g < G->N; ++g) {
        project(G, cam, g, &P);
        double *o = out + 16 * (size_t)g;
        o[0] = P.valid; o[1] = P.u; o[2] = P.v; o[3] = P.z;
        o[4] = P.conic[0]; o[5] = P.conic[1]; o[6] = P.conic[2];
        o[7] = P.cov[0]; o[8] = P.cov[1]; o[9] = P.cov[2];
        o[10] = P.opacity; o[11] = P.rgb[0]; o[12] = P.rgb[1]; o[13] = P.rgb[2];
        o[14] = P.clamp_x; o[15] = P.clamp_y;
    }
    return 0;
}

int og_sh_basis(int degree, const double *dir, double *Y) {
    sh_basis(degree, dir, Y, NULL);
    return 0;
}

int og_quat_to_rot(const double *q, double *R9) {
    const double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const double qu[4] = {q[0] / n, q[1] / n, q[2] / n, q[3] / n};
    double R[3][3];
    quat_to_rot(qu, R);
    memcpy(R9, R, sizeof R);
    return 0;
}
