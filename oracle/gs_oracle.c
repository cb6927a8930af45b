/*
 * FP64 CPU oracle of the online 3DGS optimisation step -- TEST INFRASTRUCTURE.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load this library.  It shares no code with the CUDA path.  It is the
 * plain, slow definition of what the step computes, written out in the order
 * the method states it; every function names the passage it follows.
 *
 * The paper (Sec. 3.2.3) refines "the same parameters as in prior 3DGS work"
 * by differentiable rendering, and states no formula itself.  The maths here
 * is the standard EWA-splatting definition of the cited 3DGS method with the
 * constants fixed for this build (alpha clamp 0.99, 1/255 cut-off, T < 1e-4
 * termination, L1 + D-SSIM with an 11x11 sigma=1.5 window, Adam).  Readings
 * where the paper is silent are marked READING.
 *
 * Layouts (oracle side; the Python wrapper converts, it does no arithmetic):
 *   rows   [n][60]  : mean xyz, opacity logit, log-scale xyz, pad,
 *                     quaternion wxyz, 48 SH coefficients (3*k + channel)
 *   cams   [V][20]  : R (row-major world->camera), t, fx, fy, cx, cy,
 *                     width, height, near, unused
 *   proj   [V][n][16]: u, v, depth, opacity, A, B, C, radius, r, g, b,
 *                     clamp mask, x0, y0, x1, y1   (all zero when culled)
 *   grad2d [V][n][9] : dL/du, dL/dv, dL/dA, dL/dB, dL/dC, dL/dopacity,
 *                     dL/dr, dL/dg, dL/db
 *   images : views concatenated, each planar [3][H][W]
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CAM_STRIDE 20
#define PROJ_STRIDE 16
#define G2D_STRIDE 9
#define ROW 60

/* READING: constants fixed for this build from the cited method. */
static const double ALPHA_MAX = 0.99;
static const double ALPHA_MIN = 1.0 / 255.0;
static const double T_MIN = 1e-4;
static const double DILATION = 0.3;
static const double GUARD = 1.3;

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* ------------------------------------------------------------------------
 * Real spherical harmonics, degree <= 3, order l = 0..3, m = -l..l.
 * Sec. 3.2.2 / 3.4.1: appearance is stored as SH coefficients.
 * Convention: the real form of the complex harmonics with the
 * Condon-Shortley phase kept (sqrt(2) Re Y_l^m for m > 0, sqrt(2) Im Y_l^|m|
 * for m < 0), which is the sign pattern of the cited 3DGS method.  Written as
 * polynomials of the unit direction (x, y, z); normalisations are the closed
 * forms sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the polynomial factor.
 * ---------------------------------------------------------------------- */
void or_sh_basis(const double* d, double* Y) {
    const double PI = 3.14159265358979323846;
    double x = d[0], y = d[1], z = d[2];
    double xx = x * x, yy = y * y, zz = z * z;
    double k0 = sqrt(1.0 / (4.0 * PI));
    double k1 = sqrt(3.0 / (4.0 * PI));
    double k2a = sqrt(15.0 / (4.0 * PI)), k2b = sqrt(5.0 / (16.0 * PI)), k2c = sqrt(15.0 / (16.0 * PI));
    double k3a = sqrt(35.0 / (32.0 * PI)), k3b = sqrt(105.0 / (4.0 * PI)), k3c = sqrt(21.0 / (32.0 * PI));
    double k3d = sqrt(7.0 / (16.0 * PI)), k3e = sqrt(105.0 / (16.0 * PI));
    Y[0] = k0;
    Y[1] = -k1 * y;
    Y[2] = k1 * z;
    Y[3] = -k1 * x;
    Y[4] = k2a * x * y;
    Y[5] = -k2a * y * z;
    Y[6] = k2b * (2.0 * zz - xx - yy);
    Y[7] = -k2a * x * z;
    Y[8] = k2c * (xx - yy);
    Y[9] = -k3a * y * (3.0 * xx - yy);
    Y[10] = k3b * x * y * z;
    Y[11] = -k3c * y * (4.0 * zz - xx - yy);
    Y[12] = k3d * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[13] = -k3c * x * (4.0 * zz - xx - yy);
    Y[14] = k3e * z * (xx - yy);
    Y[15] = -k3a * x * (xx - 3.0 * yy);
}

/* Partial derivatives of the polynomials above w.r.t. (x, y, z): dY[k*3+i]. */
void or_sh_basis_grad(const double* d, double* dY) {
    const double PI = 3.14159265358979323846;
    double x = d[0], y = d[1], z = d[2];
    double xx = x * x, yy = y * y, zz = z * z;
    double k1 = sqrt(3.0 / (4.0 * PI));
    double k2a = sqrt(15.0 / (4.0 * PI)), k2b = sqrt(5.0 / (16.0 * PI)), k2c = sqrt(15.0 / (16.0 * PI));
    double k3a = sqrt(35.0 / (32.0 * PI)), k3b = sqrt(105.0 / (4.0 * PI)), k3c = sqrt(21.0 / (32.0 * PI));
    double k3d = sqrt(7.0 / (16.0 * PI)), k3e = sqrt(105.0 / (16.0 * PI));
    memset(dY, 0, sizeof(double) * 48);
#define SETG(k, gx, gy, gz) do { dY[(k)*3+0] = (gx); dY[(k)*3+1] = (gy); dY[(k)*3+2] = (gz); } while (0)
    SETG(1, 0.0, -k1, 0.0);
    SETG(2, 0.0, 0.0, k1);
    SETG(3, -k1, 0.0, 0.0);
    SETG(4, k2a * y, k2a * x, 0.0);
    SETG(5, 0.0, -k2a * z, -k2a * y);
    SETG(6, -2.0 * k2b * x, -2.0 * k2b * y, 4.0 * k2b * z);
    SETG(7, -k2a * z, 0.0, -k2a * x);
    SETG(8, 2.0 * k2c * x, -2.0 * k2c * y, 0.0);
    SETG(9, -k3a * 6.0 * x * y, -k3a * (3.0 * xx - 3.0 * yy), 0.0);
    SETG(10, k3b * y * z, k3b * x * z, k3b * x * y);
    SETG(11, -k3c * y * (-2.0 * x), -k3c * (4.0 * zz - xx - 3.0 * yy), -k3c * y * 8.0 * z);
    SETG(12, k3d * z * (-6.0 * x), k3d * z * (-6.0 * y), k3d * (6.0 * zz - 3.0 * xx - 3.0 * yy));
    SETG(13, -k3c * (4.0 * zz - 3.0 * xx - yy), -k3c * x * (-2.0 * y), -k3c * x * 8.0 * z);
    SETG(14, k3e * z * 2.0 * x, k3e * z * (-2.0 * y), k3e * (xx - yy));
    SETG(15, -k3a * (3.0 * xx - 3.0 * yy), -k3a * x * (-6.0 * y), 0.0);
#undef SETG
}

/* Unit quaternion (w, x, y, z) -> rotation matrix, row-major. */
static void quat_to_rot(const double* q, double* R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

static int tiles_along(int extent, int tile) { return (extent + tile - 1) / tile; }

/* Tile rectangle [x0, x1) x [y0, y1) of the screen-space square of half-side r
 * around (u, v), clamped to the tile grid.  READING of the cited method's
 * binning: the Gaussian is evaluated at every pixel of every tile it touches. */
void or_rect(double u, double v, double r, int W, int H, int tile, int32_t* rect) {
    int TX = tiles_along(W, tile), TY = tiles_along(H, tile);
    rect[0] = (int32_t)clampd(floor((u - r) / tile), 0.0, (double)TX);
    rect[1] = (int32_t)clampd(floor((v - r) / tile), 0.0, (double)TY);
    rect[2] = (int32_t)clampd(floor((u + r + tile - 1) / tile), 0.0, (double)TX);
    rect[3] = (int32_t)clampd(floor((v + r + tile - 1) / tile), 0.0, (double)TY);
}

/* Tile rectangle of a splat.  READING (the cited method bins by the 3-sigma
 * square; the paper is silent): the square of half-side r, cut down on each
 * axis to the bounding box of the ellipse where the splat's alpha reaches
 * 1/255, q = d^T Sigma2^-1 d <= tau = 2 ln(255 o), whose half-widths are
 * sqrt(tau a) and sqrt(tau c) for the 2D covariance (a, b; b, c), widened by
 * 0.1 % + 0.01 px against rounding: the tiles holding a pixel centre within
 * that box, intersected with the square's tiles.  Every pixel that
 * compositing takes the splat at (inside the square, alpha >= 1/255) lies
 * inside this rectangle, so the rendered image is the square's; a splat whose
 * opacity is below 1/255 gets no tile. */
void or_splat_rect(double u, double v, double r, double a, double c, double o, int W, int H, int tile,
                   int32_t* rect) {
    int32_t sq[4];
    or_rect(u, v, r, W, H, tile, sq);
    double tau = 2.0 * log(255.0 * o);
    rect[0] = rect[1] = rect[2] = rect[3] = 0;
    if (!(tau >= 0.0)) return;
    double rx = sqrt(tau * a) * 1.001 + 0.01, ry = sqrt(tau * c) * 1.001 + 0.01;
    /* tiles of the pixel centres p + 0.5 within [u - rx, u + rx] (and likewise in y) */
    int32_t x0 = (int32_t)clampd(floor(ceil(u - rx - 0.5) / tile), 0.0, (double)W);
    int32_t x1 = (int32_t)clampd(floor((u + rx - 0.5) / tile) + 1.0, 0.0, (double)W);
    int32_t y0 = (int32_t)clampd(floor(ceil(v - ry - 0.5) / tile), 0.0, (double)H);
    int32_t y1 = (int32_t)clampd(floor((v + ry - 0.5) / tile) + 1.0, 0.0, (double)H);
    x0 = x0 > sq[0] ? x0 : sq[0]; x1 = x1 < sq[2] ? x1 : sq[2];
    y0 = y0 > sq[1] ? y0 : sq[1]; y1 = y1 < sq[3] ? y1 : sq[3];
    if (x1 <= x0 || y1 <= y0) return;
    rect[0] = x0; rect[1] = y0; rect[2] = x1; rect[3] = y1;
}

/* ------------------------------------------------------------------------
 * Projection + SH colour (Sec. 3.2.3: the 3DGS parameters rendered by
 * differentiable splatting; Sec. 3.2.2: SH appearance).
 * ---------------------------------------------------------------------- */
typedef struct {
    double t[3];      /* camera-space mean */
    double xt, yt;    /* guard-band clamped t_x, t_y used in J */
    int clx, cly;     /* -1 / 0 / +1: which side the guard band clamped */
    double limx, limy;
    double J[6];      /* 2x3 */
    double M[6];      /* J W, 2x3 */
    double a, b, c, det;
    double dir[3], len;
    double dir_sh[3];  /* view direction in the object frame */
    double Y[16];
} view_geom;

/* ------------------------------------------------------------------------
 * Scene dynamics (Sec. 3.4).  Rigid objects (Sec. 3.4.2): every Gaussian
 * belongs to one object (group); its mean and rotation are stored in the
 * object's frame and the engine's current object pose (rotation R_g,
 * translation t_g) is applied before each optimisation step:
 *   mu_world = R_g mu + t_g,   Sigma_world = R_g Sigma R_g^T.
 * Relighting (Sec. 3.4.1), READING: the diffuse (DC) SH coefficient is scaled
 * by a Lambertian factor of the current directional light,
 *   L = ambient + diffuse * max(0, (R_g n) . l),
 * with n the Gaussian's object-frame unit normal and l the unit vector
 * towards the light.  The poses and the light are inputs, not parameters.
 * ---------------------------------------------------------------------- */
typedef struct {
    const int32_t* group;   /* [n] or NULL (static scene) */
    const double* poses;    /* [G][8]: quaternion wxyz, translation xyz, 0 */
    const double* normals;  /* [n][3] or NULL (no relighting) */
    double light[3];
    double ambient, diffuse;
    const double* sh_light; /* [56] SH lighting (see relit_colour) or NULL */
    const uint8_t* vis;     /* [n] light visibility 0..255, or NULL (all lit) */
} dyn_t;

static void quat_to_rot(const double* q, double* R);

/* World-frame mean / covariance and DC factor of Gaussian g under `dyn`;
 * Rg receives the object rotation (identity for a static scene). */
static void apply_dynamics(const dyn_t* dyn, int64_t g, double* mu, double* Sig, double* Rg, double* L) {
    for (int i = 0; i < 9; ++i) Rg[i] = (i % 4 == 0) ? 1.0 : 0.0;
    *L = 1.0;
    if (!dyn || !dyn->group) return;
    const double* pose = dyn->poses + (int64_t)dyn->group[g] * 8;
    double qn = sqrt(pose[0] * pose[0] + pose[1] * pose[1] + pose[2] * pose[2] + pose[3] * pose[3]);
    double q[4] = {pose[0] / qn, pose[1] / qn, pose[2] / qn, pose[3] / qn};
    quat_to_rot(q, Rg);
    double m[3], S[9];
    for (int i = 0; i < 3; ++i) m[i] = Rg[i * 3] * mu[0] + Rg[i * 3 + 1] * mu[1] + Rg[i * 3 + 2] * mu[2] + pose[4 + i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += Rg[i * 3 + k] * Sig[k * 3 + l] * Rg[j * 3 + l];
            S[i * 3 + j] = acc;
        }
    memcpy(mu, m, sizeof(m));
    memcpy(Sig, S, sizeof(S));
    if (dyn->normals) {
        const double* nl = dyn->normals + g * 3;
        double nd = 0.0;
        for (int i = 0; i < 3; ++i)
            nd += (Rg[i * 3] * nl[0] + Rg[i * 3 + 1] * nl[1] + Rg[i * 3 + 2] * nl[2]) * dyn->light[i];
        *L = dyn->ambient + dyn->diffuse * fmax(0.0, nd);
    }
}

static void gauss_common(const double* p, double* mu, double* s, double* qhat, double* qnorm,
                         double* R, double* Sig, double* opac) {
    mu[0] = p[0]; mu[1] = p[1]; mu[2] = p[2];
    *opac = 1.0 / (1.0 + exp(-p[3]));
    for (int i = 0; i < 3; ++i) s[i] = exp(p[4 + i]);
    double qn = sqrt(p[8] * p[8] + p[9] * p[9] + p[10] * p[10] + p[11] * p[11]);
    *qnorm = qn;
    for (int i = 0; i < 4; ++i) qhat[i] = p[8 + i] / qn;
    quat_to_rot(qhat, R);
    /* Sigma = R diag(s^2) R^T */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[i * 3 + k] * s[k] * s[k] * R[j * 3 + k];
            Sig[i * 3 + j] = acc;
        }
}

/* Returns 1 if the Gaussian survives the near-plane and determinant tests.
 * Rg (object rotation, NULL = identity): SH colour is evaluated at the view
 * direction in the object's frame, Rg^T dir, so that an object's
 * view-dependent appearance turns with it (READING, Sec. 3.4.2). */
static int view_geometry(const double* mu, const double* Sig, const double* cam, const double* Rg,
                         view_geom* G) {
    const double* W = cam;
    const double* tc = cam + 9;
    double fx = cam[12], fy = cam[13];
    double Wimg = cam[16], Himg = cam[17], near = cam[18];
    for (int i = 0; i < 3; ++i) G->t[i] = W[i * 3] * mu[0] + W[i * 3 + 1] * mu[1] + W[i * 3 + 2] * mu[2] + tc[i];
    double tz = G->t[2];
    if (tz <= near) return 0;
    G->limx = GUARD * (Wimg / (2.0 * fx));
    G->limy = GUARD * (Himg / (2.0 * fy));
    double rx = G->t[0] / tz, ry = G->t[1] / tz;
    G->clx = rx < -G->limx ? -1 : (rx > G->limx ? 1 : 0);
    G->cly = ry < -G->limy ? -1 : (ry > G->limy ? 1 : 0);
    G->xt = clampd(rx, -G->limx, G->limx) * tz;
    G->yt = clampd(ry, -G->limy, G->limy) * tz;
    G->J[0] = fx / tz; G->J[1] = 0.0; G->J[2] = -fx * G->xt / (tz * tz);
    G->J[3] = 0.0; G->J[4] = fy / tz; G->J[5] = -fy * G->yt / (tz * tz);
    for (int k = 0; k < 2; ++k)
        for (int i = 0; i < 3; ++i) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += G->J[k * 3 + l] * W[l * 3 + i];
            G->M[k * 3 + i] = acc;
        }
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            a += G->M[i] * Sig[i * 3 + j] * G->M[j];
            b += G->M[i] * Sig[i * 3 + j] * G->M[3 + j];
            c += G->M[3 + i] * Sig[i * 3 + j] * G->M[3 + j];
        }
    G->a = a + DILATION;
    G->b = b;
    G->c = c + DILATION;
    G->det = G->a * G->c - G->b * G->b;
    if (G->det <= 0.0) return 0;
    /* view direction from the camera centre -W^T t */
    double cp[3];
    for (int i = 0; i < 3; ++i) cp[i] = -(W[i] * tc[0] + W[3 + i] * tc[1] + W[6 + i] * tc[2]);
    double dv[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
    G->len = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    for (int i = 0; i < 3; ++i) G->dir[i] = dv[i] / G->len;
    double dl[3];
    for (int i = 0; i < 3; ++i)
        dl[i] = Rg ? Rg[i] * G->dir[0] + Rg[3 + i] * G->dir[1] + Rg[6 + i] * G->dir[2] : G->dir[i];
    memcpy(G->dir_sh, dl, sizeof(dl));
    or_sh_basis(dl, G->Y);
    return 1;
}

/* ------------------------------------------------------------------------
 * SH relighting (Sec. 3.4.1).  The Gaussian's SH coefficients are read as its
 * diffuse radiance transfer T_c(w) = sum_k c_{k,c} Y_k(w) (object frame), and
 * the lighting is given as SH coefficients too.  READING: the relit colour is
 * the integral over the sphere of the transfer times the lighting that
 * reaches the object, expressed in the object's frame:
 *   rgb_c = max(0, int T_c(w) [Lenv_c(R_g w) + v E_c delta(R_g w, l)] dw + 0.5)
 * with Lenv_c(w) = sum_{k<16} e_{k,c} Y_k(w) the world-frame environment
 * lighting, l the unit vector towards the directional light of radiance E_c,
 * and v = vis / 255 the Gaussian's light visibility, which attenuates the
 * direct light only.  The delta term integrates to v E_c T_c(R_g^T l).  The
 * environment term is integrated exactly by a product rule (4-point
 * Gauss-Legendre in cos(theta) times 8 equally spaced azimuths is exact for
 * the band-limited integrand of degree <= 6).  The +0.5 is the colour offset
 * of the SH parameterisation, kept as in the view-dependent colour, so a unit
 * light along the view direction with no environment gives that colour back.
 * Lighting layout: e[16][3], then l (x, y, z, 0), then E (r, g, b, 0).
 * ---------------------------------------------------------------------- */
#define SPHERE_NQ 32
static void sphere_rule(double dirs[SPHERE_NQ][3], double w[SPHERE_NQ]) {
    const double PI = 3.14159265358979323846;
    /* Gauss-Legendre nodes and weights of order 4, closed forms */
    const double a = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0));
    const double b = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
    const double wa = (18.0 + sqrt(30.0)) / 36.0, wb = (18.0 - sqrt(30.0)) / 36.0;
    const double z[4] = {-b, -a, a, b}, wz[4] = {wb, wa, wa, wb};
    int q = 0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j, ++q) {
            double phi = 2.0 * PI * j / 8.0, rho = sqrt(1.0 - z[i] * z[i]);
            dirs[q][0] = rho * cos(phi);
            dirs[q][1] = rho * sin(phi);
            dirs[q][2] = z[i];
            w[q] = wz[i] * 2.0 * PI / 8.0;
        }
}

static double vis_of(const dyn_t* dyn, int64_t g) { return dyn->vis ? dyn->vis[g] / 255.0 : 1.0; }

/* raw[c] = int T_c(w) L_obj,c(w) dw (without the offset and the clamp) */
static void relit_raw(const double* p, int nb, const double* Rg, const double* L, double v, double* raw) {
    double dirs[SPHERE_NQ][3], wq[SPHERE_NQ];
    sphere_rule(dirs, wq);
    raw[0] = raw[1] = raw[2] = 0.0;
    for (int q = 0; q < SPHERE_NQ; ++q) {
        double ww[3], Yo[16], Yw[16];
        for (int i = 0; i < 3; ++i) ww[i] = Rg[i * 3] * dirs[q][0] + Rg[i * 3 + 1] * dirs[q][1] + Rg[i * 3 + 2] * dirs[q][2];
        or_sh_basis(dirs[q], Yo);
        or_sh_basis(ww, Yw);
        for (int ch = 0; ch < 3; ++ch) {
            double T = 0.0, Le = 0.0;
            for (int k = 0; k < nb; ++k) T += p[12 + 3 * k + ch] * Yo[k];
            for (int k = 0; k < 16; ++k) Le += L[3 * k + ch] * Yw[k];
            raw[ch] += wq[q] * T * Le;
        }
    }
    double lo[3], Yl[16];
    for (int i = 0; i < 3; ++i) lo[i] = Rg[i] * L[48] + Rg[3 + i] * L[49] + Rg[6 + i] * L[50];
    or_sh_basis(lo, Yl);
    for (int ch = 0; ch < 3; ++ch) {
        double T = 0.0;
        for (int k = 0; k < nb; ++k) T += p[12 + 3 * k + ch] * Yl[k];
        raw[ch] += v * L[52 + ch] * T;
    }
}

/* dp[12 + 3k + c] += gc[c] * d raw_c / d c_{k,c} for the channels with gc != 0 */
static void relit_grad(int nb, const double* Rg, const double* L, double v, const double* gc, double* dp) {
    double dirs[SPHERE_NQ][3], wq[SPHERE_NQ];
    sphere_rule(dirs, wq);
    for (int q = 0; q < SPHERE_NQ; ++q) {
        double ww[3], Yo[16], Yw[16];
        for (int i = 0; i < 3; ++i) ww[i] = Rg[i * 3] * dirs[q][0] + Rg[i * 3 + 1] * dirs[q][1] + Rg[i * 3 + 2] * dirs[q][2];
        or_sh_basis(dirs[q], Yo);
        or_sh_basis(ww, Yw);
        for (int ch = 0; ch < 3; ++ch) {
            if (gc[ch] == 0.0) continue;
            double Le = 0.0;
            for (int k = 0; k < 16; ++k) Le += L[3 * k + ch] * Yw[k];
            for (int k = 0; k < nb; ++k) dp[12 + 3 * k + ch] += gc[ch] * wq[q] * Yo[k] * Le;
        }
    }
    double lo[3], Yl[16];
    for (int i = 0; i < 3; ++i) lo[i] = Rg[i] * L[48] + Rg[3 + i] * L[49] + Rg[6 + i] * L[50];
    or_sh_basis(lo, Yl);
    for (int ch = 0; ch < 3; ++ch)
        for (int k = 0; k < nb; ++k) dp[12 + 3 * k + ch] += gc[ch] * v * L[52 + ch] * Yl[k];
}

static void project_impl(int64_t n, int sh_degree, const double* rows, int V, const double* cams, int tile,
                         const dyn_t* dyn, double* out) {
    int nb = (sh_degree + 1) * (sh_degree + 1);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t g = 0; g < n; ++g) {
        const double* p = rows + g * ROW;
        double mu[3], s[3], q[4], qn, R[9], Sig[9], opac, Rg[9], Ld;
        gauss_common(p, mu, s, q, &qn, R, Sig, &opac);
        apply_dynamics(dyn, g, mu, Sig, Rg, &Ld);
        for (int v = 0; v < V; ++v) {
            const double* cam = cams + (int64_t)v * CAM_STRIDE;
            double* o = out + ((int64_t)v * n + g) * PROJ_STRIDE;
            memset(o, 0, sizeof(double) * PROJ_STRIDE);
            view_geom G;
            if (!view_geometry(mu, Sig, cam, Rg, &G)) continue;
            double mid = 0.5 * (G.a + G.c);
            double lam = mid + sqrt(fmax(0.1, mid * mid - G.det));
            double r = ceil(3.0 * sqrt(lam));
            double u = cam[12] * G.t[0] / G.t[2] + cam[14];
            double vv = cam[13] * G.t[1] / G.t[2] + cam[15];
            int32_t rect[4];
            or_splat_rect(u, vv, r, G.a, G.c, opac, (int)cam[16], (int)cam[17], tile, rect);
            if ((rect[2] - rect[0]) * (rect[3] - rect[1]) == 0) continue;
            double rgb[3], raw[3];
            int mask = 0;
            if (dyn && dyn->sh_light) relit_raw(p, nb, Rg, dyn->sh_light, vis_of(dyn, g), raw);
            for (int ch = 0; ch < 3; ++ch) {
                double acc = 0.0;
                if (dyn && dyn->sh_light)
                    acc = raw[ch];
                else
                    for (int k = 0; k < nb; ++k) acc += p[12 + 3 * k + ch] * G.Y[k] * (k == 0 ? Ld : 1.0);
                acc += 0.5;
                if (acc < 0.0) { acc = 0.0; mask |= 1 << ch; }
                rgb[ch] = acc;
            }
            o[0] = u; o[1] = vv; o[2] = G.t[2]; o[3] = opac;
            o[4] = G.c / G.det; o[5] = -G.b / G.det; o[6] = G.a / G.det; o[7] = r;
            o[8] = rgb[0]; o[9] = rgb[1]; o[10] = rgb[2]; o[11] = (double)mask;
            o[12] = rect[0]; o[13] = rect[1]; o[14] = rect[2]; o[15] = rect[3];
        }
    }
}

void or_project(int64_t n, int sh_degree, const double* rows, int V, const double* cams, int tile, double* out) {
    project_impl(n, sh_degree, rows, V, cams, tile, NULL, out);
}

/* or_project with rigid-object dynamics and relighting (see apply_dynamics);
 * group: int32 [n]; poses [G][8]; normals [n][3] or NULL; light[3]. */
void or_project_dyn(int64_t n, int sh_degree, const double* rows, int V, const double* cams, int tile,
                    const int32_t* group, const double* poses, const double* normals, const double* light,
                    double ambient, double diffuse, double* out) {
    dyn_t d = {group, poses, normals, {light[0], light[1], light[2]}, ambient, diffuse, NULL, NULL};
    project_impl(n, sh_degree, rows, V, cams, tile, &d, out);
}

/* or_project with SH relighting; group / poses may be NULL (static scene),
 * vis NULL means every Gaussian is lit. */
void or_project_lit(int64_t n, int sh_degree, const double* rows, int V, const double* cams, int tile,
                    const int32_t* group, const double* poses, const double* sh_light, const uint8_t* vis,
                    double* out) {
    dyn_t d = {group, poses, NULL, {0, 0, 0}, 0.0, 0.0, sh_light, vis};
    project_impl(n, sh_degree, rows, V, cams, tile, &d, out);
}

/* ------------------------------------------------------------------------
 * Binning and sort.  Every (view, Gaussian, touched tile) becomes one entry;
 * entries are ordered lexicographically by (view, tile, depth as float32 bits,
 * Gaussian index).  READING: depth = camera-space z; the sort key uses the
 * float32 value of the depth so that float32 and float64 producers agree.
 * Tile index: per-view offset + ty * TX + tx (views in order).
 * ---------------------------------------------------------------------- */
typedef struct { uint64_t key; uint32_t g; } entry;

static int cmp_entry(const void* A, const void* B) {
    const entry* a = (const entry*)A;
    const entry* b = (const entry*)B;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->g < b->g ? -1 : (a->g > b->g ? 1 : 0);
}

int64_t or_bin_count(int V, int64_t n, const int32_t* rects) {
    int64_t K = 0;
    for (int64_t i = 0; i < (int64_t)V * n; ++i) {
        const int32_t* r = rects + i * 4;
        K += (int64_t)(r[2] - r[0]) * (r[3] - r[1]);
    }
    return K;
}

/* rects [V][n][4], depth [V][n] float32; writes keys (u64), vals (u32),
 * ranges [total_tiles][2]; returns the entry count. */
int64_t or_bin_sort(int V, int64_t n, const double* cams, int tile, const int32_t* rects,
                    const float* depth, uint64_t* keys, uint32_t* vals, uint32_t* ranges) {
    int64_t K = or_bin_count(V, n, rects);
    entry* E = (entry*)malloc(sizeof(entry) * (size_t)(K > 0 ? K : 1));
    int64_t toff = 0, k = 0;
    for (int v = 0; v < V; ++v) {
        const double* cam = cams + (int64_t)v * CAM_STRIDE;
        int TX = tiles_along((int)cam[16], tile), TY = tiles_along((int)cam[17], tile);
        for (int64_t g = 0; g < n; ++g) {
            const int32_t* r = rects + ((int64_t)v * n + g) * 4;
            uint32_t dbits;
            memcpy(&dbits, &depth[(int64_t)v * n + g], 4);
            for (int ty = r[1]; ty < r[3]; ++ty)
                for (int tx = r[0]; tx < r[2]; ++tx) {
                    E[k].key = ((uint64_t)(toff + (int64_t)ty * TX + tx) << 32) | dbits;
                    E[k].g = (uint32_t)g;
                    ++k;
                }
        }
        for (int64_t t = 0; t < (int64_t)TX * TY; ++t) { ranges[(toff + t) * 2] = 0; ranges[(toff + t) * 2 + 1] = 0; }
        toff += (int64_t)TX * TY;
    }
    qsort(E, (size_t)K, sizeof(entry), cmp_entry);
    for (int64_t i = 0; i < K; ++i) {
        keys[i] = E[i].key;
        vals[i] = E[i].g;
        uint32_t t = (uint32_t)(E[i].key >> 32);
        if (i == 0 || (uint32_t)(E[i - 1].key >> 32) != t) ranges[(int64_t)t * 2] = (uint32_t)i;
        if (i == K - 1 || (uint32_t)(E[i + 1].key >> 32) != t) ranges[(int64_t)t * 2 + 1] = (uint32_t)(i + 1);
    }
    free(E);
    return K;
}

/* The [start, end) range of every tile in the order above, without forming
 * the entries: a tile's run length is the number of (view, Gaussian) whose
 * rectangle holds it, and runs follow each other in tile order (empty tiles
 * (0, 0)), exactly as or_bin_sort writes them.  Returns the entry count. */
int64_t or_bin_ranges(int V, int64_t n, const double* cams, int tile, const int32_t* rects, uint32_t* ranges) {
    int64_t T = 0;
    for (int v = 0; v < V; ++v) {
        const double* cam = cams + (int64_t)v * CAM_STRIDE;
        T += (int64_t)tiles_along((int)cam[16], tile) * tiles_along((int)cam[17], tile);
    }
    int64_t* count = (int64_t*)calloc((size_t)(T > 0 ? T : 1), sizeof(int64_t));
    int64_t toff = 0;
    for (int v = 0; v < V; ++v) {
        const double* cam = cams + (int64_t)v * CAM_STRIDE;
        int TX = tiles_along((int)cam[16], tile), TY = tiles_along((int)cam[17], tile);
        for (int64_t g = 0; g < n; ++g) {
            const int32_t* r = rects + ((int64_t)v * n + g) * 4;
            for (int ty = r[1]; ty < r[3]; ++ty)
                for (int tx = r[0]; tx < r[2]; ++tx) count[toff + (int64_t)ty * TX + tx] += 1;
        }
        toff += (int64_t)TX * TY;
    }
    int64_t run = 0;
    for (int64_t t = 0; t < T; ++t) {
        ranges[2 * t] = count[t] ? (uint32_t)run : 0u;
        ranges[2 * t + 1] = count[t] ? (uint32_t)(run + count[t]) : 0u;
        run += count[t];
    }
    free(count);
    return run;
}

/* The sorted entries of some tiles only: for each global tile index req[i],
 * the Gaussians whose rectangle holds that tile, ordered as in or_bin_sort
 * (float32 depth bits, then Gaussian index), appended to vals; tile i's run
 * is vals[start[i], start[i + 1]).  With vals == NULL only start is filled.
 * Returns the total. */
typedef struct { uint32_t d; uint32_t g; } tile_entry;

static int cmp_tile_entry(const void* A, const void* B) {
    const tile_entry* a = (const tile_entry*)A;
    const tile_entry* b = (const tile_entry*)B;
    if (a->d != b->d) return a->d < b->d ? -1 : 1;
    return a->g < b->g ? -1 : (a->g > b->g ? 1 : 0);
}

/* view, column and row of global tile t (-1 view when t is out of range) */
static int tile_place(int V, const double* cams, int tile, int64_t t, int* tx, int* ty) {
    int64_t toff = 0;
    for (int v = 0; v < V; ++v) {
        const double* cam = cams + (int64_t)v * CAM_STRIDE;
        int TX = tiles_along((int)cam[16], tile), TY = tiles_along((int)cam[17], tile);
        if (t < toff + (int64_t)TX * TY) {
            *tx = (int)((t - toff) % TX);
            *ty = (int)((t - toff) / TX);
            return v;
        }
        toff += (int64_t)TX * TY;
    }
    return -1;
}

int64_t or_bin_tiles(int V, int64_t n, const double* cams, int tile, const int32_t* rects, const float* depth,
                     int64_t n_req, const int64_t* req, uint32_t* vals, int64_t* start) {
    int64_t* cnt = (int64_t*)calloc((size_t)(n_req > 0 ? n_req : 1), sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < n_req; ++i) {
        int tx = 0, ty = 0;
        int v = tile_place(V, cams, tile, req[i], &tx, &ty);
        if (v < 0) continue;
        int64_t c = 0;
        for (int64_t g = 0; g < n; ++g) {
            const int32_t* r = rects + ((int64_t)v * n + g) * 4;
            if (tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]) ++c;
        }
        cnt[i] = c;
    }
    start[0] = 0;
    for (int64_t i = 0; i < n_req; ++i) start[i + 1] = start[i] + cnt[i];
    if (vals) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t i = 0; i < n_req; ++i) {
            int tx = 0, ty = 0;
            int v = tile_place(V, cams, tile, req[i], &tx, &ty);
            if (v < 0 || cnt[i] == 0) continue;
            tile_entry* E = (tile_entry*)malloc(sizeof(tile_entry) * (size_t)cnt[i]);
            int64_t k = 0;
            for (int64_t g = 0; g < n; ++g) {
                const int32_t* r = rects + ((int64_t)v * n + g) * 4;
                if (tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]) {
                    memcpy(&E[k].d, &depth[(int64_t)v * n + g], 4);
                    E[k].g = (uint32_t)g;
                    ++k;
                }
            }
            qsort(E, (size_t)k, sizeof(tile_entry), cmp_tile_entry);
            for (int64_t j = 0; j < k; ++j) vals[start[i] + j] = E[j].g;
            free(E);
        }
    }
    free(cnt);
    return start[n_req];
}

/* ------------------------------------------------------------------------
 * Front-to-back alpha compositing (Sec. 3.2.3 differentiable rendering, as in
 * the cited method).  Per pixel, in sorted order, from T = 1:
 *   d = (u, v) - pixel centre, P = -(A dx^2 + C dy^2)/2 - B dx dy,
 *   skip if P > 0; alpha = min(0.99, o e^P); skip if alpha < 1/255;
 *   T' = T (1 - alpha); READING: if T' < 1e-4 stop without adding it;
 *   else C += rgb alpha T, T = T'.  Output C + T bg.  n_contrib = position
 *   (1-based, within the tile's list) of the last fragment added.
 * Pixel (x, y) is sampled at (x + 0.5, y + 0.5).
 * ---------------------------------------------------------------------- */
static int64_t view_tile_offset(const double* cams, int v, int tile) {
    int64_t off = 0;
    for (int w = 0; w < v; ++w) {
        const double* c = cams + (int64_t)w * CAM_STRIDE;
        off += (int64_t)tiles_along((int)c[16], tile) * tiles_along((int)c[17], tile);
    }
    return off;
}

static int64_t view_pixel_offset(const double* cams, int v) {
    int64_t off = 0;
    for (int w = 0; w < v; ++w) off += (int64_t)cams[w * CAM_STRIDE + 16] * (int64_t)cams[w * CAM_STRIDE + 17];
    return off;
}

void or_render(int V, int64_t n, const double* cams, int tile, const double* proj,
               const uint32_t* vals, const uint32_t* ranges, const double* bg,
               double* image, double* T_final, int32_t* n_contrib) {
    for (int v = 0; v < V; ++v) {
        const double* cam = cams + (int64_t)v * CAM_STRIDE;
        int W = (int)cam[16], H = (int)cam[17], TX = tiles_along(W, tile);
        int64_t toff = view_tile_offset(cams, v, tile), poff = view_pixel_offset(cams, v);
        double* img = image + 3 * poff;
#pragma omp parallel for schedule(dynamic, 4)
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                int64_t t = toff + (int64_t)(y / tile) * TX + x / tile;
                uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
                double px = x + 0.5, py = y + 0.5, T = 1.0, C[3] = {0, 0, 0};
                int32_t nc = 0;
                for (uint32_t j = s; j < e; ++j) {
                    const double* o = proj + ((int64_t)v * n + vals[j]) * PROJ_STRIDE;
                    double dx = o[0] - px, dy = o[1] - py;
                    double P = -0.5 * (o[4] * dx * dx + o[6] * dy * dy) - o[5] * dx * dy;
                    if (P > 0.0) continue;
                    double al = fmin(ALPHA_MAX, o[3] * exp(P));
                    if (al < ALPHA_MIN) continue;
                    double Tn = T * (1.0 - al);
                    if (Tn < T_MIN) break;
                    for (int ch = 0; ch < 3; ++ch) C[ch] += o[8 + ch] * al * T;
                    T = Tn;
                    nc = (int32_t)(j - s + 1);
                }
                int64_t pix = (int64_t)y * W + x;
                for (int ch = 0; ch < 3; ++ch) img[(int64_t)ch * W * H + pix] = C[ch] + T * bg[ch];
                T_final[poff + pix] = T;
                n_contrib[poff + pix] = nc;
            }
    }
}

/* Adjoint of or_render: per pixel, re-walk the list, keep each added
 * fragment's (alpha, T_j), then with S_j = sum_{k>j} c_k a_k T_k + T_N bg:
 *   dC/dc_j = a_j T_j,  dC/da_j = c_j T_j - S_j / (1 - a_j),
 * then a = o e^P (no gradient where clamped at 0.99) down to (u, v, A, B, C, o).
 * Discrete events (skips, termination, clamps) have zero derivative. */
void or_render_bwd(int V, int64_t n, const double* cams, int tile, const double* proj,
                   const uint32_t* vals, const uint32_t* ranges, const double* bg,
                   const double* dimage, double* grad2d) {
    memset(grad2d, 0, sizeof(double) * (size_t)V * (size_t)n * G2D_STRIDE);
    for (int v = 0; v < V; ++v) {
        const double* cam = cams + (int64_t)v * CAM_STRIDE;
        int W = (int)cam[16], H = (int)cam[17], TX = tiles_along(W, tile);
        int64_t toff = view_tile_offset(cams, v, tile), poff = view_pixel_offset(cams, v);
        const double* dimg = dimage + 3 * poff;
#pragma omp parallel
        {
            int cap = 1024;
            uint32_t* lj = (uint32_t*)malloc(sizeof(uint32_t) * cap);
            double* la = (double*)malloc(sizeof(double) * cap);
            double* lT = (double*)malloc(sizeof(double) * cap);
            double* lG = (double*)malloc(sizeof(double) * cap);
            int* lcl = (int*)malloc(sizeof(int) * cap);
#pragma omp for schedule(dynamic, 4)
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    int64_t t = toff + (int64_t)(y / tile) * TX + x / tile;
                    uint32_t s = ranges[2 * t], e = ranges[2 * t + 1];
                    double px = x + 0.5, py = y + 0.5, T = 1.0;
                    int m = 0;
                    for (uint32_t j = s; j < e; ++j) {
                        const double* o = proj + ((int64_t)v * n + vals[j]) * PROJ_STRIDE;
                        double dx = o[0] - px, dy = o[1] - py;
                        double P = -0.5 * (o[4] * dx * dx + o[6] * dy * dy) - o[5] * dx * dy;
                        if (P > 0.0) continue;
                        double Gv = exp(P);
                        double raw = o[3] * Gv;
                        double al = fmin(ALPHA_MAX, raw);
                        if (al < ALPHA_MIN) continue;
                        double Tn = T * (1.0 - al);
                        if (Tn < T_MIN) break;
                        if (m == cap) {
                            cap *= 2;
                            lj = (uint32_t*)realloc(lj, sizeof(uint32_t) * cap);
                            la = (double*)realloc(la, sizeof(double) * cap);
                            lT = (double*)realloc(lT, sizeof(double) * cap);
                            lG = (double*)realloc(lG, sizeof(double) * cap);
                            lcl = (int*)realloc(lcl, sizeof(int) * cap);
                        }
                        lj[m] = j; la[m] = al; lT[m] = T; lG[m] = Gv; lcl[m] = raw > ALPHA_MAX;
                        ++m;
                        T = Tn;
                    }
                    int64_t pix = (int64_t)y * W + x;
                    double dC[3];
                    for (int ch = 0; ch < 3; ++ch) dC[ch] = dimg[(int64_t)ch * W * H + pix];
                    double S[3] = {T * bg[0], T * bg[1], T * bg[2]};
                    for (int i = m - 1; i >= 0; --i) {
                        uint32_t g = vals[lj[i]];
                        const double* o = proj + ((int64_t)v * n + g) * PROJ_STRIDE;
                        double al = la[i], Tj = lT[i];
                        double dal = 0.0;
                        double* gg = grad2d + ((int64_t)v * n + g) * G2D_STRIDE;
                        for (int ch = 0; ch < 3; ++ch) {
                            double c = o[8 + ch];
                            dal += dC[ch] * (c * Tj - S[ch] / (1.0 - al));
#pragma omp atomic
                            gg[6 + ch] += dC[ch] * al * Tj;
                            S[ch] += c * al * Tj;
                        }
                        if (lcl[i]) continue;
                        double dx = o[0] - px, dy = o[1] - py;
                        double dP = dal * o[3] * lG[i];
                        double dO = dal * lG[i];
                        double du = dP * (-o[4] * dx - o[5] * dy);
                        double dv = dP * (-o[6] * dy - o[5] * dx);
#pragma omp atomic
                        gg[0] += du;
#pragma omp atomic
                        gg[1] += dv;
#pragma omp atomic
                        gg[2] += dP * (-0.5 * dx * dx);
#pragma omp atomic
                        gg[3] += dP * (-dx * dy);
#pragma omp atomic
                        gg[4] += dP * (-0.5 * dy * dy);
#pragma omp atomic
                        gg[5] += dO;
                    }
                }
            free(lj); free(la); free(lT); free(lG); free(lcl);
        }
    }
}

/* ------------------------------------------------------------------------
 * Adjoint of or_project: 2D gradients of every view -> parameter gradients
 * (mean, opacity logit, log-scale, quaternion, SH), summed over views.
 * ---------------------------------------------------------------------- */
static void project_bwd_impl(int64_t n, int sh_degree, const double* rows, int V, const double* cams,
                             int tile, const double* grad2d, const dyn_t* dyn, double* drows) {
    int nb = (sh_degree + 1) * (sh_degree + 1);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t g = 0; g < n; ++g) {
        const double* p = rows + g * ROW;
        double* dp = drows + g * ROW;
        memset(dp, 0, sizeof(double) * ROW);
        double mu[3], s[3], q[4], qn, R[9], Sig[9], opac, Rg[9], Ld;
        gauss_common(p, mu, s, q, &qn, R, Sig, &opac);
        apply_dynamics(dyn, g, mu, Sig, Rg, &Ld);  /* mu, Sig are world-frame from here on */
        double dmu[3] = {0, 0, 0}, dSig[9] = {0}, dlogit = 0.0;
        for (int v = 0; v < V; ++v) {
            const double* cam = cams + (int64_t)v * CAM_STRIDE;
            const double* W = cam;
            double fx = cam[12], fy = cam[13];
            view_geom G;
            if (!view_geometry(mu, Sig, cam, Rg, &G)) continue;
            /* the same culling as the forward pass */
            double mid = 0.5 * (G.a + G.c);
            double r = ceil(3.0 * sqrt(mid + sqrt(fmax(0.1, mid * mid - G.det))));
            double u = fx * G.t[0] / G.t[2] + cam[14], vv = fy * G.t[1] / G.t[2] + cam[15];
            int32_t rect[4];
            or_splat_rect(u, vv, r, G.a, G.c, opac, (int)cam[16], (int)cam[17], tile, rect);
            if ((rect[2] - rect[0]) * (rect[3] - rect[1]) == 0) continue;
            const double* gr = grad2d + ((int64_t)v * n + g) * G2D_STRIDE;
            double gu = gr[0], gv = gr[1], gA = gr[2], gB = gr[3], gC = gr[4], go = gr[5];
            /* opacity = sigmoid(logit) */
            dlogit += go * opac * (1.0 - opac);
            /* colour: rgb_c = sum_k sh[k][c] Y_k(dir) + 0.5, clamped at 0 */
            double ddl[3] = {0, 0, 0}, dY[48];  /* w.r.t. the object-frame direction */
            or_sh_basis_grad(G.dir_sh, dY);
            if (dyn && dyn->sh_light) {
                /* relit colour: no view dependence, linear in the coefficients */
                double raw[3], gcol[3];
                relit_raw(p, nb, Rg, dyn->sh_light, vis_of(dyn, g), raw);
                for (int ch = 0; ch < 3; ++ch) gcol[ch] = raw[ch] + 0.5 < 0.0 ? 0.0 : gr[6 + ch];
                relit_grad(nb, Rg, dyn->sh_light, vis_of(dyn, g), gcol, dp);
            }
            for (int ch = 0; ch < 3 && !(dyn && dyn->sh_light); ++ch) {
                double raw = 0.5;
                for (int k = 0; k < nb; ++k) raw += p[12 + 3 * k + ch] * G.Y[k] * (k == 0 ? Ld : 1.0);
                if (raw < 0.0) continue;
                double gc = gr[6 + ch];
                for (int k = 0; k < nb; ++k) {
                    dp[12 + 3 * k + ch] += gc * G.Y[k] * (k == 0 ? Ld : 1.0);
                    for (int i = 0; i < 3; ++i) ddl[i] += gc * p[12 + 3 * k + ch] * dY[k * 3 + i];
                }
            }
            /* dir_sh = Rg^T dir  ->  dL/ddir = Rg dL/ddir_sh */
            double ddir[3];
            for (int i = 0; i < 3; ++i) ddir[i] = Rg[i * 3] * ddl[0] + Rg[i * 3 + 1] * ddl[1] + Rg[i * 3 + 2] * ddl[2];
            double dd = G.dir[0] * ddir[0] + G.dir[1] * ddir[1] + G.dir[2] * ddir[2];
            for (int i = 0; i < 3; ++i) dmu[i] += (ddir[i] - G.dir[i] * dd) / G.len;
            /* conic (A, B, C) = (c, -b, a) / det */
            double a = G.a, b = G.b, c = G.c, det = G.det, d2 = det * det;
            double da = gA * (-c * c / d2) + gB * (b * c / d2) + gC * (1.0 / det - a * c / d2);
            double db = gA * (2.0 * b * c / d2) + gB * (-1.0 / det - 2.0 * b * b / d2) + gC * (2.0 * a * b / d2);
            double dc = gA * (1.0 / det - a * c / d2) + gB * (a * b / d2) + gC * (-a * a / d2);
            /* a = M0 Sig M0^T + 0.3, b = M0 Sig M1^T, c = M1 Sig M1^T + 0.3 */
            double SM0[3], SM1[3], dM[6];
            for (int i = 0; i < 3; ++i) {
                SM0[i] = Sig[i * 3] * G.M[0] + Sig[i * 3 + 1] * G.M[1] + Sig[i * 3 + 2] * G.M[2];
                SM1[i] = Sig[i * 3] * G.M[3] + Sig[i * 3 + 1] * G.M[4] + Sig[i * 3 + 2] * G.M[5];
            }
            for (int i = 0; i < 3; ++i) {
                dM[i] = 2.0 * da * SM0[i] + db * SM1[i];
                dM[3 + i] = 2.0 * dc * SM1[i] + db * SM0[i];
            }
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    dSig[i * 3 + j] += da * G.M[i] * G.M[j] + db * G.M[i] * G.M[3 + j] + dc * G.M[3 + i] * G.M[3 + j];
            /* M = J W */
            double dJ[6];
            for (int k = 0; k < 2; ++k)
                for (int l = 0; l < 3; ++l) {
                    double acc = 0.0;
                    for (int i = 0; i < 3; ++i) acc += dM[k * 3 + i] * W[l * 3 + i];
                    dJ[k * 3 + l] = acc;
                }
            double tx = G.t[0], ty = G.t[1], tz = G.t[2];
            double dt[3] = {0, 0, 0};
            dt[2] += dJ[0] * (-fx / (tz * tz)) + dJ[4] * (-fy / (tz * tz));
            dt[2] += dJ[2] * (2.0 * fx * G.xt / (tz * tz * tz)) + dJ[5] * (2.0 * fy * G.yt / (tz * tz * tz));
            double dxt = dJ[2] * (-fx / (tz * tz)), dyt = dJ[5] * (-fy / (tz * tz));
            if (G.clx == 0) dt[0] += dxt; else dt[2] += dxt * (G.clx * G.limx);
            if (G.cly == 0) dt[1] += dyt; else dt[2] += dyt * (G.cly * G.limy);
            /* u = fx tx / tz + cx, v = fy ty / tz + cy */
            dt[0] += gu * fx / tz;
            dt[1] += gv * fy / tz;
            dt[2] += -gu * fx * tx / (tz * tz) - gv * fy * ty / (tz * tz);
            /* t = W mu + t_cam */
            for (int i = 0; i < 3; ++i) dmu[i] += W[i] * dt[0] + W[3 + i] * dt[1] + W[6 + i] * dt[2];
        }
        /* back to the object frame: mu_w = Rg mu + t, Sigma_w = Rg Sigma Rg^T */
        {
            double m[3], D[9];
            for (int i = 0; i < 3; ++i) m[i] = Rg[i] * dmu[0] + Rg[3 + i] * dmu[1] + Rg[6 + i] * dmu[2];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; ++k)
                        for (int l = 0; l < 3; ++l) acc += Rg[k * 3 + i] * dSig[k * 3 + l] * Rg[l * 3 + j];
                    D[i * 3 + j] = acc;
                }
            memcpy(dmu, m, sizeof(m));
            memcpy(dSig, D, sizeof(D));
        }
        /* Sigma = R diag(s^2) R^T */
        double dR[9], ds[3];
        for (int aa = 0; aa < 3; ++aa)
            for (int bb = 0; bb < 3; ++bb) {
                double acc = 0.0;
                for (int j = 0; j < 3; ++j) acc += dSig[aa * 3 + j] * s[bb] * s[bb] * R[j * 3 + bb];
                for (int i = 0; i < 3; ++i) acc += dSig[i * 3 + aa] * R[i * 3 + bb] * s[bb] * s[bb];
                dR[aa * 3 + bb] = acc;
            }
        for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) acc += dSig[i * 3 + j] * R[i * 3 + k] * R[j * 3 + k];
            ds[k] = acc * 2.0 * s[k];
        }
        /* R(q) partials */
        double w = q[0], x = q[1], y = q[2], z = q[3];
        double dq[4];
        dq[0] = dR[1] * (-2 * z) + dR[2] * (2 * y) + dR[3] * (2 * z) + dR[5] * (-2 * x) + dR[6] * (-2 * y) + dR[7] * (2 * x);
        dq[1] = dR[1] * (2 * y) + dR[2] * (2 * z) + dR[3] * (2 * y) + dR[4] * (-4 * x) + dR[5] * (-2 * w) + dR[6] * (2 * z) + dR[7] * (2 * w) + dR[8] * (-4 * x);
        dq[2] = dR[0] * (-4 * y) + dR[1] * (2 * x) + dR[2] * (2 * w) + dR[3] * (2 * x) + dR[5] * (2 * z) + dR[6] * (-2 * w) + dR[7] * (2 * z) + dR[8] * (-4 * y);
        dq[3] = dR[0] * (-4 * z) + dR[1] * (-2 * w) + dR[2] * (2 * x) + dR[3] * (2 * w) + dR[4] * (-4 * z) + dR[5] * (2 * y) + dR[6] * (2 * x) + dR[7] * (2 * y);
        double qd = q[0] * dq[0] + q[1] * dq[1] + q[2] * dq[2] + q[3] * dq[3];
        for (int i = 0; i < 3; ++i) dp[i] = dmu[i];
        dp[3] = dlogit;
        for (int i = 0; i < 3; ++i) dp[4 + i] = ds[i] * s[i];
        for (int i = 0; i < 4; ++i) dp[8 + i] = (dq[i] - q[i] * qd) / qn;
    }
}

void or_project_bwd(int64_t n, int sh_degree, const double* rows, int V, const double* cams, int tile,
                    const double* grad2d, double* drows) {
    project_bwd_impl(n, sh_degree, rows, V, cams, tile, grad2d, NULL, drows);
}

void or_project_bwd_dyn(int64_t n, int sh_degree, const double* rows, int V, const double* cams, int tile,
                        const double* grad2d, const int32_t* group, const double* poses, const double* normals,
                        const double* light, double ambient, double diffuse, double* drows) {
    dyn_t d = {group, poses, normals, {light[0], light[1], light[2]}, ambient, diffuse, NULL, NULL};
    project_bwd_impl(n, sh_degree, rows, V, cams, tile, grad2d, &d, drows);
}

void or_project_bwd_lit(int64_t n, int sh_degree, const double* rows, int V, const double* cams, int tile,
                        const double* grad2d, const int32_t* group, const double* poses, const double* sh_light,
                        const uint8_t* vis, double* drows) {
    dyn_t d = {group, poses, NULL, {0, 0, 0}, 0.0, 0.0, sh_light, vis};
    project_bwd_impl(n, sh_degree, rows, V, cams, tile, grad2d, &d, drows);
}

/* ------------------------------------------------------------------------
 * Light visibility (Sec. 3.4.1): an orthographic camera attached to the
 * directional light renders a light-space depth map, and every Gaussian
 * centre is projected into it and tested against the stored depth.
 * READING (the paper's map is the engine's shadow pass over its meshes, which
 * this build does not have): the map is rendered from the Gaussians
 * themselves.  Texel (i, j) holds the smallest light-space depth of the
 * Gaussians whose splat alpha at the texel centre reaches alpha_min,
 *   alpha = min(0.99, o exp(-q / 2)),   q = d^T Sigma2^{-1} d,
 * Sigma2 the orthographic image of the world covariance in texel units plus
 * the renderer's 0.3 low-pass, d = texel centre - projected centre; +inf
 * where no Gaussian reaches alpha_min.  With alpha_min <= 0.99 the test is
 * q <= tau = 2 ln(o / alpha_min).  A Gaussian is lit (255) when its centre
 * falls outside the map or its depth is at most the stored depth plus bias,
 * else shadowed (0).
 * Light camera: x_l = R (mu_world - origin); u = x_l / texel + W / 2,
 * v = y_l / texel + H / 2, depth z_l; texel (i, j) is sampled at
 * (i + 0.5, j + 0.5).  lcam[17]: R[9] (rows: map x, map y, depth axis),
 * origin[3], texel, W, H, alpha_min, bias.
 * slack (tests only) moves the bound to q <= tau + slack; brute = 1 tests
 * every texel instead of the footprint's bounding box.
 * ---------------------------------------------------------------------- */
typedef struct {
    double u, v, z;
    double A, B, C;   /* conic in texel units */
    double tau;
    double lmax;      /* larger eigenvalue of Sigma2 */
} light_splat;

static void light_project(const double* p, const dyn_t* dyn, int64_t g, const double* lc, light_splat* S) {
    double mu[3], s[3], q[4], qn, R[9], Sig[9], opac, Rg[9], Ld;
    gauss_common(p, mu, s, q, &qn, R, Sig, &opac);
    apply_dynamics(dyn, g, mu, Sig, Rg, &Ld);
    const double* Rl = lc;
    double h = lc[12], W = lc[13], H = lc[14];
    double d[3] = {mu[0] - lc[9], mu[1] - lc[10], mu[2] - lc[11]};
    double xl[3];
    for (int i = 0; i < 3; ++i) xl[i] = Rl[i * 3] * d[0] + Rl[i * 3 + 1] * d[1] + Rl[i * 3 + 2] * d[2];
    S->u = xl[0] / h + W / 2.0;
    S->v = xl[1] / h + H / 2.0;
    S->z = xl[2];
    /* Sigma2 = (1 / h^2) R_2 Sigma R_2^T + 0.3 I */
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            a += Rl[i] * Sig[i * 3 + j] * Rl[j];
            b += Rl[i] * Sig[i * 3 + j] * Rl[3 + j];
            c += Rl[3 + i] * Sig[i * 3 + j] * Rl[3 + j];
        }
    a = a / (h * h) + DILATION;
    b = b / (h * h);
    c = c / (h * h) + DILATION;
    double det = a * c - b * b;
    S->A = c / det; S->B = -b / det; S->C = a / det;
    double mid = 0.5 * (a + c);
    S->lmax = mid + sqrt(fmax(0.0, mid * mid - det));
    S->tau = 2.0 * log(opac / lc[15]);
}

static void light_depth_impl(int64_t n, const double* rows, const dyn_t* dyn, const double* lc, double slack,
                             int brute, double* depth) {
    int W = (int)lc[13], H = (int)lc[14];
    for (int64_t t = 0; t < (int64_t)W * H; ++t) depth[t] = INFINITY;
    for (int64_t g = 0; g < n; ++g) {
        light_splat S;
        light_project(rows + g * ROW, dyn, g, lc, &S);
        double bound = S.tau + slack;
        if (!(bound >= 0.0) || !isfinite(S.z)) continue;
        int i0 = 0, i1 = W - 1, j0 = 0, j1 = H - 1;
        if (!brute) {
            /* q <= bound implies |d|^2 <= bound * lmax */
            double r = sqrt(bound * S.lmax);
            i0 = (int)fmax(0.0, ceil(S.u - r - 0.5));
            i1 = (int)fmin(W - 1.0, floor(S.u + r - 0.5));
            j0 = (int)fmax(0.0, ceil(S.v - r - 0.5));
            j1 = (int)fmin(H - 1.0, floor(S.v + r - 0.5));
        }
        for (int j = j0; j <= j1; ++j)
            for (int i = i0; i <= i1; ++i) {
                double dx = i + 0.5 - S.u, dy = j + 0.5 - S.v;
                double qf = S.A * dx * dx + 2.0 * S.B * dx * dy + S.C * dy * dy;
                if (qf <= bound && S.z < depth[(int64_t)j * W + i]) depth[(int64_t)j * W + i] = S.z;
            }
    }
}

/* depth [H][W]; group / poses may be NULL (static scene) */
void or_light_depth(int64_t n, const double* rows, const int32_t* group, const double* poses, const double* lcam,
                    double slack, int brute, double* depth) {
    dyn_t d = {group, poses, NULL, {0, 0, 0}, 0.0, 0.0, NULL, NULL};
    light_depth_impl(n, rows, &d, lcam, slack, brute, depth);
}

/* vis [n] (255 lit, 0 shadowed); uvz [n][3] (may be NULL) receives u, v, z */
void or_light_visibility(int64_t n, const double* rows, const int32_t* group, const double* poses,
                         const double* lcam, const double* depth, uint8_t* vis, double* uvz) {
    dyn_t d = {group, poses, NULL, {0, 0, 0}, 0.0, 0.0, NULL, NULL};
    int W = (int)lcam[13], H = (int)lcam[14];
    for (int64_t g = 0; g < n; ++g) {
        light_splat S;
        light_project(rows + g * ROW, &d, g, lcam, &S);
        if (uvz) { uvz[g * 3] = S.u; uvz[g * 3 + 1] = S.v; uvz[g * 3 + 2] = S.z; }
        double fi = floor(S.u), fj = floor(S.v);
        if (!(fi >= 0.0 && fi < W && fj >= 0.0 && fj < H)) { vis[g] = 255; continue; }
        double D = depth[(int64_t)fj * W + (int64_t)fi];
        vis[g] = S.z <= D + lcam[16] ? 255 : 0;
    }
}

/* ------------------------------------------------------------------------
 * Loss (Sec. 3.1: "compares the result to the captured ground-truth images"
 * with the configured loss).  L = w_l1 mean|x - y| + w_ssim (1 - mean SSIM).
 * SSIM: 11x11 Gaussian window (sigma 1.5, normalised), C1 = 0.01^2,
 * C2 = 0.03^2, "same"-size window sums with zero padding (READING), mean over
 * all pixels, channels and views.  Writes dL/dx.
 * ---------------------------------------------------------------------- */
static void ssim_window(double* g) {
    double s = 0.0;
    for (int i = 0; i < 11; ++i) { g[i] = exp(-(double)((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5)); s += g[i]; }
    for (int i = 0; i < 11; ++i) g[i] /= s;
}

static const double SSIM_C1 = 0.0001, SSIM_C2 = 0.0009;

/* SSIM map of one plane (and, if dmap != NULL, the three per-pixel partials
 * dS/dmu_x, dS/dE[x^2], dS/dE[xy] used by the gradient). */
void or_ssim_map(int H, int W, const double* x, const double* y, double* smap, double* dmap) {
    double g[11];
    ssim_window(g);
#pragma omp parallel for schedule(dynamic, 4)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double mx = 0, my = 0, exx = 0, eyy = 0, exy = 0;
            for (int a = -5; a <= 5; ++a)
                for (int b = -5; b <= 5; ++b) {
                    int ii = i + a, jj = j + b;
                    if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                    double w = g[a + 5] * g[b + 5];
                    double xv = x[(int64_t)ii * W + jj], yv = y[(int64_t)ii * W + jj];
                    mx += w * xv; my += w * yv; exx += w * xv * xv; eyy += w * yv * yv; exy += w * xv * yv;
                }
            double sxx = exx - mx * mx, syy = eyy - my * my, sxy = exy - mx * my;
            double n1 = 2 * mx * my + SSIM_C1, n2 = 2 * sxy + SSIM_C2;
            double d1 = mx * mx + my * my + SSIM_C1, d2 = sxx + syy + SSIM_C2;
            double S = n1 * n2 / (d1 * d2);
            int64_t p = (int64_t)i * W + j;
            smap[p] = S;
            if (dmap) {
                dmap[3 * p + 0] = S * (2 * my / n1 - 2 * my / n2 - 2 * mx / d1 + 2 * mx / d2);
                dmap[3 * p + 1] = -S / d2;
                dmap[3 * p + 2] = 2 * S / n2;
            }
        }
}

double or_loss(int V, int H, int W, const double* img, const double* tgt, double w_l1,
               double w_ssim, double* dimg) {
    double g[11];
    ssim_window(g);
    int64_t P = (int64_t)H * W, M = (int64_t)V * 3 * P;
    double l1 = 0.0, ssum = 0.0;
    double* smap = (double*)malloc(sizeof(double) * P);
    double* dmap = (double*)malloc(sizeof(double) * P * 3);
    for (int64_t pl = 0; pl < (int64_t)V * 3; ++pl) {
        const double* x = img + pl * P;
        const double* y = tgt + pl * P;
        double* dx = dimg + pl * P;
        or_ssim_map(H, W, x, y, smap, dmap);
        for (int64_t p = 0; p < P; ++p) {
            double d = x[p] - y[p];
            l1 += fabs(d);
            ssum += smap[p];
            dx[p] = w_l1 * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)M;
        }
        /* dL/dx_q -= w_ssim/M * sum_p dS_p/dx_q, with
         * dS_p/dx_q = w(p-q) (dS/dmu_x + 2 x_q dS/dE[x^2] + y_q dS/dE[xy]) */
#pragma omp parallel for schedule(dynamic, 4)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                double acc = 0.0;
                int64_t q = (int64_t)i * W + j;
                for (int a = -5; a <= 5; ++a)
                    for (int b = -5; b <= 5; ++b) {
                        int ii = i + a, jj = j + b;
                        if (ii < 0 || ii >= H || jj < 0 || jj >= W) continue;
                        int64_t pp = (int64_t)ii * W + jj;
                        double w = g[a + 5] * g[b + 5];
                        acc += w * (dmap[3 * pp] + 2.0 * x[q] * dmap[3 * pp + 1] + y[q] * dmap[3 * pp + 2]);
                    }
                dx[q] -= w_ssim * acc / (double)M;
            }
    }
    free(smap);
    free(dmap);
    return w_l1 * l1 / (double)M + w_ssim * (1.0 - ssum / (double)M);
}

/* ------------------------------------------------------------------------
 * Adam (Sec. 3.1: "updates the trainable Gaussian parameters using the
 * configured loss and learning rates"; Sec. 3.3: optimizer state is extended
 * with the model).  READING: the torch defaults beta1 0.9, beta2 0.999,
 * eps 1e-8, bias-corrected, dense.  lr is given per element.
 * ---------------------------------------------------------------------- */
void or_adam(int64_t count, double* theta, const double* grad, double* m, double* v,
             const double* lr, double b1, double b2, double eps, int step) {
    double bc1 = 1.0 - pow(b1, step), bc2 = 1.0 - pow(b2, step);
    for (int64_t i = 0; i < count; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        double mh = m[i] / bc1, vh = v[i] / bc2;
        theta[i] -= lr[i] * mh / (sqrt(vh) + eps);
    }
}

/* ------------------------------------------------------------------------
 * Changed-set extraction for the incremental stream (Sec. 3.5: tensor-delta
 * packets between snapshots; residuals relative to the previously transmitted
 * state; fresh baselines after a snapshot).
 * READING: Gaussian i is sent when max over its 59 stored attributes of
 * |theta - baseline| > thr (decided in float32, as the GPU decides it); the
 * baseline is the last transmitted float32 value; indices ascend; record =
 * u32 index, float32 mean xyz, then 56 float16 (round to nearest even):
 * log-scale xyz, quaternion wxyz, opacity logit, 48 SH.  Sent baselines are
 * replaced by theta.
 * ---------------------------------------------------------------------- */
uint16_t or_f32_to_f16(float f) {
    double a = fabs((double)f);
    uint16_t sign = signbit(f) ? 0x8000 : 0;
    if (isnan(f)) return sign | 0x7E00;
    if (a >= 65520.0) return sign | 0x7C00;          /* rounds to infinity */
    if (a < ldexp(1.0, -14)) {                       /* subnormal range */
        double m = rint(a / ldexp(1.0, -24));        /* nearest, ties to even */
        return sign | (uint16_t)m;                   /* m == 1024 encodes 2^-14 */
    }
    int e;
    frexp(a, &e);                                    /* a = f * 2^e, f in [0.5, 1) */
    e -= 1;                                          /* a in [2^e, 2^(e+1)) */
    double m = rint(a / ldexp(1.0, e - 10));         /* in [1024, 2048] */
    if (m == 2048.0) { m = 1024.0; e += 1; }
    if (e + 15 >= 31) return sign | 0x7C00;
    return sign | (uint16_t)(((e + 15) << 10) | ((int)m - 1024));
}

int64_t or_delta(int64_t n, const float* theta, float* base, float thr, uint32_t* idx, uint8_t* rec) {
    int64_t cnt = 0;
    for (int64_t g = 0; g < n; ++g) {
        const float* t = theta + g * ROW;
        float* b = base + g * ROW;
        int changed = 0;
        for (int k = 0; k < ROW; ++k) {
            float d = fabsf(t[k] - b[k]);
            if (d > thr) changed = 1;
        }
        if (!changed) continue;
        idx[cnt] = (uint32_t)g;
        uint8_t* r = rec + cnt * 128;
        uint32_t gi = (uint32_t)g;
        memcpy(r, &gi, 4);
        memcpy(r + 4, t, 12);
        /* order: log-scale (4..6), quaternion (8..11), opacity logit (3), SH (12..59) */
        int order[56], o = 0;
        for (int k = 4; k < 7; ++k) order[o++] = k;
        for (int k = 8; k < 12; ++k) order[o++] = k;
        order[o++] = 3;
        for (int k = 12; k < 60; ++k) order[o++] = k;
        for (int k = 0; k < 56; ++k) {
            uint16_t h = or_f32_to_f16(t[order[k]]);
            memcpy(r + 16 + 2 * k, &h, 2);
        }
        memcpy(b, t, sizeof(float) * ROW);
        ++cnt;
    }
    return cnt;
}

/* ------------------------------------------------------------------------
 * Tensor deltas per attribute group and their client-side replay (Sec. 3.5:
 * attribute-specific delta encoders on the server, matching replay objects on
 * the client; opacity and DC every frame, the other tensors less often).
 * Groups (bit, flat floats of a Gaussian's row, encoding):
 *   1 mean      0..2    float32
 *   2 opacity   3       float16 (logit)
 *   4 scale     4..6    float16 (log-scale)
 *   8 rotation  8..11   float16 (quaternion)
 *  16 dc        12..14  float16 (SH degree 0)
 *  32 sh_rest   15..59  float16 (SH degrees 1..3)
 * A Gaussian is sent for a group when max over the group's floats of
 * |theta - base| > thr; sent Gaussians ascend; their group floats become the
 * new baseline.  Records are the group's values, packed densely.
 * ---------------------------------------------------------------------- */
static int group_floats(int attr, int* lo, int* hi, int* f32) {
    *f32 = 0;
    switch (attr) {
        case 1: *lo = 0; *hi = 3; *f32 = 1; return 1;
        case 2: *lo = 3; *hi = 4; return 1;
        case 4: *lo = 4; *hi = 7; return 1;
        case 8: *lo = 8; *hi = 12; return 1;
        case 16: *lo = 12; *hi = 15; return 1;
        case 32: *lo = 15; *hi = 60; return 1;
        default: return 0;
    }
}

/* IEEE binary16 -> float: sign, 5-bit exponent (bias 15), 10-bit fraction;
 * subnormals are fraction * 2^-24; exponent 31 is inf / NaN. */
float or_f16_to_f32(uint16_t h) {
    const int s = (h >> 15) & 1, e = (h >> 10) & 31, f = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)f, -24);
    else if (e == 31) v = f ? NAN : INFINITY;
    else v = ldexp(1024.0 + (double)f, e - 25);
    return (float)(s ? -v : v);
}

int or_tensor_record_bytes(int attr) {
    int lo, hi, f32;
    if (!group_floats(attr, &lo, &hi, &f32)) return -1;
    return (hi - lo) * (f32 ? 4 : 2);
}

int64_t or_tensor_delta(int64_t n, const float* theta, float* base, int attr, float thr, uint32_t* idx,
                        uint8_t* vals) {
    int lo, hi, f32;
    if (!group_floats(attr, &lo, &hi, &f32)) return -1;
    const int rb = (hi - lo) * (f32 ? 4 : 2);
    int64_t cnt = 0;
    for (int64_t g = 0; g < n; ++g) {
        const float* t = theta + g * ROW;
        float* b = base + g * ROW;
        int changed = 0;
        for (int k = lo; k < hi; ++k)
            if (fabsf(t[k] - b[k]) > thr) changed = 1;
        if (!changed) continue;
        idx[cnt] = (uint32_t)g;
        uint8_t* r = vals + cnt * rb;
        for (int k = lo; k < hi; ++k) {
            if (f32) {
                memcpy(r + 4 * (k - lo), &t[k], 4);
            } else {
                const uint16_t h = or_f32_to_f16(t[k]);
                memcpy(r + 2 * (k - lo), &h, 2);
            }
            b[k] = t[k];
        }
        ++cnt;
    }
    return cnt;
}

void or_apply_tensor_delta(int64_t n, float* params, int attr, int64_t m, const uint32_t* idx,
                           const uint8_t* vals) {
    int lo, hi, f32;
    if (!group_floats(attr, &lo, &hi, &f32)) return;
    const int rb = (hi - lo) * (f32 ? 4 : 2);
    for (int64_t i = 0; i < m; ++i) {
        if ((int64_t)idx[i] >= n) continue;
        float* row = params + (int64_t)idx[i] * ROW;
        const uint8_t* r = vals + i * rb;
        for (int k = lo; k < hi; ++k) {
            if (f32) {
                memcpy(&row[k], r + 4 * (k - lo), 4);
            } else {
                uint16_t h;
                memcpy(&h, r + 2 * (k - lo), 2);
                row[k] = or_f16_to_f32(h);
            }
        }
    }
}

/* Replay of the full 128-byte records of or_delta. */
void or_apply_delta(int64_t n, float* params, int64_t m, const uint8_t* rec) {
    for (int64_t i = 0; i < m; ++i) {
        const uint8_t* r = rec + i * 128;
        uint32_t g;
        memcpy(&g, r, 4);
        if ((int64_t)g >= n) continue;
        float* row = params + (int64_t)g * ROW;
        memcpy(row, r + 4, 12);
        int order[56], o = 0;
        for (int k = 4; k < 7; ++k) order[o++] = k;
        for (int k = 8; k < 12; ++k) order[o++] = k;
        order[o++] = 3;
        for (int k = 12; k < 60; ++k) order[o++] = k;
        for (int k = 0; k < 56; ++k) {
            uint16_t h;
            memcpy(&h, r + 16 + 2 * k, 2);
            row[order[k]] = or_f16_to_f32(h);
        }
    }
}

/* ------------------------------------------------------------------------
 * Preculling (Sec. 3.3): Gaussians belong to cells of a regular 3D grid; each
 * camera keeps the cells that pass a depth test against its depth buffer;
 * only Gaussians of kept cells are rendered and optimised.  Reading (the
 * paper names no test): a conservative hierarchical depth test, evaluated in
 * float32 with explicit fused multiply-adds so that the decision is the one a
 * float32 producer takes:
 *   - the cell of a point is floor((p - origin) / size) per axis, clamped;
 *   - per view, the cell's 8 corners are moved to camera space
 *     (z = R[6] x + R[7] y + R[8] z + t[2] as nested fmaf, likewise x, y);
 *     all corners at z <= near: not seen; some: the whole image at depth
 *     near; else u = fmaf(fx, x / z, cx), v likewise, and the pixels
 *     floor(min u) .. floor(max u) by floor(min v) .. floor(max v), clipped
 *     to the image (empty: not seen), at depth min z;
 *   - the depth buffer's max pyramid: level 0 is the buffer, level k + 1 of
 *     size ((w + 1) / 2, (h + 1) / 2) holds the max of each 2x2 block;
 *   - the level L is the first at which the pixel range spans at most two
 *     texels per axis; the cell is seen when its depth <= the max over those
 *     (up to 4) texels.
 * A cell is kept when some view sees it.
 * ---------------------------------------------------------------------- */
int64_t or_cell_of(const float* p, const float* origin, float size, const int* dims) {
    int c[3];
    for (int a = 0; a < 3; ++a) {
        const float d = (p[a] - origin[a]) / size;
        long long k = (long long)floorf(d);
        if (k < 0) k = 0;
        if (k > dims[a] - 1) k = dims[a] - 1;
        c[a] = (int)k;
    }
    return ((int64_t)c[2] * dims[1] + c[1]) * dims[0] + c[0];
}

/* Max pyramid of one W x H buffer into out (levels back to back, level 0
 * first); returns the number of levels. */
int or_depth_mips(const float* depth, int W, int H, float* out) {
    memcpy(out, depth, sizeof(float) * (size_t)W * H);
    float* prev = out;
    int w = W, h = H, levels = 1;
    float* cur = out + (size_t)W * H;
    while (w > 1 || h > 1) {
        const int w2 = (w + 1) / 2, h2 = (h + 1) / 2;
        for (int j = 0; j < h2; ++j)
            for (int i = 0; i < w2; ++i) {
                float m = -INFINITY;
                for (int dj = 0; dj < 2; ++dj)
                    for (int di = 0; di < 2; ++di) {
                        const int y = 2 * j + dj, x = 2 * i + di;
                        if (y < h && x < w) m = fmaxf(m, prev[(size_t)y * w + x]);
                    }
                cur[(size_t)j * w2 + i] = m;
            }
        prev = cur;
        cur += (size_t)w2 * h2;
        w = w2; h = h2;
        ++levels;
    }
    return levels;
}

static int mip_count(int W, int H) {
    int l = 1;
    while (W > 1 || H > 1) { W = (W + 1) / 2; H = (H + 1) / 2; ++l; }
    return l;
}

static size_t mip_floats(int W, int H) {
    size_t s = 0;
    for (;;) {
        s += (size_t)W * H;
        if (W == 1 && H == 1) break;
        W = (W + 1) / 2; H = (H + 1) / 2;
    }
    return s;
}

/* cams: float32 camera records [V][20] (oracle layout); depth: the views'
 * buffers back to back; vis: [nz][ny][nx]. */
void or_cell_visible(int V, const float* cams, const float* depth, const float* origin, float size,
                     const int* dims, uint8_t* vis) {
    const int64_t ncell = (int64_t)dims[0] * dims[1] * dims[2];
    memset(vis, 0, (size_t)ncell);
    size_t doff = 0;
    for (int v = 0; v < V; ++v) {
        const float* c = cams + (int64_t)v * CAM_STRIDE;
        const int W = (int)c[16], H = (int)c[17];
        const float near = c[18];
        float* mips = (float*)malloc(sizeof(float) * mip_floats(W, H));
        or_depth_mips(depth + doff, W, H, mips);
        const int levels = mip_count(W, H);
        for (int64_t cell = 0; cell < ncell; ++cell) {
            if (vis[cell]) continue;
            const int cx = (int)(cell % dims[0]), cy = (int)((cell / dims[0]) % dims[1]),
                      cz = (int)(cell / ((int64_t)dims[0] * dims[1]));
            float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY, zmin = INFINITY;
            int behind = 0;
            for (int k = 0; k < 8; ++k) {
                const float px = fmaf(size, (float)(cx + (k & 1)), origin[0]);
                const float py = fmaf(size, (float)(cy + ((k >> 1) & 1)), origin[1]);
                const float pz = fmaf(size, (float)(cz + ((k >> 2) & 1)), origin[2]);
                const float X = fmaf(c[0], px, fmaf(c[1], py, fmaf(c[2], pz, c[9])));
                const float Y = fmaf(c[3], px, fmaf(c[4], py, fmaf(c[5], pz, c[10])));
                const float Z = fmaf(c[6], px, fmaf(c[7], py, fmaf(c[8], pz, c[11])));
                if (Z <= near) { ++behind; continue; }
                const float u = fmaf(c[12], X / Z, c[14]), w = fmaf(c[13], Y / Z, c[15]);
                umin = fminf(umin, u); umax = fmaxf(umax, u);
                vmin = fminf(vmin, w); vmax = fmaxf(vmax, w);
                zmin = fminf(zmin, Z);
            }
            if (behind == 8) continue;
            long long x0, x1, y0, y1;
            if (behind) { x0 = 0; x1 = W - 1; y0 = 0; y1 = H - 1; zmin = near; }
            else {
                x0 = (long long)floorf(umin); x1 = (long long)floorf(umax);
                y0 = (long long)floorf(vmin); y1 = (long long)floorf(vmax);
                if (x1 < 0 || y1 < 0 || x0 > W - 1 || y0 > H - 1) continue;
                if (x0 < 0) x0 = 0;
                if (y0 < 0) y0 = 0;
                if (x1 > W - 1) x1 = W - 1;
                if (y1 > H - 1) y1 = H - 1;
            }
            int L = 0;
            while (L < levels - 1 && (((x1 >> L) - (x0 >> L)) > 1 || ((y1 >> L) - (y0 >> L)) > 1)) ++L;
            /* the level's buffer and width */
            size_t off = 0;
            int w = W, h = H;
            for (int l = 0; l < L; ++l) { off += (size_t)w * h; w = (w + 1) / 2; h = (h + 1) / 2; }
            float m = -INFINITY;
            for (long long j = y0 >> L; j <= (y1 >> L); ++j)
                for (long long i = x0 >> L; i <= (x1 >> L); ++i) m = fmaxf(m, mips[off + (size_t)j * w + i]);
            if (zmin <= m) vis[cell] = 1;
        }
        free(mips);
        doff += (size_t)W * H;
    }
}

