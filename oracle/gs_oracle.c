/*
 * gs_oracle.c -- plain FP64 CPU oracle for the Gaussian-splatting RGB-D
 * renderer and the linear-blend-skinning (LBS) deformation of Gaussian avatars.
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  The CUDA product path
 * neither links nor calls it, and the two share no source.
 *
 * What it follows.  The paper renders scene Gaussians with tile-based 3D
 * Gaussian Splatting rasterisation (Sec. 2.2 and Sec. 3.2) and deforms canonical
 * avatar Gaussians to the current pose with a CUDA LBS kernel over per-frame
 * SMPL-X joint matrices (Sec. 3.1 "Asset Preparation", Sec. 3.3, Sec. 3.3.1).
 * It prints no rasteriser formulas, so this file writes out the standard
 * definitions it cites:
 *   activation  scale = exp(s), opacity = sigmoid(o), R = R(q / |q|),
 *               Sigma = R diag(scale^2) R^T (or a given posed covariance);
 *   view        d = mu - C, p = W d   (W world->camera rotation, C centre);
 *   projection  u = fx px/pz + cx, v = fy py/pz + cy; EWA Jacobian J with
 *               the lateral clamp at 1.3 x half-field; Sigma2 = J W Sigma W^T J^T
 *               plus 0.3 px^2 on the diagonal;
 *   conic       inverse of Sigma2, radius r = ceil(3 sqrt(lambda_max)) with the
 *               0.1 floor on the discriminant;
 *   footprint   pixel (i, j) is covered iff |i-u| <= r and |j-v| <= r;
 *   colour      real spherical harmonics of degree 3 at the unit view
 *               direction, + 0.5, clamped below at 0;
 *   order       per pixel, covered Gaussians by (depth key, index);
 *   blend       alpha = min(0.99, opacity exp(power)), skip alpha < 1/255,
 *               stop before blending when T (1-alpha) < 1e-4;
 *               C += c alpha T, D += z alpha T, T *= (1 - alpha);
 *   counts      n_contrib = the Gaussians blended into the pixel; n_covered =
 *               the covered Gaussians examined up to and including the last
 *               blended one (the length of the adjoint's walk).
 * Two decisions are taken in FP32 so that both sides take them in the same
 * precision: the depth key that orders and near-culls the Gaussians is
 *   zkey = fl(fl(fl(W20 d0) + fl(W21 d1)) + fl(W22 d2)),  d_i = fl(mu_i - C_i)
 * in single precision.  Everything else is double precision.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (contraction off so
 * that the FP32 key is bit-reproducible on x86-64 and aarch64).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AMB_VALUE 1u /* colour or depth may differ beyond the FP32 tolerance */
#define AMB_COUNT 2u /* the contributor count may differ by a flipped decision */
/* which decision was near its threshold (informational) */
#define AMB_FOOTPRINT 4u
#define AMB_ORDER 8u
#define AMB_ALPHA 16u
#define AMB_STOP 32u
#define AMB_CLAMP 64u /* alpha within FP32 error of the 0.99 clamp: the value is continuous there, the
                         gradient is not (it passes zero where the clamp is active) */

#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_STOP 1e-4
#define DILATION 0.3
#define FLAG_NORMALIZE_DEPTH 1

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics up to degree 3, in the ordering and sign          */
/* convention of the 3DGS reference renderer (Condon-Shortley phase folded    */
/* into the m = +-1 terms).  Normalisation constants are written from their   */
/* closed forms so that they can be checked by eye.                           */
/* ------------------------------------------------------------------------ */
static void sh_consts(double c[16])
{
    const double pi = 3.14159265358979323846;
    double c0 = sqrt(1.0 / (4.0 * pi));
    double c1 = sqrt(3.0 / (4.0 * pi));
    c[0] = c0;
    c[1] = -c1; c[2] = c1; c[3] = -c1;
    c[4] = 0.5 * sqrt(15.0 / pi);
    c[5] = -0.5 * sqrt(15.0 / pi);
    c[6] = 0.25 * sqrt(5.0 / pi);
    c[7] = -0.5 * sqrt(15.0 / pi);
    c[8] = 0.25 * sqrt(15.0 / pi);
    c[9] = -0.25 * sqrt(35.0 / (2.0 * pi));
    c[10] = 0.5 * sqrt(105.0 / pi);
    c[11] = -0.25 * sqrt(21.0 / (2.0 * pi));
    c[12] = 0.25 * sqrt(7.0 / pi);
    c[13] = -0.25 * sqrt(21.0 / (2.0 * pi));
    c[14] = 0.25 * sqrt(105.0 / pi);
    c[15] = -0.25 * sqrt(35.0 / (2.0 * pi));
}

/* Y[k](x,y,z) for a unit direction, and (optionally) its gradient dY[k][3]. */
static void sh_eval(const double dir[3], double Y[16], double dY[16][3])
{
    double c[16];
    sh_consts(c);
    double x = dir[0], y = dir[1], z = dir[2];
    double xx = x * x, yy = y * y, zz = z * z;
    Y[0] = c[0];
    Y[1] = c[1] * y;
    Y[2] = c[2] * z;
    Y[3] = c[3] * x;
    Y[4] = c[4] * x * y;
    Y[5] = c[5] * y * z;
    Y[6] = c[6] * (2.0 * zz - xx - yy);
    Y[7] = c[7] * x * z;
    Y[8] = c[8] * (xx - yy);
    Y[9] = c[9] * y * (3.0 * xx - yy);
    Y[10] = c[10] * x * y * z;
    Y[11] = c[11] * y * (4.0 * zz - xx - yy);
    Y[12] = c[12] * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[13] = c[13] * x * (4.0 * zz - xx - yy);
    Y[14] = c[14] * z * (xx - yy);
    Y[15] = c[15] * x * (xx - 3.0 * yy);
    if (!dY) return;
    memset(dY, 0, sizeof(double) * 48);
    dY[1][1] = c[1];
    dY[2][2] = c[2];
    dY[3][0] = c[3];
    dY[4][0] = c[4] * y;  dY[4][1] = c[4] * x;
    dY[5][1] = c[5] * z;  dY[5][2] = c[5] * y;
    dY[6][0] = -2.0 * c[6] * x; dY[6][1] = -2.0 * c[6] * y; dY[6][2] = 4.0 * c[6] * z;
    dY[7][0] = c[7] * z;  dY[7][2] = c[7] * x;
    dY[8][0] = 2.0 * c[8] * x; dY[8][1] = -2.0 * c[8] * y;
    dY[9][0] = 6.0 * c[9] * x * y; dY[9][1] = c[9] * (3.0 * xx - 3.0 * yy);
    dY[10][0] = c[10] * y * z; dY[10][1] = c[10] * x * z; dY[10][2] = c[10] * x * y;
    dY[11][0] = -2.0 * c[11] * x * y; dY[11][1] = c[11] * (4.0 * zz - xx - 3.0 * yy);
    dY[11][2] = 8.0 * c[11] * y * z;
    dY[12][0] = -6.0 * c[12] * x * z; dY[12][1] = -6.0 * c[12] * y * z;
    dY[12][2] = c[12] * (6.0 * zz - 3.0 * xx - 3.0 * yy);
    dY[13][0] = c[13] * (4.0 * zz - 3.0 * xx - yy); dY[13][1] = -2.0 * c[13] * x * y;
    dY[13][2] = 8.0 * c[13] * x * z;
    dY[14][0] = 2.0 * c[14] * x * z; dY[14][1] = -2.0 * c[14] * y * z; dY[14][2] = c[14] * (xx - yy);
    dY[15][0] = c[15] * (3.0 * xx - 3.0 * yy); dY[15][1] = -6.0 * c[15] * x * y;
}

void or_sh_basis(int64_t n, const double *dirs, double *out)
{
    for (int64_t i = 0; i < n; ++i) sh_eval(dirs + 3 * i, out + 16 * i, NULL);
}

/* ------------------------------------------------------------------------ */
/* Rotation of a unit quaternion (w, x, y, z) and its partial derivatives.    */
/* ------------------------------------------------------------------------ */
static void quat_rot(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* dL/dq (unit quaternion components) given dL/dR (row-major 3x3). */
static void quat_rot_vjp(const double q[4], const double gR[9], double gq[4])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    gq[0] = gR[1] * (-2 * z) + gR[2] * (2 * y) + gR[3] * (2 * z) + gR[5] * (-2 * x) + gR[6] * (-2 * y) + gR[7] * (2 * x);
    gq[1] = gR[1] * (2 * y) + gR[2] * (2 * z) + gR[3] * (2 * y) + gR[4] * (-4 * x) + gR[5] * (-2 * w) + gR[6] * (2 * z) +
            gR[7] * (2 * w) + gR[8] * (-4 * x);
    gq[2] = gR[0] * (-4 * y) + gR[1] * (2 * x) + gR[2] * (2 * w) + gR[3] * (2 * x) + gR[5] * (2 * z) + gR[6] * (-2 * w) +
            gR[7] * (2 * z) + gR[8] * (-4 * y);
    gq[3] = gR[0] * (-4 * z) + gR[1] * (-2 * w) + gR[2] * (2 * x) + gR[3] * (2 * w) + gR[4] * (-4 * z) + gR[5] * (2 * y) +
            gR[6] * (2 * x) + gR[7] * (2 * y);
}

void or_quat_to_rot(const double *q, double *R)
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qn[4] = {q[0] / n, q[1] / n, q[2] / n, q[3] / n};
    quat_rot(qn, R);
}

/* Sigma = R diag(exp(2 s)) R^T, with R = R(q / |q|). */
static void cov_from_scale_rot(const double s[3], const double q[4], double S[9])
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qn[4] = {q[0] / n, q[1] / n, q[2] / n, q[3] / n};
    double R[9];
    quat_rot(qn, R);
    double sc[3] = {exp(s[0]), exp(s[1]), exp(s[2])};
    double M[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = R[3 * r + c] * sc[c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += M[3 * r + k] * M[3 * c + k];
            S[3 * r + c] = acc;
        }
}

/* Backward of cov_from_scale_rot: given symmetric dL/dSigma, add dL/ds, dL/dq. */
static void cov_from_scale_rot_vjp(const double s[3], const double q[4], const double gS[9], double gs[3], double gq[4])
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qn[4] = {q[0] / n, q[1] / n, q[2] / n, q[3] / n};
    double R[9];
    quat_rot(qn, R);
    double sc[3] = {exp(s[0]), exp(s[1]), exp(s[2])};
    double M[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) M[3 * r + c] = R[3 * r + c] * sc[c];
    /* Sigma = M M^T, dL/dM = 2 gS M for symmetric gS */
    double gM[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += gS[3 * r + k] * M[3 * k + c];
            gM[3 * r + c] = 2.0 * acc;
        }
    double gR[9];
    for (int c = 0; c < 3; ++c) {
        double gsc = 0.0;
        for (int r = 0; r < 3; ++r) {
            gsc += gM[3 * r + c] * R[3 * r + c];
            gR[3 * r + c] = gM[3 * r + c] * sc[c];
        }
        gs[c] += gsc * sc[c];
    }
    double gqn[4];
    quat_rot_vjp(qn, gR, gqn);
    double dot = gqn[0] * qn[0] + gqn[1] * qn[1] + gqn[2] * qn[2] + gqn[3] * qn[3];
    for (int k = 0; k < 4; ++k) gq[k] += (gqn[k] - qn[k] * dot) / n;
}

/* ------------------------------------------------------------------------ */
/* Projection of one Gaussian into one view.                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    double R[9], C[3], fx, fy, cx, cy;
} cam_t;

static void load_cam(const double *c, cam_t *k)
{
    memcpy(k->R, c, 9 * sizeof(double));
    memcpy(k->C, c + 9, 3 * sizeof(double));
    k->fx = c[12]; k->fy = c[13]; k->cx = c[14]; k->cy = c[15];
}

/* Depth key in single precision, in the fixed order stated at the top. */
static float depth_key(const double mu[3], const cam_t *k)
{
    float d0 = (float)mu[0] - (float)k->C[0];
    float d1 = (float)mu[1] - (float)k->C[1];
    float d2 = (float)mu[2] - (float)k->C[2];
    float a = (float)k->R[6] * d0;
    float b = (float)k->R[7] * d1;
    float c = (float)k->R[8] * d2;
    float s = a + b;
    s = s + c;
    return s;
}

typedef struct {
    /* inputs gathered */
    double mu[3], Sigma[9];
    /* view */
    double d[3], p[3];
    float zkey;
    /* projection */
    double u, v, J[6], T[6], cov2[3], det, conic[3];
    double tx, ty;
    int clampx, clampy;
    double r3, er3; /* 3 sqrt(lambda) and its FP32 error bound */
    int32_t r, r_lo, r_hi;
    double opacity, rgb[3], raw[3], dir[3], dnorm;
    double du, dv; /* FP32 error bounds of (u, v) in pixels */
    double eA, eB, eC; /* FP32 error bounds of the conic entries */
    double ea, eb, ec; /* FP32 error bounds of the 2D covariance entries a, b, c */
    double rel_conic;  /* relative error of the conic's own roundings */
    double ez;         /* FP32 error bound of the depth key (inexact inputs only) */
    int cand;      /* footprint under r_hi touches the image */
    int visible;   /* footprint under r touches the image */
} proj_t;

static int footprint_on_image(double u, double v, int32_t r, int W, int H)
{
    /* exists integer i in [0, W-1] with |i - u| <= r, same for j */
    double ilo = ceil(u - r), ihi = floor(u + r);
    double jlo = ceil(v - r), jhi = floor(v + r);
    if (ilo < 0) ilo = 0;
    if (ihi > W - 1) ihi = W - 1;
    if (jlo < 0) jlo = 0;
    if (jhi > H - 1) jhi = H - 1;
    return ilo <= ihi && jlo <= jhi;
}

/* ------------------------------------------------------------------------ */
/* First-order FP32 error bounds.  The CUDA path computes the projection in   */
/* single precision; the ambiguity mask needs, for each decision it takes,    */
/* a bound on how far its FP32 input can lie from the FP64 value here.  Each  */
/* bound follows the CUDA path's evaluation order: an expression evaluated    */
/* with n roundings of terms of magnitudes m_i is off by at most              */
/* gamma(n) sum m_i (unit roundoff U = 2^-24, gamma(n) = nU / (1 - nU)), and  */
/* input errors propagate through absolute first-order sensitivities.         */
/* Library functions enter with their documented accuracy: expf within 2 ulp, */
/* sqrtf and division correctly rounded.  One ulp is at most 2U relative.     */
/* Posed (inexact) inputs were produced by an FP32 LBS of rigid joint         */
/* transforms applied to canonical Gaussians within 2 m (L1) of the canonical */
/* origin; their mean and covariance errors are bounded under that premise.   */
/* ------------------------------------------------------------------------ */
#define U32 (1.0 / 16777216.0)
static double gam(int n) { return n * U32 / (1.0 - n * U32); }
#define E_ALPHA (24.0 * U32)

static void fp32_bounds(proj_t *o, const double *ls, const double *q, int use_cov, int inexact, const cam_t *k)
{
    const double *d = o->d, *mu = o->mu;
    /* posed mean: blended 3x4 matrix (4 roundings per entry) applied to the
     * canonical mean (3 roundings): |dmu_r| <= 7U (|mu_r| + 3 |m|_1), |m|_1 <= 2 */
    double em[3] = {0.0, 0.0, 0.0};
    if (inexact)
        for (int r = 0; r < 3; ++r) em[r] = (gam(4) + gam(3)) * (fabs(mu[r]) + 6.0);
    /* d = mu - C (one rounding); p_r = sum_j W_rj d_j (three roundings, the
     * depth key as well); |W_rj| <= 1 */
    double ed[3], ep[3];
    for (int j = 0; j < 3; ++j) ed[j] = U32 * fabs(d[j]) + em[j];
    for (int r = 0; r < 3; ++r) {
        double a = 0.0, b = 0.0;
        for (int j = 0; j < 3; ++j) {
            a += fabs(k->R[3 * r + j]) * ed[j];
            b += fabs(k->R[3 * r + j] * d[j]);
        }
        ep[r] = a + gam(3) * b;
    }
    const double px = o->p[0], py = o->p[1], pz = o->p[2];
    o->ez = inexact ? ep[2] : 0.0; /* exact inputs: the key is the FP32 one here too */
    /* u - cx = fx (px / pz): a division and a product */
    const double tx0 = px / pz, ty0 = py / pz;
    o->du = k->fx / pz * (ep[0] + fabs(tx0) * ep[2]) + gam(2) * fabs(k->fx * tx0);
    o->dv = k->fy / pz * (ep[1] + fabs(ty0) * ep[2]) + gam(2) * fabs(k->fy * ty0);
    /* Jacobian: j00 = fx / pz, j02 = -(fx tx) / pz with tx = px / pz, or the
     * clamp limit 1.3 (W / 2) / fx (three roundings) */
    const double tx = o->tx, ty = o->ty;
    const double etx = o->clampx ? gam(3) * fabs(tx) : (ep[0] + fabs(tx0) * ep[2]) / pz + U32 * fabs(tx0);
    const double ety = o->clampy ? gam(3) * fabs(ty) : (ep[1] + fabs(ty0) * ep[2]) / pz + U32 * fabs(ty0);
    const double j00 = k->fx / pz, j02 = k->fx * fabs(tx) / pz, j11 = k->fy / pz, j12 = k->fy * fabs(ty) / pz;
    const double ej00 = j00 * (U32 + ep[2] / pz), ej11 = j11 * (U32 + ep[2] / pz);
    const double ej02 = k->fx / pz * (fabs(tx) * (gam(2) + ep[2] / pz) + etx);
    const double ej12 = k->fy / pz * (fabs(ty) * (gam(2) + ep[2] / pz) + ety);
    /* T = J W: two roundings per entry */
    double et[6];
    for (int c = 0; c < 3; ++c) {
        et[c] = fabs(k->R[c]) * ej00 + fabs(k->R[6 + c]) * ej02 + gam(2) * (j00 * fabs(k->R[c]) + j02 * fabs(k->R[6 + c]));
        et[3 + c] = fabs(k->R[3 + c]) * ej11 + fabs(k->R[6 + c]) * ej12 +
                    gam(2) * (j11 * fabs(k->R[3 + c]) + j12 * fabs(k->R[6 + c]));
    }
    const double *T = o->T, *S = o->Sigma;
    const double a = o->cov2[0], b = o->cov2[1], c = o->cov2[2], det = o->det;
    double e2[3]; /* a, b, c */
    double edet;
    o->ea = o->eb = o->ec = o->rel_conic = 0.0;
    if (!use_cov) {
        /* scale-rotation Gaussian, the factor form: M = R(q) diag(exp s) with
         * 1/|q| within 4U, the entries of R(q) within 25U absolute, exp(s)
         * within 4U: |dM_kj| <= scale_j (25U + 5U |R_kj|); G = T M (three
         * roundings); a' = |G_0|^2, b = G_0 . G_1, c' = |G_1|^2 (three each);
         * a = a' + 0.3 (one, 0.3f - 0.3 = 1.2e-8); det = (sum of the three
         * squared 2 x 2 minors of G, each minor two roundings, the sum three)
         * + 0.3 (a' + c') + 0.09 (three more; 0.09f - 0.09 = 3.6e-9) */
        double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double qn[4] = {q[0] / n, q[1] / n, q[2] / n, q[3] / n};
        double R[9];
        quat_rot(qn, R);
        double M[9], eM[9];
        for (int kk = 0; kk < 3; ++kk)
            for (int j = 0; j < 3; ++j) {
                const double sj = exp(ls[j]);
                M[3 * kk + j] = R[3 * kk + j] * sj;
                eM[3 * kk + j] = sj * (25.0 * U32 + 5.0 * U32 * fabs(R[3 * kk + j]));
            }
        double G[2][3], eG[2][3];
        for (int r = 0; r < 2; ++r)
            for (int j = 0; j < 3; ++j) {
                double v = 0.0, m = 0.0, e = 0.0;
                for (int kk = 0; kk < 3; ++kk) {
                    v += T[3 * r + kk] * M[3 * kk + j];
                    m += fabs(T[3 * r + kk] * M[3 * kk + j]);
                    e += et[3 * r + kk] * fabs(M[3 * kk + j]) + fabs(T[3 * r + kk]) * eM[3 * kk + j];
                }
                G[r][j] = v;
                eG[r][j] = gam(3) * m + e;
            }
        double ea1 = 0.0, ec1 = 0.0, eb = 0.0, sa = 0.0, sc1 = 0.0, sb = 0.0;
        for (int j = 0; j < 3; ++j) {
            sa += G[0][j] * G[0][j];
            sc1 += G[1][j] * G[1][j];
            sb += fabs(G[0][j] * G[1][j]);
            ea1 += 2.0 * fabs(G[0][j]) * eG[0][j];
            ec1 += 2.0 * fabs(G[1][j]) * eG[1][j];
            eb += fabs(G[0][j]) * eG[1][j] + eG[0][j] * fabs(G[1][j]);
        }
        ea1 += gam(3) * sa;
        ec1 += gam(3) * sc1;
        eb += gam(3) * sb;
        e2[0] = ea1 + U32 * a + 1.2e-8;
        e2[1] = eb;
        e2[2] = ec1 + U32 * c + 1.2e-8;
        const int mi[3] = {0, 0, 1}, mj[3] = {1, 2, 2};
        double dg = 0.0, edg = 0.0;
        for (int x = 0; x < 3; ++x) {
            const int i = mi[x], j = mj[x];
            const double m = G[0][i] * G[1][j] - G[0][j] * G[1][i];
            const double em = gam(2) * (fabs(G[0][i] * G[1][j]) + fabs(G[0][j] * G[1][i])) + fabs(G[1][j]) * eG[0][i] +
                              fabs(G[0][i]) * eG[1][j] + fabs(G[1][i]) * eG[0][j] + fabs(G[0][j]) * eG[1][i];
            dg += m * m;
            edg += 2.0 * fabs(m) * em;
        }
        edg += gam(3) * dg;
        edet = edg + DILATION * (ea1 + ec1) + gam(3) * det + 1.2e-8 * (sa + sc1) + 3.6e-9;
        /* conic = (c, -b, a) / det: a reciprocal and a product, errors direct */
        const double rd = edet / det + 2.0 * U32;
        o->eA = fabs(o->conic[0]) * (e2[2] / c + rd);
        o->eB = fabs(o->conic[1]) * rd + e2[1] / det;
        o->eC = fabs(o->conic[2]) * (e2[0] / a + rd);
    } else {
        /* a given covariance is exact; a posed one (A3 Sigma A3^T in FP32 from
         * the FP32 Sigma of its scales and rotation, A3 a blend of rotations)
         * within 240U tr(Sigma).  Sigma2 = T Sigma T^T + 0.3 I: u = Sigma t
         * (three roundings), a = t . u + 0.3 (four) */
        double eS[9];
        const double tr = S[0] + S[4] + S[8];
        for (int i = 0; i < 9; ++i) eS[i] = inexact ? 240.0 * U32 * tr : 0.0;
        double uu[2][3], eu[2][3];
        for (int r = 0; r < 2; ++r)
            for (int i = 0; i < 3; ++i) {
                double v = 0.0, m = 0.0, e = 0.0;
                for (int j = 0; j < 3; ++j) {
                    v += S[3 * i + j] * T[3 * r + j];
                    m += fabs(S[3 * i + j] * T[3 * r + j]);
                    e += eS[3 * i + j] * fabs(T[3 * r + j]) + fabs(S[3 * i + j]) * et[3 * r + j];
                }
                uu[r][i] = v;
                eu[r][i] = gam(3) * m + e;
            }
        for (int x = 0; x < 3; ++x) {
            const int r = x == 2 ? 1 : 0, w = x == 0 ? 0 : 1; /* a = t0 . u0, b = t0 . u1, c = t1 . u1 */
            double m = 0.0, e = 0.0;
            for (int i = 0; i < 3; ++i) {
                m += fabs(T[3 * r + i] * uu[w][i]);
                e += fabs(T[3 * r + i]) * eu[w][i] + et[3 * r + i] * fabs(uu[w][i]);
            }
            e2[x] = x == 1 ? gam(3) * m + e : gam(4) * (m + DILATION) + e + 1.2e-8;
        }
        edet = fabs(c) * e2[0] + fabs(a) * e2[2] + 2.0 * fabs(b) * e2[1] + gam(2) * (fabs(a * c) + b * b);
        /* det = a c - b b from the rounded a, b, c: an error dSigma2 moves Q =
         * Sigma2^-1 by -Q dSigma2 Q (first order) and the power by (Qd)^T
         * dSigma2 (Qd) / 2; the conic's own roundings (det under either FMA
         * contraction within U (ac + b^2) + U det, the reciprocal, the
         * product) add rel_conic relative */
        o->ea = e2[0]; o->eb = e2[1]; o->ec = e2[2];
        o->rel_conic = det > 0.0 ? U32 * (fabs(a * c) + b * b) / det + 3.0 * U32 : 0.0;
        const double Q[4] = {o->conic[0], o->conic[1], o->conic[1], o->conic[2]};
        const double E[4] = {e2[0], e2[1], e2[1], e2[2]};
        double eq[3] = {0.0, 0.0, 0.0}; /* |Q| |dSigma2| |Q| at (0,0), (0,1), (1,1) */
        const int ri[3] = {0, 0, 1}, ci[3] = {0, 1, 1};
        for (int x = 0; x < 3; ++x)
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) eq[x] += fabs(Q[2 * ri[x] + i]) * E[2 * i + j] * fabs(Q[2 * j + ci[x]]);
        o->eA = eq[0] + fabs(o->conic[0]) * o->rel_conic;
        o->eB = eq[1] + fabs(o->conic[1]) * o->rel_conic;
        o->eC = eq[2] + fabs(o->conic[2]) * o->rel_conic;
        (void)edet;
    }
    /* radius: lambda = mid + sqrt(max(0.1, hd^2 + b^2)), mid = (a + c) / 2,
     * hd = (a - c) / 2 (one rounding each), the discriminant two roundings;
     * |hd|, |b| <= sqrt(disc), so the input errors pass without amplification */
    const double mid = 0.5 * (a + c), hd = 0.5 * (a - c);
    const double emid = 0.5 * (e2[0] + e2[2]) + U32 * mid;
    const double ehd = 0.5 * (e2[0] + e2[2]) + U32 * fabs(hd);
    const double disc = hd * hd + b * b;
    const double edisc = 2.0 * fabs(hd) * ehd + 2.0 * fabs(b) * e2[1] + U32 * hd * hd + U32 * disc;
    const double xm = disc > 0.1 ? disc : 0.1;
    double esq;
    if (disc - edisc > 0.1) esq = edisc / (2.0 * sqrt(xm)) + U32 * sqrt(xm);
    else if (disc + edisc < 0.1) esq = U32 * sqrt(0.1) + 2.4e-9; /* sqrt(0.1f), 0.1f - 0.1 = 1.5e-9 */
    else esq = edisc / (2.0 * sqrt(0.1)) + U32 * sqrt(xm) + 2.4e-9;
    const double lam = mid + sqrt(xm);
    const double elam = emid + esq + U32 * lam;
    o->er3 = 1.5 * elam / sqrt(lam) + gam(2) * o->r3;
}

/* Returns 0 when the Gaussian is culled by the near plane or a singular conic. */
static int project_one(const double *mu, const double *ls, const double *q, double ologit, const double *sh,
                       const double *cov3d, int inexact, const cam_t *k, int W, int H, double near_plane, proj_t *o,
                       const double *dirmat)
{
    memset(o, 0, sizeof(*o));
    memcpy(o->mu, mu, 3 * sizeof(double));
    o->zkey = depth_key(mu, k);
    if (!(o->zkey > (float)near_plane)) return 0;
    for (int i = 0; i < 3; ++i) o->d[i] = mu[i] - k->C[i];
    for (int r = 0; r < 3; ++r) o->p[r] = k->R[3 * r] * o->d[0] + k->R[3 * r + 1] * o->d[1] + k->R[3 * r + 2] * o->d[2];
    double px = o->p[0], py = o->p[1], pz = o->p[2];
    if (cov3d) {
        double *S = o->Sigma;
        S[0] = cov3d[0]; S[1] = cov3d[1]; S[2] = cov3d[2];
        S[3] = cov3d[1]; S[4] = cov3d[3]; S[5] = cov3d[4];
        S[6] = cov3d[2]; S[7] = cov3d[4]; S[8] = cov3d[5];
    } else {
        cov_from_scale_rot(ls, q, o->Sigma);
    }
    o->u = k->fx * px / pz + k->cx;
    o->v = k->fy * py / pz + k->cy;
    /* EWA Jacobian with the lateral clamp (1.3 x the half field of view) */
    double limx = 1.3 * (0.5 * W / k->fx), limy = 1.3 * (0.5 * H / k->fy);
    double tx = px / pz, ty = py / pz;
    o->clampx = (tx < -limx || tx > limx);
    o->clampy = (ty < -limy || ty > limy);
    if (tx < -limx) tx = -limx;
    if (tx > limx) tx = limx;
    if (ty < -limy) ty = -limy;
    if (ty > limy) ty = limy;
    o->tx = tx; o->ty = ty;
    double *J = o->J; /* 2x3 row-major */
    J[0] = k->fx / pz; J[1] = 0.0; J[2] = -k->fx * tx / pz;
    J[3] = 0.0; J[4] = k->fy / pz; J[5] = -k->fy * ty / pz;
    double *T = o->T; /* T = J W */
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) T[3 * r + c] = J[3 * r] * k->R[c] + J[3 * r + 1] * k->R[3 + c] + J[3 * r + 2] * k->R[6 + c];
    double TS[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            TS[3 * r + c] = T[3 * r] * o->Sigma[c] + T[3 * r + 1] * o->Sigma[3 + c] + T[3 * r + 2] * o->Sigma[6 + c];
    double s00 = TS[0] * T[0] + TS[1] * T[1] + TS[2] * T[2];
    double s01 = TS[0] * T[3] + TS[1] * T[4] + TS[2] * T[5];
    double s11 = TS[3] * T[3] + TS[4] * T[4] + TS[5] * T[5];
    double a = s00 + DILATION, b = s01, c = s11 + DILATION;
    o->cov2[0] = a; o->cov2[1] = b; o->cov2[2] = c;
    double det = a * c - b * b;
    o->det = det;
    if (!(det > 0.0)) return 0;
    o->conic[0] = c / det; o->conic[1] = -b / det; o->conic[2] = a / det;
    double mid = 0.5 * (a + c);
    double disc = mid * mid - det;
    if (disc < 0.1) disc = 0.1;
    double lam = mid + sqrt(disc);
    o->r3 = 3.0 * sqrt(lam);
    o->r = (int32_t)ceil(o->r3);
    /* FP32 error bounds of what the CUDA path computes in single precision */
    fp32_bounds(o, ls, q, cov3d != NULL, inexact, k);
    /* FP32 can round 3 sqrt(lambda) to the other side of an integer */
    double k3 = floor(o->r3 + 0.5);
    if (fabs(o->r3 - k3) <= o->er3 && k3 >= 1.0) {
        o->r_lo = (int32_t)k3;
        o->r_hi = (int32_t)k3 + 1;
    } else {
        o->r_lo = o->r_hi = o->r;
    }
    o->cand = footprint_on_image(o->u, o->v, o->r_hi, W, H);
    o->visible = footprint_on_image(o->u, o->v, o->r, W, H);
    if (!o->cand) return 0;
    o->opacity = 1.0 / (1.0 + exp(-ologit));
    /* SH direction: the unit view direction, or -- for a posed avatar
     * Gaussian evaluated in its canonical frame -- M (mu - C) normalised,
     * M the inverse of the skinning matrix's linear part */
    double dv3[3];
    if (dirmat) {
        for (int r = 0; r < 3; ++r)
            dv3[r] = dirmat[3 * r] * o->d[0] + dirmat[3 * r + 1] * o->d[1] + dirmat[3 * r + 2] * o->d[2];
    } else {
        for (int r = 0; r < 3; ++r) dv3[r] = o->d[r];
    }
    double dn = sqrt(dv3[0] * dv3[0] + dv3[1] * dv3[1] + dv3[2] * dv3[2]);
    o->dnorm = dn;
    for (int i = 0; i < 3; ++i) o->dir[i] = dv3[i] / dn;
    double Y[16];
    sh_eval(o->dir, Y, NULL);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int kk = 0; kk < 16; ++kk) acc += Y[kk] * sh[3 * kk + ch];
        acc += 0.5;
        o->raw[ch] = acc;
        o->rgb[ch] = acc < 0.0 ? 0.0 : acc;
    }
    return 1;
}

/* Exported per-Gaussian projection (one view). */
int64_t or_project(int64_t n, const double *means, const double *log_scales, const double *quats, const double *ologits,
                   const double *sh, const double *cov3d, const uint8_t *use_cov, const uint8_t *inexact,
                   const double *dirmat, const double *cam,
                   int32_t W, int32_t H, double near_plane, int32_t *visible, double *u, double *v, double *z, float *zkey,
                   double *cov2, double *conic, double *opacity, double *rgb, int32_t *radius, double *r3,
                   double *err)
{
    cam_t k;
    load_cam(cam, &k);
    int64_t nvis = 0;
#pragma omp parallel for schedule(static) reduction(+ : nvis)
    for (int64_t g = 0; g < n; ++g) {
        proj_t o;
        const double *cv = (cov3d && use_cov && use_cov[g]) ? cov3d + 6 * g : NULL;
        int ok = project_one(means + 3 * g, log_scales + 3 * g, quats + 4 * g, ologits[g], sh + 48 * g, cv,
                             inexact ? inexact[g] : 0, &k, W, H, near_plane, &o, dirmat ? dirmat + 9 * g : NULL);
        int vis = ok && o.visible;
        visible[g] = vis;
        nvis += vis;
        u[g] = o.u; v[g] = o.v; z[g] = o.p[2]; zkey[g] = o.zkey;
        for (int i = 0; i < 3; ++i) {
            cov2[3 * g + i] = o.cov2[i];
            conic[3 * g + i] = o.conic[i];
            rgb[3 * g + i] = o.rgb[i];
        }
        opacity[g] = o.opacity;
        radius[g] = o.r;
        r3[g] = o.r3;
        if (err) { /* FP32 error bounds: u, v, 3 sqrt(lambda), conic A, B, C */
            const double e6[6] = {o.du, o.dv, o.er3, o.eA, o.eB, o.eC};
            for (int i = 0; i < 6; ++i) err[6 * g + i] = e6[i];
        }
    }
    return nvis;
}

/* ------------------------------------------------------------------------ */
/* Per-pixel front-to-back blending step.  The pixel-major and the           */
/* Gaussian-major loops both call this one function, in the same per-pixel    */
/* order, so their results agree bit for bit.                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
    double u, v, z, A, B, C, o, rgb[3], du, dv, ez;
    /* FP32 error model of the conic: direct bounds eA, eB, eC (factor-form
     * Gaussians), or the 2D covariance's errors ea, eb, ec with the conic's own
     * relative rounding rel_conic (Gaussians given by a covariance) */
    double eA, eB, eC, ea, eb, ec, rel_conic;
    int32_t r, r_lo, r_hi;
    float zkey;
    uint8_t inexact;
    int64_t idx;
} cand_t;

typedef struct {
    double T, C[3], D, relT;
    int32_t ncov, n, ncov_last, last, done;
    float prev_zkey;
    double prev_ez;
    int32_t have_prev, prev_inexact;
    uint8_t amb;
    int64_t evals;
} pix_t;

static void pix_init(pix_t *s)
{
    memset(s, 0, sizeof(*s));
    s->T = 1.0;
}

static double maxabs3(const double *c)
{
    double m = fabs(c[0]);
    if (fabs(c[1]) > m) m = fabs(c[1]);
    if (fabs(c[2]) > m) m = fabs(c[2]);
    return m;
}

static void blend_step(pix_t *s, const cand_t *g, int i, int j, int32_t pos)
{
    if (s->done) return;
    double dx = g->u - (double)i, dy = g->v - (double)j;
    double m = fabs(dx) > fabs(dy) ? fabs(dx) : fabs(dy);
    /* FP32 offsets: (u - cx) - (i - cx), i - cx exact, one rounding */
    const double edx = g->du + U32 * fabs(dx), edy = g->dv + U32 * fabs(dy);
    double eps = edx > edy ? edx : edy;
    if (m > g->r_hi + eps) return;
    double q = g->A * dx * dx + g->C * dy * dy;
    double power = -0.5 * q - g->B * dx * dy;
    /* power in FP32: three roundings on each term; the offsets' errors
     * through dpower/dd = -Q d = -w; the conic's errors directly (factor form)
     * or as the 2D covariance's through (w^T dSigma2 w) / 2 plus the conic's
     * own rounding; 1e-9 for second-order terms */
    const double wx = g->A * dx + g->B * dy, wy = g->B * dx + g->C * dy;
    double dpow = fabs(wx) * edx + fabs(wy) * edy + (gam(3) + g->rel_conic) * (0.5 * q + fabs(g->B * dx * dy)) +
                  0.5 * (g->ea * wx * wx + 2.0 * g->eb * fabs(wx * wy) + g->ec * wy * wy) +
                  0.5 * (g->eA * dx * dx + g->eC * dy * dy) + g->eB * fabs(dx * dy) + 1e-9;
    if (m >= g->r_lo - eps && m <= g->r_hi + eps) {
        /* coverage can flip under FP32 rounding of u, v or of the radius */
        s->amb |= AMB_COUNT | AMB_FOOTPRINT;
        if (power <= dpow && g->o * exp(power) >= ALPHA_MIN * (1.0 - 1e-3)) s->amb |= AMB_VALUE;
    }
    if (m > (double)g->r) return;
    if (s->have_prev && (g->inexact || s->prev_inexact)) {
        float lo = s->prev_zkey < g->zkey ? s->prev_zkey : g->zkey;
        float hi = s->prev_zkey < g->zkey ? g->zkey : s->prev_zkey;
        if ((double)hi - (double)lo <= s->prev_ez + g->ez) s->amb |= AMB_VALUE | AMB_COUNT | AMB_ORDER;
    }
    s->have_prev = 1;
    s->prev_zkey = g->zkey;
    s->prev_inexact = g->inexact;
    s->prev_ez = g->ez;
    s->ncov += 1;
    s->evals += 1;
    /* power <= 0 decision (a positive FP32 power skips the pair) */
    if (fabs(power) <= dpow && g->o >= ALPHA_MIN) s->amb |= AMB_COUNT | AMB_VALUE;
    if (power > 0.0) return;
    double G = exp(power);
    double a_raw = g->o * G;
    double alpha = a_raw < ALPHA_MAX ? a_raw : ALPHA_MAX;
    double cmax = maxabs3(g->rgb) + 1.0;
    /* alpha >= 1/255 decision: ln alpha in FP32 is off by at most dpow plus
     * E_ALPHA, the relative errors of __expf (2 + floor(1.173 |power|) ulp,
     * at most 8 ulp = 16U on the range where alpha can reach 1/255), of the
     * opacity (expf, an add and a division: 6U), of their product (U) and of
     * the FP32 threshold constants (U) */
    if (fabs(power + log(g->o) - log(ALPHA_MIN)) <= dpow + E_ALPHA) {
        s->amb |= AMB_COUNT | AMB_ALPHA;
        if (ALPHA_MIN * s->T * cmax > 0.5e-4 || ALPHA_MIN * s->T * g->z > 0.5e-4 * (s->D + ALPHA_MIN * s->T * g->z))
            s->amb |= AMB_VALUE;
    }
    if (alpha < ALPHA_MIN) return;
    /* alpha = min(0.99, .) decision: same error bound as the 1/255 test */
    if (fabs(power + log(g->o) - log(ALPHA_MAX)) <= dpow + E_ALPHA) s->amb |= AMB_CLAMP;
    double Tn = s->T * (1.0 - alpha);
    /* relative FP32 error of T: two roundings per step (1 - alpha, the
     * product), alpha's own error through alpha / (1 - alpha), and at the
     * clamp the FP32 constant: 1 - 0.99f = 0.0099999905 (16.1U off 0.01) */
    double relTn = s->relT + gam(2) +
                   (a_raw < ALPHA_MAX ? alpha / (1.0 - alpha) * (dpow + E_ALPHA) : 16.1 * U32);
    /* T (1 - alpha) < 1e-4 decision (1e-4f is within U/2 of 1e-4) */
    if (fabs(Tn - T_STOP) <= T_STOP * (relTn + U32) + 1e-15) {
        s->amb |= AMB_COUNT | AMB_STOP;
        double ec = alpha * s->T * (maxabs3(g->rgb) + 1e-30);
        double ed = alpha * s->T * g->z;
        if (ec > 0.5e-4 || ed > 0.5e-4 * (s->D + ed)) s->amb |= AMB_VALUE;
    }
    if (Tn < T_STOP) {
        s->done = 1;
        return;
    }
    double w = alpha * s->T;
    s->C[0] += g->rgb[0] * w;
    s->C[1] += g->rgb[1] * w;
    s->C[2] += g->rgb[2] * w;
    s->D += g->z * w;
    s->T = Tn;
    s->relT = relTn;
    s->n += 1;               /* n_contrib: Gaussians blended into this pixel */
    s->ncov_last = s->ncov;  /* covered Gaussians up to and including this one */
    s->last = pos + 1;
}

/* ------------------------------------------------------------------------ */
/* Candidate list: projected Gaussians whose footprint may touch the image,   */
/* sorted by (FP32 depth key, index).                                          */
/* ------------------------------------------------------------------------ */
static int cand_cmp(const void *a, const void *b)
{
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    if (x->zkey < y->zkey) return -1;
    if (x->zkey > y->zkey) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

static int64_t build_candidates(int64_t n, const double *means, const double *ls, const double *q, const double *ologit,
                                const double *sh, const double *cov3d, const uint8_t *use_cov, const uint8_t *inexact,
                                const double *dirmat, const cam_t *k, int W, int H, double near_plane, cand_t **out)
{
    cand_t *c = (cand_t *)malloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *ok = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < n; ++g) {
        proj_t o;
        const double *cv = (cov3d && use_cov && use_cov[g]) ? cov3d + 6 * g : NULL;
        int inx = inexact ? inexact[g] : 0;
        if (!project_one(means + 3 * g, ls + 3 * g, q + 4 * g, ologit[g], sh + 48 * g, cv, inx, k, W, H, near_plane, &o,
                         dirmat ? dirmat + 9 * g : NULL))
            continue;
        ok[g] = 1;
        cand_t *t = c + g;
        t->u = o.u; t->v = o.v; t->z = o.p[2];
        t->A = o.conic[0]; t->B = o.conic[1]; t->C = o.conic[2];
        t->o = o.opacity;
        for (int i = 0; i < 3; ++i) t->rgb[i] = o.rgb[i];
        t->du = o.du; t->dv = o.dv;
        t->ez = o.ez;
        const int factor = o.rel_conic == 0.0; /* the factor form sets no covariance-error terms */
        t->eA = factor ? o.eA : 0.0; t->eB = factor ? o.eB : 0.0; t->eC = factor ? o.eC : 0.0;
        t->ea = o.ea; t->eb = o.eb; t->ec = o.ec; t->rel_conic = o.rel_conic;
        t->r = o.r; t->r_lo = o.r_lo; t->r_hi = o.r_hi;
        t->zkey = o.zkey;
        t->inexact = (uint8_t)inx;
        t->idx = g;
    }
    int64_t m = 0;
    for (int64_t g = 0; g < n; ++g)
        if (ok[g]) c[m++] = c[g];
    free(ok);
    qsort(c, (size_t)m, sizeof(cand_t), cand_cmp);
    *out = c;
    return m;
}

static void finish_pixel(const pix_t *s, const double *bg, int flags, int64_t p, int64_t HW, double *rgb, double *depth,
                         double *Tout, int32_t *nout, uint8_t *amb, int32_t *last, int32_t *ncov)
{
    for (int ch = 0; ch < 3; ++ch) rgb[ch * HW + p] = s->C[ch] + s->T * bg[ch];
    double D = s->D;
    if (flags & FLAG_NORMALIZE_DEPTH) D = (1.0 - s->T) < 1e-4 ? 0.0 : s->D / (1.0 - s->T);
    depth[p] = D;
    Tout[p] = s->T;
    nout[p] = s->n;
    if (amb) amb[p] = s->amb;
    if (last) last[p] = s->last;
    if (ncov) ncov[p] = s->ncov_last;
}

static int num_threads(int32_t req)
{
#ifdef _OPENMP
    if (req > 0) return req;
    return omp_get_max_threads();
#else
    (void)req;
    return 1;
#endif
}

/* Gaussian-major walk over row bands [0, H): every band walks the whole
 * sorted candidate list and updates only its own pixels. */
static int64_t walk_gaussian_major(const cand_t *c, int64_t m, int W, int H, pix_t *st, int nthreads)
{
    int64_t evals = 0;
    int nb = nthreads > H ? H : nthreads;
    if (nb < 1) nb = 1;
#pragma omp parallel for schedule(static, 1) num_threads(nb) reduction(+ : evals)
    for (int b = 0; b < nb; ++b) {
        int j0 = (int)((int64_t)H * b / nb), j1 = (int)((int64_t)H * (b + 1) / nb);
        for (int64_t k = 0; k < m; ++k) {
            const cand_t *g = c + k;
            double ext = g->r_hi + (g->du > g->dv ? g->du : g->dv) + 1e-6 + 1.0;
            int ilo = (int)floor(g->u - ext), ihi = (int)ceil(g->u + ext);
            int jlo = (int)floor(g->v - ext), jhi = (int)ceil(g->v + ext);
            if (ilo < 0) ilo = 0;
            if (ihi > W - 1) ihi = W - 1;
            if (jlo < j0) jlo = j0;
            if (jhi > j1 - 1) jhi = j1 - 1;
            for (int j = jlo; j <= jhi; ++j)
                for (int i = ilo; i <= ihi; ++i) blend_step(st + (int64_t)j * W + i, g, i, j, (int32_t)k);
        }
        for (int j = j0; j < j1; ++j)
            for (int i = 0; i < W; ++i) evals += st[(int64_t)j * W + i].evals;
    }
    return evals;
}

/* Forward render of one view.  mode 0: pixel-major brute force over all
 * candidates; mode 1: the Gaussian-major walk.  Returns the number of
 * evaluations (covered Gaussians examined before each pixel stopped). */
int64_t or_render(int64_t n, const double *means, const double *log_scales, const double *quats, const double *ologits,
                  const double *sh, const double *cov3d, const uint8_t *use_cov, const uint8_t *inexact,
                  const double *dirmat, const double *cam,
                  int32_t W, int32_t H, double near_plane, const double *bg, int32_t mode, int32_t flags, int32_t nthreads,
                  double *out_rgb, double *out_depth, double *out_T, int32_t *out_n, uint8_t *out_amb, int32_t *out_last,
                  int32_t *out_ncov)
{
    cam_t k;
    load_cam(cam, &k);
    cand_t *c = NULL;
    int64_t m = build_candidates(n, means, log_scales, quats, ologits, sh, cov3d, use_cov, inexact, dirmat, &k, W, H,
                                 near_plane, &c);
    int64_t HW = (int64_t)W * H;
    pix_t *st = (pix_t *)malloc(sizeof(pix_t) * (size_t)HW);
    for (int64_t p = 0; p < HW; ++p) pix_init(st + p);
    int nt = num_threads(nthreads);
    int64_t evals = 0;
    if (mode == 0) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt) reduction(+ : evals)
        for (int64_t p = 0; p < HW; ++p) {
            int i = (int)(p % W), j = (int)(p / W);
            for (int64_t kk = 0; kk < m; ++kk) blend_step(st + p, c + kk, i, j, (int32_t)kk);
            evals += st[p].evals;
        }
    } else {
        evals = walk_gaussian_major(c, m, W, H, st, nt);
    }
    for (int64_t p = 0; p < HW; ++p)
        finish_pixel(st + p, bg, flags, p, HW, out_rgb, out_depth, out_T, out_n, out_amb, out_last, out_ncov);
    free(st);
    free(c);
    return evals;
}

/* ------------------------------------------------------------------------ */
/* Adjoint (FP64).  Discrete decisions (cull, radius, footprint, skip, stop)  */
/* are held at their forward values; the 0.99 clamp and the colour clamp at  */
/* zero pass the true derivative, which is zero where they are active.        */
/* ------------------------------------------------------------------------ */
typedef struct {
    double gu, gv, gA, gB, gC, go, grgb[3], gz;
} grec_t;

/* Per-Gaussian chain from the screen-space gradients back to the inputs. */
static void preprocess_vjp(const proj_t *o, const grec_t *gr, const double *ls, const double *q, const double *sh,
                           int use_cov, const cam_t *k, double *g_mu, double *g_ls, double *g_q, double *g_ologit,
                           double *g_sh, double *g_cov3d)
{
    double gp[3] = {0.0, 0.0, 0.0};
    double px = o->p[0], py = o->p[1], pz = o->p[2];
    /* u = fx px/pz + cx, v = fy py/pz + cy; depth uses pz */
    gp[0] += gr->gu * k->fx / pz;
    gp[2] += -gr->gu * k->fx * px / (pz * pz);
    gp[1] += gr->gv * k->fy / pz;
    gp[2] += -gr->gv * k->fy * py / (pz * pz);
    gp[2] += gr->gz;
    /* conic = (c, -b, a) / det of the dilated 2D covariance (a, b, c) */
    double a = o->cov2[0], b = o->cov2[1], c = o->cov2[2], det = o->det, d2 = det * det;
    double ga = gr->gA * (-c * c / d2) + gr->gB * (b * c / d2) + gr->gC * (-b * b / d2);
    double gb = gr->gA * (2.0 * b * c / d2) + gr->gB * (-(a * c + b * b) / d2) + gr->gC * (2.0 * a * b / d2);
    double gc = gr->gA * (-b * b / d2) + gr->gB * (a * b / d2) + gr->gC * (-a * a / d2);
    double G2[4] = {ga, 0.5 * gb, 0.5 * gb, gc};
    const double *T = o->T, *S = o->Sigma;
    /* dL/dSigma = T^T G2 T ; dL/dT = 2 G2 T Sigma */
    double gS[9];
    for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) {
            double acc = 0.0;
            for (int x = 0; x < 2; ++x)
                for (int y = 0; y < 2; ++y) acc += T[3 * x + r] * G2[2 * x + y] * T[3 * y + cc];
            gS[3 * r + cc] = acc;
        }
    double GT[6];
    for (int x = 0; x < 2; ++x)
        for (int cc = 0; cc < 3; ++cc) GT[3 * x + cc] = G2[2 * x] * T[cc] + G2[2 * x + 1] * T[3 + cc];
    double gT[6];
    for (int x = 0; x < 2; ++x)
        for (int cc = 0; cc < 3; ++cc) {
            double acc = 0.0;
            for (int kk = 0; kk < 3; ++kk) acc += GT[3 * x + kk] * S[3 * kk + cc];
            gT[3 * x + cc] = 2.0 * acc;
        }
    /* T = J W -> dL/dJ = dL/dT W^T */
    double gJ[6];
    for (int x = 0; x < 2; ++x)
        for (int cc = 0; cc < 3; ++cc)
            gJ[3 * x + cc] = gT[3 * x] * k->R[3 * cc] + gT[3 * x + 1] * k->R[3 * cc + 1] + gT[3 * x + 2] * k->R[3 * cc + 2];
    /* J00 = fx/pz, J02 = -fx tx/pz (tx = px/pz unless clamped), J11, J12 alike */
    gp[2] += gJ[0] * (-k->fx / (pz * pz));
    gp[2] += gJ[4] * (-k->fy / (pz * pz));
    if (!o->clampx) {
        gp[0] += gJ[2] * (-k->fx / (pz * pz));
        gp[2] += gJ[2] * (2.0 * k->fx * px / (pz * pz * pz));
    } else {
        gp[2] += gJ[2] * (k->fx * o->tx / (pz * pz));
    }
    if (!o->clampy) {
        gp[1] += gJ[5] * (-k->fy / (pz * pz));
        gp[2] += gJ[5] * (2.0 * k->fy * py / (pz * pz * pz));
    } else {
        gp[2] += gJ[5] * (k->fy * o->ty / (pz * pz));
    }
    /* p = W d -> dL/dd = W^T dL/dp */
    double gd[3];
    for (int cc = 0; cc < 3; ++cc) gd[cc] = k->R[cc] * gp[0] + k->R[3 + cc] * gp[1] + k->R[6 + cc] * gp[2];
    /* colour: rgb = max(0, sum Y(dir) k + 0.5), dir = d / |d| */
    double Y[16], dY[16][3];
    sh_eval(o->dir, Y, dY);
    double gdir[3] = {0.0, 0.0, 0.0};
    for (int ch = 0; ch < 3; ++ch) {
        double g = o->raw[ch] < 0.0 ? 0.0 : gr->grgb[ch];
        if (g == 0.0) continue;
        for (int kk = 0; kk < 16; ++kk) {
            g_sh[3 * kk + ch] += Y[kk] * g;
            double w = sh[3 * kk + ch] * g;
            gdir[0] += dY[kk][0] * w;
            gdir[1] += dY[kk][1] * w;
            gdir[2] += dY[kk][2] * w;
        }
    }
    double dot = gdir[0] * o->dir[0] + gdir[1] * o->dir[1] + gdir[2] * o->dir[2];
    for (int cc = 0; cc < 3; ++cc) gd[cc] += (gdir[cc] - o->dir[cc] * dot) / o->dnorm;
    for (int cc = 0; cc < 3; ++cc) g_mu[cc] += gd[cc];
    /* covariance */
    if (use_cov) {
        if (g_cov3d) {
            g_cov3d[0] += gS[0];
            g_cov3d[1] += gS[1] + gS[3];
            g_cov3d[2] += gS[2] + gS[6];
            g_cov3d[3] += gS[4];
            g_cov3d[4] += gS[5] + gS[7];
            g_cov3d[5] += gS[8];
        }
    } else {
        cov_from_scale_rot_vjp(ls, q, gS, g_ls, g_q);
    }
    /* opacity = sigmoid(logit) */
    *g_ologit += gr->go * o->opacity * (1.0 - o->opacity);
}

/* Backward of one view: dL/d(inputs) for L = <d_rgb, rgb> + <d_depth, depth>.
 * Gradients are accumulated (+=).  The raw (unnormalised) depth is assumed. */
int32_t or_render_backward(int64_t n, const double *means, const double *log_scales, const double *quats,
                           const double *ologits, const double *sh, const double *cov3d, const uint8_t *use_cov,
                           const double *cam, int32_t W, int32_t H, double near_plane, const double *bg,
                           const double *d_rgb, const double *d_depth, double *g_means, double *g_log_scales,
                           double *g_quats, double *g_ologits, double *g_sh, double *g_cov3d)
{
    cam_t k;
    load_cam(cam, &k);
    cand_t *c = NULL;
    int64_t m = build_candidates(n, means, log_scales, quats, ologits, sh, cov3d, use_cov, NULL, NULL, &k, W, H,
                                 near_plane, &c);
    int64_t HW = (int64_t)W * H;
    pix_t *st = (pix_t *)malloc(sizeof(pix_t) * (size_t)HW);
    for (int64_t p = 0; p < HW; ++p) pix_init(st + p);
    walk_gaussian_major(c, m, W, H, st, 1);
    /* reverse walk: T is rebuilt by division, S accumulates what lies behind */
    double *Tc = (double *)malloc(sizeof(double) * (size_t)HW);
    double *Sc = (double *)malloc(sizeof(double) * (size_t)HW * 4);
    for (int64_t p = 0; p < HW; ++p) {
        Tc[p] = st[p].T;
        for (int ch = 0; ch < 3; ++ch) Sc[4 * p + ch] = st[p].T * bg[ch];
        Sc[4 * p + 3] = 0.0;
    }
    grec_t *gr = (grec_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(grec_t));
    for (int64_t kk = m - 1; kk >= 0; --kk) {
        const cand_t *g = c + kk;
        grec_t *q = gr + kk;
        int r = g->r;
        int ilo = (int)ceil(g->u - r) - 1, ihi = (int)floor(g->u + r) + 1;
        int jlo = (int)ceil(g->v - r) - 1, jhi = (int)floor(g->v + r) + 1;
        if (ilo < 0) ilo = 0;
        if (ihi > W - 1) ihi = W - 1;
        if (jlo < 0) jlo = 0;
        if (jhi > H - 1) jhi = H - 1;
        for (int j = jlo; j <= jhi; ++j)
            for (int i = ilo; i <= ihi; ++i) {
                int64_t p = (int64_t)j * W + i;
                if (kk >= st[p].last) continue;
                double dx = g->u - i, dy = g->v - j;
                if (fabs(dx) > r || fabs(dy) > r) continue;
                double power = -0.5 * (g->A * dx * dx + g->C * dy * dy) - g->B * dx * dy;
                if (power > 0.0) continue;
                double G = exp(power);
                double a_raw = g->o * G;
                double alpha = a_raw < ALPHA_MAX ? a_raw : ALPHA_MAX;
                if (alpha < ALPHA_MIN) continue;
                double Ti = Tc[p] / (1.0 - alpha);
                double w = alpha * Ti;
                double gal = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    double dl = d_rgb[ch * HW + p];
                    q->grgb[ch] += w * dl;
                    gal += dl * (g->rgb[ch] * Ti - Sc[4 * p + ch] / (1.0 - alpha));
                    Sc[4 * p + ch] += g->rgb[ch] * w;
                }
                double dd = d_depth[p];
                q->gz += w * dd;
                gal += dd * (g->z * Ti - Sc[4 * p + 3] / (1.0 - alpha));
                Sc[4 * p + 3] += g->z * w;
                Tc[p] = Ti;
                if (a_raw < ALPHA_MAX) {
                    q->go += gal * G;
                    double gpow = gal * alpha;
                    q->gu += gpow * (-(g->A * dx + g->B * dy));
                    q->gv += gpow * (-(g->C * dy + g->B * dx));
                    q->gA += gpow * (-0.5 * dx * dx);
                    q->gC += gpow * (-0.5 * dy * dy);
                    q->gB += gpow * (-dx * dy);
                }
            }
    }
    for (int64_t kk = 0; kk < m; ++kk) {
        int64_t g = c[kk].idx;
        proj_t o;
        int uc = (cov3d && use_cov && use_cov[g]) ? 1 : 0;
        project_one(means + 3 * g, log_scales + 3 * g, quats + 4 * g, ologits[g], sh + 48 * g, uc ? cov3d + 6 * g : NULL, 0,
                    &k, W, H, near_plane, &o, NULL);
        preprocess_vjp(&o, gr + kk, log_scales + 3 * g, quats + 4 * g, sh + 48 * g, uc, &k, g_means + 3 * g,
                       g_log_scales + 3 * g, g_quats + 4 * g, g_ologits + g, g_sh + 48 * g,
                       g_cov3d ? g_cov3d + 6 * g : NULL);
    }
    free(gr);
    free(Sc);
    free(Tc);
    free(st);
    free(c);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Linear blend skinning (Sec. 3.3): A = sum_k w_k G[j_k] (3x4),              */
/* mu' = A3 mu_c + a, Sigma' = A3 Sigma_c A3^T with Sigma_c from (s, q).      */
/* Weights are used as given (no renormalisation).                            */
/* ------------------------------------------------------------------------ */
static void blend_joints(const int32_t *ids, const double *w, const double *Gav, double A[12])
{
    memset(A, 0, 12 * sizeof(double));
    for (int kk = 0; kk < 4; ++kk) {
        const double *Gj = Gav + 12 * ids[kk];
        for (int e = 0; e < 12; ++e) A[e] += w[kk] * Gj[e];
    }
}

/* The blended skinning matrices A = sum_k w_k G[avatar][j_k] (3x4 each). */
void or_lbs_matrices(int64_t m, const int32_t *joint_ids, const double *weights, const int32_t *avatar_of,
                     const double *G, int32_t n_joints, double *out_A)
{
    for (int64_t g = 0; g < m; ++g)
        blend_joints(joint_ids + 4 * g, weights + 4 * g, G + (int64_t)12 * n_joints * avatar_of[g], out_A + 12 * g);
}

void or_lbs(int64_t m, const double *means_c, const double *log_scales_c, const double *quats_c, const int32_t *joint_ids,
            const double *weights, const int32_t *avatar_of, const double *G, int32_t n_joints, double *out_means,
            double *out_cov)
{
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < m; ++g) {
        double A[12];
        blend_joints(joint_ids + 4 * g, weights + 4 * g, G + (int64_t)12 * n_joints * avatar_of[g], A);
        const double *mu = means_c + 3 * g;
        for (int r = 0; r < 3; ++r) out_means[3 * g + r] = A[4 * r] * mu[0] + A[4 * r + 1] * mu[1] + A[4 * r + 2] * mu[2] + A[4 * r + 3];
        double S[9];
        cov_from_scale_rot(log_scales_c + 3 * g, quats_c + 4 * g, S);
        double AS[9], P[9];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) AS[3 * r + cc] = A[4 * r] * S[cc] + A[4 * r + 1] * S[3 + cc] + A[4 * r + 2] * S[6 + cc];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) P[3 * r + cc] = AS[3 * r] * A[4 * cc] + AS[3 * r + 1] * A[4 * cc + 1] + AS[3 * r + 2] * A[4 * cc + 2];
        double *o = out_cov + 6 * g;
        o[0] = P[0]; o[1] = P[1]; o[2] = P[2]; o[3] = P[4]; o[4] = P[5]; o[5] = P[8];
    }
}

void or_lbs_backward(int64_t m, const double *means_c, const double *log_scales_c, const double *quats_c,
                     const int32_t *joint_ids, const double *weights, const int32_t *avatar_of, const double *G,
                     int32_t n_joints, const double *g_means, const double *g_cov, double *g_means_c,
                     double *g_log_scales_c, double *g_quats_c, double *g_G)
{
    for (int64_t g = 0; g < m; ++g) {
        const double *Gav = G + (int64_t)12 * n_joints * avatar_of[g];
        double A[12];
        blend_joints(joint_ids + 4 * g, weights + 4 * g, Gav, A);
        const double *mu = means_c + 3 * g;
        const double *gm = g_means + 3 * g, *gc = g_cov + 6 * g;
        double S[9];
        cov_from_scale_rot(log_scales_c + 3 * g, quats_c + 4 * g, S);
        double Gs[9] = {gc[0], 0.5 * gc[1], 0.5 * gc[2], 0.5 * gc[1], gc[3], 0.5 * gc[4], 0.5 * gc[2], 0.5 * gc[4], gc[5]};
        /* dL/dA3 = gm mu^T + 2 Gs A3 S ; dL/da = gm */
        double gA[12];
        for (int r = 0; r < 3; ++r) {
            for (int cc = 0; cc < 3; ++cc) {
                double acc = 0.0;
                for (int x = 0; x < 3; ++x)
                    for (int y = 0; y < 3; ++y) acc += Gs[3 * r + x] * A[4 * x + y] * S[3 * y + cc];
                gA[4 * r + cc] = gm[r] * mu[cc] + 2.0 * acc;
            }
            gA[4 * r + 3] = gm[r];
        }
        /* dL/dmu_c = A3^T gm ; dL/dSigma_c = A3^T Gs A3 */
        for (int cc = 0; cc < 3; ++cc) g_means_c[3 * g + cc] += A[cc] * gm[0] + A[4 + cc] * gm[1] + A[8 + cc] * gm[2];
        double gSc[9];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                double acc = 0.0;
                for (int x = 0; x < 3; ++x)
                    for (int y = 0; y < 3; ++y) acc += A[4 * x + r] * Gs[3 * x + y] * A[4 * y + cc];
                gSc[3 * r + cc] = acc;
            }
        cov_from_scale_rot_vjp(log_scales_c + 3 * g, quats_c + 4 * g, gSc, g_log_scales_c + 3 * g, g_quats_c + 4 * g);
        double *gGav = g_G + (int64_t)12 * n_joints * avatar_of[g];
        for (int kk = 0; kk < 4; ++kk) {
            double *gj = gGav + 12 * joint_ids[4 * g + kk];
            for (int e = 0; e < 12; ++e) gj[e] += weights[4 * g + kk] * gA[e];
        }
    }
}

/* ------------------------------------------------------------------------
 * Nearest-fragment composite (Sec. 3.2, the full-screen pass that merges the
 * 3DGS colour/depth with another layer -- the mesh pass, or the avatars'
 * Gaussian pass): per pixel (C, D) = (D_a < D_b) ? (C_a, D_a) : (C_b, D_b).
 * Reading: a depth that is not a positive finite number marks a pixel the
 * layer does not cover and compares as +infinity, so the formula's else branch
 * also decides when neither layer covers the pixel.
 * rgb [V,3,H,W], depth [V,H,W].
 * ------------------------------------------------------------------------ */
static double layer_depth(double d) { return (d > 0.0 && d <= DBL_MAX) ? d : INFINITY; }

void or_composite_nearest(int64_t n_views, int64_t hw, const double *rgb_a, const double *depth_a, const double *rgb_b,
                          const double *depth_b, double *rgb_out, double *depth_out)
{
    for (int64_t v = 0; v < n_views; ++v)
        for (int64_t p = 0; p < hw; ++p) {
            const int64_t i = v * hw + p;
            const int take_a = layer_depth(depth_a[i]) < layer_depth(depth_b[i]);
            depth_out[i] = take_a ? depth_a[i] : depth_b[i];
            for (int c = 0; c < 3; ++c) {
                const int64_t k = (3 * v + c) * hw + p;
                rgb_out[k] = take_a ? rgb_a[k] : rgb_b[k];
            }
        }
}

/* ------------------------------------------------------------------------
 * Forward kinematics of a joint tree (the per-frame joint matrices the
 * avatar module feeds to LBS, Sec. 3.3.1): for avatar a,
 *   G_0 = [R_root R_0 | t_root],  G_j = G_parent(j) [R_j | J_j - J_parent(j)],
 *   M_j = G_j [I | -J_j]   (the skinning matrix of joint j, 3x4 row-major),
 * with J the rest-pose joint positions and parent(j) < j.
 *   local_rot [A,J,3,3], root [A,3,4] (R_root | t_root), rest [J,3],
 *   parents [J] (parents[0] ignored) -> out [A,J,3,4].
 * ------------------------------------------------------------------------ */
static void mat3_mul(const double *a, const double *b, double *o)
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) o[3 * r + c] = a[3 * r] * b[c] + a[3 * r + 1] * b[3 + c] + a[3 * r + 2] * b[6 + c];
}

void or_forward_kinematics(int32_t n_avatars, int32_t n_joints, const double *local_rot, const double *root,
                           const double *rest, const int32_t *parents, double *out)
{
    double *GR = (double *)malloc((size_t)n_joints * 9 * sizeof(double));
    double *Gt = (double *)malloc((size_t)n_joints * 3 * sizeof(double));
    for (int32_t a = 0; a < n_avatars; ++a) {
        const double *Rl = local_rot + (int64_t)a * n_joints * 9;
        const double *rt = root + 12 * a;
        const double Rr[9] = {rt[0], rt[1], rt[2], rt[4], rt[5], rt[6], rt[8], rt[9], rt[10]};
        mat3_mul(Rr, Rl, GR);
        Gt[0] = rt[3]; Gt[1] = rt[7]; Gt[2] = rt[11];
        for (int32_t j = 1; j < n_joints; ++j) {
            const int32_t p = parents[j];
            mat3_mul(GR + 9 * p, Rl + 9 * j, GR + 9 * j);
            for (int r = 0; r < 3; ++r) {
                double acc = Gt[3 * p + r];
                for (int c = 0; c < 3; ++c) acc += GR[9 * p + 3 * r + c] * (rest[3 * j + c] - rest[3 * p + c]);
                Gt[3 * j + r] = acc;
            }
        }
        for (int32_t j = 0; j < n_joints; ++j) {
            double *M = out + ((int64_t)a * n_joints + j) * 12;
            for (int r = 0; r < 3; ++r) {
                double t = Gt[3 * j + r];
                for (int c = 0; c < 3; ++c) {
                    M[4 * r + c] = GR[9 * j + 3 * r + c];
                    t -= GR[9 * j + 3 * r + c] * rest[3 * j + c];
                }
                M[4 * r + 3] = t;
            }
        }
    }
    free(GR);
    free(Gt);
}

/* ------------------------------------------------------------------------
 * Joint matrices at simulation time (Sec. 3.3.1: the per-frame matrices are
 * interpolated at the current time).  Reading: linear interpolation of the
 * 3x4 matrices of the two frames around the fractional frame position t,
 *   f = clamp(floor(t), 0, F-1), w = clamp(t - f, 0, 1), g = min(f+1, F-1),
 *   M(t) = (1 - w) M_f + w M_g   -- LBS itself blends matrices linearly.
 * frames [A,F,J,12], t [A] -> out [A,J,12].
 * ------------------------------------------------------------------------ */
void or_interpolate_frames(int32_t n_avatars, int32_t n_frames, int32_t n_joints, const double *frames, const double *t,
                           double *out)
{
    for (int32_t a = 0; a < n_avatars; ++a) {
        double tf = t[a];
        double f = floor(tf);
        if (!(f >= 0.0)) f = 0.0;
        if (f > n_frames - 1) f = n_frames - 1;
        double w = tf - f;
        if (!(w >= 0.0)) w = 0.0;
        if (w > 1.0) w = 1.0;
        const int32_t f0 = (int32_t)f, f1 = f0 + 1 < n_frames ? f0 + 1 : n_frames - 1;
        const double *A0 = frames + ((int64_t)a * n_frames + f0) * n_joints * 12;
        const double *A1 = frames + ((int64_t)a * n_frames + f1) * n_joints * 12;
        double *o = out + (int64_t)a * n_joints * 12;
        for (int32_t e = 0; e < n_joints * 12; ++e) o[e] = (1.0 - w) * A0[e] + w * A1[e];
    }
}

/* ------------------------------------------------------------------------
 * Triangle-mesh layer (the mesh pass whose colour and depth the composite of
 * Sec. 3.2 merges with the Gaussian pass).  Reading of a plain z-buffered
 * rasteriser:
 *   q_k = R (P_k - C); a triangle with any q_k.z <= near is culled;
 *   s_k = (fx q.x / q.z + cx, fy q.y / q.z + cy);
 *   pixel (i, j) is covered iff its centre lies inside or on the edge of the
 *   screen triangle (edge functions of one sign with the area, zero allowed);
 *   screen barycentrics l_k, perspective-correct w_k = l_k / z_k,
 *   depth z = 1 / sum w_k, colour = z sum w_k c_k (per-vertex colours);
 *   the smallest depth wins, equal depths keep the lower triangle index.
 * Uncovered pixels get bg and depth 0.  amb flags pixels whose coverage by
 * some triangle, or whose winner, FP32 rounding could change.
 * verts [V,3], colors [V,3], tris [T,3] -> rgb [3,H,W], depth [H,W].
 * ------------------------------------------------------------------------ */
void or_raster_mesh(int64_t n_verts, const double *verts, const double *colors, int64_t n_tris, const int32_t *tris,
                    const double *cam, int32_t W, int32_t H, double near_plane, const double *bg, double *out_rgb,
                    double *out_depth, uint8_t *out_amb)
{
    cam_t k;
    load_cam(cam, &k);
    (void)n_verts;
    const int64_t HW = (int64_t)W * H;
    /* per-triangle screen data */
    double *sx = (double *)malloc((size_t)(n_tris > 0 ? n_tris : 1) * 3 * sizeof(double));
    double *sy = (double *)malloc((size_t)(n_tris > 0 ? n_tris : 1) * 3 * sizeof(double));
    double *sz = (double *)malloc((size_t)(n_tris > 0 ? n_tris : 1) * 3 * sizeof(double));
    uint8_t *live = (uint8_t *)calloc((size_t)(n_tris > 0 ? n_tris : 1), 1);
    for (int64_t t = 0; t < n_tris; ++t) {
        int ok = 1;
        for (int a = 0; a < 3; ++a) {
            const double *P = verts + 3 * tris[3 * t + a];
            double d[3] = {P[0] - k.C[0], P[1] - k.C[1], P[2] - k.C[2]};
            double q[3];
            for (int r = 0; r < 3; ++r) q[r] = k.R[3 * r] * d[0] + k.R[3 * r + 1] * d[1] + k.R[3 * r + 2] * d[2];
            if (!(q[2] > near_plane)) ok = 0;
            sz[3 * t + a] = q[2];
            sx[3 * t + a] = k.fx * q[0] / q[2] + k.cx;
            sy[3 * t + a] = k.fy * q[1] / q[2] + k.cy;
        }
        double area = (sx[3 * t + 1] - sx[3 * t]) * (sy[3 * t + 2] - sy[3 * t]) -
                      (sy[3 * t + 1] - sy[3 * t]) * (sx[3 * t + 2] - sx[3 * t]);
        live[t] = ok && area != 0.0;
    }
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t p = 0; p < HW; ++p) {
        const double px = (double)(p % W), py = (double)(p / W);
        double best = INFINITY, second = INFINITY, col[3] = {bg[0], bg[1], bg[2]};
        uint8_t amb = 0;
        for (int64_t t = 0; t < n_tris; ++t) {
            if (!live[t]) continue;
            const double *X = sx + 3 * t, *Y = sy + 3 * t, *Z = sz + 3 * t;
            const double area = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
            double e[3], scale[3];
            for (int a = 0; a < 3; ++a) {
                const int b = (a + 1) % 3;
                e[a] = (X[b] - X[a]) * (py - Y[a]) - (Y[b] - Y[a]) * (px - X[a]);
                scale[a] = (fabs(X[b] - X[a]) + fabs(Y[b] - Y[a])) * (fabs(px - X[a]) + fabs(py - Y[a]) + 1.0);
            }
            const double sgn = area > 0.0 ? 1.0 : -1.0;
            int inside = 1, near_edge = 0;
            for (int a = 0; a < 3; ++a) {
                if (sgn * e[a] < 0.0) inside = 0;
                /* FP32 screen positions and edge products: a few 1e-7 relative */
                if (fabs(e[a]) <= 1e-5 * scale[a] + 1e-6) near_edge = 1;
            }
            if (near_edge) amb = 1;
            if (!inside) continue;
            /* barycentrics: the edge opposite each vertex over the area */
            const double l0 = e[1] / area, l1 = e[2] / area, l2 = e[0] / area;
            const double w0 = l0 / Z[0], w1 = l1 / Z[1], w2 = l2 / Z[2];
            const double z = 1.0 / (w0 + w1 + w2);
            if (z < best) {
                second = best;
                best = z;
                const int32_t *tv = tris + 3 * t;
                for (int c = 0; c < 3; ++c)
                    col[c] = z * (w0 * colors[3 * tv[0] + c] + w1 * colors[3 * tv[1] + c] + w2 * colors[3 * tv[2] + c]);
            } else if (z < second) {
                second = z;
            }
        }
        if (second - best <= 1e-5 * best) amb = 1;
        for (int c = 0; c < 3; ++c) out_rgb[c * HW + p] = col[c];
        out_depth[p] = best < INFINITY ? best : 0.0;
        out_amb[p] = amb;
    }
    free(sx);
    free(sy);
    free(sz);
    free(live);
}

/* ------------------------------------------------------------------------ */
/* Proxy capsules and the two avatar queries (Sec. 3.3.2, Sec. 3.4).         */
/* A capsule is the set of points within radius rho of the segment [a, b];   */
/* one per joint j: the bone from the posed position of parent(j) to that of */
/* j (the root: a = b, a sphere).  The posed position of joint j is          */
/* M_j [J_j; 1], M_j its skinning matrix and J_j its rest position (the      */
/* skinning matrix maps the rest pose to the posed one).  The agent is a     */
/* sphere of radius r at p; a step moves it from p0 to p1.                    */
/* Capsule rows: (ax, ay, az, rho, bx, by, bz, 0).                            */
/* ------------------------------------------------------------------------ */
void or_avatar_capsules(int32_t n_avatars, int32_t n_joints, const double *M, const double *rest,
                        const int32_t *parents, const double *radius, double *out)
{
    for (int32_t a = 0; a < n_avatars; ++a) {
        for (int32_t j = 0; j < n_joints; ++j) {
            double pj[3], pp[3];
            const int32_t par = parents[j] < 0 ? j : parents[j];
            const double *Mj = M + ((size_t)a * n_joints + j) * 12, *Mp = M + ((size_t)a * n_joints + par) * 12;
            for (int r = 0; r < 3; ++r) {
                pj[r] = Mj[4 * r] * rest[3 * j] + Mj[4 * r + 1] * rest[3 * j + 1] + Mj[4 * r + 2] * rest[3 * j + 2] +
                        Mj[4 * r + 3];
                pp[r] = Mp[4 * r] * rest[3 * par] + Mp[4 * r + 1] * rest[3 * par + 1] +
                        Mp[4 * r + 2] * rest[3 * par + 2] + Mp[4 * r + 3];
            }
            double *o = out + ((size_t)a * n_joints + j) * 8;
            o[0] = pp[0]; o[1] = pp[1]; o[2] = pp[2]; o[3] = radius[j];
            o[4] = pj[0]; o[5] = pj[1]; o[6] = pj[2]; o[7] = 0.0;
        }
    }
}

/* Distance from point p to the segment [a, b]. */
static double point_segment_distance(const double *p, const double *a, const double *b)
{
    double ab[3], ap[3], ll = 0.0, t = 0.0;
    for (int i = 0; i < 3; ++i) {
        ab[i] = b[i] - a[i];
        ap[i] = p[i] - a[i];
        ll += ab[i] * ab[i];
        t += ap[i] * ab[i];
    }
    t = ll > 0.0 ? t / ll : 0.0;
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    double d2 = 0.0;
    for (int i = 0; i < 3; ++i) {
        const double e = ap[i] - t * ab[i];
        d2 += e * e;
    }
    return sqrt(d2);
}

/* Per query q (env query_env[q]): dist = min over the env's capsules of
 * |p0 - segment| - rho, nearest = that capsule's index (the lowest on ties,
 * -1 without capsules); along the step p0 -> p1 the agent sphere first touches
 * a capsule at the smallest t in [0, 1] with |p(t) - segment| <= rho + r:
 * tclip = that t (0 when it starts in contact, 1 when it never touches),
 * blocked = some contact.  f(t) = |p(t) - segment| is convex, so the contact
 * set is an interval: its minimum over [0, 1] (golden-section search) decides
 * contact and bisection on [0, argmin] finds the first t. */
void or_capsule_query(int64_t n_queries, const double *caps, const int64_t *env_cap_off, const int32_t *query_env,
                      const double *p0, const double *p1, double agent_radius, double *out_dist, int32_t *out_nearest,
                      double *out_tclip, uint8_t *out_blocked)
{
    for (int64_t q = 0; q < n_queries; ++q) {
        const int32_t e = query_env[q];
        const double *P0 = p0 + 3 * q, *P1 = p1 ? p1 + 3 * q : p0 + 3 * q;
        double best = INFINITY, tmin = 1.0;
        int32_t arg = -1;
        int blocked = 0;
        for (int64_t c = env_cap_off[e]; c < env_cap_off[e + 1]; ++c) {
            const double *cp = caps + 8 * c;
            const double d = point_segment_distance(P0, cp, cp + 4) - cp[3];
            if (d < best) {
                best = d;
                arg = (int32_t)(c - env_cap_off[e]);
            }
            const double R = cp[3] + agent_radius;
            double pt[3];
#define PT(t) (pt[0] = P0[0] + (t) * (P1[0] - P0[0]), pt[1] = P0[1] + (t) * (P1[1] - P0[1]), \
               pt[2] = P0[2] + (t) * (P1[2] - P0[2]), point_segment_distance(pt, cp, cp + 4))
            if (PT(0.0) <= R) {
                blocked = 1;
                tmin = 0.0;
                continue;
            }
            /* golden-section search for the minimum of the convex f on [0, 1] */
            double lo = 0.0, hi = 1.0;
            const double g = 0.5 * (sqrt(5.0) - 1.0);
            double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo), f1 = PT(x1), f2 = PT(x2);
            for (int it = 0; it < 100; ++it) {
                if (f1 <= f2) {
                    hi = x2; x2 = x1; f2 = f1; x1 = hi - g * (hi - lo); f1 = PT(x1);
                } else {
                    lo = x1; x1 = x2; f1 = f2; x2 = lo + g * (hi - lo); f2 = PT(x2);
                }
            }
            double ts = 0.5 * (lo + hi);
            if (PT(1.0) < PT(ts)) ts = 1.0;
            if (PT(ts) > R) continue;
            /* first crossing: f(0) > R >= f(ts), f decreasing on [0, ts] */
            double a = 0.0, b = ts;
            for (int it = 0; it < 100; ++it) {
                const double m = 0.5 * (a + b);
                if (PT(m) <= R) b = m;
                else a = m;
            }
#undef PT
            blocked = 1;
            if (b < tmin) tmin = b;
        }
        out_dist[q] = arg >= 0 ? best : INFINITY;
        out_nearest[q] = arg;
        if (out_tclip) out_tclip[q] = blocked ? tmin : 1.0;
        if (out_blocked) out_blocked[q] = (uint8_t)blocked;
    }
}

int32_t or_abi_version(void) { return 1; }
