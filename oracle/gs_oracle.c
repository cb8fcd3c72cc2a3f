/*
 * gs_oracle.c -- plain, slow FP64 CPU oracle of the 3D-Gaussian registration
 * hot path of LoopSplat (arXiv 2408.10154).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the CPU
 * baseline leg of bench.py load this library.  The product path (the CUDA
 * library and its Python binding) never loads, calls or links it, and the two
 * share no code, header, table or constant generator.
 *
 * What is computed, and where the paper defines it:
 *   - A submap is a set of Gaussians {mu, Sigma, o, C} (Eq. 1), without
 *     spherical harmonics (end of Sec. 3.3).  Sigma is parameterised by
 *     per-axis log-scales s and a unit quaternion q, Sigma = R(q) S^2 R(q)^T
 *     with S = diag(e^s) (the scale s_k of Eq. 5); o = sigmoid(logit).
 *   - Rigid transform of a submap: mu <- R mu + t, Sigma <- R Sigma R^T
 *     (Eq. 8 / Eq. 9).
 *   - Registration as keyframe localisation (Sec. 3.2): render RGB and depth
 *     of the transformed submap at a keyframe, loss L = L_col + L_depth, both
 *     L1, descended on the rigid transform (rotation and translation, Supp. B,
 *     "3DGS Registration"), learning rates per Supp. B loop-closure table.
 *     The residual eps of each estimate is the loss at the final pose.
 *   - The renderer is the 3D Gaussian splatting forward model the paper builds
 *     on (Sec. 3.2, citing Kerbl et al.); the paper gives no kernel.  It is
 *     restated here from the mathematics: EWA projection with a 2D low-pass
 *     dilation, 16x16 screen tiles, front-to-back alpha compositing.
 *   - Weighted rotation averaging (Eq. 7) is in oracle/__init__.py (numpy).
 *
 * Precision contract.  Every VALUE is computed in FP64 from the FP32 inputs.
 * Every DISCRETE choice -- visibility (near plane, positive determinant),
 * pixel radius and tile rectangle, the depth bits that order the tile lists,
 * skipped contributors (positive exponent, alpha below alpha_min), the alpha
 * clamp, and the transmittance early stop -- is taken in IEEE-754 single
 * precision by the "mirror" below, which follows a fixed operation sequence
 * (round-to-nearest, fmaf only where written, no other contraction; compile
 * with -ffp-contract=off).  The CUDA kernels take the same choices in the
 * same precision, so both sides agree on every integer outcome and differ in
 * values only by rounding.  The mirror's exponential is Cody-Waite range
 * reduction (k = round(x log2 e), r = x - k ln2 with a two-part ln2) followed
 * by the degree-6 Taylor polynomial of e^r and an exact scaling by 2^k.
 */
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_OOM 2

/* ------------------------------------------------------------------------ */
/* options: float opt[11] = {tile, z_near, dilation, alpha_min, alpha_max,    */
/*                            t_min, bg_r, bg_g, bg_b, smooth, tight}         */
/* smooth != 0: every visible Gaussian covers every tile (no radius cull).    */
/* tight != 0: tile rectangles shrunk to the alpha-threshold box (m_tighten). */
/* ------------------------------------------------------------------------ */
typedef struct {
    int tile;
    float z_near, dilation, alpha_min, alpha_max, t_min;
    float bg[3];
    int smooth;
    int tight;
} opts_t;

static void read_opts(const float *o, opts_t *p)
{
    p->tile = (int)o[0];
    p->z_near = o[1];
    p->dilation = o[2];
    p->alpha_min = o[3];
    p->alpha_max = o[4];
    p->t_min = o[5];
    p->bg[0] = o[6];
    p->bg[1] = o[7];
    p->bg[2] = o[8];
    p->smooth = o[9] != 0.0f;
    p->tight = o[10] != 0.0f;
}

/* camera: float cam[18] = {fx, fy, cx, cy, width, height, w2c[12] row-major} */

/* ======================================================================== */
/* FP32 decision mirror                                                      */
/* ======================================================================== */

/* e^x in FP32: Cody-Waite reduction + degree-6 Taylor, argument clamped to
 * [-80, 80] so that 2^k stays a normal number. */
float or_exp32(float x)
{
    x = fminf(fmaxf(x, -80.0f), 80.0f);
    const float magic = 12582912.0f; /* 1.5 * 2^23: rounds to an integer */
    float t = fmaf(x, 1.4426950408889634f, magic);
    float kf = t - magic;
    float r = fmaf(kf, -0.693145751953125f, x);
    r = fmaf(kf, -1.428606820309417e-06f, r);
    float p = 1.0f / 720.0f;
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int k = (int)kf;
    uint32_t bits = (uint32_t)(k + 127) << 23;
    float scale;
    memcpy(&scale, &bits, sizeof scale);
    return p * scale;
}

/* How many floats x with bit patterns in [lo, hi] have or_exp32(x) > 1
 * (a property check for the tests: for every exponent x <= 0 the mirror's
 * e^x is at most 1, so x o can exceed alpha_max only when the opacity o
 * does).  Multi-threaded under or_set_threads. */
int64_t or_exp32_count_above_one(uint32_t lo, uint32_t hi)
{
    int64_t bad = 0;
    const int64_t n = (int64_t)hi - (int64_t)lo + 1;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t u = lo + (uint32_t)i;
        float x;
        memcpy(&x, &u, sizeof x);
        if (!(or_exp32(x) <= 1.0f))
            ++bad;
    }
    return bad;
}

/* ln x in FP32 for a positive normal x, as the tight tile rectangles take
 * it: x = m 2^e with the mantissa m moved into [sqrt(1/2), sqrt(2)) (halved,
 * e raised, when above sqrt(2)); ln m = 2 artanh(s), s = (m - 1)/(m + 1),
 * summed as 2 s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9) by Horner in s^2 (|s| is
 * at most 0.1716, so the next term is below 2e-10); result e ln2 + that. */
float or_log32(float x)
{
    uint32_t b;
    memcpy(&b, &x, sizeof b);
    int e = (int)(b >> 23) - 127;
    uint32_t mb = (b & 0x007fffffu) | 0x3f800000u;
    float m;
    memcpy(&m, &mb, sizeof m);
    if (m > 1.41421354f) {
        m = m * 0.5f;
        e = e + 1;
    }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    float p = 0.222222222f;
    p = fmaf(p, s2, 0.285714286f);
    p = fmaf(p, s2, 0.4f);
    p = fmaf(p, s2, 0.666666667f);
    p = fmaf(p, s2, 2.0f);
    return fmaf((float)e, 0.693147181f, s * p);
}

/* camera-from-object transform M = V o T in FP32 (3x4 row-major each). */
static void m_compose(const float V[12], const float T[12], float M[12])
{
    for (int i = 0; i < 3; ++i) {
        const float *v = V + 4 * i;
        for (int j = 0; j < 3; ++j)
            M[4 * i + j] = fmaf(v[2], T[8 + j], fmaf(v[1], T[4 + j], v[0] * T[j]));
        M[4 * i + 3] = fmaf(v[2], T[11], fmaf(v[1], T[7], fmaf(v[0], T[3], v[3])));
    }
}

typedef struct {
    int vis;            /* survives the near-plane, determinant and rect culls */
    int r;              /* pixel radius */
    int x0, x1, y0, y1; /* tile rectangle [x0,x1) x [y0,y1) */
    float u, v, z;      /* pixel centre, camera depth */
    float ca, cb, cc;   /* exponent = ca dx^2 + cb dx dy + cc dy^2 */
    float o;            /* opacity */
} m32_t;

/* The tight tile rectangle: the tiles of the 3-sigma rectangle whose pixel
 * centres can reach the alpha threshold.  A pixel passes the alpha test only
 * where o e^power >= alpha_min, i.e. power >= ln(alpha_min / o); with a
 * margin of 0.06 for the FP32 evaluation, tau = ln alpha_min - ln o - 0.06,
 * and power >= tau is the ellipse d^T Q d <= -2 tau about (u, v), with
 * Q = [[A, B], [B, C]] = -[[2 ca, cb], [cb, 2 cc]].  Its axis-aligned box has
 * half-widths sqrt(-2 tau C / det) and sqrt(-2 tau A / det), det = AC - B^2,
 * taken 0.1 % + 0.01 px wider; tile t of side B (pixel centres B t + 0.5 ..
 * B t + B - 0.5) meets it when ceil((u - ex - (B - 0.5)) / B) <= t <=
 * floor((u + ex - 0.5) / B).
 * tau >= 0 (opacity below alpha_min e^-0.06) empties the rectangle; a nearly
 * singular conic (B^2 > 0.998 AC) keeps the 3-sigma one. */
static void m_tighten(const m32_t *g, float alpha_min, int tile, int TX, int TY, int *x0, int *x1, int *y0,
                      int *y1)
{
    float tau = (or_log32(alpha_min) - or_log32(g->o)) - 0.06f;
    if (!(tau < 0.0f)) {
        *x1 = *x0;
        return;
    }
    float A = -2.0f * g->ca, B = -g->cb, C = -2.0f * g->cc;
    float AC = A * C, BB = B * B;
    float det = AC - BB;
    if (!(det > 0.0f) || !(BB <= 0.998f * AC))
        return;
    float s = (-2.0f * tau) / det;
    float ex = fmaf(sqrtf(s * C), 1.001f, 0.01f);
    float ey = fmaf(sqrtf(s * A), 1.001f, 0.01f);
    if (!(ex >= 0.0f) || !(ey >= 0.0f))
        return;
    const float Bt = (float)tile, hi = Bt - 0.5f;
    float tx0 = fminf(fmaxf(ceilf(((g->u - ex) - hi) / Bt), 0.0f), (float)TX);
    float tx1 = fminf(fmaxf(floorf(((g->u + ex) - 0.5f) / Bt) + 1.0f, 0.0f), (float)TX);
    float ty0 = fminf(fmaxf(ceilf(((g->v - ey) - hi) / Bt), 0.0f), (float)TY);
    float ty1 = fminf(fmaxf(floorf(((g->v + ey) - 0.5f) / Bt) + 1.0f, 0.0f), (float)TY);
    if ((int)tx0 > *x0) *x0 = (int)tx0;
    if ((int)tx1 < *x1) *x1 = (int)tx1;
    if ((int)ty0 > *y0) *y0 = (int)ty0;
    if ((int)ty1 < *y1) *y1 = (int)ty1;
}

static void m_project(const float *mu, const float *s, const float *q, float logit,
                      const float M[12], const float *cam, const opts_t *op, m32_t *g)
{
    memset(g, 0, sizeof *g);
    const float fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
    const int W = (int)cam[4], H = (int)cam[5];
    const int TX = (W + op->tile - 1) / op->tile, TY = (H + op->tile - 1) / op->tile;

    float x = fmaf(M[2], mu[2], fmaf(M[1], mu[1], fmaf(M[0], mu[0], M[3])));
    float y = fmaf(M[6], mu[2], fmaf(M[5], mu[1], fmaf(M[4], mu[0], M[7])));
    float z = fmaf(M[10], mu[2], fmaf(M[9], mu[1], fmaf(M[8], mu[0], M[11])));
    if (!(z > op->z_near))
        return;

    float qw = q[0], qx = q[1], qy = q[2], qz = q[3];
    float n2 = fmaf(qw, qw, fmaf(qx, qx, fmaf(qy, qy, qz * qz)));
    if (!(n2 > 0.0f))
        return;
    float inv = 1.0f / sqrtf(n2);
    qw = qw * inv;
    qx = qx * inv;
    qy = qy * inv;
    qz = qz * inv;
    float xx = qx * qx, yy = qy * qy, zz = qz * qz;
    float xy = qx * qy, xz = qx * qz, yz = qy * qz;
    float wx = qw * qx, wy = qw * qy, wz = qw * qz;
    float Rq[3][3];
    Rq[0][0] = 1.0f - 2.0f * (yy + zz);
    Rq[0][1] = 2.0f * (xy - wz);
    Rq[0][2] = 2.0f * (xz + wy);
    Rq[1][0] = 2.0f * (xy + wz);
    Rq[1][1] = 1.0f - 2.0f * (xx + zz);
    Rq[1][2] = 2.0f * (yz - wx);
    Rq[2][0] = 2.0f * (xz - wy);
    Rq[2][1] = 2.0f * (yz + wx);
    Rq[2][2] = 1.0f - 2.0f * (xx + yy);

    float sig[3] = {or_exp32(s[0]), or_exp32(s[1]), or_exp32(s[2])};
    /* A = M_R Rq diag(sig);  Sigma_cam = A A^T */
    float A[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            float b = fmaf(M[4 * i + 2], Rq[2][j], fmaf(M[4 * i + 1], Rq[1][j], M[4 * i] * Rq[0][j]));
            A[i][j] = b * sig[j];
        }
    float S[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j)
            S[i][j] = fmaf(A[i][2], A[j][2], fmaf(A[i][1], A[j][1], A[i][0] * A[j][0]));

    float iz = 1.0f / z;
    float tx = x * iz, ty = y * iz;
    float j00 = fx * iz, j11 = fy * iz;
    float j02 = -(j00 * tx), j12 = -(j11 * ty);
    /* rows of J Sigma_cam (J = [[j00,0,j02],[0,j11,j12]]) */
    float r00 = fmaf(j00, S[0][0], j02 * S[0][2]);
    float r01 = fmaf(j00, S[0][1], j02 * S[1][2]);
    float r02 = fmaf(j00, S[0][2], j02 * S[2][2]);
    float r11 = fmaf(j11, S[1][1], j12 * S[1][2]);
    float r12 = fmaf(j11, S[1][2], j12 * S[2][2]);
    float a = fmaf(r00, j00, r02 * j02) + op->dilation;
    float b = fmaf(r01, j11, r02 * j12);
    float c = fmaf(r11, j11, r12 * j12) + op->dilation;
    float det = fmaf(a, c, -(b * b));
    if (!(det > 0.0f))
        return;
    float idet = 1.0f / det;
    g->ca = -0.5f * (c * idet);
    g->cb = b * idet;
    g->cc = -0.5f * (a * idet);
    float mid = 0.5f * (a + c);
    float disc = fmaxf(0.1f, fmaf(mid, mid, -det));
    float lam = mid + sqrtf(disc);
    float rf = ceilf(3.0f * sqrtf(lam));
    float u = fmaf(fx, tx, cx);
    float v = fmaf(fy, ty, cy);
    if (!(rf < 1.0e7f) || !(fabsf(u) < 1.0e7f) || !(fabsf(v) < 1.0e7f))
        return; /* non-finite or absurd footprint: culled */
    int r = (int)rf;
    const float B = (float)op->tile;
    int x0, x1, y0, y1;
    if (op->smooth) {
        x0 = 0; x1 = TX; y0 = 0; y1 = TY;
    } else {
        float fx0 = floorf((u - rf) / B), fx1 = floorf((u + rf) / B) + 1.0f;
        float fy0 = floorf((v - rf) / B), fy1 = floorf((v + rf) / B) + 1.0f;
        x0 = (int)fminf(fmaxf(fx0, 0.0f), (float)TX);
        x1 = (int)fminf(fmaxf(fx1, 0.0f), (float)TX);
        y0 = (int)fminf(fmaxf(fy0, 0.0f), (float)TY);
        y1 = (int)fminf(fmaxf(fy1, 0.0f), (float)TY);
    }
    g->u = u;
    g->v = v;
    g->z = z;
    g->o = 1.0f / (1.0f + or_exp32(-logit));
    if (op->tight && !op->smooth && op->alpha_min >= FLT_MIN)
        m_tighten(g, op->alpha_min, op->tile, TX, TY, &x0, &x1, &y0, &y1);
    if (x0 >= x1 || y0 >= y1)
        return;
    g->vis = 1;
    g->r = r;
    g->x0 = x0; g->x1 = x1; g->y0 = y0; g->y1 = y1;
    (void)H;
}

/* Contribution decision of Gaussian g at pixel (px,py).  Returns 1 and the
 * FP32 alpha if it contributes (before the transmittance test). */
/* the exponent of the Gaussian density at pixel sample (pxf, pyf) in the
 * mirror's FP32 sequence: dx, dy, h = ca dx + (cb dy), (cc dy) dy, h dx + that */
static float m_power(float u, float v, float ca, float cb, float cc, float pxf, float pyf)
{
    float dx = u - pxf, dy = v - pyf;
    float h = fmaf(ca, dx, cb * dy);
    float k = (cc * dy) * dy;
    return fmaf(h, dx, k);
}

static int m_alpha(const m32_t *g, int px, int py, const opts_t *op, float *alpha, int *clamped)
{
    float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    float power = m_power(g->u, g->v, g->ca, g->cb, g->cc, pxf, pyf);
    if (power > 0.0f)
        return 0;
    float x = g->o * or_exp32(power);
    int cl = x > op->alpha_max;
    float a = cl ? op->alpha_max : x;
    if (a < op->alpha_min)
        return 0;
    *alpha = a;
    *clamped = cl;
    return 1;
}

/* How many of n (conic, mean, pixel sample) cases have a positive mirror
 * exponent (a property check for the tests: a well-conditioned conic's
 * exponent never rounds above 0).  Multi-threaded under or_set_threads. */
int64_t or_count_positive_power(int64_t n, const float *ca, const float *cb, const float *cc, const float *u,
                                const float *v, const float *pxf, const float *pyf)
{
    int64_t pos = 0;
#pragma omp parallel for schedule(static) reduction(+ : pos)
    for (int64_t i = 0; i < n; ++i)
        if (m_power(u[i], v[i], ca[i], cb[i], cc[i], pxf[i], pyf[i]) > 0.0f)
            ++pos;
    return pos;
}

/* ======================================================================== */
/* FP64 values                                                               */
/* ======================================================================== */

typedef struct {
    double mw[3];     /* mu' = R mu + t */
    double Sw[3][3];  /* Sigma' = R Sigma R^T */
    double m[3];      /* camera-space mean */
    double Sc[3][3];  /* camera-space covariance */
    double J[2][3];   /* projection Jacobian at m */
    double A, B, C;   /* conic = inverse of the dilated 2D covariance */
    double U, V;      /* pixel-space mean */
    double o;         /* opacity */
    double sig[3];    /* e^s */
    double Rq[3][3];  /* rotation of the Gaussian */
    double qn[4];     /* normalised quaternion */
    double qlen;      /* |q| */
} v64_t;

static void mat3_mul(const double a[3][3], const double b[3][3], double c[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            c[i][j] = a[i][0] * b[0][j] + a[i][1] * b[1][j] + a[i][2] * b[2][j];
}

static void mat3_mul_bt(const double a[3][3], const double b[3][3], double c[3][3])
{ /* c = a b^T */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            c[i][j] = a[i][0] * b[j][0] + a[i][1] * b[j][1] + a[i][2] * b[j][2];
}

static void mat3_tmul(const double a[3][3], const double b[3][3], double c[3][3])
{ /* c = a^T b */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            c[i][j] = a[0][i] * b[0][j] + a[1][i] * b[1][j] + a[2][i] * b[2][j];
}

static void rot_of(const double *P12, double R[3][3], double t[3])
{
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            R[i][j] = P12[4 * i + j];
        t[i] = P12[4 * i + 3];
    }
}

static void quat_to_rot(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z);
    R[0][1] = 2 * (x * y - w * z);
    R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);
    R[1][1] = 1 - 2 * (x * x + z * z);
    R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);
    R[2][1] = 2 * (y * z + w * x);
    R[2][2] = 1 - 2 * (x * x + y * y);
}

/* FP64 projection of one Gaussian under pose T (object -> world) and the
 * view's world -> camera transform. */
static void v_project(const float *mu, const float *s, const float *q, float logit,
                      const double T[12], const double Vw[12], const float *cam, double dil, v64_t *g)
{
    double R[3][3], t[3], Rv[3][3], tv[3];
    rot_of(T, R, t);
    rot_of(Vw, Rv, tv);
    const double fx = cam[0], fy = cam[1], cx = cam[2], cy = cam[3];
    double m0[3] = {mu[0], mu[1], mu[2]};
    for (int i = 0; i < 3; ++i)
        g->mw[i] = R[i][0] * m0[0] + R[i][1] * m0[1] + R[i][2] * m0[2] + t[i];
    for (int i = 0; i < 3; ++i)
        g->m[i] = Rv[i][0] * g->mw[0] + Rv[i][1] * g->mw[1] + Rv[i][2] * g->mw[2] + tv[i];

    double ql = sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] + (double)q[3] * q[3]);
    g->qlen = ql;
    for (int k = 0; k < 4; ++k)
        g->qn[k] = q[k] / ql;
    quat_to_rot(g->qn, g->Rq);
    for (int k = 0; k < 3; ++k)
        g->sig[k] = exp((double)s[k]);
    /* Sigma = Rq S^2 Rq^T */
    double RS[3][3], Sig[3][3], tmp[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            RS[i][j] = g->Rq[i][j] * g->sig[j] * g->sig[j];
    mat3_mul_bt(RS, g->Rq, Sig);
    /* Sigma' = R Sigma R^T (Eq. 9) */
    mat3_mul(R, Sig, tmp);
    mat3_mul_bt(tmp, R, g->Sw);
    /* camera frame */
    mat3_mul(Rv, g->Sw, tmp);
    mat3_mul_bt(tmp, Rv, g->Sc);

    double x = g->m[0], y = g->m[1], z = g->m[2];
    g->J[0][0] = fx / z; g->J[0][1] = 0; g->J[0][2] = -fx * x / (z * z);
    g->J[1][0] = 0; g->J[1][1] = fy / z; g->J[1][2] = -fy * y / (z * z);
    double JS[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            JS[i][j] = g->J[i][0] * g->Sc[0][j] + g->J[i][1] * g->Sc[1][j] + g->J[i][2] * g->Sc[2][j];
    double a = JS[0][0] * g->J[0][0] + JS[0][1] * g->J[0][1] + JS[0][2] * g->J[0][2] + dil;
    double b = JS[0][0] * g->J[1][0] + JS[0][1] * g->J[1][1] + JS[0][2] * g->J[1][2];
    double c = JS[1][0] * g->J[1][0] + JS[1][1] * g->J[1][1] + JS[1][2] * g->J[1][2] + dil;
    double det = a * c - b * b;
    g->A = c / det;
    g->B = -b / det;
    g->C = a / det;
    g->U = fx * x / z + cx;
    g->V = fy * y / z + cy;
    g->o = 1.0 / (1.0 + exp(-(double)logit));
}

/* ======================================================================== */
/* per-camera preparation: projection (both precisions) + binning            */
/* ======================================================================== */

typedef struct {
    uint64_t key;  /* (tile << 32) | float bits of z */
    uint64_t seq;  /* emission order: Gaussian index major, tile row-major */
    uint32_t gid;
} dup_t;

static int dup_cmp(const void *pa, const void *pb)
{
    const dup_t *a = pa, *b = pb;
    if (a->key != b->key)
        return a->key < b->key ? -1 : 1;
    if (a->seq != b->seq)
        return a->seq < b->seq ? -1 : 1;
    return 0;
}

typedef struct {
    int n, W, H, TX, TY;
    m32_t *g32;
    v64_t *g64;
    dup_t *dups;
    long ndup;
    long *rstart, *rend; /* per tile */
} prep_t;

static void prep_free(prep_t *p)
{
    free(p->g32);
    free(p->g64);
    free(p->dups);
    free(p->rstart);
    free(p->rend);
    memset(p, 0, sizeof *p);
}

static int prep_camera(int n, const float *means4, const float *scales4, const float *quats4,
                       const float *logits, const double pose[12], const float *cam, const opts_t *op,
                       prep_t *p)
{
    memset(p, 0, sizeof *p);
    p->n = n;
    p->W = (int)cam[4];
    p->H = (int)cam[5];
    p->TX = (p->W + op->tile - 1) / op->tile;
    p->TY = (p->H + op->tile - 1) / op->tile;
    p->g32 = calloc((size_t)(n > 0 ? n : 1), sizeof(m32_t));
    p->g64 = calloc((size_t)(n > 0 ? n : 1), sizeof(v64_t));
    long ntiles = (long)p->TX * p->TY;
    p->rstart = calloc((size_t)(ntiles > 0 ? ntiles : 1), sizeof(long));
    p->rend = calloc((size_t)(ntiles > 0 ? ntiles : 1), sizeof(long));
    if (!p->g32 || !p->g64 || !p->rstart || !p->rend)
        return OR_ERR_OOM;
    float P32[12], V32[12], M32[12];
    double Vw[12];
    for (int k = 0; k < 12; ++k) {
        P32[k] = (float)pose[k];
        V32[k] = cam[6 + k];
        Vw[k] = cam[6 + k];
    }
    m_compose(V32, P32, M32);
    long total = 0;
    for (int i = 0; i < n; ++i) {
        m_project(means4 + 4 * i, scales4 + 4 * i, quats4 + 4 * i, logits[i], M32, cam, op, &p->g32[i]);
        if (p->g32[i].vis) {
            v_project(means4 + 4 * i, scales4 + 4 * i, quats4 + 4 * i, logits[i], pose, Vw, cam,
                      op->dilation, &p->g64[i]);
            total += (long)(p->g32[i].x1 - p->g32[i].x0) * (p->g32[i].y1 - p->g32[i].y0);
        }
    }
    p->dups = malloc((size_t)(total > 0 ? total : 1) * sizeof(dup_t));
    if (!p->dups)
        return OR_ERR_OOM;
    long e = 0;
    for (int i = 0; i < n; ++i) {
        const m32_t *g = &p->g32[i];
        if (!g->vis)
            continue;
        uint32_t zb;
        memcpy(&zb, &g->z, 4);
        for (int ty = g->y0; ty < g->y1; ++ty)
            for (int tx = g->x0; tx < g->x1; ++tx) {
                p->dups[e].key = ((uint64_t)(ty * p->TX + tx) << 32) | zb;
                p->dups[e].seq = (uint64_t)e;
                p->dups[e].gid = (uint32_t)i;
                ++e;
            }
    }
    p->ndup = e;
    qsort(p->dups, (size_t)e, sizeof(dup_t), dup_cmp);
    for (long k = 0; k < e; ++k) {
        long t = (long)(p->dups[k].key >> 32);
        if (k == 0 || (long)(p->dups[k - 1].key >> 32) != t)
            p->rstart[t] = k;
        if (k == e - 1 || (long)(p->dups[k + 1].key >> 32) != t)
            p->rend[t] = k + 1;
    }
    return OR_OK;
}

/* ======================================================================== */
/* compositing (FP64 values, FP32 decisions)                                 */
/* ======================================================================== */

typedef struct {
    int gid;
    double alpha, T, e, dx, dy;
    int clamped;
} contrib_t;

/* Walks the tile list of pixel (px,py); fills the contributor list (if cl is
 * not NULL) and returns their number.  *Tf64, *Tf32: final transmittance;
 * *D32: the FP32 mirror of the depth (sum of z * (alpha * T) by fused
 * multiply-adds in list order, alpha and T the mirror's); *last: one past
 * the list position of the last contributor. */
static int walk_pixel(const prep_t *p, const opts_t *op, int px, int py, contrib_t *cl,
                      double *rgb, double *depth, const float *rgb4, double *Tf64, float *Tf32, float *D32,
                      long *last)
{
    int tx = px / op->tile, ty = py / op->tile;
    long t = (long)ty * p->TX + tx;
    double T = 1.0, C[3] = {0, 0, 0}, D = 0.0;
    float T32 = 1.0f, Dm = 0.0f;
    long lst = 0;
    int k = 0;
    double pxc = px + 0.5, pyc = py + 0.5;
    for (long j = p->rstart[t]; j < p->rend[t]; ++j) {
        int gi = (int)p->dups[j].gid;
        float a32;
        int clamped;
        if (!m_alpha(&p->g32[gi], px, py, op, &a32, &clamped))
            continue;
        float Tn32 = T32 * (1.0f - a32);
        if (Tn32 < op->t_min)
            break;
        const v64_t *g = &p->g64[gi];
        double dx = g->U - pxc, dy = g->V - pyc;
        double power = -0.5 * (g->A * dx * dx + g->C * dy * dy) - g->B * dx * dy;
        double e = exp(power);
        double a = clamped ? (double)op->alpha_max : g->o * e;
        double w = a * T;
        for (int ch = 0; ch < 3; ++ch)
            C[ch] += rgb4[4 * gi + ch] * w;
        D += g->m[2] * w;
        if (cl) {
            cl[k].gid = gi;
            cl[k].alpha = a;
            cl[k].T = T;
            cl[k].e = e;
            cl[k].dx = dx;
            cl[k].dy = dy;
            cl[k].clamped = clamped;
        }
        ++k;
        Dm = fmaf(p->g32[gi].z, a32 * T32, Dm);
        T = T * (1.0 - a);
        T32 = Tn32;
        lst = j - p->rstart[t] + 1;
    }
    for (int ch = 0; ch < 3; ++ch)
        rgb[ch] = C[ch] + T * op->bg[ch];
    *depth = D;
    *Tf64 = T;
    *Tf32 = T32;
    if (D32)
        *D32 = Dm;
    *last = lst;
    return k;
}

static long max_list(const prep_t *p)
{
    long m = 0;
    for (long t = 0; t < (long)p->TX * p->TY; ++t)
        if (p->rend[t] - p->rstart[t] > m)
            m = p->rend[t] - p->rstart[t];
    return m;
}

static void composite(const prep_t *p, const opts_t *op, const float *rgb4, double *out_rgb,
                      double *out_depth, double *out_alpha, double *out_tf, float *out_tf32,
                      int32_t *out_last, float *out_depth32)
{
    const long HW = (long)p->W * p->H;
    /* pixels are independent: rows may run on several threads */
#pragma omp parallel for schedule(dynamic, 4)
    for (int py = 0; py < p->H; ++py)
        for (int px = 0; px < p->W; ++px) {
            double c[3], d, Tf;
            float Tf32, D32;
            long last;
            walk_pixel(p, op, px, py, NULL, c, &d, rgb4, &Tf, &Tf32, &D32, &last);
            long pix = (long)py * p->W + px;
            if (out_depth32) out_depth32[pix] = D32;
            for (int ch = 0; ch < 3; ++ch)
                if (out_rgb)
                    out_rgb[ch * HW + pix] = c[ch];
            if (out_depth) out_depth[pix] = d;
            if (out_alpha) out_alpha[pix] = 1.0 - Tf;
            if (out_tf) out_tf[pix] = Tf;
            if (out_tf32) out_tf32[pix] = Tf32;
            if (out_last) out_last[pix] = (int32_t)last;
        }
}

/* ======================================================================== */
/* adjoint                                                                   */
/* ======================================================================== */

/* per-Gaussian accumulated screen-space gradient */
enum { G_U, G_V, G_A, G_B, G_C, G_Z, G_O, G_R, G_G, G_BL, G_N };

/* Accumulates dL/d(screen parameters) of every Gaussian, given per-pixel
 * cotangents of the rendered colour (3 planes), depth and alpha.  The image
 * is cut into OR_CHUNKS bands of tile rows; each band sums its pixels'
 * contributions (row-major) into its own accumulator, and the bands are
 * added in band order, so the result does not depend on how many threads
 * run the bands. */
#define OR_CHUNKS 16

static int adjoint_band(const prep_t *p, const opts_t *op, const float *rgb4, const double *g_rgb,
                        const double *g_depth, const double *g_alpha, int py0, int py1, double *acc)
{
    const long HW = (long)p->W * p->H;
    long ml = max_list(p);
    contrib_t *cl = malloc((size_t)(ml > 0 ? ml : 1) * sizeof(contrib_t));
    double *Sc = malloc((size_t)(ml > 0 ? ml : 1) * 4 * sizeof(double));
    if (!cl || !Sc) {
        free(cl);
        free(Sc);
        return OR_ERR_OOM;
    }
    for (int py = py0; py < py1; ++py)
        for (int px = 0; px < p->W; ++px) {
            long pix = (long)py * p->W + px;
            double gc[3], gd, ga;
            for (int ch = 0; ch < 3; ++ch)
                gc[ch] = g_rgb ? g_rgb[ch * HW + pix] : 0.0;
            gd = g_depth ? g_depth[pix] : 0.0;
            ga = g_alpha ? g_alpha[pix] : 0.0;
            double c[3], d, Tf;
            float Tf32;
            long last;
            int K = walk_pixel(p, op, px, py, cl, c, &d, rgb4, &Tf, &Tf32, NULL, &last);
            /* suffix sums S_i = sum_{j>i} c_j alpha_j T_j (+ T_f bg for colour) */
            double s[4] = {Tf * op->bg[0], Tf * op->bg[1], Tf * op->bg[2], 0.0};
            for (int i = K - 1; i >= 0; --i) {
                for (int q = 0; q < 4; ++q)
                    Sc[4 * i + q] = s[q];
                int gi = cl[i].gid;
                double w = cl[i].alpha * cl[i].T;
                for (int ch = 0; ch < 3; ++ch)
                    s[ch] += rgb4[4 * gi + ch] * w;
                s[3] += p->g64[gi].m[2] * w;
            }
            for (int i = 0; i < K; ++i) {
                int gi = cl[i].gid;
                const v64_t *g = &p->g64[gi];
                double a = cl[i].alpha, T = cl[i].T, om = 1.0 - a;
                double dLda = 0.0;
                for (int ch = 0; ch < 3; ++ch)
                    dLda += gc[ch] * (rgb4[4 * gi + ch] * T - Sc[4 * i + ch] / om);
                dLda += gd * (g->m[2] * T - Sc[4 * i + 3] / om);
                dLda += ga * (Tf / om);
                double *A = acc + (size_t)gi * G_N;
                A[G_R] += gc[0] * a * T;
                A[G_G] += gc[1] * a * T;
                A[G_BL] += gc[2] * a * T;
                A[G_Z] += gd * a * T;
                if (!cl[i].clamped) {
                    /* alpha = o e^power */
                    A[G_O] += dLda * cl[i].e;
                    double dp = dLda * a;
                    double dx = cl[i].dx, dy = cl[i].dy;
                    /* power = -1/2 (A dx^2 + C dy^2) - B dx dy, dx = U - px */
                    A[G_U] += dp * (-(g->A * dx + g->B * dy));
                    A[G_V] += dp * (-(g->B * dx + g->C * dy));
                    A[G_A] += dp * (-0.5 * dx * dx);
                    A[G_B] += dp * (-dx * dy);
                    A[G_C] += dp * (-0.5 * dy * dy);
                }
            }
        }
    free(cl);
    free(Sc);
    return OR_OK;
}

static int adjoint_screen(const prep_t *p, const opts_t *op, const float *rgb4, const double *g_rgb,
                          const double *g_depth, const double *g_alpha, double *acc /* n x G_N */)
{
    const size_t na = (size_t)(p->n > 0 ? p->n : 1) * G_N;
    double *band = calloc(na * OR_CHUNKS, sizeof(double));
    if (!band)
        return OR_ERR_OOM;
    int st = OR_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < OR_CHUNKS; ++c) {
        /* band c: tile rows [c TY / K, (c + 1) TY / K) */
        const int ty0 = (int)((long)c * p->TY / OR_CHUNKS), ty1 = (int)((long)(c + 1) * p->TY / OR_CHUNKS);
        const int py0 = ty0 * op->tile, py1 = ty1 * op->tile < p->H ? ty1 * op->tile : p->H;
        if (py0 < py1 && adjoint_band(p, op, rgb4, g_rgb, g_depth, g_alpha, py0, py1, band + na * c) != OR_OK) {
#pragma omp critical
            st = OR_ERR_OOM;
        }
    }
    if (st == OR_OK)
        for (int c = 0; c < OR_CHUNKS; ++c)
            for (size_t k = 0; k < na; ++k)
                acc[k] += band[na * c + k];
    free(band);
    return st;
}

/* Threads used by the parallel loops (1 unless the library was built with
 * OpenMP); returns the number in effect. */
int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Chains the screen-space gradient of every Gaussian to (a) the left twist
 * (omega, v) of the pose about the pivot c: mu' -> exp(omega)(mu' - c) + c + v,
 * Sigma' -> exp(omega) Sigma' exp(omega)^T, and (b) optionally every
 * Gaussian parameter. */
static void chain(const prep_t *p, const double pose[12], const float *cam, const double *acc,
                  const double pivot[3], const float *logits, double twist[6], double *g_means,
                  double *g_scales, double *g_quats, double *g_logits, double *g_rgb)
{
    double R[3][3], t[3], Rv[3][3], tv[3], Vw[12];
    for (int k = 0; k < 12; ++k)
        Vw[k] = cam[6 + k];
    rot_of(pose, R, t);
    rot_of(Vw, Rv, tv);
    const double fx = cam[0], fy = cam[1];
    for (int gi = 0; gi < p->n; ++gi) {
        if (!p->g32[gi].vis)
            continue;
        const double *A = acc + (size_t)gi * G_N;
        const v64_t *g = &p->g64[gi];
        if (g_rgb) {
            g_rgb[3 * gi + 0] += A[G_R];
            g_rgb[3 * gi + 1] += A[G_G];
            g_rgb[3 * gi + 2] += A[G_BL];
        }
        if (g_logits)
            g_logits[gi] += A[G_O] * g->o * (1.0 - g->o);
        /* conic -> 2D covariance: dL/dSigma2 = -Q G_Q Q */
        double Q[2][2] = {{g->A, g->B}, {g->B, g->C}};
        double GQ[2][2] = {{A[G_A], 0.5 * A[G_B]}, {0.5 * A[G_B], A[G_C]}};
        double t1[2][2], G2[2][2];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                t1[i][j] = Q[i][0] * GQ[0][j] + Q[i][1] * GQ[1][j];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                G2[i][j] = -(t1[i][0] * Q[0][j] + t1[i][1] * Q[1][j]);
        /* Sigma2 = J Sc J^T + dI: dL/dSc = J^T G2 J, dL/dJ = 2 G2 J Sc */
        double Gc[3][3], GJ[2][3], G2J[2][3];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                G2J[i][j] = G2[i][0] * g->J[0][j] + G2[i][1] * g->J[1][j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Gc[i][j] = g->J[0][i] * G2J[0][j] + g->J[1][i] * G2J[1][j];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                GJ[i][j] = 2.0 * (G2J[i][0] * g->Sc[0][j] + G2J[i][1] * g->Sc[1][j] + G2J[i][2] * g->Sc[2][j]);
        double x = g->m[0], y = g->m[1], z = g->m[2];
        double gm[3];
        gm[0] = A[G_U] * fx / z;
        gm[1] = A[G_V] * fy / z;
        gm[2] = -A[G_U] * fx * x / (z * z) - A[G_V] * fy * y / (z * z) + A[G_Z];
        /* J = [[fx/z, 0, -fx x/z^2], [0, fy/z, -fy y/z^2]] */
        gm[0] += GJ[0][2] * (-fx / (z * z));
        gm[1] += GJ[1][2] * (-fy / (z * z));
        gm[2] += GJ[0][0] * (-fx / (z * z)) + GJ[1][1] * (-fy / (z * z)) +
                 GJ[0][2] * (2.0 * fx * x / (z * z * z)) + GJ[1][2] * (2.0 * fy * y / (z * z * z));
        /* world (target) frame: m = Rv mu' + tv, Sc = Rv Sigma' Rv^T */
        double gmw[3], Gw[3][3], tmp[3][3];
        for (int i = 0; i < 3; ++i)
            gmw[i] = Rv[0][i] * gm[0] + Rv[1][i] * gm[1] + Rv[2][i] * gm[2];
        mat3_tmul(Rv, Gc, tmp);
        mat3_mul(tmp, Rv, Gw);
        if (twist) {
            double rel[3] = {g->mw[0] - pivot[0], g->mw[1] - pivot[1], g->mw[2] - pivot[2]};
            double cr[3];
            cross3(rel, gmw, cr);
            double GS[3][3], SG[3][3];
            mat3_mul(Gw, g->Sw, GS);
            mat3_mul(g->Sw, Gw, SG);
            /* 2 vee(G Sigma' - Sigma' G) */
            double K21 = GS[2][1] - SG[2][1], K02 = GS[0][2] - SG[0][2], K10 = GS[1][0] - SG[1][0];
            twist[0] += cr[0] + 2.0 * K21;
            twist[1] += cr[1] + 2.0 * K02;
            twist[2] += cr[2] + 2.0 * K10;
            twist[3] += gmw[0];
            twist[4] += gmw[1];
            twist[5] += gmw[2];
        }
        if (g_means || g_scales || g_quats) {
            /* object frame: mu' = R mu + t, Sigma' = R Sigma R^T */
            double GS0[3][3];
            mat3_tmul(R, Gw, tmp);
            mat3_mul(tmp, R, GS0);
            if (g_means)
                for (int i = 0; i < 3; ++i)
                    g_means[3 * gi + i] += R[0][i] * gmw[0] + R[1][i] * gmw[1] + R[2][i] * gmw[2];
            /* Sigma = Rq S^2 Rq^T: dL/ds_k = 2 sig_k^2 (Rq^T G Rq)_kk; dL/dRq = 2 G Rq S^2 */
            double RtG[3][3], RtGR[3][3];
            mat3_tmul(g->Rq, GS0, RtG);
            mat3_mul(RtG, g->Rq, RtGR);
            if (g_scales)
                for (int k = 0; k < 3; ++k)
                    g_scales[3 * gi + k] += 2.0 * g->sig[k] * g->sig[k] * RtGR[k][k];
            if (g_quats) {
                double GR[3][3], dR[3][3];
                mat3_mul(GS0, g->Rq, GR);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j)
                        dR[i][j] = 2.0 * GR[i][j] * g->sig[j] * g->sig[j];
                double w = g->qn[0], qx = g->qn[1], qy = g->qn[2], qz = g->qn[3];
                double gw = 0, gx = 0, gy = 0, gz = 0;
                gy += dR[0][0] * (-4 * qy); gz += dR[0][0] * (-4 * qz);
                gw += dR[0][1] * (-2 * qz); gx += dR[0][1] * (2 * qy); gy += dR[0][1] * (2 * qx); gz += dR[0][1] * (-2 * w);
                gw += dR[0][2] * (2 * qy); gx += dR[0][2] * (2 * qz); gy += dR[0][2] * (2 * w); gz += dR[0][2] * (2 * qx);
                gw += dR[1][0] * (2 * qz); gx += dR[1][0] * (2 * qy); gy += dR[1][0] * (2 * qx); gz += dR[1][0] * (2 * w);
                gx += dR[1][1] * (-4 * qx); gz += dR[1][1] * (-4 * qz);
                gw += dR[1][2] * (-2 * qx); gx += dR[1][2] * (-2 * w); gy += dR[1][2] * (2 * qz); gz += dR[1][2] * (2 * qy);
                gw += dR[2][0] * (-2 * qy); gx += dR[2][0] * (2 * qz); gy += dR[2][0] * (-2 * w); gz += dR[2][0] * (2 * qx);
                gw += dR[2][1] * (2 * qx); gx += dR[2][1] * (2 * w); gy += dR[2][1] * (2 * qz); gz += dR[2][1] * (2 * qy);
                gx += dR[2][2] * (-4 * qx); gy += dR[2][2] * (-4 * qy);
                /* q_hat = q / |q|: dL/dq = (g - q_hat (q_hat . g)) / |q| */
                double gq[4] = {gw, gx, gy, gz};
                double dot = g->qn[0] * gw + g->qn[1] * gx + g->qn[2] * gy + g->qn[3] * gz;
                for (int k = 0; k < 4; ++k)
                    g_quats[4 * gi + k] += (gq[k] - g->qn[k] * dot) / g->qlen;
            }
        }
    }
    (void)logits;
}

/* ======================================================================== */
/* exported entry points                                                     */
/* ======================================================================== */

static int check_cam(const float *cam, const opts_t *op)
{
    if (!cam || op->tile <= 0)
        return 0;
    if (!(cam[4] >= 1.0f) || !(cam[5] >= 1.0f))
        return 0;
    return 1;
}

/* FP32 mirror of the projection of n Gaussians (one pose, one camera).
 * Per Gaussian: out_f[8] = {u, v, z, ca, cb, cc, o, 0},
 * out_i[6] = {visible, radius, x0, x1, y0, y1}. */
int or_project32(int n, const float *means4, const float *scales4, const float *quats4,
                 const float *logits, const double *pose, const float *cam, const float *opt,
                 float *out_f, int32_t *out_i)
{
    opts_t op;
    read_opts(opt, &op);
    if (n < 0 || !check_cam(cam, &op))
        return OR_ERR_ARG;
    float P32[12], V32[12], M32[12];
    for (int k = 0; k < 12; ++k) {
        P32[k] = (float)pose[k];
        V32[k] = cam[6 + k];
    }
    m_compose(V32, P32, M32);
    for (int i = 0; i < n; ++i) {
        m32_t g;
        m_project(means4 + 4 * i, scales4 + 4 * i, quats4 + 4 * i, logits[i], M32, cam, &op, &g);
        float *f = out_f + 8 * i;
        int32_t *q = out_i + 6 * i;
        f[0] = g.u; f[1] = g.v; f[2] = g.z; f[3] = g.ca; f[4] = g.cb; f[5] = g.cc; f[6] = g.o; f[7] = 0.0f;
        q[0] = g.vis; q[1] = g.r; q[2] = g.x0; q[3] = g.x1; q[4] = g.y0; q[5] = g.y1;
    }
    return OR_OK;
}

/* FP64 projection of n Gaussians.  Per Gaussian (visible or not):
 * out[16] = {U, V, z, A, B, C, o, x, y, Sc00, Sc01, Sc02, Sc11, Sc12, Sc22, 0}
 * where (A,B,C) is the conic of the dilated 2D covariance. */
int or_project64(int n, const float *means4, const float *scales4, const float *quats4,
                 const float *logits, const double *pose, const float *cam, const float *opt, double *out)
{
    opts_t op;
    read_opts(opt, &op);
    if (n < 0 || !check_cam(cam, &op))
        return OR_ERR_ARG;
    double Vw[12];
    for (int k = 0; k < 12; ++k)
        Vw[k] = cam[6 + k];
    for (int i = 0; i < n; ++i) {
        v64_t g;
        v_project(means4 + 4 * i, scales4 + 4 * i, quats4 + 4 * i, logits[i], pose, Vw, cam, op.dilation, &g);
        double *o = out + 16 * i;
        o[0] = g.U; o[1] = g.V; o[2] = g.m[2]; o[3] = g.A; o[4] = g.B; o[5] = g.C; o[6] = g.o;
        o[7] = g.m[0]; o[8] = g.m[1];
        o[9] = g.Sc[0][0]; o[10] = g.Sc[0][1]; o[11] = g.Sc[0][2];
        o[12] = g.Sc[1][1]; o[13] = g.Sc[1][2]; o[14] = g.Sc[2][2]; o[15] = 0.0;
    }
    return OR_OK;
}

/* Binning of n Gaussians seen by n_cams cameras (pose i for camera i).
 * Record index of (camera c, Gaussian g) is c*n + g; tile ids are global:
 * camera c's tiles follow those of cameras 0..c-1.  Writes the sorted keys
 * and values (up to cap) and per-tile [start, end) ranges; returns the
 * number of duplicates in *ndup.  ranges: 2 * total_tiles int64. */
int or_bin(int n, const float *means4, const float *scales4, const float *quats4, const float *logits,
           int n_cams, const double *poses, const float *cams, const float *opt, uint64_t *keys,
           uint32_t *vals, long cap, int64_t *ranges, long *ndup)
{
    opts_t op;
    read_opts(opt, &op);
    long tile_base = 0, out = 0;
    for (int c = 0; c < n_cams; ++c) {
        const float *cam = cams + 18 * c;
        if (!check_cam(cam, &op))
            return OR_ERR_ARG;
        prep_t p;
        int st = prep_camera(n, means4, scales4, quats4, logits, poses + 12 * c, cam, &op, &p);
        if (st != OR_OK) {
            prep_free(&p);
            return st;
        }
        for (long k = 0; k < p.ndup; ++k) {
            if (out + k < cap) {
                uint64_t tile = (p.dups[k].key >> 32) + (uint64_t)tile_base;
                keys[out + k] = (tile << 32) | (p.dups[k].key & 0xffffffffull);
                vals[out + k] = (uint32_t)((long)c * n + p.dups[k].gid);
            }
        }
        long ntiles = (long)p.TX * p.TY;
        for (long t = 0; t < ntiles; ++t) {
            int64_t s = p.rend[t] > p.rstart[t] ? p.rstart[t] + out : 0;
            int64_t e = p.rend[t] > p.rstart[t] ? p.rend[t] + out : 0;
            ranges[2 * (tile_base + t)] = s;
            ranges[2 * (tile_base + t) + 1] = e;
        }
        out += p.ndup;
        tile_base += ntiles;
        prep_free(&p);
    }
    *ndup = out;
    return OR_OK;
}

/* Renders n Gaussians transformed by pose at one camera.  Colour is planar
 * [3][H][W]; any output may be NULL.  tf32 and depth32 are the mirror's FP32
 * final transmittance and depth, last is one past the tile-list position of
 * the last contributor (0 if none). */
int or_render(int n, const float *means4, const float *scales4, const float *quats4, const float *logits,
              const float *rgb4, const double *pose, const float *cam, const float *opt, double *out_rgb,
              double *out_depth, double *out_alpha, double *out_tf, float *out_tf32, int32_t *out_last,
              float *out_depth32)
{
    opts_t op;
    read_opts(opt, &op);
    if (n < 0 || !check_cam(cam, &op))
        return OR_ERR_ARG;
    prep_t p;
    int st = prep_camera(n, means4, scales4, quats4, logits, pose, cam, &op, &p);
    if (st == OR_OK)
        composite(&p, &op, rgb4, out_rgb, out_depth, out_alpha, out_tf, out_tf32, out_last, out_depth32);
    prep_free(&p);
    return st;
}

/* Per-pixel signature of the contributor sequence of or_render (FNV-1a over
 * (Gaussian index, clamped) of each contributor in list order, then the
 * count): two renders whose signatures agree at every pixel take the same
 * discrete choices (alpha test, clamp, early stop) everywhere, so a finite
 * difference between them crosses no threshold.  sig[H][W]. */
int or_contrib_sig(int n, const float *means4, const float *scales4, const float *quats4, const float *logits,
                   const float *rgb4, const double *pose, const float *cam, const float *opt, uint64_t *sig)
{
    opts_t op;
    read_opts(opt, &op);
    if (n < 0 || !check_cam(cam, &op))
        return OR_ERR_ARG;
    prep_t p;
    int st = prep_camera(n, means4, scales4, quats4, logits, pose, cam, &op, &p);
    long ml = st == OR_OK ? max_list(&p) : 0;
    contrib_t *cl = st == OR_OK ? malloc((size_t)(ml > 0 ? ml : 1) * sizeof(contrib_t)) : NULL;
    if (st == OR_OK && !cl)
        st = OR_ERR_OOM;
    for (int py = 0; st == OR_OK && py < p.H; ++py)
        for (int px = 0; px < p.W; ++px) {
            double c[3], d, Tf;
            float Tf32;
            long last;
            int K = walk_pixel(&p, &op, px, py, cl, c, &d, rgb4, &Tf, &Tf32, NULL, &last);
            uint64_t h = 1469598103934665603ull;
            for (int i = 0; i < K; ++i)
                h = (h ^ (uint64_t)(2 * (uint64_t)cl[i].gid + (uint64_t)cl[i].clamped)) * 1099511628211ull;
            sig[(long)py * p.W + px] = (h ^ (uint64_t)K) * 1099511628211ull;
        }
    free(cl);
    prep_free(&p);
    return st;
}

/* L1 colour + L1 depth loss of one view (Sec. 3.2): returns
 * L = mean|I^ - I| over 3HW + mean|D^ - D| over HW; writes the gradients
 * dL/dI^ = sign(I^ - I)/(3HW), dL/dD^ = sign(D^ - D)/(HW) (sign(0) = 0)
 * when the pointers are not NULL. */
double or_loss(int H, int W, const double *rgb, const double *depth, const double *t_rgb,
               const double *t_depth, double *g_rgb, double *g_depth)
{
    const long HW = (long)H * W;
    double lc = 0.0, ld = 0.0;
    for (long k = 0; k < 3 * HW; ++k) {
        double d = rgb[k] - t_rgb[k];
        lc += fabs(d);
        if (g_rgb)
            g_rgb[k] = (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (3.0 * (double)HW);
    }
    for (long k = 0; k < HW; ++k) {
        double d = depth[k] - t_depth[k];
        ld += fabs(d);
        if (g_depth)
            g_depth[k] = (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)HW;
    }
    return lc / (3.0 * (double)HW) + ld / (double)HW;
}

/* Registration loss with exposure compensation (Supp. B: the exposure of
 * each keyframe is optimised with its pose).  The compensated colour is
 * e^a I^ + b (one gain and one offset per keyframe, shared by the three
 * channels); returns or_loss of the compensated colour, and writes
 * g_rgb = dL/dI^ (the raw render's cotangent, e^a times the compensated
 * one), g_depth, and g_ab = (dL/da, dL/db). */
double or_exposure_loss(int H, int W, const double *rgb, const double *depth, const double *t_rgb,
                        const double *t_depth, const double *ab, double *g_rgb, double *g_depth, double *g_ab)
{
    const long HW = (long)H * W;
    double *x = malloc((size_t)(3 * HW > 0 ? 3 * HW : 1) * sizeof(double));
    double *gx = malloc((size_t)(3 * HW > 0 ? 3 * HW : 1) * sizeof(double));
    if (!x || !gx) {
        free(x);
        free(gx);
        return NAN;
    }
    const double ea = exp(ab[0]);
    for (long k = 0; k < 3 * HW; ++k)
        x[k] = ea * rgb[k] + ab[1];
    const double L = or_loss(H, W, x, depth, t_rgb, t_depth, gx, g_depth);
    double ga = 0.0, gb = 0.0;
    for (long k = 0; k < 3 * HW; ++k) {
        ga += gx[k] * ea * rgb[k];
        gb += gx[k];
        if (g_rgb)
            g_rgb[k] = ea * gx[k];
    }
    if (g_ab) {
        g_ab[0] = ga;
        g_ab[1] = gb;
    }
    free(x);
    free(gx);
    return L;
}

/* One Adam step on the exposure (a, b): the pose's moments and cosine
 * schedule (hyper as in or_pose_step) with learning rate lr_exposure;
 * state[5] = m_a, m_b, v_a, v_b, steps taken. */
static void exposure_step(double *ab, double *state, const double *g, const double *hyper, double lr_exposure, int k,
                          int iters)
{
    const double b1 = hyper[2], b2 = hyper[3], eps = hyper[4], f = hyper[5];
    const double t = state[4] + 1.0;
    state[4] = t;
    const double sched = f + (1.0 - f) * 0.5 * (1.0 + cos(M_PI * (double)k / (double)iters));
    for (int i = 0; i < 2; ++i) {
        state[i] = b1 * state[i] + (1.0 - b1) * g[i];
        state[2 + i] = b2 * state[2 + i] + (1.0 - b2) * g[i] * g[i];
        const double mh = state[i] / (1.0 - pow(b1, t));
        const double vh = state[2 + i] / (1.0 - pow(b2, t));
        ab[i] -= lr_exposure * sched * mh / (sqrt(vh) + eps);
    }
}

static int cmp_float(const void *a, const void *b)
{
    const float x = *(const float *)a, y = *(const float *)b;
    return (x > y) - (x < y);
}

/* Frame-to-model tracking loss of one view (Eq. 2, masks of Supp. A):
 *   L = sum over pixels of M_in * M_a * (lambda_c |I^ - I|_1 + (1 - lambda_c) |D^ - D|)
 * with |.|_1 over the three colour channels, M_a = alpha^3 (alpha = 1 - final
 * transmittance; a weight, not differentiated), and the inlier mask M_in:
 * pixels with a valid input depth (D > 0) whose depth error e = |D^ - D| is at
 * most 50 times the median depth error over the valid pixels.  The median is
 * the lower one (rank floor((m - 1) / 2) of the m valid errors); e and the
 * threshold are taken in FP32 from the FP32 mirror of the rendered depth
 * (depth32), as the kernels take them, so that the inlier decisions are
 * exact.  Writes g_rgb = dL/dI^ and g_depth = dL/dD^ (mask held fixed;
 * sign(0) = 0), inlier[HW] (1/0) and *median when the pointers are not NULL.
 * Returns L, or NaN when out of memory. */
double or_track_loss(int H, int W, const double *rgb, const double *depth, const double *tf,
                     const float *depth32, const float *t_rgb, const float *t_depth, double lambda_c,
                     double *g_rgb, double *g_depth, int8_t *inlier, float *median)
{
    const long HW = (long)H * W;
    float *e = malloc((size_t)(HW > 0 ? HW : 1) * sizeof(float));
    float *sorted = malloc((size_t)(HW > 0 ? HW : 1) * sizeof(float));
    if (!e || !sorted) {
        free(e);
        free(sorted);
        return NAN;
    }
    long m = 0;
    for (long k = 0; k < HW; ++k) {
        e[k] = fabsf(depth32[k] - t_depth[k]);
        if (t_depth[k] > 0.0f)
            sorted[m++] = e[k];
    }
    qsort(sorted, (size_t)m, sizeof(float), cmp_float);
    const float med = m > 0 ? sorted[(m - 1) / 2] : 0.0f;
    const float thr = 50.0f * med;
    if (median)
        *median = med;
    double L = 0.0;
    for (long k = 0; k < HW; ++k) {
        const int in = m > 0 && t_depth[k] > 0.0f && e[k] <= thr;
        if (inlier)
            inlier[k] = (int8_t)in;
        const double a = 1.0 - tf[k];
        const double w = in ? a * a * a : 0.0;
        double lc = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            const double d = rgb[ch * HW + k] - (double)t_rgb[ch * HW + k];
            lc += fabs(d);
            if (g_rgb)
                g_rgb[ch * HW + k] = w * lambda_c * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0));
        }
        const double dd = depth[k] - (double)t_depth[k];
        if (g_depth)
            g_depth[k] = w * (1.0 - lambda_c) * (dd > 0 ? 1.0 : (dd < 0 ? -1.0 : 0.0));
        L += w * (lambda_c * lc + (1.0 - lambda_c) * fabs(dd));
    }
    free(e);
    free(sorted);
    return L;
}

/* Adjoint of or_render for given cotangents (any may be NULL).  twist[6]
 * (may be NULL) receives dL/d(omega, v) of a left perturbation of the pose
 * about pivot[3]; the parameter gradients (each may be NULL) are ADDED to:
 * g_means[n][3], g_scales[n][3] (log-scales), g_quats[n][4], g_logits[n],
 * g_rgb[n][3]. */
int or_backward(int n, const float *means4, const float *scales4, const float *quats4, const float *logits,
                const float *rgb4, const double *pose, const float *cam, const float *opt,
                const double *cot_rgb, const double *cot_depth, const double *cot_alpha,
                const double *pivot, double *twist, double *g_means, double *g_scales, double *g_quats,
                double *g_logits, double *g_rgb)
{
    opts_t op;
    read_opts(opt, &op);
    if (n < 0 || !check_cam(cam, &op))
        return OR_ERR_ARG;
    prep_t p;
    int st = prep_camera(n, means4, scales4, quats4, logits, pose, cam, &op, &p);
    double *acc = NULL;
    if (st == OR_OK) {
        acc = calloc((size_t)(n > 0 ? n : 1) * G_N, sizeof(double));
        if (!acc)
            st = OR_ERR_OOM;
    }
    if (st == OR_OK)
        st = adjoint_screen(&p, &op, rgb4, cot_rgb, cot_depth, cot_alpha, acc);
    if (st == OR_OK) {
        double zero[3] = {0, 0, 0};
        if (twist)
            memset(twist, 0, 6 * sizeof(double));
        chain(&p, pose, cam, acc, pivot ? pivot : zero, logits, twist, g_means, g_scales, g_quats,
              g_logits, g_rgb);
    }
    free(acc);
    prep_free(&p);
    return st;
}

/* ------------------------------------------------------------------------ */
/* pose update and registration                                              */
/* ------------------------------------------------------------------------ */

/* Rodrigues: R = exp([w]x) */
static void so3_exp(const double w[3], double R[3][3])
{
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double a, b;
    if (th < 1e-8) {
        a = 1.0 - th2 / 6.0;
        b = 0.5 - th2 / 24.0;
    } else {
        a = sin(th) / th;
        b = (1.0 - cos(th)) / th2;
    }
    double K[3][3] = {{0, -w[2], w[1]}, {w[2], 0, -w[0]}, {-w[1], w[0], 0}}, K2[3][3];
    mat3_mul(K, K, K2);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            R[i][j] = (i == j ? 1.0 : 0.0) + a * K[i][j] + b * K2[i][j];
}

/* The moving centroid mu_bar of the submap (pivot = R mu_bar + t). */
static void centroid(int n, const float *means4, double mbar[3])
{
    double s[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k)
            s[k] += means4[4 * i + k];
    for (int k = 0; k < 3; ++k)
        mbar[k] = n > 0 ? s[k] / n : 0.0;
}

/* One Adam step on the twist and the pose update about the pivot.
 * hyper[6] = {lr_rot, lr_trans, beta1, beta2, eps, final_lr_fraction};
 * state[13] = {m[6], v[6], step count}; k = iteration index in [0, iters).
 * The learning rate follows a cosine from 1 to final_lr_fraction. */
int or_pose_step(double *pose, double *state, const double *grad, const double *pivot,
                 const double *hyper, int k, int iters)
{
    if (iters <= 0 || k < 0)
        return OR_ERR_ARG;
    const double b1 = hyper[2], b2 = hyper[3], eps = hyper[4], f = hyper[5];
    double *m = state, *v = state + 6;
    double t = state[12] + 1.0;
    state[12] = t;
    double sched = f + (1.0 - f) * 0.5 * (1.0 + cos(M_PI * (double)k / (double)iters));
    double xi[6];
    for (int i = 0; i < 6; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        double mh = m[i] / (1.0 - pow(b1, t));
        double vh = v[i] / (1.0 - pow(b2, t));
        double lr = (i < 3 ? hyper[0] : hyper[1]) * sched;
        xi[i] = -lr * mh / (sqrt(vh) + eps);
    }
    double R[3][3], tt[3], dR[3][3], Rn[3][3];
    rot_of(pose, R, tt);
    so3_exp(xi, dR);
    mat3_mul(dR, R, Rn);
    double rel[3] = {tt[0] - pivot[0], tt[1] - pivot[1], tt[2] - pivot[2]};
    for (int i = 0; i < 3; ++i) {
        double tn = dR[i][0] * rel[0] + dR[i][1] * rel[1] + dR[i][2] * rel[2] + pivot[i] + xi[3 + i];
        for (int j = 0; j < 3; ++j)
            pose[4 * i + j] = Rn[i][j];
        pose[4 * i + 3] = tn;
    }
    return OR_OK;
}

/* Registration of one keyframe (Sec. 3.2): optimises the rigid transform
 * applied to the moving submap so that its render at the keyframe camera
 * matches the keyframe's colour and depth.  pose (in/out) starts at the
 * given value; eps_out = loss at the final pose; loss_hist[iters] (may be
 * NULL) records the loss at each iteration before its update.  track NULL:
 * the registration loss (or_loss); otherwise the tracking loss of Eq. 2
 * (or_track_loss) with lambda_c = track[0].  expo NULL: no exposure
 * compensation; otherwise the keyframe's exposure (a, b), starting at 0, is
 * optimised with the pose at learning rate expo[0] (or_exposure_loss;
 * registration loss only) and returned in ab_out[2] (may be NULL). */
int or_register_view(int n, const float *means4, const float *scales4, const float *quats4,
                     const float *logits, const float *rgb4, const float *cam, const float *opt,
                     const float *t_rgb, const float *t_depth, const double *hyper, int iters,
                     double *pose, double *eps_out, double *loss_hist, const double *track, const double *expo,
                     double *ab_out)
{
    opts_t op;
    read_opts(opt, &op);
    if (n < 0 || iters < 0 || !check_cam(cam, &op) || (track && expo))
        return OR_ERR_ARG;
    double ab[2] = {0.0, 0.0}, ab_state[5] = {0, 0, 0, 0, 0}, gab[2] = {0.0, 0.0};
    const int W = (int)cam[4], H = (int)cam[5];
    const long HW = (long)W * H;
    double *rgb = malloc((size_t)HW * 3 * sizeof(double));
    double *dep = malloc((size_t)HW * sizeof(double));
    double *grgb = malloc((size_t)HW * 3 * sizeof(double));
    double *gdep = malloc((size_t)HW * sizeof(double));
    double *acc = calloc((size_t)(n > 0 ? n : 1) * G_N, sizeof(double));
    double *trgb = malloc((size_t)HW * 3 * sizeof(double));
    double *tdep = malloc((size_t)HW * sizeof(double));
    double *tf = malloc((size_t)HW * sizeof(double));
    float *dep32 = malloc((size_t)HW * sizeof(float));
    int st = (rgb && dep && grgb && gdep && acc && trgb && tdep && tf && dep32) ? OR_OK : OR_ERR_OOM;
    for (long k = 0; st == OR_OK && k < 3 * HW; ++k)
        trgb[k] = t_rgb[k];
    for (long k = 0; st == OR_OK && k < HW; ++k)
        tdep[k] = t_depth[k];
    double mbar[3], state[13] = {0};
    centroid(n, means4, mbar);
    for (int k = 0; k <= iters && st == OR_OK; ++k) {
        prep_t p;
        st = prep_camera(n, means4, scales4, quats4, logits, pose, cam, &op, &p);
        if (st == OR_OK) {
            composite(&p, &op, rgb4, rgb, dep, NULL, tf, NULL, NULL, dep32);
            double L = track  ? or_track_loss(H, W, rgb, dep, tf, dep32, t_rgb, t_depth, track[0], grgb, gdep, NULL,
                                              NULL)
                       : expo ? or_exposure_loss(H, W, rgb, dep, trgb, tdep, ab, grgb, gdep, gab)
                              : or_loss(H, W, rgb, dep, trgb, tdep, grgb, gdep);
            if (L != L)
                st = OR_ERR_OOM;
            if (k == iters) {
                *eps_out = L;
            } else {
                if (loss_hist)
                    loss_hist[k] = L;
                memset(acc, 0, (size_t)(n > 0 ? n : 1) * G_N * sizeof(double));
                st = adjoint_screen(&p, &op, rgb4, grgb, gdep, NULL, acc);
                if (st == OR_OK) {
                    double R[3][3], t[3], c[3], tw[6] = {0};
                    rot_of(pose, R, t);
                    for (int i = 0; i < 3; ++i)
                        c[i] = R[i][0] * mbar[0] + R[i][1] * mbar[1] + R[i][2] * mbar[2] + t[i];
                    chain(&p, pose, cam, acc, c, logits, tw, NULL, NULL, NULL, NULL, NULL);
                    or_pose_step(pose, state, tw, c, hyper, k, iters);
                    if (expo)
                        exposure_step(ab, ab_state, gab, hyper, expo[0], k, iters);
                }
            }
        }
        prep_free(&p);
    }
    free(rgb);
    free(dep);
    free(grgb);
    free(gdep);
    free(acc);
    free(trgb);
    free(tdep);
    free(tf);
    free(dep32);
    if (ab_out) {
        ab_out[0] = ab[0];
        ab_out[1] = ab[1];
    }
    return st;
}

/* Rigid transform of a submap (Eq. 8 / Eq. 9): mu <- R mu + t and
 * Sigma <- R Sigma R^T, the latter by rotating each Gaussian's frame:
 * R(q') = R R(q), q' read back from the rotated matrix.  Scales, opacities
 * and colours are unchanged.  Outputs are float [n][4] (w unused = 0 for
 * means; quaternion as w, x, y, z with w >= 0). */
int or_transform(int n, const float *means4, const float *quats4, const double *T, float *out_means4,
                 float *out_quats4)
{
    double R[3][3], t[3];
    rot_of(T, R, t);
    for (int i = 0; i < n; ++i) {
        const float *mu = means4 + 4 * i;
        for (int k = 0; k < 3; ++k)
            out_means4[4 * i + k] = (float)(R[k][0] * mu[0] + R[k][1] * mu[1] + R[k][2] * mu[2] + t[k]);
        out_means4[4 * i + 3] = 0.0f;
        const float *q = quats4 + 4 * i;
        double ql = sqrt((double)q[0] * q[0] + (double)q[1] * q[1] + (double)q[2] * q[2] + (double)q[3] * q[3]);
        double qn[4] = {q[0] / ql, q[1] / ql, q[2] / ql, q[3] / ql}, Rq[3][3], M[3][3];
        quat_to_rot(qn, Rq);
        mat3_mul(R, Rq, M);
        /* matrix -> quaternion (largest-diagonal branch for stability) */
        double tr = M[0][0] + M[1][1] + M[2][2], w, x, y, z;
        if (tr > 0) {
            double s = sqrt(tr + 1.0) * 2;
            w = 0.25 * s;
            x = (M[2][1] - M[1][2]) / s;
            y = (M[0][2] - M[2][0]) / s;
            z = (M[1][0] - M[0][1]) / s;
        } else if (M[0][0] > M[1][1] && M[0][0] > M[2][2]) {
            double s = sqrt(1.0 + M[0][0] - M[1][1] - M[2][2]) * 2;
            w = (M[2][1] - M[1][2]) / s;
            x = 0.25 * s;
            y = (M[0][1] + M[1][0]) / s;
            z = (M[0][2] + M[2][0]) / s;
        } else if (M[1][1] > M[2][2]) {
            double s = sqrt(1.0 + M[1][1] - M[0][0] - M[2][2]) * 2;
            w = (M[0][2] - M[2][0]) / s;
            x = (M[0][1] + M[1][0]) / s;
            y = 0.25 * s;
            z = (M[1][2] + M[2][1]) / s;
        } else {
            double s = sqrt(1.0 + M[2][2] - M[0][0] - M[1][1]) * 2;
            w = (M[1][0] - M[0][1]) / s;
            x = (M[0][2] + M[2][0]) / s;
            y = (M[1][2] + M[2][1]) / s;
            z = 0.25 * s;
        }
        if (w < 0) {
            w = -w; x = -x; y = -y; z = -z;
        }
        out_quats4[4 * i + 0] = (float)w;
        out_quats4[4 * i + 1] = (float)x;
        out_quats4[4 * i + 2] = (float)y;
        out_quats4[4 * i + 3] = (float)z;
    }
    return OR_OK;
}

/* ======================================================================== */
/* overlap ratio (loop filter, Supp.: reciprocal closest-point matching)     */
/* ======================================================================== */

/* p' = R p + t in FP32, fused multiply-adds translation first (the
 * projection's convention); T is [R|t] rounded to FP32 */
static void rigid32(const float T[12], const float *p, float *out)
{
    for (int i = 0; i < 3; ++i)
        out[i] = fmaf(T[4 * i + 2], p[2], fmaf(T[4 * i + 1], p[1], fmaf(T[4 * i], p[0], T[4 * i + 3])));
}

/* squared distance in FP32: dx = b - a per axis, fma(dz, dz, fma(dy, dy, dx*dx)) */
static float dist2_32(const float *a, const float *b)
{
    const float dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

/* nearest neighbour of each of the na points a (xyz, stride 4) among the nb
 * points b: the smallest FP32 squared distance, ties to the smaller index;
 * -1 if nb = 0 */
static void nearest(const float *a, int na, const float *b, int nb, int32_t *nn, float *d2)
{
    for (int i = 0; i < na; ++i) {
        float best = INFINITY;
        int32_t bi = -1;
        for (int j = 0; j < nb; ++j) {
            const float d = dist2_32(a + 4 * (size_t)i, b + 4 * (size_t)j);
            if (d < best) {
                best = d;
                bi = j;
            }
        }
        nn[i] = bi;
        if (d2)
            d2[i] = best;
    }
}

/* Overlap ratio of submaps P and Q under T = T_{P->Q} (the loop filter of
 * the supplement): the means of P are moved by T (FP32, rigid32), K is the
 * set of reciprocal nearest-neighbour pairs (p, q) -- q the nearest of T p
 * in Q and T p the nearest of q in T P -- and OR is the fraction of K with
 * |T p - q| < tau, decided as d2 < tau * tau in FP32.  Writes nn_pq[np],
 * nn_qp[nq] (may be NULL) and *n_corr = |K|; returns OR (0 when K is
 * empty), or -1 when out of memory. */
double or_overlap_ratio(int np, const float *p_means4, int nq, const float *q_means4, const double *T, float tau,
                        int32_t *nn_pq_out, int32_t *nn_qp_out, long *n_corr)
{
    float T32[12];
    for (int k = 0; k < 12; ++k)
        T32[k] = (float)T[k];
    float *pt = malloc((size_t)(np > 0 ? np : 1) * 4 * sizeof(float));
    int32_t *pq = malloc((size_t)(np > 0 ? np : 1) * sizeof(int32_t));
    int32_t *qp = malloc((size_t)(nq > 0 ? nq : 1) * sizeof(int32_t));
    float *d2 = malloc((size_t)(np > 0 ? np : 1) * sizeof(float));
    if (!pt || !pq || !qp || !d2) {
        free(pt);
        free(pq);
        free(qp);
        free(d2);
        return -1.0;
    }
    for (int i = 0; i < np; ++i) {
        rigid32(T32, p_means4 + 4 * (size_t)i, pt + 4 * (size_t)i);
        pt[4 * (size_t)i + 3] = 0.0f;
    }
    nearest(pt, np, q_means4, nq, pq, d2);
    nearest(q_means4, nq, pt, np, qp, NULL);
    const float tau2 = tau * tau;
    long k = 0, in = 0;
    for (int i = 0; i < np; ++i) {
        const int32_t j = pq[i];
        if (j >= 0 && qp[j] == i) {
            ++k;
            if (d2[i] < tau2)
                ++in;
        }
    }
    if (nn_pq_out)
        memcpy(nn_pq_out, pq, (size_t)np * sizeof(int32_t));
    if (nn_qp_out)
        memcpy(nn_qp_out, qp, (size_t)nq * sizeof(int32_t));
    if (n_corr)
        *n_corr = k;
    free(pt);
    free(pq);
    free(qp);
    free(d2);
    return k > 0 ? (double)in / (double)k : 0.0;
}

/* nearest neighbours in Q of a subset of P's moved means (for parity checks
 * at full size): idx[m] indices into P; writes nn[m] */
int or_nearest_subset(int np, const float *p_means4, int nq, const float *q_means4, const double *T, int m,
                      const int32_t *idx, int32_t *nn)
{
    float T32[12], pt[4];
    for (int k = 0; k < 12; ++k)
        T32[k] = (float)T[k];
    for (int s = 0; s < m; ++s) {
        if (idx[s] < 0 || idx[s] >= np)
            return OR_ERR_ARG;
        rigid32(T32, p_means4 + 4 * (size_t)idx[s], pt);
        pt[3] = 0.0f;
        nearest(pt, 1, q_means4, nq, nn + s, NULL);
    }
    return OR_OK;
}

/* the FP32 moved means of the overlap ratio (rigid32), [n][4] with w = 0 */
int or_moved_means(int n, const float *means4, const double *T, float *out4)
{
    float T32[12];
    for (int k = 0; k < 12; ++k)
        T32[k] = (float)T[k];
    for (int i = 0; i < n; ++i) {
        rigid32(T32, means4 + 4 * (size_t)i, out4 + 4 * (size_t)i);
        out4[4 * (size_t)i + 3] = 0.0f;
    }
    return OR_OK;
}
