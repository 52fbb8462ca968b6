/*
 * FP64 CPU oracle for delivery-state rendering of a dynamic Gaussian scene.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  It shares no code with the
 * CUDA library: it is a plain, slow, literal statement of what the renderer
 * computes, in double precision, one Gaussian and one pixel at a time.
 *
 * What the paper fixes (cited by section / equation of the paper):
 *   - Section 3: N fixed-identity Gaussians grouped in clusters; every cluster
 *     has one base completion group and three refinement groups; scale,
 *     rotation, opacity and colour are "base plus learned refinements"; every
 *     dependency-closed subset decodes to a valid scene.
 *   - Eq. 1: mu_{i,t} = A_{c,t} mubar_i + sum_r b_{t,r} q_{i,r} + delta2 + delta3.
 *     The cluster affine A_{c,t} is the identity here (the temporal low-rank
 *     term and the two residual levels are kept).
 *   - Section 4 and Section 7.4: packet dependencies are enforced after
 *     delivery (a chunk is usable only when its whole dependency closure is
 *     usable), then turned into cluster-layer masks.
 *   - Section 6: many delivery states of one scene are rasterized in one batch;
 *     the abstract states batched evaluation equals serial evaluation.
 *   - Eq. 3: the distortion D between the state's render and the reference.
 * The paper delegates rasterization to an external EWA-splatting library and
 * does not describe it.  The rasterizer below is the published EWA-splatting
 * formulation (Zwicker et al.; Kerbl et al. 2023) written out from the
 * mathematics with these readings (all are listed in the design notes):
 *   closure = leading delivered layers per cluster; depth 0 = cluster absent;
 *   OpenCV pinhole; near plane z <= 0.01 culled; Jacobian evaluated with x/z,
 *   y/z clamped to +-1.3 * (W/2)/fx, (H/2)/fy; 2D covariance dilated by 0.3 px^2;
 *   radius r = ceil(3 sqrt(lambda_max)); a Gaussian touches pixel p iff
 *   |p_centre - m| <= r on both axes; power > 0 skipped;
 *   alpha = min(0.99, o e^power), skipped below 1/255; a pixel stops before the
 *   Gaussian that would bring T below 1e-4; order = (float32 depth, index);
 *   colour = max(rgb, 0) (degree 0) or max(SH(dir) + 0.5, 0) (degree 3).
 *
 * Marginal bookkeeping: every threshold above is a discontinuity.  When an
 * FP64 quantity lies within a small tolerance of a threshold the pixel is
 * flagged "marginal"; an FP32 implementation may legitimately decide such a
 * case the other way, so comparisons exclude flagged pixels and report them.
 *
 * Parity pins for every function here live in the CPU test-suite: closed
 * forms (single and double Gaussian composites, on-axis EWA covariance,
 * in-plane rotation), brute force (row-filtered vs full-scan compositing,
 * tile lists), invariants (empty/full delivery, undelivered packets, temporal
 * period) and central finite differences of the adjoint.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int32_t n, n_clusters, n_layers, sh_degree, temporal_rank;
    const int32_t *cluster_offsets;   /* [C+1] */
    const float *mu0;                 /* [n][3] */
    const float *u;                   /* [R][n][3] */
    const float *log_scale;           /* [n][3] */
    const float *quat;                /* [n][4] w,x,y,z */
    const float *opacity_logit;       /* [n] */
    const float *colour;              /* [n][nc] */
    const float *res;                 /* [L-1][n][11+nc] */
    const float *affine;              /* [C][T][12] cluster affine keyframes of Eq. 1, or NULL (identity) */
    int32_t affine_T;                 /* keyframes per cluster, keyframe k at time k / T (period 1) */
    const int16_t *res_q;             /* [L-1][n][K] quantized refinement symbols (res_mode 1) */
    const float *res_step;            /* [L-1][K] quantization steps (res_mode 1 and 2) */
    int32_t res_mode;                 /* 0: res as given; 1: res_q * step; 2: res quantized to step */
} OScene;

typedef struct {
    double R[9], t[3], fx, fy, cx, cy;
    int32_t width, height;
} OCam;

typedef struct {            /* tolerances of the marginal rule */
    double box_px;          /* |dist - r| below this (pixels) */
    double rel_alpha;       /* relative distance of alpha to 1/255 and 0.99 */
    double rel_T;           /* relative distance of T(1-alpha) to 1e-4 */
    double rel_depth;       /* relative depth gap between neighbours */
    double rel_radius;      /* 3 sqrt(lambda) relative distance to an integer */
    double near_abs;        /* |z - 0.01| below this */
} OEps;

static const OEps kDefaultEps = {2e-3, 1e-4, 1e-4, 4e-7, 1e-5, 1e-6};

enum { REC_W = 20 };
/* Projected record of one present Gaussian (FP64). */
typedef struct {
    int valid;
    int idx;
    double mx, my, A, B, Cc, z, o, rgb[3], r;
    int xlo, xhi, ylo, yhi;       /* exact pixel box (clamped to the image) */
    int marg_rad, marg_near;
    int has_proj;                 /* projection computed (z > 0, det > 0) */
    float z32;
} ORec;

static int n_colour(const OScene *s) { return 3 * (s->sh_degree + 1) * (s->sh_degree + 1); }
static int res_width(const OScene *s) { return 11 + n_colour(s); }

/* ---- Section 4 / 7.4: closure of a raw delivery mask into delivered depths ---- */
void o_closure(int C, int L, const uint32_t *mask, uint8_t *depth)
{
    for (int c = 0; c < C; ++c) {
        int d = 0;
        while (d < L) {
            int b = c * L + d;
            if (!((mask[b >> 5] >> (b & 31)) & 1u)) break;   /* layer d unusable: stop */
            ++d;
        }
        depth[c] = (uint8_t)d;
    }
}

/* ---- Section 3: base plus the delivered refinements l = 1..d-1 ---- */
typedef struct { double mu[3], ls[3], q[4], logit, col[48]; } OAttr;

/* Quantization of a refinement value to step st (the learned steps of
 * Section 3): the signed 16-bit symbol v = round(x / st) (x / st in FP32, ties
 * to even), clipped to [-32768, 32767]; returns v and whether it was clipped. */
static double quant_symbol(float x, float st, int *clipped)
{
    float u = x / st;
    double v = rint((double)u);
    *clipped = 0;
    if (v > 32767.0) { v = 32767.0; *clipped = 1; }
    if (v < -32768.0) { v = -32768.0; *clipped = 1; }
    return v;
}

/* Component k of refinement layer l (1-based) of Gaussian i as decoded. */
static double res_value(const OScene *s, int l, int i, int k)
{
    int K = res_width(s);
    size_t o = ((size_t)(l - 1) * s->n + i) * K + k;
    if (s->res_mode == 1) return (double)s->res_q[o] * (double)s->res_step[(size_t)(l - 1) * K + k];
    if (s->res_mode == 2) {
        int cl;
        float st = s->res_step[(size_t)(l - 1) * K + k];
        return quant_symbol(s->res[o], st, &cl) * (double)st;
    }
    return s->res[o];
}

static void decode(const OScene *s, int i, int d, OAttr *a)
{
    int nc = n_colour(s);
    for (int k = 0; k < 3; ++k) { a->mu[k] = s->mu0[3 * i + k]; a->ls[k] = s->log_scale[3 * i + k]; }
    for (int k = 0; k < 4; ++k) a->q[k] = s->quat[4 * i + k];
    a->logit = s->opacity_logit[i];
    for (int k = 0; k < nc; ++k) a->col[k] = s->colour[(size_t)nc * i + k];
    for (int l = 1; l < d; ++l) {
        for (int k = 0; k < 3; ++k) { a->mu[k] += res_value(s, l, i, k); a->ls[k] += res_value(s, l, i, 3 + k); }
        for (int k = 0; k < 4; ++k) a->q[k] += res_value(s, l, i, 6 + k);
        a->logit += res_value(s, l, i, 10);
        for (int k = 0; k < nc; ++k) a->col[k] += res_value(s, l, i, 11 + k);
    }
}

/* Cluster affine A_{c,t} of Eq. 1 (3x4, row-major: linear part | translation):
 * keyframe k of cluster c holds A at time k / T; between keyframes the twelve
 * entries are interpolated linearly, periodically in t with period 1.  Returns
 * the keyframes used (k0, k1) and the weight w of k1 (NULL affine: identity). */
static void affine_at(const OScene *s, int c, double t, double A[12], int *k0, int *k1, double *w)
{
    if (!s->affine) {
        for (int k = 0; k < 12; ++k) A[k] = (k == 0 || k == 5 || k == 10) ? 1.0 : 0.0;
        *k0 = *k1 = -1; *w = 0.0;
        return;
    }
    int T = s->affine_T;
    double u = t * T;
    double fl = floor(u);
    *w = u - fl;
    long kk = (long)fl % T;
    if (kk < 0) kk += T;
    *k0 = (int)kk; *k1 = (int)((kk + 1) % T);
    const float *a0 = s->affine + ((size_t)c * T + *k0) * 12, *a1 = s->affine + ((size_t)c * T + *k1) * 12;
    for (int k = 0; k < 12; ++k) A[k] = (1.0 - *w) * a0[k] + *w * a1[k];
}

static int cluster_of_idx(const OScene *s, int i)
{
    int c = 0;
    while (!(i >= s->cluster_offsets[c] && i < s->cluster_offsets[c + 1])) ++c;
    return c;
}

/* Shared temporal basis of Eq. 1: b_{2j-1}(t) = cos(2 pi j t), b_{2j}(t) = sin(2 pi j t). */
static double basis(int k, double t)
{
    int j = k / 2 + 1;
    return (k % 2 == 0) ? cos(2.0 * M_PI * j * t) : sin(2.0 * M_PI * j * t);
}

/* Real spherical harmonics of degree <= 3 on a unit direction (orthonormal on
 * the sphere), order (l, m) = (0,0), (1,-1), (1,0), (1,1), (2,-2) ... (3,3). */
void o_sh_basis(const double *d, int deg, double *Y)
{
    double x = d[0], y = d[1], z = d[2];
    Y[0] = 0.5 * sqrt(1.0 / M_PI);
    if (deg < 1) return;
    double k1 = sqrt(3.0 / (4.0 * M_PI));
    Y[1] = k1 * y; Y[2] = k1 * z; Y[3] = k1 * x;
    if (deg < 2) return;
    double k2a = 0.5 * sqrt(15.0 / M_PI), k2b = 0.25 * sqrt(5.0 / M_PI), k2c = 0.25 * sqrt(15.0 / M_PI);
    Y[4] = k2a * x * y; Y[5] = k2a * y * z; Y[6] = k2b * (3.0 * z * z - 1.0);
    Y[7] = k2a * x * z; Y[8] = k2c * (x * x - y * y);
    if (deg < 3) return;
    double k3a = 0.25 * sqrt(35.0 / (2.0 * M_PI)), k3b = 0.5 * sqrt(105.0 / M_PI);
    double k3c = 0.25 * sqrt(21.0 / (2.0 * M_PI)), k3d = 0.25 * sqrt(7.0 / M_PI);
    double k3e = 0.25 * sqrt(105.0 / M_PI);
    Y[9] = k3a * y * (3.0 * x * x - y * y);
    Y[10] = k3b * x * y * z;
    Y[11] = k3c * y * (5.0 * z * z - 1.0);
    Y[12] = k3d * z * (5.0 * z * z - 3.0);
    Y[13] = k3c * x * (5.0 * z * z - 1.0);
    Y[14] = k3e * z * (x * x - y * y);
    Y[15] = k3a * x * (x * x - 3.0 * y * y);
}

/* Partial derivatives dY_j / d(x,y,z) of the polynomials above (treating x,y,z
 * as free variables; the caller projects onto the sphere's tangent plane). */
static void sh_basis_grad(const double *d, int deg, double (*dY)[3])
{
    double x = d[0], y = d[1], z = d[2];
    memset(dY, 0, sizeof(double) * 3 * 16);
    if (deg < 1) return;
    double k1 = sqrt(3.0 / (4.0 * M_PI));
    dY[1][1] = k1; dY[2][2] = k1; dY[3][0] = k1;
    if (deg < 2) return;
    double k2a = 0.5 * sqrt(15.0 / M_PI), k2b = 0.25 * sqrt(5.0 / M_PI), k2c = 0.25 * sqrt(15.0 / M_PI);
    dY[4][0] = k2a * y; dY[4][1] = k2a * x;
    dY[5][1] = k2a * z; dY[5][2] = k2a * y;
    dY[6][2] = k2b * 6.0 * z;
    dY[7][0] = k2a * z; dY[7][2] = k2a * x;
    dY[8][0] = k2c * 2.0 * x; dY[8][1] = -k2c * 2.0 * y;
    if (deg < 3) return;
    double k3a = 0.25 * sqrt(35.0 / (2.0 * M_PI)), k3b = 0.5 * sqrt(105.0 / M_PI);
    double k3c = 0.25 * sqrt(21.0 / (2.0 * M_PI)), k3d = 0.25 * sqrt(7.0 / M_PI);
    double k3e = 0.25 * sqrt(105.0 / M_PI);
    dY[9][0] = k3a * 6.0 * x * y; dY[9][1] = k3a * (3.0 * x * x - 3.0 * y * y);
    dY[10][0] = k3b * y * z; dY[10][1] = k3b * x * z; dY[10][2] = k3b * x * y;
    dY[11][1] = k3c * (5.0 * z * z - 1.0); dY[11][2] = k3c * 10.0 * y * z;
    dY[12][2] = k3d * (15.0 * z * z - 3.0);
    dY[13][0] = k3c * (5.0 * z * z - 1.0); dY[13][2] = k3c * 10.0 * x * z;
    dY[14][0] = k3e * 2.0 * x * z; dY[14][1] = -k3e * 2.0 * y * z; dY[14][2] = k3e * (x * x - y * y);
    dY[15][0] = k3a * (3.0 * x * x - 3.0 * y * y); dY[15][1] = -k3a * 6.0 * x * y;
}

static void quat_to_rot(const double *q, double *R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Forward quantities of one present Gaussian kept for the adjoint. */
typedef struct {
    OAttr a;
    double mu[3], p[3], qn[4], qnorm, Rq[9], S[3], M[9], S3[9], J[6], T[6];
    double a2, b2, c2, det, campos[3], dir[3], dist, shv[3];
    int clampx, clampy;
} OFwd;

static void camera_centre(const OCam *cam, double *c)
{
    for (int k = 0; k < 3; ++k)
        c[k] = -(cam->R[0 + k] * cam->t[0] + cam->R[3 + k] * cam->t[1] + cam->R[6 + k] * cam->t[2]);
}

/* Eq. 1 deformation + EWA projection of Gaussian i at delivered depth d (>= 1). */
static void project_one(const OScene *s, int i, int d, double t, const OCam *cam,
                        const OEps *eps, ORec *rec, OFwd *f)
{
    OFwd local;
    if (!f) f = &local;
    memset(rec, 0, sizeof(*rec));
    rec->idx = i;
    decode(s, i, d, &f->a);
    if (s->affine) {   /* Eq. 1: A_{c,t} mubar + (delivered position residuals) */
        double A[12], w;
        int k0, k1;
        affine_at(s, cluster_of_idx(s, i), t, A, &k0, &k1, &w);
        const float *m0 = s->mu0 + 3 * i;
        for (int k = 0; k < 3; ++k)
            f->mu[k] = A[4 * k] * m0[0] + A[4 * k + 1] * m0[1] + A[4 * k + 2] * m0[2] + A[4 * k + 3] +
                       (f->a.mu[k] - m0[k]);
    } else {
        for (int k = 0; k < 3; ++k) f->mu[k] = f->a.mu[k];
    }
    for (int r = 0; r < s->temporal_rank; ++r) {
        double b = basis(r, t);
        for (int k = 0; k < 3; ++k) f->mu[k] += b * s->u[((size_t)r * s->n + i) * 3 + k];
    }
    for (int k = 0; k < 3; ++k)
        f->p[k] = cam->R[3 * k] * f->mu[0] + cam->R[3 * k + 1] * f->mu[1] + cam->R[3 * k + 2] * f->mu[2] + cam->t[k];
    double x = f->p[0], y = f->p[1], z = f->p[2];
    rec->z = z;
    rec->z32 = (float)z;
    rec->marg_near = fabs(z - 0.01) <= eps->near_abs;
    if (!(z > 0)) return;   /* behind the camera: nothing to keep, even for the marginal rule */
    rec->mx = cam->fx * x / z + cam->cx;
    rec->my = cam->fy * y / z + cam->cy;
    /* rotation and scale */
    f->qnorm = sqrt(f->a.q[0] * f->a.q[0] + f->a.q[1] * f->a.q[1] + f->a.q[2] * f->a.q[2] + f->a.q[3] * f->a.q[3]);
    for (int k = 0; k < 4; ++k) f->qn[k] = f->a.q[k] / f->qnorm;
    quat_to_rot(f->qn, f->Rq);
    for (int k = 0; k < 3; ++k) f->S[k] = exp(f->a.ls[k]);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) f->M[3 * r + c] = f->Rq[3 * r + c] * f->S[c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += f->M[3 * r + k] * f->M[3 * c + k];
            f->S3[3 * r + c] = acc;
        }
    /* Jacobian of the pinhole at the (clamped) direction */
    double limx = 1.3 * (0.5 * cam->width) / cam->fx, limy = 1.3 * (0.5 * cam->height) / cam->fy;
    double txz = x / z, tyz = y / z;
    f->clampx = (txz < -limx || txz > limx);
    f->clampy = (tyz < -limy || tyz > limy);
    txz = txz < -limx ? -limx : (txz > limx ? limx : txz);
    tyz = tyz < -limy ? -limy : (tyz > limy ? limy : tyz);
    f->J[0] = cam->fx / z; f->J[1] = 0; f->J[2] = -cam->fx * txz / z;
    f->J[3] = 0; f->J[4] = cam->fy / z; f->J[5] = -cam->fy * tyz / z;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            f->T[3 * r + c] = f->J[3 * r] * cam->R[c] + f->J[3 * r + 1] * cam->R[3 + c] + f->J[3 * r + 2] * cam->R[6 + c];
    double S2[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += f->T[3 * r + k] * f->S3[3 * k + l] * f->T[3 * c + l];
            S2[2 * r + c] = acc;
        }
    f->a2 = S2[0] + 0.3; f->b2 = S2[1]; f->c2 = S2[3] + 0.3;
    f->det = f->a2 * f->c2 - f->b2 * f->b2;
    if (!(f->det > 0)) return;
    rec->A = f->c2 / f->det; rec->B = -f->b2 / f->det; rec->Cc = f->a2 / f->det;
    double mid = 0.5 * (f->a2 + f->c2);
    double disc = mid * mid - f->det;
    double lam = mid + sqrt(disc > 0 ? disc : 0);
    double r3 = 3.0 * sqrt(lam);
    rec->r = ceil(r3);
    double frac = r3 - floor(r3);
    rec->marg_rad = (frac <= eps->rel_radius * r3) || (1.0 - frac <= eps->rel_radius * r3);
    double xl = ceil(rec->mx - rec->r - 0.5), xh = floor(rec->mx + rec->r - 0.5);
    double yl = ceil(rec->my - rec->r - 0.5), yh = floor(rec->my + rec->r - 0.5);
    /* clamp to the image; an off-image box becomes empty (lo > hi) */
    xl = xl < 0 ? 0 : (xl > cam->width ? cam->width : xl);
    yl = yl < 0 ? 0 : (yl > cam->height ? cam->height : yl);
    xh = xh > cam->width - 1 ? cam->width - 1 : (xh < -1 ? -1 : xh);
    yh = yh > cam->height - 1 ? cam->height - 1 : (yh < -1 ? -1 : yh);
    rec->xlo = (int)xl; rec->xhi = (int)xh; rec->ylo = (int)yl; rec->yhi = (int)yh;
    rec->o = 1.0 / (1.0 + exp(-f->a.logit));
    int nc = n_colour(s);
    if (s->sh_degree == 0) {
        for (int k = 0; k < 3; ++k) { f->shv[k] = f->a.col[k]; rec->rgb[k] = f->a.col[k] > 0 ? f->a.col[k] : 0; }
    } else {
        camera_centre(cam, f->campos);
        double v[3], nrm = 0;
        for (int k = 0; k < 3; ++k) { v[k] = f->mu[k] - f->campos[k]; nrm += v[k] * v[k]; }
        f->dist = sqrt(nrm);
        for (int k = 0; k < 3; ++k) f->dir[k] = v[k] / f->dist;
        double Y[16];
        o_sh_basis(f->dir, s->sh_degree, Y);
        int nb = nc / 3;
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0;
            for (int j = 0; j < nb; ++j) acc += Y[j] * f->a.col[3 * j + ch];
            f->shv[ch] = acc + 0.5;
            rec->rgb[ch] = f->shv[ch] > 0 ? f->shv[ch] : 0;
        }
    }
    rec->has_proj = 1;
    /* live: in front of the near plane, positive-definite, non-empty pixel box */
    rec->valid = (z > 0.01) && (rec->xlo <= rec->xhi && rec->ylo <= rec->yhi);
}

/* Exported per-Gaussian projection (FP64) for tests and the tile-list check.
 * out[i*REC_W + ...] = valid, mx, my, A, B, C, z, o, r, g, b, radius,
 * xlo, xhi, ylo, yhi, marg_rad, marg_near, z32 (as double), depth d. */
int o_project(const OScene *s, const uint8_t *depth, double t, const OCam *cam, double *out)
{
    for (int c = 0; c < s->n_clusters; ++c)
        for (int i = s->cluster_offsets[c]; i < s->cluster_offsets[c + 1]; ++i) {
            double *o = out + (size_t)i * REC_W;
            memset(o, 0, sizeof(double) * REC_W);
            int d = depth[c];
            o[19] = d;
            if (d < 1) continue;
            ORec r;
            project_one(s, i, d, t, cam, &kDefaultEps, &r, NULL);
            o[0] = r.valid; o[1] = r.mx; o[2] = r.my; o[3] = r.A; o[4] = r.B; o[5] = r.Cc;
            o[6] = r.z; o[7] = r.o; o[8] = r.rgb[0]; o[9] = r.rgb[1]; o[10] = r.rgb[2];
            o[11] = r.r; o[12] = r.xlo; o[13] = r.xhi; o[14] = r.ylo; o[15] = r.yhi;
            o[16] = r.marg_rad; o[17] = r.marg_near; o[18] = (double)r.z32;
        }
    return 0;
}

static int cmp_rec(const void *pa, const void *pb)
{
    const ORec *a = (const ORec *)pa, *b = (const ORec *)pb;
    if (a->z32 < b->z32) return -1;
    if (a->z32 > b->z32) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* Project every present Gaussian and order by (float32 depth, index). */
static ORec *project_sorted(const OScene *s, const uint8_t *depth, double t, const OCam *cam,
                            const OEps *eps, int *count)
{
    ORec *recs = (ORec *)malloc(sizeof(ORec) * (size_t)(s->n > 0 ? s->n : 1));
    int m = 0;
    for (int c = 0; c < s->n_clusters; ++c) {
        int d = depth[c];
        if (d < 1) continue;
        for (int i = s->cluster_offsets[c]; i < s->cluster_offsets[c + 1]; ++i) {
            ORec r;
            project_one(s, i, d, t, cam, eps, &r, NULL);
            /* dead records that an FP32 evaluation could still keep (near-plane or
               marginal radius) stay in the list for the marginal rule only */
            if (r.valid || (r.has_proj && (r.marg_rad || r.marg_near))) recs[m++] = r;
        }
    }
    qsort(recs, (size_t)m, sizeof(ORec), cmp_rec);
    *count = m;
    return recs;
}

/* One pixel, front to back.  Returns colour in out[3]; sets *marg when any
 * threshold decision was within tolerance; counts evaluated candidates.
 *
 * *bound (when not NULL) receives a bound on how far, per channel, an
 * evaluation that decides the flagged thresholds the other way can move the
 * pixel.  With M bounding every colour behind a decision (the candidates' rgb
 * and |bg|; a composite behind any point is a convex combination of those):
 *   - including or skipping one Gaussian of opacity a at transmittance T
 *     (alpha near 1/255, pixel-box edge, radius rounding, near plane) moves
 *     the pixel by at most a T 2M;
 *   - swapping two adjacent Gaussians i, j (depths within rounding) moves it
 *     by T a_i a_j |rgb_i - rgb_j| <= T a_i a_j 2M (the transmittance after
 *     both is the same);
 *   - stopping one Gaussian earlier or later (T (1 - alpha) near 1e-4) moves it
 *     by at most T 2M, T the transmittance before that Gaussian; earlier
 *     flipped inclusions change T by up to their summed opacities, so the stop
 *     window widens by that sum (a cascaded stop flip);
 *   - the 0.99 clamp is continuous: the pixel does not jump there.
 * The bound is the sum over the pixel's flagged decisions. */
static void shade_pixel(const ORec *recs, const int *list, int nlist, int px, int py,
                        const double *bg, const OEps *eps, double *out, int *marg, int64_t *n_eval,
                        double *bound)
{
    double pcx = px + 0.5, pcy = py + 0.5;
    double T = 1.0, C[3] = {0, 0, 0};
    int mg = 0;
    int64_t ne = 0;
    float prev_z = 0; int have_prev = 0;
    /* colour scale of the bound: |bg| and the rgb of every candidate reaching the pixel */
    double M = 0.0, bnd = 0.0, flip_a = 0.0, T_prev = 1.0, a_prev = 0.0;
    for (int ch = 0; ch < 3; ++ch) M = fabs(bg[ch]) > M ? fabs(bg[ch]) : M;
    for (int k = 0; k < nlist; ++k) {
        const ORec *r = &recs[list[k]];
        if (fabs(pcx - r->mx) <= r->r + 2.0 && fabs(pcy - r->my) <= r->r + 2.0)
            for (int ch = 0; ch < 3; ++ch) M = r->rgb[ch] > M ? r->rgb[ch] : M;
    }
    for (int k = 0; k < nlist; ++k) {
        const ORec *r = &recs[list[k]];
        double ax = fabs(pcx - r->mx), ay = fabs(pcy - r->my);
        double dx = r->mx - pcx, dy = r->my - pcy;
        double pw = -0.5 * (r->A * dx * dx + r->Cc * dy * dy) - r->B * dx * dy;
        double pmag = 0.5 * fabs(r->A * dx * dx) + 0.5 * fabs(r->Cc * dy * dy) + fabs(r->B * dx * dy);
        double araw = r->o * exp(pw);
        int could = (pw <= 1e-5 * pmag) && araw >= (1.0 / 255.0) * (1.0 - eps->rel_alpha);
        double reach = r->r + (r->marg_rad ? 1.0 : 0.0) + eps->box_px;
        if (!r->valid) {
            /* kept for the marginal rule only: an FP32 evaluation may keep it */
            if (ax <= reach && ay <= reach && could && T > 1e-4) {
                mg = 1;
                const double a = araw < 0.99 ? araw : 0.99;
                bnd += a * T * 2.0 * M;
                flip_a += a;
            }
            continue;
        }
        int inside = px >= r->xlo && px <= r->xhi && py >= r->ylo && py <= r->yhi;
        int edge_x = fabs(ax - r->r) <= eps->box_px, edge_y = fabs(ay - r->r) <= eps->box_px;
        if (r->marg_rad) {
            if (ax > r->r - 1 - eps->box_px && ax <= reach) edge_x = 1;
            if (ay > r->r - 1 - eps->box_px && ay <= reach) edge_y = 1;
        }
        int edge = (edge_x && ay <= reach) || (edge_y && ax <= reach) || r->marg_near;
        if (!inside) {
            if (edge && ax <= reach && ay <= reach && could && T > 1e-4) {
                mg = 1;
                const double a = araw < 0.99 ? araw : 0.99;
                bnd += a * T * 2.0 * M;
                flip_a += a;
            }
            continue;
        }
        ++ne;
        if (fabs(pw) <= 1e-5 * pmag && pmag > 0 && araw >= 1.0 / 255.0) {
            mg = 1;                 /* power ~ 0: the sign test may go either way */
            const double a = r->o < 0.99 ? r->o : 0.99;
            bnd += a * T * 2.0 * M;
            flip_a += a;
        }
        if (pw > 0) continue;
        double alpha = araw < 0.99 ? araw : 0.99;
        if (fabs(araw - 0.99) <= eps->rel_alpha * 0.99) mg = 1;
        if (fabs(alpha - 1.0 / 255.0) <= eps->rel_alpha / 255.0) {
            mg = 1;
            const double a = (1.0 / 255.0) * (1.0 + eps->rel_alpha);
            bnd += a * T * 2.0 * M;
            flip_a += a;
        }
        if (alpha < 1.0 / 255.0) continue;
        if (edge) mg = 1;
        if (edge) { bnd += alpha * T * 2.0 * M; flip_a += alpha; }
        if (have_prev && fabs((double)r->z32 - (double)prev_z) <= eps->rel_depth * fabs((double)prev_z)) {
            mg = 1;
            bnd += T_prev * a_prev * alpha * 2.0 * M;
        }
        prev_z = r->z32; have_prev = 1;
        T_prev = T; a_prev = alpha;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn - 1e-4) <= eps->rel_T * 1e-4) mg = 1;
        if (fabs(Tn - 1e-4) <= (eps->rel_T + 1.01 * flip_a) * 1e-4) bnd += T * 2.0 * M;
        if (Tn < 1e-4) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += r->rgb[ch] * alpha * T;
        T = Tn;
    }
    for (int ch = 0; ch < 3; ++ch) out[ch] = C[ch] + T * bg[ch];
    *marg = mg;
    *n_eval += ne;
    if (bound) *bound = bnd;
}

/* Candidate pre-filter: a record may affect row py only if the row centre is
 * within r of its mean (widened by two pixels, which only feeds the marginal
 * rule).  Filtering keeps the (depth, index) order of the sorted list. */
static int row_candidates(const ORec *recs, int m, int py, int *list)
{
    int n = 0;
    for (int k = 0; k < m; ++k) {
        const ORec *r = &recs[k];
        double reach = r->r + 2.0;
        if (fabs(py + 0.5 - r->my) <= reach) list[n++] = k;
    }
    return n;
}

/*
 * Render one delivery state (depth table per cluster, time t, camera).
 * pix == NULL: every pixel, image_out [H][W][3], marg [H][W];
 * else pix [npix][2] = (x, y), image_out [npix][3], marg [npix].
 * full_scan != 0 walks the whole sorted list per pixel (brute force).
 * eps == NULL uses the default tolerances.  Returns the marginal count.
 */
/* Rows [y0, y1) of the image into image_out [(y1 - y0)][W][3] (marg likewise). */
static void render_rows(const ORec *recs, int m, int W, int y0, int y1, const double *bg, const OEps *eps,
                        int full_scan, double *image_out, uint8_t *marg, double *bound, int64_t *total_marg,
                        int64_t *total_eval)
{
    int64_t tm = 0, te = 0;
    #pragma omp parallel for schedule(dynamic, 1) reduction(+:tm, te)
    for (int py = y0; py < y1; ++py) {
        int *list = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
        int nl;
        if (full_scan) { for (int k = 0; k < m; ++k) list[k] = k; nl = m; }
        else nl = row_candidates(recs, m, py, list);
        for (int px = 0; px < W; ++px) {
            int mg = 0; int64_t ne = 0;
            const size_t o = (size_t)(py - y0) * W + px;
            shade_pixel(recs, list, nl, px, py, bg, eps, image_out + o * 3, &mg, &ne, bound ? bound + o : NULL);
            if (marg) marg[o] = (uint8_t)mg;
            tm += mg; te += ne;
        }
        free(list);
    }
    *total_marg += tm;
    *total_eval += te;
}

/* A band of whole rows [y0, y1) (row filter as in the full render): the
 * bounded sample a timing of the oracle extrapolates from. */
int64_t o_render_rows(const OScene *s, const uint8_t *depth, double t, const OCam *cam, const double *bg,
                      int y0, int y1, double *image_out, uint8_t *marg, int64_t *n_eval)
{
    int m = 0;
    ORec *recs = project_sorted(s, depth, t, cam, &kDefaultEps, &m);
    int64_t total_marg = 0, total_eval = 0;
    render_rows(recs, m, cam->width, y0, y1, bg, &kDefaultEps, 0, image_out, marg, NULL, &total_marg, &total_eval);
    free(recs);
    if (n_eval) *n_eval = total_eval;
    return total_marg;
}

int64_t o_render(const OScene *s, const uint8_t *depth, double t, const OCam *cam,
                 const double *bg, int npix, const int32_t *pix, double *image_out,
                 uint8_t *marg, int64_t *n_eval, int full_scan, const OEps *eps_in, double *bound)
{
    const OEps *eps = eps_in ? eps_in : &kDefaultEps;
    int m = 0;
    ORec *recs = project_sorted(s, depth, t, cam, eps, &m);
    int64_t total_marg = 0, total_eval = 0;
    int W = cam->width, H = cam->height;
    if (pix == NULL) {
        render_rows(recs, m, W, 0, H, bg, eps, full_scan, image_out, marg, bound, &total_marg, &total_eval);
    } else {
        #pragma omp parallel for schedule(dynamic, 16) reduction(+:total_marg, total_eval)
        for (int q = 0; q < npix; ++q) {
            int *list = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
            for (int k = 0; k < m; ++k) list[k] = k;
            int mg = 0; int64_t ne = 0;
            shade_pixel(recs, list, m, pix[2 * q], pix[2 * q + 1], bg, eps, image_out + (size_t)q * 3, &mg, &ne,
                        bound ? bound + q : NULL);
            if (marg) marg[q] = (uint8_t)mg;
            total_marg += mg; total_eval += ne;
            free(list);
        }
    }
    free(recs);
    if (n_eval) *n_eval = total_eval;
    return total_marg;
}

/*
 * Tile membership from the footprint alone (the definition tile binning must
 * cover; it uses no acceleration structure and none of the GPU path's
 * constants).  For every Gaussian present in the state, the tiles of side
 * `tile` that hold at least one pixel centre p with |p - m| <= r on both axes,
 * power <= 0 and alpha = min(0.99, o e^power) >= 1/255: exactly the pixels
 * the compositing of S11/S12 can include it at.  A (Gaussian, tile) pair that
 * only pixels near a threshold qualify for (alpha within rel_alpha of 1/255,
 * |p - m| within box_px of r, a radius that may round the other way, a mean
 * at the near plane) is marked marginal: an FP32 evaluation may take or drop
 * it.  Writes up to cap pairs (Gaussian index, tile index = ty * tiles_x + tx,
 * marginal) in (Gaussian, tile) order; returns the number of pairs.
 */
int64_t o_footprint_tiles(const OScene *s, const uint8_t *depth, double t, const OCam *cam, int tile,
                          int64_t cap, int32_t *gauss, int32_t *tiles, uint8_t *marg)
{
    const OEps *eps = &kDefaultEps;
    const int W = cam->width, H = cam->height, tiles_x = (W + tile - 1) / tile;
    int64_t n = 0;
    for (int c = 0; c < s->n_clusters; ++c) {
        const int d = depth[c];
        if (d < 1) continue;
        for (int i = s->cluster_offsets[c]; i < s->cluster_offsets[c + 1]; ++i) {
            ORec r;
            project_one(s, i, d, t, cam, eps, &r, NULL);
            if (!r.has_proj || !(r.valid || r.marg_rad || r.marg_near)) continue;
            const double reach = r.r + (r.marg_rad ? 1.0 : 0.0) + eps->box_px;
            int x0 = (int)ceil(r.mx - reach - 0.5), x1 = (int)floor(r.mx + reach - 0.5);
            int y0 = (int)ceil(r.my - reach - 0.5), y1 = (int)floor(r.my + reach - 0.5);
            x0 = x0 < 0 ? 0 : x0; y0 = y0 < 0 ? 0 : y0;
            x1 = x1 > W - 1 ? W - 1 : x1; y1 = y1 > H - 1 ? H - 1 : y1;
            if (x0 > x1 || y0 > y1) continue;
            const int tx0 = x0 / tile, tx1 = x1 / tile, ty0 = y0 / tile, ty1 = y1 / tile;
            const int tw = tx1 - tx0 + 1, th = ty1 - ty0 + 1;
            uint8_t *flag = (uint8_t *)calloc((size_t)tw * th, 1);   /* bit 0: sure, bit 1: maybe */
            for (int py = y0; py <= y1; ++py)
                for (int px = x0; px <= x1; ++px) {
                    const double dx = r.mx - (px + 0.5), dy = r.my - (py + 0.5);
                    const double ax = fabs(dx), ay = fabs(dy);
                    const double pw = -0.5 * (r.A * dx * dx + r.Cc * dy * dy) - r.B * dx * dy;
                    const double pmag = 0.5 * fabs(r.A * dx * dx) + 0.5 * fabs(r.Cc * dy * dy) + fabs(r.B * dx * dy);
                    const double araw = r.o * exp(pw);
                    const double alpha = araw < 0.99 ? araw : 0.99;
                    const int inside = r.valid && px >= r.xlo && px <= r.xhi && py >= r.ylo && py <= r.yhi;
                    const int edge = fabs(ax - r.r) <= eps->box_px || fabs(ay - r.r) <= eps->box_px ||
                                     (r.marg_rad && (ax > r.r - 1 - eps->box_px || ay > r.r - 1 - eps->box_px)) ||
                                     r.marg_near;
                    const int sure = inside && !edge && pw <= 0 && fabs(pw) > 1e-5 * pmag &&
                                     alpha >= (1.0 / 255.0) * (1.0 + eps->rel_alpha);
                    const int maybe = pw <= 1e-5 * pmag && alpha >= (1.0 / 255.0) * (1.0 - eps->rel_alpha);
                    uint8_t *f = &flag[(size_t)(py / tile - ty0) * tw + (px / tile - tx0)];
                    if (sure) *f |= 1;
                    else if (maybe) *f |= 2;
                }
            for (int ty = 0; ty < th; ++ty)
                for (int tx = 0; tx < tw; ++tx) {
                    const uint8_t f = flag[(size_t)ty * tw + tx];
                    if (!f) continue;
                    if (n < cap) {
                        gauss[n] = i;
                        tiles[n] = (ty0 + ty) * tiles_x + (tx0 + tx);
                        marg[n] = (uint8_t)((f & 1) ? 0 : 1);
                    }
                    ++n;
                }
            free(flag);
        }
    }
    return n;
}

/* ---------------- adjoint ---------------- */

typedef struct { double mx, my, A, B, Cc, o, rgb[3]; } OGrad2;

/* Accumulate the chain rule of one record into the scene gradient arrays. */
static void backprop_record(const OScene *s, int i, int d, double t, const OCam *cam,
                            const OGrad2 *g, double *g_mu0, double *g_u, double *g_ls,
                            double *g_quat, double *g_logit, double *g_col, double *g_res, double *g_aff,
                            double *g_step)
{
    ORec rec;
    OFwd f;
    project_one(s, i, d, t, cam, &kDefaultEps, &rec, &f);
    int nc = n_colour(s), K = res_width(s);
    double gmu[3] = {0, 0, 0}, gp[3] = {0, 0, 0}, gls[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0};
    double glogit = g->o * rec.o * (1.0 - rec.o);
    double gcol[48];
    memset(gcol, 0, sizeof(gcol));
    /* colour */
    if (s->sh_degree == 0) {
        for (int k = 0; k < 3; ++k) gcol[k] = f.a.col[k] > 0 ? g->rgb[k] : 0;
    } else {
        double Y[16], dY[16][3];
        o_sh_basis(f.dir, s->sh_degree, Y);
        sh_basis_grad(f.dir, s->sh_degree, dY);
        int nb = nc / 3;
        double gdir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            if (!(f.shv[ch] > 0)) continue;
            for (int j = 0; j < nb; ++j) {
                gcol[3 * j + ch] += Y[j] * g->rgb[ch];
                for (int k = 0; k < 3; ++k) gdir[k] += g->rgb[ch] * f.a.col[3 * j + ch] * dY[j][k];
            }
        }
        double dd = gdir[0] * f.dir[0] + gdir[1] * f.dir[1] + gdir[2] * f.dir[2];
        for (int k = 0; k < 3; ++k) gmu[k] += (gdir[k] - f.dir[k] * dd) / f.dist;
    }
    /* conic -> 2D covariance: G_sigma = -Q G Q with G = [[gA, gB/2], [gB/2, gC]] */
    double Q[4] = {rec.A, rec.B, rec.B, rec.Cc};
    double G[4] = {g->A, 0.5 * g->B, 0.5 * g->B, g->Cc};
    double QG[4], GS[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) QG[2 * r + c] = Q[2 * r] * G[c] + Q[2 * r + 1] * G[2 + c];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) GS[2 * r + c] = -(QG[2 * r] * Q[c] + QG[2 * r + 1] * Q[2 + c]);
    /* Sigma2 = T Sigma3 T^T + 0.3 I:  gSigma3 = T^T GS T,  gT = 2 GS T Sigma3 */
    double gS3[9], gT[6];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) acc += f.T[3 * a + r] * GS[2 * a + b] * f.T[3 * b + c];
            gS3[3 * r + c] = acc;
        }
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int b = 0; b < 2; ++b)
                for (int k = 0; k < 3; ++k) acc += GS[2 * r + b] * f.T[3 * b + k] * f.S3[3 * k + c];
            gT[3 * r + c] = 2.0 * acc;
        }
    /* T = J W  ->  gJ = gT W^T */
    double gJ[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            gJ[3 * r + c] = gT[3 * r] * cam->R[3 * c] + gT[3 * r + 1] * cam->R[3 * c + 1] + gT[3 * r + 2] * cam->R[3 * c + 2];
    double x = f.p[0], y = f.p[1], z = f.p[2], z2 = z * z, z3 = z2 * z;
    double fx = cam->fx, fy = cam->fy;
    /* mean2d */
    gp[0] += g->mx * fx / z;
    gp[1] += g->my * fy / z;
    gp[2] += -g->mx * fx * x / z2 - g->my * fy * y / z2;
    /* Jacobian entries */
    gp[2] += gJ[0] * (-fx / z2) + gJ[4] * (-fy / z2);
    if (!f.clampx) { gp[0] += gJ[2] * (-fx / z2); gp[2] += gJ[2] * (2.0 * fx * x / z3); }
    else { double limx = 1.3 * (0.5 * cam->width) / fx; double txz = x / z < 0 ? -limx : limx; gp[2] += gJ[2] * (fx * txz / z2); }
    if (!f.clampy) { gp[1] += gJ[5] * (-fy / z2); gp[2] += gJ[5] * (2.0 * fy * y / z3); }
    else { double limy = 1.3 * (0.5 * cam->height) / fy; double tyz = y / z < 0 ? -limy : limy; gp[2] += gJ[5] * (fy * tyz / z2); }
    for (int k = 0; k < 3; ++k) gmu[k] += cam->R[k] * gp[0] + cam->R[3 + k] * gp[1] + cam->R[6 + k] * gp[2];
    /* Sigma3 = M M^T -> gM = 2 gS3 M;  M = Rq diag(S) */
    double gM[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += gS3[3 * r + k] * f.M[3 * k + c];
            gM[3 * r + c] = 2.0 * acc;
        }
    double gR[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) gR[3 * r + c] = gM[3 * r + c] * f.S[c];
    for (int c = 0; c < 3; ++c) {
        double acc = 0;
        for (int r = 0; r < 3; ++r) acc += gM[3 * r + c] * f.Rq[3 * r + c];
        gls[c] = acc * f.S[c];
    }
    double w = f.qn[0], qx = f.qn[1], qy = f.qn[2], qz = f.qn[3];
    double gqn[4];
    gqn[0] = 2 * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
    gqn[1] = 2 * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2 * qx * gR[4] - w * gR[5] + qz * gR[6] + w * gR[7] - 2 * qx * gR[8]);
    gqn[2] = 2 * (-2 * qy * gR[0] + qx * gR[1] + w * gR[2] + qx * gR[3] + qz * gR[5] - w * gR[6] + qz * gR[7] - 2 * qy * gR[8]);
    gqn[3] = 2 * (-2 * qz * gR[0] - w * gR[1] + qx * gR[2] + w * gR[3] - 2 * qz * gR[4] + qy * gR[5] + qx * gR[6] + qy * gR[7]);
    double dq = gqn[0] * f.qn[0] + gqn[1] * f.qn[1] + gqn[2] * f.qn[2] + gqn[3] * f.qn[3];
    for (int k = 0; k < 4; ++k) gq[k] = (gqn[k] - f.qn[k] * dq) / f.qnorm;
    /* scatter to base, temporal coefficients and delivered residual layers */
    if (s->affine) {   /* mu = A mubar + ...: d/dmubar = A_lin^T, d/dA = (mubar, 1) per row */
        double A[12], w;
        int k0, k1;
        const int c = cluster_of_idx(s, i);
        affine_at(s, c, t, A, &k0, &k1, &w);
        const float *m0 = s->mu0 + 3 * i;
        for (int k = 0; k < 3; ++k) g_mu0[3 * i + k] += A[k] * gmu[0] + A[4 + k] * gmu[1] + A[8 + k] * gmu[2];
        if (g_aff) {
            const double pv[4] = {m0[0], m0[1], m0[2], 1.0};
            double *ga0 = g_aff + ((size_t)c * s->affine_T + k0) * 12, *ga1 = g_aff + ((size_t)c * s->affine_T + k1) * 12;
            for (int r = 0; r < 3; ++r)
                for (int k = 0; k < 4; ++k) {
                    ga0[4 * r + k] += (1.0 - w) * gmu[r] * pv[k];
                    ga1[4 * r + k] += w * gmu[r] * pv[k];
                }
        }
        for (int k = 0; k < 3; ++k) g_ls[3 * i + k] += gls[k];
    } else {
        for (int k = 0; k < 3; ++k) { g_mu0[3 * i + k] += gmu[k]; g_ls[3 * i + k] += gls[k]; }
    }
    for (int r = 0; r < s->temporal_rank; ++r) {
        double b = basis(r, t);
        for (int k = 0; k < 3; ++k) g_u[((size_t)r * s->n + i) * 3 + k] += b * gmu[k];
    }
    for (int k = 0; k < 4; ++k) g_quat[4 * i + k] += gq[k];
    g_logit[i] += glogit;
    for (int k = 0; k < nc; ++k) g_col[(size_t)nc * i + k] += gcol[k];
    for (int l = 1; l < d; ++l) {
        double gv[64];     /* gradient of the decoded refinement components */
        for (int k = 0; k < 3; ++k) { gv[k] = gmu[k]; gv[3 + k] = gls[k]; }
        for (int k = 0; k < 4; ++k) gv[6 + k] = gq[k];
        gv[10] = glogit;
        for (int k = 0; k < nc; ++k) gv[11 + k] = gcol[k];
        if (s->res_mode == 1) continue;      /* decoded symbols: no gradient */
        double *gr = g_res + ((size_t)(l - 1) * s->n + i) * K;
        for (int k = 0; k < K; ++k) {
            if (s->res_mode == 2) {
                /* straight-through: the rounding passes the gradient, the clip stops it;
                 * the step receives g (v - x / st) in range and g v when clipped */
                int cl;
                const float x = s->res[((size_t)(l - 1) * s->n + i) * K + k];
                const float st = s->res_step[(size_t)(l - 1) * K + k];
                const double v = quant_symbol(x, st, &cl);
                if (!cl) gr[k] += gv[k];
                if (g_step) g_step[(size_t)(l - 1) * K + k] += gv[k] * (cl ? v : v - (double)(x / st));
            } else {
                gr[k] += gv[k];
            }
        }
    }
}

/*
 * Adjoint of o_render for one state: given dL/dI [H][W][3], accumulate (+=)
 * dL/d(parameters) in the scene layout.  Per pixel the included Gaussians
 * 1..K with T_1 = 1, T_{k+1} = T_k (1 - alpha_k) give
 *   dC/drgb_k   = alpha_k T_k
 *   dC/dalpha_k = rgb_k T_k - (sum_{j>k} rgb_j alpha_j T_j + T_{K+1} bg) / (1 - alpha_k)
 * and alpha = o e^power (zero derivative where the 0.99 clamp is active).
 * Optionally writes the per-Gaussian screen-space gradients g2d [n][9] =
 * (mx, my, A, B, C, o, r, g, b).
 */
int o_render_backward(const OScene *s, const uint8_t *depth, double t, const OCam *cam,
                      const double *bg, const double *dL_dimg,
                      double *g_mu0, double *g_u, double *g_ls, double *g_quat,
                      double *g_logit, double *g_col, double *g_res, double *g2d_out, double *g_aff,
                      double *g_step)
{
    int m = 0;
    ORec *recs = project_sorted(s, depth, t, cam, &kDefaultEps, &m);
    OGrad2 *g2 = (OGrad2 *)calloc((size_t)(m > 0 ? m : 1), sizeof(OGrad2));
    int W = cam->width, H = cam->height;
    int *inc = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
    double *al = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *ex = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *Tk = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            const double *gC = dL_dimg + ((size_t)py * W + px) * 3;
            if (gC[0] == 0 && gC[1] == 0 && gC[2] == 0) continue;
            double pcx = px + 0.5, pcy = py + 0.5, T = 1.0;
            int K = 0;
            for (int k = 0; k < m; ++k) {
                const ORec *r = &recs[k];
                if (!r->valid) continue;
                if (px < r->xlo || px > r->xhi || py < r->ylo || py > r->yhi) continue;
                double dx = r->mx - pcx, dy = r->my - pcy;
                double pw = -0.5 * (r->A * dx * dx + r->Cc * dy * dy) - r->B * dx * dy;
                if (pw > 0) continue;
                double e = exp(pw);
                double araw = r->o * e;
                double alpha = araw < 0.99 ? araw : 0.99;
                if (alpha < 1.0 / 255.0) continue;
                double Tn = T * (1.0 - alpha);
                if (Tn < 1e-4) break;
                inc[K] = k; al[K] = araw < 0.99 ? alpha : -alpha; ex[K] = e; Tk[K] = T; ++K;
                T = Tn;
            }
            double suffix[3] = {T * bg[0], T * bg[1], T * bg[2]};
            for (int q = K - 1; q >= 0; --q) {
                const ORec *r = &recs[inc[q]];
                OGrad2 *g = &g2[inc[q]];
                int clamped = al[q] < 0;
                double alpha = clamped ? -al[q] : al[q];
                double T_q = Tk[q], galpha = 0;
                for (int ch = 0; ch < 3; ++ch) {
                    g->rgb[ch] += gC[ch] * alpha * T_q;
                    galpha += gC[ch] * (r->rgb[ch] * T_q - suffix[ch] / (1.0 - alpha));
                }
                for (int ch = 0; ch < 3; ++ch) suffix[ch] += r->rgb[ch] * alpha * T_q;
                if (clamped) continue;
                double dx = r->mx - pcx, dy = r->my - pcy;
                g->o += galpha * ex[q];
                double gpw = galpha * alpha;
                g->mx += gpw * (-(r->A * dx + r->B * dy));
                g->my += gpw * (-(r->Cc * dy + r->B * dx));
                g->A += gpw * (-0.5 * dx * dx);
                g->B += gpw * (-dx * dy);
                g->Cc += gpw * (-0.5 * dy * dy);
            }
        }
    for (int k = 0; k < m; ++k) {
        const ORec *r = &recs[k];
        if (!r->valid) continue;
        int i = r->idx;
        int c = 0;
        while (!(i >= s->cluster_offsets[c] && i < s->cluster_offsets[c + 1])) ++c;
        backprop_record(s, i, depth[c], t, cam, &g2[k], g_mu0, g_u, g_ls, g_quat, g_logit, g_col, g_res, g_aff,
                        g_step);
        if (g2d_out) {
            double *o = g2d_out + (size_t)i * 9;
            o[0] += g2[k].mx; o[1] += g2[k].my; o[2] += g2[k].A; o[3] += g2[k].B; o[4] += g2[k].Cc;
            o[5] += g2[k].o; o[6] += g2[k].rgb[0]; o[7] += g2[k].rgb[1]; o[8] += g2[k].rgb[2];
        }
    }
    free(inc); free(al); free(ex); free(Tk); free(g2); free(recs);
    return 0;
}

int o_rec_width(void) { return REC_W; }
