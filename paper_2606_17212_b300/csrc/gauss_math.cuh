// Per-Gaussian FP32 math of the renderer: masked prefix decode (Section 3),
// the low-rank temporal deformation of Eq. 1, EWA projection to a 2D conic,
// colour, and the adjoint of all of it.  Shared by the projection kernel and
// the backward projection kernel so both evaluate exactly the same forward.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "dgs_internal.cuh"

namespace dgs {

template <int SH> struct NCol { static constexpr int value = 3 * (SH + 1) * (SH + 1); };

template <int SH>
struct Attr {
    float mu[3], ls[3], q[4], logit;
    float mu0[3];              // the base mean alone (the cluster affine applies to it)
    float col[NCol<SH>::value];
};

template <int SH>
__device__ __forceinline__ void load_base(const SceneDev &s, int i, Attr<SH> &a)
{
    constexpr int NC = NCol<SH>::value;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a.mu[k] = a.mu0[k] = __ldg(s.mu0 + 3 * i + k);
        a.ls[k] = __ldg(s.ls + 3 * i + k);
    }
    const float4 q = __ldg(reinterpret_cast<const float4 *>(s.quat) + i);
    a.q[0] = q.x; a.q[1] = q.y; a.q[2] = q.z; a.q[3] = q.w;
    a.logit = __ldg(s.logit + i);
#pragma unroll
    for (int k = 0; k < NC; ++k) a.col[k] = __ldg(s.colour + (size_t)NC * i + k);
}

// Symbol of a refinement value x quantized to step st (the learned steps of
// Section 3): round(x / st) (IEEE FP32 quotient, ties to even) clipped to the
// signed 16-bit range.
__device__ __forceinline__ float quant_symbol(float x, float st, bool &clipped)
{
    float v = rintf(__fdiv_rn(x, st));
    clipped = v > 32767.0f || v < -32768.0f;
    return fminf(fmaxf(v, -32768.0f), 32767.0f);
}

// Component k of refinement layer l (1-based) of Gaussian i as decoded (res_mode 1, 2).
__device__ __forceinline__ float res_value(const SceneDev &s, int l, int i, int k)
{
    const size_t o = ((size_t)(l - 1) * s.n + i) * s.K + k;
    const float st = __ldg(s.res_step + (size_t)(l - 1) * s.K + k);
    if (s.res_mode == 1) return __fmul_rn((float)__ldg(s.res_q + o), st);
    bool cl;
    return __fmul_rn(quant_symbol(__ldg(s.res + o), st, cl), st);
}

// attribute += refinement layer l (1-based) of Gaussian i, in a fixed order
template <int SH>
__device__ __forceinline__ void add_layer(const SceneDev &s, int i, int l, Attr<SH> &a)
{
    constexpr int NC = NCol<SH>::value;
    constexpr int K = 11 + NC;
    if (s.res_mode != 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { a.mu[k] += res_value(s, l, i, k); a.ls[k] += res_value(s, l, i, 3 + k); }
#pragma unroll
        for (int k = 0; k < 4; ++k) a.q[k] += res_value(s, l, i, 6 + k);
        a.logit += res_value(s, l, i, 10);
#pragma unroll
        for (int k = 0; k < NC; ++k) a.col[k] += res_value(s, l, i, 11 + k);
        return;
    }
    const float *r = s.res + ((size_t)(l - 1) * s.n + i) * K;
#pragma unroll
    for (int k = 0; k < 3; ++k) { a.mu[k] += __ldg(r + k); a.ls[k] += __ldg(r + 3 + k); }
#pragma unroll
    for (int k = 0; k < 4; ++k) a.q[k] += __ldg(r + 6 + k);
    a.logit += __ldg(r + 10);
#pragma unroll
    for (int k = 0; k < NC; ++k) a.col[k] += __ldg(r + 11 + k);
}

// Cluster affine A_{c,t} of Eq. 1: keyframe k at time k / T, linear
// interpolation of the twelve entries between keyframes, periodic in t.
// Returns the keyframes used and the weight w of k1.
__device__ __forceinline__ void affine_at(const SceneDev &s, int c, float t, float *A, int &k0, int &k1, float &w)
{
    const float u = t * (float)s.aT;
    const float fl = floorf(u);
    w = u - fl;
    int kk = (int)fl % s.aT;
    if (kk < 0) kk += s.aT;
    k0 = kk;
    k1 = (kk + 1) % s.aT;
    const float *a0 = s.affine + ((size_t)c * s.aT + k0) * 12, *a1 = s.affine + ((size_t)c * s.aT + k1) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) A[k] = fmaf(w, __ldg(a1 + k), (1.0f - w) * __ldg(a0 + k));
}

// Shared temporal basis of Eq. 1: b_{2j-1}(t) = cos(2 pi j t), b_{2j}(t) = sin(2 pi j t).
__device__ __forceinline__ float temporal_basis(int k, float t)
{
    float s, c;
    sincospif(2.0f * (float)(k / 2 + 1) * t, &s, &c);
    return (k & 1) ? s : c;
}

// Real spherical harmonics (orthonormal on the sphere) up to degree 3 on a unit
// direction; order (0,0), (1,-1), (1,0), (1,1), (2,-2) .. (2,2), (3,-3) .. (3,3).
// Normalisations: 1/(2 sqrt(pi)), sqrt(3/(4 pi)), sqrt(15/pi)/2, sqrt(5/pi)/4,
// sqrt(15/pi)/4, sqrt(35/(2 pi))/4, sqrt(105/pi)/2, sqrt(21/(2 pi))/4,
// sqrt(7/pi)/4, sqrt(105/pi)/4.
struct SHK {
    static constexpr float c00 = 0.28209479177387814f, c1 = 0.4886025119029199f;
    static constexpr float c2a = 1.0925484305920792f, c2b = 0.31539156525252005f, c2c = 0.5462742152960396f;
    static constexpr float c3a = 0.5900435899266435f, c3b = 2.890611442640554f, c3c = 0.4570457994644658f;
    static constexpr float c3d = 0.3731763325901154f, c3e = 1.445305721320277f;
};

__device__ __forceinline__ void sh3_basis(float x, float y, float z, float *Y)
{
    Y[0] = SHK::c00;
    Y[1] = SHK::c1 * y; Y[2] = SHK::c1 * z; Y[3] = SHK::c1 * x;
    const float zz = z * z;
    Y[4] = SHK::c2a * x * y; Y[5] = SHK::c2a * y * z; Y[6] = SHK::c2b * (3.0f * zz - 1.0f);
    Y[7] = SHK::c2a * x * z; Y[8] = SHK::c2c * (x * x - y * y);
    Y[9] = SHK::c3a * y * (3.0f * x * x - y * y);
    Y[10] = SHK::c3b * x * y * z;
    Y[11] = SHK::c3c * y * (5.0f * zz - 1.0f);
    Y[12] = SHK::c3d * z * (5.0f * zz - 3.0f);
    Y[13] = SHK::c3c * x * (5.0f * zz - 1.0f);
    Y[14] = SHK::c3e * z * (x * x - y * y);
    Y[15] = SHK::c3a * x * (x * x - 3.0f * y * y);
}

// d(sum_j w_j Y_j)/d(x, y, z) for weights w (polynomial extension off the sphere).
__device__ __forceinline__ void sh3_grad_dot(float x, float y, float z, const float *w, float *g)
{
    const float zz = z * z;
    float gx = 0, gy = 0, gz = 0;
    gy += w[1] * SHK::c1; gz += w[2] * SHK::c1; gx += w[3] * SHK::c1;
    gx += w[4] * SHK::c2a * y; gy += w[4] * SHK::c2a * x;
    gy += w[5] * SHK::c2a * z; gz += w[5] * SHK::c2a * y;
    gz += w[6] * SHK::c2b * 6.0f * z;
    gx += w[7] * SHK::c2a * z; gz += w[7] * SHK::c2a * x;
    gx += w[8] * SHK::c2c * 2.0f * x; gy -= w[8] * SHK::c2c * 2.0f * y;
    gx += w[9] * SHK::c3a * 6.0f * x * y; gy += w[9] * SHK::c3a * 3.0f * (x * x - y * y);
    gx += w[10] * SHK::c3b * y * z; gy += w[10] * SHK::c3b * x * z; gz += w[10] * SHK::c3b * x * y;
    gy += w[11] * SHK::c3c * (5.0f * zz - 1.0f); gz += w[11] * SHK::c3c * 10.0f * y * z;
    gz += w[12] * SHK::c3d * (15.0f * zz - 3.0f);
    gx += w[13] * SHK::c3c * (5.0f * zz - 1.0f); gz += w[13] * SHK::c3c * 10.0f * x * z;
    gx += w[14] * SHK::c3e * 2.0f * x * z; gy -= w[14] * SHK::c3e * 2.0f * y * z; gz += w[14] * SHK::c3e * (x * x - y * y);
    gx += w[15] * SHK::c3a * 3.0f * (x * x - y * y); gy -= w[15] * SHK::c3a * 6.0f * x * y;
    g[0] = gx; g[1] = gy; g[2] = gz;
}

// Forward intermediates of one projected variant (kept for the adjoint).
struct Fwd {
    float mu[3];          // deformed mean (world)
    float p[3];           // camera-space mean
    float iz;
    float qn[4], qinv;    // normalised quaternion, 1 / |q|
    float Rq[9], S[3];
    float T[6];           // J W
    float V[6];           // J W Rq diag(S)
    float a, b, c, det;   // dilated 2D covariance and its determinant
    float dir[3], idist;  // SH view direction (degree 3)
    float shv[3];         // colour before the clamp at zero
    int clampx, clampy;
};

struct Proj {
    float mx, my, A, B, C, o, rgb[3], z, r;
    int xlo, xhi, ylo, yhi;
    bool live;
    bool rclip;                // the 3-sigma box is narrower than the alpha >= 1/255 box on some axis
    bool aclamp;               // alpha = o 2^p2 may reach the 0.99 clamp at some pixel
};

// Eq. 1 deformation and EWA projection of decoded attributes `a` of Gaussian i.
template <int SH>
__device__ __forceinline__ void project_fwd(const SceneDev &s, int i, int c, const Attr<SH> &a,
                                            const ViewGroup &vg, Proj &P, Fwd &F)
{
    P.live = false;
    P.rclip = false;
    P.aclamp = true;
    if (s.affine) {   // A_{c,t} mubar + (position residuals)
        float A[12], w;
        int k0, k1;
        affine_at(s, c, vg.time, A, k0, k1, w);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            F.mu[k] = fmaf(A[4 * k], a.mu0[0], fmaf(A[4 * k + 1], a.mu0[1], fmaf(A[4 * k + 2], a.mu0[2], A[4 * k + 3]))) +
                      (a.mu[k] - a.mu0[k]);
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) F.mu[k] = a.mu[k];
    }
    for (int r = 0; r < s.R; ++r) {
        const float bk = temporal_basis(r, vg.time);
        const float *ur = s.u + ((size_t)r * s.n + i) * 3;
#pragma unroll
        for (int k = 0; k < 3; ++k) F.mu[k] = fmaf(bk, __ldg(ur + k), F.mu[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
        F.p[k] = fmaf(vg.R[3 * k], F.mu[0], fmaf(vg.R[3 * k + 1], F.mu[1], fmaf(vg.R[3 * k + 2], F.mu[2], vg.t[k])));
    const float x = F.p[0], y = F.p[1], z = F.p[2];
    P.z = z;
    if (!(z > 0.01f)) return;                 // near plane
    F.iz = 1.0f / z;
    P.mx = fmaf(vg.fx * x, F.iz, vg.cx);
    P.my = fmaf(vg.fy * y, F.iz, vg.cy);
    // rotation from the normalised quaternion, axis scales
    const float qq = a.q[0] * a.q[0] + a.q[1] * a.q[1] + a.q[2] * a.q[2] + a.q[3] * a.q[3];
    F.qinv = 1.0f / sqrtf(qq);
#pragma unroll
    for (int k = 0; k < 4; ++k) F.qn[k] = a.q[k] * F.qinv;
    {
        const float w = F.qn[0], qx = F.qn[1], qy = F.qn[2], qz = F.qn[3];
        F.Rq[0] = 1.f - 2.f * (qy * qy + qz * qz); F.Rq[1] = 2.f * (qx * qy - w * qz);       F.Rq[2] = 2.f * (qx * qz + w * qy);
        F.Rq[3] = 2.f * (qx * qy + w * qz);       F.Rq[4] = 1.f - 2.f * (qx * qx + qz * qz); F.Rq[5] = 2.f * (qy * qz - w * qx);
        F.Rq[6] = 2.f * (qx * qz - w * qy);       F.Rq[7] = 2.f * (qy * qz + w * qx);       F.Rq[8] = 1.f - 2.f * (qx * qx + qy * qy);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) F.S[k] = expf(a.ls[k]);
    // pinhole Jacobian at the direction clamped to 1.3x the half field of view
    const float limx = 1.3f * 0.5f * (float)vg.width / vg.fx;
    const float limy = 1.3f * 0.5f * (float)vg.height / vg.fy;
    float txz = x * F.iz, tyz = y * F.iz;
    F.clampx = (txz < -limx) || (txz > limx);
    F.clampy = (tyz < -limy) || (tyz > limy);
    txz = fminf(fmaxf(txz, -limx), limx);
    tyz = fminf(fmaxf(tyz, -limy), limy);
    const float J00 = vg.fx * F.iz, J02 = -vg.fx * txz * F.iz;
    const float J11 = vg.fy * F.iz, J12 = -vg.fy * tyz * F.iz;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        F.T[j] = fmaf(J00, vg.R[j], J02 * vg.R[6 + j]);
        F.T[3 + j] = fmaf(J11, vg.R[3 + j], J12 * vg.R[6 + j]);
    }
    // V = T Rq diag(S): Sigma2D = V V^T + 0.3 I
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k)
            F.V[3 * r + k] = (F.T[3 * r] * F.Rq[k] + F.T[3 * r + 1] * F.Rq[3 + k] + F.T[3 * r + 2] * F.Rq[6 + k]) * F.S[k];
    const float v00 = F.V[0] * F.V[0] + F.V[1] * F.V[1] + F.V[2] * F.V[2];
    const float v11 = F.V[3] * F.V[3] + F.V[4] * F.V[4] + F.V[5] * F.V[5];
    const float v01 = F.V[0] * F.V[3] + F.V[1] * F.V[4] + F.V[2] * F.V[5];
    F.a = v00 + 0.3f; F.c = v11 + 0.3f; F.b = v01;
    // det = |V0 x V1|^2 + 0.3 (|V0|^2 + |V1|^2) + 0.09 (Lagrange identity): no cancellation
    const float cx_ = F.V[1] * F.V[5] - F.V[2] * F.V[4];
    const float cy_ = F.V[2] * F.V[3] - F.V[0] * F.V[5];
    const float cz_ = F.V[0] * F.V[4] - F.V[1] * F.V[3];
    F.det = (cx_ * cx_ + cy_ * cy_ + cz_ * cz_) + 0.3f * (v00 + v11) + 0.09f;
    if (!(F.det > 0.0f)) return;
    const float idet = 1.0f / F.det;
    P.A = F.c * idet; P.B = -F.b * idet; P.C = F.a * idet;
    const float hd = 0.5f * (F.a - F.c);
    const float lam = 0.5f * (F.a + F.c) + sqrtf(hd * hd + F.b * F.b);
    P.r = ceilf(3.0f * sqrtf(lam));
    P.o = 1.0f / (1.0f + expf(-a.logit));
    // Visible box.  The definition's box is |p_centre - m| <= r.  A pixel also
    // needs alpha = o e^power >= 1/255, i.e. d^T Q d <= rho = 2 ln(255 o), whose
    // bounding box has half-widths sqrt(rho a) and sqrt(rho c) (a, c: diagonal
    // of the dilated covariance).  Intersecting both boxes removes only pixels
    // the compositing would skip; the alpha half-widths are inflated by 1e-3
    // relative + 0.05 px so FP32 rounding never drops a pixel that composites.
    // A Gaussian with o < 1/255 never composites at all.
    if (!(P.o >= (1.0f / 255.0f))) return;
    const float rho = 2.0f * logf(255.0f * P.o);
    const float ax = fmaf(sqrtf(fmaxf(rho, 0.0f) * F.a), 1.001f, 0.05f);
    const float ay = fmaf(sqrtf(fmaxf(rho, 0.0f) * F.c), 1.001f, 0.05f);
    const float hx = fminf(P.r, ax), hy = fminf(P.r, ay);
    // Where the 3-sigma box is not the narrower one, the box holds every pixel
    // the alpha test keeps, so the raster needs no per-pixel box test.
    P.rclip = (P.r < ax) || (P.r < ay);
    // The raster evaluates the exponent p2 = dT Q' d (Q' the scaled negative-
    // definite conic) in FP32 as fma(fma(c2, dy, b2 dx), dy, a2 dx dx); its
    // rounding error is below 16 * 2^-24 * lambda_max |d|^2 while the exact
    // value is at most -lambda_min |d|^2, so for a condition number below 2^20
    // the evaluated p2 is never positive and alpha <= o (1 + 2^-21).  Below
    // o = 0.98 and a condition number of 1e4 the 0.99 clamp is then
    // unreachable and the raster may skip it; every other record keeps it.
    P.aclamp = !(P.o <= 0.98f) || !(lam * lam <= 1e4f * F.det);
    // pixel ranges: |x + 0.5 - mx| <= h  <=>  ceil(mx - h - 0.5) <= x <= floor(mx + h - 0.5),
    // evaluated in FP32 (rounding moves an edge only for pixel centres within
    // ~1e-5 px of the boundary), clamped to the image before the integer cast
    float xl = ceilf(__fsub_rn(__fsub_rn(P.mx, hx), 0.5f)), xh = floorf(__fsub_rn(__fadd_rn(P.mx, hx), 0.5f));
    float yl = ceilf(__fsub_rn(__fsub_rn(P.my, hy), 0.5f)), yh = floorf(__fsub_rn(__fadd_rn(P.my, hy), 0.5f));
    xl = fminf(fmaxf(xl, 0.0f), (float)vg.width);  xh = fmaxf(fminf(xh, (float)(vg.width - 1)), -1.0f);
    yl = fminf(fmaxf(yl, 0.0f), (float)vg.height); yh = fmaxf(fminf(yh, (float)(vg.height - 1)), -1.0f);
    P.xlo = (int)xl; P.xhi = (int)xh; P.ylo = (int)yl; P.yhi = (int)yh;
    if (SH == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { F.shv[k] = a.col[k]; P.rgb[k] = fmaxf(a.col[k], 0.0f); }
    } else {
        float v[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) v[k] = F.mu[k] - vg.campos[k];
        F.idist = 1.0f / sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
#pragma unroll
        for (int k = 0; k < 3; ++k) F.dir[k] = v[k] * F.idist;
        float Y[16];
        sh3_basis(F.dir[0], F.dir[1], F.dir[2], Y);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < (NCol<SH>::value / 3); ++j) acc = fmaf(Y[j], a.col[3 * j + ch], acc);
            F.shv[ch] = acc + 0.5f;
            P.rgb[ch] = fmaxf(F.shv[ch], 0.0f);
        }
    }
    P.live = (P.xlo <= P.xhi) && (P.ylo <= P.yhi);
}

// Adjoint of project_fwd for one variant: given the screen-space gradient
// g = (mx, my, A, B, C, o, r, g, b), accumulate the gradient w.r.t. the decoded
// attributes into ga and return the gradient w.r.t. the deformed mean in gmu.
template <int SH>
__device__ __forceinline__ void project_bwd(const Attr<SH> &a, const ViewGroup &vg, const Proj &P,
                                            const Fwd &F, const float *g, Attr<SH> &ga, float *gmu)
{
    constexpr int NC = NCol<SH>::value;
    const float gmx = g[0], gmy = g[1], gA = g[2], gB = g[3], gC = g[4], go = g[5];
    gmu[0] = gmu[1] = gmu[2] = 0.0f;
    ga.logit += go * P.o * (1.0f - P.o);
    if (SH == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) ga.col[k] += F.shv[k] > 0.0f ? g[6 + k] : 0.0f;
    } else {
        float Y[16], w[16], gd[3];
        sh3_basis(F.dir[0], F.dir[1], F.dir[2], Y);
        const float m0 = F.shv[0] > 0.0f ? g[6] : 0.0f;
        const float m1 = F.shv[1] > 0.0f ? g[7] : 0.0f;
        const float m2 = F.shv[2] > 0.0f ? g[8] : 0.0f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            ga.col[3 * j + 0] += Y[j] * m0;
            ga.col[3 * j + 1] += Y[j] * m1;
            ga.col[3 * j + 2] += Y[j] * m2;
            w[j] = m0 * a.col[3 * j] + m1 * a.col[3 * j + 1] + m2 * a.col[3 * j + 2];
        }
        sh3_grad_dot(F.dir[0], F.dir[1], F.dir[2], w, gd);
        const float dd = gd[0] * F.dir[0] + gd[1] * F.dir[1] + gd[2] * F.dir[2];
#pragma unroll
        for (int k = 0; k < 3; ++k) gmu[k] += (gd[k] - F.dir[k] * dd) * F.idist;
    }
    // conic Q = Sigma^-1:  dL/dSigma = -Q G Q with G = [[gA, gB/2], [gB/2, gC]]
    const float A = P.A, B = P.B, C = P.C, hB = 0.5f * gB;
    const float qa = A * gA + B * hB, qb = A * hB + B * gC;
    const float qc = B * gA + C * hB, qd = B * hB + C * gC;
    const float gs00 = -(qa * A + qb * B), gs01 = -(qa * B + qb * C), gs11 = -(qc * B + qd * C);
    // Sigma = V V^T + 0.3 I
    float gV[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        gV[k] = 2.0f * gs00 * F.V[k] + 2.0f * gs01 * F.V[3 + k];
        gV[3 + k] = 2.0f * gs11 * F.V[3 + k] + 2.0f * gs01 * F.V[k];
    }
    // V = T Rq diag(S)
#pragma unroll
    for (int k = 0; k < 3; ++k) ga.ls[k] += gV[k] * F.V[k] + gV[3 + k] * F.V[3 + k];
    float gT[6], gR[9];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            gT[3 * r + j] = gV[3 * r] * F.Rq[3 * j] * F.S[0] + gV[3 * r + 1] * F.Rq[3 * j + 1] * F.S[1] +
                            gV[3 * r + 2] * F.Rq[3 * j + 2] * F.S[2];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) gR[3 * j + k] = (gV[k] * F.T[j] + gV[3 + k] * F.T[3 + j]) * F.S[k];
    // T = J W with J = [[fx/z, 0, -fx tx/z], [0, fy/z, -fy ty/z]]
    const float gJ00 = gT[0] * vg.R[0] + gT[1] * vg.R[1] + gT[2] * vg.R[2];
    const float gJ02 = gT[0] * vg.R[6] + gT[1] * vg.R[7] + gT[2] * vg.R[8];
    const float gJ11 = gT[3] * vg.R[3] + gT[4] * vg.R[4] + gT[5] * vg.R[5];
    const float gJ12 = gT[3] * vg.R[6] + gT[4] * vg.R[7] + gT[5] * vg.R[8];
    const float x = F.p[0], y = F.p[1], iz = F.iz, iz2 = iz * iz;
    float gx = gmx * vg.fx * iz, gy = gmy * vg.fy * iz;
    float gz = -(gmx * vg.fx * x + gmy * vg.fy * y) * iz2;
    gz += -(gJ00 * vg.fx + gJ11 * vg.fy) * iz2;
    if (!F.clampx) { gx += -gJ02 * vg.fx * iz2; gz += 2.0f * gJ02 * vg.fx * x * iz2 * iz; }
    else { const float lim = 1.3f * 0.5f * (float)vg.width / vg.fx; gz += gJ02 * vg.fx * (x > 0.0f ? lim : -lim) * iz2; }
    if (!F.clampy) { gy += -gJ12 * vg.fy * iz2; gz += 2.0f * gJ12 * vg.fy * y * iz2 * iz; }
    else { const float lim = 1.3f * 0.5f * (float)vg.height / vg.fy; gz += gJ12 * vg.fy * (y > 0.0f ? lim : -lim) * iz2; }
#pragma unroll
    for (int k = 0; k < 3; ++k) gmu[k] += vg.R[k] * gx + vg.R[3 + k] * gy + vg.R[6 + k] * gz;
    // rotation matrix of the unit quaternion, then the normalisation
    const float w = F.qn[0], qx = F.qn[1], qy = F.qn[2], qz = F.qn[3];
    float gq[4];
    gq[0] = 2.f * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
    gq[1] = 2.f * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2.f * qx * gR[4] - w * gR[5] + qz * gR[6] + w * gR[7] - 2.f * qx * gR[8]);
    gq[2] = 2.f * (-2.f * qy * gR[0] + qx * gR[1] + w * gR[2] + qx * gR[3] + qz * gR[5] - w * gR[6] + qz * gR[7] - 2.f * qy * gR[8]);
    gq[3] = 2.f * (-2.f * qz * gR[0] - w * gR[1] + qx * gR[2] + w * gR[3] - 2.f * qz * gR[4] + qy * gR[5] + qx * gR[6] + qy * gR[7]);
    const float dq = gq[0] * w + gq[1] * qx + gq[2] * qy + gq[3] * qz;
#pragma unroll
    for (int k = 0; k < 4; ++k) ga.q[k] += (gq[k] - F.qn[k] * dq) * F.qinv;
#pragma unroll
    for (int k = 0; k < 3; ++k) ga.mu[k] += gmu[k];
    (void)NC;
}

}  // namespace dgs
