// EWA projection with SH colour (Sec. 3.1, Eq. 1) and its adjoint, per
// Gaussian: the device functions shared by the projection kernels and the
// fused decode-and-project kernels.
#pragma once

#include <cmath>

#include "common.cuh"

namespace qn {
namespace {


struct CamArgs {
    float R[9], t[3];
    float fx, fy, cx, cy, near_plane, limx, limy;
    float cp[3];
    int W, H, TX, TY;
};

// Real spherical harmonics without the Condon-Shortley phase, k = l^2 + l + m.
// Constants are the closed-form normalisations sqrt((2l+1)/4pi (l-|m|)!/(l+|m|)!)
// (times sqrt 2 for m != 0) folded into the Cartesian polynomials.
constexpr float SH_C0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float SH_C1 = 0.4886025119029199f;    // sqrt(3/(4 pi))
constexpr float SH_A2 = 1.0925484305920792f;    // sqrt(15/pi)/2
constexpr float SH_B2 = 0.31539156525252005f;   // sqrt(5/pi)/4
constexpr float SH_C2 = 0.5462742152960396f;    // sqrt(15/pi)/4
constexpr float SH_D3 = 0.5900435899266435f;    // sqrt(35/(2 pi))/4
constexpr float SH_E3 = 2.890611442640554f;     // sqrt(105/pi)/2
constexpr float SH_F3 = 0.4570457994644658f;    // sqrt(21/(2 pi))/4
constexpr float SH_G3 = 0.3731763325901154f;    // sqrt(7/pi)/4
constexpr float SH_H3 = 1.445305721320277f;     // sqrt(105/pi)/4

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float Y[16]) {
    Y[0] = SH_C0;
    if (deg < 1) return;
    Y[1] = SH_C1 * y;
    Y[2] = SH_C1 * z;
    Y[3] = SH_C1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = SH_A2 * x * y;
    Y[5] = SH_A2 * y * z;
    Y[6] = SH_B2 * (3.f * zz - 1.f);
    Y[7] = SH_A2 * x * z;
    Y[8] = SH_C2 * (xx - yy);
    if (deg < 3) return;
    Y[9] = SH_D3 * y * (3.f * xx - yy);
    Y[10] = SH_E3 * x * y * z;
    Y[11] = SH_F3 * y * (5.f * zz - 1.f);
    Y[12] = SH_G3 * z * (5.f * zz - 3.f);
    Y[13] = SH_F3 * x * (5.f * zz - 1.f);
    Y[14] = SH_H3 * z * (xx - yy);
    Y[15] = SH_D3 * x * (xx - 3.f * yy);
}

// g += sum_k w[k] grad Y_k(x, y, z) (gradient of the polynomials above).
__device__ __forceinline__ void sh_grad(int deg, float x, float y, float z, const float w[16],
                                        float &gx, float &gy, float &gz) {
    if (deg < 1) return;
    gy += SH_C1 * w[1];
    gz += SH_C1 * w[2];
    gx += SH_C1 * w[3];
    if (deg < 2) return;
    gx += SH_A2 * (y * w[4] + z * w[7]) + 2.f * SH_C2 * x * w[8];
    gy += SH_A2 * (x * w[4] + z * w[5]) - 2.f * SH_C2 * y * w[8];
    gz += SH_A2 * (y * w[5] + x * w[7]) + 6.f * SH_B2 * z * w[6];
    if (deg < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += SH_D3 * 6.f * x * y * w[9] + SH_E3 * y * z * w[10] + SH_F3 * (5.f * zz - 1.f) * w[13] +
          2.f * SH_H3 * x * z * w[14] + SH_D3 * 3.f * (xx - yy) * w[15];
    gy += SH_D3 * 3.f * (xx - yy) * w[9] + SH_E3 * x * z * w[10] + SH_F3 * (5.f * zz - 1.f) * w[11] -
          2.f * SH_H3 * y * z * w[14] - SH_D3 * 6.f * x * y * w[15];
    gz += SH_E3 * x * y * w[10] + 10.f * SH_F3 * y * z * w[11] + SH_G3 * (15.f * zz - 3.f) * w[12] +
          10.f * SH_F3 * x * z * w[13] + SH_H3 * (xx - yy) * w[14];
}

__device__ __forceinline__ void quat_rot(float w, float x, float y, float z, float R[9]) {
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// a d - b c to about one rounding (Kahan's difference of products: the
// product b c is split into its rounded value and its exact rounding error,
// which an FMA recovers).
__device__ __forceinline__ float diff_prod(float a, float d, float b, float c) {
    const float w = __fmul_rn(b, c);
    const float e = __fmaf_rn(-b, c, w);   // w - b c, exactly
    const float f = __fmaf_rn(a, d, -w);
    return __fadd_rn(f, e);
}

// Forward intermediates shared by the projection and its adjoint.
struct Fwd {
    float t[3], ux, uy, uxc, uyc, Tm[6], v[6], Rq[9], S[3], qn[4], qinv;
    float a, b, c, det0;
};

// Returns false when culled by depth (the determinant is tested by the caller).
__device__ __forceinline__ bool geometry(const CamArgs &cm, const float *__restrict__ A, size_t S_,
                                         int i, Fwd &f) {
    const float px = A[i], py = A[S_ + i], pz = A[2 * S_ + i];
#pragma unroll
    for (int r = 0; r < 3; ++r) f.t[r] = cm.R[3 * r] * px + cm.R[3 * r + 1] * py + cm.R[3 * r + 2] * pz + cm.t[r];
    const float tz = f.t[2];
    if (!(tz > cm.near_plane)) return false;
    const float qw = A[3 * S_ + i], qx = A[4 * S_ + i], qy = A[5 * S_ + i], qz = A[6 * S_ + i];
    f.qinv = 1.f / sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    f.qn[0] = qw * f.qinv; f.qn[1] = qx * f.qinv; f.qn[2] = qy * f.qinv; f.qn[3] = qz * f.qinv;
    quat_rot(f.qn[0], f.qn[1], f.qn[2], f.qn[3], f.Rq);
#pragma unroll
    for (int k = 0; k < 3; ++k) f.S[k] = expf(A[(7 + k) * S_ + i]);
    f.ux = f.t[0] / tz;
    f.uy = f.t[1] / tz;
    f.uxc = fminf(cm.limx, fmaxf(-cm.limx, f.ux));
    f.uyc = fminf(cm.limy, fmaxf(-cm.limy, f.uy));
    const float j00 = cm.fx / tz, j02 = -cm.fx * f.uxc / tz;
    const float j11 = cm.fy / tz, j12 = -cm.fy * f.uyc / tz;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        f.Tm[c] = j00 * cm.R[c] + j02 * cm.R[6 + c];
        f.Tm[3 + c] = j11 * cm.R[3 + c] + j12 * cm.R[6 + c];
    }
    // Sigma' - blur I = T Rq S^2 Rq^T T^T = V V^T with V = T Rq S (2 x 3):
    // column c of V is S_c v_c, v_c = T Rq[:, c] the axis c seen through T.
    // Formed from V, a and c are sums of squares, and the determinant is the
    // sum of the squared 2 x 2 minors of V (Cauchy-Binet), each to about one
    // rounding: no cancellation by the condition number, as a c - b^2 of a
    // needle-like Gaussian would have.
    const float *T = f.Tm;
    float V[6];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        f.v[c] = T[0] * f.Rq[c] + T[1] * f.Rq[3 + c] + T[2] * f.Rq[6 + c];
        f.v[3 + c] = T[3] * f.Rq[c] + T[4] * f.Rq[3 + c] + T[5] * f.Rq[6 + c];
        V[c] = f.S[c] * f.v[c];
        V[3 + c] = f.S[c] * f.v[3 + c];
    }
    f.a = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    f.b = V[0] * V[3] + V[1] * V[4] + V[2] * V[5];
    f.c = V[3] * V[3] + V[4] * V[4] + V[5] * V[5];
    const float m01 = diff_prod(V[0], V[4], V[1], V[3]);
    const float m02 = diff_prod(V[0], V[5], V[2], V[3]);
    const float m12 = diff_prod(V[1], V[5], V[2], V[4]);
    f.det0 = m01 * m01 + m02 * m02 + m12 * m12;
    return true;
}

// det(Sigma') for Sigma' = V V^T + blur I: det(V V^T) + blur tr(V V^T) + blur^2,
// every term non-negative.
__device__ __forceinline__ float proj_det(const Fwd &f, float blur) {
    return f.det0 + blur * (f.a + f.c + blur);
}

// Bounding box of the region where o exp(-q/2) can reach 1/255, i.e. the
// ellipse q(d) = d^T conic d <= k, k = 2 ln(255 o); its half-widths are
// sqrt(k Sigma'_xx) and sqrt(k Sigma'_yy).  k is widened by 0.01 and then 1%,
// the half-widths by 0.01 px, so that FP32 rounding of alpha outside the box
// stays far below 1/255.  Returns false when no pixel can pass (o < 0.995/255).
__device__ __forceinline__ bool alpha_box(float opac, float a, float c, float &hx, float &hy) {
    const float k = 2.f * logf(255.f * opac) + 0.01f;
    if (!(k > 0.f)) return false;
    hx = sqrtf(1.01f * k * a) + 0.01f;
    hy = sqrtf(1.01f * k * c) + 0.01f;
    return true;
}

// DEG: the SH degree, a template parameter so the basis and its loops are
// unrolled into registers.
// The projected record and tile rect of Gaussian i, its attribute planes
// read at A[k * S + i] (global planes, or a tile staged in shared memory).
template <int DEG>
__device__ __forceinline__ void project_one(const CamArgs &cm, float blur, int tight, const float *__restrict__ A,
                                            size_t S, int i, float4 &s0, float4 &s1, float4 &s2, int4 &rc) {
    constexpr int deg = DEG;
    Fwd f;
    s0 = make_float4(0.f, 0.f, 0.f, 0.f);
    s1 = s0;
    s2 = s0;
    rc = make_int4(0, 0, 0, 0);
    bool vis = geometry(cm, A, S, i, f);
    s0.w = f.t[2];
    if (vis) {
        const float a = f.a + blur, b = f.b, c = f.c + blur;
        const float det = proj_det(f, blur);
        vis = det > 0.f;
        if (vis) {
            const float mx = cm.fx * f.ux + cm.cx, my = cm.fy * f.uy + cm.cy;
            const float mid = 0.5f * (a + c);
            const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - det));
            const float rad = ceilf(3.f * sqrtf(lam));
            const float fx0 = floorf((mx - rad) * (1.f / QN_TILE)), fy0 = floorf((my - rad) * (1.f / QN_TILE));
            const float fx1 = floorf((mx + rad + (QN_TILE - 1)) * (1.f / QN_TILE));
            const float fy1 = floorf((my + rad + (QN_TILE - 1)) * (1.f / QN_TILE));
            rc.x = (int)fminf(fmaxf(fx0, 0.f), (float)cm.TX);
            rc.y = (int)fminf(fmaxf(fy0, 0.f), (float)cm.TY);
            rc.z = (int)fminf(fmaxf(fx1, 0.f), (float)cm.TX);
            rc.w = (int)fminf(fmaxf(fy1, 0.f), (float)cm.TY);
            const float opac = 1.f / (1.f + expf(-A[10 * S + i]));
            if (tight) {
                // keep only tiles the alpha >= 1/255 ellipse can reach; the
                // dropped (tile, Gaussian) pairs are skipped by every pixel
                float hx, hy;
                if (alpha_box(opac, a, c, hx, hy)) {
                    const float ex0 = floorf((mx - hx) * (1.f / QN_TILE)), ey0 = floorf((my - hy) * (1.f / QN_TILE));
                    const float ex1 = floorf((mx + hx) * (1.f / QN_TILE)) + 1.f;
                    const float ey1 = floorf((my + hy) * (1.f / QN_TILE)) + 1.f;
                    rc.x = max(rc.x, (int)fminf(fmaxf(ex0, 0.f), (float)cm.TX));
                    rc.y = max(rc.y, (int)fminf(fmaxf(ey0, 0.f), (float)cm.TY));
                    rc.z = min(rc.z, (int)fminf(fmaxf(ex1, 0.f), (float)cm.TX));
                    rc.w = min(rc.w, (int)fminf(fmaxf(ey1, 0.f), (float)cm.TY));
                } else {
                    rc = make_int4(0, 0, 0, 0);
                }
            }
            vis = rc.z > rc.x && rc.w > rc.y;
            if (vis) {
                const float id = 1.f / det;
                s0.x = mx;
                s0.y = my;
                s0.z = opac;
                s1 = make_float4(c * id, -b * id, a * id, 0.f);
                float dx = A[i] - cm.cp[0], dy = A[S + i] - cm.cp[1], dz = A[2 * S + i] - cm.cp[2];
                const float inv = 1.f / sqrtf(dx * dx + dy * dy + dz * dz);
                dx *= inv; dy *= inv; dz *= inv;
                float Y[16];
                sh_basis(deg, dx, dy, dz, Y);
                constexpr int K = (deg + 1) * (deg + 1);
                float col[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
                for (int k = 0; k < K; ++k)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) col[ch] = fmaf(A[(11 + 3 * k + ch) * S + i], Y[k], col[ch]);
                s2 = make_float4(fmaxf(col[0], 0.f), fmaxf(col[1], 0.f), fmaxf(col[2], 0.f), 0.f);
            }
        }
    }
    if (!vis) rc = make_int4(0, 0, 0, 0);
}

// The adjoint of project_one for Gaussian i: attribute planes read at
// A[k * S + i], the gradient record dsp[3 i .. 3 i + 2], dL/dA written to
// dA[k * dstride + di] (zero for a culled Gaussian).
template <int DEG>
__device__ __forceinline__ void project_bwd_one(const CamArgs &cm, float blur, const float *__restrict__ A, size_t S,
                                                int i, const float4 *__restrict__ dsp, float *__restrict__ dA,
                                                size_t dstride, int di) {
    constexpr int deg = DEG;
    constexpr int n_attr = 11 + 3 * (DEG + 1) * (DEG + 1);
    Fwd f;
    bool vis = geometry(cm, A, S, i, f);
    float a = 0.f, b = 0.f, c = 0.f, det = 0.f;
    if (vis) {
        a = f.a + blur; b = f.b; c = f.c + blur;
        det = proj_det(f, blur);
        vis = det > 0.f;
        if (vis) {
            const float mx = cm.fx * f.ux + cm.cx, my = cm.fy * f.uy + cm.cy;
            const float mid = 0.5f * (a + c);
            const float rad = ceilf(3.f * sqrtf(mid + sqrtf(fmaxf(0.1f, mid * mid - det))));
            const float fx0 = fminf(fmaxf(floorf((mx - rad) * (1.f / QN_TILE)), 0.f), (float)cm.TX);
            const float fy0 = fminf(fmaxf(floorf((my - rad) * (1.f / QN_TILE)), 0.f), (float)cm.TY);
            const float fx1 = fminf(fmaxf(floorf((mx + rad + (QN_TILE - 1)) * (1.f / QN_TILE)), 0.f), (float)cm.TX);
            const float fy1 = fminf(fmaxf(floorf((my + rad + (QN_TILE - 1)) * (1.f / QN_TILE)), 0.f), (float)cm.TY);
            vis = fx1 > fx0 && fy1 > fy0;
        }
    }
    if (!vis) {
#pragma unroll
        for (int k = 0; k < n_attr; ++k) dA[k * dstride + di] = 0.f;
        return;
    }
    const float4 g0 = dsp[3 * (size_t)i], g1 = dsp[3 * (size_t)i + 1], g2 = dsp[3 * (size_t)i + 2];
    const float tx = f.t[0], ty = f.t[1], tz = f.t[2];
    float dp[3] = {0.f, 0.f, 0.f}, dt[3] = {0.f, 0.f, 0.f};
    // opacity = sigmoid(logit)
    const float op = 1.f / (1.f + expf(-A[10 * S + i]));
    dA[10 * dstride + di] = g0.z * op * (1.f - op);
    // colour
    {
        float vx = A[i] - cm.cp[0], vy = A[S + i] - cm.cp[1], vz = A[2 * S + i] - cm.cp[2];
        const float vn = sqrtf(vx * vx + vy * vy + vz * vz), inv = 1.f / vn;
        const float x = vx * inv, y = vy * inv, z = vz * inv;
        float Y[16];
        sh_basis(deg, x, y, z, Y);
        constexpr int K = (deg + 1) * (deg + 1);
        float col[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) col[ch] = fmaf(A[(11 + 3 * k + ch) * S + i], Y[k], col[ch]);
        const float gr[3] = {col[0] > 0.f ? g2.x : 0.f, col[1] > 0.f ? g2.y : 0.f, col[2] > 0.f ? g2.z : 0.f};
        float w[16];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float s = 0.f;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                dA[(11 + 3 * k + ch) * dstride + di] = gr[ch] * Y[k];
                s = fmaf(gr[ch], A[(11 + 3 * k + ch) * S + i], s);
            }
            w[k] = s;
        }
        float gx = 0.f, gy = 0.f, gz = 0.f;
        sh_grad(deg, x, y, z, w, gx, gy, gz);
        const float dd = gx * x + gy * y + gz * z;
        dp[0] += (gx - x * dd) * inv;
        dp[1] += (gy - y * dd) * inv;
        dp[2] += (gz - z * dd) * inv;
    }
    // mean2d = (fx tx/tz + cx, fy ty/tz + cy)
    const float itz = 1.f / tz, itz2 = itz * itz;
    dt[0] += g0.x * cm.fx * itz;
    dt[1] += g0.y * cm.fy * itz;
    dt[2] -= (g0.x * cm.fx * tx + g0.y * cm.fy * ty) * itz2;
    // conic = Sigma'^-1 with Sigma' = [[a, b], [b, c]], so dL/dSigma' =
    // G = -conic D conic, D = [[dA, dB/2], [dB/2, dC]] the conic's gradient.
    // G is never formed in the image axes: for a needle-like Gaussian its
    // entries there are ~1/lambda2^2 while the long axis sees only its
    // ~1/lambda1^2 part, so v^T G v along the long axis would cancel by
    // kappa^2 (kappa = lambda1 / lambda2).  Instead, in the eigenbasis
    // E = (e1, e2) of Sigma' (lambda1 = mid + r, lambda2 = det / lambda1 with
    // the determinant to one rounding), G = -E L^-1 g L^-1 E^T with
    // g = E^T D E and L = diag(lambda1, lambda2); with u = L^-1 E^T v,
    //   v^T G v = -u^T g u,   G v = -E L^-1 (g u),
    // every term of which is formed without cancellation.
    const float mid = 0.5f * (a + c), hd = 0.5f * (a - c);
    const float rr = sqrtf(hd * hd + b * b);
    const float l1 = mid + rr, il1 = 1.f / l1, il2 = l1 / det;          // 1 / lambda1, 1 / lambda2
    float ex = hd >= 0.f ? hd + rr : b, ey = hd >= 0.f ? b : rr - hd;  // e1, the larger of the two forms
    float nn = ex * ex + ey * ey;
    if (nn == 0.f) { ex = 1.f; ey = 0.f; nn = 1.f; }                    // a == c, b == 0: any basis
    const float en = 1.f / sqrtf(nn);
    const float e1x = ex * en, e1y = ey * en, e2x = -e1y, e2y = e1x;
    const float hb = 0.5f * g1.y;
    const float De1x = g1.x * e1x + hb * e1y, De1y = hb * e1x + g1.z * e1y;
    const float De2x = g1.x * e2x + hb * e2y, De2y = hb * e2x + g1.z * e2y;
    const float q11 = e1x * De1x + e1y * De1y, q12 = e1x * De2x + e1y * De2y, q22 = e2x * De2x + e2y * De2y;
    const float *T = f.Tm;
    // Sigma = Rq diag(S^2) Rq^T, so per axis c with v_c = T Rq[:, c] (column c
    // of Rq seen through T) and w_c = G v_c:
    //   dL/ds_c = S_c dL/dS_c = 2 S_c^2 v_c^T G v_c,
    //   dL/dRq[:, c] = 2 S_c^2 T^T w_c,
    //   dL/dT = 2 G T Sigma = sum_c 2 S_c^2 w_c Rq[:, c]^T.
    float dRq[9], ds[3], dT[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
        const float v0 = f.v[cc], v1 = f.v[3 + cc];
        const float u1 = (e1x * v0 + e1y * v1) * il1, u2 = (e2x * v0 + e2y * v1) * il2;
        const float h1 = q11 * u1 + q12 * u2, h2 = q12 * u1 + q22 * u2;  // g u
        const float s2 = 2.f * f.S[cc] * f.S[cc];
        ds[cc] = -s2 * (u1 * h1 + u2 * h2);
        const float k1 = h1 * il1, k2 = h2 * il2;
        const float w0 = -(e1x * k1 + e2x * k2), w1 = -(e1y * k1 + e2y * k2);
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            dRq[3 * r + cc] = s2 * (T[r] * w0 + T[3 + r] * w1);
            dT[r] = fmaf(s2 * w0, f.Rq[3 * r + cc], dT[r]);
            dT[3 + r] = fmaf(s2 * w1, f.Rq[3 * r + cc], dT[3 + r]);
        }
    }
    // T = J W: dJ = dT W^T; only J00, J02, J11, J12 depend on t
    const float dJ00 = dT[0] * cm.R[0] + dT[1] * cm.R[1] + dT[2] * cm.R[2];
    const float dJ02 = dT[0] * cm.R[6] + dT[1] * cm.R[7] + dT[2] * cm.R[8];
    const float dJ11 = dT[3] * cm.R[3] + dT[4] * cm.R[4] + dT[5] * cm.R[5];
    const float dJ12 = dT[3] * cm.R[6] + dT[4] * cm.R[7] + dT[5] * cm.R[8];
    dt[2] -= (dJ00 * cm.fx + dJ11 * cm.fy) * itz2;
    if (f.ux == f.uxc) {
        dt[0] -= dJ02 * cm.fx * itz2;
        dt[2] += dJ02 * 2.f * cm.fx * tx * itz2 * itz;
    } else {
        dt[2] += dJ02 * cm.fx * f.uxc * itz2;
    }
    if (f.uy == f.uyc) {
        dt[1] -= dJ12 * cm.fy * itz2;
        dt[2] += dJ12 * 2.f * cm.fy * ty * itz2 * itz;
    } else {
        dt[2] += dJ12 * cm.fy * f.uyc * itz2;
    }
#pragma unroll
    for (int e = 0; e < 3; ++e) dp[e] += cm.R[e] * dt[0] + cm.R[3 + e] * dt[1] + cm.R[6 + e] * dt[2];
    const float qw = f.qn[0], qx = f.qn[1], qy = f.qn[2], qz = f.qn[3];
    float dq[4];
    dq[0] = 2.f * (-qz * dRq[1] + qy * dRq[2] + qz * dRq[3] - qx * dRq[5] - qy * dRq[6] + qx * dRq[7]);
    dq[1] = 2.f * (qy * dRq[1] + qz * dRq[2] + qy * dRq[3] - 2.f * qx * dRq[4] - qw * dRq[5] + qz * dRq[6] +
                   qw * dRq[7] - 2.f * qx * dRq[8]);
    dq[2] = 2.f * (-2.f * qy * dRq[0] + qx * dRq[1] + qw * dRq[2] + qx * dRq[3] + qz * dRq[5] - qw * dRq[6] +
                   qz * dRq[7] - 2.f * qy * dRq[8]);
    dq[3] = 2.f * (-2.f * qz * dRq[0] - qw * dRq[1] + qx * dRq[2] + qw * dRq[3] - 2.f * qz * dRq[4] +
                   qy * dRq[5] + qx * dRq[6] + qy * dRq[7]);
    const float qd = qw * dq[0] + qx * dq[1] + qy * dq[2] + qz * dq[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) dA[(3 + k) * dstride + di] = (dq[k] - f.qn[k] * qd) * f.qinv;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        dA[(7 + k) * dstride + di] = ds[k];
        dA[k * dstride + di] = dp[k];
    }
}

inline int cam_args(const qn_camera *cam, CamArgs *c) {
    QN_REQUIRE(cam, "camera is required");
    QN_REQUIRE(cam->width > 0 && cam->height > 0 && cam->width <= QN_TILE * QN_MAX_TILES_X &&
                   cam->height <= QN_TILE * QN_MAX_TILES_Y,
               "image size %dx%d out of range", cam->width, cam->height);
    QN_REQUIRE(cam->fx > 0.f && cam->fy > 0.f && cam->near_plane > 0.f, "bad intrinsics or near plane");
    for (int k = 0; k < 9; ++k) c->R[k] = cam->R[k];
    for (int k = 0; k < 3; ++k) {
        c->t[k] = cam->t[k];
        c->cp[k] = cam->campos[k];
    }
    c->fx = cam->fx; c->fy = cam->fy; c->cx = cam->cx; c->cy = cam->cy;
    c->near_plane = cam->near_plane;
    c->limx = (float)(1.3 * 0.5 * cam->width / cam->fx);
    c->limy = (float)(1.3 * 0.5 * cam->height / cam->fy);
    c->W = cam->width; c->H = cam->height;
    c->TX = (cam->width + QN_TILE - 1) / QN_TILE;
    c->TY = (cam->height + QN_TILE - 1) / QN_TILE;
    return QN_OK;
}

}  // namespace
}  // namespace qn
