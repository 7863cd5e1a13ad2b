/*
 * queen_oracle.c -- plain CPU FP64 oracle of QUEEN's per-frame residual
 * training path (arXiv 2412.04469).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker: it is compiled into
 * liboracle.so and called only by tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py.  The product library never
 * links, loads or calls it, and it shares no code, header, table or
 * constant with the CUDA sources.
 *
 * Everything is written as the plain definition of what the paper computes,
 * in double precision, with no blocking, fusion or reordering beyond what the
 * definition states.  OpenMP pragmas only split independent outer loops
 * (tiles / Gaussians) across host cores.
 *
 *   Sec. 3.1, Eq. 1   EWA projection  p' = Pi(p), Sigma' = J W Sigma W^T J^T
 *   Sec. 3.1, Eq. 2   front-to-back alpha compositing
 *   Sec. 3.2, Eq. 4   A_t = A_{t-1} + R_t
 *   Sec. 3.2.1, Eq. 5 r = D float(round(l_hat))   (straight-through estimator)
 *   Sec. 3.2.2, Eq. 6-8  hard-concrete gate and its L0 penalty
 *
 * Readings where the paper is silent (it only cites the 3D-GS rasterizer):
 *   - alpha = min(0.99, o exp(power)); skipped when alpha < 1/255;
 *     compositing stops before the Gaussian that would push T below 1e-4.
 *     (power <= 0 for a positive definite conic; the 3D-GS rasterizer's
 *     "power > 0" skip only fires on rounding at a footprint's centre, where
 *     it would drop the Gaussian's largest term, and is not taken.)
 *   - pixel (u, v) is sampled at (u + 0.5, v + 0.5); p' = (fx x/z + cx, fy y/z + cy).
 *   - Sigma' gets `blur` added to its diagonal (opacity is not rescaled).
 *   - radius = ceil(3 sqrt(lambda_max)), lambda_max = mid + sqrt(max(0.1, mid^2 - det));
 *     tile rect = [floor((p'-r)/16), floor((p'+r+15)/16)) clamped to the grid.
 *   - Gaussians with t_z <= near, det <= 0 or an empty rect are culled.
 *   - In J the ratios x/z, y/z are clamped to +-1.3 * (half-extent / focal);
 *     the clamp passes no gradient to its argument.
 *   - residuals are added to raw parameters: position, unnormalised quaternion
 *     (w,x,y,z), log-scale, logit-opacity, SH coefficients.
 *   - real spherical harmonics without the Condon-Shortley phase, index
 *     k = l^2 + l + m; colour = sum_k h_k Y_k(dir) + 0.5, clamped at 0.
 *   - latents round half to even and saturate to [-128, 127]; the backward is
 *     the identity (plain straight-through estimator).
 *   - the 0.99 alpha cap passes zero gradient.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_TILE 16
#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics, built from the general polynomial formula.      */
/*   r^l Y_l^m = sqrt((2l+1)/4pi) * Pi_l^|m|(z) * {sqrt2 A_m | 1 | sqrt2 B_|m|}*/
/*   Pi_l^m(z) = sqrt((l-m)!/(l+m)!) sum_k (-1)^k 2^-l C(l,k) C(2l-2k,l)      */
/*               (l-2k)!/(l-2k-m)! r^2k z^(l-2k-m)                             */
/*   A_m = sum_p C(m,p) x^p y^(m-p) cos((m-p) pi/2), B_m likewise with sin.   */
/* Stored as homogeneous polynomials c[a][b] * x^a y^b z^(l-a-b).             */
/* ------------------------------------------------------------------------ */
#define OR_SH_MAXDEG 3
#define OR_SH_MAXK 16

typedef struct {
    int l;
    double c[OR_SH_MAXDEG + 1][OR_SH_MAXDEG + 1];
} or_shpoly;

static or_shpoly g_sh[OR_SH_MAXK];
static int g_sh_ready = 0;

static double or_fact(int k) {
    double r = 1.0;
    for (int i = 2; i <= k; ++i) r *= (double)i;
    return r;
}

static double or_binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    return or_fact(n) / (or_fact(k) * or_fact(n - k));
}

static void or_sh_build(void) {
    if (g_sh_ready) return;
    for (int l = 0; l <= OR_SH_MAXDEG; ++l) {
        for (int m = -l; m <= l; ++m) {
            or_shpoly *P = &g_sh[l * l + l + m];
            memset(P, 0, sizeof(*P));
            P->l = l;
            int am = m < 0 ? -m : m;
            double norm = sqrt((2.0 * l + 1.0) / (4.0 * OR_PI)) * (m != 0 ? sqrt(2.0) : 1.0) *
                          sqrt(or_fact(l - am) / or_fact(l + am));
            double xy[OR_SH_MAXDEG + 1] = {0};   /* coefficient of x^p y^(am-p) */
            if (m == 0) {
                xy[0] = 1.0;
            } else {
                for (int p = 0; p <= am; ++p) {
                    int r = (am - p) % 4;
                    double trig;
                    if (m > 0) trig = (r == 0) ? 1.0 : (r == 2 ? -1.0 : 0.0);   /* cos */
                    else       trig = (r == 1) ? 1.0 : (r == 3 ? -1.0 : 0.0);   /* sin */
                    xy[p] = or_binom(am, p) * trig;
                }
            }
            for (int k = 0; 2 * k <= l - am; ++k) {
                double zc = ((k & 1) ? -1.0 : 1.0) * pow(2.0, -l) * or_binom(l, k) *
                            or_binom(2 * l - 2 * k, l) * or_fact(l - 2 * k) / or_fact(l - 2 * k - am);
                /* r^2k = sum_{i+j+h=k} k!/(i! j! h!) x^2i y^2j z^2h */
                for (int i = 0; i <= k; ++i)
                    for (int j = 0; i + j <= k; ++j) {
                        int h = k - i - j;
                        double mc = or_fact(k) / (or_fact(i) * or_fact(j) * or_fact(h));
                        for (int p = 0; p <= am; ++p) {
                            if (xy[p] == 0.0) continue;
                            P->c[2 * i + p][2 * j + (am - p)] += norm * zc * mc * xy[p];
                        }
                    }
            }
        }
    }
    g_sh_ready = 1;
}

static double or_ipow(double x, int e) {
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

/* Y[k] and, if dY != NULL, the gradient of the polynomial dY[3k+0..2] at d. */
static void or_sh_eval(int degree, const double d[3], double *Y, double *dY) {
    or_sh_build();
    int K = (degree + 1) * (degree + 1);
    for (int k = 0; k < K; ++k) {
        const or_shpoly *P = &g_sh[k];
        int l = P->l;
        double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int a = 0; a <= l; ++a)
            for (int b = 0; a + b <= l; ++b) {
                double c = P->c[a][b];
                if (c == 0.0) continue;
                int e = l - a - b;
                v += c * or_ipow(d[0], a) * or_ipow(d[1], b) * or_ipow(d[2], e);
                if (a > 0) gx += c * a * or_ipow(d[0], a - 1) * or_ipow(d[1], b) * or_ipow(d[2], e);
                if (b > 0) gy += c * b * or_ipow(d[0], a) * or_ipow(d[1], b - 1) * or_ipow(d[2], e);
                if (e > 0) gz += c * e * or_ipow(d[0], a) * or_ipow(d[1], b) * or_ipow(d[2], e - 1);
            }
        Y[k] = v;
        if (dY) {
            dY[3 * k + 0] = gx;
            dY[3 * k + 1] = gy;
            dY[3 * k + 2] = gz;
        }
    }
}

/* Exported for the basis pins (orthonormality, library comparison). */
void or_sh_basis(int degree, const double *dirs, int n, double *Y, double *dY) {
    int K = (degree + 1) * (degree + 1);
    for (int i = 0; i < n; ++i)
        or_sh_eval(degree, dirs + 3 * i, Y + (size_t)K * i, dY ? dY + (size_t)3 * K * i : NULL);
}

/* ------------------------------------------------------------------------ */
/* Residual decode + gate (Eq. 4-8).                                         */
/* ------------------------------------------------------------------------ */
static double or_sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

static double or_latent(double v, int round_latents) {
    if (!round_latents) return v;
    double r = nearbyint(v);           /* round half to even (default FP mode) */
    if (r > 127.0) r = 127.0;
    if (r < -128.0) r = -128.0;
    return r;
}

/*
 * prev/out: [n_attr][n] raw attributes; lat: [sum L_c][n]; dec: per category
 * c a row-major M_c x L_c block, categories concatenated; lp: [3][n];
 * log_alpha: [n].  Category c adds to attribute planes
 * attr_begin[c] .. attr_begin[c] + attr_count[c] - 1.
 */
void or_decode(int n, int n_attr, const double *prev, int n_cat, const int *attr_begin,
               const int *attr_count, const int *lat_dim, const double *lat, const double *dec,
               int round_latents, const double *lp, const double *log_alpha, double tau,
               double gamma0, double gamma1, double *out, double *gate, double *lreg) {
    memcpy(out, prev, sizeof(double) * (size_t)n_attr * n);
    double reg = 0.0;
    double shift = tau * log(-gamma0 / gamma1);
    for (int i = 0; i < n; ++i) {
        double gh = or_sigmoid(log_alpha[i] / tau);               /* Eq. 6 */
        double gt = gh * (gamma1 - gamma0) + gamma0;              /* Eq. 7 */
        double g = fmin(1.0, fmax(0.0, gt));
        gate[i] = g;
        for (int d = 0; d < 3; ++d) out[(size_t)d * n + i] += g * lp[(size_t)d * n + i];
        reg += or_sigmoid(log_alpha[i] - shift);                  /* Eq. 8 */
    }
    int lo = 0, dofs = 0;
    for (int c = 0; c < n_cat; ++c) {
        int M = attr_count[c], L = lat_dim[c];
        for (int i = 0; i < n; ++i)
            for (int r = 0; r < M; ++r) {
                double acc = 0.0;                                 /* Eq. 5: D float(l) */
                for (int k = 0; k < L; ++k)
                    acc += dec[dofs + r * L + k] * or_latent(lat[(size_t)(lo + k) * n + i], round_latents);
                out[(size_t)(attr_begin[c] + r) * n + i] += acc;  /* Eq. 4 */
            }
        lo += L;
        dofs += M * L;
    }
    *lreg = reg;
}

void or_decode_bwd(int n, int n_attr, int n_cat, const int *attr_begin, const int *attr_count,
                   const int *lat_dim, const double *lat, const double *dec, int round_latents,
                   const double *lp, const double *log_alpha, double tau, double gamma0,
                   double gamma1, const double *d_out, double d_lreg, const uint8_t *skip,
                   double *d_lat, double *d_dec, double *d_lp, double *d_log_alpha) {
    (void)n_attr;
    double shift = tau * log(-gamma0 / gamma1);
    for (int i = 0; i < n; ++i) {
        int sk = skip ? skip[i] : 0;
        double gh = or_sigmoid(log_alpha[i] / tau);
        double gt = gh * (gamma1 - gamma0) + gamma0;
        double g = fmin(1.0, fmax(0.0, gt));
        double dg_dla = (gt > 0.0 && gt < 1.0) ? (gamma1 - gamma0) * gh * (1.0 - gh) / tau : 0.0;
        double dot = 0.0;
        for (int d = 0; d < 3; ++d) {
            double dp = d_out[(size_t)d * n + i];
            d_lp[(size_t)d * n + i] = sk ? 0.0 : g * dp;
            dot += dp * lp[(size_t)d * n + i];
        }
        double p = or_sigmoid(log_alpha[i] - shift);
        d_log_alpha[i] = sk ? 0.0 : dot * dg_dla + d_lreg * p * (1.0 - p);
    }
    int lo = 0, dofs = 0;
    for (int c = 0; c < n_cat; ++c) {
        int M = attr_count[c], L = lat_dim[c];
        for (int r = 0; r < M; ++r)
            for (int k = 0; k < L; ++k) d_dec[dofs + r * L + k] = 0.0;
        for (int i = 0; i < n; ++i) {
            int sk = skip ? skip[i] : 0;
            for (int k = 0; k < L; ++k) {
                double acc = 0.0;                                 /* STE: D^T dr */
                for (int r = 0; r < M; ++r)
                    acc += dec[dofs + r * L + k] * d_out[(size_t)(attr_begin[c] + r) * n + i];
                d_lat[(size_t)(lo + k) * n + i] = sk ? 0.0 : acc;
            }
            if (sk) continue;
            for (int r = 0; r < M; ++r) {
                double dr = d_out[(size_t)(attr_begin[c] + r) * n + i];
                for (int k = 0; k < L; ++k)
                    d_dec[dofs + r * L + k] += dr * or_latent(lat[(size_t)(lo + k) * n + i], round_latents);
            }
        }
        lo += L;
        dofs += M * L;
    }
}

/* ------------------------------------------------------------------------ */
/* EWA projection + SH colour (Eq. 1).                                       */
/* cam: R[9] (row-major world->camera), t[3], fx, fy, cx, cy, near, campos[3] */
/* ------------------------------------------------------------------------ */
static void or_quat_rot(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static int or_clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* distance of v to the nearest integer, relative to max(1, |v|) */
static int or_near_int(double v, double eps) {
    double f = v - floor(v);
    double d = f < 0.5 ? f : 1.0 - f;
    return d <= eps * fmax(1.0, fabs(v));
}

typedef struct {
    double t[3], ux, uy, uxc, uyc, J[6], T[6], Sig[9], M[9], Rq[9], S[3], qn[4], qnorm;
    double a, b, c, det, dir[3], vnorm, raw[3];
} or_proj_tmp;

/* Projection of one Gaussian; returns 1 if visible.  fr gets fragility bits
 * (a decision that FP32 rounding could flip, within eps_g relative):
 *   1 near plane, 2 radius ceil, 4 rect floor, 8 det sign, 16 opacity bound,
 *   and 32 << k for the rect edges k (x0, y0, x1, y1) such a flip can move
 *   (a radius flip moves all four).
 * out2d = (mx, my, conic a, b, c, opacity, r, g, b, depth); for a fragile
 * Gaussian the 2D footprint is filled in even when it is culled, so that the
 * renderer can tell which pixels the flipped decision could reach. */
static int or_project_one(int i, int n, int sh_degree, const double *A, const double *cam,
                          int W, int H, double blur, int tight, double eps_g, or_proj_tmp *w,
                          double out2d[10], int *radius_out, int rect_out[4], int frag_rect[4],
                          int *fr) {
    const double *R = cam, *tv = cam + 9;
    double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15], nearp = cam[16];
    const double *cpos = cam + 17;
    int TX = (W + OR_TILE - 1) / OR_TILE, TY = (H + OR_TILE - 1) / OR_TILE;
    double p[3] = {A[(size_t)0 * n + i], A[(size_t)1 * n + i], A[(size_t)2 * n + i]};
    *fr = 0;
    memset(out2d, 0, sizeof(double) * 10);
    *radius_out = 0;
    for (int k = 0; k < 4; ++k) rect_out[k] = frag_rect[k] = 0;

    for (int r = 0; r < 3; ++r) w->t[r] = R[3 * r] * p[0] + R[3 * r + 1] * p[1] + R[3 * r + 2] * p[2] + tv[r];
    double tz = w->t[2];
    out2d[9] = tz;                                        /* depth */
    if (tz <= 1e-6) return 0;                             /* behind the camera: never fragile */
    if (fabs(tz - nearp) <= eps_g * nearp) *fr |= 1;

    double qr[4], qq = 0.0;
    for (int k = 0; k < 4; ++k) { qr[k] = A[(size_t)(3 + k) * n + i]; qq += qr[k] * qr[k]; }
    w->qnorm = sqrt(qq);
    for (int k = 0; k < 4; ++k) w->qn[k] = qr[k] / w->qnorm;
    or_quat_rot(w->qn, w->Rq);
    for (int k = 0; k < 3; ++k) w->S[k] = exp(A[(size_t)(7 + k) * n + i]);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) w->M[3 * r + c] = w->Rq[3 * r + c] * w->S[c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += w->M[3 * r + k] * w->M[3 * c + k];
            w->Sig[3 * r + c] = s;                        /* Sigma = R S S^T R^T */
        }

    double limx = 1.3 * 0.5 * W / fx, limy = 1.3 * 0.5 * H / fy;
    w->ux = w->t[0] / tz;
    w->uy = w->t[1] / tz;
    w->uxc = fmin(limx, fmax(-limx, w->ux));
    w->uyc = fmin(limy, fmax(-limy, w->uy));
    double *J = w->J;                                     /* affine Jacobian of the projection */
    J[0] = fx / tz; J[1] = 0.0;     J[2] = -fx * w->uxc / tz;
    J[3] = 0.0;     J[4] = fy / tz; J[5] = -fy * w->uyc / tz;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += J[3 * r + k] * R[3 * k + c];
            w->T[3 * r + c] = s;                          /* T = J W */
        }
    double C2[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) s += w->T[3 * r + k] * w->Sig[3 * k + l] * w->T[3 * c + l];
            C2[2 * r + c] = s;                            /* Sigma' = T Sigma T^T */
        }
    w->a = C2[0] + blur;
    w->b = C2[1];
    w->c = C2[3] + blur;
    w->det = w->a * w->c - w->b * w->b;
    if (fabs(w->det) <= eps_g * w->a * w->c) *fr |= 8;

    double mx = fx * w->ux + cx, my = fy * w->uy + cy;
    double mid = 0.5 * (w->a + w->c);
    double lam = mid + sqrt(fmax(0.1, mid * mid - w->det));
    double r3 = 3.0 * sqrt(lam);
    int rad = (int)ceil(r3);
    if (or_near_int(r3, eps_g)) *fr |= 2 | (15 << 5);
    double ex[4] = {(mx - rad) / OR_TILE, (my - rad) / OR_TILE, (mx + rad + OR_TILE - 1) / OR_TILE,
                    (my + rad + OR_TILE - 1) / OR_TILE};
    for (int k = 0; k < 4; ++k)
        if (or_near_int(ex[k], eps_g)) *fr |= 4 | (32 << k);
    int rc[4] = {or_clampi((int)floor(ex[0]), 0, TX), or_clampi((int)floor(ex[1]), 0, TY),
                 or_clampi((int)floor(ex[2]), 0, TX), or_clampi((int)floor(ex[3]), 0, TY)};
    if (tight) {
        /* tiles the alpha >= 1/255 region can reach: the bounding box of the
         * ellipse q(d) <= k, k = 2 ln(255 o) (+0.01, then +1%), half-widths
         * sqrt(k Sigma'_xx) + 0.01 and sqrt(k Sigma'_yy) + 0.01 */
        double op = or_sigmoid(A[(size_t)10 * n + i]);
        double k = 2.0 * log(255.0 * op) + 0.01;
        if (fabs(k) <= eps_g * 10.0) *fr |= 16;
        if (k <= 0.0) {
            rc[0] = rc[1] = rc[2] = rc[3] = 0;
        } else {
            double hx = sqrt(1.01 * k * w->a) + 0.01, hy = sqrt(1.01 * k * w->c) + 0.01;
            double tb[4] = {(mx - hx) / OR_TILE, (my - hy) / OR_TILE, (mx + hx) / OR_TILE, (my + hy) / OR_TILE};
            for (int q = 0; q < 4; ++q)
                if (or_near_int(tb[q], eps_g)) *fr |= 4 | (32 << q);
            int t0 = or_clampi((int)floor(tb[0]), 0, TX), t1 = or_clampi((int)floor(tb[1]), 0, TY);
            int t2 = or_clampi((int)floor(tb[2]) + 1, 0, TX), t3 = or_clampi((int)floor(tb[3]) + 1, 0, TY);
            rc[0] = rc[0] > t0 ? rc[0] : t0;
            rc[1] = rc[1] > t1 ? rc[1] : t1;
            rc[2] = rc[2] < t2 ? rc[2] : t2;
            rc[3] = rc[3] < t3 ? rc[3] : t3;
        }
    }
    if (*fr) {
        frag_rect[0] = or_clampi(rc[0] - 1, 0, TX);
        frag_rect[1] = or_clampi(rc[1] - 1, 0, TY);
        frag_rect[2] = or_clampi(rc[2] + 1, 0, TX);
        frag_rect[3] = or_clampi(rc[3] + 1, 0, TY);
    }
    int visible = tz > nearp && w->det > 0.0 && (rc[2] - rc[0]) * (rc[3] - rc[1]) > 0;
    if (!visible && !(*fr && w->det > 0.0)) return 0;

    double K2[3] = {w->c / w->det, -w->b / w->det, w->a / w->det};   /* conic = Sigma'^-1 */
    double v[3] = {p[0] - cpos[0], p[1] - cpos[1], p[2] - cpos[2]};
    w->vnorm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int k = 0; k < 3; ++k) w->dir[k] = v[k] / w->vnorm;
    double Y[OR_SH_MAXK];
    or_sh_eval(sh_degree, w->dir, Y, NULL);
    int K = (sh_degree + 1) * (sh_degree + 1);
    double rgb[3];
    for (int ch = 0; ch < 3; ++ch) {
        double s = 0.5;
        for (int k = 0; k < K; ++k) s += A[(size_t)(11 + 3 * k + ch) * n + i] * Y[k];
        w->raw[ch] = s;
        rgb[ch] = s > 0.0 ? s : 0.0;
    }
    out2d[0] = mx; out2d[1] = my;
    out2d[2] = K2[0]; out2d[3] = K2[1]; out2d[4] = K2[2];
    out2d[5] = or_sigmoid(A[(size_t)10 * n + i]);
    out2d[6] = rgb[0]; out2d[7] = rgb[1]; out2d[8] = rgb[2];
    if (!visible) return 0;
    *radius_out = rad;
    for (int k = 0; k < 4; ++k) rect_out[k] = rc[k];
    return 1;
}

/*
 * Outputs (all [.][n] planes): mean2d[2], conic[3] (a, b, c of Sigma'^-1 with
 * power = -0.5 (a dx^2 + c dy^2) - b dx dy), opac, rgb[3], depth, radius,
 * rect[4] = (x0, y0, x1, y1) in tiles (half-open; all 0 when culled; with
 * `tight` also limited to the tiles the alpha >= 1/255 ellipse can reach),
 * fragile bits, and frag_rect[4] = the tiles whose pixels a fragile Gaussian
 * may reach.
 */
void or_project(int n, int n_attr, int sh_degree, const double *A, const double *cam, int W,
                int H, double blur, int tight, double eps_g, double *mean2d, double *conic,
                double *opac, double *rgb, double *depth, int *radius, int *rect, int *fragile,
                int *frag_rect) {
    (void)n_attr;
    or_sh_build();
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        or_proj_tmp w;
        double o[10];
        int rad, rc[4], frc[4], fr;
        or_project_one(i, n, sh_degree, A, cam, W, H, blur, tight, eps_g, &w, o, &rad, rc, frc, &fr);
        mean2d[i] = o[0]; mean2d[(size_t)n + i] = o[1];
        conic[i] = o[2]; conic[(size_t)n + i] = o[3]; conic[(size_t)2 * n + i] = o[4];
        opac[i] = o[5];
        rgb[i] = o[6]; rgb[(size_t)n + i] = o[7]; rgb[(size_t)2 * n + i] = o[8];
        depth[i] = o[9];
        radius[i] = rad;
        for (int k = 0; k < 4; ++k) {
            rect[(size_t)k * n + i] = rc[k];
            frag_rect[(size_t)k * n + i] = frc[k];
        }
        fragile[i] = fr;
    }
}

/* Analytic adjoint of or_project: d_attrs[n_attr][n] from the 2D gradients. */
void or_project_bwd(int n, int n_attr, int sh_degree, const double *A, const double *cam, int W,
                    int H, double blur, const double *d_mean2d, const double *d_conic,
                    const double *d_opac, const double *d_rgb, double *d_attrs) {
    or_sh_build();
    memset(d_attrs, 0, sizeof(double) * (size_t)n_attr * n);
    const double *R = cam;
    double fx = cam[12], fy = cam[13];
    int K = (sh_degree + 1) * (sh_degree + 1);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        or_proj_tmp w;
        double o[10];
        int rad, rc[4], frc[4], fr;
        if (!or_project_one(i, n, sh_degree, A, cam, W, H, blur, 0, 0.0, &w, o, &rad, rc, frc, &fr))
            continue;
        double dp[3] = {0, 0, 0}, dt[3] = {0, 0, 0};
        /* opacity = sigmoid(logit) */
        double op = o[5];
        d_attrs[(size_t)10 * n + i] = d_opac[i] * op * (1.0 - op);
        /* colour: c = max(0, 0.5 + sum_k h_k Y_k(dir)) */
        double Y[OR_SH_MAXK], dY[3 * OR_SH_MAXK];
        or_sh_eval(sh_degree, w.dir, Y, dY);
        double ddir[3] = {0, 0, 0};
        for (int ch = 0; ch < 3; ++ch) {
            if (!(w.raw[ch] > 0.0)) continue;
            double g = d_rgb[(size_t)ch * n + i];
            for (int k = 0; k < K; ++k) {
                d_attrs[(size_t)(11 + 3 * k + ch) * n + i] = g * Y[k];
                double h = A[(size_t)(11 + 3 * k + ch) * n + i];
                for (int e = 0; e < 3; ++e) ddir[e] += g * h * dY[3 * k + e];
            }
        }
        double dd = ddir[0] * w.dir[0] + ddir[1] * w.dir[1] + ddir[2] * w.dir[2];
        for (int e = 0; e < 3; ++e) dp[e] += (ddir[e] - w.dir[e] * dd) / w.vnorm;
        /* mean2d = (fx tx/tz + cx, fy ty/tz + cy) */
        double tx = w.t[0], ty = w.t[1], tz = w.t[2];
        double gmx = d_mean2d[i], gmy = d_mean2d[(size_t)n + i];
        dt[0] += gmx * fx / tz;
        dt[1] += gmy * fy / tz;
        dt[2] += -(gmx * fx * tx + gmy * fy * ty) / (tz * tz);
        /* conic (A,B,C) = (c, -b, a)/det  ->  (a, b, c) of Sigma' */
        double a = w.a, b = w.b, c = w.c, det = w.det, d2 = det * det;
        double gA = d_conic[i], gB = d_conic[(size_t)n + i], gC = d_conic[(size_t)2 * n + i];
        double da = (-c * c * gA + b * c * gB - b * b * gC) / d2;
        double dc = (-b * b * gA + a * b * gB - a * a * gC) / d2;
        double db = (2.0 * b * c * gA - (det + 2.0 * b * b) * gB + 2.0 * a * b * gC) / d2;
        /* Sigma' = T Sigma T^T: G = dL/dSigma' (symmetric) */
        double G[4] = {da, 0.5 * db, 0.5 * db, dc};
        double dT[6], dSig[9];
        for (int r = 0; r < 2; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                double s = 0.0;                            /* dT = 2 G T Sigma */
                for (int k = 0; k < 2; ++k)
                    for (int l = 0; l < 3; ++l) s += G[2 * r + k] * w.T[3 * k + l] * w.Sig[3 * l + cc];
                dT[3 * r + cc] = 2.0 * s;
            }
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                double s = 0.0;                            /* dSigma = T^T G T */
                for (int k = 0; k < 2; ++k)
                    for (int l = 0; l < 2; ++l) s += w.T[3 * k + r] * G[2 * k + l] * w.T[3 * l + cc];
                dSig[3 * r + cc] = s;
            }
        /* T = J W  ->  dJ = dT W^T */
        double dJ[6];
        for (int r = 0; r < 2; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += dT[3 * r + k] * R[3 * cc + k];
                dJ[3 * r + cc] = s;
            }
        dt[2] += -dJ[0] * fx / (tz * tz) - dJ[4] * fy / (tz * tz);
        if (w.ux == w.uxc) {                              /* J02 = -fx tx / tz^2 */
            dt[0] += -dJ[2] * fx / (tz * tz);
            dt[2] += dJ[2] * 2.0 * fx * tx / (tz * tz * tz);
        } else {                                          /* J02 = -fx uxc / tz */
            dt[2] += dJ[2] * fx * w.uxc / (tz * tz);
        }
        if (w.uy == w.uyc) {
            dt[1] += -dJ[5] * fy / (tz * tz);
            dt[2] += dJ[5] * 2.0 * fy * ty / (tz * tz * tz);
        } else {
            dt[2] += dJ[5] * fy * w.uyc / (tz * tz);
        }
        /* t = W p + t_w */
        for (int e = 0; e < 3; ++e) dp[e] += R[e] * dt[0] + R[3 + e] * dt[1] + R[6 + e] * dt[2];
        /* Sigma = M M^T, M = Rq diag(S) */
        double dM[9];
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += (dSig[3 * r + k] + dSig[3 * k + r]) * w.M[3 * k + cc];
                dM[3 * r + cc] = s;
            }
        double dRq[9], ds[3];
        for (int cc = 0; cc < 3; ++cc) {
            double s = 0.0;
            for (int r = 0; r < 3; ++r) {
                dRq[3 * r + cc] = dM[3 * r + cc] * w.S[cc];
                s += dM[3 * r + cc] * w.Rq[3 * r + cc];
            }
            ds[cc] = s * w.S[cc];
        }
        /* Rq(q_n): partial derivatives of each entry w.r.t. (w, x, y, z) */
        double qw = w.qn[0], qx = w.qn[1], qy = w.qn[2], qz = w.qn[3];
        double dq[4];
        dq[0] = 2 * (-qz * dRq[1] + qy * dRq[2] + qz * dRq[3] - qx * dRq[5] - qy * dRq[6] + qx * dRq[7]);
        dq[1] = 2 * (qy * dRq[1] + qz * dRq[2] + qy * dRq[3] - 2 * qx * dRq[4] - qw * dRq[5] + qz * dRq[6] +
                     qw * dRq[7] - 2 * qx * dRq[8]);
        dq[2] = 2 * (-2 * qy * dRq[0] + qx * dRq[1] + qw * dRq[2] + qx * dRq[3] + qz * dRq[5] - qw * dRq[6] +
                     qz * dRq[7] - 2 * qy * dRq[8]);
        dq[3] = 2 * (-2 * qz * dRq[0] - qw * dRq[1] + qx * dRq[2] + qw * dRq[3] - 2 * qz * dRq[4] + qy * dRq[5] +
                     qx * dRq[6] + qy * dRq[7]);
        double qd = 0.0;
        for (int k = 0; k < 4; ++k) qd += w.qn[k] * dq[k];
        for (int k = 0; k < 4; ++k) d_attrs[(size_t)(3 + k) * n + i] = (dq[k] - w.qn[k] * qd) / w.qnorm;
        for (int k = 0; k < 3; ++k) d_attrs[(size_t)(7 + k) * n + i] = ds[k];
        for (int k = 0; k < 3; ++k) d_attrs[(size_t)k * n + i] = dp[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Tile binning (integer path).  Pairs are emitted in Gaussian index order,  */
/* tiles row-major inside each rect; key = (tile << 32) | bits(float depth). */
/* The result is the stable sort of the pairs by key.                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint64_t key;
    uint64_t seq;
    uint32_t val;
} or_pair;

static int or_pair_cmp(const void *pa, const void *pb) {
    const or_pair *a = (const or_pair *)pa, *b = (const or_pair *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->seq != b->seq) return a->seq < b->seq ? -1 : 1;
    return 0;
}

/* rect: [4][n] (x0, y0, x1, y1); a Gaussian with an empty rect emits nothing. */
int64_t or_bin_count(int n, const int *rect) {
    int64_t P = 0;
    for (int i = 0; i < n; ++i) {
        int w = rect[(size_t)2 * n + i] - rect[i], h = rect[(size_t)3 * n + i] - rect[(size_t)n + i];
        if (w > 0 && h > 0) P += (int64_t)w * h;
    }
    return P;
}

/* ranges: [n_tiles][2] = (#pairs with tile < t, #pairs with tile <= t). */
int64_t or_bin_sort(int n, const float *depth, const int *rect, int tiles_x, int tiles_y,
                    uint64_t *keys, uint32_t *vals, uint32_t *ranges) {
    int64_t P = or_bin_count(n, rect);
    or_pair *pr = (or_pair *)malloc(sizeof(or_pair) * (size_t)(P > 0 ? P : 1));
    if (!pr) return -1;
    int64_t e = 0;
    for (int i = 0; i < n; ++i) {
        int x0 = rect[i], y0 = rect[(size_t)n + i], x1 = rect[(size_t)2 * n + i], y1 = rect[(size_t)3 * n + i];
        if (x1 <= x0 || y1 <= y0) continue;
        uint32_t bits;
        memcpy(&bits, &depth[i], 4);
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = x0; tx < x1; ++tx) {
                pr[e].key = ((uint64_t)(uint32_t)(ty * tiles_x + tx) << 32) | bits;
                pr[e].seq = (uint64_t)e;
                pr[e].val = (uint32_t)i;
                ++e;
            }
    }
    qsort(pr, (size_t)P, sizeof(or_pair), or_pair_cmp);
    int nt = tiles_x * tiles_y;
    for (int t = 0; t < nt; ++t) ranges[2 * t] = ranges[2 * t + 1] = 0;
    int64_t *cnt = (int64_t *)calloc((size_t)nt + 1, sizeof(int64_t));
    for (int64_t k = 0; k < P; ++k) {
        keys[k] = pr[k].key;
        vals[k] = pr[k].val;
        cnt[(pr[k].key >> 32) + 1] += 1;
    }
    for (int t = 0; t < nt; ++t) {
        cnt[t + 1] += cnt[t];
        ranges[2 * t] = (uint32_t)cnt[t];
        ranges[2 * t + 1] = (uint32_t)cnt[t + 1];
    }
    free(cnt);
    free(pr);
    return P;
}

/* ------------------------------------------------------------------------ */
/* Compositing (Eq. 2) and its adjoint.                                      */
/* For every tile, the list is every visible Gaussian whose rect contains    */
/* the tile, ordered by (depth, index).                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    double depth;
    int idx;
} or_dk;

static int or_dk_cmp(const void *pa, const void *pb) {
    const or_dk *a = (const or_dk *)pa, *b = (const or_dk *)pb;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static int or_tile_list(int n, const int *rect, const double *depth, int tx, int ty, or_dk *buf) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
        int x0 = rect[i], y0 = rect[(size_t)n + i], x1 = rect[(size_t)2 * n + i], y1 = rect[(size_t)3 * n + i];
        if (x1 <= x0 || y1 <= y0) continue;
        if (tx >= x0 && tx < x1 && ty >= y0 && ty < y1) {
            buf[m].depth = depth[i];
            buf[m].idx = i;
            ++m;
        }
    }
    qsort(buf, (size_t)m, sizeof(or_dk), or_dk_cmp);
    return m;
}

typedef struct {
    double alpha_min, alpha_max, t_min;
} or_consts;

static const or_consts OR_C = {1.0 / 255.0, 0.99, 1e-4};

/* contributor record for the adjoint replay */
typedef struct {
    int g;
    double alpha, G, T, dx, dy;
    int capped;
} or_contrib;

/*
 * Composites one pixel.  Returns the number of list entries up to and
 * including the last contributor (0 if none); writes color, final T and the
 * fragility bits (1 alpha near 1/255 or 0.99 within eps relative, 2 T near
 * 1e-4 within eps_t relative; 4 consecutive contributors whose depths lie
 * within eps_d relative, an order FP32 depths could swap).  If rec != NULL
 * the contributors are stored.
 */
static int or_pixel(const or_dk *list, int m, int n, double px, double py, const double *mean2d,
                    const double *conic, const double *opac, const double *rgb, const double *bg,
                    double eps, double eps_t, double eps_d, double col[3], double *Tout, int *frag, or_contrib *rec,
                    int *nrec) {
    double T = 1.0, C[3] = {0, 0, 0};
    int last = 0, fr = 0, nr = 0;
    double prev_depth = -1.0;
    for (int k = 0; k < m; ++k) {
        int g = list[k].idx;
        double dx = px - mean2d[g], dy = py - mean2d[(size_t)n + g];
        double a = conic[g], b = conic[(size_t)n + g], c = conic[(size_t)2 * n + g];
        double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
        double G = exp(power);
        double v = opac[g] * G;
        if (fabs(v - OR_C.alpha_min) <= eps * OR_C.alpha_min) fr |= 1;
        if (fabs(v - OR_C.alpha_max) <= eps * OR_C.alpha_max) fr |= 1;
        int capped = v > OR_C.alpha_max;
        double alpha = capped ? OR_C.alpha_max : v;
        if (alpha < OR_C.alpha_min) continue;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn - OR_C.t_min) <= eps_t * OR_C.t_min) fr |= 2;
        if (Tn < OR_C.t_min) break;
        if (prev_depth >= 0.0 && fabs(list[k].depth - prev_depth) <= eps_d * list[k].depth) fr |= 4;
        prev_depth = list[k].depth;
        for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[(size_t)ch * n + g] * alpha * T;
        if (rec) {
            rec[nr].g = g; rec[nr].alpha = alpha; rec[nr].G = G; rec[nr].T = T;
            rec[nr].dx = dx; rec[nr].dy = dy; rec[nr].capped = capped;
        }
        ++nr;
        T = Tn;
        last = k + 1;
    }
    for (int ch = 0; ch < 3; ++ch) col[ch] = C[ch] + T * bg[ch];
    *Tout = T;
    *frag = fr;
    if (nrec) *nrec = nr;
    return last;
}

static int or_max_list(int n, const int *rect, int TX, int TY) {
    int *cnt = (int *)calloc((size_t)TX * TY, sizeof(int));
    int mx = 0;
    for (int i = 0; i < n; ++i) {
        int x0 = rect[i], y0 = rect[(size_t)n + i], x1 = rect[(size_t)2 * n + i], y1 = rect[(size_t)3 * n + i];
        for (int ty = y0; ty < y1; ++ty)
            for (int tx = x0; tx < x1; ++tx) cnt[ty * TX + tx]++;
    }
    for (int t = 0; t < TX * TY; ++t) mx = cnt[t] > mx ? cnt[t] : mx;
    free(cnt);
    return mx;
}

/*
 * tiles (nullable): composite only these n_tiles_sel tile indices (a bounded
 * sample); other pixels are left untouched.
 * img: [3][H][W]; T_final, last, fragile: [H][W].  fragile pixel bits: see
 * or_pixel, plus 8 when a fragile Gaussian (frag_g != 0) could change the
 * pixel: it reaches alpha >= (1 - eps)/255 there, and the pixel's tile lies in
 * its frag_rect when the flippable decision is the near plane, the
 * determinant's sign or the opacity bound, or when the Gaussian is culled (the
 * whole footprint can appear or vanish), or else (rect and radius decisions of
 * a visible Gaussian) in the band of tiles a flippable rect edge can add or
 * remove: columns x0 - 1, x0 or x1 - 1, x1 (rows y0 - 1 .. y1) for a vertical
 * edge, likewise rows for a horizontal one.
 */
void or_render_fwd(int n, const double *mean2d, const double *conic, const double *opac,
                   const double *rgb, const double *depth, const int *rect, const int *frag_g,
                   const int *frag_rect, int W, int H, const double *bg, double eps, double eps_t, double eps_d,
                   const int *tiles, int n_tiles_sel, double *img, double *T_final, int *last,
                   int *fragile) {
    int TX = (W + OR_TILE - 1) / OR_TILE, TY = (H + OR_TILE - 1) / OR_TILE;
    int NT = tiles ? n_tiles_sel : TX * TY;
    int maxl = or_max_list(n, rect, TX, TY);
    int nfrag = 0;
    if (frag_g)
        for (int i = 0; i < n; ++i) nfrag += frag_g[i] != 0;
    int *fidx = (int *)malloc(sizeof(int) * (size_t)(nfrag > 0 ? nfrag : 1));
    nfrag = 0;
    if (frag_g)
        for (int i = 0; i < n; ++i)
            if (frag_g[i]) fidx[nfrag++] = i;
#pragma omp parallel
    {
        or_dk *buf = (or_dk *)malloc(sizeof(or_dk) * (size_t)(maxl > 0 ? maxl : 1));
#pragma omp for schedule(dynamic, 1)
        for (int q = 0; q < NT; ++q) {
            int t = tiles ? tiles[q] : q;
            int tx = t % TX, ty = t / TX;
            int m = or_tile_list(n, rect, depth, tx, ty, buf);
            for (int v = ty * OR_TILE; v < (ty + 1) * OR_TILE && v < H; ++v)
                for (int u = tx * OR_TILE; u < (tx + 1) * OR_TILE && u < W; ++u) {
                    double col[3], T;
                    int fr;
                    int l = or_pixel(buf, m, n, u + 0.5, v + 0.5, mean2d, conic, opac, rgb, bg, eps, eps_t, eps_d, col,
                                     &T, &fr, NULL, NULL);
                    for (int f = 0; f < nfrag; ++f) {
                        int i = fidx[f];
                        if (!(tx >= frag_rect[i] && tx < frag_rect[(size_t)2 * n + i] &&
                              ty >= frag_rect[(size_t)n + i] && ty < frag_rect[(size_t)3 * n + i]))
                            continue;
                        if (frag_g[i] & 8) { fr |= 8; continue; }
                        const int x0 = rect[i], y0 = rect[(size_t)n + i], x1 = rect[(size_t)2 * n + i],
                                  y1 = rect[(size_t)3 * n + i];
                        if (!(frag_g[i] & (1 | 16)) && x1 > x0 && y1 > y0) {
                            /* rect or radius decisions of a visible Gaussian only: the edge bands
                             * (a culled one keeps the whole frag_rect) */
                            const int g = frag_g[i];
                            const int iny = ty >= y0 - 1 && ty <= y1, inx = tx >= x0 - 1 && tx <= x1;
                            const int band = ((g & 32) && iny && (tx == x0 - 1 || tx == x0)) ||
                                             ((g & 128) && iny && (tx == x1 - 1 || tx == x1)) ||
                                             ((g & 64) && inx && (ty == y0 - 1 || ty == y0)) ||
                                             ((g & 256) && inx && (ty == y1 - 1 || ty == y1));
                            if (!band) continue;
                        }
                        double dx = u + 0.5 - mean2d[i], dy = v + 0.5 - mean2d[(size_t)n + i];
                        double power = -0.5 * (conic[i] * dx * dx + conic[(size_t)2 * n + i] * dy * dy) -
                                       conic[(size_t)n + i] * dx * dy;
                        if (opac[i] * exp(power) >= (1.0 - eps) * OR_C.alpha_min) fr |= 8;
                    }
                    size_t px = (size_t)v * W + u;
                    for (int ch = 0; ch < 3; ++ch) img[(size_t)ch * W * H + px] = col[ch];
                    T_final[px] = T;
                    last[px] = l;
                    fragile[px] = fr;
                }
        }
        free(buf);
    }
    free(fidx);
}

/*
 * Adjoint of or_render_fwd for an upstream d_img[3][H][W].  Each pixel replays
 * its forward pass to record the contributors, then walks them back to front:
 *   dC/dc_k     = alpha_k T_k
 *   dC/dalpha_k = T_k (c_k - B_k),  B_last = bg,  B_{k-1} = alpha_k c_k + (1 - alpha_k) B_k
 * and alpha_k = o G (uncapped) carries dL/do = dL/dalpha G and
 * dL/dpower = dL/dalpha alpha into the conic and mean.
 * Outputs are [.][n] planes, zeroed first.
 * mag (nullable, [9][n] in the order d_mean2d, d_conic, d_opac, d_rgb):
 * the same sums with every term replaced by its magnitude, each factor that
 * is itself a sum of signed parts by the sum of their magnitudes
 * (dL/dalpha_k by T_k sum_ch |dC_ch| (|c_k| + |B_k|)).  An entry computed in
 * floating point with relative precision u cannot be trusted beyond a small
 * multiple of u mag: where it cancels, mag says by how much.
 */
void or_render_bwd(int n, const double *mean2d, const double *conic, const double *opac,
                   const double *rgb, const double *depth, const int *rect, int W, int H,
                   const double *bg, const double *d_img, const int *tiles, int n_tiles_sel,
                   double *d_mean2d, double *d_conic, double *d_opac, double *d_rgb, double *mag) {
    int TX = (W + OR_TILE - 1) / OR_TILE, TY = (H + OR_TILE - 1) / OR_TILE;
    int NT = tiles ? n_tiles_sel : TX * TY;
    int maxl = or_max_list(n, rect, TX, TY);
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    double *acc = (double *)calloc((size_t)nthr * 9 * n, sizeof(double));
    double *macc = mag ? (double *)calloc((size_t)nthr * 9 * n, sizeof(double)) : NULL;
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = acc + (size_t)tid * 9 * n;
        double *mm = macc ? macc + (size_t)tid * 9 * n : NULL;
        or_dk *buf = (or_dk *)malloc(sizeof(or_dk) * (size_t)(maxl > 0 ? maxl : 1));
        or_contrib *rec = (or_contrib *)malloc(sizeof(or_contrib) * (size_t)(maxl > 0 ? maxl : 1));
#pragma omp for schedule(static, 1)   /* fixed tile -> thread map: reproducible sums */
        for (int q = 0; q < NT; ++q) {
            int t = tiles ? tiles[q] : q;
            int tx = t % TX, ty = t / TX;
            int m = or_tile_list(n, rect, depth, tx, ty, buf);
            for (int v = ty * OR_TILE; v < (ty + 1) * OR_TILE && v < H; ++v)
                for (int u = tx * OR_TILE; u < (tx + 1) * OR_TILE && u < W; ++u) {
                    double col[3], T;
                    int fr, nr;
                    or_pixel(buf, m, n, u + 0.5, v + 0.5, mean2d, conic, opac, rgb, bg, 0.0, 0.0, 0.0, col, &T, &fr, rec,
                             &nr);
                    size_t px = (size_t)v * W + u;
                    double dC[3];
                    for (int ch = 0; ch < 3; ++ch) dC[ch] = d_img[(size_t)ch * W * H + px];
                    double B[3] = {bg[0], bg[1], bg[2]};
                    double Bm[3] = {fabs(bg[0]), fabs(bg[1]), fabs(bg[2])};
                    for (int j = nr - 1; j >= 0; --j) {
                        const or_contrib *r = &rec[j];
                        int g = r->g;
                        double dalpha = 0.0, dalpha_m = 0.0;
                        for (int ch = 0; ch < 3; ++ch) {
                            double c = rgb[(size_t)ch * n + g];
                            my[(size_t)(6 + ch) * n + g] += dC[ch] * r->alpha * r->T;
                            dalpha += dC[ch] * r->T * (c - B[ch]);
                            B[ch] = r->alpha * c + (1.0 - r->alpha) * B[ch];
                            if (mm) {
                                mm[(size_t)(6 + ch) * n + g] += fabs(dC[ch]) * r->alpha * r->T;
                                dalpha_m += fabs(dC[ch]) * r->T * (fabs(c) + Bm[ch]);
                                Bm[ch] = r->alpha * fabs(c) + (1.0 - r->alpha) * Bm[ch];
                            }
                        }
                        if (r->capped) continue;
                        my[(size_t)5 * n + g] += dalpha * r->G;
                        double dpow = dalpha * r->alpha;
                        double a = conic[g], b = conic[(size_t)n + g], c = conic[(size_t)2 * n + g];
                        my[(size_t)0 * n + g] += dpow * (a * r->dx + b * r->dy);
                        my[(size_t)1 * n + g] += dpow * (b * r->dx + c * r->dy);
                        my[(size_t)2 * n + g] += dpow * (-0.5 * r->dx * r->dx);
                        my[(size_t)3 * n + g] += dpow * (-r->dx * r->dy);
                        my[(size_t)4 * n + g] += dpow * (-0.5 * r->dy * r->dy);
                        if (mm) {
                            double pm = dalpha_m * r->alpha;
                            mm[(size_t)5 * n + g] += dalpha_m * r->G;
                            mm[(size_t)0 * n + g] += pm * (fabs(a * r->dx) + fabs(b * r->dy));
                            mm[(size_t)1 * n + g] += pm * (fabs(b * r->dx) + fabs(c * r->dy));
                            mm[(size_t)2 * n + g] += pm * (0.5 * r->dx * r->dx);
                            mm[(size_t)3 * n + g] += pm * fabs(r->dx * r->dy);
                            mm[(size_t)4 * n + g] += pm * (0.5 * r->dy * r->dy);
                        }
                    }
                }
        }
        free(buf);
        free(rec);
    }
    for (int i = 0; i < n; ++i) {
        double s[9] = {0};
        for (int th = 0; th < nthr; ++th)
            for (int k = 0; k < 9; ++k) s[k] += acc[(size_t)th * 9 * n + (size_t)k * n + i];
        d_mean2d[i] = s[0]; d_mean2d[(size_t)n + i] = s[1];
        d_conic[i] = s[2]; d_conic[(size_t)n + i] = s[3]; d_conic[(size_t)2 * n + i] = s[4];
        d_opac[i] = s[5];
        d_rgb[i] = s[6]; d_rgb[(size_t)n + i] = s[7]; d_rgb[(size_t)2 * n + i] = s[8];
        if (mag)
            for (int k = 0; k < 9; ++k) {
                double m = 0.0;
                for (int th = 0; th < nthr; ++th) m += macc[(size_t)th * 9 * n + (size_t)k * n + i];
                mag[(size_t)k * n + i] = m;
            }
    }
    free(acc);
    free(macc);
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
