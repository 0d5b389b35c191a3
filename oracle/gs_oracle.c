/*
 * gs_oracle.c -- plain FP64 CPU oracle for the differentiable tile rasterizer of
 * "3D Gaussian Splatting for Real-Time Radiance Field Rendering" (Kerbl et al. 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline leg of
 * bench.py may load this library.  It shares no code, header, table or constant
 * generator with the CUDA path under paper_2308_04079_gb300/csrc, and the product path
 * never calls it.
 *
 * What it computes (one function per step, in the paper's order):
 *   - Sec. 4: 3D Gaussian G(x) = exp(-1/2 x^T Sigma^-1 x), Sigma = R S S^T R^T with R(q)
 *     from eq. (quat) of App. A after normalising q; EWA projection
 *     Sigma' = J W Sigma W^T J^T (eq. volume-render), upper 2x2, plus a 0.3 px^2
 *     low-pass dilation on the diagonal.
 *   - Sec. 6: cull (near plane, guard band, 3-sigma screen extent), 16x16 tiles,
 *     one instance per overlapped tile, 64-bit key (tile id high, fp32 depth bits low),
 *     one stable sort, per-tile ranges (App. C, Algorithm 2).
 *   - Eq. (front-to-back): C = sum_i c_i a_i prod_{j<i}(1 - a_j) per pixel, with the
 *     App. C numerical-stability rules (skip a < 1/255, clamp a <= 0.99, stop before the
 *     accumulated opacity would exceed 0.9999).
 *   - App. A: analytic gradients through Sigma' -> Sigma -> M = RS -> (s, q) and the
 *     quaternion normalisation; the view-direction and Jacobian terms the appendix leaves
 *     out are included (they are part of the exact derivative).
 *
 * Per-pixel rendering is the plain definition: every pixel walks the Gaussians whose
 * tile rectangle covers its tile, ordered by (fp32 depth, index), in FP64.  No batching,
 * no early tile termination, no transmittance recovery by division: the backward pass
 * re-runs the pixel's forward walk and keeps every T_i.
 *
 * Decisions (cull, radius, tile rectangle, skip, clamp, stop, depth order) whose FP64 value
 * lies within the error margin of an FP32 evaluation of the same definition are reported, and
 * each one is also evaluated the other way: the forward pass returns the pixel's colour, T and
 * last Gaussian with that decision flipped, and the backward pass adds up, per Gaussian, the
 * magnitude of the change the flip makes to its gradients.  A test can then check every pixel
 * and every Gaussian: against the definition, against one of the flipped alternatives, or
 * within the definition plus the summed effect of the flips, instead of excluding them.
 *
 * Build: gcc -O2 -std=c11 -fopenmp -ffp-contract=off -fPIC -shared (see build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Camera / configuration, passed from Python as flat double arrays.          */
/* ------------------------------------------------------------------------- */
typedef struct {
    int width, height;
    double fx, fy, cx, cy;
    double W[9];   /* world -> camera rotation ("viewing transformation W", Sec. 4), row-major */
    double t[3];   /* world -> camera translation */
    double near_z;
} ocam;

typedef struct {
    int tile_w, tile_h;
    double alpha_min;   /* 1/255, App. C */
    double alpha_max;   /* 0.99, App. C */
    double T_min;       /* 1 - 0.9999, App. C */
    double dilation;    /* 0.3 px^2 low-pass filter on the diagonal of Sigma' */
    double guard;       /* guard band factor on the view-frustum tangents (Sec. 6) */
    double extent;      /* 3 (sigma multiple of the screen extent, Sec. 6) */
    int radius_max;     /* radius clamp in pixels */
    double eps_geom;    /* relative margin for geometric decisions (cull, floor, ceil) */
    double eps_alpha;   /* relative margin for the alpha skip / clamp decisions */
    double eps_T;       /* relative margin for the transmittance stop decision */
    int grad_limit;     /* > 0: only the grad_limit front-most blended Gaussians of a pixel receive
                           gradients (Limited-BW ablation, Sec. 7.3); 0: all of them */
    double eps_power;   /* margin of the splat power, relative to the magnitude sum of the terms of
                           the quadratic form: see power_margin */
} ocfg;

static void read_cam(const double* c, ocam* o) {
    o->width = (int)c[0]; o->height = (int)c[1];
    o->fx = c[2]; o->fy = c[3]; o->cx = c[4]; o->cy = c[5];
    for (int k = 0; k < 9; ++k) o->W[k] = c[6 + k];
    for (int k = 0; k < 3; ++k) o->t[k] = c[15 + k];
    o->near_z = c[18];
}

static void read_cfg(const double* c, ocfg* o) {
    o->tile_w = (int)c[0]; o->tile_h = (int)c[1];
    o->alpha_min = c[2]; o->alpha_max = c[3]; o->T_min = c[4];
    o->dilation = c[5]; o->guard = c[6]; o->extent = c[7];
    o->radius_max = (int)c[8]; o->eps_geom = c[9]; o->eps_alpha = c[10];
    o->eps_T = c[11];
    o->grad_limit = (int)c[12];
    o->eps_power = c[13];
}

/* Per-Gaussian bits: decisions of the per-Gaussian stage near their threshold. */
#define AMB_CULL   1u   /* a cull decision lies within eps_geom of its threshold                */
#define AMB_RECT   2u   /* floor(u), floor(v) or the radius ceiling may round the other way     */
#define AMB_RGB    4u   /* an SH colour channel lies within eps_geom (relative) of the 0 clamp  */

/* ------------------------------------------------------------------------- */
/* Small linear algebra.                                                       */
/* ------------------------------------------------------------------------- */
static void matmul33(const double* A, const double* B, double* C) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}

static void transpose33(const double* A, double* At) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) At[3 * j + i] = A[3 * i + j];
}

static int floor_div(int a, int b) {   /* floor(a / b) for b > 0 */
    return (a >= 0) ? a / b : -((-a + b - 1) / b);
}

static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* True when x lies within a relative margin eps of the threshold th. */
static int near_threshold(double x, double th, double eps) {
    double s = fabs(th) > fabs(x) ? fabs(th) : fabs(x);
    return fabs(x - th) <= eps * s;
}

/* ------------------------------------------------------------------------- */
/* Eq. (quat), App. A: rotation matrix of a unit quaternion q = (q_r, q_i, q_j, q_k). */
/* ------------------------------------------------------------------------- */
void orc_quat_to_rot(const double* q, double* R) {
    double r = q[0], i = q[1], j = q[2], k = q[3];
    R[0] = 2.0 * (0.5 - (j * j + k * k)); R[1] = 2.0 * (i * j - r * k);         R[2] = 2.0 * (i * k + r * j);
    R[3] = 2.0 * (i * j + r * k);         R[4] = 2.0 * (0.5 - (i * i + k * k)); R[5] = 2.0 * (j * k - r * i);
    R[6] = 2.0 * (i * k - r * j);         R[7] = 2.0 * (j * k + r * i);         R[8] = 2.0 * (0.5 - (i * i + j * j));
}

/* ------------------------------------------------------------------------- */
/* Real spherical harmonics, bands 0..3 (Sec. 4 / Sec. 7.1 use SH for colour).   */
/* Textbook definition with the Condon-Shortley phase:                           */
/*   Y_l^0  = K_l^0 P_l(z)                                                       */
/*   Y_l^m  = sqrt2 K_l^m (-1)^m (d^m P_l / dz^m)(z) Re[(x + i y)^m],  m > 0       */
/*   Y_l^-m = sqrt2 K_l^m (-1)^m (d^m P_l / dz^m)(z) Im[(x + i y)^m],  m > 0       */
/*   K_l^m  = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)                                   */
/* for a unit direction (x, y, z); (1 - z^2)^{m/2} e^{i m phi} = (x + i y)^m there. */
/* Coefficient index k = l^2 + l + m.                                             */
/* ------------------------------------------------------------------------- */
static double factorial(int n) { double f = 1.0; for (int k = 2; k <= n; ++k) f *= k; return f; }

/* Legendre polynomial coefficients, Bonnet recursion (l+1) P_{l+1} = (2l+1) z P_l - l P_{l-1}. */
static void legendre_coeffs(int lmax, double P[4][4]) {
    memset(P, 0, sizeof(double) * 16);
    P[0][0] = 1.0;
    if (lmax >= 1) P[1][1] = 1.0;
    for (int l = 1; l < 3 && l < lmax; ++l)
        for (int p = 0; p < 4; ++p) {
            double v = -l * P[l - 1][p];
            if (p > 0) v += (2 * l + 1) * P[l][p - 1];
            P[l + 1][p] = v / (l + 1);
        }
}

/* Evaluate the m-th and (m+1)-th derivative of a cubic polynomial c at z. */
static void poly_deriv_eval(const double* c, int m, double z, double* val, double* dval) {
    double d[4];
    for (int p = 0; p < 4; ++p) d[p] = c[p];
    for (int k = 0; k < m; ++k) {
        for (int p = 0; p < 3; ++p) d[p] = (p + 1) * d[p + 1];
        d[3] = 0.0;
    }
    *val = d[0] + z * (d[1] + z * (d[2] + z * d[3]));
    *dval = d[1] + z * (2.0 * d[2] + z * 3.0 * d[3]);
}

/* Y[k] and dY[k][3] = gradient w.r.t. (x, y, z) of the polynomial form above. */
static void sh_basis(int deg, const double* dir, double* Y, double* dY) {
    double P[4][4];
    legendre_coeffs(3, P);
    double x = dir[0], y = dir[1], z = dir[2];
    for (int l = 0; l <= deg; ++l) {
        for (int m = 0; m <= l; ++m) {
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - m) / factorial(l + m));
            double pl, dpl;
            poly_deriv_eval(P[l], m, z, &pl, &dpl);
            double sign = (m % 2) ? -1.0 : 1.0;
            /* (x + i y)^m and its x-derivative m (x + i y)^{m-1} (y-derivative = i times that). */
            double re = 1.0, im = 0.0, dre = 0.0, dim = 0.0;
            for (int k = 0; k < m; ++k) {
                double nre = re * x - im * y, nim = re * y + im * x;
                if (k == m - 1) { dre = m * re; dim = m * im; }
                re = nre; im = nim;
            }
            if (m == 0) {
                int k = l * l + l;
                Y[k] = K * pl;
                if (dY) { dY[3 * k + 0] = 0.0; dY[3 * k + 1] = 0.0; dY[3 * k + 2] = K * dpl; }
            } else {
                double c = M_SQRT2 * K * sign;
                int kp = l * l + l + m, km = l * l + l - m;
                Y[kp] = c * pl * re;
                Y[km] = c * pl * im;
                if (dY) {
                    /* d/dx (x+iy)^m = m (x+iy)^{m-1};  d/dy (x+iy)^m = i m (x+iy)^{m-1} */
                    dY[3 * kp + 0] = c * pl * dre;
                    dY[3 * kp + 1] = c * pl * (-dim);
                    dY[3 * kp + 2] = c * dpl * re;
                    dY[3 * km + 0] = c * pl * dim;
                    dY[3 * km + 1] = c * pl * dre;
                    dY[3 * km + 2] = c * dpl * im;
                }
            }
        }
    }
}

void orc_sh_eval(int deg, int n, const double* dirs, double* Y, double* dY) {
    int D = (deg + 1) * (deg + 1);
    for (int i = 0; i < n; ++i) sh_basis(deg, dirs + 3 * i, Y + (size_t)D * i, dY ? dY + (size_t)3 * D * i : NULL);
}

/* ------------------------------------------------------------------------- */
/* Per-Gaussian forward state (Algorithm 2: CullGaussian, ScreenspaceGaussians). */
/* ------------------------------------------------------------------------- */
typedef struct {
    int valid;          /* all inputs finite, z > 0: the quantities below are defined */
    int visible;        /* survives every cull */
    double tcam[3];     /* camera-space mean t = W mu + t_w */
    double qn[4];       /* normalised quaternion */
    double qnorm;
    double R[9];        /* R(q) */
    double M[9];        /* M = R S */
    double Sigma[9];    /* Sigma = M M^T */
    double J[6];        /* 2x3 Jacobian of the perspective projection at t */
    double U[6];        /* U = J W (first two rows) */
    double cov2[3];     /* Sigma' = upper 2x2 of U Sigma U^T + dilation I: (A, B, C) */
    double det;
    double conic[3];    /* Sigma'^{-1}: (a, b, c) = (C, -B, A) / det */
    double lambda_max;
    int radius;
    double uv[2];       /* screen-space mean (pixels) */
    int rect[4];        /* tile rectangle [x0, x1) x [y0, y1) */
    int rect_in[4];     /* intersection of the rectangles reachable under ambiguous rounding */
    int rect_out[4];    /* union (bounding box) of those rectangles */
    double dirv[3];     /* mu - camera centre */
    double dnorm;
    double dhat[3];
    double Y[16];
    double dY[48];
    double rgb_raw[3];
    double rgb[3];
    unsigned amb;
    unsigned rgb_amb;   /* bit ch: channel ch near the 0 clamp */
} ogauss;

static int rect_of(double u, double v, int r, const ocam* cam, const ocfg* cfg, int fu_off, int fv_off, int out[4]) {
    int TX = (cam->width + cfg->tile_w - 1) / cfg->tile_w;
    int TY = (cam->height + cfg->tile_h - 1) / cfg->tile_h;
    /* floor((u -/+ r) / tile) computed exactly: r is an integer, so it equals
       floor_div(floor(u) -/+ r, tile). */
    int fu = (int)floor(u) + fu_off, fv = (int)floor(v) + fv_off;
    out[0] = clampi(floor_div(fu - r, cfg->tile_w), 0, TX);
    out[1] = clampi(floor_div(fu + r, cfg->tile_w) + 1, 0, TX);
    out[2] = clampi(floor_div(fv - r, cfg->tile_h), 0, TY);
    out[3] = clampi(floor_div(fv + r, cfg->tile_h) + 1, 0, TY);
    return out[0] < out[1] && out[2] < out[3];
}

static void gauss_forward(size_t i, const double* means, const double* scales, const double* quats,
                          const double* opac, const double* sh, int deg, int sh_stride,
                          const ocam* cam, const ocfg* cfg, ogauss* g) {
    memset(g, 0, sizeof(*g));
    const double* mu = means + 3 * i;
    const double* s = scales + 3 * i;
    const double* q = quats + 4 * i;
    int D = (deg + 1) * (deg + 1);
    int finite = isfinite(opac[i]);
    for (int k = 0; k < 3; ++k) finite &= isfinite(mu[k]) && isfinite(s[k]);
    for (int k = 0; k < 4; ++k) finite &= isfinite(q[k]);
    for (int k = 0; k < D * 3; ++k) finite &= isfinite(sh[(size_t)i * sh_stride * 3 + k]);
    if (!finite) return;

    /* Camera-space mean: t = W mu + t_w. */
    for (int r = 0; r < 3; ++r)
        g->tcam[r] = cam->W[3 * r] * mu[0] + cam->W[3 * r + 1] * mu[1] + cam->W[3 * r + 2] * mu[2] + cam->t[r];
    double tx = g->tcam[0], ty = g->tcam[1], tz = g->tcam[2];
    double qn2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    if (!(tz > 0.0) || !(qn2 > 0.0)) return;   /* nothing can be projected */
    g->valid = 1;

    /* Guard band and near plane (Sec. 6): reject, do not clamp. */
    double tanx = 0.5 * cam->width / cam->fx, tany = 0.5 * cam->height / cam->fy;
    int keep = 1;
    if (tz <= cam->near_z) keep = 0;
    if (near_threshold(tz, cam->near_z, cfg->eps_geom)) g->amb |= AMB_CULL;
    double rx = fabs(tx / tz), ry = fabs(ty / tz);
    if (rx > cfg->guard * tanx) keep = 0;
    if (ry > cfg->guard * tany) keep = 0;
    if (near_threshold(rx, cfg->guard * tanx, cfg->eps_geom)) g->amb |= AMB_CULL;
    if (near_threshold(ry, cfg->guard * tany, cfg->eps_geom)) g->amb |= AMB_CULL;

    /* Sigma = R S S^T R^T with q normalised (Sec. 4). */
    g->qnorm = sqrt(qn2);
    for (int k = 0; k < 4; ++k) g->qn[k] = q[k] / g->qnorm;
    orc_quat_to_rot(g->qn, g->R);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) g->M[3 * r + c] = g->R[3 * r + c] * s[c];
    double Mt[9];
    transpose33(g->M, Mt);
    matmul33(g->M, Mt, g->Sigma);

    /* EWA: Sigma' = J W Sigma W^T J^T (eq. volume-render), upper 2x2, + dilation. */
    g->J[0] = cam->fx / tz; g->J[1] = 0.0;            g->J[2] = -cam->fx * tx / (tz * tz);
    g->J[3] = 0.0;          g->J[4] = cam->fy / tz;   g->J[5] = -cam->fy * ty / (tz * tz);
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            g->U[3 * r + c] = g->J[3 * r] * cam->W[c] + g->J[3 * r + 1] * cam->W[3 + c] + g->J[3 * r + 2] * cam->W[6 + c];
    double US[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            US[3 * r + c] = g->U[3 * r] * g->Sigma[c] + g->U[3 * r + 1] * g->Sigma[3 + c] + g->U[3 * r + 2] * g->Sigma[6 + c];
    double S00 = US[0] * g->U[0] + US[1] * g->U[1] + US[2] * g->U[2];
    double S01 = US[0] * g->U[3] + US[1] * g->U[4] + US[2] * g->U[5];
    double S11 = US[3] * g->U[3] + US[4] * g->U[4] + US[5] * g->U[5];
    g->cov2[0] = S00 + cfg->dilation;
    g->cov2[1] = S01;
    g->cov2[2] = S11 + cfg->dilation;
    g->det = g->cov2[0] * g->cov2[2] - g->cov2[1] * g->cov2[1];
    if (!(g->det > 0.0)) { g->valid = 0; return; }
    g->conic[0] = g->cov2[2] / g->det;
    g->conic[1] = -g->cov2[1] / g->det;
    g->conic[2] = g->cov2[0] / g->det;

    /* 3-sigma extent of the largest eigenvalue, integer pixels. */
    double m = 0.5 * (g->cov2[0] + g->cov2[2]);
    double disc = m * m - g->det;
    g->lambda_max = m + sqrt(disc > 0.0 ? disc : 0.0);
    double rr = cfg->extent * sqrt(g->lambda_max);
    int rclamped = rr >= (double)cfg->radius_max;
    g->radius = rclamped ? cfg->radius_max : (int)ceil(rr);
    g->uv[0] = cam->fx * tx / tz + cam->cx;
    g->uv[1] = cam->fy * ty / tz + cam->cy;

    /* Tile rectangle and its sensitivity to rounding of floor(u), floor(v), ceil(3 sqrt(lambda)).
       Only meaningful inside the guard band, which also bounds |u| and |v|. */
    if (!keep && !(g->amb & AMB_CULL)) return;
    int nonempty = rect_of(g->uv[0], g->uv[1], g->radius, cam, cfg, 0, 0, g->rect);
    if (!nonempty) keep = 0;
    int du_alt[2] = {0, 0}, dv_alt[2] = {0, 0}, r_alt[2] = {g->radius, g->radius};
    double fu_frac = g->uv[0] - floor(g->uv[0]), fv_frac = g->uv[1] - floor(g->uv[1]);
    double su = fabs(g->uv[0]) > 1.0 ? fabs(g->uv[0]) : 1.0, sv = fabs(g->uv[1]) > 1.0 ? fabs(g->uv[1]) : 1.0;
    if (fu_frac <= cfg->eps_geom * su) du_alt[0] = -1;
    if (1.0 - fu_frac <= cfg->eps_geom * su) du_alt[1] = 1;
    if (fv_frac <= cfg->eps_geom * sv) dv_alt[0] = -1;
    if (1.0 - fv_frac <= cfg->eps_geom * sv) dv_alt[1] = 1;
    if (!rclamped) {
        double rfrac = rr - floor(rr);
        double sr = rr > 1.0 ? rr : 1.0;
        /* an fp32 value of rr on the other side of the integer below (above) changes ceil by one */
        if (rfrac <= cfg->eps_geom * sr && rfrac > 0.0 && rr >= 1.0) r_alt[0] = g->radius - 1;
        if (1.0 - rfrac <= cfg->eps_geom * sr || rfrac == 0.0) r_alt[1] = g->radius + 1;
    } else if (near_threshold(rr, cfg->radius_max, cfg->eps_geom)) {
        r_alt[0] = cfg->radius_max - 1;
    }
    for (int k = 0; k < 4; ++k) { g->rect_in[k] = g->rect[k]; g->rect_out[k] = g->rect[k]; }
    int any_empty = !nonempty, any_full = nonempty;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                int alt[4];
                int ne = rect_of(g->uv[0], g->uv[1], r_alt[c], cam, cfg, du_alt[a], dv_alt[b], alt);
                if (!ne) { any_empty = 1; continue; }
                if (alt[0] != g->rect[0] || alt[1] != g->rect[1] || alt[2] != g->rect[2] || alt[3] != g->rect[3])
                    g->amb |= AMB_RECT;
                if (!any_full) { for (int k = 0; k < 4; ++k) g->rect_out[k] = alt[k]; any_full = 1; }
                if (alt[0] < g->rect_out[0]) g->rect_out[0] = alt[0];
                if (alt[1] > g->rect_out[1]) g->rect_out[1] = alt[1];
                if (alt[2] < g->rect_out[2]) g->rect_out[2] = alt[2];
                if (alt[3] > g->rect_out[3]) g->rect_out[3] = alt[3];
                if (alt[0] > g->rect_in[0]) g->rect_in[0] = alt[0];
                if (alt[1] < g->rect_in[1]) g->rect_in[1] = alt[1];
                if (alt[2] > g->rect_in[2]) g->rect_in[2] = alt[2];
                if (alt[3] < g->rect_in[3]) g->rect_in[3] = alt[3];
            }
    if (any_empty && any_full && nonempty) g->amb |= AMB_RECT;
    if (any_empty) { g->rect_in[0] = g->rect_in[1] = 0; }   /* nothing is certain */
    if (g->amb & AMB_CULL) { g->rect_in[0] = g->rect_in[1] = 0; }
    if (!any_full) { g->rect_out[0] = g->rect_out[1] = 0; }

    /* View-dependent colour: rgb = max(0, sum_k sh_k Y_k(d)), d = (mu - C)/|mu - C|,
       C = -W^T t the camera centre. */
    double C[3];
    for (int r = 0; r < 3; ++r) C[r] = -(cam->W[r] * cam->t[0] + cam->W[3 + r] * cam->t[1] + cam->W[6 + r] * cam->t[2]);
    for (int r = 0; r < 3; ++r) g->dirv[r] = mu[r] - C[r];
    g->dnorm = sqrt(g->dirv[0] * g->dirv[0] + g->dirv[1] * g->dirv[1] + g->dirv[2] * g->dirv[2]);
    for (int r = 0; r < 3; ++r) g->dhat[r] = g->dirv[r] / g->dnorm;
    sh_basis(deg, g->dhat, g->Y, g->dY);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0, mag = 0.0;
        for (int k = 0; k < D; ++k) {
            double term = sh[((size_t)i * sh_stride + k) * 3 + ch] * g->Y[k];
            acc += term;
            mag += fabs(term);
        }
        g->rgb_raw[ch] = acc;
        g->rgb[ch] = acc > 0.0 ? acc : 0.0;
        if (fabs(acc) <= cfg->eps_geom * mag) { g->amb |= AMB_RGB; g->rgb_amb |= 1u << ch; }   /* clamp at 0 may flip */
    }
    g->visible = keep;
    (void)opac;
}

/* ------------------------------------------------------------------------- */
/* Scene-level state shared by forward and backward.                           */
/* ------------------------------------------------------------------------- */
typedef struct {
    size_t n;
    int deg, sh_stride;
    const double *means, *scales, *quats, *opac, *sh;
    ocam cam;
    ocfg cfg;
    ogauss* g;
    int TX, TY;
    /* per-tile candidate lists (only tiles in the mask) */
    int64_t* tile_start;   /* [T+1] */
    int32_t* tile_list;    /* certain-or-main candidates, sorted by (fp32 depth, index) */
    int64_t* shadow_start; /* [T+1] */
    int32_t* shadow_list;  /* uncertain candidates not in the main list */
} oscene;

typedef struct { uint32_t dkey; int32_t idx; } dkey_t;

static int cmp_dkey(const void* a, const void* b) {
    const dkey_t* x = (const dkey_t*)a;
    const dkey_t* y = (const dkey_t*)b;
    if (x->dkey != y->dkey) return x->dkey < y->dkey ? -1 : 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Depth key: IEEE-754 fp32 bits of the camera-space depth (App. C: "the lower 32 bits
   encode its projected depth"); positive floats order like their bit patterns. */
static uint32_t depth_key(double z) {
    float f = (float)z;
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

static int in_rect(const int* rc, int tx, int ty) { return tx >= rc[0] && tx < rc[1] && ty >= rc[2] && ty < rc[3]; }

static void scene_build(oscene* S, const uint8_t* tile_mask) {
    S->TX = (S->cam.width + S->cfg.tile_w - 1) / S->cfg.tile_w;
    S->TY = (S->cam.height + S->cfg.tile_h - 1) / S->cfg.tile_h;
    S->g = (ogauss*)malloc(sizeof(ogauss) * (S->n ? S->n : 1));
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)S->n; ++i)
        gauss_forward((size_t)i, S->means, S->scales, S->quats, S->opac, S->sh, S->deg, S->sh_stride, &S->cam, &S->cfg, &S->g[i]);

    /* One instance per (Gaussian, overlapped tile), in Gaussian order then row-major tile order. */
    int T = S->TX * S->TY;
    S->tile_start = (int64_t*)calloc((size_t)T + 1, sizeof(int64_t));
    S->shadow_start = (int64_t*)calloc((size_t)T + 1, sizeof(int64_t));
    for (size_t i = 0; i < S->n; ++i) {
        const ogauss* g = &S->g[i];
        if (!g->valid) continue;
        int lo_x = g->rect_out[0], hi_x = g->rect_out[1], lo_y = g->rect_out[2], hi_y = g->rect_out[3];
        if (g->visible) {
            if (g->rect[0] < lo_x) lo_x = g->rect[0];
            if (g->rect[1] > hi_x) hi_x = g->rect[1];
            if (g->rect[2] < lo_y) lo_y = g->rect[2];
            if (g->rect[3] > hi_y) hi_y = g->rect[3];
        }
        for (int ty = lo_y; ty < hi_y; ++ty)
            for (int tx = lo_x; tx < hi_x; ++tx) {
                int t = ty * S->TX + tx;
                if (tile_mask && !tile_mask[t]) continue;
                int main_c = g->visible && in_rect(g->rect, tx, ty);
                int uncertain = ((g->amb & (AMB_CULL | AMB_RECT)) != 0) && in_rect(g->rect_out, tx, ty) && !in_rect(g->rect_in, tx, ty);
                if (main_c) S->tile_start[t + 1]++;
                else if (uncertain) S->shadow_start[t + 1]++;
            }
    }
    for (int t = 0; t < T; ++t) { S->tile_start[t + 1] += S->tile_start[t]; S->shadow_start[t + 1] += S->shadow_start[t]; }
    S->tile_list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(S->tile_start[T] + 1));
    S->shadow_list = (int32_t*)malloc(sizeof(int32_t) * (size_t)(S->shadow_start[T] + 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
    int64_t* sfill = (int64_t*)malloc(sizeof(int64_t) * (size_t)T);
    for (int t = 0; t < T; ++t) { fill[t] = S->tile_start[t]; sfill[t] = S->shadow_start[t]; }
    for (size_t i = 0; i < S->n; ++i) {
        const ogauss* g = &S->g[i];
        if (!g->valid) continue;
        int lo_x = g->rect_out[0], hi_x = g->rect_out[1], lo_y = g->rect_out[2], hi_y = g->rect_out[3];
        if (g->visible) {
            if (g->rect[0] < lo_x) lo_x = g->rect[0];
            if (g->rect[1] > hi_x) hi_x = g->rect[1];
            if (g->rect[2] < lo_y) lo_y = g->rect[2];
            if (g->rect[3] > hi_y) hi_y = g->rect[3];
        }
        for (int ty = lo_y; ty < hi_y; ++ty)
            for (int tx = lo_x; tx < hi_x; ++tx) {
                int t = ty * S->TX + tx;
                if (tile_mask && !tile_mask[t]) continue;
                int main_c = g->visible && in_rect(g->rect, tx, ty);
                int uncertain = ((g->amb & (AMB_CULL | AMB_RECT)) != 0) && in_rect(g->rect_out, tx, ty) && !in_rect(g->rect_in, tx, ty);
                if (main_c) S->tile_list[fill[t]++] = (int32_t)i;
                else if (uncertain) S->shadow_list[sfill[t]++] = (int32_t)i;
            }
    }
    free(fill); free(sfill);
    /* Per-tile order by (fp32 depth bits, Gaussian index): the result of one stable sort
       of the (tile | depth) keys emitted in Gaussian order (App. C). */
#pragma omp parallel for schedule(dynamic, 4)
    for (int t = 0; t < T; ++t) {
        int64_t a = S->tile_start[t], b = S->tile_start[t + 1];
        if (b - a < 2) continue;
        dkey_t* tmp = (dkey_t*)malloc(sizeof(dkey_t) * (size_t)(b - a));
        for (int64_t k = a; k < b; ++k) { tmp[k - a].idx = S->tile_list[k]; tmp[k - a].dkey = depth_key(S->g[S->tile_list[k]].tcam[2]); }
        qsort(tmp, (size_t)(b - a), sizeof(dkey_t), cmp_dkey);
        for (int64_t k = a; k < b; ++k) S->tile_list[k] = tmp[k - a].idx;
        free(tmp);
    }
}

static void scene_free(oscene* S) {
    free(S->g); free(S->tile_start); free(S->tile_list); free(S->shadow_start); free(S->shadow_list);
}

/* Record of one blended Gaussian at one pixel (kept for the backward walk). */
typedef struct {
    int32_t idx;
    double alpha, G, T;   /* T = transmittance before this Gaussian */
    double dx, dy;
    int clamped;
} contrib_t;

/* Screen-space gradient terms that one pixel gives one Gaussian: dL/d(u, v), dL/d(conic a, b,
   c) with b the off-diagonal entry as it enters the power once, dL/do, dL/d(r, g, b). */
typedef struct {
    int32_t idx;
    double uv[2], conic[3], op, rgb[3];
} pgrad_t;

/* Evaluate the 2D Gaussian of g at pixel centre (px + 0.5, py + 0.5). */
static double eval_power(const ogauss* g, double pxc, double pyc, double* dx, double* dy) {
    *dx = pxc - g->uv[0];
    *dy = pyc - g->uv[1];
    return -0.5 * (g->conic[0] * (*dx) * (*dx) + g->conic[2] * (*dy) * (*dy)) - g->conic[1] * (*dx) * (*dy);
}

/* Margin of the power for an fp32 evaluation (ocfg.eps_power).  The plain definition's form
   P = (a dx^2 + c dy^2)/2 + b dx dy (power = -P) is evaluated from fp32 values; with unit
   roundoff u = 2^-24 and Q = (|a| dx^2 + |c| dy^2)/2 + |b dx dy| (the magnitude sum of its
   terms), first-order error analysis gives |P_fp32 - P| <= eps Q with
     conic entries a, c within 6u relative and b within 6u sqrt(a c)        12u Q
       (|db dx dy| <= 6u sqrt(a) |dx| sqrt(c) |dy| <= 6u (a dx^2 + c dy^2)/2)
     pixel offsets dx, dy within 2u relative, entering squared               4u Q
     the evaluation: at most two products and two sums on any term's path   4u Q
   eps = 20u = 1.19e-6.  Q equals |P| when the terms share a sign and exceeds it by the
   conditioning of the form when they cancel (an elongated splat, far along its major axis),
   which is where an fp32 evaluation may decide a threshold differently. */
static double power_margin(const ogauss* g, double dx, double dy, const ocfg* cfg) {
    double Q = 0.5 * (fabs(g->conic[0]) * dx * dx + fabs(g->conic[2]) * dy * dy) + fabs(g->conic[1] * dx * dy);
    return cfg->eps_power * Q;
}

/* ------------------------------------------------------------------------- */
/* Discrete decisions of a pixel's walk, and the walk with one of them taken   */
/* the other way.  A decision is "near its threshold" when the FP64 quantity   */
/* lies within the margin that an FP32 evaluation of the same definition may   */
/* err by (ocfg eps_*); for each such decision the walk is also run with the   */
/* decision flipped, so that a test can accept either outcome (and bound the   */
/* effect of several flips by the sum of their effects) instead of skipping    */
/* the pixel or the Gaussians it touches.                                      */
/* ------------------------------------------------------------------------- */
#define DEC_SKIP  1   /* alpha < 1/255 (App. C)                                                */
#define DEC_CLAMP 2   /* alpha clamped at 0.99 (App. C): continuous value, not its derivative  */
#define DEC_STOP  3   /* T (1 - alpha) < 1e-4: stop before this Gaussian (App. C)              */
#define DEC_SWAP  4   /* equal or adjacent fp32 depth keys: the two Gaussians may swap places  */
#define DEC_DROP  5   /* tile membership near its threshold (cull, rectangle): may be absent   */
#define DEC_ADD   6   /* a Gaussian outside the tile's list whose membership is near threshold */

typedef struct { int kind; int32_t g0, g1; } odec_t;

/* Per-thread scratch of the pixel walks. */
typedef struct {
    int32_t* cand;   /* walk order */
    contrib_t* rec;  /* blended Gaussians, main walk */
    contrib_t* rec2; /* blended Gaussians, alternative walk */
    pgrad_t* pg;     /* gradient terms, main walk */
    pgrad_t* pg2;    /* gradient terms, alternative walk */
    odec_t* dec;     /* decisions near their threshold */
    int dec_cap;
} oscratch;

#define DEC_CAP 512

static void scratch_alloc(oscratch* W, int64_t maxlen) {
    size_t m = (size_t)maxlen + 2;
    W->cand = (int32_t*)malloc(sizeof(int32_t) * m);
    W->rec = (contrib_t*)malloc(sizeof(contrib_t) * m);
    W->rec2 = (contrib_t*)malloc(sizeof(contrib_t) * m);
    W->pg = (pgrad_t*)malloc(sizeof(pgrad_t) * m);
    W->pg2 = (pgrad_t*)malloc(sizeof(pgrad_t) * m);
    W->dec = (odec_t*)malloc(sizeof(odec_t) * DEC_CAP);
    W->dec_cap = DEC_CAP;
}

static void scratch_free(oscratch* W) {
    free(W->cand); free(W->rec); free(W->rec2); free(W->pg); free(W->pg2); free(W->dec);
}

/* Walk order of the definition: (fp32 depth bits, index) ascending. */
static int walk_before(const oscene* S, int32_t x, int32_t y) {
    uint32_t kx = depth_key(S->g[x].tcam[2]), ky = depth_key(S->g[y].tcam[2]);
    return kx != ky ? kx < ky : x < y;
}

static int flips(const odec_t* f, int kind, int32_t gi) { return f && f->kind == kind && f->g0 == gi; }

/*
 * One pixel's walk over its tile's list: eq. front-to-back with the App. C rules (skip
 * alpha < 1/255 after the 0.99 clamp, stop before T (1 - alpha) < 1e-4), in (fp32 depth,
 * index) order.  flip == NULL: the definition, and (if ndec is given) the decisions that lie
 * near their threshold are listed in W->dec.  flip != NULL: the same walk with that one decision
 * taken the other way.  Writes C (before the background), T, the 1-based list position and the
 * index of the last blended Gaussian; returns the number of blended Gaussians (recorded in rec
 * when given).
 */
static int pixel_walk(const oscene* S, int t, int px, int py, const odec_t* flip, oscratch* W, contrib_t* rec,
                      double* C_out, double* T_out, int* last_pos, int32_t* last_id, int* ndec) {
    const ocfg* cfg = &S->cfg;
    const double pxc = px + 0.5, pyc = py + 0.5;
    const int tx = t % S->TX, ty = t / S->TX;
    const int main_walk = flip == NULL;
    const int want_dec = main_walk && ndec != NULL;
    int nd = 0;
#define ADD_DEC(k, a, b)                                                                           \
    do {                                                                                           \
        if (nd < W->dec_cap) { W->dec[nd].kind = (k); W->dec[nd].g0 = (a); W->dec[nd].g1 = (b); } \
        ++nd;                                                                                      \
    } while (0)

    /* walk order: the tile's list, with the flipped membership or order applied */
    int64_t a = S->tile_start[t], b = S->tile_start[t + 1];
    int m = 0, added = 0;
    for (int64_t k = a; k < b; ++k) {
        int32_t gi = S->tile_list[k];
        if (flips(flip, DEC_DROP, gi)) continue;
        if (flip && flip->kind == DEC_ADD && !added && walk_before(S, flip->g0, gi)) { W->cand[m++] = flip->g0; added = 1; }
        W->cand[m++] = gi;
    }
    if (flip && flip->kind == DEC_ADD && !added) W->cand[m++] = flip->g0;
    if (flip && flip->kind == DEC_SWAP) {
        int p0 = -1, p1 = -1;
        for (int w = 0; w < m; ++w) {
            if (W->cand[w] == flip->g0) p0 = w;
            if (W->cand[w] == flip->g1) p1 = w;
        }
        if (p0 >= 0 && p1 >= 0) { W->cand[p0] = flip->g1; W->cand[p1] = flip->g0; }
    }

    double T = 1.0, C[3] = {0.0, 0.0, 0.0};
    int nrec = 0, lp = 0;
    int32_t lid = -1;
    uint32_t prev_key = 0;
    int32_t prev = -1;
    for (int w = 0; w < m; ++w) {
        const int32_t gi = W->cand[w];
        const ogauss* g = &S->g[gi];
        double dx, dy;
        const double power = eval_power(g, pxc, pyc, &dx, &dy);
        const double G = exp(power);
        const double oG = S->opac[gi] * G;
        const double eps_a = cfg->eps_alpha + power_margin(g, dx, dy, cfg);   /* relative, on o G */
        if (want_dec) {
            if (oG >= cfg->alpha_min * (1.0 - eps_a)) {
                if ((g->amb & (AMB_CULL | AMB_RECT)) && !in_rect(g->rect_in, tx, ty)) ADD_DEC(DEC_DROP, gi, -1);
                const uint32_t key = depth_key(g->tcam[2]);
                if (prev >= 0 && key - prev_key <= 1u) ADD_DEC(DEC_SWAP, prev, gi);
                prev_key = key;
                prev = gi;
            }
            if (near_threshold(oG, cfg->alpha_min, eps_a)) ADD_DEC(DEC_SKIP, gi, -1);
            if (near_threshold(oG, cfg->alpha_max, eps_a)) ADD_DEC(DEC_CLAMP, gi, -1);
        }
        int clamped = oG > cfg->alpha_max;
        if (flips(flip, DEC_CLAMP, gi)) clamped = !clamped;
        const double alpha = clamped ? cfg->alpha_max : oG;
        int skip = alpha < cfg->alpha_min;                      /* skip (App. C) */
        if (flips(flip, DEC_SKIP, gi)) skip = !skip;
        if (skip) continue;
        const double test_T = T * (1.0 - alpha);
        /* (1 - alpha) is uncertain by alpha (eps_a - eps_alpha) relative to alpha */
        if (want_dec && near_threshold(test_T, cfg->T_min, cfg->eps_T + alpha / (1.0 - alpha) * (eps_a - cfg->eps_alpha)))
            ADD_DEC(DEC_STOP, gi, -1);
        int stop = test_T < cfg->T_min;                         /* stop before exceeding 0.9999 */
        if (flips(flip, DEC_STOP, gi)) stop = !stop;
        if (stop) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += g->rgb[ch] * alpha * T;
        if (rec) {
            rec[nrec].idx = gi; rec[nrec].alpha = alpha; rec[nrec].G = G; rec[nrec].T = T;
            rec[nrec].dx = dx; rec[nrec].dy = dy; rec[nrec].clamped = clamped;
        }
        nrec++;
        T = test_T;
        lp = w + 1;
        lid = gi;
    }
    if (want_dec) {
        /* Gaussians outside this tile's list whose membership is near its threshold */
        for (int64_t k = S->shadow_start[t]; k < S->shadow_start[t + 1]; ++k) {
            const int32_t gi = S->shadow_list[k];
            const ogauss* g = &S->g[gi];
            double dx, dy;
            const double oG = S->opac[gi] * exp(eval_power(g, pxc, pyc, &dx, &dy));
            if (oG >= cfg->alpha_min * (1.0 - cfg->eps_alpha - power_margin(g, dx, dy, cfg))) ADD_DEC(DEC_ADD, gi, -1);
        }
        *ndec = nd;
    }
#undef ADD_DEC
    for (int ch = 0; ch < 3; ++ch) C_out[ch] = C[ch];
    *T_out = T;
    if (last_pos) *last_pos = main_walk ? lp : 0;
    if (last_id) *last_id = lid;
    return nrec;
}

/*
 * Backward walk of one pixel (Sec. 6): back to front over the blended Gaussians, with the
 * colour behind each one (normalised by the transmittance in front of it) carried from the
 * background.  pg[k] receives the screen-space gradient terms of rec[k].  With a gradient limit
 * N (Limited-BW, Sec. 7.3) only the N front-most blended Gaussians get terms; the colour behind
 * still takes in every one.
 */
static void pixel_backward(const oscene* S, const contrib_t* rec, int nrec, const double* dC, const double* bg,
                           pgrad_t* pg) {
    double Rb[3] = {bg[0], bg[1], bg[2]};
    for (int k = nrec - 1; k >= 0; --k) {
        const contrib_t* c = &rec[k];
        const ogauss* g = &S->g[c->idx];
        pgrad_t* p = &pg[k];
        memset(p, 0, sizeof(*p));
        p->idx = c->idx;
        const int grad = S->cfg.grad_limit <= 0 || k < S->cfg.grad_limit;
        double dL_dalpha = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            if (grad) p->rgb[ch] = c->T * c->alpha * dC[ch];
            dL_dalpha += c->T * (g->rgb[ch] - Rb[ch]) * dC[ch];
            Rb[ch] = c->alpha * g->rgb[ch] + (1.0 - c->alpha) * Rb[ch];
        }
        if (!grad || c->clamped) continue;   /* derivative of min(o G, 0.99) is 0 when clamped */
        const double o = S->opac[c->idx];
        p->op = c->G * dL_dalpha;
        const double dL_dpower = o * c->G * dL_dalpha;
        p->conic[0] = -0.5 * c->dx * c->dx * dL_dpower;
        p->conic[1] = -c->dx * c->dy * dL_dpower;
        p->conic[2] = -0.5 * c->dy * c->dy * dL_dpower;
        /* d = p - mean: d(power)/du = a dx + b dy, d(power)/dv = b dx + c dy */
        p->uv[0] = (g->conic[0] * c->dx + g->conic[1] * c->dy) * dL_dpower;
        p->uv[1] = (g->conic[1] * c->dx + g->conic[2] * c->dy) * dL_dpower;
    }
}

/* dL/dSigma' from dL/dconic, conic = Sigma'^-1: dL/dSigma' = -Q G_Q Q with G_Q the symmetric
   gradient of Q (the off-diagonal b enters the power once, as the symmetric entry); returns the
   full-matrix entries (00, 01, 11). */
static void conic_to_cov_grad(const ogauss* g, const double* dconic, double* H4) {
    double Q[4] = {g->conic[0], g->conic[1], g->conic[1], g->conic[2]};
    double GQ[4] = {dconic[0], 0.5 * dconic[1], 0.5 * dconic[1], dconic[2]};
    double QG[4];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) QG[2 * r + c] = Q[2 * r] * GQ[c] + Q[2 * r + 1] * GQ[2 + c];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) H4[2 * r + c] = -(QG[2 * r] * Q[c] + QG[2 * r + 1] * Q[2 + c]);
}

/*
 * Chain rule of App. A for Gaussian i, linear in the screen-space gradients: dL/d(u, v),
 * dL/dconic and dL/drgb (the latter already masked by the colour clamp) to dL/d(mu, s, q, SH).
 * dsh receives the first D x 3 coefficients.
 */
static void gauss_chain_g(const oscene* S, size_t i, const ogauss* g, const double* d_uv, const double* d_conic,
                          const double* drgb, double* dmu, double* ds, double* dq, double* dsh) {
    const double* s = S->scales + 3 * i;
    const int D = (S->deg + 1) * (S->deg + 1);
    double H[4];
    conic_to_cov_grad(g, d_conic, H);

    /* App. A: dSigma'/dSigma_ij = [[U1i U1j, U1i U2j], [U1j U2i, U2i U2j]] with U = J W. */
    double GS[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double* U = g->U;
            GS[3 * a + b] = H[0] * U[a] * U[b] + H[1] * U[a] * U[3 + b] + H[2] * U[b] * U[3 + a] + H[3] * U[3 + a] * U[3 + b];
        }
    /* Sigma = M M^T: dL/dM = (G + G^T) M. */
    double GSs[9], dM[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) GSs[3 * a + b] = GS[3 * a + b] + GS[3 * b + a];
    matmul33(GSs, g->M, dM);
    /* dM_ij/ds_k = R_ik if j == k. */
    for (int k = 0; k < 3; ++k) ds[k] = dM[k] * g->R[k] + dM[3 + k] * g->R[3 + k] + dM[6 + k] * g->R[6 + k];
    /* dM/dq from App. A (q normalised). */
    double qr = g->qn[0], qi = g->qn[1], qj = g->qn[2], qk = g->qn[3];
    double sx = s[0], sy = s[1], sz = s[2];
    double dMr[9] = {0, -sy * qk, sz * qj, sx * qk, 0, -sz * qi, -sx * qj, sy * qi, 0};
    double dMi[9] = {0, sy * qj, sz * qk, sx * qj, -2 * sy * qi, -sz * qr, sx * qk, sy * qr, -2 * sz * qi};
    double dMj[9] = {-2 * sx * qj, sy * qi, sz * qr, sx * qi, 0, sz * qk, -sx * qr, sy * qk, -2 * sz * qj};
    double dMk[9] = {-2 * sx * qk, -sy * qr, sz * qi, sx * qr, -2 * sy * qk, sz * qj, sx * qi, sy * qj, 0};
    double dqn[4] = {0, 0, 0, 0};
    for (int e = 0; e < 9; ++e) {
        dqn[0] += 2.0 * dMr[e] * dM[e];
        dqn[1] += 2.0 * dMi[e] * dM[e];
        dqn[2] += 2.0 * dMj[e] * dM[e];
        dqn[3] += 2.0 * dMk[e] * dM[e];
    }
    /* q_hat = q / |q|: dL/dq = (dL/dq_hat - q_hat (q_hat . dL/dq_hat)) / |q|. */
    double proj = dqn[0] * qr + dqn[1] * qi + dqn[2] * qj + dqn[3] * qk;
    for (int k = 0; k < 4; ++k) dq[k] = (dqn[k] - g->qn[k] * proj) / g->qnorm;

    /* Jacobian and screen position depend on the camera-space mean t. */
    /* Sigma'_raw = U Sigma U^T: dL/dU = (H + H^T) U Sigma; U = J W: dL/dJ = dL/dU W^T. */
    double Hs[4] = {2 * H[0], H[1] + H[2], H[1] + H[2], 2 * H[3]};
    double USg[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            USg[3 * r + c] = g->U[3 * r] * g->Sigma[c] + g->U[3 * r + 1] * g->Sigma[3 + c] + g->U[3 * r + 2] * g->Sigma[6 + c];
    double dU[6], dJ[6];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c) dU[3 * r + c] = Hs[2 * r] * USg[c] + Hs[2 * r + 1] * USg[3 + c];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            dJ[3 * r + c] = dU[3 * r] * S->cam.W[3 * c] + dU[3 * r + 1] * S->cam.W[3 * c + 1] + dU[3 * r + 2] * S->cam.W[3 * c + 2];
    double tx = g->tcam[0], ty = g->tcam[1], tz = g->tcam[2];
    double fx = S->cam.fx, fy = S->cam.fy;
    double du = d_uv[0], dv = d_uv[1];
    double dt[3];
    dt[0] = du * fx / tz + dJ[2] * (-fx / (tz * tz));
    dt[1] = dv * fy / tz + dJ[5] * (-fy / (tz * tz));
    dt[2] = du * (-fx * tx / (tz * tz)) + dv * (-fy * ty / (tz * tz)) + dJ[0] * (-fx / (tz * tz)) +
            dJ[2] * (2.0 * fx * tx / (tz * tz * tz)) + dJ[4] * (-fy / (tz * tz)) + dJ[5] * (2.0 * fy * ty / (tz * tz * tz));
    for (int k = 0; k < 3; ++k) dmu[k] = S->cam.W[k] * dt[0] + S->cam.W[3 + k] * dt[1] + S->cam.W[6 + k] * dt[2];

    /* Colour: rgb = max(0, sum_k sh_k Y_k(d_hat)); drgb is already zero on clamped channels. */
    double dd[3] = {0, 0, 0};
    for (int k = 0; k < D; ++k) {
        double w = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            dsh[3 * k + ch] = g->Y[k] * drgb[ch];
            w += S->sh[((size_t)i * S->sh_stride + k) * 3 + ch] * drgb[ch];
        }
        for (int r = 0; r < 3; ++r) dd[r] += w * g->dY[3 * k + r];
    }
    double dproj = dd[0] * g->dhat[0] + dd[1] * g->dhat[1] + dd[2] * g->dhat[2];
    for (int r = 0; r < 3; ++r) dmu[r] += (dd[r] - g->dhat[r] * dproj) / g->dnorm;
}

static void gauss_chain(const oscene* S, size_t i, const double* d_uv, const double* d_conic, const double* drgb,
                        double* dmu, double* ds, double* dq, double* dsh) {
    gauss_chain_g(S, i, &S->g[i], d_uv, d_conic, drgb, dmu, ds, dq, dsh);
}

/*
 * Conditioning of the chain rule in fp32 (test allowance; see orc_render_backward): the
 * first-order change of dL/d(mu, s, q, SH) when the quantities every fp32 implementation of
 * App. A must form from the fp32 inputs -- the rotation R(q_hat) (with M = R S), the projection
 * U = J W, the camera-space mean t and the view direction d_hat (with its SH basis) -- carry
 * relative rounding errors of COND_ROUNDINGS units in the last place.  Per quantity, two
 * perturbations of all its entries with pseudo-random signs (relative step COND_STEP) give a
 * finite-difference sensitivity; the larger of the two, summed over the quantities and times
 * COND_ROUNDINGS u, is added to out[] entry by entry.  The screen-space sums are held fixed:
 * their own conditioning depends on the frame an implementation accumulates them in.
 */
#define COND_ROUNDINGS 4.0
#define COND_STEP 9.5367431640625e-07   /* 2^-20 */
#define COND_U 5.9604644775390625e-08   /* 2^-24, unit roundoff of IEEE fp32 */

static double sign_hash(size_t i, int a, int t, int j) {
    uint64_t x = (uint64_t)i * 0x9E3779B97F4A7C15ull ^ (uint64_t)(a * 131 + t * 17 + j + 1) * 0xBF58476D1CE4E5B9ull;
    x ^= x >> 31; x *= 0x94D049BB133111EBull; x ^= x >> 29;
    return (x & 1) ? 1.0 : -1.0;
}

static void chain_conditioning(const oscene* S, size_t i, const double* d_uv, const double* d_conic,
                               const double* drgb, double* out /* [3 + 3 + 4 + 3D] */) {
    const ogauss* g = &S->g[i];
    const int D = (S->deg + 1) * (S->deg + 1), NY = 10 + 3 * D;
    double y0[58], y[58], sens[58], tot[58];
    gauss_chain_g(S, i, g, d_uv, d_conic, drgb, y0, y0 + 3, y0 + 6, y0 + 10);
    for (int e = 0; e < NY; ++e) tot[e] = 0.0;
    const double* s = S->scales + 3 * i;
    for (int a = 0; a < 4; ++a) {
        for (int e = 0; e < NY; ++e) sens[e] = 0.0;
        for (int t = 0; t < 2; ++t) {
            ogauss gp = *g;
            if (a == 0) {          /* R, and M = R S formed from it */
                for (int j = 0; j < 9; ++j) gp.R[j] *= 1.0 + COND_STEP * sign_hash(i, a, t, j);
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) gp.M[3 * r + c] = gp.R[3 * r + c] * s[c];
            } else if (a == 1) {   /* U = J W */
                for (int j = 0; j < 6; ++j) gp.U[j] *= 1.0 + COND_STEP * sign_hash(i, a, t, j);
            } else if (a == 2) {   /* camera-space mean */
                for (int j = 0; j < 3; ++j) gp.tcam[j] *= 1.0 + COND_STEP * sign_hash(i, a, t, j);
            } else {               /* view direction and its SH basis */
                for (int j = 0; j < 3; ++j) gp.dhat[j] *= 1.0 + COND_STEP * sign_hash(i, a, t, j);
                sh_basis(S->deg, gp.dhat, gp.Y, gp.dY);
            }
            gauss_chain_g(S, i, &gp, d_uv, d_conic, drgb, y, y + 3, y + 6, y + 10);
            for (int e = 0; e < NY; ++e) {
                const double d = fabs(y[e] - y0[e]) / COND_STEP;
                if (d > sens[e]) sens[e] = d;
            }
        }
        for (int e = 0; e < NY; ++e) tot[e] += sens[e];
    }
    for (int e = 0; e < NY; ++e) out[e] = COND_ROUNDINGS * COND_U * tot[e];
}

static void scene_init(oscene* S, long n, const double* means, const double* scales, const double* quats,
                       const double* opac, const double* sh, int deg, int sh_stride, const double* cam, const double* cfg) {
    memset(S, 0, sizeof(*S));
    S->n = (size_t)n; S->deg = deg; S->sh_stride = sh_stride;
    S->means = means; S->scales = scales; S->quats = quats; S->opac = opac; S->sh = sh;
    read_cam(cam, &S->cam);
    read_cfg(cfg, &S->cfg);
}

static int64_t max_list(const oscene* S) {
    int64_t m = 1;
    for (int t = 0; t < S->TX * S->TY; ++t) {
        int64_t l = S->tile_start[t + 1] - S->tile_start[t];
        if (l > m) m = l;
    }
    return m;
}

/* ------------------------------------------------------------------------- */
/* Exported: per-Gaussian preprocess outputs.                                  */
/* ------------------------------------------------------------------------- */
void orc_preprocess(long n, const double* means, const double* scales, const double* quats, const double* opac,
                    const double* sh, int deg, int sh_stride, const double* cam, const double* cfg,
                    int32_t* visible, double* uv, double* depth, double* cov2d, double* conic, int32_t* radius,
                    int32_t* rect, double* rgb, double* rgb_raw, uint32_t* amb, int32_t* rect_in, int32_t* rect_out) {
    ocam c; ocfg f;
    read_cam(cam, &c); read_cfg(cfg, &f);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        ogauss g;
        gauss_forward((size_t)i, means, scales, quats, opac, sh, deg, sh_stride, &c, &f, &g);
        visible[i] = g.visible;
        uv[2 * i] = g.uv[0]; uv[2 * i + 1] = g.uv[1];
        depth[i] = g.tcam[2];
        for (int k = 0; k < 3; ++k) { cov2d[3 * i + k] = g.cov2[k]; conic[3 * i + k] = g.conic[k]; rgb[3 * i + k] = g.rgb[k]; rgb_raw[3 * i + k] = g.rgb_raw[k]; }
        radius[i] = g.visible ? g.radius : 0;
        for (int k = 0; k < 4; ++k) { rect[4 * i + k] = g.visible ? g.rect[k] : 0; rect_in[4 * i + k] = g.rect_in[k]; rect_out[4 * i + k] = g.rect_out[k]; }
        amb[i] = g.amb;
    }
}

/* ------------------------------------------------------------------------- */
/* Exported: forward render (Algorithm 2, eq. front-to-back).                  */
/* tile_mask (may be NULL) selects the tiles to render; other pixels are left   */
/* untouched.  Images are planar [3, H, W].  out_pix_dec[p] has bit (kind - 1)  */
/* set for every kind of decision near its threshold at pixel p.  For each such */
/* decision one alternative is written (up to alt_cap): the pixel, the decision */
/* (kind, g0, g1), and the pixel's colour, T and last Gaussian with that        */
/* decision flipped.  counts[0] = alternatives found, counts[1] = decisions     */
/* beyond the per-pixel list capacity (not flipped; a test must see 0).         */
/* ------------------------------------------------------------------------- */
void orc_render_forward(long n, const double* means, const double* scales, const double* quats, const double* opac,
                        const double* sh, int deg, int sh_stride, const double* cam, const double* cfg,
                        const double* bg, const uint8_t* tile_mask, double* out_img, double* out_T, int32_t* out_last,
                        int32_t* out_last_id, uint8_t* out_pix_dec, uint32_t* out_gauss_amb, long alt_cap,
                        int64_t* alt_pix, int32_t* alt_dec, double* alt_img, double* alt_T, int32_t* alt_last_id,
                        long* counts) {
    oscene S;
    scene_init(&S, n, means, scales, quats, opac, sh, deg, sh_stride, cam, cfg);
    scene_build(&S, tile_mask);
    int W = S.cam.width, H = S.cam.height, T = S.TX * S.TY;
    size_t P = (size_t)W * H;
    if (out_gauss_amb)
        for (size_t i = 0; i < S.n; ++i) out_gauss_amb[i] = S.g[i].amb;
    const int64_t maxlen = max_list(&S);
    long nalt = 0, overflow = 0;
#pragma omp parallel
    {
        oscratch Wk;
        scratch_alloc(&Wk, maxlen);
#pragma omp for schedule(dynamic, 1) reduction(+ : overflow)
        for (int t = 0; t < T; ++t) {
            if (tile_mask && !tile_mask[t]) continue;
            int tx = t % S.TX, ty = t / S.TX;
            for (int ly = 0; ly < S.cfg.tile_h; ++ly)
                for (int lx = 0; lx < S.cfg.tile_w; ++lx) {
                    int px = tx * S.cfg.tile_w + lx, py = ty * S.cfg.tile_h + ly;
                    if (px >= W || py >= H) continue;
                    double C[3], Tf;
                    int last, ndec;
                    int32_t last_id;
                    pixel_walk(&S, t, px, py, NULL, &Wk, NULL, C, &Tf, &last, &last_id, &ndec);
                    size_t p = (size_t)py * W + px;
                    if (out_last_id) out_last_id[p] = last_id;
                    for (int ch = 0; ch < 3; ++ch) out_img[ch * P + p] = C[ch] + Tf * bg[ch];
                    out_T[p] = Tf;
                    out_last[p] = last;
                    if (ndec > Wk.dec_cap) { overflow += ndec - Wk.dec_cap; ndec = Wk.dec_cap; }
                    uint8_t bits = 0;
                    for (int d = 0; d < ndec; ++d) {
                        const odec_t dec = Wk.dec[d];
                        bits |= (uint8_t)(1u << (dec.kind - 1));
                        double C2[3], T2;
                        int32_t lid2;
                        pixel_walk(&S, t, px, py, &dec, &Wk, NULL, C2, &T2, NULL, &lid2, NULL);
                        long slot;
#pragma omp atomic capture
                        slot = nalt++;
                        if (slot < alt_cap) {
                            alt_pix[slot] = (int64_t)p;
                            alt_dec[3 * slot] = dec.kind; alt_dec[3 * slot + 1] = dec.g0; alt_dec[3 * slot + 2] = dec.g1;
                            for (int ch = 0; ch < 3; ++ch) alt_img[3 * slot + ch] = C2[ch] + T2 * bg[ch];
                            alt_T[slot] = T2;
                            alt_last_id[slot] = lid2;
                        }
                    }
                    if (out_pix_dec) out_pix_dec[p] = bits;
                }
        }
        scratch_free(&Wk);
    }
    counts[0] = nalt;
    counts[1] = overflow;
    scene_free(&S);
}

/* ------------------------------------------------------------------------- */
/* Exported: backward pass.  Per pixel: the forward walk keeping every T_i,   */
/* then the reverse walk (Sec. 6) gives dL/d(mean2D, conic, opacity, colour)   */
/* of each blended Gaussian; per Gaussian: chain rule of App. A down to        */
/* (mu, s, q, o, SH).                                                          */
/* allow_screen [n, 9] (dL/du, dL/dv, dL/dSigma' 00, 01, 11, dL/do, dL/drgb)   */
/* and allow_* (may all be NULL): for every decision near its threshold, the   */
/* pixel's gradient terms are recomputed with the decision flipped, and the    */
/* magnitude of the change they make to each Gaussian's gradients (screen      */
/* space, and through the chain rule the inputs) is added up; a colour channel */
/* near the 0 clamp adds the magnitude of its own chain-rule terms.  A test    */
/* can accept |g - g*| <= tolerance + allowance for every Gaussian.            */
/* cond_* (may be NULL): per gradient entry, the fp32 conditioning allowance  */
/* of the chain rule (chain_conditioning).                                     */
/* counts[0] = decisions flipped, counts[1] = decisions beyond the per-pixel   */
/* list capacity.                                                              */
/* ------------------------------------------------------------------------- */
static void atomic_add(double* p, double v) {
#pragma omp atomic
    *p += v;
}

typedef struct {
    double *screen, *means, *scales, *quats, *opac, *sh;
} oallow;

/* |change| of one Gaussian's gradients between two pixel walks: screen space and chained. */
static void allow_add(const oscene* S, const oallow* A, const pgrad_t* d) {
    const size_t i = (size_t)d->idx;
    const ogauss* g = &S->g[i];
    double H[4];
    conic_to_cov_grad(g, d->conic, H);
    double sc[9] = {d->uv[0], d->uv[1], H[0], H[1], H[3], d->op, d->rgb[0], d->rgb[1], d->rgb[2]};
    for (int k = 0; k < 9; ++k) if (sc[k] != 0.0) atomic_add(&A->screen[9 * i + k], fabs(sc[k]));
    if (d->op != 0.0) atomic_add(&A->opac[i], fabs(d->op));
    if (!g->valid) return;
    double drgb[3], dmu[3], ds[3], dq[4], dsh[48];
    for (int ch = 0; ch < 3; ++ch) drgb[ch] = g->rgb_raw[ch] > 0.0 ? d->rgb[ch] : 0.0;
    gauss_chain(S, i, d->uv, d->conic, drgb, dmu, ds, dq, dsh);
    for (int k = 0; k < 3; ++k) { atomic_add(&A->means[3 * i + k], fabs(dmu[k])); atomic_add(&A->scales[3 * i + k], fabs(ds[k])); }
    for (int k = 0; k < 4; ++k) atomic_add(&A->quats[4 * i + k], fabs(dq[k]));
    const int D = (S->deg + 1) * (S->deg + 1);
    for (int k = 0; k < 3 * D; ++k) if (dsh[k] != 0.0) atomic_add(&A->sh[(size_t)i * S->sh_stride * 3 + k], fabs(dsh[k]));
}

static int cmp_pg(const void* a, const void* b) {
    int32_t x = ((const pgrad_t*)a)->idx, y = ((const pgrad_t*)b)->idx;
    return (x > y) - (x < y);
}

/* Add |alt - main| per Gaussian (both lists sorted by index). */
static void allow_delta(const oscene* S, const oallow* A, const pgrad_t* p1, int n1, const pgrad_t* p2, int n2) {
    int a = 0, b = 0;
    while (a < n1 || b < n2) {
        pgrad_t d;
        memset(&d, 0, sizeof(d));
        int take1 = b >= n2 || (a < n1 && p1[a].idx <= p2[b].idx);
        int take2 = a >= n1 || (b < n2 && p2[b].idx <= p1[a].idx);
        d.idx = take1 ? p1[a].idx : p2[b].idx;
        for (int k = 0; k < 2; ++k) d.uv[k] = (take2 ? p2[b].uv[k] : 0.0) - (take1 ? p1[a].uv[k] : 0.0);
        for (int k = 0; k < 3; ++k) d.conic[k] = (take2 ? p2[b].conic[k] : 0.0) - (take1 ? p1[a].conic[k] : 0.0);
        for (int k = 0; k < 3; ++k) d.rgb[k] = (take2 ? p2[b].rgb[k] : 0.0) - (take1 ? p1[a].rgb[k] : 0.0);
        d.op = (take2 ? p2[b].op : 0.0) - (take1 ? p1[a].op : 0.0);
        allow_add(S, A, &d);
        if (take1) ++a;
        if (take2) ++b;
    }
}

void orc_render_backward(long n, const double* means, const double* scales, const double* quats, const double* opac,
                         const double* sh, int deg, int sh_stride, const double* cam, const double* cfg,
                         const double* bg, const uint8_t* tile_mask, const double* dL_dimg,
                         double* d_means, double* d_scales, double* d_quats, double* d_opac, double* d_sh,
                         double* d_uv, double* d_conic, double* d_rgb, double* d_cov2d,
                         uint8_t* out_pix_dec, uint32_t* out_gauss_amb,
                         double* allow_screen, double* allow_means, double* allow_scales, double* allow_quats,
                         double* allow_opac, double* allow_sh, double* cond_means, double* cond_scales,
                         double* cond_quats, double* cond_sh, long* counts) {
    oscene S;
    scene_init(&S, n, means, scales, quats, opac, sh, deg, sh_stride, cam, cfg);
    scene_build(&S, tile_mask);
    int W = S.cam.width, H = S.cam.height, T = S.TX * S.TY;
    size_t P = (size_t)W * H;
    int D = (deg + 1) * (deg + 1);
    memset(d_uv, 0, sizeof(double) * 2 * S.n);
    memset(d_conic, 0, sizeof(double) * 3 * S.n);
    memset(d_rgb, 0, sizeof(double) * 3 * S.n);
    memset(d_opac, 0, sizeof(double) * S.n);
    oallow A = {allow_screen, allow_means, allow_scales, allow_quats, allow_opac, allow_sh};
    const int want_allow = allow_screen != NULL;
    if (want_allow) {
        memset(allow_screen, 0, sizeof(double) * 9 * S.n);
        memset(allow_means, 0, sizeof(double) * 3 * S.n);
        memset(allow_scales, 0, sizeof(double) * 3 * S.n);
        memset(allow_quats, 0, sizeof(double) * 4 * S.n);
        memset(allow_opac, 0, sizeof(double) * S.n);
        memset(allow_sh, 0, sizeof(double) * 3 * (size_t)sh_stride * S.n);
    }
    if (cond_means) {
        memset(cond_means, 0, sizeof(double) * 3 * S.n);
        memset(cond_scales, 0, sizeof(double) * 3 * S.n);
        memset(cond_quats, 0, sizeof(double) * 4 * S.n);
        memset(cond_sh, 0, sizeof(double) * 3 * (size_t)sh_stride * S.n);
    }
    if (out_gauss_amb)
        for (size_t i = 0; i < S.n; ++i) out_gauss_amb[i] = S.g[i].amb;
    const int64_t maxlen = max_list(&S);
    long nflip = 0, overflow = 0;

#pragma omp parallel
    {
        oscratch Wk;
        scratch_alloc(&Wk, maxlen);
#pragma omp for schedule(dynamic, 1) reduction(+ : nflip, overflow)
        for (int t = 0; t < T; ++t) {
            if (tile_mask && !tile_mask[t]) continue;
            int tx = t % S.TX, ty = t / S.TX;
            for (int ly = 0; ly < S.cfg.tile_h; ++ly)
                for (int lx = 0; lx < S.cfg.tile_w; ++lx) {
                    int px = tx * S.cfg.tile_w + lx, py = ty * S.cfg.tile_h + ly;
                    if (px >= W || py >= H) continue;
                    size_t p = (size_t)py * W + px;
                    double C[3], Tf;
                    int last, ndec;
                    int32_t last_id;
                    int nrec = pixel_walk(&S, t, px, py, NULL, &Wk, Wk.rec, C, &Tf, &last, &last_id, &ndec);
                    if (ndec > Wk.dec_cap) { overflow += ndec - Wk.dec_cap; ndec = Wk.dec_cap; }
                    const double dC[3] = {dL_dimg[p], dL_dimg[P + p], dL_dimg[2 * P + p]};
                    pixel_backward(&S, Wk.rec, nrec, dC, bg, Wk.pg);
                    for (int k = 0; k < nrec; ++k) {
                        const pgrad_t* q = &Wk.pg[k];
                        const int32_t i = q->idx;
                        for (int c = 0; c < 3; ++c) if (q->rgb[c] != 0.0) atomic_add(&d_rgb[3 * i + c], q->rgb[c]);
                        if (q->op != 0.0) {
                            atomic_add(&d_opac[i], q->op);
                            for (int c = 0; c < 3; ++c) atomic_add(&d_conic[3 * i + c], q->conic[c]);
                            for (int c = 0; c < 2; ++c) atomic_add(&d_uv[2 * i + c], q->uv[c]);
                        }
                    }
                    uint8_t bits = 0;
                    for (int d = 0; d < ndec; ++d) bits |= (uint8_t)(1u << (Wk.dec[d].kind - 1));
                    if (out_pix_dec) out_pix_dec[p] = bits;
                    if (!want_allow || ndec == 0) continue;
                    qsort(Wk.pg, (size_t)nrec, sizeof(pgrad_t), cmp_pg);
                    for (int d = 0; d < ndec; ++d) {
                        double C2[3], T2;
                        const odec_t dec = Wk.dec[d];
                        int n2 = pixel_walk(&S, t, px, py, &dec, &Wk, Wk.rec2, C2, &T2, NULL, NULL, NULL);
                        pixel_backward(&S, Wk.rec2, n2, dC, bg, Wk.pg2);
                        qsort(Wk.pg2, (size_t)n2, sizeof(pgrad_t), cmp_pg);
                        allow_delta(&S, &A, Wk.pg, nrec, Wk.pg2, n2);
                        ++nflip;
                    }
                }
        }
        scratch_free(&Wk);
    }
    if (counts) { counts[0] = nflip; counts[1] = overflow; }

    /* Per Gaussian: chain rule of App. A. */
#pragma omp parallel for schedule(static)
    for (long i = 0; i < (long)S.n; ++i) {
        const ogauss* g = &S.g[i];
        double* dmu = d_means + 3 * i;
        double* ds = d_scales + 3 * i;
        double* dq = d_quats + 4 * i;
        double* dsh = d_sh + (size_t)i * sh_stride * 3;
        for (int k = 0; k < 3; ++k) { dmu[k] = 0.0; ds[k] = 0.0; }
        for (int k = 0; k < 4; ++k) dq[k] = 0.0;
        for (int k = 0; k < sh_stride * 3; ++k) dsh[k] = 0.0;
        d_cov2d[3 * i] = d_cov2d[3 * i + 1] = d_cov2d[3 * i + 2] = 0.0;
        if (!g->visible) { d_opac[i] = 0.0; continue; }
        double Hc[4];
        conic_to_cov_grad(g, d_conic + 3 * i, Hc);
        d_cov2d[3 * i + 0] = Hc[0];
        d_cov2d[3 * i + 1] = Hc[1];
        d_cov2d[3 * i + 2] = Hc[3];
        double drgb[3];
        for (int ch = 0; ch < 3; ++ch) drgb[ch] = g->rgb_raw[ch] > 0.0 ? d_rgb[3 * i + ch] : 0.0;
        gauss_chain(&S, (size_t)i, d_uv + 2 * i, d_conic + 3 * i, drgb, dmu, ds, dq, dsh);
        if (cond_means) {
            double c[58];
            chain_conditioning(&S, (size_t)i, d_uv + 2 * i, d_conic + 3 * i, drgb, c);
            for (int k = 0; k < 3; ++k) { cond_means[3 * i + k] = c[k]; cond_scales[3 * i + k] = c[3 + k]; }
            for (int k = 0; k < 4; ++k) cond_quats[4 * i + k] = c[6 + k];
            for (int k = 0; k < 3 * D; ++k) cond_sh[(size_t)i * sh_stride * 3 + k] = c[10 + k];
        }
        if (!want_allow) continue;
        /* a colour channel near the 0 clamp: its gradient terms may be absent or present */
        for (int ch = 0; ch < 3; ++ch) {
            if (!(g->rgb_amb & (1u << ch)) || d_rgb[3 * i + ch] == 0.0) continue;
            const double zero2[2] = {0.0, 0.0}, zero3[3] = {0.0, 0.0, 0.0};
            double one[3] = {0.0, 0.0, 0.0}, amu[3], as[3], aq[4], ash[48];
            one[ch] = d_rgb[3 * i + ch];
            gauss_chain(&S, (size_t)i, zero2, zero3, one, amu, as, aq, ash);
            for (int k = 0; k < 3; ++k) allow_means[3 * i + k] += fabs(amu[k]);
            for (int k = 0; k < 3 * D; ++k) allow_sh[(size_t)i * sh_stride * 3 + k] += fabs(ash[k]);
        }
    }
    scene_free(&S);
}

/* ------------------------------------------------------------------------- */
/* Reachable-tile rule (this implementation's refinement of the Sec. 6 tile      */
/* rectangle; the paper has no counterpart).  A pixel at offset d from the mean   */
/* is blended only if o exp(-|L^T d|^2 / 2) >= alpha_min, i.e. |L^T d|^2 <= tau,  */
/* tau = 2 ln(o / alpha_min), with L = [[l11, 0], [l21, l22]] the Cholesky factor */
/* of the conic.  Of the rectangle's tiles, a row keeps the column interval whose */
/* pixel centres meet the (slightly widened) ellipse.  The decision is taken in   */
/* IEEE fp32 round-to-nearest arithmetic, written out step by step below, which  */
/* is the precision the rasterizer decides it in; -ffp-contract=off keeps every  */
/* product and sum separately rounded.                                            */
/*   t    = tau (1 + 2^-10) + 2^-10           (no tiles when t <= 0)             */
/*   ylim = sqrt(t) / l22                      (|dy| bound of the ellipse)         */
/*   S    = (L L^T)^-1:  S00 = (l21^2 + l22^2) / (l11 l22)^2,                     */
/*                       S01 = -l21 / ((l11 l22) l22)                             */
/*   y*   = S01 sqrt(t / S00)                  (dy of the ellipse's rightmost point) */
/*   X(y, s) = (s sqrt(max(t - (l22 y)^2, 0)) - l21 y) * (1 / l11)                */
/* Row ty: pixel-centre offsets dy in [ya, yb] = [ty th + 0.5 - v, ty th + th - 0.5 - v] */
/* clipped to [-ylim, ylim]; the rightmost reach over that band is X(clip(y*), +1), */
/* the leftmost X(clip(-y*), -1) (each branch is concave/convex in y); widened by */
/* 0.01 px they bound the columns px with px + 0.5 - u inside; the tiles holding  */
/* those columns, cut to the rectangle, are kept.                                 */
/* This rule is a restatement of a decision the rasterizer takes in fp32, not a   */
/* definition from the paper: it serves the bit-exact binning test of the         */
/* default schedule only.  It is pinned apart from the rasterizer by FP64 brute   */
/* force over pixel centres (every tile with a pixel reaching alpha_min is kept,  */
/* every kept tile lies in the rectangle and near the ellipse; orc_reach_needed), */
/* and on the benchmark frame the GPU's kept tiles are checked against that FP64  */
/* set directly; images are shown identical to the rectangle rule's.              */
/* ------------------------------------------------------------------------- */
static float reach_x32(float t, float inv11, float l21, float l22, float y, float s) {
    float q = l22 * y;
    float q2 = q * q;
    float h = t - q2;
    h = sqrtf(h > 0.0f ? h : 0.0f);
    float num = s * h - l21 * y;
    return num * inv11;
}

static float clampf32(float x, float lo, float hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* Columns [*txa, *txb) of tile row ty inside the rectangle columns [x0, x1). */
static int reach_row32(const float* L, float tau, float u, float v, int ty, int tw, int th, int x0, int x1,
                       int* txa, int* txb) {
    const float w = 0.0009765625f;
    float t = tau * (1.0f + w) + w;
    if (!(t > 0.0f)) return 0;
    float l11 = L[0], l21 = L[1], l22 = L[2];
    float inv11 = 1.0f / l11;
    float ylim = sqrtf(t) / l22;
    float a = l11 * l22;
    float s00 = (l21 * l21 + l22 * l22) / (a * a);
    float s01 = (-l21) / (a * l22);
    float ystar = s01 * sqrtf(t / s00);
    float ya = ((float)(ty * th) + 0.5f) - v;
    float yb = ((float)(ty * th + th) - 0.5f) - v;
    if (ya < -ylim) ya = -ylim;
    if (yb > ylim) yb = ylim;
    if (ya > yb) return 0;
    float xb = reach_x32(t, inv11, l21, l22, clampf32(ystar, ya, yb), 1.0f) + 0.01f;
    float xa = reach_x32(t, inv11, l21, l22, clampf32(-ystar, ya, yb), -1.0f) - 0.01f;
    float fa = ceilf((u + xa) - 0.5f), fb = floorf((u + xb) - 0.5f);
    const float lim = 1048576.0f;
    int pa = (int)clampf32(fa, -lim, lim), pb = (int)clampf32(fb, -lim, lim);
    if (pb < pa) return 0;
    int lo = floor_div(pa, tw), hi = floor_div(pb, tw) + 1;
    *txa = lo > x0 ? lo : x0;
    *txb = hi < x1 ? hi : x1;
    return *txa < *txb;
}

/* ------------------------------------------------------------------------- */
/* Exported: binning definition (App. C) on given fp32 screen-space values.     */
/* Emits one key per (Gaussian, tile) in Gaussian order then row-major tile      */
/* order, key = (tile id << 32) | fp32 bits of depth, stable-sorts by key (ties   */
/* keep emission order), and finds each tile's [start, end).  The tiles are the   */
/* 3-sigma rectangle's (Sec. 6); when chol and tau are given, only those the     */
/* reachable-tile rule above keeps.  radius <= 0 marks a culled Gaussian.         */
/* Returns the number of instances, or -1 if it exceeds capacity (nothing is     */
/* written past capacity).                                                       */
/* ------------------------------------------------------------------------- */
typedef struct { uint64_t key; int64_t seq; uint32_t val; } inst_t;

static int cmp_inst(const void* a, const void* b) {
    const inst_t* x = (const inst_t*)a;
    const inst_t* y = (const inst_t*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->seq > y->seq) - (x->seq < y->seq);
}

/* Tiles of Gaussian i in row ty: [*a, *b); 0 if none. */
static int bin_row(long i, int ty, const float* uv, const int32_t* radius, const float* chol, const float* tau,
                   int TX, int TY, int tile_w, int tile_h, int* a, int* b) {
    if (radius[i] <= 0) return 0;
    int fu = (int)floorf(uv[2 * i]), fv = (int)floorf(uv[2 * i + 1]), r = radius[i];
    int x0 = clampi(floor_div(fu - r, tile_w), 0, TX), x1 = clampi(floor_div(fu + r, tile_w) + 1, 0, TX);
    int y0 = clampi(floor_div(fv - r, tile_h), 0, TY), y1 = clampi(floor_div(fv + r, tile_h) + 1, 0, TY);
    if (ty < y0 || ty >= y1 || x0 >= x1) return 0;
    if (!chol) { *a = x0; *b = x1; return 1; }
    return reach_row32(&chol[3 * i], tau[i], uv[2 * i], uv[2 * i + 1], ty, tile_w, tile_h, x0, x1, a, b);
}

long orc_bin(long n, const float* uv, const float* depth, const int32_t* radius, const float* chol, const float* tau,
             int width, int height, int tile_w, int tile_h, long capacity, uint64_t* keys, uint32_t* vals,
             uint32_t* ranges) {
    int TX = (width + tile_w - 1) / tile_w, TY = (height + tile_h - 1) / tile_h;
    long K = 0;
    for (long i = 0; i < n; ++i)
        for (int ty = 0; ty < TY; ++ty) {
            int a, b;
            if (bin_row(i, ty, uv, radius, chol, tau, TX, TY, tile_w, tile_h, &a, &b)) K += b - a;
        }
    for (long t = 0; t < (long)TX * TY; ++t) { ranges[2 * t] = 0; ranges[2 * t + 1] = 0; }
    if (K > capacity) return -K;
    if (!keys) return K;
    inst_t* inst = (inst_t*)malloc(sizeof(inst_t) * (size_t)(K ? K : 1));
    long k = 0;
    for (long i = 0; i < n; ++i) {
        uint32_t dbits;
        memcpy(&dbits, &depth[i], 4);
        for (int ty = 0; ty < TY; ++ty) {
            int a, b;
            if (!bin_row(i, ty, uv, radius, chol, tau, TX, TY, tile_w, tile_h, &a, &b)) continue;
            for (int tx = a; tx < b; ++tx) {
                inst[k].key = ((uint64_t)(uint32_t)(ty * TX + tx) << 32) | dbits;
                inst[k].seq = k;
                inst[k].val = (uint32_t)i;
                ++k;
            }
        }
    }
    qsort(inst, (size_t)K, sizeof(inst_t), cmp_inst);
    for (long j = 0; j < K; ++j) {
        keys[j] = inst[j].key;
        vals[j] = inst[j].val;
        uint32_t t = (uint32_t)(inst[j].key >> 32);
        if (j == 0 || (uint32_t)(inst[j - 1].key >> 32) != t) ranges[2 * t] = (uint32_t)j;
        if (j == K - 1 || (uint32_t)(inst[j + 1].key >> 32) != t) ranges[2 * t + 1] = (uint32_t)(j + 1);
    }
    free(inst);
    return K;
}

/* ------------------------------------------------------------------------- */
/* Exported: (Gaussian, tile) pairs of the Sec. 6 rectangle that any binning   */
/* must keep: tiles that every rounding of the rectangle contains (rect_in) in */
/* which some pixel centre certainly reaches alpha_min in FP64, i.e.           */
/* o G >= alpha_min (1 + eps_alpha + power margin); found by brute force over  */
/* the tile's pixels.  Writes keys i * tiles + t (up to cap); returns the      */
/* number of pairs.                                                            */
/* ------------------------------------------------------------------------- */
long orc_reach_needed(long n, const double* means, const double* scales, const double* quats, const double* opac,
                      const double* sh, int deg, int sh_stride, const double* cam, const double* cfg, long cap,
                      int64_t* out) {
    ocam c; ocfg f;
    read_cam(cam, &c); read_cfg(cfg, &f);
    const int TX = (c.width + f.tile_w - 1) / f.tile_w, TY = (c.height + f.tile_h - 1) / f.tile_h;
    long count = 0;
#pragma omp parallel for schedule(dynamic, 256)
    for (long i = 0; i < n; ++i) {
        ogauss g;
        gauss_forward((size_t)i, means, scales, quats, opac, sh, deg, sh_stride, &c, &f, &g);
        if (!g.visible || (g.amb & AMB_CULL)) continue;
        for (int ty = g.rect_in[2]; ty < g.rect_in[3]; ++ty)
            for (int tx = g.rect_in[0]; tx < g.rect_in[1]; ++tx) {
                int hit = 0;
                for (int ly = 0; ly < f.tile_h && !hit; ++ly)
                    for (int lx = 0; lx < f.tile_w && !hit; ++lx) {
                        const int px = tx * f.tile_w + lx, py = ty * f.tile_h + ly;
                        if (px >= c.width || py >= c.height) continue;
                        double dx, dy;
                        const double oG = opac[i] * exp(eval_power(&g, px + 0.5, py + 0.5, &dx, &dy));
                        hit = oG >= f.alpha_min * (1.0 + f.eps_alpha + power_margin(&g, dx, dy, &f));
                    }
                if (!hit) continue;
                long slot;
#pragma omp atomic capture
                slot = count++;
                if (slot < cap) out[slot] = (int64_t)i * TX * TY + (int64_t)(ty * TX + tx);
            }
    }
    return count;
}

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
