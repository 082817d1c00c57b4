/*
 * FP64 CPU oracle for the vortex-particle hot path of the NL-UVLM-VPM method
 * (Fu & Laurendeau, arXiv 2511.11430).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only tests/, the smoke check and the CPU-baseline leg of bench.py do.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * Every routine is the plain definition written out in double precision: direct
 * double loops, no blocking, no truncation of the Gaussian kernel, no FMM.
 * OpenMP only splits the independent outer loop over targets (or sources for the
 * adjoint); each target's sum runs in source order.
 *
 * Layouts (row-major, "AoS"):
 *   particles  pos[n][4] = (x, y, z, volume)   str[n][4] = (Gx, Gy, Gz, unused)
 *   targets    tgt[n][4] = (x, y, z, unused)
 *   segments   a[m][4]   = (ax, ay, az, circulation)   b[m][4] = (bx, by, bz, unused)
 *   outputs    u[n][3], J[n][9] with J[3*a+b] = d u_a / d x_b
 *
 * Readings of the paper that this file fixes are listed next to the routine.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const double PI = 3.14159265358979323846264338327950288;

/* Levi-Civita symbol e_{abc}. */
static double levi(int a, int b, int c)
{
    if (a == b || b == c || a == c) return 0.0;
    if ((a == 0 && b == 1 && c == 2) || (a == 1 && b == 2 && c == 0) || (a == 2 && b == 0 && c == 1))
        return 1.0;
    return -1.0;
}

static void cross(const double* p, const double* q, double* out)
{
    out[0] = p[1] * q[2] - p[2] * q[1];
    out[1] = p[2] * q[0] - p[0] * q[2];
    out[2] = p[0] * q[1] - p[1] * q[0];
}

static double dot(const double* p, const double* q) { return p[0] * q[0] + p[1] * q[1] + p[2] * q[2]; }

/* ------------------------------------------------------------------------- */
/* Gaussian blob radial functions (Eq. 2-3).                                  */
/*                                                                            */
/* zeta_sigma(rho) = (2 pi sigma^2)^(-3/2) exp(-rho^2/2) integrates to 1 over  */
/* space (Eq. 3; the nomenclature's 1/m^2 unit is read as 1/m^3).  The share  */
/* of one blob's vorticity inside radius rho*sigma is                         */
/*     g(rho) = sqrt(2/pi) * int_0^rho s^2 exp(-s^2/2) ds                      */
/*            = erf(rho/sqrt2) - sqrt(2/pi) rho exp(-rho^2/2),                 */
/* and with it the regularised Biot-Savart kernel of one blob reads           */
/*     u(x) = K(r) Gamma x r,  K = g(rho) / (4 pi r^3),  r = x - x_j.           */
/* Its radial derivative enters the gradient through                          */
/*     H = K'(r)/r = F(rho) / (4 pi r^5),  F = rho g'(rho) - 3 g(rho).           */
/* Below rho = 1 the closed form loses digits to cancellation, so the Taylor  */
/* series of the integrand, integrated term by term, is used instead (with    */
/* x = rho^2/2):                                                              */
/*     g/rho^3 =  sqrt(2/pi) sum_k (-x)^k / (k! (2k+3))                        */
/*     F/rho^5 = -sqrt(2/pi) sum_k (-x)^k / (k! (2k+5))                        */
/* (the second from rho g' - 3 g = sqrt(2/pi) sum_k (-1)^k 2k rho^(2k+3) /     */
/* (2^k k! (2k+3)), re-indexed).                                              */
/* ------------------------------------------------------------------------- */
static const double SQRT_2_OVER_PI = 0.79788456080286535587989211986876373;

/* q = g(rho)/rho^3 and f = F(rho)/rho^5; valid for rho >= 0 (limits at 0). */
static void blob_qf(double rho, double* q, double* f)
{
    if (rho < 1.0) {
        const double x = 0.5 * rho * rho;
        double qs = 0.0, fs = 0.0;
        double term = 1.0; /* (-x)^k / k! */
        for (int k = 0; k < 60; ++k) {
            if (k > 0) term *= -x / (double)k;
            qs += term / (2.0 * k + 3.0);
            fs += term / (2.0 * k + 5.0);
            if (fabs(term) < 1e-20) break;
        }
        *q = SQRT_2_OVER_PI * qs;
        *f = -SQRT_2_OVER_PI * fs;
        return;
    }
    const double e = exp(-0.5 * rho * rho);
    const double g = erf(rho / sqrt(2.0)) - SQRT_2_OVER_PI * rho * e;
    const double F = SQRT_2_OVER_PI * rho * rho * rho * e - 3.0 * g;
    const double r3 = rho * rho * rho;
    *q = g / r3;
    *f = F / (r3 * rho * rho);
}

/* g(rho) and F(rho) at given rho values (exposed so tests can pin them). */
void orc_blob_gF(const double* rho, int64_t n, double* g, double* F)
{
    for (int64_t i = 0; i < n; ++i) {
        double q, f;
        blob_qf(rho[i], &q, &f);
        const double r = rho[i];
        g[i] = q * r * r * r;
        F[i] = f * r * r * r * r * r;
    }
}

/* K(r) and H(r) for one pair; returns 0 when r == 0 (no self-induction). */
static int blob_KH(double r, double sigma, double* K, double* H)
{
    if (r == 0.0) return 0;
    double q, f;
    const double rho = r / sigma;
    blob_qf(rho, &q, &f);
    const double s3 = sigma * sigma * sigma;
    *K = q / (4.0 * PI * s3);            /* g/(4 pi r^3) = (g/rho^3)/(4 pi sigma^3) */
    *H = f / (4.0 * PI * s3 * sigma * sigma); /* F/(4 pi r^5) */
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Particle -> point velocity and velocity gradient (Eq. 2-4; the gradient is */
/* the one the VPM needs for stretching and the SGS model).                   */
/*   u_a(x)  = sum_j K (Gamma_j x r)_a                                        */
/*   J_ab(x) = sum_j [ K e_{acb} Gamma_{j,c} + H (Gamma_j x r)_a r_b ]         */
/* A pair with r == 0 contributes nothing, which excludes a particle's own    */
/* term when the targets are the particles themselves.                        */
/* ------------------------------------------------------------------------- */
void orc_p2p(const double* pos, const double* str, int64_t n_src, const double* tgt, int64_t n_tgt,
             double sigma, double* u, double* J)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_tgt; ++i) {
        double ui[3] = {0, 0, 0};
        double Ji[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t j = 0; j < n_src; ++j) {
            double r[3] = {tgt[4 * i + 0] - pos[4 * j + 0], tgt[4 * i + 1] - pos[4 * j + 1],
                           tgt[4 * i + 2] - pos[4 * j + 2]};
            const double rr = sqrt(dot(r, r));
            double K, H;
            if (!blob_KH(rr, sigma, &K, &H)) continue;
            const double* G = &str[4 * j];
            double c[3];
            cross(G, r, c);
            for (int a = 0; a < 3; ++a) ui[a] += K * c[a];
            if (J) {
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        double t = 0.0;
                        for (int cc = 0; cc < 3; ++cc) t += levi(a, cc, b) * G[cc];
                        Ji[3 * a + b] += K * t + H * c[a] * r[b];
                    }
            }
        }
        for (int a = 0; a < 3; ++a) u[3 * i + a] = ui[a];
        if (J)
            for (int k = 0; k < 9; ++k) J[9 * i + k] = Ji[k];
    }
}

/* ------------------------------------------------------------------------- */
/* Straight vortex segment a->b of circulation Gs with a Vatistas core        */
/* (the blade and near-wake vortex lines).  The singular Biot-Savart law of a */
/* finite segment,                                                            */
/*   u = Gs/(4 pi) (r1 x r2) [r0 . (r1/|r1| - r2/|r2|)] / |r1 x r2|^2,          */
/* with r0 = b - a, r1 = x - a, r2 = x - b, has |r1 x r2|^2 = h^2 |r0|^2 for    */
/* the distance h to the line; the Vatistas kernel of exponent n replaces     */
/* h^2 by (h^(2n) + rc^(2n))^(1/n), i.e. the denominator becomes               */
/*   D = (|r1 x r2|^(2n) + (rc |r0|)^(2n))^(1/n).                              */
/* The gradient is the analytic x-derivative of that expression.  Points      */
/* within 1e-10 |r0| (or 1e-15 m) of an end point get zero, as does D == 0   */
/* (no core, on the line).                                                    */
/* ------------------------------------------------------------------------- */
static void segment_uJ(const double* A, const double* B, double Gs, const double* x, double rc, int vn,
                       double* u, double* J)
{
    double r0[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double r1[3] = {x[0] - A[0], x[1] - A[1], x[2] - A[2]};
    double r2[3] = {x[0] - B[0], x[1] - B[1], x[2] - B[2]};
    const double L = sqrt(dot(r0, r0));
    const double n1 = sqrt(dot(r1, r1));
    const double n2 = sqrt(dot(r2, r2));
    for (int k = 0; k < 3; ++k) u[k] = 0.0;
    if (J)
        for (int k = 0; k < 9; ++k) J[k] = 0.0;
    if (L == 0.0 || n1 <= 1e-10 * L || n2 <= 1e-10 * L || n1 <= 1e-15 || n2 <= 1e-15) return;

    double c[3];
    cross(r1, r2, c);
    const double c2 = dot(c, c);
    const double d = dot(r0, r1) / n1 - dot(r0, r2) / n2;
    const double e = pow(rc * L, 2.0 * vn);
    const double D = pow(pow(c2, (double)vn) + e, 1.0 / vn);
    if (D == 0.0) return;
    const double pref = Gs / (4.0 * PI);
    for (int a = 0; a < 3; ++a) u[a] = pref * c[a] * d / D;
    if (!J) return;

    /* d c_a / d x_m = e_{a b m} r0_b  (c = r1 x r2 = r0 x r1). */
    /* d d / d x_m   = sum_k r0_k [ (delta_km - r1h_k r1h_m)/|r1| - (delta_km - r2h_k r2h_m)/|r2| ] */
    /* d D / d x_m   = (1/n) (c2^n + e)^(1/n - 1) * n c2^(n-1) * d c2/d x_m,  d c2/d x_m = 2 c_a dc_a/dx_m */
    double dd[3], dc2[3], dD[3];
    for (int m = 0; m < 3; ++m) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double dk = (k == m) ? 1.0 : 0.0;
            s += r0[k] * ((dk - r1[k] * r1[m] / (n1 * n1)) / n1 - (dk - r2[k] * r2[m] / (n2 * n2)) / n2);
        }
        dd[m] = s;
        double t = 0.0;
        for (int a = 0; a < 3; ++a) {
            double dca = 0.0;
            for (int b = 0; b < 3; ++b) dca += levi(a, b, m) * r0[b];
            t += 2.0 * c[a] * dca;
        }
        dc2[m] = t;
        const double dDdc2 = (vn == 1) ? 1.0 : pow(pow(c2, (double)vn) + e, 1.0 / vn - 1.0) * pow(c2, vn - 1.0);
        dD[m] = dDdc2 * dc2[m];
    }
    for (int a = 0; a < 3; ++a)
        for (int m = 0; m < 3; ++m) {
            double dca = 0.0;
            for (int b = 0; b < 3; ++b) dca += levi(a, b, m) * r0[b];
            /* quotient and product rule on c_a d / D */
            J[3 * a + m] = pref * (dca * d / D + c[a] * dd[m] / D - c[a] * d * dD[m] / (D * D));
        }
}

void orc_segments(const double* sa, const double* sb, int64_t m, const double* tgt, int64_t n_tgt, double rc,
                  int vn, double* u, double* J)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_tgt; ++i) {
        double ui[3] = {0, 0, 0}, Ji[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t s = 0; s < m; ++s) {
            double us[3], Js[9];
            segment_uJ(&sa[4 * s], &sb[4 * s], sa[4 * s + 3], &tgt[4 * i], rc, vn, us, J ? Js : NULL);
            for (int a = 0; a < 3; ++a) ui[a] += us[a];
            if (J)
                for (int k = 0; k < 9; ++k) Ji[k] += Js[k];
        }
        for (int a = 0; a < 3; ++a) u[3 * i + a] = ui[a];
        if (J)
            for (int k = 0; k < 9; ++k) J[9 * i + k] = Ji[k];
    }
}

/* ------------------------------------------------------------------------- */
/* Vreman (2004) eddy viscosity, the SGS model of the VPM (coefficient c_V,   */
/* 0.07 in the paper).  With alpha_ij = d u_j / d x_i, beta_ij = Delta^2      */
/* sum_m alpha_mi alpha_mj and                                                */
/*   B = b11 b22 - b12^2 + b11 b33 - b13^2 + b22 b33 - b23^2,                  */
/* nu_t = c_V sqrt(B / (alpha_ij alpha_ij)), zero when alpha = 0 (or B <= 0   */
/* by rounding).  Reading: the filter width Delta is the core size sigma.     */
/* ------------------------------------------------------------------------- */
void orc_vreman(const double* J, int64_t n, double delta, double c_v, double* nu_t)
{
    for (int64_t p = 0; p < n; ++p) {
        const double* Jp = &J[9 * p];
        double al[3][3], be[3][3];
        double aa = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                al[i][j] = Jp[3 * j + i]; /* alpha_ij = d u_j / d x_i = J_ji */
                aa += al[i][j] * al[i][j];
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int m = 0; m < 3; ++m) s += al[m][i] * al[m][j];
                be[i][j] = delta * delta * s;
            }
        const double B = be[0][0] * be[1][1] - be[0][1] * be[0][1] + be[0][0] * be[2][2] - be[0][2] * be[0][2] +
                         be[1][1] * be[2][2] - be[1][2] * be[1][2];
        nu_t[p] = (aa > 0.0 && B > 0.0) ? c_v * sqrt(B / aa) : 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* Vortex stretching of Eq. 5, (Gamma . grad^T) u = J^T Gamma, the default;   */
/* the classic form of Eq. 1, (Gamma . grad) u = J Gamma, when classic != 0.  */
/* ------------------------------------------------------------------------- */
void orc_stretch(const double* J, const double* str, int64_t n, int classic, double* s)
{
    for (int64_t p = 0; p < n; ++p) {
        const double* Jp = &J[9 * p];
        const double* G = &str[4 * p];
        for (int a = 0; a < 3; ++a) {
            double t = 0.0;
            for (int b = 0; b < 3; ++b) t += classic ? Jp[3 * a + b] * G[b] : Jp[3 * b + a] * G[b];
            s[3 * p + a] = t;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Viscous diffusion nu lap(omega) of Eq. 5 by particle strength exchange.    */
/* The paper defers the scheme to earlier work; the reading here is the       */
/* Degond-Mas-Gallic form with the Eq. 3 Gaussian as exchange kernel:         */
/*   p_i = (2/sigma^2) sum_j nu_ij (v_i Gamma_j - v_j Gamma_i) zeta_sigma(r)    */
/* with nu_ij = nu + (nu_t,i + nu_t,j)/2 carrying the Vreman eddy viscosity.  */
/* The i == j term is zero by construction.                                   */
/* ------------------------------------------------------------------------- */
static void pse_one(const double* pos, const double* str, const double* nu_t, int64_t n, int64_t i, double sigma,
                    double nu, double* p)
{
    const double norm = 1.0 / pow(2.0 * PI * sigma * sigma, 1.5);
    double acc[3] = {0, 0, 0};
    const double vi = pos[4 * i + 3];
    for (int64_t j = 0; j < n; ++j) {
        double r[3] = {pos[4 * i] - pos[4 * j], pos[4 * i + 1] - pos[4 * j + 1], pos[4 * i + 2] - pos[4 * j + 2]};
        const double rho2 = dot(r, r) / (sigma * sigma);
        const double zeta = norm * exp(-0.5 * rho2);
        const double nij = nu + 0.5 * ((nu_t ? nu_t[i] : 0.0) + (nu_t ? nu_t[j] : 0.0));
        const double vj = pos[4 * j + 3];
        for (int a = 0; a < 3; ++a) acc[a] += nij * (vi * str[4 * j + a] - vj * str[4 * i + a]) * zeta;
    }
    for (int a = 0; a < 3; ++a) p[a] = 2.0 / (sigma * sigma) * acc[a];
}

void orc_pse(const double* pos, const double* str, const double* nu_t, int64_t n, double sigma, double nu,
             double* p)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) pse_one(pos, str, nu_t, n, i, sigma, nu, &p[3 * i]);
}

/* The same sum at the k particles idx[0..k) only, each over all n particles
 * (p[k][3]); for sampled checks of large particle sets. */
void orc_pse_at(const double* pos, const double* str, const double* nu_t, int64_t n, const int64_t* idx, int64_t k,
                double sigma, double nu, double* p)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < k; ++t) pse_one(pos, str, nu_t, n, idx[t], sigma, nu, &p[3 * t]);
}

/* ------------------------------------------------------------------------- */
/* Right-hand side of Eq. 4-5 for every particle:                             */
/*   dx/dt = u + U_inf,   dGamma/dt = stretching + PSE diffusion,              */
/* where u and its gradient come from all other particles plus the segments.  */
/* flags bit 0: classic stretching (J Gamma) instead of the transposed form.  */
/* ------------------------------------------------------------------------- */
void orc_rhs(const double* pos, const double* str, int64_t n, const double* sa, const double* sb, int64_t m,
             double sigma, double nu, double c_v, double seg_core, int vn, const double* u_inf, int flags,
             double* dxdt, double* dGdt, double* nu_t_out)
{
    double* u = (double*)calloc((size_t)(3 * n), sizeof(double));
    double* J = (double*)calloc((size_t)(9 * n), sizeof(double));
    double* us = (double*)calloc((size_t)(3 * n), sizeof(double));
    double* Js = (double*)calloc((size_t)(9 * n), sizeof(double));
    double* nut = (double*)calloc((size_t)n, sizeof(double));
    double* s = (double*)calloc((size_t)(3 * n), sizeof(double));
    double* p = (double*)calloc((size_t)(3 * n), sizeof(double));
    orc_p2p(pos, str, n, pos, n, sigma, u, J);
    if (m > 0) {
        orc_segments(sa, sb, m, pos, n, seg_core, vn, us, Js);
        for (int64_t k = 0; k < 3 * n; ++k) u[k] += us[k];
        for (int64_t k = 0; k < 9 * n; ++k) J[k] += Js[k];
    }
    orc_vreman(J, n, sigma, c_v, nut);
    orc_stretch(J, str, n, flags & 1, s);
    orc_pse(pos, str, nut, n, sigma, nu, p);
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            dxdt[3 * i + a] = u[3 * i + a] + u_inf[a];
            dGdt[3 * i + a] = s[3 * i + a] + p[3 * i + a];
        }
    if (nu_t_out)
        for (int64_t i = 0; i < n; ++i) nu_t_out[i] = nut[i];
    free(u);
    free(J);
    free(us);
    free(Js);
    free(nut);
    free(s);
    free(p);
}

/* ------------------------------------------------------------------------- */
/* One step of the low-storage third-order Runge-Kutta scheme of Williamson   */
/* (1980), which the paper uses for both Eq. 4 and Eq. 5:                     */
/*   for k = 1..3:  q <- A_k q + dt f(y);  y <- y + B_k q                      */
/*   A = (0, -5/9, -153/128),  B = (1/3, 15/16, 8/15).                         */
/* y = (x, Gamma) in double; segments stay frozen during the step.  When     */
/* cast_f32 != 0 each stage evaluates f on the state rounded to float, the    */
/* precision in which the pair sums read their inputs.                        */
/* x[n][3], G[n][3], vol[n].                                                  */
/* ------------------------------------------------------------------------- */
void orc_step(double* x, double* G, const double* vol, int64_t n, const double* sa, const double* sb, int64_t m,
              double sigma, double nu, double c_v, double seg_core, int vn, const double* u_inf, int flags,
              double dt, int cast_f32)
{
    static const double Ak[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
    static const double Bk[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
    double* qx = (double*)calloc((size_t)(3 * n), sizeof(double));
    double* qG = (double*)calloc((size_t)(3 * n), sizeof(double));
    double* pos = (double*)calloc((size_t)(4 * n), sizeof(double));
    double* str = (double*)calloc((size_t)(4 * n), sizeof(double));
    double* fx = (double*)calloc((size_t)(3 * n), sizeof(double));
    double* fG = (double*)calloc((size_t)(3 * n), sizeof(double));
    for (int k = 0; k < 3; ++k) {
        for (int64_t i = 0; i < n; ++i) {
            for (int a = 0; a < 3; ++a) {
                pos[4 * i + a] = cast_f32 ? (double)(float)x[3 * i + a] : x[3 * i + a];
                str[4 * i + a] = cast_f32 ? (double)(float)G[3 * i + a] : G[3 * i + a];
            }
            pos[4 * i + 3] = vol[i];
            str[4 * i + 3] = 0.0;
        }
        orc_rhs(pos, str, n, sa, sb, m, sigma, nu, c_v, seg_core, vn, u_inf, flags, fx, fG, NULL);
        for (int64_t i = 0; i < 3 * n; ++i) {
            qx[i] = Ak[k] * qx[i] + dt * fx[i];
            qG[i] = Ak[k] * qG[i] + dt * fG[i];
            x[i] += Bk[k] * qx[i];
            G[i] += Bk[k] * qG[i];
        }
    }
    free(qx);
    free(qG);
    free(pos);
    free(str);
    free(fx);
    free(fG);
}

/* ------------------------------------------------------------------------- */
/* Influence matrix of the blade vortex rings (Neumann condition at the      */
/* collocation points): A_kl = u(ring l, unit circulation)(y_k) . n_k, a ring */
/* being the four segments c0->c1->c2->c3->c0 of its corners.                 */
/* rings[n][4][4] (corner xyz + pad), colloc[n][4], normal[n][4], A[n][n].    */
/* The right-hand side b_k = -(v_k + w_k) . n_k with v the kinematic plus     */
/* free-stream velocity and w the velocity induced by everything else.        */
/* ------------------------------------------------------------------------- */
void orc_aic_build(const double* rings, const double* colloc, const double* normal, int64_t n, double rc, int vn,
                   double* A)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < n; ++k) {
        for (int64_t l = 0; l < n; ++l) {
            double tot[3] = {0, 0, 0};
            for (int s = 0; s < 4; ++s) {
                const double* P = &rings[16 * l + 4 * s];
                const double* Q = &rings[16 * l + 4 * ((s + 1) % 4)];
                double us[3];
                segment_uJ(P, Q, 1.0, &colloc[4 * k], rc, vn, us, NULL);
                for (int a = 0; a < 3; ++a) tot[a] += us[a];
            }
            A[n * k + l] = dot(tot, &normal[4 * k]);
        }
    }
}

void orc_aic_rhs(const double* v_rel, const double* w_ind, const double* normal, int64_t n, double* b)
{
    for (int64_t k = 0; k < n; ++k) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += (v_rel[4 * k + a] + (w_ind ? w_ind[3 * k + a] : 0.0)) * normal[4 * k + a];
        b[k] = -s;
    }
}

/* Textbook Gaussian elimination with partial pivoting in double; A[n][n]     */
/* row-major is copied.  Returns 0 on success, -1 if a pivot is exactly 0.    */
int orc_lu_solve(const double* A_in, const double* b, int64_t n, double* x)
{
    double* A = (double*)malloc(sizeof(double) * (size_t)(n * n));
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(A, A_in, sizeof(double) * (size_t)(n * n));
    memcpy(y, b, sizeof(double) * (size_t)n);
    int rc = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t piv = k;
        for (int64_t i = k + 1; i < n; ++i)
            if (fabs(A[n * i + k]) > fabs(A[n * piv + k])) piv = i;
        if (A[n * piv + k] == 0.0) {
            rc = -1;
            break;
        }
        if (piv != k) {
            for (int64_t j = 0; j < n; ++j) {
                const double t = A[n * k + j];
                A[n * k + j] = A[n * piv + j];
                A[n * piv + j] = t;
            }
            const double t = y[k];
            y[k] = y[piv];
            y[piv] = t;
        }
        for (int64_t i = k + 1; i < n; ++i) {
            const double l = A[n * i + k] / A[n * k + k];
            A[n * i + k] = l;
            for (int64_t j = k + 1; j < n; ++j) A[n * i + j] -= l * A[n * k + j];
            y[i] -= l * y[k];
        }
    }
    if (rc == 0) {
        for (int64_t i = n - 1; i >= 0; --i) {
            double s = y[i];
            for (int64_t j = i + 1; j < n; ++j) s -= A[n * i + j] * x[j];
            x[i] = s / A[n * i + i];
        }
    }
    free(A);
    free(y);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Adjoint of the particle -> point velocity.  For u_k = sum_j K (Gamma_j x r) */
/* with r = y_k - x_j and a loss gradient g_k = dL/du_k, the chain rule gives */
/*   dL/dGamma_j = sum_k (du_k/dGamma_j)^T g_k,  du_k/dGamma_j = -K [r x]      */
/*   dL/dx_j     = sum_k (du_k/dx_j)^T g_k,      du_k/dx_j = -M_kj              */
/* where M_kj is the pair's velocity-gradient matrix (the J summand above).   */
/* tgt[nt][4], g[nt][3]; outputs dx[ns][3], dG[ns][3].                         */
/* ------------------------------------------------------------------------- */
void orc_p2p_adjoint(const double* pos, const double* str, int64_t n_src, const double* tgt, int64_t n_tgt,
                     double sigma, const double* g, double* dx, double* dG)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t j = 0; j < n_src; ++j) {
        double ax[3] = {0, 0, 0}, aG[3] = {0, 0, 0};
        const double* G = &str[4 * j];
        for (int64_t k = 0; k < n_tgt; ++k) {
            double r[3] = {tgt[4 * k] - pos[4 * j], tgt[4 * k + 1] - pos[4 * j + 1], tgt[4 * k + 2] - pos[4 * j + 2]};
            const double rr = sqrt(dot(r, r));
            double K, H;
            if (!blob_KH(rr, sigma, &K, &H)) continue;
            const double* gk = &g[3 * k];
            /* (-K [r x])^T g = K (r x g) since [r x]^T = -[r x] */
            double rxg[3];
            cross(r, gk, rxg);
            for (int a = 0; a < 3; ++a) aG[a] += K * rxg[a];
            double c[3];
            cross(G, r, c);
            double M[9];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double t = 0.0;
                    for (int cc = 0; cc < 3; ++cc) t += levi(a, cc, b) * G[cc];
                    M[3 * a + b] = K * t + H * c[a] * r[b];
                }
            for (int b = 0; b < 3; ++b) {
                double t = 0.0;
                for (int a = 0; a < 3; ++a) t += M[3 * a + b] * gk[a];
                ax[b] -= t;
            }
        }
        for (int a = 0; a < 3; ++a) {
            dx[3 * j + a] = ax[a];
            dG[3 * j + a] = aG[a];
        }
    }
}

/* ------------------------------------------------------------------------------
 * Wake panel -> particle conversion (Sec. II.C, Eq. 6-8).
 *
 * An edge is one straight vortex line of the wake lattice, from a to b, owned by the
 * wake panel of circulation gamma (the ring's circulation runs along a -> b).  Its
 * circulation difference (Eq. 7) is gamma - gamma_nb when the panel on the other side
 * of the edge is converted together with it (has_nb), else gamma.  The edge becomes
 * n particles of strength Delta Gamma (b - a) / n (Eq. 6).  A trailed (streamwise)
 * edge gets n = ceil(|b - a| / ds_tip * n_tip) particles (Eq. 8, the adaptive count
 * scaled on the tip edge of length ds_tip that carries n_tip); a shed (spanwise) edge
 * gets n_shed.  A negative n_tip selects the conventional strategy the paper compares
 * against: -n_tip particles on every trailed edge whatever its length.
 *
 * Readings: the paper places the particles along the edge without stating where; they
 * sit at the centres of the n equal pieces, x_k = a + (k + 1/2)/n (b - a).  The count
 * is computed in double precision as ceil((len / ds_tip) * n_tip) with
 * len = sqrt(dx*dx + dy*dy + dz*dz) (no contraction; the library takes the same
 * integer decision in the same precision).  Particles are written edge by edge.
 *
 * Edges a[m][3], b[m][3]; outputs x[cap][3], G[cap][3], counts[m].  Returns the number
 * of particles, -1 (nothing written) if it exceeds cap, or -2 (nothing written) if an
 * edge's count is not a finite number of at most 2^30 (NaN or runaway edge lengths).
 * ------------------------------------------------------------------------------ */
static int64_t wake_count(const double* a, const double* b, int trailed, double ds_tip, int n_tip, int n_shed)
{
    if (!trailed) return n_shed;
    if (n_tip < 0) return -n_tip; /* the conventional strategy: the same count on every trailed edge */
    const double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
    const double len = sqrt(dx * dx + dy * dy + dz * dz);
    const double v = ceil((len / ds_tip) * (double)n_tip);
    if (!(v <= 1073741824.0)) return -1; /* not a finite count of at most 2^30 particles: refused */
    return v < 1.0 ? 1 : (int64_t)v;  /* a zero-length edge still gets one particle (of zero strength) */
}

int64_t orc_wake_convert(const double* a, const double* b, const double* gamma, const double* gamma_nb,
                         const int* has_nb, const int* trailed, int64_t m, double ds_tip, int n_tip, int n_shed,
                         int64_t cap, double* x, double* G, int64_t* counts)
{
    int64_t total = 0;
    for (int64_t i = 0; i < m; ++i) {
        counts[i] = wake_count(&a[3 * i], &b[3 * i], trailed[i], ds_tip, n_tip, n_shed);
        if (counts[i] < 0) return -2; /* an edge whose count is not finite (NaN or huge lengths) */
        total += counts[i];
    }
    if (total > cap) return -1;
    int64_t o = 0;
    for (int64_t i = 0; i < m; ++i) {
        const double* ai = &a[3 * i];
        const double* bi = &b[3 * i];
        const double dG = (has_nb && has_nb[i]) ? gamma[i] - gamma_nb[i] : gamma[i]; /* Eq. 7 */
        const double d[3] = {bi[0] - ai[0], bi[1] - ai[1], bi[2] - ai[2]};
        const int64_t n = counts[i];
        for (int64_t k = 0; k < n; ++k, ++o) {
            const double t = ((double)k + 0.5) / (double)n;
            for (int c = 0; c < 3; ++c) {
                x[3 * o + c] = ai[c] + t * d[c];
                G[3 * o + c] = (dG * d[c]) / (double)n; /* Eq. 6 */
            }
        }
    }
    return total;
}

/* The edges of one wake panel row for its conversion.  The row has S panels between
 * an upstream node line U[0..S] (towards the blade) and a downstream line D[0..S];
 * panel p is the ring U[p] -> U[p+1] -> D[p+1] -> D[p] -> U[p] of circulation
 * gamma[p].  Edges, in this order (3 S + 1 of them):
 *   trailed q = 0..S-1: D[q] -> U[q], owned by panel q, neighbour panel q-1 (q > 0);
 *   trailed S:          U[S] -> D[S], owned by panel S-1, no neighbour;
 *   shed back p:        D[p+1] -> D[p], owned by panel p, no neighbour (the older row
 *                       is converted already);
 *   shed front p:       U[p] -> U[p+1], owned by panel p, no neighbour (the younger row
 *                       stays a panel row and keeps its own ring, so the converted
 *                       line carries this ring's strength alone).
 * U, D [S+1][3]; outputs a, b [3S+1][3], g, gnb [3S+1], has_nb, trailed [3S+1]. */
void orc_wake_row_edges(const double* U, const double* D, const double* gamma, int64_t S, double* a, double* b,
                        double* g, double* gnb, int* has_nb, int* trailed)
{
    int64_t e = 0;
    for (int64_t q = 0; q <= S; ++q, ++e) {
        const int end = q == S;
        const double* from = end ? &U[3 * q] : &D[3 * q];
        const double* to = end ? &D[3 * q] : &U[3 * q];
        memcpy(&a[3 * e], from, 3 * sizeof(double));
        memcpy(&b[3 * e], to, 3 * sizeof(double));
        g[e] = end ? gamma[S - 1] : gamma[q];
        has_nb[e] = (!end && q > 0);
        gnb[e] = has_nb[e] ? gamma[q - 1] : 0.0;
        trailed[e] = 1;
    }
    for (int64_t p = 0; p < S; ++p, ++e) {
        memcpy(&a[3 * e], &D[3 * (p + 1)], 3 * sizeof(double));
        memcpy(&b[3 * e], &D[3 * p], 3 * sizeof(double));
        g[e] = gamma[p], gnb[e] = 0.0, has_nb[e] = 0, trailed[e] = 0;
    }
    for (int64_t p = 0; p < S; ++p, ++e) {
        memcpy(&a[3 * e], &U[3 * p], 3 * sizeof(double));
        memcpy(&b[3 * e], &U[3 * (p + 1)], 3 * sizeof(double));
        g[e] = gamma[p], gnb[e] = 0.0, has_nb[e] = 0, trailed[e] = 0;
    }
}

/* Thread count of the OpenMP loops above (the CPU baseline reports a multi-core and a
 * single-thread figure). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------------
 * Blade loads (Sec. II.A): the steady part by the Kutta-Joukowski theorem on every
 * bound segment (panel side), F_s = rho Gamma_s (V_s x (b_s - a_s)), V_s the air
 * velocity relative to the blade at the segment midpoint,
 *   V_s = u_inf - omega x (mid - hub) + u_ind(mid),
 * and the unsteady part at the centre of every panel (unsteady Bernoulli),
 *   F_p = rho (Gamma_p - Gamma_p,prev) / dt  A_p n_p,
 * A_p the area of the ring's quadrilateral (half the norm of the cross product of its
 * diagonals).  out[0..2] = total force, out[3..5] = total moment about hub.  The
 * caller lists the bound segments: every ring's four sides with the ring's
 * circulation, so that shared sides carry their net circulation, the trailing-edge
 * sides with zero (their net circulation with the row shed at the same step vanishes).
 * seg_a [m][4] (a, Gamma), seg_b [m][4]; u_ind [m][3]; rings [n][4][4] corners;
 * normal [n][4]; gamma, gamma_prev [n] (gamma_prev NULL: no unsteady part).
 * ------------------------------------------------------------------------------ */
void orc_blade_loads(const double* sa, const double* sb, int64_t m, const double* u_ind, const double* omega,
                     const double* hub, const double* u_inf, const double* rings, const double* normal,
                     const double* gamma, const double* gamma_prev, int64_t n, double dt, double rho, double* out)
{
    double F[3] = {0, 0, 0}, M[3] = {0, 0, 0};
    for (int64_t s = 0; s < m; ++s) {
        const double* a = &sa[4 * s];
        const double* b = &sb[4 * s];
        double mid[3], dl[3], rel[3], w[3], V[3], f[3], mom[3];
        for (int c = 0; c < 3; ++c) {
            mid[c] = 0.5 * (a[c] + b[c]);
            dl[c] = b[c] - a[c];
            rel[c] = mid[c] - hub[c];
        }
        cross(omega, rel, w);
        for (int c = 0; c < 3; ++c) V[c] = u_inf[c] - w[c] + u_ind[3 * s + c];
        cross(V, dl, f);
        for (int c = 0; c < 3; ++c) f[c] *= rho * a[3];
        cross(rel, f, mom);
        for (int c = 0; c < 3; ++c) F[c] += f[c], M[c] += mom[c];
    }
    if (gamma_prev) {
        for (int64_t p = 0; p < n; ++p) {
            const double* r = &rings[16 * p];
            double d1[3], d2[3], cr[3], ctr[3], rel[3], f[3], mom[3];
            for (int c = 0; c < 3; ++c) {
                d1[c] = r[8 + c] - r[c];      /* corner 2 - corner 0 */
                d2[c] = r[12 + c] - r[4 + c]; /* corner 3 - corner 1 */
                ctr[c] = 0.25 * (r[c] + r[4 + c] + r[8 + c] + r[12 + c]);
                rel[c] = ctr[c] - hub[c];
            }
            cross(d1, d2, cr);
            const double area = 0.5 * sqrt(dot(cr, cr));
            const double k = rho * (gamma[p] - gamma_prev[p]) / dt * area;
            for (int c = 0; c < 3; ++c) f[c] = k * normal[4 * p + c];
            cross(rel, f, mom);
            for (int c = 0; c < 3; ++c) F[c] += f[c], M[c] += mom[c];
        }
    }
    for (int c = 0; c < 3; ++c) out[c] = F[c], out[3 + c] = M[c];
}
