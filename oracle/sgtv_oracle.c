/*
 * sgtv_oracle.c -- plain FP64 CPU oracle for one ADMM iteration of spectrally
 * grouped TV (SGTV) reconstruction under a Poisson model.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * restatement of the method that the CUDA path is checked against. Only the
 * tests, the package's smoke check and the benchmark's CPU-baseline leg may
 * load it. It shares no code, header, table or constant with the CUDA path.
 *
 * Problem (Sec. II, Eq. 1 and Eq. 2; Sec. III, Eq. 4):
 *   y_i ~ Poisson((A f)_i + r_i),  A >= 0 of size I x J, J = S * Q,
 *   minimise L(f) + beta * R(w . G f)  subject to f >= 0, where
 *   L(f) = sum_i [ybar_i - y_i log ybar_i]  (negative log-likelihood),
 *   R(d) = sum_s sqrt( sum_q sum_p d_{s,q,p}^2 )  (group TV, Eq. 2), or with
 *   per_bin = 1 the isotropic standard TV the paper compares against, whose
 *   sum over q sits outside the square root (Sec. II, after Eq. 2):
 *   R(d) = sum_s sum_q sqrt( sum_p d_{s,q,p}^2 ),
 *   (G_p f)_{s,q} = f_{s,q} - f_{nbr_p(s),q}, the neighbour outside the
 *   domain being a zero ghost (Dirichlet, Sec. III).
 *
 * ADMM / split Bregman (Sec. III, Eqs. 5-7) with penalty rho (the paper's
 * lambda) and scaled dual c:
 *   f^{k+1} = argmin_f L(f) + rho/2 || d^k - w.(G f) - c^k ||^2      (Eq. 5)
 *   d^{k+1} = argmin_d beta R(d) + rho/2 || d - w.(G f^{k+1}) - c^k ||^2 (Eq. 6)
 *   c^{k+1} = c^k + w.(G f^{k+1}) - d^{k+1}                            (Eq. 7)
 * Eq. 5 is solved approximately by one step (n_inner steps, u fixed) of
 * optimisation transfer: the separable EM surrogate of L and De Pierro's
 * convexity split of the quadratic (Sec. III, last paragraph), which makes the
 * update separable and closed-form per hyper-voxel.
 *
 * Conventions (readings where the paper is silent):
 *   j = (x * Nz + z) * Nq + q, q fastest (Sec. II "lexicographical ordering").
 *   Directions: n_dirs = 4 -> p = 0:+x, 1:-x, 2:+z, 3:-z;
 *               n_dirs = 2 -> p = 0:+x, 1:+z (forward differences only).
 *   d and c are direction-major: d[p * J + j].
 *   One weight per direction, w[p].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const int DX4[4] = {+1, -1, 0, 0};
static const int DZ4[4] = {0, 0, +1, -1};
static const int DX2[2] = {+1, 0};
static const int DZ2[2] = {0, +1};

/* Spatial neighbour of hyper-voxel j in direction p, same q; -1 for a ghost. */
static int64_t nbr(int32_t Nx, int32_t Nz, int32_t Nq, int n_dirs, int64_t j, int p)
{
    int64_t s = j / Nq, q = j % Nq;
    int64_t x = s / Nz, z = s % Nz;
    int dx = (n_dirs == 4) ? DX4[p] : DX2[p];
    int dz = (n_dirs == 4) ? DZ4[p] : DZ2[p];
    int64_t xn = x + dx, zn = z + dz;
    if (xn < 0 || xn >= Nx || zn < 0 || zn >= Nz) return -1;
    return (xn * Nz + zn) * Nq + q;
}

/* O1 (Eq. 1): ybar = A f + r (CSR, one row at a time); ratio = y / ybar,
 * with ratio = 0 where y = 0. r has length 1 (scalar) or I. */
void oracle_forward(int64_t I, const int64_t *rowptr, const int32_t *col,
                    const double *val, const double *f, const double *r,
                    int64_t r_len, const double *y, double *ybar, double *ratio)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < I; i++) {
        double acc = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++)
            acc += val[k] * f[col[k]];
        double yb = acc + (r_len == 1 ? r[0] : r[i]);
        ybar[i] = yb;
        if (ratio) ratio[i] = (y[i] == 0.0) ? 0.0 : y[i] / yb;
    }
}

/* O2: out = A^T v (CSC, one column at a time). With v = ratio this is the
 * backprojection e of the EM surrogate; with v = 1 it is the sensitivity s. */
void oracle_backproject(int64_t J, const int64_t *colptr, const int32_t *row,
                        const double *val, const double *v, double *out)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < J; j++) {
        double acc = 0.0;
        for (int64_t k = colptr[j]; k < colptr[j + 1]; k++)
            acc += val[k] * v[row[k]];
        out[j] = acc;
    }
}

/* s_j = sum_i a_ij (column sums, the EM surrogate's linear coefficient). */
void oracle_sensitivity(int64_t J, const int64_t *colptr, const double *val, double *s)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < J; j++) {
        double acc = 0.0;
        for (int64_t k = colptr[j]; k < colptr[j + 1]; k++) acc += val[k];
        s[j] = acc;
    }
}

/* O4-O5: quadratic and linear coefficients of De Pierro's separable majoriser
 * of P(t) = rho/2 * sum_{j,p} (u_{j,p} - w_p (t_j - t_{nbr_p(j)}))^2 at f.
 *
 * Each term with a in-domain neighbour b = nbr_p(a) is split with weights 1/2,
 * 1/2 around f:  w(t_a - t_b) - u = 1/2 (2w t_a - K) + 1/2 (K' - 2w t_b)
 * with K = w(f_a + f_b) + u and K' = w(f_a + f_b) - u; convexity of the square
 * gives the majoriser rho/4 (2w t_a - K)^2 + rho/4 (2w t_b - K')^2, which
 * touches the term at t = f. Expanded, it adds rho w^2 to alpha_a and alpha_b,
 * rho w K to gamma_a and rho w K' to gamma_b (as the t^2 and -t coefficients).
 * A ghost term (f_b = t_b = 0) is already separable: rho/2 (w t_a - u)^2 adds
 * rho w^2 / 2 to alpha_a and rho w u to gamma_a.
 * The separable majoriser is then sum_j [alpha_j t_j^2 - gamma_j t_j] + const. */
void oracle_surrogate_coeffs(int32_t Nx, int32_t Nz, int32_t Nq, int n_dirs,
                             const double *w, double rho, const double *f,
                             const double *u, double *alpha, double *gamma)
{
    int64_t J = (int64_t)Nx * Nz * Nq;
    memset(alpha, 0, sizeof(double) * J);
    memset(gamma, 0, sizeof(double) * J);
    for (int p = 0; p < n_dirs; p++) {
        for (int64_t a = 0; a < J; a++) {
            double wp = w[p];
            double uap = u[(int64_t)p * J + a];
            int64_t b = nbr(Nx, Nz, Nq, n_dirs, a, p);
            if (b >= 0) {
                double K = wp * (f[a] + f[b]) + uap;
                double Kp = wp * (f[a] + f[b]) - uap;
                alpha[a] += rho * wp * wp;
                gamma[a] += rho * wp * K;
                alpha[b] += rho * wp * wp;
                gamma[b] += rho * wp * Kp;
            } else {
                alpha[a] += 0.5 * rho * wp * wp;
                gamma[a] += rho * wp * uap;
            }
        }
    }
}

/* O5: minimiser over t >= 0 of the separable surrogate
 *   phi_j(t) = s_j t - E_j log t + alpha_j t^2 - gamma_j t,  E_j = f_j e_j,
 * i.e. the nonnegative root of 2 alpha t^2 + (s - gamma) t - E = 0:
 *   t = (-B + sqrt(B^2 + 8 alpha E)) / (4 alpha),  B = s - gamma,
 * evaluated as 2E / (B + sqrt(B^2 + 8 alpha E)) when B >= 0 (no cancellation).
 * alpha = 0 (rho = 0) gives the MLEM step E / s (0 where s = 0). */
double oracle_root(double alpha, double B, double E, double s)
{
    if (alpha == 0.0) return (s > 0.0) ? E / s : 0.0;
    double disc = sqrt(B * B + 8.0 * alpha * E);
    if (B >= 0.0) {
        double den = B + disc;
        return (den > 0.0) ? 2.0 * E / den : 0.0;
    }
    return (-B + disc) / (4.0 * alpha);
}

void oracle_f_update(int64_t J, const double *f, const double *e, const double *s,
                     const double *alpha, const double *gamma, double *f_new)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < J; j++) {
        double E = f[j] * e[j];
        double B = s[j] - gamma[j];
        f_new[j] = oracle_root(alpha[j], B, E, s[j]);
    }
}

/* w . G f : out[p * J + j] = w_p (f_j - f_{nbr_p(j)}), ghost = 0. */
void oracle_wgrad(int32_t Nx, int32_t Nz, int32_t Nq, int n_dirs, const double *w,
                  const double *f, double *out)
{
    int64_t J = (int64_t)Nx * Nz * Nq;
    for (int p = 0; p < n_dirs; p++)
        for (int64_t j = 0; j < J; j++) {
            int64_t b = nbr(Nx, Nz, Nq, n_dirs, j, p);
            out[(int64_t)p * J + j] = w[p] * (f[j] - (b >= 0 ? f[b] : 0.0));
        }
}

/* (w . G)^T z : out_j = sum_p w_p z_{j,p} - sum over terms (a, p) with
 * nbr_p(a) = j of w_p z_{a,p}  (the adjoint of oracle_wgrad). */
void oracle_wgrad_adjoint(int32_t Nx, int32_t Nz, int32_t Nq, int n_dirs,
                          const double *w, const double *z, double *out)
{
    int64_t J = (int64_t)Nx * Nz * Nq;
    memset(out, 0, sizeof(double) * J);
    for (int p = 0; p < n_dirs; p++)
        for (int64_t a = 0; a < J; a++) {
            double t = w[p] * z[(int64_t)p * J + a];
            out[a] += t;
            int64_t b = nbr(Nx, Nz, Nq, n_dirs, a, p);
            if (b >= 0) out[b] -= t;
        }
}

/* O6-O7 (Eqs. 6, 7): v = w.(G f) + c; per spatial site s the group norm
 * n_s = || v_{s,.,.} ||_2 over all q and p (the grouping of Eq. 2);
 * d_s = max(1 - tau / n_s, 0) v_s (d_s = 0 when n_s = 0), tau = beta / rho;
 * c = v - d. d and c are overwritten. */
void oracle_shrink_dual(int32_t Nx, int32_t Nz, int32_t Nq, int n_dirs, const double *w,
                        double tau, int per_bin, const double *f, double *d, double *c)
{
    int64_t J = (int64_t)Nx * Nz * Nq;
    int64_t S = (int64_t)Nx * Nz;
    double *v = (double *)malloc(sizeof(double) * J * n_dirs);
    oracle_wgrad(Nx, Nz, Nq, n_dirs, w, f, v);
    for (int64_t k = 0; k < J * n_dirs; k++) v[k] += c[k];
    if (per_bin) {
        /* standard TV: one group per (s, q), over the directions p only */
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < J; j++) {
            double n2 = 0.0;
            for (int p = 0; p < n_dirs; p++) {
                double t = v[(int64_t)p * J + j];
                n2 += t * t;
            }
            double n = sqrt(n2);
            double scale = (n > 0.0) ? 1.0 - tau / n : 0.0;
            if (scale < 0.0) scale = 0.0;
            for (int p = 0; p < n_dirs; p++) {
                int64_t k = (int64_t)p * J + j;
                d[k] = scale * v[k];
                c[k] = v[k] - d[k];
            }
        }
        free(v);
        return;
    }
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < S; s++) {
        double n2 = 0.0;
        for (int p = 0; p < n_dirs; p++)
            for (int64_t q = 0; q < Nq; q++) {
                double t = v[(int64_t)p * J + s * Nq + q];
                n2 += t * t;
            }
        double n = sqrt(n2);
        double scale = (n > 0.0) ? 1.0 - tau / n : 0.0;
        if (scale < 0.0) scale = 0.0;
        for (int p = 0; p < n_dirs; p++)
            for (int64_t q = 0; q < Nq; q++) {
                int64_t k = (int64_t)p * J + s * Nq + q;
                d[k] = scale * v[k];
                c[k] = v[k] - d[k];
            }
    }
    free(v);
}

/* Poisson deviance D = sum_i [ybar_i - y_i + y_i log(y_i / ybar_i)], 0 log 0 = 0:
 * the negative log-likelihood minus its saturated value (so D >= 0). */
double oracle_deviance(int64_t I, const double *ybar, const double *y)
{
    double acc = 0.0;
    for (int64_t i = 0; i < I; i++) {
        double t = ybar[i] - y[i];
        if (y[i] > 0.0) t += y[i] * log(y[i] / ybar[i]);
        acc += t;
    }
    return acc;
}

/* Negative log-likelihood L = sum_i [ybar_i - y_i log ybar_i] (no constant). */
double oracle_nll(int64_t I, const double *ybar, const double *y)
{
    double acc = 0.0;
    for (int64_t i = 0; i < I; i++) {
        acc += ybar[i];
        if (y[i] > 0.0) acc -= y[i] * log(ybar[i]);
    }
    return acc;
}

/* Group TV of Eq. 2 applied to a direction-major field g (g = w.G f or d);
 * per_bin = 1: the standard TV, one square root per (s, q). */
double oracle_group_tv(int32_t Nx, int32_t Nz, int32_t Nq, int n_dirs, int per_bin, const double *g)
{
    int64_t J = (int64_t)Nx * Nz * Nq, S = (int64_t)Nx * Nz;
    double acc = 0.0;
    if (per_bin) {
        for (int64_t j = 0; j < J; j++) {
            double n2 = 0.0;
            for (int p = 0; p < n_dirs; p++) {
                double t = g[(int64_t)p * J + j];
                n2 += t * t;
            }
            acc += sqrt(n2);
        }
        return acc;
    }
    for (int64_t s = 0; s < S; s++) {
        double n2 = 0.0;
        for (int p = 0; p < n_dirs; p++)
            for (int64_t q = 0; q < Nq; q++) {
                double t = g[(int64_t)p * J + s * Nq + q];
                n2 += t * t;
            }
        acc += sqrt(n2);
    }
    return acc;
}

/* O9 (initialisation): f0_j = kappa with
 * kappa = sum_i (y_i - r_i) / sum_j s_j, falling back to sum_i y_i and then 1
 * in the numerator when that is not positive; d0 = w.G f0; c0 = 0. */
void oracle_init(int32_t Nx, int32_t Nz, int32_t Nq, int n_dirs, const double *w,
                 int64_t I, const double *y, const double *r, int64_t r_len,
                 const double *s, double *f, double *d, double *c)
{
    int64_t J = (int64_t)Nx * Nz * Nq;
    double sy = 0.0, syr = 0.0, ss = 0.0;
    for (int64_t i = 0; i < I; i++) {
        sy += y[i];
        syr += y[i] - (r_len == 1 ? r[0] : r[i]);
    }
    for (int64_t j = 0; j < J; j++) ss += s[j];
    double num = (syr > 0.0) ? syr : ((sy > 0.0) ? sy : 1.0);
    double kappa = (ss > 0.0) ? num / ss : 0.0;
    for (int64_t j = 0; j < J; j++) f[j] = kappa;
    oracle_wgrad(Nx, Nz, Nq, n_dirs, w, f, d);
    memset(c, 0, sizeof(double) * J * n_dirs);
}

/* One or more full ADMM iterations (Eqs. 5-7) in the paper's order:
 *   repeat n_inner times with u = d - c fixed:
 *     ybar = A f + r, ratio = y / ybar            (O1)
 *     e = A^T ratio                               (O2)
 *     alpha, gamma from the surrogate at f        (O4)
 *     f = closed-form minimiser                   (O5)
 *   d, c = group shrink and dual update           (O6, O7)
 * s (= A^T 1) is given. f [J], d and c [n_dirs * J] are updated in place. */
void oracle_iterate(int32_t Nx, int32_t Nz, int32_t Nq, int n_dirs, const double *w,
                    int64_t I, const int64_t *rowptr, const int32_t *col, const double *rval,
                    const int64_t *colptr, const int32_t *row, const double *cval,
                    const double *y, const double *r, int64_t r_len, const double *s,
                    double beta, double rho, int n_iter, int n_inner, int per_bin,
                    double *f, double *d, double *c)
{
    int64_t J = (int64_t)Nx * Nz * Nq;
    double *ybar = (double *)malloc(sizeof(double) * I);
    double *ratio = (double *)malloc(sizeof(double) * I);
    double *e = (double *)malloc(sizeof(double) * J);
    double *alpha = (double *)malloc(sizeof(double) * J);
    double *gamma = (double *)malloc(sizeof(double) * J);
    double *u = (double *)malloc(sizeof(double) * J * n_dirs);
    double *fn = (double *)malloc(sizeof(double) * J);
    double tau = (rho > 0.0) ? beta / rho : 0.0;
    for (int it = 0; it < n_iter; it++) {
        for (int64_t k = 0; k < J * n_dirs; k++) u[k] = d[k] - c[k];
        for (int inner = 0; inner < n_inner; inner++) {
            oracle_forward(I, rowptr, col, rval, f, r, r_len, y, ybar, ratio);
            oracle_backproject(J, colptr, row, cval, ratio, e);
            oracle_surrogate_coeffs(Nx, Nz, Nq, n_dirs, w, rho, f, u, alpha, gamma);
            oracle_f_update(J, f, e, s, alpha, gamma, fn);
            memcpy(f, fn, sizeof(double) * J);
        }
        if (rho > 0.0) oracle_shrink_dual(Nx, Nz, Nq, n_dirs, w, tau, per_bin, f, d, c);
    }
    free(ybar); free(ratio); free(e); free(alpha); free(gamma); free(u); free(fn);
}
