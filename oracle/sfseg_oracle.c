/*
 * sfseg_oracle.c -- plain FP64 CPU oracle for the SFSeg power iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path.
 *
 * What it computes is the plain definition, written out edge by edge with
 * the adjacency matrix M never factored into convolutions:
 *
 *   sp_i   = s_i^p                                            (Eq. 1, unary)
 *   M_ij   = sp_i sp_j [1 - alpha (f_i - f_j)^2] G_ij          (Eq. 2, Taylor)
 *   G_ij   = g_t(t_i-t_j) g_y(y_i-y_j) g_x(x_i-x_j),  g(d) = exp(-d^2/2sigma^2)
 *            for |dt|<=rt, |dy|<=ry, |dx|<=rx, j inside the volume, i included
 *   y      = M x                                              (Eq. 4)
 *   r_k    = x.y / x.x   (Rayleigh quotient of Eq. 3)
 *   rho_k  = ||y - r_k x|| / ||x||
 *   x^{k+1} = y / ||y||                                       (Eq. 8, Alg. 1)
 *
 * Readings of the paper taken here (each one also listed in the design notes):
 *   - G is the per-axis Gaussian with peak 1, truncated to the stated radii,
 *     not renormalised; the volume border is zero padding (a neighbour
 *     outside the volume does not exist), which keeps M symmetric.
 *   - N(i) of Eq. 4 contains i itself.
 *   - Eq. 7 lacks the leading alpha of Eq. 6; this oracle applies M of Eq. 2.
 *   - Eq. 3 divides by ||x||; read as the Rayleigh quotient (divide by x.x).
 *   - Multiple channels (Eq. 9): the result is the sum over channels c of the
 *     single-channel operator with F_c, i.e.
 *       M_ij = sp_i sp_j G_ij sum_c [1 - alpha (f_ci - f_cj)^2].
 *   - mode 1 uses the exact exponential pairwise term of Eq. 1 instead of
 *     its Taylor form (single channel only), for the approximation study.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC (no -ffast-math: IEEE FP64 order).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* g[d + r] = exp(-d^2 / (2 sigma^2)), d = -r..r  (Gaussian of Eq. 1, peak 1) */
void oracle_taps(int r, double sigma, double *g)
{
    for (int d = -r; d <= r; ++d)
        g[d + r] = exp(-((double)d * (double)d) / (2.0 * sigma * sigma));
}

/* sp_i = s_i^p (unary term of Eq. 1/Eq. 2).  pow(0, 0) = 1, pow(0, p>0) = 0. */
void oracle_unary(const double *s, int64_t n, double p, double *sp)
{
    for (int64_t i = 0; i < n; ++i)
        sp[i] = pow(s[i], p);
}

/* The pairwise factor of M_ij without the unary terms and without G. */
static double pair_term(int mode, int nc, int64_t n, double alpha,
                        const double *f, int64_t i, int64_t j)
{
    if (mode == 1) {                          /* Eq. 1: exp(-alpha (fi-fj)^2) */
        double d = f[i] - f[j];
        return exp(-alpha * d * d);
    }
    double acc = 0.0;                         /* Eq. 2 (summed over Eq. 9 channels) */
    for (int c = 0; c < nc; ++c) {
        double d = f[(int64_t)c * n + i] - f[(int64_t)c * n + j];
        acc += 1.0 - alpha * d * d;
    }
    return acc;
}

/* y_i = sum_{j in N(i)} M_ij x_j for one voxel i = (t, yy, xx). */
static double apply_one(int64_t nf, int64_t h, int64_t w, int rt, int ry, int rx,
                        const double *gt, const double *gy, const double *gx,
                        double alpha, int mode, int nc, const double *sp,
                        const double *f, const double *x,
                        int64_t t, int64_t yy, int64_t xx)
{
    const int64_t n = nf * h * w;
    const int64_t i = (t * h + yy) * w + xx;
    double acc = 0.0;
    for (int dt = -rt; dt <= rt; ++dt) {
        int64_t tj = t + dt;
        if (tj < 0 || tj >= nf) continue;
        for (int dy = -ry; dy <= ry; ++dy) {
            int64_t yj = yy + dy;
            if (yj < 0 || yj >= h) continue;
            for (int dx = -rx; dx <= rx; ++dx) {
                int64_t xj = xx + dx;
                if (xj < 0 || xj >= w) continue;
                int64_t j = (tj * h + yj) * w + xj;
                double gij = gt[dt + rt] * gy[dy + ry] * gx[dx + rx];
                double mij = sp[i] * sp[j] * pair_term(mode, nc, n, alpha, f, i, j) * gij;
                acc += mij * x[j];
            }
        }
    }
    return acc;
}

/* y = M x over the whole volume (Eq. 4 before normalisation). */
void oracle_apply(int64_t nf, int64_t h, int64_t w, int rt, int ry, int rx,
                  const double *gt, const double *gy, const double *gx,
                  double alpha, int mode, int nc, const double *sp,
                  const double *f, const double *x, double *y)
{
    int64_t rows = nf * h;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t row = 0; row < rows; ++row) {
        int64_t t = row / h, yy = row % h;
        for (int64_t xx = 0; xx < w; ++xx)
            y[row * w + xx] = apply_one(nf, h, w, rt, ry, rx, gt, gy, gx, alpha,
                                        mode, nc, sp, f, x, t, yy, xx);
    }
}

/* (M x)_i at the listed flat indices only. */
void oracle_apply_at(int64_t nf, int64_t h, int64_t w, int rt, int ry, int rx,
                     const double *gt, const double *gy, const double *gx,
                     double alpha, int mode, int nc, const double *sp,
                     const double *f, const double *x, const int64_t *idx,
                     int64_t m, double *y_at)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = idx[k];
        int64_t t = i / (h * w), rem = i % (h * w);
        y_at[k] = apply_one(nf, h, w, rt, ry, rx, gt, gy, gx, alpha, mode, nc,
                            sp, f, x, t, rem / w, rem % w);
    }
}

static double dot(const double *a, const double *b, int64_t n)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/*
 * Power iteration (Eq. 4 + Eq. 8, Alg. 1 without binarisation): x^0 = x0,
 * K steps.  Writes x^K, and per step k the Rayleigh quotient r_k, the
 * residual rho_k and ||y_k|| (nullable outputs).  If keep != NULL it receives
 * the K+1 iterates x^0..x^K (row k at keep + k*n), for the adjoint.
 * Returns 0, or 1 if some ||y_k|| = 0 (x then holds the last valid iterate
 * and k_done the number of completed steps).
 */
int oracle_power(int64_t nf, int64_t h, int64_t w, int rt, int ry, int rx,
                 const double *gt, const double *gy, const double *gx,
                 double alpha, int mode, int nc, const double *sp,
                 const double *f, const double *x0, int K, double *x_out,
                 double *rayleigh, double *residual, double *norms,
                 double *keep, int *k_done)
{
    const int64_t n = nf * h * w;
    double *x = (double *)malloc(sizeof(double) * n);
    double *y = (double *)malloc(sizeof(double) * n);
    if (!x || !y) { free(x); free(y); return 2; }
    memcpy(x, x0, sizeof(double) * n);
    if (keep) memcpy(keep, x, sizeof(double) * n);
    int status = 0, k;
    for (k = 0; k < K; ++k) {
        oracle_apply(nf, h, w, rt, ry, rx, gt, gy, gx, alpha, mode, nc, sp, f, x, y);
        double xx = dot(x, x, n), xy = dot(x, y, n), yy = dot(y, y, n);
        double r = xy / xx;
        double rr = 0.0;                       /* ||y - r x||^2, two-pass */
        for (int64_t i = 0; i < n; ++i) { double d = y[i] - r * x[i]; rr += d * d; }
        if (rayleigh) rayleigh[k] = r;
        if (residual) residual[k] = sqrt(rr) / sqrt(xx);
        double ny = sqrt(yy);
        if (norms) norms[k] = ny;
        if (!(ny > 0.0)) { status = 1; break; }
        for (int64_t i = 0; i < n; ++i) x[i] = y[i] / ny;
        if (keep) memcpy(keep + (int64_t)(k + 1) * n, x, sizeof(double) * n);
    }
    if (k_done) *k_done = k;
    memcpy(x_out, x, sizeof(double) * n);
    free(x); free(y);
    return status;
}

/*
 * Reverse-mode derivative of the K-step normalised power iteration
 * (single channel, Taylor form), for a loss L with dL/dx^K = gK.
 *
 * Forward: y_k = M x^k, x^{k+1} = y_k / ||y_k||.  Backward, k = K-1..0:
 *   u_k   = (g_{k+1} - x^{k+1} (x^{k+1} . g_{k+1})) / ||y_k||   (d/dy_k)
 *   g_k   = M^T u_k                                           (d/dx^k)
 *   dL/dM_ij += u_k,i x^k_j, pushed through M_ij's definition:
 *     dM_ij/dsp_i = sp_j K_ij,  dM_ij/dsp_j = sp_i K_ij,  K_ij = [1-a(fi-fj)^2] G_ij
 *     dM_ij/df_i  = -2a (f_i - f_j) sp_i sp_j G_ij = -dM_ij/df_j
 * xs holds x^0..x^K (from oracle_power's keep), norms the ||y_k||.
 * Outputs: g_x0 = dL/dx^0, g_sp = dL/dsp, g_f = dL/df (all length n).
 */
void oracle_adjoint(int64_t nf, int64_t h, int64_t w, int rt, int ry, int rx,
                    const double *gt, const double *gy, const double *gx,
                    double alpha, const double *sp, const double *f,
                    const double *xs, const double *norms, int K,
                    const double *gK, double *g_x0, double *g_sp, double *g_f)
{
    const int64_t n = nf * h * w;
    double *g = (double *)malloc(sizeof(double) * n);
    double *u = (double *)malloc(sizeof(double) * n);
    memcpy(g, gK, sizeof(double) * n);
    memset(g_sp, 0, sizeof(double) * n);
    memset(g_f, 0, sizeof(double) * n);
    const int64_t rows = nf * h;
    for (int k = K - 1; k >= 0; --k) {
        const double *xk = xs + (int64_t)k * n;
        const double *xk1 = xs + (int64_t)(k + 1) * n;
        double c = dot(xk1, g, n);
        for (int64_t i = 0; i < n; ++i) u[i] = (g[i] - xk1[i] * c) / norms[k];
        /* gather per voxel m over its box; M_ij = M_ji so both edge
           directions (m,j) and (j,m) are visited from m. */
#pragma omp parallel for schedule(dynamic, 4)
        for (int64_t row = 0; row < rows; ++row) {
            int64_t t = row / h, yy = row % h;
            for (int64_t xx = 0; xx < w; ++xx) {
                int64_t m = row * w + xx;
                double gm = 0.0, dsp = 0.0, df = 0.0;
                for (int dt = -rt; dt <= rt; ++dt) {
                    int64_t tj = t + dt;
                    if (tj < 0 || tj >= nf) continue;
                    for (int dy = -ry; dy <= ry; ++dy) {
                        int64_t yj = yy + dy;
                        if (yj < 0 || yj >= h) continue;
                        for (int dx = -rx; dx <= rx; ++dx) {
                            int64_t xj = xx + dx;
                            if (xj < 0 || xj >= w) continue;
                            int64_t j = (tj * h + yj) * w + xj;
                            double G = gt[dt + rt] * gy[dy + ry] * gx[dx + rx];
                            double d = f[m] - f[j];
                            double Kmj = (1.0 - alpha * d * d) * G;
                            double Mjm = sp[j] * sp[m] * Kmj;   /* M_jm */
                            gm += Mjm * u[j];                   /* (M^T u)_m */
                            /* edge (m,j): dL/dM_mj = u_m x_j ; edge (j,m): u_j x_m */
                            dsp += u[m] * xk[j] * sp[j] * Kmj   /* d/dsp_m via (m,j) */
                                 + u[j] * xk[m] * sp[j] * Kmj;  /* d/dsp_m via (j,m) */
                            double dMdfm = -2.0 * alpha * d * sp[m] * sp[j] * G;
                            df += (u[m] * xk[j] + u[j] * xk[m]) * dMdfm;
                        }
                    }
                }
                g_sp[m] += dsp;
                g_f[m] += df;
                g_x0[m] = gm;          /* new g, copied into g after the sweep */
            }
        }
        memcpy(g, g_x0, sizeof(double) * n);
    }
    free(g); free(u);
}
