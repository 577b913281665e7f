/*
 * FP64 CPU oracle for the SPIIR hot path.  TEST INFRASTRUCTURE ONLY: this file is
 * compiled and called by the tests, by the smoke check and by the benchmark's CPU
 * baseline.  The product library never links, loads or calls it, and it shares no
 * code, header, table or constant with the CUDA path.
 *
 * Everything here is the plain definition written out in double precision, loop by
 * loop, so that it can be read against the paper:
 *
 *   oracle_filter_bank      Sec. II.B.1, Eq. (zk), read per filter (the printed
 *                           equation feeds back the summed output; the commented
 *                           closed form u(t) = sum_m b_m a_m^(t - t_m) beside it fixes
 *                           the per-filter reading):
 *                             y_l[k] = a1_l y_l[k-1] + b0_l x[k - d_l]
 *                             z_t[k] = sum_{l in template t} y_l[k]
 *   oracle_coherent         Sec. II.C.1 Eq. (llr_form) with App. A Eqs. (Ax), (svd):
 *                           the maximised network statistic is the squared norm of the
 *                           projection of the delayed SNR vector w onto the column
 *                           space of G_sigma.  Here the projector is built from the
 *                           normal equations, Pi = G (G^T G)^-1 G^T, with no SVD, so it
 *                           is independent of any U table.  Null: Eq. (null_def),
 *                           sum_I |w_I|^2 - rho_C^2.
 *   oracle_impulse_forward  impulse response of the bank with initial states s_l:
 *                           y_l[-1] = s_l, x = unit impulse at k = 0.
 *   oracle_impulse_backward reverse-mode derivative of a real loss of that response
 *                           (adjoint recurrence, see the function comment).
 *   oracle_autocorr         the correlation of a template with itself (Sec. II.C.2):
 *                             R[j] = sum_k conj(u[k]) u[k + j],  A[j] = R[j] / R[0],
 *                             A[-j] = conj(A[j]).
 *   oracle_xi2              Sec. II.C.2 signal-consistency statistic, per sample:
 *                             xi^2[k] = sum_{j=-Nj}^{Nj} |z[k + j] - z[k] A[j]|^2
 *                                       / sum_{j=-Nj}^{Nj} (2 - 2 |A[j]|^2).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

/*
 * Streaming filter bank.  Complex input so that complex exponentials can be fed in
 * directly; real strain passes a zero imaginary part.
 *   x      [n_det][D + n]: D history samples, then the n samples of this call.
 *          Sample k of the call is x[I][D + k]; x[I][D + k - d] for d <= D.
 *   state  [n_det][F] in/out: y_l[-1] on entry, y_l[n-1] on exit.
 *   z      [T][n_det][n] out.
 * Returns 0, or -1 when a delay exceeds the history D.
 */
int oracle_filter_bank(int n_det, int T, const int64_t *off, const cplx *a1, const cplx *b0,
                       const int32_t *d, const cplx *x, int64_t D, int64_t n, cplx *state,
                       cplx *z)
{
    const int64_t F = off[T];
    for (int64_t l = 0; l < F; ++l)
        if (d[l] < 0 || d[l] > D) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < T; ++t) {
        for (int di = 0; di < n_det; ++di) {
            const cplx *xi = x + (int64_t)di * (D + n) + D;
            cplx *zi = z + ((int64_t)t * n_det + di) * n;
            for (int64_t k = 0; k < n; ++k) {
                cplx acc = 0.0;
                for (int64_t l = off[t]; l < off[t + 1]; ++l) {
                    cplx *y = state + (int64_t)di * F + l;
                    *y = a1[l] * (*y) + b0[l] * xi[k - d[l]];
                    acc += *y;
                }
                zi[k] = acc;
            }
        }
    }
    return 0;
}

/*
 * Coherent sky scan by the projector form.
 *   G      [P][n_det][2]   noise-weighted antenna matrix G_sigma per pixel (Eq. svd).
 *   delay  [P][n_det]      integer arrival offset of detector I for pixel p (samples).
 *   z      [T][n_det][pitch] SNR; output sample k reads z_I[H + k + delay[p][I]].
 *   out:   max_stat[T][n], argmax[T][n] (lowest pixel among equal maxima),
 *          null_stat[T][n] = sum_I |w_I|^2 - rho_C^2 at the argmax pixel,
 *          skymap[T][n][P] (may be NULL).
 * A pixel whose G_sigma has sigma_min / sigma_max < 1e-6 is projected onto its
 * dominant direction only (rank 1); the paper does not treat this measure-zero case.
 * Returns 0, or -1 if a read would fall outside [0, pitch).
 */
/*
 * Projector onto the column space of G_sigma for every pixel: Pi = G (G^T G)^-1 G^T from the
 * normal equations (no SVD); rank <= 1 pixels project onto the dominant direction.
 * Pi [P][n_det][n_det] out.
 */
static void build_projectors(int n_det, int P, const double *G, double *Pi)
{
    for (int p = 0; p < P; ++p) {
        const double *g = G + (int64_t)p * n_det * 2;
        double m00 = 0, m01 = 0, m11 = 0; /* G^T G */
        for (int di = 0; di < n_det; ++di) {
            m00 += g[2 * di] * g[2 * di];
            m01 += g[2 * di] * g[2 * di + 1];
            m11 += g[2 * di + 1] * g[2 * di + 1];
        }
        /* eigenvalues of the 2x2 Gram matrix are the squared singular values */
        double tr = m00 + m11, det = m00 * m11 - m01 * m01;
        double disc = sqrt(fmax(0.0, 0.25 * tr * tr - det));
        double l1 = 0.5 * tr + disc, l2 = 0.5 * tr - disc;
        double *pp = Pi + (int64_t)p * n_det * n_det;
        if (l1 > 0 && l2 > 1e-12 * l1) {
            double i00 = m11 / det, i01 = -m01 / det, i11 = m00 / det; /* (G^T G)^-1 */
            for (int di = 0; di < n_det; ++di)
                for (int dj = 0; dj < n_det; ++dj)
                    pp[di * n_det + dj] = g[2 * di] * (i00 * g[2 * dj] + i01 * g[2 * dj + 1]) +
                                        g[2 * di + 1] * (i01 * g[2 * dj] + i11 * g[2 * dj + 1]);
        } else {
            /* rank <= 1: unit vector along the dominant column direction */
            double vx = m01, vy = l1 - m00;
            if (fabs(vx) + fabs(vy) == 0) { vx = (m00 >= m11) ? 1 : 0; vy = 1 - vx; }
            double vn = sqrt(vx * vx + vy * vy);
            vx /= vn; vy /= vn;
            double un = 0;
            double u[8];
            for (int di = 0; di < n_det; ++di) { u[di] = g[2 * di] * vx + g[2 * di + 1] * vy; un += u[di] * u[di]; }
            for (int di = 0; di < n_det; ++di)
                for (int dj = 0; dj < n_det; ++dj) pp[di * n_det + dj] = (un > 0) ? u[di] * u[dj] / un : 0.0;
        }
    }
}

int oracle_coherent(int n_det, int P, const double *G, const int32_t *delay, int T,
                    const cplx *z, int64_t pitch, int64_t H, int64_t n, double *max_stat,
                    int32_t *argmax, double *null_stat, double *skymap)
{
    for (int p = 0; p < P; ++p)
        for (int di = 0; di < n_det; ++di) {
            int dd = delay[(int64_t)p * n_det + di];
            if (H + dd < 0 || H + dd + n > pitch) return -1;
        }
    double *Pi = (double *)malloc(sizeof(double) * (size_t)P * n_det * n_det);
    if (!Pi) return -2;
    build_projectors(n_det, P, G, Pi);
#pragma omp parallel
    {
        cplx *w = (cplx *)malloc(sizeof(cplx) * n_det);
#pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < T; ++t) {
            for (int64_t k = 0; k < n; ++k) {
                double best = -INFINITY, best_null = 0.0;
                int32_t best_p = -1;
                for (int p = 0; p < P; ++p) {
                    double norm2 = 0.0;
                    for (int di = 0; di < n_det; ++di) {
                        w[di] = z[((int64_t)t * n_det + di) * pitch + H + k + delay[(int64_t)p * n_det + di]];
                        norm2 += creal(w[di]) * creal(w[di]) + cimag(w[di]) * cimag(w[di]);
                    }
                    const double *pp = Pi + (int64_t)p * n_det * n_det;
                    double rho2 = 0.0; /* w^H Pi w, Pi real symmetric */
                    for (int di = 0; di < n_det; ++di)
                        for (int dj = 0; dj < n_det; ++dj)
                            rho2 += pp[di * n_det + dj] * creal(conj(w[di]) * w[dj]);
                    if (skymap) skymap[((int64_t)t * n + k) * P + p] = rho2;
                    if (rho2 > best) { best = rho2; best_p = p; best_null = norm2 - rho2; }
                }
                max_stat[(int64_t)t * n + k] = best;
                argmax[(int64_t)t * n + k] = best_p;
                null_stat[(int64_t)t * n + k] = best_null;
            }
        }
        free(w);
    }
    free(Pi);
    return 0;
}

/*
 * Impulse response of a bank with initial states:
 *   y_l[-1] = s_l,  y_l[k] = a1_l y_l[k-1] + b0_l [k == d_l],  u_t[k] = sum_{l in t} y_l[k]
 * for k = 0 .. n-1.  u is [T][n].  If yend is not NULL it receives y_l[n-1].
 */
void oracle_impulse_forward(int T, const int64_t *off, const cplx *a1, const cplx *b0,
                            const int32_t *d, const cplx *s0, int64_t n, cplx *u, cplx *yend)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < T; ++t) {
        cplx *ut = u + (int64_t)t * n;
        for (int64_t k = 0; k < n; ++k) ut[k] = 0.0;
        for (int64_t l = off[t]; l < off[t + 1]; ++l) {
            cplx y = s0[l];
            for (int64_t k = 0; k < n; ++k) {
                y = a1[l] * y + (k == d[l] ? b0[l] : 0.0);
                ut[k] += y;
            }
            if (yend) yend[l] = y;
        }
    }
}

/*
 * Reverse mode of oracle_impulse_forward for a real loss L(u).
 *   g [T][n] holds dL/dRe(u) + i dL/dIm(u) (the PyTorch gradient convention, so that
 *   dL = Re(sum conj(g) du)).
 * The adjoint state of filter l obeys, for k = n-1 down to 0 with lambda[n] = 0,
 *   lambda_l[k] = g_t[k] + conj(a1_l) lambda_l[k+1]
 * and the gradients in the same convention are
 *   grad_a1_l = sum_k lambda_l[k] conj(y_l[k-1])     (y_l[-1] = s_l)
 *   grad_b0_l = sum_k lambda_l[k] x[k - d_l]  = lambda_l[d_l]  (d_l < n, else 0)
 *   grad_s_l  = conj(a1_l) lambda_l[0].
 * The forward states are stored in full (this is the slow, obviously correct form).
 */
int oracle_impulse_backward(int T, const int64_t *off, const cplx *a1, const cplx *b0,
                            const int32_t *d, const cplx *s0, int64_t n, const cplx *g,
                            cplx *ga1, cplx *gb0, cplx *gs0)
{
    int err = 0;
#pragma omp parallel
    {
        cplx *y = (cplx *)malloc(sizeof(cplx) * (size_t)(n + 1));
        if (!y) err = -2;
#pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < T; ++t) {
            if (!y) continue;
            const cplx *gt = g + (int64_t)t * n;
            for (int64_t l = off[t]; l < off[t + 1]; ++l) {
                /* y[k + 1] holds y_l[k]; y[0] = y_l[-1] = s_l */
                y[0] = s0[l];
                for (int64_t k = 0; k < n; ++k) y[k + 1] = a1[l] * y[k] + (k == d[l] ? b0[l] : 0.0);
                cplx lam = 0.0, sa = 0.0, sb = 0.0;
                for (int64_t k = n - 1; k >= 0; --k) {
                    lam = gt[k] + conj(a1[l]) * lam;
                    sa += lam * conj(y[k]);
                    if (k == d[l]) sb = lam;
                }
                ga1[l] = sa;
                gb0[l] = sb;
                gs0[l] = conj(a1[l]) * lam;
            }
        }
        free(y);
    }
    return err;
}

/*
 * Template autocorrelation.  u [T][nr] (a template's response), A [T][2 Nj + 1] out with
 * A[t][Nj + j] the lag-j value for -Nj <= j <= Nj.  Lags beyond the response are zero terms.
 */
void oracle_autocorr(int T, const cplx *u, int64_t nr, int Nj, cplx *A)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < T; ++t) {
        const cplx *ut = u + (int64_t)t * nr;
        cplx *At = A + (int64_t)t * (2 * Nj + 1);
        cplx R0 = 0.0;
        for (int64_t k = 0; k < nr; ++k) R0 += conj(ut[k]) * ut[k];
        for (int j = 0; j <= Nj; ++j) {
            cplx R = 0.0;
            for (int64_t k = 0; k + j < nr; ++k) R += conj(ut[k]) * ut[k + j];
            At[Nj + j] = R / R0;
            At[Nj - j] = conj(R / R0);
        }
    }
}

/*
 * Signal-consistency statistic of every sample of SNR series.
 *   z   [T][n_det][pitch]: entry Nj + k is sample k, so samples -Nj .. n + Nj - 1 are read.
 *   A   [T][2 Nj + 1]: autocorrelation of each template, A[t][Nj + j] = A_t[j].
 *   out [T][n_det][n].
 */
void oracle_xi2(int T, int n_det, const cplx *z, int64_t pitch, const cplx *A, int Nj, int64_t n,
                double *out)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < T; ++t) {
        const cplx *At = A + (int64_t)t * (2 * Nj + 1);
        double den = 0.0;
        for (int j = -Nj; j <= Nj; ++j) den += 2.0 - 2.0 * creal(At[Nj + j] * conj(At[Nj + j]));
        for (int di = 0; di < n_det; ++di) {
            const cplx *zr = z + ((int64_t)t * n_det + di) * pitch + Nj;
            for (int64_t k = 0; k < n; ++k) {
                double num = 0.0;
                for (int j = -Nj; j <= Nj; ++j) {
                    const cplx d = zr[k + j] - zr[k] * At[Nj + j];
                    num += creal(d * conj(d));
                }
                out[((int64_t)t * n_det + di) * n + k] = num / den;
            }
        }
    }
}

/*
 * Coherent statistic at given points instead of on a grid of geocentric times.  Point i names
 * a template t, a reference detector r and the buffer entry e of the reference detector's
 * sample, plus an extra offset per detector (0 for the foreground; the time shifts of a
 * background event).  For every pixel p the delayed vector is
 *     w_I = z[t][I][e + Delta_I(p) - Delta_r(p) + shift_I],
 * i.e. the reference detector is read at its own sample and the others at the times a source
 * in direction p implies; the statistic is w^H Pi_p w (Sec. II.C.1 Eq. (llr_form)).
 *   pts    [n_pts][3] int64: t, r, e;   shifts [n_pts][n_det] int64
 *   out: max_stat, argmax (lowest p among equals), null (sum |w|^2 - rho^2 at the argmax).
 * Returns 0, or -1 if a read falls outside [0, pitch).
 */
int oracle_coherent_points(int n_det, int P, const double *G, const int32_t *delay, const cplx *z,
                           int64_t pitch, int64_t n_pts, const int64_t *pts, const int64_t *shifts,
                           double *max_stat, int32_t *argmax, double *null_stat)
{
    double *Pi = (double *)malloc(sizeof(double) * (size_t)P * n_det * n_det);
    if (!Pi) return -2;
    build_projectors(n_det, P, G, Pi);
    int err = 0;
#pragma omp parallel
    {
        cplx w[8];
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < n_pts; ++i) {
            const int64_t t = pts[3 * i], r = pts[3 * i + 1], e = pts[3 * i + 2];
            double best = -INFINITY, best_null = 0.0;
            int32_t best_p = -1;
            for (int p = 0; p < P; ++p) {
                double norm2 = 0.0;
                for (int di = 0; di < n_det; ++di) {
                    const int64_t x = e + delay[(int64_t)p * n_det + di] - delay[(int64_t)p * n_det + r] +
                                      shifts[i * n_det + di];
                    if (x < 0 || x >= pitch) { err = -1; w[di] = 0.0; continue; }
                    w[di] = z[(t * n_det + di) * pitch + x];
                    norm2 += creal(w[di]) * creal(w[di]) + cimag(w[di]) * cimag(w[di]);
                }
                const double *pp = Pi + (int64_t)p * n_det * n_det;
                double rho2 = 0.0;
                for (int di = 0; di < n_det; ++di)
                    for (int dj = 0; dj < n_det; ++dj) rho2 += pp[di * n_det + dj] * creal(conj(w[di]) * w[dj]);
                if (rho2 > best) { best = rho2; best_p = p; best_null = norm2 - rho2; }
            }
            max_stat[i] = best;
            argmax[i] = best_p;
            null_stat[i] = best_null;
        }
    }
    free(Pi);
    return err;
}
