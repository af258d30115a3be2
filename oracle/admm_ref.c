/*
 * ORACLE (test infrastructure only; never linked into the library).
 *
 * Plain FP64 ADMM of Algorithm 1 on the consensus form of Eq. OurModel:
 *
 *   global update  (Eq. closed_1): for every global i,
 *       x_i = clip( (sum_{k: g(k)=i} (rho x_k - lam_k) - c_i) / (rho N_i), lb_i, ub_i )
 *     which is the minimiser of the separable 1-D problem stated above it
 *     (the printed fraction lacks the factor rho on the local copies; the
 *     stationarity condition of that 1-D problem gives this form);
 *   local update   (Eq. closed_2): for every subsystem s,
 *       x_s = (1/rho) Abar_s d_s + bbar_s,  d_s = -rho B_s x - lam_s
 *     with Abar_s given as a dense n_s x n_s matrix (row-major);
 *   dual update    (Eq. ADMM-3):  lam_s += rho (B_s x - x_s);
 *   residuals      (Sec. III-C):  pres, dres, eps_prim, eps_dual with every
 *     norm over all local slots stacked (B_s has one 1 per row and at most
 *     one per column, so |B_s^T v| = |v|).
 *
 * Update order global -> local -> dual as in Algorithm 1; residuals use the
 * values after the update of the same iteration.  Loops run in index order,
 * one thread, no FMA contraction (built with -ffp-contract=off).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* hist (optional) receives 5 doubles per iteration: pres, dres, eps_prim/eps_rel
 * (the max of the two norms), eps_dual/eps_rel (|lam|), objective c^T x.
 * Returns the number of iterations run, or -1 if a global variable has no
 * local copy. */
int oracle_admm(int n, const double *c, const double *lb, const double *ub,
                int S, const long *off, const int *gidx,
                const double *abar, const long *aoff, const double *bbar,
                double rho, double eps_rel, double eps_abs_pres,
                int max_iter, int check_every,
                double *xs, double *lam, double *x, double *hist,
                int *converged)
{
    long L = off[S];
    double *sigma = (double *)calloc((size_t)n, sizeof(double));
    int *cnt = (int *)calloc((size_t)n, sizeof(int));
    double *xn = (double *)malloc(sizeof(double) * (size_t)(L > 0 ? L : 1));
    double *d = (double *)malloc(sizeof(double) * (size_t)(L > 0 ? L : 1));
    int t, i, s;
    long k;
    *converged = 0;
    for (k = 0; k < L; k++) cnt[gidx[k]] += 1;
    for (i = 0; i < n; i++) {
        if (cnt[i] == 0) { free(sigma); free(cnt); free(xn); free(d); return -1; }
    }
    for (t = 0; t < max_iter; t++) {
        /* global update, Eq. closed_1 */
        for (i = 0; i < n; i++) sigma[i] = 0.0;
        for (k = 0; k < L; k++) sigma[gidx[k]] += rho * xs[k] - lam[k];
        for (i = 0; i < n; i++) {
            double xh = (sigma[i] - c[i]) / (rho * (double)cnt[i]);
            if (xh < lb[i]) xh = lb[i];
            if (xh > ub[i]) xh = ub[i];
            x[i] = xh;
        }
        /* local update, Eq. closed_2 */
        for (k = 0; k < L; k++) d[k] = -rho * x[gidx[k]] - lam[k];
        for (s = 0; s < S; s++) {
            long o = off[s];
            int ns = (int)(off[s + 1] - off[s]);
            const double *A = abar + aoff[s];
            int r, q;
            for (r = 0; r < ns; r++) {
                double acc = 0.0;
                for (q = 0; q < ns; q++) acc += A[(long)r * ns + q] * d[o + q];
                xn[o + r] = acc / rho + bbar[o + r];
            }
        }
        /* dual update, Eq. ADMM-3, and the residuals of Sec. III-C */
        {
            double p2 = 0.0, d2 = 0.0, bx2 = 0.0, xs2 = 0.0, l2 = 0.0, obj = 0.0;
            double pres, dres, eprim, edual;
            for (k = 0; k < L; k++) {
                double xg = x[gidx[k]];
                double r = xg - xn[k];
                double dx = xn[k] - xs[k];
                lam[k] = lam[k] + rho * r;
                p2 += r * r;
                d2 += dx * dx;
                bx2 += xg * xg;
                xs2 += xn[k] * xn[k];
                l2 += lam[k] * lam[k];
                xs[k] = xn[k];
            }
            for (i = 0; i < n; i++) obj += c[i] * x[i];
            pres = sqrt(p2);
            dres = rho * sqrt(d2);
            eprim = sqrt(bx2) > sqrt(xs2) ? sqrt(bx2) : sqrt(xs2);
            edual = sqrt(l2);
            if (hist) {
                hist[5L * t + 0] = pres;
                hist[5L * t + 1] = dres;
                hist[5L * t + 2] = eprim;
                hist[5L * t + 3] = edual;
                hist[5L * t + 4] = obj;
            }
            if (check_every > 0 && (t + 1) % check_every == 0 &&
                pres <= eps_rel * eprim && dres <= eps_rel * edual && pres <= eps_abs_pres) {
                *converged = 1;
                t++;
                break;
            }
        }
    }
    free(sigma); free(cnt); free(xn); free(d);
    return t;
}
