/*
 * pd_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of what the entropic optimal transport
 * method for persistence diagrams computes (Lacombe, Cuturi & Oudot, NeurIPS
 * 2018, "Large Scale computation of Means and Clusters for Persistence
 * Diagrams using Optimal Transport").  It is the parity oracle for the CUDA
 * library and shares no code with it.  Only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it; the product path
 * never does.
 *
 * What is here, each following the passage named beside it:
 *   or_rasterize      -- Sec. 3 "Discretization": a_ij = number of points in
 *                        grid cell (i,j); supplementary "Error control due to
 *                        discretization" snaps (x,y) to (floor(xd)/d,
 *                        floor(yd)/d).
 *   or_cost           -- Prop. 1 block cost matrix with the Delta row/column
 *                        and the grid cost of Sec. 3 "Convolutions"
 *                        (squared Euclidean, p = 2, physical units on [0,1]^2);
 *                        or_cost_p: the same for ||.||_p^p.
 *   or_sinkhorn_w     -- Eq. (SinkhornMap) iterated in the log domain on the
 *                        explicit cost matrix (no separability is used), the
 *                        marginal error dist(P, Pi(a,b)) of Eq. (Altschuler
 *                        bounds) and the transport cost <P, C> of
 *                        Sec. 2 (Sinkhorn divergence).  Zero-mass cells are
 *                        skipped in the sums, which is exact: their weight
 *                        in every sum is exp(-inf) = 0.
 *   or_sinkhorn_pd    -- Alg. 1 for one pair: rasterised histograms augmented
 *                        as a = (hist_A, |B|), b = (hist_B, |A|) (Prop. 1).
 *   or_barycenter     -- Alg. 2 (smoothed barycenter) with the gradient of
 *                        Prop. (gradient of E^gamma) and the multiplicative
 *                        update; or_barycenter_e adds the barycenter
 *                        experiment's stop |E_{t+1}/E_t - 1| < tol (Sec. 5).
 *   or_kmeans         -- Sec. 5 k-means: assignment by Alg. 1 cost, centroid
 *                        update by Alg. 2.
 *   or_sharpen        -- entropic sharpening of a measure (Solomon et al., the
 *                        extension the paper names for smeared barycenters);
 *                        or_barycenter_s applies it after every Alg. 2 step.
 *   or_round_bound    -- the rounding algorithm of the supplementary (Altschuler
 *                        et al.) applied to the plan P(f, g), written out on the
 *                        explicit dense matrices, and the transport cost of the
 *                        rounded plan R, <R, C> (the upper bound of Prop. 3).
 *   or_ctransform_bound -- the lower bound m_t of Sec. 3 "Upper and Lower
 *                        Bounds" from the C- and C^T-transforms of alpha =
 *                        gamma log u, by plain minimisation over the supports.
 *
 * Conventions (shared with the CUDA library by specification only):
 *   - Grid cell (i,j): i = birth index (row), j = death index (column), both in
 *     [0,d).  Flattened index x = i*d + j; index d*d is the Delta bin.
 *   - The plan is parametrised as P_xy = a_x b_y exp((f_x + g_y - C_xy)/gamma),
 *     i.e. u = a*exp(f/gamma), v = b*exp(g/gamma) in the notation of
 *     Eq. (SinkhornTransportPlan).
 *   - One iteration t: f-update (u = a / Kv), then the marginal error err_t of
 *     the plan (u_t, v_{t-1}) on the column side, then the g-update
 *     (v = b / K^T u).  The loop stops after iteration t if
 *     err_t / (total mass) <= tol or t == max_iter.  Cost and marginals are
 *     those of (u_t, v_t).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------- */
/* Compensated (Neumaier) summation.                                      */
typedef struct { double s, c; } or_ksum;
static void ks_add(or_ksum* k, double x) {
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
    else k->c += (x - t) + k->s;
    k->s = t;
}
static double ks_val(const or_ksum* k) { return k->s + k->c; }

/* ---------------------------------------------------------------------- */
/* Sec. 3 "Discretization" and supplementary snapping: the cell of a point
 * (birth, death) is (floor(birth*d), floor(death*d)), clamped to d-1 so that
 * the closed edge at 1 belongs to the last cell.  Returns 0, or -1 if an
 * input is not a finite point of [0,1]^2 with birth <= death.              */
int or_rasterize(const double* birth, const double* death, const int64_t* offsets,
                 int B, int d, uint32_t* hist, uint32_t* mass) {
    if (d < 2 || B < 0) return -1;
    memset(hist, 0, sizeof(uint32_t) * (size_t)B * d * d);
    for (int b = 0; b < B; ++b) {
        uint32_t n = 0;
        for (int64_t p = offsets[b]; p < offsets[b + 1]; ++p) {
            double s = birth[p], t = death[p];
            if (!(s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0 && s <= t)) return -1;
            long i = (long)floor(s * (double)d), j = (long)floor(t * (double)d);
            if (i > d - 1) i = d - 1;
            if (j > d - 1) j = d - 1;
            hist[(size_t)b * d * d + (size_t)i * d + j] += 1u;
            ++n;
        }
        mass[b] = n;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Prop. 1 block cost with p = 2 on the grid of Sec. 3, in physical units
 * (cell (i,j) represented by (i/d, j/d)):
 *   grid-grid:  ((i-k)^2 + (j-l)^2) / d^2          (squared Euclidean)
 *   grid-Delta: squared distance of (i/d, j/d) to its orthogonal projection
 *               on the diagonal = (j-i)^2 / (2 d^2)
 *   Delta-Delta: 0.                                                         */
double or_cost(int d, int x, int y) {
    const int D = d * d;
    if (x == D && y == D) return 0.0;
    if (x == D || y == D) {
        int z = (x == D) ? y : x;
        double i = z / d, j = z % d;
        return (j - i) * (j - i) / (2.0 * d * d);
    }
    double i = x / d, j = x % d, k = y / d, l = y % d;
    return ((i - k) * (i - k) + (j - l) * (j - l)) / ((double)d * d);
}

/* The same block cost for a ground cost ||.||_p^p (p >= 1), separable on the
 * grid: |i-k|^p / d^p + |j-l|^p / d^p; a grid cell to the diagonal bin costs
 * ||x - pi_Delta(x)||_p^p with pi_Delta the orthogonal projection, i.e.
 * 2 |(j-i) / (2d)|^p; Delta-Delta costs 0.  p = 2 is or_cost itself. */
double or_cost_p(int d, double p, int x, int y) {
    if (p == 2.0) return or_cost(d, x, y);
    const int D = d * d;
    if (x == D && y == D) return 0.0;
    if (x == D || y == D) {
        int z = (x == D) ? y : x;
        double i = z / d, j = z % d;
        return 2.0 * pow(fabs(j - i) / (2.0 * d), p);
    }
    double i = x / d, j = x % d, k = y / d, l = y % d;
    return pow(fabs(i - k) / d, p) + pow(fabs(j - l) / d, p);
}

/* log-sum-exp of n values (two passes: max, then sum). */
static double lse(const double* v, int n) {
    double m = -INFINITY;
    for (int i = 0; i < n; ++i) if (v[i] > m) m = v[i];
    if (m == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += exp(v[i] - m);
    return m + log(s);
}

/* ---------------------------------------------------------------------- */
/* Entropic OT between two nonnegative weight vectors a, b of length n = d*d+1
 * (last entry = Delta bin) with the cost of or_cost, by Sinkhorn iterations
 * of Eq. (SinkhornMap) written in the log domain:
 *   f_x = -gamma * LSE_y [ log b_y + (g_y - C_xy)/gamma ]   (u = a / K v)
 *   g_y = -gamma * LSE_x [ log a_x + (f_x - C_xy)/gamma ]   (v = b / K^T u)
 * Marginal error (Eq. Altschuler bounds): err_t = sum_y |sum_x P_xy - b_y|
 * with P of (f_t, g_{t-1}); the row side is exact after the f-update.
 * Inputs g_init (length n, or NULL for g = 0, i.e. v_0 = b).
 * Outputs (any may be NULL): cost = <P, C>; f, g on all n entries (zero-mass
 * entries get the same formula, a soft c-transform, finite); rmarg, cmarg the
 * two marginals of P; iters; err (relative to the total mass).
 * Returns 0, or -1 on bad input (negative weight, unequal total mass).     */
int or_sinkhorn_wp(int d, double pw, double gamma, const double* a, const double* b,
                   int max_iter, double tol, const double* g_init,
                   double* cost, double* f_out, double* g_out,
                   double* rmarg, double* cmarg, int* iters, double* err_out) {
    const int n = d * d + 1;
    double ma = 0, mb = 0;
    for (int x = 0; x < n; ++x) {
        if (!(a[x] >= 0) || !(b[x] >= 0)) return -1;
        ma += a[x]; mb += b[x];
    }
    if (fabs(ma - mb) > 1e-9 * (ma > 1 ? ma : 1)) return -1;
    const double total = ma;
    int na = 0, nb = 0;
    int* sa = (int*)malloc(sizeof(int) * n);
    int* sb = (int*)malloc(sizeof(int) * n);
    for (int x = 0; x < n; ++x) { if (a[x] > 0) sa[na++] = x; if (b[x] > 0) sb[nb++] = x; }
    double* C = (double*)malloc(sizeof(double) * (size_t)na * (nb > 0 ? nb : 1));
    for (int p = 0; p < na; ++p)
        for (int q = 0; q < nb; ++q) C[(size_t)p * nb + q] = or_cost_p(d, pw, sa[p], sb[q]);
    double* la = (double*)malloc(sizeof(double) * (na + 1));
    double* lb = (double*)malloc(sizeof(double) * (nb + 1));
    for (int p = 0; p < na; ++p) la[p] = log(a[sa[p]]);
    for (int q = 0; q < nb; ++q) lb[q] = log(b[sb[q]]);
    double* f = (double*)calloc(na + 1, sizeof(double));
    double* g = (double*)calloc(nb + 1, sizeof(double));
    if (g_init) for (int q = 0; q < nb; ++q) g[q] = g_init[sb[q]];
    int big = na > nb ? na : nb;
    double* tmp = (double*)malloc(sizeof(double) * (big + 1));
    double err = INFINITY;
    int t = 0;
    if (na > 0 && nb > 0) {
        for (t = 1; t <= max_iter; ++t) {
            for (int p = 0; p < na; ++p) {
                for (int q = 0; q < nb; ++q) tmp[q] = lb[q] + (g[q] - C[(size_t)p * nb + q]) / gamma;
                f[p] = -gamma * lse(tmp, nb);
            }
            or_ksum e = {0, 0};
            for (int q = 0; q < nb; ++q) {
                for (int p = 0; p < na; ++p) tmp[p] = la[p] + (f[p] - C[(size_t)p * nb + q]) / gamma;
                double colsum = exp(lb[q] + g[q] / gamma + lse(tmp, na));
                ks_add(&e, fabs(colsum - b[sb[q]]));
                g[q] = -gamma * lse(tmp, na);
            }
            err = ks_val(&e) / total;
            if (err <= tol) break;
        }
        if (t > max_iter) t = max_iter;
    } else {
        err = 0.0;
    }
    /* cost and marginals of P(f_t, g_t) */
    or_ksum ck = {0, 0};
    if (rmarg) memset(rmarg, 0, sizeof(double) * n);
    if (cmarg) memset(cmarg, 0, sizeof(double) * n);
    for (int p = 0; p < na; ++p) {
        or_ksum rk = {0, 0};
        for (int q = 0; q < nb; ++q) {
            double c = C[(size_t)p * nb + q];
            double P = exp(la[p] + lb[q] + (f[p] + g[q] - c) / gamma);
            ks_add(&ck, P * c);
            ks_add(&rk, P);
            if (cmarg) cmarg[sb[q]] += P;
        }
        if (rmarg) rmarg[sa[p]] = ks_val(&rk);
    }
    if (cost) *cost = ks_val(&ck);
    /* potentials on every entry: the update formulas evaluated everywhere */
    if (f_out) {
        for (int x = 0; x < n; ++x) {
            for (int q = 0; q < nb; ++q) tmp[q] = lb[q] + (g[q] - or_cost_p(d, pw, x, sb[q])) / gamma;
            f_out[x] = nb > 0 ? -gamma * lse(tmp, nb) : 0.0;
        }
        for (int p = 0; p < na; ++p) f_out[sa[p]] = f[p];
    }
    if (g_out) {
        for (int y = 0; y < n; ++y) {
            for (int p = 0; p < na; ++p) tmp[p] = la[p] + (f[p] - or_cost_p(d, pw, sa[p], y)) / gamma;
            g_out[y] = na > 0 ? -gamma * lse(tmp, na) : 0.0;
        }
        for (int q = 0; q < nb; ++q) g_out[sb[q]] = g[q];
    }
    if (iters) *iters = t;
    if (err_out) *err_out = err;
    free(sa); free(sb); free(C); free(la); free(lb); free(f); free(g); free(tmp);
    return 0;
}

/* Eq. (SinkhornMap) with the p = 2 cost (see or_sinkhorn_wp). */
int or_sinkhorn_w(int d, double gamma, const double* a, const double* b,
                  int max_iter, double tol, const double* g_init,
                  double* cost, double* f_out, double* g_out,
                  double* rmarg, double* cmarg, int* iters, double* err_out) {
    return or_sinkhorn_wp(d, 2.0, gamma, a, b, max_iter, tol, g_init, cost, f_out, g_out, rmarg, cmarg, iters, err_out);
}

/* Prop. 1 augmentation: a = (hist_A, |B|), b = (hist_B, |A|). */
static void augment(int d, const uint32_t* hA, const uint32_t* hB, double* a, double* b) {
    const int D = d * d;
    double mA = 0, mB = 0;
    for (int x = 0; x < D; ++x) { a[x] = hA[x]; b[x] = hB[x]; mA += hA[x]; mB += hB[x]; }
    a[D] = mB; b[D] = mA;
}

/* Alg. 1 for one pair of rasterised diagrams. */
int or_sinkhorn_pdp(int d, double pw, double gamma, const uint32_t* hA, const uint32_t* hB,
                   int max_iter, double tol, const double* g_init,
                   double* cost, double* f, double* g, double* rmarg, double* cmarg,
                   int* iters, double* err) {
    const int n = d * d + 1;
    double* a = (double*)malloc(sizeof(double) * n);
    double* b = (double*)malloc(sizeof(double) * n);
    augment(d, hA, hB, a, b);
    int rc = or_sinkhorn_wp(d, pw, gamma, a, b, max_iter, tol, g_init, cost, f, g, rmarg, cmarg, iters, err);
    free(a); free(b);
    return rc;
}

int or_sinkhorn_pd(int d, double gamma, const uint32_t* hA, const uint32_t* hB,
                   int max_iter, double tol, const double* g_init,
                   double* cost, double* f, double* g, double* rmarg, double* cmarg, int* iters, double* err) {
    return or_sinkhorn_pdp(d, 2.0, gamma, hA, hB, max_iter, tol, g_init, cost, f, g, rmarg, cmarg, iters, err);
}

/* Alg. 1 over P pairs (histA[p], histB[p]), parallel over pairs.  Outputs are
 * per pair; f, g, rmarg, cmarg have n = d*d+1 entries per pair (may be NULL). */
int or_sinkhorn_pd_batchp(int d, double pw, double gamma, const uint32_t* hA, const uint32_t* hB, int P,
                         int max_iter, double tol, double* cost, double* f, double* g,
                         double* rmarg, double* cmarg, int* iters, double* err) {
    const size_t D = (size_t)d * d, n = D + 1;
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int p = 0; p < P; ++p) {
        int rc = or_sinkhorn_pdp(d, pw, gamma, hA + p * D, hB + p * D, max_iter, tol, NULL,
                                cost ? cost + p : NULL, f ? f + p * n : NULL, g ? g + p * n : NULL,
                                rmarg ? rmarg + p * n : NULL, cmarg ? cmarg + p * n : NULL,
                                iters ? iters + p : NULL, err ? err + p : NULL);
        bad |= (rc != 0);
    }
    return bad ? -1 : 0;
}

int or_sinkhorn_pd_batch(int d, double gamma, const uint32_t* hA, const uint32_t* hB, int P,
                         int max_iter, double tol, double* cost, double* f, double* g,
                         double* rmarg, double* cmarg, int* iters, double* err) {
    return or_sinkhorn_pd_batchp(d, 2.0, gamma, hA, hB, P, max_iter, tol, cost, f, g, rmarg, cmarg, iters, err);
}

/* ---------------------------------------------------------------------- */
/* Alg. 2: smoothed barycenter of N rasterised diagrams.
 * z starts as z_init (d*d, may be NULL): NULL means the uniform measure above
 * the diagonal, i.e. every cell with j >= i gets mass (mean_i |D_i|) /
 * (d(d+1)/2).  Each outer step:
 *   for every i, Sinkhorn between (z + R a_i) and (a_i + R z), warm-started
 *   from the previous outer step's g_i, stopped at (tol, max_iter);
 *   grad(x) = (1/N) sum_i [ gamma*log u_i(x) + gamma*log v_i(Delta) ]
 *           = (1/N) sum_i [ gamma*log z(x) + f_i(x) + gamma*log|z| + g_i(Delta) ]
 *   (gradient proposition of Sec. 4; R^T maps the Delta value to a constant
 *   on the grid), divided by N so that it is the gradient of the mean energy;
 *   z <- z * exp(-lambda * grad) on the cells where z > 0.
 * energy[t] = (1/N) sum_i <P_i, C_i> of the step-t plans (energy of z_t).
 * Outputs z_out (d*d) and energy (outer_iters entries, may be NULL).        */
/* Entropy of the normalised measure w^beta / sum w^beta, w = z / |z| (z >= 0,
 * zeros skipped).  The powers are taken of v = z / max z (the normalised
 * measure is the same, since w and v differ by a constant factor), so the
 * largest term is 1 and the sum cannot underflow however large beta is:
 * H(beta) = log S - beta T / S with S = sum v^beta, T = sum v^beta log v. */
static double sharp_entropy(const double* z, int D, double zmax, double beta) {
    or_ksum S = {0, 0}, T = {0, 0};
    for (int x = 0; x < D; ++x) {
        if (!(z[x] > 0)) continue;
        const double lv = log(z[x] / zmax);
        const double vb = exp(beta * lv);
        ks_add(&S, vb);
        ks_add(&T, vb * lv);
    }
    return log(ks_val(&S)) - beta * ks_val(&T) / ks_val(&S);
}

/* Entropic sharpening (Solomon et al., the reference of the paper's Sec. 4
 * remark on smeared barycenters): when the entropy of the normalised measure
 * z / |z| exceeds H0, z is replaced by |z| w^beta / sum w^beta with the beta >= 1
 * for which that entropy equals H0 (the entropy decreases with beta; bisection
 * in FP64).  Returns beta (1 when no sharpening was needed). */
double or_sharpen(int d, double* z, double H0) {
    const int D = d * d;
    double zm = 0, zmax = 0;
    for (int x = 0; x < D; ++x) { zm += z[x]; zmax = fmax(zmax, z[x]); }
    if (!(zm > 0) || !(sharp_entropy(z, D, zmax, 1.0) > H0)) return 1.0;
    double lo = 1.0, hi = 2.0;
    while (sharp_entropy(z, D, zmax, hi) > H0 && hi < 1e6) { lo = hi; hi *= 2.0; }
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sharp_entropy(z, D, zmax, mid) > H0) lo = mid; else hi = mid;
    }
    const double beta = 0.5 * (lo + hi);
    or_ksum S = {0, 0};
    for (int x = 0; x < D; ++x) if (z[x] > 0) ks_add(&S, exp(beta * log(z[x] / zmax)));
    const double Sv = ks_val(&S);
    for (int x = 0; x < D; ++x) if (z[x] > 0) z[x] = zm * exp(beta * log(z[x] / zmax)) / Sv;
    return beta;
}

/* Alg. 2 with the stopping rule of the barycenter experiment (Sec. 5, Fig. 5):
 * after step t (its Sinkhorn solves give the energy E_t of z_t, then z is
 * updated), stop when t >= 1 and |E_t / E_{t-1} - 1| < rel_energy_tol
 * (rel_energy_tol <= 0: run all outer_iters steps).  *steps_out (if not NULL)
 * receives the number of steps run; energy[0 .. steps-1] is written. */
int or_barycenter_e(int d, double gamma, const uint32_t* hists, int N, double lambda,
                    int outer_iters, int max_iter, double tol, const double* z_init,
                    double* z_out, double* energy, int sharpen, double rel_energy_tol, int* steps_out) {
    const int D = d * d, n = D + 1;
    if (N <= 0 || d < 2) return -1;
    double* z = (double*)malloc(sizeof(double) * D);
    if (z_init) memcpy(z, z_init, sizeof(double) * D);
    else {
        double mean = 0;
        for (int i = 0; i < N; ++i) for (int x = 0; x < D; ++x) mean += hists[(size_t)i * D + x];
        mean /= N;
        double per = mean / (d * (d + 1) / 2.0);
        for (int i = 0; i < d; ++i) for (int j = 0; j < d; ++j) z[i * d + j] = (j >= i) ? per : 0.0;
    }
    double* gs = (double*)calloc((size_t)N * n, sizeof(double));
    double* fs = (double*)calloc((size_t)N * n, sizeof(double));
    double* costs = (double*)calloc(N, sizeof(double));
    int bad = 0;
    /* sharpening target: the largest entropy among the normalised input histograms */
    double H0 = -INFINITY;
    if (sharpen) {
        double* w = (double*)malloc(sizeof(double) * D);
        for (int i = 0; i < N; ++i) {
            double m = 0;
            for (int x = 0; x < D; ++x) { w[x] = hists[(size_t)i * D + x]; m += w[x]; }
            double mx = 0;
            for (int x = 0; x < D; ++x) mx = fmax(mx, w[x]);
            if (m > 0) H0 = fmax(H0, sharp_entropy(w, D, mx, 1.0));
        }
        free(w);
    }
    double e_prev = NAN;
    int steps = 0;
    for (int t = 0; t < outer_iters; ++t) {
        double zm = 0;
        for (int x = 0; x < D; ++x) zm += z[x];
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
        for (int i = 0; i < N; ++i) {
            double* a = (double*)malloc(sizeof(double) * n);
            double* b = (double*)malloc(sizeof(double) * n);
            double mi = 0;
            for (int x = 0; x < D; ++x) { a[x] = z[x]; b[x] = hists[(size_t)i * D + x]; mi += b[x]; }
            a[D] = mi; b[D] = zm;
            double* gw = (double*)malloc(sizeof(double) * n);
            memcpy(gw, gs + (size_t)i * n, sizeof(double) * n);
            int rc = or_sinkhorn_w(d, gamma, a, b, max_iter, tol, gw, costs + i,
                                   fs + (size_t)i * n, gs + (size_t)i * n, NULL, NULL, NULL, NULL);
            bad |= (rc != 0);
            free(a); free(b); free(gw);
        }
        or_ksum ek = {0, 0};
        for (int i = 0; i < N; ++i) ks_add(&ek, costs[i]);
        const double e_t = ks_val(&ek) / N;
        if (energy) energy[t] = e_t;
        double lzm = log(zm);
        for (int x = 0; x < D; ++x) {
            if (!(z[x] > 0)) continue;
            or_ksum s = {0, 0};
            for (int i = 0; i < N; ++i)
                ks_add(&s, gamma * log(z[x]) + fs[(size_t)i * n + x] + gamma * lzm + gs[(size_t)i * n + D]);
            double grad = ks_val(&s) / N;
            z[x] *= exp(-lambda * grad);
        }
        if (sharpen) or_sharpen(d, z, H0);
        steps = t + 1;
        if (rel_energy_tol > 0 && t >= 1 && fabs(e_t / e_prev - 1.0) < rel_energy_tol) break;
        e_prev = e_t;
    }
    memcpy(z_out, z, sizeof(double) * D);
    if (steps_out) *steps_out = steps;
    free(z); free(gs); free(fs); free(costs);
    return bad ? -1 : 0;
}

int or_barycenter_s(int d, double gamma, const uint32_t* hists, int N, double lambda,
                    int outer_iters, int max_iter, double tol, const double* z_init,
                    double* z_out, double* energy, int sharpen) {
    return or_barycenter_e(d, gamma, hists, N, lambda, outer_iters, max_iter, tol, z_init, z_out, energy,
                           sharpen, 0.0, NULL);
}

/* ---------------------------------------------------------------------- */
/* Alg. 2 without sharpening. */
int or_barycenter(int d, double gamma, const uint32_t* hists, int N, double lambda,
                  int outer_iters, int max_iter, double tol, const double* z_init,
                  double* z_out, double* energy) {
    return or_barycenter_s(d, gamma, hists, N, lambda, outer_iters, max_iter, tol, z_init, z_out, energy, 0);
}

/* splitmix64 (Steele, Lea & Flood 2014), used for the k-means seeding. */
static uint64_t splitmix64(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* k-means on diagrams (Sec. 5): centroids start as k distinct input
 * histograms drawn with splitmix64(seed) (draw r mod N, skip repeats).  Each
 * round: assign every diagram n to argmin_c <P, C> of the pair
 * (a_n + R z_c, z_c + R a_n) (ties -> lowest c; cold start, (tol, max_iter));
 * then each non-empty cluster's centroid takes bary_steps outer steps of
 * Alg. 2 over its members starting from the current centroid (an empty
 * cluster keeps its centroid).  objective[r] = sum_n min_c cost at round r.
 * Outputs assign (N), centroids (k*d*d), objective (rounds, may be NULL).   */
int or_kmeans(int d, double gamma, const uint32_t* hists, int N, int k, double lambda,
              int rounds, int bary_steps, int max_iter, double tol, uint64_t seed,
              int32_t* assign, double* centroids, double* objective) {
    const int D = d * d, n = D + 1;
    if (k <= 0 || k > N) return -1;
    uint64_t st = seed;
    int* chosen = (int*)malloc(sizeof(int) * k);
    for (int c = 0; c < k;) {
        int r = (int)(splitmix64(&st) % (uint64_t)N);
        int dup = 0;
        for (int q = 0; q < c; ++q) dup |= (chosen[q] == r);
        if (!dup) chosen[c++] = r;
    }
    for (int c = 0; c < k; ++c)
        for (int x = 0; x < D; ++x) centroids[(size_t)c * D + x] = hists[(size_t)chosen[c] * D + x];
    double* cst = (double*)malloc(sizeof(double) * (size_t)N * k);
    int bad = 0;
    for (int r = 0; r < rounds; ++r) {
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
        for (int q = 0; q < N * k; ++q) {
            int i = q / k, c = q % k;
            double* a = (double*)malloc(sizeof(double) * n);
            double* b = (double*)malloc(sizeof(double) * n);
            double mi = 0, mz = 0;
            for (int x = 0; x < D; ++x) {
                a[x] = hists[(size_t)i * D + x]; b[x] = centroids[(size_t)c * D + x];
                mi += a[x]; mz += b[x];
            }
            a[D] = mz; b[D] = mi;
            int rc = or_sinkhorn_w(d, gamma, a, b, max_iter, tol, NULL, cst + q,
                                   NULL, NULL, NULL, NULL, NULL, NULL);
            bad |= (rc != 0);
            free(a); free(b);
        }
        or_ksum obj = {0, 0};
        for (int i = 0; i < N; ++i) {
            int best = 0;
            for (int c = 1; c < k; ++c) if (cst[(size_t)i * k + c] < cst[(size_t)i * k + best]) best = c;
            assign[i] = best;
            ks_add(&obj, cst[(size_t)i * k + best]);
        }
        if (objective) objective[r] = ks_val(&obj);
        for (int c = 0; c < k; ++c) {
            int m = 0;
            for (int i = 0; i < N; ++i) m += (assign[i] == c);
            if (m == 0) continue;
            uint32_t* mem = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)m * D);
            int w = 0;
            for (int i = 0; i < N; ++i)
                if (assign[i] == c) memcpy(mem + (size_t)(w++) * D, hists + (size_t)i * D, sizeof(uint32_t) * D);
            double* zc = centroids + (size_t)c * D;
            int rc = or_barycenter(d, gamma, mem, m, lambda, bary_steps, max_iter, tol, zc, zc, NULL);
            bad |= (rc != 0);
            free(mem);
        }
    }
    free(chosen); free(cst);
    return bad ? -1 : 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Rounding (supplementary, algorithm of Altschuler et al.) of the plan
 * P_xy = a_x b_y exp((f_x + g_y - C_xy)/gamma) onto Pi(a, b), and <R, C>.
 * Literal, on the dense (d^2+1) x (d^2+1) matrices (no separability):
 *   X = min(a / r(P), 1), P' = diag(X) P, Y = min(b / c(P'), 1),
 *   P'' = P' diag(Y), e_r = a - r(P''), e_c = b - c(P''),
 *   R = P'' + e_r e_c^T / ||e_c||_1.
 * A zero row or column sum of P gives a factor 1 (min(+inf, 1)).
 * Outputs: *upper = <R, C>; *row_dev, *col_dev = max |r(R) - a|, max |c(R) - b|
 * (R has the marginals (a, b) exactly, up to rounding); *er, *ec = ||e_r||_1,
 * ||e_c||_1.  Returns -1 when d > 64 (the dense plan would not fit). */
int or_round_bound(int d, double gamma, const double* a, const double* b, const double* f, const double* g,
                   double* upper, double* row_dev, double* col_dev, double* er, double* ec) {
    if (d > 64) return -1;
    const int n = d * d + 1;
    double* P = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* rs = (double*)calloc(n, sizeof(double));
    double* cs = (double*)calloc(n, sizeof(double));
    double* X = (double*)malloc(sizeof(double) * n);
    double* Y = (double*)malloc(sizeof(double) * n);
    double* e_r = (double*)malloc(sizeof(double) * n);
    double* e_c = (double*)malloc(sizeof(double) * n);
    for (int x = 0; x < n; ++x)
        for (int y = 0; y < n; ++y) {
            double v = 0.0;
            if (a[x] > 0 && b[y] > 0) v = exp(log(a[x]) + log(b[y]) + (f[x] + g[y] - or_cost(d, x, y)) / gamma);
            P[(size_t)x * n + y] = v;
        }
    /* X, then P' = diag(X) P */
    for (int x = 0; x < n; ++x) {
        or_ksum k = {0, 0};
        for (int y = 0; y < n; ++y) ks_add(&k, P[(size_t)x * n + y]);
        rs[x] = ks_val(&k);
        X[x] = rs[x] > 0 ? fmin(a[x] / rs[x], 1.0) : 1.0;
        for (int y = 0; y < n; ++y) P[(size_t)x * n + y] *= X[x];
    }
    /* Y, then P'' = P' diag(Y) */
    for (int y = 0; y < n; ++y) {
        or_ksum k = {0, 0};
        for (int x = 0; x < n; ++x) ks_add(&k, P[(size_t)x * n + y]);
        cs[y] = ks_val(&k);
        Y[y] = cs[y] > 0 ? fmin(b[y] / cs[y], 1.0) : 1.0;
    }
    for (int x = 0; x < n; ++x)
        for (int y = 0; y < n; ++y) P[(size_t)x * n + y] *= Y[y];
    /* marginal errors of P'' */
    or_ksum ner = {0, 0}, nec = {0, 0};
    for (int x = 0; x < n; ++x) {
        or_ksum k = {0, 0};
        for (int y = 0; y < n; ++y) ks_add(&k, P[(size_t)x * n + y]);
        e_r[x] = a[x] - ks_val(&k);
        ks_add(&ner, e_r[x]);
    }
    for (int y = 0; y < n; ++y) {
        or_ksum k = {0, 0};
        for (int x = 0; x < n; ++x) ks_add(&k, P[(size_t)x * n + y]);
        e_c[y] = b[y] - ks_val(&k);
        ks_add(&nec, e_c[y]);
    }
    const double ecn = ks_val(&nec);
    /* R = P'' + e_r e_c^T / ||e_c||_1, its cost and its marginals */
    if (ecn > 0)
        for (int x = 0; x < n; ++x)
            for (int y = 0; y < n; ++y) P[(size_t)x * n + y] += e_r[x] * e_c[y] / ecn;
    or_ksum ck = {0, 0};
    double rd = 0, cd = 0;
    for (int x = 0; x < n; ++x) {
        or_ksum k = {0, 0};
        for (int y = 0; y < n; ++y) {
            ks_add(&ck, P[(size_t)x * n + y] * or_cost(d, x, y));
            ks_add(&k, P[(size_t)x * n + y]);
        }
        rd = fmax(rd, fabs(ks_val(&k) - a[x]));
    }
    for (int y = 0; y < n; ++y) {
        or_ksum k = {0, 0};
        for (int x = 0; x < n; ++x) ks_add(&k, P[(size_t)x * n + y]);
        cd = fmax(cd, fabs(ks_val(&k) - b[y]));
    }
    if (upper) *upper = ks_val(&ck);
    if (row_dev) *row_dev = rd;
    if (col_dev) *col_dev = cd;
    if (er) *er = ks_val(&ner);
    if (ec) *ec = ecn;
    free(P); free(rs); free(cs); free(X); free(Y); free(e_r); free(e_c);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Lower bound m_t of Sec. 3 "Upper and Lower Bounds": from the first dual
 * variable alpha = gamma log u (u = a exp(f/gamma), so alpha = f + gamma log a
 * on the support of a), its C-transform and the C^T-transform of that,
 *   alpha^c(y)   = min_{x in supp a} C(x,y) - alpha(x),     y in supp b,
 *   alpha^cc(x)  = min_{y in supp b} C(x,y) - alpha^c(y),   x in supp a,
 * (the transforms are infima: the pair (alpha^cc, alpha^c) then satisfies the
 * dual constraint alpha^cc(x) + alpha^c(y) <= C(x,y) on the supports), and
 *   m = <alpha^cc, a> + <alpha^c, b>  <=  the exact transport cost (weak duality).
 * Plain double loops over the supports with the explicit cost. */
int or_ctransform_bound(int d, double gamma, const double* a, const double* b, const double* f, double* lower) {
    const int n = d * d + 1;
    int na = 0, nb = 0;
    int* sa = (int*)malloc(sizeof(int) * n);
    int* sb = (int*)malloc(sizeof(int) * n);
    for (int x = 0; x < n; ++x) { if (a[x] > 0) sa[na++] = x; if (b[x] > 0) sb[nb++] = x; }
    double* alpha = (double*)malloc(sizeof(double) * (na + 1));
    double* ac = (double*)malloc(sizeof(double) * (nb + 1));
    for (int p = 0; p < na; ++p) alpha[p] = f[sa[p]] + gamma * log(a[sa[p]]);
    for (int q = 0; q < nb; ++q) {
        double m = INFINITY;
        for (int p = 0; p < na; ++p) m = fmin(m, or_cost(d, sa[p], sb[q]) - alpha[p]);
        ac[q] = m;
    }
    or_ksum s = {0, 0};
    for (int p = 0; p < na; ++p) {
        double m = INFINITY;
        for (int q = 0; q < nb; ++q) m = fmin(m, or_cost(d, sa[p], sb[q]) - ac[q]);
        ks_add(&s, a[sa[p]] * m);
    }
    for (int q = 0; q < nb; ++q) ks_add(&s, b[sb[q]] * ac[q]);
    if (lower) *lower = (na > 0 && nb > 0) ? ks_val(&s) : 0.0;
    free(sa); free(sb); free(alpha); free(ac);
    return 0;
}
