// bounds.cu -- the lower bound m_t of Sec. 3 "Upper and Lower Bounds".
//
// From the first dual variable alpha = gamma log u = f + gamma log a (on the
// support of a), the C-transform alpha^c(y) = min_x C(x,y) - alpha(x) (y on the
// support of b) and the C^T-transform of that, alpha^cc(x) = min_y C(x,y) -
// alpha^c(y) (x on the support of a), give a pair satisfying the dual
// constraint on the supports, so m = <alpha^cc, a> + <alpha^c, b> is below the
// exact transport cost (weak duality).  The transforms are inf-convolutions
// with the separable cost of Prop. 1, evaluated in the (min, +) semiring with
// the same two stages as the kernel application (rows first, then columns),
// restricted to the supports, in FP64: exact up to the rounding of the sums.
#include "sk_common.cuh"

// Non-empty input rows and output columns of a transform.
static __device__ void ct_lines(const int* __restrict__ rpin, const int* __restrict__ cpout, int d, int* rows,
                                int* cols, int* colpos, int* nrc) {
    if (threadIdx.x == 0) {
        int nr = 0, nc = 0;
        for (int k = 0; k < d; ++k) if (rpin[k + 1] > rpin[k]) rows[nr++] = k;
        for (int j = 0; j < d; ++j) {
            colpos[j] = -1;
            if (cpout[j + 1] > cpout[j]) { colpos[j] = nc; cols[nc++] = j; }
        }
        nrc[0] = nr; nrc[1] = nc;
    }
    __syncthreads();
}

// Stage 1 of a transform: A[r][c] = min over the input cells (i, j) of row
// rows[r] of c_{j, cols[c]} - in(i, j).
template <class In>
static __device__ void ct_rows(const int* __restrict__ rpin, const int* __restrict__ listin, In in, double* A, int d,
                               int dp, const int* rows, const int* cols, int nr, int nc, double pw) {
    for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
        const int r = e / nc, c = e - r * nc, i = rows[r], l = cols[c];
        double m = INFINITY;
        for (int q = rpin[i]; q < rpin[i + 1]; ++q) {
            const int cell = listin[q];
            m = fmin(m, pd_c1p(cell % dp, l, d, pw) - in(cell));
        }
        A[(size_t)r * nc + c] = m;
    }
    __syncthreads();
}

// Stage 2 at one output cell (k, l): min over rows of c_{rows[r], k} + A[r][colpos[l]],
// and the input Delta term cD(k, l) - inD when the input side has a Delta mass.
static __device__ __forceinline__ double ct_cell(int cell, const double* A, int d, int dp, const int* rows,
                                                 const int* colpos, int nr, int nc, double inD, bool hasD, double pw) {
    const int k = cell / dp, l = cell % dp, c = colpos[l];
    double m = hasD ? pd_cdiagp(k, l, d, pw) - inD : INFINITY;
    for (int r = 0; r < nr; ++r) m = fmin(m, pd_c1p(rows[r], k, d, pw) + A[(size_t)r * nc + c]);
    return m;
}

// Delta entry of a transform: min( min over the input support of cD(x) - in(x), -inD ).
template <class In>
static __device__ double ct_delta(const int* __restrict__ listin, int nin, In in, double inD, bool hasD, int d, int dp,
                                  double* shd, double pw) {
    double m = INFINITY;
    for (int e = threadIdx.x; e < nin; e += blockDim.x) {
        const int cell = listin[e];
        m = fmin(m, pd_cdiagp(cell / dp, cell % dp, d, pw) - in(cell));
    }
    m = -block_max(-m, shd, (double)-INFINITY);
    if (hasD) m = fmin(m, -inD);
    return m;
}

__global__ void __launch_bounds__(256) sk_ctransform_kernel(SkWS w, double* __restrict__ lower) {
    __shared__ int rows[256], cols[256], colpos[256], nrc[2];
    __shared__ double shd[32];
    const int p = blockIdx.x, t = threadIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    const int st = q.ic[IC_STATUS];
    if (!((st == ST_CONVERGED || st == ST_MAXITER) && q.sc[SC_TOTAL] > 0)) {
        if (t == 0) lower[p] = (st == ST_CONVERGED && q.sc[SC_TOTAL] == 0) ? 0.0 : NAN;
        return;
    }
    const int d = w.d, dp = w.dp, n1 = w.n - 1, na = q.ic[IC_NA], nb = q.ic[IC_NB];
    const double gamma = w.gamma;
    const double aD = q.sc[SC_AD], bD = q.sc[SC_BD];
    const bool hasA = aD > 0, hasB = bD > 0;
    double* A = q.L64;                          // [nr][nc] stage buffer (<= dp*dp doubles)
    double* ac = q.L64 + (size_t)dp * dp;       // [dp*dp] alpha^c by padded cell (b support)
    const double* phi = q.phi;
    const double* la = q.la;
    auto alpha = [=](int cell) { return gamma * (phi[cell] + la[cell]); };   // gamma log u
    auto acf = [=](int cell) { return ac[cell]; };
    const double alphaD = hasA ? gamma * (phi[n1] + log(aD)) : 0.0;
    // alpha^c on the b support and its Delta entry
    ct_lines(q.rpa, q.cpb, d, rows, cols, colpos, nrc);
    int nr = nrc[0], nc = nrc[1];
    ct_rows(q.rpa, q.sa, alpha, A, d, dp, rows, cols, nr, nc, w.p);
    double sum = 0.0;
    for (int e = t; e < nb; e += blockDim.x) {
        const int cell = q.sb[e];
        const double v = ct_cell(cell, A, d, dp, rows, colpos, nr, nc, alphaD, hasA, w.p);
        ac[cell] = v;
        sum += exp(q.lb[cell]) * v;
    }
    const double acD = hasB ? ct_delta(q.sa, na, alpha, alphaD, hasA, d, dp, shd, w.p) : 0.0;
    __syncthreads();
    // alpha^cc on the a support (summed with the weights a) and its Delta entry
    ct_lines(q.rpb, q.cpa, d, rows, cols, colpos, nrc);
    nr = nrc[0]; nc = nrc[1];
    ct_rows(q.rpb, q.sb, acf, A, d, dp, rows, cols, nr, nc, w.p);
    for (int e = t; e < na; e += blockDim.x) {
        const int cell = q.sa[e];
        sum += exp(q.la[cell]) * ct_cell(cell, A, d, dp, rows, colpos, nr, nc, acD, hasB, w.p);
    }
    const double accD = hasA ? ct_delta(q.sb, nb, acf, acD, hasB, d, dp, shd, w.p) : 0.0;
    const double s = block_sum(sum, shd);
    if (t == 0) lower[p] = s + (hasA ? aD * accD : 0.0) + (hasB ? bD * acD : 0.0);
}

cudaError_t sk_launch_ctransform(const SkWS& w, double* lower, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_ctransform_kernel<<<w.P, 256, 0, s>>>(w, lower);
    return cudaGetLastError();
}
