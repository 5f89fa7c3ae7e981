// sinkhorn_lse.cu -- exact log-domain Sinkhorn for persistence diagrams.
//
// Prop. 1's separable kernel application, K(v)_(i,j) = sum_k k_ik sum_l k_jl
// v_kl + v_Delta k_Delta, is evaluated in the log semiring (sum -> log-sum-exp,
// product -> sum), restricted to the supports of the histograms: zero-mass
// cells contribute exp(-inf) = 0 to every sum and their scalings are never
// read, so only
//   stage 1: L[k,j] = LSE_{l: (k,l) in supp(in)} ( h_kl - c_jl/gamma ),
//            k over the non-empty input rows, j over the output support's columns
//   stage 2: out_(i,j) = -LSE( LSE_k ( L[k,j] - c_ik/gamma ), h_Delta - cD_(i,j)/gamma )
//            for (i,j) on the output support
// are computed; h = log(weight) + potential/gamma of the input side.  The
// u-update (phi from psi) and the v-update (psi from phi) are the same
// routine with the two sides swapped (the cost is symmetric).  This is the
// log-domain form of Eq. (SinkhornMap): phi = f/gamma = -log(K v / ...),
// exact up to rounding and free of any over/underflow, whatever gamma.
//
// Precision: potentials are FP64.  Exponent arguments are formed in
// double-float (two FP32 words, TwoSum) so their error is ulp-level of the
// small centred argument, exponentials are FP32, and sums use Kahan
// compensation; the resulting log-values are accurate to a few 1e-7.
#define T_CTA 256
#include "sk_common.cuh"
#include <atomic>

struct df { float hi, lo; };

__device__ __forceinline__ df df_from(double x) {
    float h = (float)x;
    return {h, (float)(x - (double)h)};
}
// a - b for double-floats: the leading words are subtracted with TwoSum.
__device__ __forceinline__ df df_sub(df a, float bh, float bl) {
    float e;
    float s = two_sum(a.hi, -bh, e);
    return {s, e + (a.lo - bl)};
}
__device__ __forceinline__ double df_val(df a) { return (double)a.hi + (double)a.lo; }

// log(x) for x >= 1 (a sum whose largest term is 1): FP32 logf refined by one
// Newton step, L = L0 + (x e^-L0 - 1), so the absolute error is ~1e-7 whatever
// the size of log(x) (logf alone errs by |log x| * 2^-23).
__device__ __forceinline__ float log_acc(float x) {
    float l0 = logf(x);
    return l0 + fmaf(x, expf(-l0), -1.0f);
}

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Warp-wide max / compensated sum (all lanes get the result).
__device__ __forceinline__ float wmax(float v) { return warp_max(v); }
__device__ __forceinline__ float wsum_kahan(Kahan k) {
    float v = k.s - k.c;
    return warp_sum(v);
}

// One log-domain half-step.  Input side: weights' logs lin (FP64, by padded
// cell), potentials hin_pot (FP64), CSR of its support (rpin, listin), Delta
// log-weight + potential lD_in.  Output side: support list (listout, nout),
// column pointers (cpout) to know which columns are needed, output potentials
// written to out_pot (FP64) at the cells, and out_D.  Scratch: Hh/Hl (FP32
// dp*dp, the input h as double-float), Lh/Ll (FP32 dp*dp, stage-1 values).
// If err != NULL, the previous output potentials are compared with the new ones
// and sum_y w_y |exp(old_y - new_y) - 1| (with w the output weights) is added
// to *err (the marginal error of Eq. Altschuler bounds for the plan before the
// update).  all_cols: compute stage 1 for every column (for full-grid outputs).
struct HalfArgs {
    const double* lin; const double* pin; const int* rpin; const int* listin; int nin; double lD_in;
    const double* lout; const float* wout; double* pout; const int* listout; int nout; const int* cpout;
    double* pD_out; double lwD_out; double wD_out;
    float *Hh, *Hl, *Lh, *Ll;
};

__device__ void lse_stage1(const HalfArgs& a, const float* chi, const float* clo, int d, int dp, const int* rows,
                           int nr, const int* cols, int nc) {
    const int t = threadIdx.x;
    // input h = log w + pot as double-float
    for (int q = t; q < a.nin; q += blockDim.x) {
        int c = a.listin[q];
        df h = df_from(a.lin[c] + a.pin[c]);
        a.Hh[c] = h.hi; a.Hl[c] = h.lo;
    }
    __syncthreads();
    for (int e = t; e < nr * nc; e += blockDim.x) {
        const int k = rows[e / nc], j = cols[e % nc];
        const int q0 = a.rpin[k], q1 = a.rpin[k + 1];
        float m = -INFINITY;
        for (int q = q0; q < q1; ++q) {
            int c = a.listin[q], mm = abs(j - c % dp);
            df v = df_sub({a.Hh[c], a.Hl[c]}, chi[mm], clo[mm]);
            m = fmaxf(m, v.hi);
        }
        Kahan s;
        for (int q = q0; q < q1; ++q) {
            int c = a.listin[q], mm = abs(j - c % dp);
            df v = df_sub({a.Hh[c], a.Hl[c]}, chi[mm], clo[mm]);
            s.add(expf((v.hi - m) + v.lo));
        }
        a.Lh[k * dp + j] = m;
        a.Ll[k * dp + j] = log_acc(s.s - s.c);
    }
    __syncthreads();
}

// Stage 2 for one output cell (i,j), executed by one warp.  Returns -LSE as FP64.
__device__ __forceinline__ double lse_stage2_cell(const HalfArgs& a, const float* chi, const float* clo, int i,
                                                  int j, int d, int dp, const int* rows, int nr, df hD,
                                                  float cDh, float cDl) {
    const int lane = threadIdx.x & 31;
    float m = -INFINITY;
    for (int r = lane; r < nr; r += 32) {
        int k = rows[r], mm = abs(i - k);
        df v = df_sub({a.Lh[k * dp + j], a.Ll[k * dp + j]}, chi[mm], clo[mm]);
        m = fmaxf(m, v.hi);
    }
    df vD = df_sub(hD, cDh, cDl);
    m = fmaxf(wmax(m), vD.hi);
    Kahan s;
    for (int r = lane; r < nr; r += 32) {
        int k = rows[r], mm = abs(i - k);
        df v = df_sub({a.Lh[k * dp + j], a.Ll[k * dp + j]}, chi[mm], clo[mm]);
        s.add(expf((v.hi - m) + v.lo));
    }
    float tot = wsum_kahan(s);
    if (hD.hi > -INFINITY) tot += expf((vD.hi - m) + vD.lo);
    return -((double)m + (double)log_acc(tot));
}

// Delta output: -LSE( {h_y - cD_y/g : y in supp(in)} u {h_Delta} ).
__device__ double lse_delta(const HalfArgs& a, const float* chi2, const float* clo2, int dp, double* shd) {
    const int t = threadIdx.x;
    float m = -INFINITY;
    for (int q = t; q < a.nin; q += blockDim.x) {
        int c = a.listin[q], mm = abs(c % dp - c / dp);
        df v = df_sub({a.Hh[c], a.Hl[c]}, chi2[mm], clo2[mm]);
        m = fmaxf(m, v.hi);
    }
    df hD = df_from(a.lD_in);
    float mf = block_max(m, reinterpret_cast<float*>(shd), -INFINITY);
    mf = fmaxf(mf, hD.hi);
    Kahan s;
    for (int q = t; q < a.nin; q += blockDim.x) {
        int c = a.listin[q], mm = abs(c % dp - c / dp);
        df v = df_sub({a.Hh[c], a.Hl[c]}, chi2[mm], clo2[mm]);
        s.add(expf((v.hi - mf) + v.lo));
    }
    float tot = block_sum(s.s - s.c, reinterpret_cast<float*>(shd));
    if (hD.hi > -INFINITY) tot += expf((hD.hi - mf) + hD.lo);
    if (!(mf > -INFINITY)) return INFINITY;
    return -((double)mf + (double)log_acc(tot));
}

// Full half-step on the output support; returns the marginal-error contribution
// (FP64, only if want_err) of the output side.
__device__ double lse_halfstep(HalfArgs a, const float* chi, const float* clo, const float* chi2, const float* clo2,
                               int d, int dp, int* rows, int* cols, int* nrc, bool want_err, double* shd) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    if (t == 0) {
        int nr = 0, nc = 0;
        for (int k = 0; k < d; ++k) if (a.rpin[k + 1] > a.rpin[k]) rows[nr++] = k;
        for (int j = 0; j < d; ++j) if (a.cpout[j + 1] > a.cpout[j]) cols[nc++] = j;
        nrc[0] = nr; nrc[1] = nc;
    }
    __syncthreads();
    const int nr = nrc[0], nc = nrc[1];
    lse_stage1(a, chi, clo, d, dp, rows, nr, cols, nc);
    const df hD = df_from(a.lD_in);
    double err = 0.0;
    for (int e = wid; e < a.nout; e += nw) {
        const int c = a.listout[e], i = c / dp, j = c % dp, mm = abs(j - i);
        double nv = lse_stage2_cell(a, chi, clo, i, j, d, dp, rows, nr, hD, chi2[mm], clo2[mm]);
        if (lane == 0) {
            if (want_err) err += (double)(a.wout[c] * fabsf(expm1f((float)(a.pout[c] - nv))));
            a.pout[c] = nv;
        }
    }
    double nD = lse_delta(a, chi2, clo2, dp, shd);
    if (t == 0 && a.lwD_out > -INFINITY) {
        if (want_err) err += a.wD_out * (double)fabsf(expm1f((float)(*a.pD_out - nD)));
        *a.pD_out = nD;
    }
    __syncthreads();
    return want_err ? block_sum(err, shd) : 0.0;
}

__device__ __forceinline__ HalfArgs u_args(PairPtrs& q, const SkWS& w) {
    HalfArgs a;
    a.lin = q.lb; a.pin = q.psi; a.rpin = q.rpb; a.listin = q.sb; a.nin = q.ic[IC_NB];
    a.lD_in = (q.sc[SC_BD] > 0) ? log(q.sc[SC_BD]) + q.psi[w.n - 1] : -INFINITY;
    a.lout = q.la; a.wout = q.am; a.pout = q.phi; a.listout = q.sa; a.nout = q.ic[IC_NA]; a.cpout = q.cpa;
    a.pD_out = &q.phi[w.n - 1];
    a.lwD_out = (q.sc[SC_AD] > 0) ? log(q.sc[SC_AD]) : -INFINITY;
    a.wD_out = q.sc[SC_AD];
    a.Hh = q.Wt; a.Hl = q.Rt; a.Lh = q.K1u; a.Ll = q.K2u;
    return a;
}
__device__ __forceinline__ HalfArgs v_args(PairPtrs& q, const SkWS& w) {
    HalfArgs a;
    a.lin = q.la; a.pin = q.phi; a.rpin = q.rpa; a.listin = q.sa; a.nin = q.ic[IC_NA];
    a.lD_in = (q.sc[SC_AD] > 0) ? log(q.sc[SC_AD]) + q.phi[w.n - 1] : -INFINITY;
    a.lout = q.lb; a.wout = q.bm; a.pout = q.psi; a.listout = q.sb; a.nout = q.ic[IC_NB]; a.cpout = q.cpb;
    a.pD_out = &q.psi[w.n - 1];
    a.lwD_out = (q.sc[SC_BD] > 0) ? log(q.sc[SC_BD]) : -INFINITY;
    a.wD_out = q.sc[SC_BD];
    a.Hh = q.Wt; a.Hl = q.Rt; a.Lh = q.K1u; a.Ll = q.K2u;
    return a;
}

// Iterations: u-update, then the v-update which also yields err_t.
__global__ void __launch_bounds__(T_CTA) sk_lse_iter_kernel(SkWS w, SkRun r, int n_inner, int* active_count,
                                                             int min_big) {
    __shared__ int rows[256], cols[256], nrc[2];
    __shared__ double shd[32];
    const int p = blockIdx.x, t = threadIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    if (q.ic[IC_STATUS] != ST_ACTIVE || q.ic[IC_BIG] < min_big) return;
    const int d = w.d, dp = w.dp;
    const float* chi = w.ctab;             // c_m/gamma, hi / lo
    const float* clo = w.ctab + dp;
    const float* chi2 = w.ctab + 2 * dp;   // c_m/(2 gamma): cost to the diagonal bin, m = |j - i|
    const float* clo2 = w.ctab + 3 * dp;
    const double total = q.sc[SC_TOTAL];
    int iters = q.ic[IC_ITERS];
    double err = q.sc[SC_ERR];
    int status = ST_ACTIVE;
    for (int it = 0; it < n_inner; ++it) {
        lse_halfstep(u_args(q, w), chi, clo, chi2, clo2, d, dp, rows, cols, nrc, false, shd);
        err = lse_halfstep(v_args(q, w), chi, clo, chi2, clo2, d, dp, rows, cols, nrc, true, shd) / total;
        ++iters;
        if (r.tol > 0 && err <= r.tol) { status = ST_CONVERGED; break; }
        if (iters >= r.max_iter) { status = ST_MAXITER; break; }
        if (!isfinite(err)) { status = ST_RANGE; break; }
    }
    if (t == 0) {
        q.sc[SC_ERR] = err;
        q.ic[IC_ITERS] = iters;
        q.ic[IC_STATUS] = status;
        q.ic[IC_ABSORB] = 0;
        if (status == ST_ACTIVE) atomicAdd(active_count, 1);
    }
}

cudaError_t sk_launch_lse_iter(const SkWS& w, SkRun r, int n_inner, int* active_count, int min_big,
                               cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_lse_iter_kernel<<<w.P, T_CTA, 0, s>>>(w, r, n_inner, active_count, min_big < 1 ? 1 : min_big);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Finalize: cost by Prop. 2 in the log domain, marginals and potentials.
//   cost = sum_{x in supp a} u_x [ sum_k c_ik k_ik W[k,j] + sum_k k_ik Wm[k,j] ]
//        + v_Delta sum_x u_x k_xDelta cD_x + u_Delta sum_y v_y k_Deltay cD_y
// with W[k,j] = sum_l k_jl v_kl and Wm[k,j] = sum_l c_jl k_jl v_kl (m = k . c),
// each evaluated as a log-sum-exp; the outer sums are FP64.
__global__ void __launch_bounds__(T_CTA) sk_lse_finalize_kernel(SkWS w, double* __restrict__ cost,
                                                                float* __restrict__ row_marg,
                                                                float* __restrict__ col_marg,
                                                                double* __restrict__ fo, double* __restrict__ go,
                                                                int32_t* __restrict__ iters_o,
                                                                float* __restrict__ err_o,
                                                                int32_t* __restrict__ status_o, int pso,
                                                                const int* __restrict__ plist) {
    __shared__ int rows[256], cols[256], nrc[2];
    __shared__ double shd[32];
    const int p = plist ? plist[blockIdx.x] : blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5,
              nw = blockDim.x >> 5;
    PairPtrs q = pair_ptrs(w, p);
    const int d = w.d, dp = w.dp, n_out = d * d + 1, na = q.ic[IC_NA], nb = q.ic[IC_NB];
    const int st = q.ic[IC_STATUS];
    if (t == 0) {
        if (iters_o) iters_o[p] = q.ic[IC_ITERS];
        if (err_o) err_o[p] = (float)q.sc[SC_ERR];
        if (status_o) status_o[p] = st == ST_CONVERGED ? 0 : (st == ST_MAXITER ? 6 : (st == ST_INVALID ? 1 : 8));
    }
    const bool usable = (st == ST_CONVERGED || st == ST_MAXITER) && q.sc[SC_TOTAL] > 0;
    if (!usable) {
        if (t == 0) cost[p] = (st == ST_CONVERGED && q.sc[SC_TOTAL] == 0) ? 0.0 : NAN;
        for (int x = t; x < n_out; x += blockDim.x) {
            if (row_marg) row_marg[(size_t)p * n_out + x] = 0.f;
            if (col_marg) col_marg[(size_t)p * n_out + x] = 0.f;
            if (fo) fo[(size_t)p * n_out + x] = NAN;
            if (go) go[(size_t)p * n_out + x] = NAN;
        }
        return;
    }
    const float* chi = w.ctab;
    const float* clo = w.ctab + dp;
    const float* chi2 = w.ctab + 2 * dp;
    const float* clo2 = w.ctab + 3 * dp;
    const float* lcm = w.ctab + 4 * dp;    // log(c_m) (physical units), -inf at m = 0
    const double gamma = w.gamma;
    const double lAD = q.sc[SC_AD] > 0 ? log(q.sc[SC_AD]) : -INFINITY;
    const double lBD = q.sc[SC_BD] > 0 ? log(q.sc[SC_BD]) : -INFINITY;
    const double phiD = q.phi[w.n - 1], psiD = q.psi[w.n - 1];
    HalfArgs ua = u_args(q, w);
    // stage 1 of the u-side application over every column, from psi_t
    if (t == 0) {
        int nr = 0;
        for (int k = 0; k < d; ++k) if (q.rpb[k + 1] > q.rpb[k]) rows[nr++] = k;
        for (int j = 0; j < d; ++j) cols[j] = j;
        nrc[0] = nr; nrc[1] = d;
    }
    __syncthreads();
    const int nr = nrc[0];
    lse_stage1(ua, chi, clo, d, dp, rows, nr, cols, d);
    // Wm[k,j] (log) into L64 as float pairs: LSE_l (h_kl - c_jl/g + log c_jl)
    float* Mh = reinterpret_cast<float*>(q.L64);
    float* Ml = Mh + (size_t)dp * dp;
    for (int e = t; e < nr * d; e += blockDim.x) {
        const int k = rows[e / d], j = e % d;
        float m = -INFINITY;
        for (int qq = q.rpb[k]; qq < q.rpb[k + 1]; ++qq) {
            int c = q.sb[qq], mm = abs(j - c % dp);
            df v = df_sub({ua.Hh[c], ua.Hl[c]}, chi[mm], clo[mm]);
            m = fmaxf(m, v.hi + lcm[mm]);
        }
        Kahan s;
        for (int qq = q.rpb[k]; qq < q.rpb[k + 1]; ++qq) {
            int c = q.sb[qq], mm = abs(j - c % dp);
            df v = df_sub({ua.Hh[c], ua.Hl[c]}, chi[mm], clo[mm]);
            if (lcm[mm] > -INFINITY) s.add(expf((v.hi - m) + v.lo + lcm[mm]));
        }
        Mh[k * dp + j] = m;
        Ml[k * dp + j] = (m > -INFINITY) ? log_acc(s.s - s.c) : 0.f;
    }
    __syncthreads();
    // per output cell (all grid cells when f is requested, else the a-support)
    const df hDb = df_from(lBD + psiD);
    double cs = 0.0, rowD = 0.0;
    const bool allx = fo && !pso;
    const int nx = allx ? d * d : na;
    for (int e = wid; e < nx; e += nw) {
        int i, j;
        if (allx) { i = e / d; j = e % d; } else { int c = q.sa[e]; i = c / dp; j = c % dp; }
        const int c = i * dp + j, mmD = abs(j - i);
        // -log (K v)_x  (phi' of the final v)
        double phip = lse_stage2_cell(ua, chi, clo, i, j, d, dp, rows, nr, hDb, chi2[mmD], clo2[mmD]);
        const bool ina = q.am[c] > 0.f;
        if (ina) {
            // log T1 = LSE_k (log c_ik - c_ik/g + L[k,j]); log T2 = LSE_k (-c_ik/g + Wm[k,j])
            float m1 = -INFINITY, m2 = -INFINITY;
            for (int r = lane; r < nr; r += 32) {
                int k = rows[r], mm = abs(i - k);
                df v1 = df_sub({ua.Lh[k * dp + j], ua.Ll[k * dp + j]}, chi[mm], clo[mm]);
                m1 = fmaxf(m1, v1.hi + lcm[mm]);
                df v2 = df_sub({Mh[k * dp + j], Ml[k * dp + j]}, chi[mm], clo[mm]);
                m2 = fmaxf(m2, v2.hi);
            }
            m1 = wmax(m1); m2 = wmax(m2);
            Kahan s1, s2;
            for (int r = lane; r < nr; r += 32) {
                int k = rows[r], mm = abs(i - k);
                df v1 = df_sub({ua.Lh[k * dp + j], ua.Ll[k * dp + j]}, chi[mm], clo[mm]);
                if (lcm[mm] > -INFINITY) s1.add(expf((v1.hi - m1) + v1.lo + lcm[mm]));
                df v2 = df_sub({Mh[k * dp + j], Ml[k * dp + j]}, chi[mm], clo[mm]);
                if (v2.hi > -INFINITY) s2.add(expf((v2.hi - m2) + v2.lo));
            }
            float t1 = wsum_kahan(s1), t2 = wsum_kahan(s2);
            if (lane == 0) {
                const double lu = q.la[c] + q.phi[c];
                if (m1 > -INFINITY) cs += exp(lu + (double)m1 + (double)log_acc(t1));
                if (m2 > -INFINITY) cs += exp(lu + (double)m2 + (double)log_acc(t2));
                const double cd = pd_cdiagp(i, j, d, w.p);
                if (lBD > -INFINITY && cd > 0) cs += exp(lu + lBD + psiD - cd / gamma) * cd;
                rowD += exp(lu + lBD + psiD - cd / gamma);
                if (row_marg) row_marg[(size_t)p * n_out + i * d + j] = (float)exp(lu - phip);
            }
        } else if (lane == 0 && row_marg && allx) {
            row_marg[(size_t)p * n_out + i * d + j] = 0.f;
        }
        if (lane == 0 && fo) fo[(size_t)p * n_out + i * d + j] = gamma * (ina ? q.phi[c] : phip);
    }
    if (row_marg && !allx) {
        for (int x = t; x < d * d; x += blockDim.x) {
            int c = (x / d) * dp + x % d;
            if (!(q.am[c] > 0.f)) row_marg[(size_t)p * n_out + x] = 0.f;
        }
    }
    // the b-side Delta term of the cost and the Delta entries
    double csb = 0.0, colD = 0.0;
    for (int e = t; e < nb; e += blockDim.x) {
        int c = q.sb[e], k = c / dp, l = c % dp;
        double cd = pd_cdiagp(k, l, d, w.p);
        double lv = q.lb[c] + q.psi[c];
        if (lAD > -INFINITY && cd > 0) csb += exp(lv + lAD + phiD - cd / gamma) * cd;
        colD += exp(lv + lAD + phiD - cd / gamma);
    }
    cs = block_sum(cs, shd);
    csb = block_sum(csb, shd);
    rowD = block_sum(rowD, shd);
    colD = block_sum(colD, shd);
    if (t == 0) cost[p] = cs + csb;
    if (row_marg && t == 0) {
        // Delta row: sum_y P_Delta,y + P_Delta,Delta
        double dd = (lAD > -INFINITY && lBD > -INFINITY) ? exp(lAD + phiD + lBD + psiD) : 0.0;
        row_marg[(size_t)p * n_out + d * d] = (float)(colD + dd);
    }
    // column marginal and g from (u_t, v_t)
    if (col_marg || go) {
        __syncthreads();
        HalfArgs va = v_args(q, w);
        if (t == 0) {
            int nr2 = 0;
            for (int k = 0; k < d; ++k) if (q.rpa[k + 1] > q.rpa[k]) rows[nr2++] = k;
            for (int j = 0; j < d; ++j) cols[j] = j;
            nrc[0] = nr2; nrc[1] = d;
        }
        __syncthreads();
        const int nr2 = nrc[0];
        lse_stage1(va, chi, clo, d, dp, rows, nr2, cols, d);
        const df hDa = df_from(lAD + phiD);
        for (int e = wid; e < d * d; e += nw) {
            const int k = e / d, l = e % d, c = k * dp + l, mmD = abs(l - k);
            const bool inb = q.bm[c] > 0.f;
            if (!inb && (!go || pso)) continue;
            double psip = lse_stage2_cell(va, chi, clo, k, l, d, dp, rows, nr2, hDa, chi2[mmD], clo2[mmD]);
            if (lane == 0) {
                if (col_marg) col_marg[(size_t)p * n_out + e] = inb ? (float)exp(q.lb[c] + q.psi[c] - psip) : 0.f;
                if (go) go[(size_t)p * n_out + e] = gamma * (inb ? q.psi[c] : psip);
            }
        }
        if (col_marg && (!go || pso)) {
            // cells off the b-support were skipped above: their marginal is 0
            for (int y = t; y < d * d; y += blockDim.x) {
                const int c = (y / d) * dp + y % d;
                if (!(q.bm[c] > 0.f)) col_marg[(size_t)p * n_out + y] = 0.f;
            }
        }
        if (t == 0) {
            double dd = (lAD > -INFINITY && lBD > -INFINITY) ? exp(lAD + phiD + lBD + psiD) : 0.0;
            if (col_marg) col_marg[(size_t)p * n_out + d * d] = (float)(rowD + dd);
        }
    }
    if (t == 0) {
        if (fo) fo[(size_t)p * n_out + d * d] = gamma * phiD;
        if (go) go[(size_t)p * n_out + d * d] = gamma * psiD;
    }
}

cudaError_t sk_launch_lse_finalize(const SkWS& w, double* cost, float* row_marg, float* col_marg, double* f,
                                   double* g, int32_t* iters, float* err, int32_t* status, int pso, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_lse_finalize_kernel<<<w.P, T_CTA, 0, s>>>(w, cost, row_marg, col_marg, f, g, iters, err, status, pso,
                                                 nullptr);
    return cudaGetLastError();
}
// Finalize of the pairs plist[0..np) only; outputs are indexed by pair.
cudaError_t sk_launch_lse_finalize_list(const SkWS& w, double* cost, float* row_marg, float* col_marg, double* f,
                                        double* g, int32_t* iters, float* err, int32_t* status, int pso,
                                        const int* plist, int np, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    sk_lse_finalize_kernel<<<np, T_CTA, 0, s>>>(w, cost, row_marg, col_marg, f, g, iters, err, status, pso, plist);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// On-chip iteration kernel.  For pairs whose supports fit (the common case for
// persistence diagrams of a few hundred points), everything an iteration
// touches lives in shared memory for the whole launch: the support lists, the
// FP64 potentials, the log-weights, the cost tables, the stage-1 buffer L and
// the input h.  Global memory is read at the start of the launch and written
// at its end only.  Pairs that do not fit are marked and left to the
// global-memory kernel above.
#define LSE_SM_THREADS 768

struct SideS {
    int n;                 // support size
    int nr, nc;            // non-empty rows / columns
    int* cell;             // [n] padded cell index, row-major order
    double* pot;           // [n] potential / gamma
    float *lwh, *lwl;      // [n] log weight as double-float
    float* w;              // [n] weight
    int* rp;               // [d+1] row pointers into cell
    short *rows, *cols;    // [nr], [nc]
    short* colpos;         // [d] position of a column in cols (or -1)
    double lD;             // log of the Delta weight (-inf if 0)
    double wD;             // Delta weight
    double potD;           // Delta potential / gamma
};

__device__ __forceinline__ size_t align_up(size_t x, size_t a) { return (x + a - 1) & ~(a - 1); }

// Shared-memory bytes needed for a pair (same formula on the host side check).
__device__ __forceinline__ size_t lse_smem_need(int nA, int nB, int nrA, int ncA, int nrB, int ncB, int d, int dp) {
    size_t b = 0;
    b += align_up((size_t)(nA + nB) * 8, 16);             // potentials
    b += align_up((size_t)(nA + nB) * 4 * 4, 16);         // cell, lwh, lwl, w
    b += align_up((size_t)2 * (d + 1) * 4, 16);           // row pointers
    b += align_up((size_t)6 * 256 * 2, 16);               // rows, cols, colpos (x2)
    b += align_up((size_t)4 * dp * 4, 16);                // cost tables
    int nmax = nA > nB ? nA : nB;
    b += align_up((size_t)nmax * 8, 16);                  // h
    size_t la = (size_t)nrB * (ncA | 1), lb = (size_t)nrA * (ncB | 1);
    b += align_up((la > lb ? la : lb) * 8, 16);           // L
    return b;
}

__device__ void sm_stage1(const SideS& in, const SideS& out, const float* Hh, const float* Hl, float* Lh, float* Ll,
                          int ld, const float* chi, const float* clo, int dp) {
    for (int e = threadIdx.x; e < in.nr * out.nc; e += blockDim.x) {
        const int r = e / out.nc, c = e - r * out.nc;
        const int k = in.rows[r], j = out.cols[c];
        const int q0 = in.rp[k], q1 = in.rp[k + 1];
        float m, tot;
        if (q1 - q0 <= 8) {
            // the row's arguments, formed once (double-float), then max and sum from registers
            float vh[8], vl[8];
            m = -INFINITY;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (q0 + u < q1) {
                    const int q = q0 + u, mm = abs(j - in.cell[q] % dp);
                    df v = df_sub({Hh[q], Hl[q]}, chi[mm], clo[mm]);
                    vh[u] = v.hi; vl[u] = v.lo;
                    m = fmaxf(m, v.hi);
                } else {
                    vh[u] = -INFINITY; vl[u] = 0.f;
                }
            }
            Kahan s;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (q0 + u < q1) s.add(expf((vh[u] - m) + vl[u]));
            tot = s.s - s.c;
        } else {
            m = -INFINITY;
            for (int q = q0; q < q1; ++q) {
                int mm = abs(j - in.cell[q] % dp);
                df v = df_sub({Hh[q], Hl[q]}, chi[mm], clo[mm]);
                m = fmaxf(m, v.hi);
            }
            Kahan s;
            for (int q = q0; q < q1; ++q) {
                int mm = abs(j - in.cell[q] % dp);
                df v = df_sub({Hh[q], Hl[q]}, chi[mm], clo[mm]);
                s.add(expf((v.hi - m) + v.lo));
            }
            tot = s.s - s.c;
        }
        Lh[r * ld + c] = m;
        Ll[r * ld + c] = log_acc(tot);
    }
    __syncthreads();
}

// One half-step in shared memory: out.pot <- -LSE over in.  Returns the
// (block-reduced) marginal error contribution if want_err.
__device__ double sm_halfstep(SideS& in, SideS& out, float* Hh, float* Hl, float* Lh, float* Ll, const float* chi,
                              const float* clo, const float* chi2, const float* clo2, int dp, bool want_err,
                              double* shd) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    for (int q = t; q < in.n; q += blockDim.x) {
        df h = df_from((double)in.lwh[q] + (double)in.lwl[q] + in.pot[q]);
        Hh[q] = h.hi; Hl[q] = h.lo;
    }
    __syncthreads();
    const int ld = out.nc | 1;
    sm_stage1(in, out, Hh, Hl, Lh, Ll, ld, chi, clo, dp);
    const df hD = df_from(in.lD + in.potD);
    double err = 0.0;
    // warp per non-empty output row i; lane holds rows r = lane + 32u of the input (u < 8)
    for (int rr = wid; rr < out.nr; rr += nw) {
        const int i = out.rows[rr];
        float kh[8], kl[8];
        int roff[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int r = lane + 32 * u;
            if (r < in.nr) {
                const int mm = abs(i - in.rows[r]);
                kh[u] = chi[mm]; kl[u] = clo[mm]; roff[u] = r * ld;
            } else {
                kh[u] = 0.f; kl[u] = 0.f; roff[u] = -1;
            }
        }
        for (int e = out.rp[i]; e < out.rp[i + 1]; ++e) {
            const int cell = out.cell[e], j = cell - i * dp, c = out.colpos[j];
            const int mmD = abs(j - i);
            float vh[8], vl[8];
            float m = -INFINITY;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (roff[u] >= 0) {
                    df v = df_sub({Lh[roff[u] + c], Ll[roff[u] + c]}, kh[u], kl[u]);
                    vh[u] = v.hi; vl[u] = v.lo;
                    m = fmaxf(m, v.hi);
                } else {
                    vh[u] = -INFINITY; vl[u] = 0.f;
                }
            }
            df vD = df_sub(hD, chi2[mmD], clo2[mmD]);
            m = fmaxf(warp_max(m), vD.hi);
            Kahan s;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (roff[u] >= 0) s.add(expf((vh[u] - m) + vl[u]));
            float tot = warp_sum(s.s - s.c);
            if (hD.hi > -INFINITY) tot += expf((vD.hi - m) + vD.lo);
            if (lane == 0) {
                double nv = -((double)m + (double)log_acc(tot));
                if (want_err) err += (double)(out.w[e] * fabsf(expm1f((float)(out.pot[e] - nv))));
                out.pot[e] = nv;
            }
        }
    }
    // Delta output
    float m = -INFINITY;
    for (int q = t; q < in.n; q += blockDim.x) {
        int cell = in.cell[q], mm = abs(cell % dp - cell / dp);
        df v = df_sub({Hh[q], Hl[q]}, chi2[mm], clo2[mm]);
        m = fmaxf(m, v.hi);
    }
    float mf = fmaxf(block_max(m, reinterpret_cast<float*>(shd), -INFINITY), hD.hi);
    Kahan s;
    for (int q = t; q < in.n; q += blockDim.x) {
        int cell = in.cell[q], mm = abs(cell % dp - cell / dp);
        df v = df_sub({Hh[q], Hl[q]}, chi2[mm], clo2[mm]);
        s.add(expf((v.hi - mf) + v.lo));
    }
    float tot = block_sum(s.s - s.c, reinterpret_cast<float*>(shd));
    if (t == 0 && out.wD > 0) {
        if (hD.hi > -INFINITY) tot += expf((hD.hi - mf) + hD.lo);
        double nD = (mf > -INFINITY) ? -((double)mf + (double)log_acc(tot)) : INFINITY;
        if (want_err) err += out.wD * (double)fabsf(expm1f((float)(out.potD - nD)));
        out.potD = nD;
    }
    __syncthreads();
    double e = want_err ? block_sum(err, shd) : 0.0;
    // every thread needs the new Delta potential of `out`
    __shared__ double potD_sh;
    if (t == 0) potD_sh = out.potD;
    __syncthreads();
    out.potD = potD_sh;
    __syncthreads();
    return e;
}

__device__ void compact_nonempty(const int* __restrict__ ptr, int d, short* out, int* count, short* pos) {
    // rows (or columns) i with ptr[i+1] > ptr[i], in increasing order; pos[i] = index or -1
    __shared__ int warp_cnt[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    // d <= 256 <= blockDim.x: one pass
    bool f = false;
    int i = threadIdx.x;
    if (i < d) f = ptr[i + 1] > ptr[i];
    unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_cnt[wid] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int q = 0; q < nw; ++q) { if (q < wid) off += warp_cnt[q]; tot += warp_cnt[q]; }
    int idx = off + __popc(bal & ((1u << lane) - 1u));
    if (i < d) {
        if (f) out[idx] = (short)i;
        if (pos) pos[i] = f ? (short)idx : (short)-1;
    }
    if (threadIdx.x == 0) *count = tot;
    __syncthreads();
}

__global__ void __launch_bounds__(LSE_SM_THREADS) sk_lse_smem_kernel(SkWS w, SkRun r, int n_inner, int* active_count,
                                                                      int smem_cap, int* big_count) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ double shd[32];
    __shared__ int cnt[8];
    __shared__ int fits;
    const int p = blockIdx.x, t = threadIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    if (q.ic[IC_STATUS] != ST_ACTIVE || q.ic[IC_BIG]) return;
    const int d = w.d, dp = w.dp, nA = q.ic[IC_NA], nB = q.ic[IC_NB];
    // non-empty rows / columns of both supports (row pointers rpa/rpb, column pointers cpa/cpb)
    short* tmp = reinterpret_cast<short*>(smraw);   // provisional, moved below once the layout is known
    compact_nonempty(q.rpa, d, tmp, &cnt[0], nullptr);
    compact_nonempty(q.cpa, d, tmp, &cnt[1], nullptr);
    compact_nonempty(q.rpb, d, tmp, &cnt[2], nullptr);
    compact_nonempty(q.cpb, d, tmp, &cnt[3], nullptr);
    const int nrA = cnt[0], ncA = cnt[1], nrB = cnt[2], ncB = cnt[3];
    if (t == 0) fits = lse_smem_need(nA, nB, nrA, ncA, nrB, ncB, d, dp) <= (size_t)smem_cap;
    __syncthreads();
    if (!fits) {
        if (t == 0) { q.ic[IC_BIG] = 1; atomicAdd(big_count, 1); }
        return;
    }
    // ---- carve shared memory
    unsigned char* sp = smraw;
    auto take = [&](size_t bytes) { unsigned char* r0 = sp; sp += align_up(bytes, 16); return r0; };
    SideS A, B;
    A.n = nA; B.n = nB; A.nr = nrA; A.nc = ncA; B.nr = nrB; B.nc = ncB;
    A.pot = reinterpret_cast<double*>(take((size_t)(nA + nB) * 8)); B.pot = A.pot + nA;
    A.cell = reinterpret_cast<int*>(take((size_t)(nA + nB) * 16));
    B.cell = A.cell + nA;
    A.lwh = reinterpret_cast<float*>(B.cell + nB); B.lwh = A.lwh + nA;
    A.lwl = B.lwh + nB; B.lwl = A.lwl + nA;
    A.w = B.lwl + nB; B.w = A.w + nA;
    A.rp = reinterpret_cast<int*>(take((size_t)2 * (d + 1) * 4)); B.rp = A.rp + (d + 1);
    short* sh16 = reinterpret_cast<short*>(take((size_t)6 * 256 * 2));
    A.rows = sh16; A.cols = sh16 + 256; A.colpos = sh16 + 512;
    B.rows = sh16 + 768; B.cols = sh16 + 1024; B.colpos = sh16 + 1280;
    float* tab = reinterpret_cast<float*>(take((size_t)4 * dp * 4));
    const int nmax = nA > nB ? nA : nB;
    float* Hh = reinterpret_cast<float*>(take((size_t)nmax * 8));
    float* Hl = Hh + nmax;
    const size_t la = (size_t)nrB * (ncA | 1), lb = (size_t)nrA * (ncB | 1);
    const size_t lmax = la > lb ? la : lb;
    float* Lh = reinterpret_cast<float*>(take(lmax * 8));
    float* Ll = Lh + lmax;
    // ---- load
    compact_nonempty(q.rpa, d, A.rows, &cnt[0], nullptr);
    compact_nonempty(q.cpa, d, A.cols, &cnt[1], A.colpos);
    compact_nonempty(q.rpb, d, B.rows, &cnt[2], nullptr);
    compact_nonempty(q.cpb, d, B.cols, &cnt[3], B.colpos);
    for (int i = t; i <= d; i += blockDim.x) { A.rp[i] = q.rpa[i]; B.rp[i] = q.rpb[i]; }
    for (int e = t; e < nA; e += blockDim.x) {
        int c = q.sa[e];
        A.cell[e] = c; A.pot[e] = q.phi[c]; A.w[e] = q.am[c];
        df l = df_from(q.la[c]); A.lwh[e] = l.hi; A.lwl[e] = l.lo;
    }
    for (int e = t; e < nB; e += blockDim.x) {
        int c = q.sb[e];
        B.cell[e] = c; B.pot[e] = q.psi[c]; B.w[e] = q.bm[c];
        df l = df_from(q.lb[c]); B.lwh[e] = l.hi; B.lwl[e] = l.lo;
    }
    for (int m = t; m < 4 * dp; m += blockDim.x) tab[m] = w.ctab[m];
    A.wD = q.sc[SC_AD]; B.wD = q.sc[SC_BD];
    A.lD = A.wD > 0 ? log(A.wD) : -INFINITY; B.lD = B.wD > 0 ? log(B.wD) : -INFINITY;
    A.potD = q.phi[w.n - 1]; B.potD = q.psi[w.n - 1];
    __syncthreads();
    const float *chi = tab, *clo = tab + dp, *chi2 = tab + 2 * dp, *clo2 = tab + 3 * dp;
    const double total = q.sc[SC_TOTAL];
    int iters = q.ic[IC_ITERS];
    double err = q.sc[SC_ERR];
    int status = ST_ACTIVE;
    for (int it = 0; it < n_inner; ++it) {
        sm_halfstep(B, A, Hh, Hl, Lh, Ll, chi, clo, chi2, clo2, dp, false, shd);   // u-update: phi from psi
        err = sm_halfstep(A, B, Hh, Hl, Lh, Ll, chi, clo, chi2, clo2, dp, true, shd) / total;  // v-update
        ++iters;
        if (r.tol > 0 && err <= r.tol) { status = ST_CONVERGED; break; }
        if (iters >= r.max_iter) { status = ST_MAXITER; break; }
        if (!isfinite(err)) { status = ST_RANGE; break; }
    }
    // ---- store
    for (int e = t; e < nA; e += blockDim.x) q.phi[A.cell[e]] = A.pot[e];
    for (int e = t; e < nB; e += blockDim.x) q.psi[B.cell[e]] = B.pot[e];
    if (t == 0) {
        q.phi[w.n - 1] = A.potD; q.psi[w.n - 1] = B.potD;
        q.sc[SC_ERR] = err;
        q.ic[IC_ITERS] = iters;
        q.ic[IC_STATUS] = status;
        if (status == ST_ACTIVE) atomicAdd(active_count, 1);
    }
}

cudaError_t sk_launch_lse_smem(const SkWS& w, SkRun r, int n_inner, int* active_count, int* big_count,
                               cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    static std::atomic<int> configured{-1};
    int dev = 0;
    cudaGetDevice(&dev);
    int cap = 0;
    cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cap -= 2048;   // static shared memory of the kernel
    if (configured != cap) {
        cudaError_t e = cudaFuncSetAttribute(sk_lse_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
        if (e != cudaSuccess) return e;
        configured = cap;
    }
    sk_lse_smem_kernel<<<w.P, LSE_SM_THREADS, cap, s>>>(w, r, n_inner, active_count, cap, big_count);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Prop. 3: cost of the rounded plan R (the rounding algorithm of the
// supplementary, after Altschuler et al.) from the final potentials, without
// forming any plan.  Write phi_u(psi) = -log(K (b e^psi)) for the value the
// u-update would give and psi_v(phi) = -log(K^T (a e^phi)) for the v-update.
// The row marginal of P is r(P) = a e^(phi - phi_u(psi)), so
//   X = min(a / r(P), 1)          <=>  phi1 = min(phi, phi_u(psi)),
//   c(diag(X) P) = b e^(psi - psi_v(phi1)),
//   Y = min(b / c(diag(X) P), 1)  <=>  psi2 = min(psi, psi_v(phi1)),
//   e_c = b - c(P2) = b max(0, 1 - e^(psi - psi_v(phi1))),
//   e_r = a - r(P2) = a (1 - e^(phi1 - phi_u(psi2))),
// with P2 = diag(X) P diag(Y), and <R, C> = <P2, C> + e_r^T C e_c / |e_c|_1.
// <P2, C> is Prop. 2 with the potentials (phi1, psi2), which this kernel
// leaves in place of (phi, psi).  The rank-one term uses the separable cost:
// sum_{x,y} e_r(x) e_c(y) C(x,y) = sum_{ik} c_ik ER_i EC_k + sum_{jl} c_jl
// ER'_j EC'_l (row / column sums of the grid parts) + e_c(Delta) <e_r, cD> +
// e_r(Delta) <e_c, cD>.
__global__ void __launch_bounds__(T_CTA) sk_round_bound_kernel(SkWS w) {
    __shared__ int rows[256], cols[256], nrc[2];
    __shared__ double shd[32];
    __shared__ double sums[4][256];   // e_r row sums, e_r column sums, e_c row sums, e_c column sums
    __shared__ double dval[2];
    const int p = blockIdx.x, t = threadIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    const int st = q.ic[IC_STATUS];
    if (t == 0) q.sc[SC_CORR] = 0.0;
    if (!((st == ST_CONVERGED || st == ST_MAXITER) && q.sc[SC_TOTAL] > 0)) return;
    const int d = w.d, dp = w.dp, n1 = w.n - 1, na = q.ic[IC_NA], nb = q.ic[IC_NB];
    const float* chi = w.ctab;
    const float* clo = w.ctab + dp;
    const float* chi2 = w.ctab + 2 * dp;
    const float* clo2 = w.ctab + 3 * dp;
    double* S1 = q.L64;                       // [dp*dp] u-side values by padded cell
    double* S2 = q.L64 + (size_t)dp * dp;     // [dp*dp] v-side values
    const double aD = q.sc[SC_AD], bD = q.sc[SC_BD];
    for (int i = t; i < 4 * 256; i += blockDim.x) (&sums[0][0])[i] = 0.0;
    // ---- phi_u(psi), then phi1 = min(phi, phi_u(psi))
    {
        HalfArgs ua = u_args(q, w);
        ua.pout = S1;
        ua.pD_out = &dval[0];
        if (t == 0) dval[0] = q.phi[n1];
        __syncthreads();
        lse_halfstep(ua, chi, clo, chi2, clo2, d, dp, rows, cols, nrc, false, shd);
        for (int e = t; e < na; e += blockDim.x) {
            const int c = q.sa[e];
            q.phi[c] = fmin(q.phi[c], S1[c]);
        }
        if (t == 0 && aD > 0) q.phi[n1] = fmin(q.phi[n1], dval[0]);
        __syncthreads();
    }
    // ---- psi_v(phi1), e_c, then psi2 = min(psi, psi_v(phi1))
    double ec_sum = 0.0, ec_cd = 0.0, ecD = 0.0;
    {
        HalfArgs va = v_args(q, w);
        va.pout = S2;
        va.pD_out = &dval[1];
        if (t == 0) dval[1] = q.psi[n1];
        __syncthreads();
        lse_halfstep(va, chi, clo, chi2, clo2, d, dp, rows, cols, nrc, false, shd);
        for (int e = t; e < nb; e += blockDim.x) {
            const int c = q.sb[e], k = c / dp, l = c % dp;
            const double ec = exp(q.lb[c]) * fmax(0.0, -expm1(q.psi[c] - S2[c]));
            ec_sum += ec;
            ec_cd += ec * pd_cdiagp(k, l, d, w.p);
            atomicAdd(&sums[2][k], ec);
            atomicAdd(&sums[3][l], ec);
            q.psi[c] = fmin(q.psi[c], S2[c]);
        }
        if (bD > 0) ecD = bD * fmax(0.0, -expm1(q.psi[n1] - dval[1]));
        __syncthreads();
        if (t == 0 && bD > 0) q.psi[n1] = fmin(q.psi[n1], dval[1]);
        __syncthreads();
    }
    // ---- phi_u(psi2), e_r
    double er_cd = 0.0, erD = 0.0;
    {
        HalfArgs ua = u_args(q, w);
        ua.pout = S1;
        ua.pD_out = &dval[0];
        __syncthreads();
        lse_halfstep(ua, chi, clo, chi2, clo2, d, dp, rows, cols, nrc, false, shd);
        for (int e = t; e < na; e += blockDim.x) {
            const int c = q.sa[e], i = c / dp, j = c % dp;
            const double er = exp(q.la[c]) * fmax(0.0, -expm1(q.phi[c] - S1[c]));
            er_cd += er * pd_cdiagp(i, j, d, w.p);
            atomicAdd(&sums[0][i], er);
            atomicAdd(&sums[1][j], er);
        }
        if (aD > 0) erD = aD * fmax(0.0, -expm1(q.phi[n1] - dval[0]));
        __syncthreads();
    }
    // ---- rank-one term
    double bil = 0.0;
    for (int e = t; e < d * d; e += blockDim.x) {
        const int i = e / d, k = e % d;
        bil += pd_c1p(i, k, d, w.p) * (sums[0][i] * sums[2][k] + sums[1][i] * sums[3][k]);
    }
    bil = block_sum(bil, shd);
    ec_sum = block_sum(ec_sum, shd);
    ec_cd = block_sum(ec_cd, shd);
    er_cd = block_sum(er_cd, shd);
    if (t == 0) {
        const double ec_tot = ec_sum + ecD;
        const double num = bil + ecD * er_cd + erD * ec_cd;
        q.sc[SC_CORR] = ec_tot > 0 ? num / ec_tot : 0.0;
    }
}

__global__ void sk_add_corr_kernel(SkWS w, double* __restrict__ upper) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < w.P) upper[p] += w.sc[(size_t)p * SC_N + SC_CORR];
}

cudaError_t sk_launch_round_bound(const SkWS& w, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_round_bound_kernel<<<w.P, T_CTA, 0, s>>>(w);
    return cudaGetLastError();
}
cudaError_t sk_launch_add_corr(const SkWS& w, double* upper, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_add_corr_kernel<<<(w.P + 255) / 256, 256, 0, s>>>(w, upper);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// gamma-continuation step (see sk_launch_regamma): phi, psi hold f/gamma and
// g/gamma; a new gamma keeps f and g, so both scale by old/new.  Pairs that
// stopped (converged or at max_iter of the stage) are made active again unless
// they are invalid, out of range, have no mass, or used up max_iter.
__global__ void sk_regamma_kernel(SkWS w, double ratio, int max_iter) {
    const int p = blockIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    const int st = q.ic[IC_STATUS];
    if (st == ST_INVALID || st == ST_RANGE || !(q.sc[SC_TOTAL] > 0)) return;
    const int na = q.ic[IC_NA], nb = q.ic[IC_NB];
    for (int e = threadIdx.x; e < na; e += blockDim.x) q.phi[q.sa[e]] *= ratio;
    for (int e = threadIdx.x; e < nb; e += blockDim.x) q.psi[q.sb[e]] *= ratio;
    if (threadIdx.x == 0) {
        q.phi[w.n - 1] *= ratio;
        q.psi[w.n - 1] *= ratio;
        if (q.ic[IC_ITERS] < max_iter) {
            q.ic[IC_STATUS] = ST_ACTIVE;
            q.sc[SC_ERR] = INFINITY;
        }
    }
}

cudaError_t sk_launch_regamma(const SkWS& w, double ratio, int max_iter, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_regamma_kernel<<<w.P, 128, 0, s>>>(w, ratio, max_iter);
    return cudaGetLastError();
}
