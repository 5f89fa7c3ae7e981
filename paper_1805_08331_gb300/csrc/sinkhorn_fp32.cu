// sinkhorn_fp32.cu -- batched Sinkhorn for persistence diagrams (Alg. 1) with
// the separable kernel of Prop. 1 applied by CUDA-core FP32 GEMMs, log-domain
// stabilisation by separable absorption, and the transport cost of Prop. 2.
//
// Representation (per pair).  With u = a*exp(phi), v = b*exp(psi) (phi =
// f/gamma, psi = g/gamma) the potentials are split into an absorbed part that
// is SEPARABLE on the grid plus a residual scaling:
//     u_x = exp(Fb_x) * ut_x,   Fb_(i,j) = ap_i + bp_j,   Fb_Delta = FD
//     v_y = exp(Gb_y) * vt_y,   Gb_(k,l) = al_k + be_l,   Gb_Delta = GD
// so the absorbed kernel Kt_xy = exp(Fb_x + Gb_y - C_xy/gamma) stays a Kronecker
// product on the grid block (C_xy = c_ik + c_jl, Sec. 3 "Convolutions"):
//     Kt_(ij),(kl) = exp(ap_i + al_k - c_ik/gamma) * exp(bp_j + be_l - c_jl/gamma)
// and every kernel application is two d x d x d GEMMs (Prop. 1) plus the
// rank-one Delta terms.  Schmitzer-style absorption of the residual into the
// potentials keeps ut, vt near a, b; the separable part is re-fitted by least
// squares on the supports at each absorption.  The intermediate of the two
// GEMMs gets its own separable shift (Au, Bu), fitted on the entries that
// contribute to an output on the support, so every term that matters stays in
// FP32 range.
//
// u-update (v -> u):   Wt = rs_u .* (vt * K1u^T)         [k,j]
//                      R  = K2u * Wt                        [i,j]
//                      ut = a ./ (cf_u[j] R + KDu vt_Delta)
//   K1u[j,l] = exp(be_l - c_jl/g - Bu_j), K2u[i,k] = exp(ap_i + Au_k - c_ik/g),
//   rs_u[k] = exp(al_k - Au_k),           cf_u[j] = exp(bp_j + Bu_j).
// v-update symmetric with (K1v, K2v, rs_v, cf_v, Av, Bv).
#include "sk_common.cuh"

// ---------------------------------------------------------------------------
// CTA-wide FP32 GEMM, "NT" form: C(m,n) = sum_k A[m*dp+k] * B[n*dp+k] for
// m, n, k < dp (dp a multiple of 64).  256 threads, 64x64 output tiles, each
// thread a 4x4 register tile; K staged through shared memory in steps of 32.
// ATr/BTr transform loaded elements (identity for plain GEMMs); Epi receives
// every output element.
struct Ident { __device__ float operator()(int, int, float v) const { return v; } };

template <class ATr, class BTr, class Epi>
__device__ void cta_gemm_nt(const float* __restrict__ A, const float* __restrict__ B, int dp, ATr atr,
                            BTr btr, Epi epi, float* sm) {
    float* sA = sm;              // [32][68]
    float* sB = sm + 32 * 68;    // [32][68]
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    for (int m0 = 0; m0 < dp; m0 += 64) {
        for (int n0 = 0; n0 < dp; n0 += 64) {
            float acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
            for (int k0 = 0; k0 < dp; k0 += 32) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    int idx = t + 256 * e, r = idx >> 3, q = idx & 7;
                    float4 va = *reinterpret_cast<const float4*>(A + (size_t)(m0 + r) * dp + k0 + 4 * q);
                    float4 vb = *reinterpret_cast<const float4*>(B + (size_t)(n0 + r) * dp + k0 + 4 * q);
                    int kk = k0 + 4 * q;
                    sA[(4 * q + 0) * 68 + r] = atr(m0 + r, kk + 0, va.x);
                    sA[(4 * q + 1) * 68 + r] = atr(m0 + r, kk + 1, va.y);
                    sA[(4 * q + 2) * 68 + r] = atr(m0 + r, kk + 2, va.z);
                    sA[(4 * q + 3) * 68 + r] = atr(m0 + r, kk + 3, va.w);
                    sB[(4 * q + 0) * 68 + r] = btr(n0 + r, kk + 0, vb.x);
                    sB[(4 * q + 1) * 68 + r] = btr(n0 + r, kk + 1, vb.y);
                    sB[(4 * q + 2) * 68 + r] = btr(n0 + r, kk + 2, vb.z);
                    sB[(4 * q + 3) * 68 + r] = btr(n0 + r, kk + 3, vb.w);
                }
                __syncthreads();
#pragma unroll 8
                for (int kk = 0; kk < 32; ++kk) {
                    float4 a4 = *reinterpret_cast<const float4*>(sA + kk * 68 + ty * 4);
                    float4 b4 = *reinterpret_cast<const float4*>(sB + kk * 68 + tx * 4);
                    float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
                }
                __syncthreads();
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) epi(m0 + ty * 4 + a, n0 + tx * 4 + b, acc[a][b]);
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Setup: dense a, b, support lists (row- and column-major), initial psi.
__device__ void build_lists(const float* m, int d, int dp, int* list, int* rowptr, int* colptr,
                            int* colrows, int* cnt_out, int* sh) {
    // row-major compaction (order preserved) using warp ballots
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    int base = 0;
    for (int c0 = 0; c0 < d * d; c0 += blockDim.x) {
        int c = c0 + t;
        bool f = false;
        int cell = 0;
        if (c < d * d) { int i = c / d, j = c % d; cell = i * dp + j; f = m[cell] > 0.f; }
        unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) sh[wid] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int q = 0; q < nw; ++q) { if (q < wid) off += sh[q]; tot += sh[q]; }
        if (f) list[base + off + __popc(bal & ((1u << lane) - 1u))] = cell;
        base += tot;
        __syncthreads();
    }
    if (t == 0) *cnt_out = base;
    // row pointers: count per row
    for (int i = t; i <= d; i += blockDim.x) rowptr[i] = 0;
    for (int i = t; i <= d; i += blockDim.x) colptr[i] = 0;
    __syncthreads();
    for (int q = t; q < base; q += blockDim.x) {
        int cell = list[q];
        atomicAdd(&rowptr[cell / dp + 1], 1);
        atomicAdd(&colptr[cell % dp + 1], 1);
    }
    __syncthreads();
    if (t == 0) {
        for (int i = 0; i < d; ++i) rowptr[i + 1] += rowptr[i];
        for (int j = 0; j < d; ++j) colptr[j + 1] += colptr[j];
    }
    __syncthreads();
    // column-major row indices: thread per column walks the rows in order
    for (int j = t; j < d; j += blockDim.x) {
        int w = colptr[j];
        for (int i = 0; i < d; ++i)
            if (m[i * dp + j] > 0.f) colrows[w++] = i;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(T_CTA) sk_setup_kernel(SkWS w, const double* __restrict__ g_init,
                                                         const int* __restrict__ plist) {
    __shared__ int sh[64];
    __shared__ double shd[32];
    const int p = plist ? plist[blockIdx.x] : blockIdx.x, t = threadIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    const int d = w.d, dp = w.dp;
    int ia = w.pairs ? w.pairs[2 * p] : p, ib = w.pairs ? w.pairs[2 * p + 1] : p;
    const uint32_t* hA = w.histA ? w.histA + (size_t)ia * d * d : nullptr;
    const uint32_t* hB = w.histB ? w.histB + (size_t)ib * d * d : nullptr;
    const double* rA = w.wA ? w.wA + (size_t)ia * d * d : nullptr;
    const double* rB = w.wB ? w.wB + (size_t)ib * d * d : nullptr;
    double sA = 0, sB = 0;
    for (int c = t; c < dp * dp; c += blockDim.x) {
        int i = c / dp, j = c % dp;
        double va = 0.0, vb = 0.0;
        if (i < d && j < d) {
            va = rA ? rA[i * d + j] : (double)hA[i * d + j];
            vb = rB ? rB[i * d + j] : (double)hB[i * d + j];
            if (!(va >= 0.0)) va = 0.0;   // negative / NaN weights are treated as 0 (validated on the host)
            if (!(vb >= 0.0)) vb = 0.0;
            sA += va; sB += vb;
        }
        q.am[c] = (float)va; q.bm[c] = (float)vb; q.ut[c] = 0.f; q.vt[c] = 0.f;
        q.la[c] = va > 0.0 ? log(va) : -INFINITY;
        q.lb[c] = vb > 0.0 ? log(vb) : -INFINITY;
    }
    sA = block_sum(sA, shd);
    sB = block_sum(sB, shd);
    __syncthreads();
    build_lists(q.am, d, dp, q.sa, q.rpa, q.cpa, q.cia, &q.ic[IC_NA], sh);
    build_lists(q.bm, d, dp, q.sb, q.rpb, q.cpb, q.cib, &q.ic[IC_NB], sh);
    const double nA = rA ? sA : (double)w.massA[ia], nB = rB ? sB : (double)w.massB[ib];
    for (int x = t; x < w.n; x += blockDim.x) { q.phi[x] = 0.0; q.psi[x] = 0.0; }
    __syncthreads();
    if (g_init) {
        const double* gi = g_init + (size_t)p * (d * d + 1);
        for (int c = t; c < d * d; c += blockDim.x) {
            int i = c / d, j = c % d;
            q.psi[i * dp + j] = gi[c] / w.gamma;   // psi stored at padded index for grid cells
        }
        if (t == 0) q.psi[w.n - 1] = gi[d * d] / w.gamma;
    }
    if (t == 0) {
        q.sc[SC_FD] = 0; q.sc[SC_GD] = 0; q.sc[SC_UTD] = 0; q.sc[SC_VTD] = 0; q.sc[SC_DD] = 0;
        q.sc[SC_AD] = nB; q.sc[SC_BD] = nA; q.sc[SC_TOTAL] = nA + nB; q.sc[SC_ERR] = INFINITY;
        q.ic[IC_ITERS] = 0; q.ic[IC_ABSORB] = 1; q.ic[IC_FROMLIN] = 0; q.ic[IC_RANGE] = 0; q.ic[IC_BIG] = 0;
        q.ic[IC_STAGE] = 0;
        int st = ST_ACTIVE;
        if ((!rA && sA != nA) || (!rB && sB != nB)) st = ST_INVALID;
        else if (nA + nB == 0) { st = ST_CONVERGED; q.sc[SC_ERR] = 0; }
        q.ic[IC_STATUS] = st;
    }
}

// phi/psi address grid cells by the padded index i*dp + j and hold dp*dp + 1
// entries (w.n = dp*dp + 1); the Delta entry is index n - 1.

cudaError_t sk_launch_setup(const SkWS& w, const double* g_init, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_setup_kernel<<<w.P, T_CTA, 0, s>>>(w, g_init, nullptr);
    return cudaGetLastError();
}
// Set-up of the pairs plist[0..np) only (the others keep their state).
cudaError_t sk_launch_setup_list(const SkWS& w, const double* g_init, const int* plist, int np, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    sk_setup_kernel<<<np, T_CTA, 0, s>>>(w, g_init, plist);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Separable log-domain half-step (exact up to FP64 rounding):
//   out_x = -log( sum_y wgt_y exp(h_y - C_xy/gamma) ),  x in out-support
// with h = log-potential of the input side (psi for the u-update).  Evaluated
// through the Kronecker structure: L[k,j] = LSE_{l in row k} (log w_kl + h_kl
// - c_jl/g), then out_(i,j) = -LSE_k (L[k,j] - c_ik/g) (+) (log w_D + h_D -
// cD_(i,j)/g).  Maxima and sums in FP64, exponentials of centred arguments in
// FP32.  `L` is FP64 dp*dp scratch.
__device__ void log_halfstep(const float* __restrict__ win, const double* __restrict__ hin,
                             const int* __restrict__ rpin, const int* __restrict__ listin, double wD,
                             double hD, const int* __restrict__ listout, int nout, double* __restrict__ out,
                             double* __restrict__ outD, const float* __restrict__ wout_for_D, double* L,
                             int d, int dp, double ginv, int nin, int* __restrict__ rowsin, int* nrows_sh) {
    const int t = threadIdx.x;
    // nonempty input rows
    if (t == 0) {
        int c = 0;
        for (int k = 0; k < d; ++k) if (rpin[k + 1] > rpin[k]) rowsin[c++] = k;
        *nrows_sh = c;
    }
    __syncthreads();
    const int nr = *nrows_sh;
    // stage 1: L[k,j] for nonempty rows k, all j < d
    for (int e = t; e < nr * d; e += blockDim.x) {
        int k = rowsin[e / d], j = e % d;
        double mx = -INFINITY;
        for (int q = rpin[k]; q < rpin[k + 1]; ++q) {
            int cell = listin[q], l = cell % dp;
            double a = log((double)win[cell]) + hin[cell] - pd_c1(j, l, d) * ginv;
            mx = fmax(mx, a);
        }
        double s = 0.0;
        for (int q = rpin[k]; q < rpin[k + 1]; ++q) {
            int cell = listin[q], l = cell % dp;
            double a = log((double)win[cell]) + hin[cell] - pd_c1(j, l, d) * ginv;
            s += (double)expf((float)(a - mx));
        }
        L[k * dp + j] = mx + log(s);
    }
    __syncthreads();
    // stage 2: outputs on the out-support
    const double lwD = (wD > 0) ? log(wD) + hD : -INFINITY;
    for (int e = t; e < nout; e += blockDim.x) {
        int cell = listout[e], i = cell / dp, j = cell % dp;
        double mx = lwD - pd_cdiag(i, j, d) * ginv;
        for (int r = 0; r < nr; ++r) { int k = rowsin[r]; mx = fmax(mx, L[k * dp + j] - pd_c1(i, k, d) * ginv); }
        double s = (lwD > -INFINITY) ? (double)expf((float)(lwD - pd_cdiag(i, j, d) * ginv - mx)) : 0.0;
        for (int r = 0; r < nr; ++r) { int k = rowsin[r]; s += (double)expf((float)(L[k * dp + j] - pd_c1(i, k, d) * ginv - mx)); }
        out[cell] = -(mx + log(s));
    }
    // Delta output: -LSE_y (log w_y + h_y - cD_y/g) (+) (log w_D + h_D)
    __shared__ double shd[32];
    double mx = -INFINITY;
    for (int q = t; q < nin; q += blockDim.x) {
        int cell = listin[q];
        mx = fmax(mx, log((double)win[cell]) + hin[cell] - pd_cdiag(cell / dp, cell % dp, d) * ginv);
    }
    mx = block_max(mx, shd, (double)-INFINITY);
    mx = fmax(mx, lwD);
    double s = 0.0;
    for (int q = t; q < nin; q += blockDim.x) {
        int cell = listin[q];
        s += (double)expf((float)(log((double)win[cell]) + hin[cell] - pd_cdiag(cell / dp, cell % dp, d) * ginv - mx));
    }
    s = block_sum(s, shd);
    if (t == 0) {
        if (lwD > -INFINITY) s += (double)expf((float)(lwD - mx));
        *outD = (mx > -INFINITY) ? -(mx + log(s)) : INFINITY;
    }
    __syncthreads();
}

// First iteration, exact in the log domain: phi_1 from psi_0, err_1, psi_1.
__global__ void __launch_bounds__(T_CTA) sk_logstep_kernel(SkWS w, SkRun r) {
    __shared__ int nrows;
    __shared__ int rows[256];
    __shared__ double shd[32];
    const int p = blockIdx.x, t = threadIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    if (q.ic[IC_STATUS] != ST_ACTIVE) return;
    const int d = w.d, dp = w.dp, na = q.ic[IC_NA], nb = q.ic[IC_NB];
    const double ginv = 1.0 / w.gamma, aD = q.sc[SC_AD], bD = q.sc[SC_BD];
    double* phiD = &q.phi[w.n - 1];
    double* psiD = &q.psi[w.n - 1];
    // u-update from psi_0
    log_halfstep(q.bm, q.psi, q.rpb, q.sb, bD, *psiD, q.sa, na, q.phi, phiD, q.am, q.L64, d, dp, ginv, nb,
                 rows, &nrows);
    // v-update from phi_1, with the column error of (phi_1, psi_0): the new psi_1
    // satisfies v_1 (K^T u_1) = b, so v_0 (K^T u_1) = b exp(psi_0 - psi_1).
    __shared__ double psi0D;
    if (t == 0) psi0D = *psiD;
    __syncthreads();
    double* psi0 = q.L64;   // first half of L64 is free once the u-update is done
    for (int e = t; e < nb; e += blockDim.x) psi0[e] = q.psi[q.sb[e]];
    __syncthreads();
    log_halfstep(q.am, q.phi, q.rpa, q.sa, aD, *phiD, q.sb, nb, q.psi, psiD, q.bm,
                 q.L64 + (size_t)dp * dp, d, dp, ginv, na, rows, &nrows);
    double e = 0.0;
    for (int k = t; k < nb; k += blockDim.x) {
        int cell = q.sb[k];
        e += (double)q.bm[cell] * fabs(expm1(psi0[k] - q.psi[cell]));
    }
    e = block_sum(e, shd);
    if (t == 0) {
        if (bD > 0) e += bD * fabs(expm1(psi0D - *psiD));
        double err = e / q.sc[SC_TOTAL];
        q.sc[SC_ERR] = err;
        q.ic[IC_ITERS] = 1;
        q.ic[IC_ABSORB] = 1;
        q.ic[IC_FROMLIN] = 0;
        if (r.tol > 0 && err <= r.tol) q.ic[IC_STATUS] = ST_CONVERGED;
        else if (r.max_iter <= 1) q.ic[IC_STATUS] = ST_MAXITER;
    }
}
// L64 holds 2*dp*dp doubles per pair: the second half-step's stage-1 scratch
// is the upper half, the saved psi_0 the start of the lower half.

cudaError_t sk_launch_logstep(const SkWS& w, SkRun r, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_logstep_kernel<<<w.P, T_CTA, 0, s>>>(w, r);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Least-squares separable fits (alternating means), computed in FP32 and
// rounded to FP32-representable shifts.  Rows/columns without data take the
// value of the nearest row/column that has data (they only need to be finite).
__device__ void fill_nearest(float* v, const int* cnt, int d) {
    __syncthreads();
    float* tmp = v + 256;   // caller provides 512 floats
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        float r = 0.f;
        if (cnt[i] > 0) r = v[i];
        else {
            for (int s = 1; s < d; ++s) {
                if (i - s >= 0 && cnt[i - s] > 0) { r = v[i - s]; break; }
                if (i + s < d && cnt[i + s] > 0) { r = v[i + s]; break; }
            }
        }
        tmp[i] = r;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d; i += blockDim.x) v[i] = tmp[i];
    __syncthreads();
}

// Fit val[cell] ~ al[i] + be[j] over a support given in CSR (rows) and CSC
// (columns) form by alternating row / column MIDRANGES of the residual, which
// centres the residual's range (what must fit the FP32 exponent range) rather
// than its mean.  al, be: shared float[512] each; rc, cc: shared int[256].
__device__ void fit_sparse(const double* __restrict__ val, const int* __restrict__ rowptr,
                          const int* __restrict__ list, const int* __restrict__ colptr,
                          const int* __restrict__ colrows, int d, int dp, float* al, float* be, int* rc,
                          int* cc, int sweeps) {
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        al[i] = 0.f; be[i] = 0.f;
        rc[i] = rowptr[i + 1] - rowptr[i];
        cc[i] = colptr[i + 1] - colptr[i];
    }
    __syncthreads();
    for (int s = 0; s < sweeps; ++s) {
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            if (rc[i]) {
                float lo = INFINITY, hi = -INFINITY;
                for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
                    int c = list[q];
                    float r = (float)val[c] - be[c % dp];
                    lo = fminf(lo, r); hi = fmaxf(hi, r);
                }
                al[i] = 0.5f * (lo + hi);
            }
        }
        __syncthreads();
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            if (cc[j]) {
                float lo = INFINITY, hi = -INFINITY;
                for (int q = colptr[j]; q < colptr[j + 1]; ++q) {
                    int i = colrows[q];
                    float r = (float)val[i * dp + j] - al[i];
                    lo = fminf(lo, r); hi = fmaxf(hi, r);
                }
                be[j] = 0.5f * (lo + hi);
            }
        }
        __syncthreads();
    }
    fill_nearest(al, rc, d);
    fill_nearest(be, cc, d);
}

// Midrange fit L[k*dp+j] ~ al[k] + be[j] over entries with rel[k*dp+j] > thr.
__device__ void fit_masked(const float* __restrict__ L, const float* __restrict__ rel, float thr, int d, int dp,
                           float* al, float* be, int* rc, int* cc, int sweeps) {
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        al[i] = 0.f; be[i] = 0.f;
        int n = 0;
        for (int j = 0; j < d; ++j) n += rel[i * dp + j] > thr;
        rc[i] = n;
        int m = 0;
        for (int k = 0; k < d; ++k) m += rel[k * dp + i] > thr;
        cc[i] = m;
    }
    __syncthreads();
    for (int s = 0; s < sweeps; ++s) {
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            if (rc[i]) {
                float lo = INFINITY, hi = -INFINITY;
                for (int j = 0; j < d; ++j)
                    if (rel[i * dp + j] > thr) { float r = L[i * dp + j] - be[j]; lo = fminf(lo, r); hi = fmaxf(hi, r); }
                al[i] = 0.5f * (lo + hi);
            }
        }
        __syncthreads();
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            if (cc[j]) {
                float lo = INFINITY, hi = -INFINITY;
                for (int k = 0; k < d; ++k)
                    if (rel[k * dp + j] > thr) { float r = L[k * dp + j] - al[k]; lo = fminf(lo, r); hi = fmaxf(hi, r); }
                be[j] = 0.5f * (lo + hi);
            }
        }
        __syncthreads();
    }
    fill_nearest(al, rc, d);
    fill_nearest(be, cc, d);
}

// Min-max balancing of the factors of one kernel application (named for the
// u-update; the v-update passes its own arrays in the same roles).  The terms
// that matter are those within exp(thr) of their sum:
//   output-relevant (i,k,j): x=(i,j) on the out-support, -c_ik/g + L[k,j] - LO[x] > thr
//   intermediate-relevant (k,j): rel[k,j] > thr
//   GEMM1-relevant (k,l,j): (k,j) relevant, l in row k of the input support,
//                           lw[k,l] - c_jl/g - L[k,j] > thr   (lw = log w + h)
// Their factors, in log units:
//   K2[i,k] = oa_i + A_k - c_ik/g        W[k,j] = L[k,j] - A_k - B_j
//   cf[j]   = ob_j + B_j                 K1[j,l] = ib_l - B_j - c_jl/g
//   GEMM1 operand row k: rs[k] * vt[k,l] = lw[k,l] - ib_l - A_k
// A row shift of A_k moves range between K2 (+) and W, operand (-); a column
// shift of B_j between cf (+) and W, K1 (-).  Each round picks, per row then
// per column, the shift minimising the largest |log factor| it touches (the
// largest entry of K1's row is also kept below e^80+M).  A, B: shared floats.
__device__ void balance(const float* __restrict__ L, const float* __restrict__ LO, const float* __restrict__ rel,
                        const int* __restrict__ outlist, int nout, const int* __restrict__ outcp,
                        const int* __restrict__ outcr, const float* __restrict__ win, const double* __restrict__ hin,
                        const int* __restrict__ rpin, const int* __restrict__ listin,
                        const double* __restrict__ oa, const double* __restrict__ ob, const double* __restrict__ ib,
                        float* A, float* B, const int* rows, int nr, int d, int dp, float ginv, float thr,
                        int rounds) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float invd = 1.0f / d;
    for (int rd = 0; rd < rounds; ++rd) {
        // rows k (warp per row)
        for (int r = wid; r < nr; r += nw) {
            const int k = rows[r];
            const float Ak = A[k];
            float ulo = INFINITY, uhi = -INFINITY, dlo = INFINITY, dhi = -INFINITY;
            for (int e = lane; e < nout; e += 32) {          // K2 column k
                int cell = outlist[e], i = cell / dp, j = cell % dp;
                float dk = (i - k) * invd, cik = dk * dk * ginv;
                if (-cik + L[k * dp + j] - LO[cell] > thr) {
                    float k2 = (float)oa[i] + Ak - cik;
                    ulo = fminf(ulo, k2); uhi = fmaxf(uhi, k2);
                }
            }
            for (int j = lane; j < d; j += 32) {             // W row k
                if (rel[k * dp + j] > thr) {
                    float w = L[k * dp + j] - Ak - B[j];
                    dlo = fminf(dlo, w); dhi = fmaxf(dhi, w);
                }
            }
            for (int q = rpin[k] + lane; q < rpin[k + 1]; q += 32) {   // GEMM1 operand row k
                int cell = listin[q];
                float op = logf(win[cell]) + (float)hin[cell] - (float)ib[cell % dp] - Ak;
                dlo = fminf(dlo, op); dhi = fmaxf(dhi, op);
            }
            ulo = -warp_max(-ulo); uhi = warp_max(uhi); dlo = -warp_max(-dlo); dhi = warp_max(dhi);
            if (lane == 0 && (uhi > -INFINITY || dhi > -INFINITY)) {
                float inc = fmaxf(uhi, -dlo), dec = fmaxf(-ulo, dhi);
                A[k] = Ak + 0.5f * (dec - inc);
            }
        }
        __syncthreads();
        // columns j of the out-support (warp per column)
        for (int j = wid; j < d; j += nw) {
            if (outcp[j + 1] == outcp[j]) continue;
            const float Bj = B[j];
            float dlo = INFINITY, dhi = -INFINITY, k1 = -INFINITY;
            for (int r = 0; r < nr; ++r) {
                const int k = rows[r];
                if (!(rel[k * dp + j] > thr)) continue;
                const float Lkj = L[k * dp + j];
                if (lane == 0) { float w = Lkj - A[k] - Bj; dlo = fminf(dlo, w); dhi = fmaxf(dhi, w); }
                for (int q = rpin[k] + lane; q < rpin[k + 1]; q += 32) {
                    int cell = listin[q], l = cell % dp;
                    float dl = (j - l) * invd, cjl = dl * dl * ginv;
                    if (logf(win[cell]) + (float)hin[cell] - cjl - Lkj > thr) {
                        float k1v = (float)ib[l] - Bj - cjl;
                        dlo = fminf(dlo, k1v); dhi = fmaxf(dhi, k1v);
                    }
                }
            }
            for (int l = lane; l < d; l += 32) {
                float dl = (j - l) * invd;
                k1 = fmaxf(k1, (float)ib[l] - Bj - dl * dl * ginv);
            }
            dlo = -warp_max(-dlo); dhi = warp_max(dhi); k1 = warp_max(k1);
            if (lane == 0) {
                float z = (float)ob[j] + Bj;
                float inc = (dlo < INFINITY) ? fmaxf(z, -dlo) : z;
                float dec = (dhi > -INFINITY) ? fmaxf(fmaxf(-z, dhi), k1 - 80.f) : fmaxf(-z, k1 - 80.f);
                B[j] = Bj + 0.5f * (dec - inc);
            }
        }
        __syncthreads();
    }
}

// Relevance of the GEMM intermediate (FP32 log domain).
//   L[k,j]  = LSE_{l in row k of the input support} (log w_kl + h_kl - c_jl/g)
//   LO[x]   = LSE_k (L[k,j] - c_ik/g) (+) (log w_D + h_D - cD_x/g),  x=(i,j) in out support
//   rel[k,j] = max_{i: (i,j) in out support} (L[k,j] - c_ik/g - LO[i,j])
// L -> Lbuf, LO -> LObuf (at cell index), rel -> relbuf (-inf where irrelevant).
__device__ void relevance(const float* __restrict__ win, const double* __restrict__ hin, const int* __restrict__ rpin,
                          const int* __restrict__ listin, double lwD, const int* __restrict__ listout, int nout,
                          const int* __restrict__ cpout, const int* __restrict__ crout, int d, int dp, float ginv,
                          float* __restrict__ Lbuf, float* __restrict__ LObuf, float* __restrict__ relbuf,
                          int* rows, int* nrows_sh) {
    const int t = threadIdx.x;
    if (t == 0) {
        int c = 0;
        for (int k = 0; k < d; ++k) if (rpin[k + 1] > rpin[k]) rows[c++] = k;
        *nrows_sh = c;
    }
    for (int c = t; c < dp * dp; c += blockDim.x) { Lbuf[c] = -INFINITY; relbuf[c] = -INFINITY; }
    __syncthreads();
    const int nr = *nrows_sh;
    const float invd = 1.0f / d;
    for (int e = t; e < nr * d; e += blockDim.x) {
        int k = rows[e / d], j = e % d;
        float mx = -INFINITY;
        for (int q = rpin[k]; q < rpin[k + 1]; ++q) {
            int cell = listin[q], l = cell % dp;
            float dl = (j - l) * invd;
            mx = fmaxf(mx, logf(win[cell]) + (float)hin[cell] - dl * dl * ginv);
        }
        float s = 0.f;
        for (int q = rpin[k]; q < rpin[k + 1]; ++q) {
            int cell = listin[q], l = cell % dp;
            float dl = (j - l) * invd;
            s += expf(logf(win[cell]) + (float)hin[cell] - dl * dl * ginv - mx);
        }
        Lbuf[k * dp + j] = mx + logf(s);
    }
    __syncthreads();
    const float lD = (float)lwD;
    for (int e = t; e < nout; e += blockDim.x) {
        int cell = listout[e], i = cell / dp, j = cell % dp;
        float dd = (j - i) * invd;
        float mx = lD - 0.5f * dd * dd * ginv;
        for (int r = 0; r < nr; ++r) { int k = rows[r]; float dk = (i - k) * invd; mx = fmaxf(mx, Lbuf[k * dp + j] - dk * dk * ginv); }
        float s = (lD > -INFINITY) ? expf(lD - 0.5f * dd * dd * ginv - mx) : 0.f;
        for (int r = 0; r < nr; ++r) { int k = rows[r]; float dk = (i - k) * invd; s += expf(Lbuf[k * dp + j] - dk * dk * ginv - mx); }
        LObuf[cell] = mx + logf(s);
    }
    __syncthreads();
    for (int e = t; e < nr * d; e += blockDim.x) {
        int k = rows[e / d], j = e % d;
        float best = -INFINITY;
        float Lkj = Lbuf[k * dp + j];
        for (int q = cpout[j]; q < cpout[j + 1]; ++q) {
            int i = crout[q];
            float dk = (i - k) * invd;
            best = fmaxf(best, Lkj - dk * dk * ginv - LObuf[i * dp + j]);
        }
        relbuf[k * dp + j] = best;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(T_CTA) sk_absorb_kernel(SkWS w, SkRun r) {
    __shared__ float s_a[512], s_b[512];
    __shared__ int s_rc[256], s_cc[256];
    __shared__ int rows[256];
    __shared__ int nrows;
    __shared__ int bad;
    const int p = blockIdx.x, t = threadIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    if (q.ic[IC_STATUS] != ST_ACTIVE && q.ic[IC_STATUS] != ST_CONVERGED && q.ic[IC_STATUS] != ST_MAXITER) return;
    if (!q.ic[IC_ABSORB]) return;
    const int d = w.d, dp = w.dp, na = q.ic[IC_NA], nb = q.ic[IC_NB];
    const double aD = q.sc[SC_AD], bD = q.sc[SC_BD];
    double* phiD = &q.phi[w.n - 1];
    double* psiD = &q.psi[w.n - 1];
    if (t == 0) bad = 0;
    __syncthreads();
    // (a) potentials from the current residuals
    if (q.ic[IC_FROMLIN]) {
        for (int e = t; e < na; e += blockDim.x) {
            int c = q.sa[e];
            float ratio = q.ut[c] / q.am[c];
            if (!(ratio > 0.f) || !isfinite(ratio)) bad = 1;
            q.phi[c] = (q.ap[c / dp] + q.bp[c % dp]) + (double)logf(ratio);
        }
        for (int e = t; e < nb; e += blockDim.x) {
            int c = q.sb[e];
            float ratio = q.vt[c] / q.bm[c];
            if (!(ratio > 0.f) || !isfinite(ratio)) bad = 1;
            q.psi[c] = (q.al[c / dp] + q.be[c % dp]) + (double)logf(ratio);
        }
        if (t == 0) {
            if (aD > 0) *phiD = q.sc[SC_FD] + log(q.sc[SC_UTD] / aD);
            if (bD > 0) *psiD = q.sc[SC_GD] + log(q.sc[SC_VTD] / bD);
        }
    }
    __syncthreads();
    if (bad) {
        if (t == 0) { q.ic[IC_STATUS] = ST_RANGE; q.ic[IC_ABSORB] = 0; }
        return;
    }
    // (b) separable fits of the potentials on the supports
    fit_sparse(q.phi, q.rpa, q.sa, q.cpa, q.cia, d, dp, s_a, s_b, s_rc, s_cc, 16);
    for (int i = t; i < dp; i += blockDim.x) { q.ap[i] = i < d ? (double)s_a[i] : 0.0; q.bp[i] = i < d ? (double)s_b[i] : 0.0; }
    __syncthreads();
    fit_sparse(q.psi, q.rpb, q.sb, q.cpb, q.cib, d, dp, s_a, s_b, s_rc, s_cc, 16);
    for (int i = t; i < dp; i += blockDim.x) { q.al[i] = i < d ? (double)s_a[i] : 0.0; q.be[i] = i < d ? (double)s_b[i] : 0.0; }
    if (t == 0) {
        q.sc[SC_FD] = (aD > 0) ? as_f32(*phiD) : 0.0;
        q.sc[SC_GD] = (bD > 0) ? as_f32(*psiD) : 0.0;
    }
    __syncthreads();
    const float ginvf = (float)(1.0 / w.gamma);
    float* relf = reinterpret_cast<float*>(q.L64);
    // (c) intermediate of the u-update
    relevance(q.bm, q.psi, q.rpb, q.sb, bD > 0 ? log(bD) + *psiD : -INFINITY, q.sa, na, q.cpa, q.cia, d, dp, ginvf,
              q.Wt, q.Rt, relf, rows, &nrows);
    fit_masked(q.Wt, relf, (float)r.rel_thresh, d, dp, s_a, s_b, s_rc, s_cc, 16);
    balance(q.Wt, q.Rt, relf, q.sa, na, q.cpa, q.cia, q.bm, q.psi, q.rpb, q.sb, q.ap, q.bp, q.be, s_a, s_b, rows,
            nrows, d, dp, ginvf, (float)r.rel_thresh, 6);
    for (int i = t; i < dp; i += blockDim.x) { q.Au[i] = i < d ? (double)s_a[i] : 0.0; q.Bu[i] = i < d ? (double)s_b[i] : 0.0; }
    __syncthreads();
    // (d) intermediate of the v-update
    relevance(q.am, q.phi, q.rpa, q.sa, aD > 0 ? log(aD) + *phiD : -INFINITY, q.sb, nb, q.cpb, q.cib, d, dp, ginvf,
              q.Wt, q.Rt, relf, rows, &nrows);
    fit_masked(q.Wt, relf, (float)r.rel_thresh, d, dp, s_a, s_b, s_rc, s_cc, 16);
    balance(q.Wt, q.Rt, relf, q.sb, nb, q.cpb, q.cib, q.am, q.phi, q.rpa, q.sa, q.al, q.be, q.bp, s_a, s_b, rows,
            nrows, d, dp, ginvf, (float)r.rel_thresh, 6);
    for (int i = t; i < dp; i += blockDim.x) { q.Av[i] = i < d ? (double)s_a[i] : 0.0; q.Bv[i] = i < d ? (double)s_b[i] : 0.0; }
    __syncthreads();
    // (e) absorbed kernel factors.  c_m/gamma split hi/lo from the shared table.
    const float* chi = w.ctab;
    const float* clo = w.ctab + dp;
    for (int c = t; c < dp * dp; c += blockDim.x) {
        int a = c / dp, b = c % dp;
        float k1u = 0.f, k2u = 0.f, k1v = 0.f, k2v = 0.f;
        if (a < d && b < d) {
            int m = abs(a - b);
            // K1u[j=a, l=b] = exp(be_l - Bu_j - c_jl/g)
            k1u = exp3((float)q.be[b], -(float)q.Bu[a], chi[m], clo[m]);
            // K2u[i=a, k=b] = exp(ap_i + Au_k - c_ik/g)
            k2u = exp3((float)q.ap[a], (float)q.Au[b], chi[m], clo[m]);
            // K1v[l=a, j=b] = exp(bp_j - Bv_l - c_jl/g)
            k1v = exp3((float)q.bp[b], -(float)q.Bv[a], chi[m], clo[m]);
            // K2v[k=a, i=b] = exp(al_k + Av_i - c_ik/g)
            k2v = exp3((float)q.al[a], (float)q.Av[b], chi[m], clo[m]);
        }
        q.K1u[c] = k1u; q.K2u[c] = k2u; q.K1v[c] = k1v; q.K2v[c] = k2v;
    }
    for (int i = t; i < dp; i += blockDim.x) {
        bool in = i < d;
        q.rs_u[i] = in ? exp_split(q.al[i] - q.Au[i]) : 0.f;
        q.cf_u[i] = in ? exp_split(q.bp[i] + q.Bu[i]) : 0.f;
        q.rs_v[i] = in ? exp_split(q.ap[i] - q.Av[i]) : 0.f;
        q.cf_v[i] = in ? exp_split(q.be[i] + q.Bv[i]) : 0.f;
    }
    // (f) Delta factors and residual scalings on the supports
    const double ginv = 1.0 / w.gamma, FD = q.sc[SC_FD], GD = q.sc[SC_GD];
    float maxres = 0.f;
    for (int e = t; e < na; e += blockDim.x) {
        int c = q.sa[e], i = c / dp, j = c % dp;
        double Fb = q.ap[i] + q.bp[j];
        q.KDu[c] = exp_split(Fb + GD - pd_cdiag(i, j, d) * ginv);
        float u = q.am[c] * exp_split(q.phi[c] - Fb);
        if (!(u > 0.f) || !isfinite(u)) bad = 1;
        maxres = fmaxf(maxres, fabsf((float)(q.phi[c] - Fb)));
        q.ut[c] = u;
    }
    for (int e = t; e < nb; e += blockDim.x) {
        int c = q.sb[e], k = c / dp, l = c % dp;
        double Gb = q.al[k] + q.be[l];
        q.KDv[c] = exp_split(FD + Gb - pd_cdiag(k, l, d) * ginv);
        float v = q.bm[c] * exp_split(q.psi[c] - Gb);
        if (!(v > 0.f) || !isfinite(v)) bad = 1;
        maxres = fmaxf(maxres, fabsf((float)(q.psi[c] - Gb)));
        q.vt[c] = v;
    }
    maxres = block_max(maxres, reinterpret_cast<float*>(s_rc), 0.f);
    __syncthreads();
    if (t == 0) {
        q.sc[SC_DD] = exp_split(FD + GD);
        q.sc[SC_UTD] = (aD > 0) ? aD * exp(*phiD - FD) : 0.0;
        q.sc[SC_VTD] = (bD > 0) ? bD * exp(*psiD - GD) : 0.0;
        q.sc[SC_TAU] = fmin(60.0, fmax(r.tau, (double)maxres + 15.0));
        q.ic[IC_ABSORB] = 0;
        q.ic[IC_FROMLIN] = 1;
        q.ic[IC_SINCE] = 0;
        if (bad) q.ic[IC_STATUS] = ST_RANGE;
    }
}

cudaError_t sk_launch_absorb(const SkWS& w, SkRun r, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_absorb_kernel<<<w.P, T_CTA, 0, s>>>(w, r);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Linear-domain iterations with FP32 CUDA-core GEMMs (the plain FP32 form).
struct EpiStoreT {   // Wt[n*dp + m] = acc, saturated to the finite range
    float* out; int dp;
    __device__ void operator()(int m, int n, float v) const { out[(size_t)n * dp + m] = fminf(v, 3.4028235e38f); }
};
struct RowScale {    // A element (m, k) times rs[m]: the row scale of the GEMM1 operand
    const float* rs;
    __device__ float operator()(int m, int, float v) const { return v * rs[m]; }
};
struct EpiStore {    // R[m*dp + n] = acc
    float* out; int dp;
    __device__ void operator()(int m, int n, float v) const { out[(size_t)m * dp + n] = v; }
};

// One Sinkhorn iteration on the residual representation.  Returns the
// relative marginal error err_t; sets *range if a scaling left [e^-tau, e^tau]
// relative to its weight or became non-finite.
__device__ float sk_iteration_fp32(PairPtrs& q, int d, int dp, int na, int nb, float aD, float bD, float total,
                                   float DD, float& utD, float& vtD, float tau, int* range, float* sm, float* shf) {
    const int t = threadIdx.x;
    // ---- u-update
    cta_gemm_nt(q.vt, q.K1u, dp, RowScale{q.rs_u}, Ident(), EpiStoreT{q.Wt, dp}, sm);
    cta_gemm_nt(q.K2u, q.Wt, dp, Ident(), Ident(), EpiStore{q.Rt, dp}, sm);
    for (int e = t; e < na; e += blockDim.x) {
        int c = q.sa[e];
        float den = q.cf_u[c % dp] * q.Rt[c] + q.KDu[c] * vtD;
        float u = q.am[c] / den;
        float lr = logf(u / q.am[c]), lo = logf(u * q.rs_v[c / dp]);
        if (!(fabsf(lr) <= tau) || !(fabsf(lo) <= 85.f)) *range = 1;
        q.ut[c] = u;
    }
    float s = 0.f;
    for (int e = t; e < nb; e += blockDim.x) { int c = q.sb[e]; s += q.KDv[c] * q.vt[c]; }
    s = block_sum(s, shf);
    float utD_new = (aD > 0.f) ? aD / (s + DD * vtD) : 0.f;
    if (aD > 0.f && !(fabsf(logf(utD_new / aD)) <= tau)) *range = 1;
    utD = utD_new;
    __syncthreads();
    // ---- v-update (with the column error of (u_t, v_{t-1}))
    cta_gemm_nt(q.ut, q.K1v, dp, RowScale{q.rs_v}, Ident(), EpiStoreT{q.Wt, dp}, sm);
    cta_gemm_nt(q.K2v, q.Wt, dp, Ident(), Ident(), EpiStore{q.Rt, dp}, sm);
    float err = 0.f;
    for (int e = t; e < nb; e += blockDim.x) {
        int c = q.sb[e];
        float qv = q.cf_v[c % dp] * q.Rt[c] + q.KDv[c] * utD;
        err += fabsf(q.vt[c] * qv - q.bm[c]);
        float v = q.bm[c] / qv;
        if (!(fabsf(logf(v / q.bm[c])) <= tau) || !(fabsf(logf(v * q.rs_u[c / dp])) <= 85.f)) *range = 1;
        q.vt[c] = v;
    }
    float s2 = 0.f;
    for (int e = t; e < na; e += blockDim.x) { int c = q.sa[e]; s2 += q.KDu[c] * q.ut[c]; }
    s2 = block_sum(s2, shf);
    err = block_sum(err, shf);
    float qD = s2 + DD * utD;
    if (bD > 0.f) {
        err += fabsf(vtD * qD - bD);
        float v = bD / qD;
        if (!(fabsf(logf(v / bD)) <= tau)) *range = 1;
        vtD = v;
    }
    __syncthreads();
    return err / total;
}

__global__ void __launch_bounds__(T_CTA) sk_iter_fp32_kernel(SkWS w, SkRun r, int n_inner, int* active_count) {
    extern __shared__ float sm[];
    __shared__ float shf[32];
    __shared__ int range;
    const int p = blockIdx.x, t = threadIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    if (q.ic[IC_STATUS] != ST_ACTIVE) return;
    if (q.ic[IC_ABSORB]) { if (t == 0) atomicAdd(active_count, 1); return; }
    const int d = w.d, dp = w.dp, na = q.ic[IC_NA], nb = q.ic[IC_NB];
    const float aD = (float)q.sc[SC_AD], bD = (float)q.sc[SC_BD], total = (float)q.sc[SC_TOTAL];
    const float DD = (float)q.sc[SC_DD];
    float utD = (float)q.sc[SC_UTD], vtD = (float)q.sc[SC_VTD];
    const float tau = (float)q.sc[SC_TAU];
    int iters = q.ic[IC_ITERS], since = q.ic[IC_SINCE];
    int status = ST_ACTIVE, absorb = 0;
    float err = (float)q.sc[SC_ERR];
    if (t == 0) range = 0;
    __syncthreads();
    for (int it = 0; it < n_inner; ++it) {
        err = sk_iteration_fp32(q, d, dp, na, nb, aD, bD, total, DD, utD, vtD, tau, &range, sm, shf);
        ++iters; ++since;
        __syncthreads();
        if (!isfinite(err)) { absorb = 1; break; }
        if (r.tol > 0 && err <= r.tol) { status = ST_CONVERGED; break; }
        if (iters >= r.max_iter) { status = ST_MAXITER; break; }
        if (range || since >= r.absorb_every) { absorb = 1; break; }
    }
    __syncthreads();
    if (t == 0) {
        q.sc[SC_UTD] = utD; q.sc[SC_VTD] = vtD; q.sc[SC_ERR] = err;
        q.ic[IC_ITERS] = iters; q.ic[IC_SINCE] = since;
        if (status != ST_ACTIVE) q.ic[IC_STATUS] = status;
        if (absorb) {
            // a range failure right after an absorption means the separable
            // representation cannot hold this pair
            if (range && since == 1) { q.ic[IC_RANGE] += 1; } else q.ic[IC_RANGE] = 0;
            if (q.ic[IC_RANGE] >= 2 || !isfinite(err)) q.ic[IC_STATUS] = ST_RANGE;
            else q.ic[IC_ABSORB] = 1;
        }
        if (q.ic[IC_STATUS] == ST_ACTIVE) atomicAdd(active_count, 1);
    }
}

cudaError_t sk_launch_iter_fp32(const SkWS& w, SkRun r, int n_inner, int* active_count, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    const int smem = 2 * 32 * 68 * sizeof(float);
    sk_iter_fp32_kernel<<<w.P, T_CTA, smem, s>>>(w, r, n_inner, active_count);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Finalize: transport cost by Prop. 2 (three GEMMs with m = k (.) c, reduced in
// FP64), marginals and potentials of the final (u_t, v_t).
struct BScaleC {   // B element (n, k) times c_nk = ((n-k)/d)^2
    const float* c1; 
    __device__ float operator()(int n, int k, float v) const { return v * c1[abs(n - k)]; }
};
struct EpiStoreAdd {   // R[m*dp+n] += acc
    float* out; int dp;
    __device__ void operator()(int m, int n, float v) const { out[(size_t)m * dp + n] += v; }
};

__global__ void __launch_bounds__(T_CTA) sk_finalize_kernel(SkWS w, double* __restrict__ cost, float* __restrict__ row_marg,
                                                            float* __restrict__ col_marg, double* __restrict__ fo,
                                                            double* __restrict__ go, int32_t* __restrict__ iters_o,
                                                            float* __restrict__ err_o, int32_t* __restrict__ status_o) {
    extern __shared__ float sm[];
    __shared__ float c1[256];
    __shared__ double shd[32];
    const int p = blockIdx.x, t = threadIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    const int d = w.d, dp = w.dp, na = q.ic[IC_NA], nb = q.ic[IC_NB], n_out = d * d + 1;
    const int st = q.ic[IC_STATUS];
    if (t == 0) {
        if (iters_o) iters_o[p] = q.ic[IC_ITERS];
        if (err_o) err_o[p] = (float)q.sc[SC_ERR];
        if (status_o) status_o[p] = st == ST_CONVERGED ? 0 : (st == ST_MAXITER ? 6 : (st == ST_INVALID ? 1 : 8));
    }
    const bool usable = (st == ST_CONVERGED || st == ST_MAXITER) && q.sc[SC_TOTAL] > 0 && !q.ic[IC_ABSORB];
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
    for (int m = t; m < 256; m += blockDim.x) { float z = (float)m / d; c1[m] = z * z; }
    __syncthreads();
    const double gamma = w.gamma, ginv = 1.0 / gamma;
    const double utD = q.sc[SC_UTD], vtD = q.sc[SC_VTD], DD = q.sc[SC_DD];
    const double aD = q.sc[SC_AD], bD = q.sc[SC_BD], FD = q.sc[SC_FD], GD = q.sc[SC_GD];
    float* W1 = q.Wt;                                   // [j][k]
    float* W2 = reinterpret_cast<float*>(q.L64);        // [j][k]
    float* T = W2 + (size_t)dp * dp;                    // [i][j]
    // W1 = rs_u .* (vt K1u^T), W2 = rs_u .* (vt M1u^T)
    cta_gemm_nt(q.vt, q.K1u, dp, RowScale{q.rs_u}, Ident(), EpiStoreT{W1, dp}, sm);
    cta_gemm_nt(q.vt, q.K1u, dp, RowScale{q.rs_u}, BScaleC{c1}, EpiStoreT{W2, dp}, sm);
    // T = M2u W1 + K2u W2 ;  R = K2u W1
    cta_gemm_nt(q.K2u, W1, dp, BScaleC{c1}, Ident(), EpiStore{T, dp}, sm);
    cta_gemm_nt(q.K2u, W2, dp, Ident(), Ident(), EpiStoreAdd{T, dp}, sm);
    cta_gemm_nt(q.K2u, W1, dp, Ident(), Ident(), EpiStore{q.Rt, dp}, sm);
    // grid-grid cost and the grid->Delta cost, FP64 reduction
    double cs = 0.0;
    for (int e = t; e < na; e += blockDim.x) {
        int c = q.sa[e], i = c / dp, j = c % dp;
        cs += (double)q.ut[c] * ((double)q.cf_u[j] * (double)T[c] + (double)q.KDu[c] * vtD * pd_cdiag(i, j, d));
    }
    for (int e = t; e < nb; e += blockDim.x) {
        int c = q.sb[e], k = c / dp, l = c % dp;
        cs += utD * (double)q.KDv[c] * (double)q.vt[c] * pd_cdiag(k, l, d);
    }
    cs = block_sum(cs, shd);
    if (t == 0) cost[p] = cs;
    // row marginal and f: support cells from u_t, other cells as the soft c-transform of v_t
    if (row_marg || fo) {
        double sD = 0.0;
        for (int e = t; e < nb; e += blockDim.x) { int c = q.sb[e]; sD += (double)q.KDv[c] * q.vt[c]; }
        sD = block_sum(sD, shd);
        for (int x = t; x < d * d; x += blockDim.x) {
            int i = x / d, j = x % d, c = i * dp + j;
            double Fb = q.ap[i] + q.bp[j];
            double kdu = exp_split(Fb + GD - pd_cdiag(i, j, d) * ginv);
            double den = (double)q.cf_u[j] * q.Rt[c] + kdu * vtD;
            float a = q.am[c];
            if (row_marg) row_marg[(size_t)p * n_out + x] = a > 0.f ? (float)(q.ut[c] * den) : 0.f;
            if (fo) fo[(size_t)p * n_out + x] = a > 0.f ? gamma * (Fb + log((double)q.ut[c] / a)) : gamma * (Fb - log(den));
        }
        if (t == 0) {
            if (row_marg) row_marg[(size_t)p * n_out + d * d] = (float)(utD * (sD + DD * vtD));
            if (fo) fo[(size_t)p * n_out + d * d] = aD > 0 ? gamma * (FD + log(utD / aD)) : gamma * (FD - log(sD + DD * vtD));
        }
    }
    // column marginal and g from (u_t, v_t)
    if (col_marg || go) {
        cta_gemm_nt(q.ut, q.K1v, dp, RowScale{q.rs_v}, Ident(), EpiStoreT{q.Wt, dp}, sm);
        cta_gemm_nt(q.K2v, q.Wt, dp, Ident(), Ident(), EpiStore{q.Rt, dp}, sm);
        double sD = 0.0;
        for (int e = t; e < na; e += blockDim.x) { int c = q.sa[e]; sD += (double)q.KDu[c] * q.ut[c]; }
        sD = block_sum(sD, shd);
        for (int y = t; y < d * d; y += blockDim.x) {
            int k = y / d, l = y % d, c = k * dp + l;
            double Gb = q.al[k] + q.be[l];
            double kdv = exp_split(FD + Gb - pd_cdiag(k, l, d) * ginv);
            double qv = (double)q.cf_v[l] * q.Rt[c] + kdv * utD;
            float b = q.bm[c];
            if (col_marg) col_marg[(size_t)p * n_out + y] = b > 0.f ? (float)(q.vt[c] * qv) : 0.f;
            if (go) go[(size_t)p * n_out + y] = b > 0.f ? gamma * (Gb + log((double)q.vt[c] / b)) : gamma * (Gb - log(qv));
        }
        if (t == 0) {
            if (col_marg) col_marg[(size_t)p * n_out + d * d] = (float)(vtD * (sD + DD * utD));
            if (go) go[(size_t)p * n_out + d * d] = bD > 0 ? gamma * (GD + log(vtD / bD)) : gamma * (GD - log(sD + DD * utD));
        }
    }
}

cudaError_t sk_launch_finalize(const SkWS& w, double* cost, float* row_marg, float* col_marg, double* f, double* g,
                               int32_t* iters, float* err, int32_t* status, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    const int smem = 2 * 32 * 68 * sizeof(float);
    sk_finalize_kernel<<<w.P, T_CTA, smem, s>>>(w, cost, row_marg, col_marg, f, g, iters, err, status);
    return cudaGetLastError();
}

