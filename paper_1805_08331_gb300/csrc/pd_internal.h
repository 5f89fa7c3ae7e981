// pd_internal.h -- library-internal declarations (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Per-pair scalar slots (double) of the Sinkhorn workspace.
enum {
    SC_FD = 0,   // absorbed Delta potential of the u side (log units, f_Delta/gamma part)
    SC_GD,       // absorbed Delta potential of the v side
    SC_UTD,      // residual scaling u~_Delta
    SC_VTD,      // residual scaling v~_Delta
    SC_DD,       // absorbed Delta-Delta kernel entry exp(FD + GD)
    SC_AD,       // a_Delta = |B|
    SC_BD,       // b_Delta = |A|
    SC_TOTAL,    // total mass |A| + |B|
    SC_ERR,      // last relative marginal error
    SC_TAU,      // residual threshold that triggers the next absorption
    SC_CORR,     // Prop. 3: rank-one correction term of the rounded plan's cost
    SC_N
};
// Per-pair int slots.
enum {
    IC_NA = 0,   // support size of a on the grid
    IC_NB,       // support size of b on the grid
    IC_ITERS,    // iterations done
    IC_STATUS,   // ST_*
    IC_ABSORB,   // 1 = needs (re-)absorption before iterating
    IC_FROMLIN,  // 1 = potentials must be rebuilt from the linear residuals
    IC_RANGE,    // consecutive range failures
    IC_SINCE,    // iterations since the last absorption
    IC_BIG,      // 1 = supports too large for the on-chip log-domain kernel
    IC_STAGE,    // gamma-continuation inside the base-2 kernel: current stage k (gamma * 4^k)
    IC_N
};
enum { ST_ACTIVE = 0, ST_CONVERGED = 1, ST_MAXITER = 2, ST_RANGE = 3, ST_INVALID = 4 };

// Device-side view of the batched Sinkhorn workspace.  Every per-pair array is
// stored pair-major with the stride given in the comment (dp = padded d, a
// multiple of 64; n = d*d + 1).
struct SkWS {
    int d, dp, n, P;
    double gamma;
    double p;                       // ground cost ||.||_p^p (2: squared Euclidean)
    // FP32 [P][dp*dp]
    float *K1u, *K2u, *K1v, *K2v;   // absorbed separable kernel factors (u- and v-updates)
    float *ut, *vt;                 // residual scalings on the grid (0 off support)
    float *Wt, *Rt;                 // GEMM intermediate (transposed) and output scratch
    float *KDu, *KDv;               // absorbed grid<->Delta kernel entries
    float *am, *bm;                 // dense a, b on the grid (FP32)
    // FP32 [P][dp]
    float *rs_u, *cf_u, *rs_v, *cf_v;  // intermediate row scales / output column factors
    // FP64 [P][dp]
    double *ap, *bp, *al, *be;      // separable absorbed potentials: u side (alpha', beta'), v side (alpha, beta)
    double *Au, *Bu, *Av, *Bv;      // intermediate shifts of the u- and v-updates
    // FP64 [P][n]
    double *phi, *psi;              // current log potentials f/gamma, g/gamma on the supports
    double *sc;                     // [P][SC_N]
    int *sa, *sb;                   // [P][dp*dp] support lists (row-major order)
    int *ic;                        // [P][IC_N]
    // auxiliary per-pair arrays
    double* L64;                    // [P][2*dp*dp] FP64 scratch
    double *la, *lb;                // [P][dp*dp] log a, log b on the supports (FP64)
    int *rpa, *rpb, *cpa, *cpb;     // [P][dp+1] row / column pointers of the support lists
    int *cia, *cib;                 // [P][dp*dp] row indices of the column-major support lists
    float* ctab;                    // [5*dp] hi / lo FP32 splits of c_m/gamma and cD_m/gamma, log c_m
    int* order_buf;                 // [P] launch order of the pairs (filled by the host)
    const int* order;               // NULL: CTA b runs pair b; else CTA b runs pair order[b]
    // device copies of workspace descriptors read by the base-2 kernel: with
    // ngroups == 1 groups[0] is this workspace; a launch over several
    // workspaces (several grid sizes) has ngroups > 1 and order codes
    // group << 24 | pair
    struct SkWS* groups;
    int ngroups;
    // inputs: integer histograms (histA/massA, histB/massB) or, when wA / wB is
    // non-NULL, real-valued weights [N][d*d] for that side (its mass is their sum)
    const uint32_t *histA, *histB, *massA, *massB;
    const double *wA, *wB;
    const int32_t* pairs;
};

cudaError_t pd_launch_raster(const double* birth, const double* death, const int64_t* offsets, int B,
                             int d, int64_t npts, uint32_t* hist, uint32_t* mass, int* bad,
                             cudaStream_t s);

// internal value of SkRun::form (never accepted from pd_sinkhorn_params)
constexpr int SK_FORM_AUTO2 = 3;

struct SkRun {
    int max_iter;
    double tol;
    double tau;
    int absorb_every;
    double rel_thresh;   // relevance threshold (log) for the intermediate fits
    int pot_support_only; // finalize: potentials on the supports and Delta only
    int eps_stages;       // gamma-continuation stages before the target gamma (PD_FP32)
    // on-chip base-2 kernel: once counter[4] (pairs of the launch that stopped
    // or moved tier) reaches exit_at, the pairs still iterating save their
    // state and return, so that the host relaunches them in wider CTAs
    // (0: never)
    int exit_at;
    int cta_threads;      // fixed CTA width of the base-2 kernel (0: automatic)
    int base_threads;     // automatic mode: width of the first launch (0: 256; from the tuning table)
    int tier;             // 0 automatic, 1 global-memory variant, 2 FP64 kernel for every pair
    int max_inner;        // iterations per launch at most (0: run to the stop)
    int diag_tc_timeout;  // tensor-core kernel: skip the first GEMM issue, wait with a spin limit of 0
    // base-2 kernel: gamma-continuation inside the launch (0: off); each pair
    // starts at stage ic[IC_STAGE] (gamma * 4^k) and moves to the next stage
    // once its error is <= stage_tol
    int kstages;
    double stage_tol;
    int form;             // base-2 kernel: 0 automatic, 1 separable only, 2 pairwise wherever p = 2,
                          // SK_FORM_AUTO2 automatic with the term ratio 2 (serving)
    // form 0 in an outer loop (Alg. 2, k-means: results that depend on the
    // whole batch): the separable form for the whole call where the pairwise
    // records of the automatic forms would lower the on-chip CTAs per SM
    int batch_form;
};

cudaError_t sk_launch_setup(const SkWS& w, const double* g_init, cudaStream_t s);
// gamma-continuation step: potentials/gamma scaled by `ratio` (old gamma / new
// gamma, f unchanged) and every pair that stopped at the previous gamma (and is
// below max_iter) made active again
cudaError_t sk_launch_regamma(const SkWS& w, double ratio, int max_iter, cudaStream_t s);
cudaError_t sk_launch_setup_list(const SkWS& w, const double* g_init, const int* plist, int np, cudaStream_t s);
cudaError_t sk_launch_logstep(const SkWS& w, SkRun r, cudaStream_t s);
cudaError_t sk_launch_absorb(const SkWS& w, SkRun r, cudaStream_t s);
cudaError_t sk_launch_iter_fp32(const SkWS& w, SkRun r, int n_inner, int* active_count, cudaStream_t s);
// FP64 global-memory iteration kernel for the pairs with IC_BIG >= min_big
cudaError_t sk_launch_lse_iter(const SkWS& w, SkRun r, int n_inner, int* active_count, int min_big, cudaStream_t s);
cudaError_t sk_launch_iter_bf16(const SkWS& w, SkRun r, int n_inner, int* active_count, int* error_flag,
                                cudaStream_t s);
cudaError_t sk_launch_refine_prep(const SkWS& w, cudaStream_t s);
// PD_BF16 for dp = 64: two pairs per CTA, factors by TMA (sinkhorn_bf16x2.cu);
// pairs are taken two by two in w.order (or index order)
bool sk_bf16x2_applies(const SkWS& w);
cudaError_t sk_launch_iter_bf16x2(const SkWS& w, SkRun r, int n_inner, int* active_count, int* error_flag,
                                  cudaStream_t s);
// potentials phi, psi from the linear-domain residual representation (pairs keep their status)
cudaError_t sk_launch_rebuild_potentials(const SkWS& w, cudaStream_t s);
// PD_OK pairs whose exact marginal error (row / col: [P][d*d+1] exact marginals) exceeds thr -> PD_ERR_RANGE
cudaError_t sk_launch_range_check(const SkWS& w, const float* row, const float* col, int32_t* status, float* err,
                                  double thr, cudaStream_t s);
cudaError_t sk_launch_lse_smem(const SkWS& w, SkRun r, int n_inner, int* active_count, int* big_count,
                               cudaStream_t s);
// base-2 on-chip iteration kernel (sinkhorn_log2.cu)
int sk_lse2_grid_bits(double gamma);
// gamma-continuation inside the iteration kernel: ic[IC_STAGE] = K for every pair
cudaError_t sk_launch_set_stage(const SkWS& w, int K, cudaStream_t s);
// Shared memory of the on-chip pairs: max_need[0] = the largest need;
// max_need[1] += pairs not pairwise in both half-steps.
cudaError_t sk_launch_lse2_need(const SkWS& w, int* max_need, int form, cudaStream_t s);
// counter: [0] active pairs, [1] pairs moved to the global-memory variant,
// [2] (need kernel) max shared bytes, [3] pairs moved to the FP64 kernel.
cudaError_t sk_launch_lse2(const SkWS& w, SkRun r, int n_inner, int* counter, size_t smem, int gbits, int threads,
                           cudaStream_t s);
cudaError_t sk_launch_lse2_gm(const SkWS& w, SkRun r, int n_inner, int* counter, int gbits, size_t gcap,
                              cudaStream_t s);
cudaError_t sk_launch_lse_finalize(const SkWS& w, double* cost, float* row_marg, float* col_marg, double* f,
                                   double* g, int32_t* iters, float* err, int32_t* status, int pot_support_only,
                                   cudaStream_t s);
cudaError_t sk_launch_lse_finalize_list(const SkWS& w, double* cost, float* row_marg, float* col_marg, double* f,
                                        double* g, int32_t* iters, float* err, int32_t* status, int pso,
                                        const int* plist, int np, cudaStream_t s);
// Prop. 3 upper bound (sinkhorn_lse.cu): replaces every usable pair's potentials
// by those of the rescaled plan P2 of the rounding and stores the rank-one term
// in sc[SC_CORR]; the finalize cost of the new potentials plus that term is
// <R, C> (sk_launch_add_corr adds it).
cudaError_t sk_launch_round_bound(const SkWS& w, cudaStream_t s);
cudaError_t sk_launch_add_corr(const SkWS& w, double* upper, cudaStream_t s);
// lower bound m_t of every usable pair from its current potentials (bounds.cu)
cudaError_t sk_launch_ctransform(const SkWS& w, double* lower, cudaStream_t s);
// workspace helpers (api.cu)
size_t pd_carve_ws(char* base, int P, int d, int dp, double gamma, SkWS* w, int** counter);
cudaError_t pd_upload_cost_tables(const SkWS& w, double gamma, cudaStream_t s);
// outer loops (outer.cu)
cudaError_t outer_bary_init_uniform(double* z, const uint32_t* mass, int N, int d, cudaStream_t s);
cudaError_t outer_measure_mass(const double* z, int k, int d, double* out, cudaStream_t s);
cudaError_t outer_bary_step(double* z, const double* zmass, const double* f, const double* g, const int32_t* owner,
                            int N, int k, int d, double gamma, double lambda, cudaStream_t s);
cudaError_t outer_mean(const double* cost, int N, double* out, cudaStream_t s);
// sharded Alg. 2 step: per-shard sums (gsum [k][d*d], count [k]), then the update from the summed values
cudaError_t outer_bary_grad(const double* z, const double* f, const double* g, const int32_t* owner, int N, int k,
                            int d, double* gsum, double* count, cudaStream_t s);
cudaError_t outer_bary_apply(double* z, const double* gsum, const double* count, int k, int d, double gamma,
                             double lambda, cudaStream_t s);
cudaError_t outer_cost_sum(const double* cost, const int32_t* owner, int N, int k, double* out, cudaStream_t s);
cudaError_t outer_km_assign(const double* cost, int N, int k, int32_t* assign, double* objective, cudaStream_t s);
cudaError_t outer_km_seed(const uint32_t* hist, const int32_t* idx, int k, int d, double* z, cudaStream_t s);
cudaError_t outer_km_pairs(int N, int k, int32_t* pairs, cudaStream_t s);
cudaError_t outer_owner_pairs(const int32_t* owner, int N, int32_t* pairs, cudaStream_t s);
cudaError_t outer_check_owner(const int32_t* owner, int N, int k, int* flag, cudaStream_t s);
// entropic sharpening: H0 = largest input entropy (stored as the bits of a non-negative double)
cudaError_t outer_input_entropy(const uint32_t* hist, int N, int d, unsigned long long* H0bits, cudaStream_t s);
cudaError_t outer_sharpen(double* z, int k, int d, const unsigned long long* H0bits, cudaStream_t s);
cudaError_t sk_launch_finalize(const SkWS& w, double* cost, float* row_marg, float* col_marg, double* f,
                               double* g, int32_t* iters, float* err, int32_t* status, cudaStream_t s);
