/*
 * pd_ot.h -- C ABI of the GB300 (sm_103a) library for entropic optimal
 * transport between persistence diagrams rasterised on a d x d grid plus one
 * diagonal bin (Lacombe, Cuturi & Oudot, NeurIPS 2018).
 *
 * Conventions for every entry point
 *   - Returns pd_status; PD_OK (0) on success.  No call aborts the process.
 *     pd_last_error(ctx) gives a message for the last failing call on ctx
 *     (owned by ctx, valid until the next call on ctx).
 *   - Array arguments are DEVICE pointers unless their name ends in _host.
 *     The caller owns every input and output buffer; the library never frees
 *     them.  The library allocates only its own workspace, held by pd_ctx and
 *     released by pd_ctx_destroy.
 *   - Every call takes a CUDA stream (pd_stream is cudaStream_t; NULL is the
 *     legacy default stream).  Work is enqueued on that stream; calls return
 *     after enqueueing unless stated otherwise.  Calls that must inspect
 *     device-side results on the host (convergence loops) synchronise the
 *     stream and say so.
 *   - Grid cell (i, j): i = birth index (row), j = death index (column),
 *     0 <= i, j < d; flattened index x = i*d + j.  Index d*d is the Delta
 *     (diagonal) bin.  Histograms are row-major uint32 [d][d].
 *   - A pd_ctx must not be used by two host threads at once.
 */
#ifndef PD_OT_H
#define PD_OT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* pd_stream; /* == cudaStream_t */
typedef struct pd_ctx pd_ctx;
typedef int pd_status;

enum {
    PD_OK = 0,
    PD_ERR_INVALID = 1,   /* bad argument: d outside [2,256], gamma <= 0, bad point, NULL output ... */
    PD_ERR_OOM = 2,       /* workspace allocation failed */
    PD_ERR_CUDA = 3,      /* a CUDA runtime call failed (message in pd_last_error) */
    PD_ERR_TIMEOUT = 4,   /* a bounded wait ran out */
    PD_ERR_QUEUE_FULL = 5,/* serving queue has no free slot */
    PD_NOT_CONVERGED = 6, /* per pair: max_iter reached before tol (not fatal) */
    PD_PENDING = 7,       /* serving: result not ready yet */
    PD_ERR_RANGE = 8      /* per pair: a scaling left the floating-point range even after absorption */
};

/* Engines of pd_sinkhorn_batch:
 *   PD_FP32       exact log-domain separable evaluation (Prop. 1 in the log semiring) on the
 *                 histogram supports, FP32 double-float arithmetic, FP64 potentials; any gamma.
 *   PD_BF16       absorbed-potential linear-domain separable GEMMs on the tensor cores (tcgen05,
 *                 BF16 operands, FP32 accumulation), then FP32 refinement by the PD_FP32 engine.
 *   PD_FP32_DENSE absorbed-potential linear-domain separable GEMMs on the CUDA cores (FP32),
 *                 one pair per CTA, all pairs in each launch: the batched dense form.
 *   PD_FP32_PLAIN the same FP32 arithmetic as PD_FP32_DENSE with one pair per launch (pairs solved
 *                 one after the other): the plain FP32 form, kept as the comparator of the
 *                 batched tensor-core form. */
enum { PD_FP32 = 0, PD_BF16 = 1, PD_FP32_DENSE = 2, PD_FP32_PLAIN = 3 };

/* Version of this ABI (increments on incompatible change). */
int pd_abi_version(void);

/* Create a context bound to CUDA device `device` (makes it current for the
 * calling thread).  *out receives the context. */
pd_status pd_ctx_create(int device, pd_ctx** out);
/* Release the context and its workspace.  Safe on NULL. */
void pd_ctx_destroy(pd_ctx* ctx);
/* Message of the last failing call on ctx ("" if none). */
const char* pd_last_error(const pd_ctx* ctx);

/*
 * pd_rasterize -- Sec. 3 "Discretization": hist[b][i][j] = number of points
 * of diagram b in grid cell (i, j), with i = floor(birth * d), j =
 * floor(death * d) computed in IEEE FP64 and clamped to d-1 (the closed edge at
 * 1 belongs to the last cell); mass[b] = number of points of diagram b.
 *   birth, death : double [offsets[B]]  points in CSR order (device)
 *   offsets      : int64  [B+1]         diagram b owns points offsets[b] .. offsets[b+1]-1 (device)
 *   B, d         : number of diagrams, grid size (2 <= d <= 256)
 *   hist         : uint32 [B][d][d]     output, overwritten (device)
 *   mass         : uint32 [B]           output (device)
 * Errors: PD_ERR_INVALID if B < 0, d outside [2,256], or any point is not a
 * finite point of [0,1]^2 with birth <= death (checked on the device; this call
 * then synchronises the stream to report it).
 */
pd_status pd_rasterize(pd_ctx* ctx, const double* birth, const double* death, const int64_t* offsets,
                       int B, int d, uint32_t* hist, uint32_t* mass, pd_stream stream);

/* Parameters of a batched Sinkhorn solve. */
typedef struct {
    double gamma;      /* entropic regularisation gamma > 0 (Eq. SinkhornMinimizationProblem) */
    int d;             /* grid size, 2 <= d <= 256 */
    int max_iter;      /* maximum number of Sinkhorn iterations (each = u-update then v-update), >= 1 */
    double tol;        /* stop after iteration t if err_t / total mass <= tol (0 = run max_iter) */
    int precision;     /* engine: PD_FP32, PD_BF16, PD_FP32_DENSE or PD_FP32_PLAIN (see above) */
    int refine_iters;  /* PD_BF16 only: FP32 iterations run after the BF16 phase stops (0 = none) */
    double absorb_tau; /* re-absorb when |log(u~/a)| or |log(v~/b)| exceeds this (<= 0: default 20) */
    int absorb_every;  /* also re-absorb every this many iterations (<= 0: default 64; the PD_BF16 kernel
                          for d <= 64, whose split operands keep their precision, uses at least 512) */
    double rel_log_thresh; /* a term counts as relevant to an output when it is within exp(rel_log_thresh)
                              of the output's sum; the absorbed representation keeps every relevant
                              term in range (>= 0: default, -21 for PD_FP32 and -14 for PD_BF16) */
    int eps_stages;    /* PD_FP32: gamma-continuation (epsilon-scaling) stages before the target gamma:
                          stage k = eps_stages..1 iterates at gamma * 4^k until err <= max(tol, 1e-4),
                          the potentials f, g carried over; then gamma itself to tol.  The result is the
                          same fixed point; iters counts all stages.  0 (default) = off */
    double p;          /* ground cost ||.||_p^p, 1 <= p <= 8 (default 2, squared Euclidean): grid cost
                          |i-k|^p/d^p + |j-l|^p/d^p, cell to diagonal 2 |(j-i)/(2d)|^p (the orthogonal
                          projection).  p != 2: PD_FP32 engine of pd_sinkhorn_batch only */
    int bary_sharpen;  /* pd_barycenter only: 1 = entropic sharpening after every Alg. 2 step (the
                          extension the paper names for smeared barycenters, after Solomon et al.): when
                          the entropy of z/|z| exceeds the largest entropy of the normalised input
                          histograms, z <- |z| w^beta / sum w^beta (w = z/|z|), beta >= 1 chosen to meet
                          it.  0 (default) = off */
    int cta_threads;   /* PD_FP32 iteration kernel: threads of the CTA that runs one pair, 128, 256, 512 or
                          1024; 0 (default) = automatic: the context's tuning table (pd_sinkhorn_tune) when it
                          has an entry for the batch's profile, else the built-in rule (256 while several pairs
                          share an SM, wider CTAs for the last pairs of a launch unless every pair takes the
                          pairwise form in both half-steps, see lse_form).  A fixed width turns the
                          hand-over of the last pairs to wider CTAs off.  Results do not depend on it: every
                          sum of the kernel has a fixed order whatever the width */
    int kernel_tier;   /* PD_FP32: 0 (default) = automatic (on-chip kernel; its global-memory variant for
                          supports beyond shared memory; the FP64 kernel beyond that or for potentials outside
                          the exact range); 1 = every pair in the global-memory variant; 2 = every pair in the
                          FP64 kernel (for checking the tiers against each other) */
    int max_inner;     /* PD_FP32: iterations per launch at most; 0 (default) = every pair runs to its stop
                          inside one launch */
    int diag_tc_timeout; /* PD_BF16 diagnostic of the tensor-core kernel's bounded waits: 1 = its first GEMM
                          is not issued and the wait for it has a spin limit of 0, so the wait gives up at once
                          with no tensor-core work in flight; the kernel frees its tensor memory and the call
                          returns PD_ERR_TIMEOUT (the context stays usable).  0 (default) = off */
    int lse_form;      /* PD_FP32 iteration kernel (on chip), form of each half-step's log-sum-exp (Prop. 1
                          restricted to the supports): 1 = separable (stage 1 over the input's cells and the
                          output's columns, stage 2 over the input's rows and the output's cells); 2 = pairwise
                          over the two supports, c_xy = |x - y|^2 / d^2 computed exactly per term, wherever
                          p = 2; 0 (default) = per half-step, pairwise while it has at most 5 times the separable
                          form's terms (p = 2), else separable.  The pairwise form also needs its records
                          (16 bytes per cell) to fit in shared memory beside the pair's other arrays (else
                          the separable form runs on chip) and exact scaled units at the gamma of the stage
                          (n1 = rint(log2(e) / (gamma d^2) 2^G) >= 1; a continuation stage without them runs
                          separable, and the pair switches at the first stage that has them).  In
                          pd_barycenter, pd_barycenter_grad, pd_kmeans and pd_kmeans_assign, whose results
                          depend on the whole batch, form 0 runs a call in the separable form where the
                          pairwise records would lower the on-chip CTAs per SM (a dense barycenter side at
                          d = 64).  pd_sinkhorn_batch keeps each pair's form independent of the batch; for a
                          batch of small diagrams against dense histograms of varying sizes, lse_form = 1
                          can be faster (2048 such pairs at d = 64: 83 against 124 ms).  Both forms are
                          exact sums of the same terms in FP32; results agree within rounding */
} pd_sinkhorn_params;

/* Fill *p with defaults for (gamma, d): max_iter 20000, tol 1e-6, PD_FP32,
 * refine_iters 0, absorb_tau 20, absorb_every 64, rel_log_thresh 0 (default). */
void pd_sinkhorn_default_params(pd_sinkhorn_params* p, double gamma, int d);

/*
 * pd_sinkhorn_batch -- Alg. 1: for each pair p, the entropic transport between
 * the augmented histograms a = (histA[ia], massB[ib]) and b = (histB[ib],
 * massA[ia]) (Prop. 1) with the squared-Euclidean grid cost in physical units
 * on [0,1]^2 and cost (j-i)^2/(2 d^2) to the diagonal bin, by Sinkhorn
 * iterations of Eq. (SinkhornMap) applied through the separable kernel of
 * Prop. 1 (Sec. 3 "Convolutions").  Iteration t is the u-update then the
 * v-update; err_t = sum_y |v_{t-1,y} (K^T u_t)_y - b_y| (the marginal error of
 * Eq. Altschuler bounds, row side exact after the u-update) divided by the total
 * mass; the loop stops after iteration t when err_t <= tol or t == max_iter.
 * Potentials use P_xy = a_x b_y exp((f_x + g_y - C_xy)/gamma).
 *   histA, massA : uint32 [NA][d][d], uint32 [NA]   (device)
 *   histB, massB : uint32 [NB][d][d], uint32 [NB]   (device)
 *   pairs        : int32 [P][2] (ia, ib) indices, or NULL meaning pair p = (p, p) (device);
 *                  the arrays' lengths are not passed, so the caller keeps ia and ib
 *                  within histA / histB (not checked)
 *   P            : number of pairs (>= 0)
 *   params       : host pointer
 *   g_init       : double [P][d*d+1] initial g (warm start), or NULL for g = 0 (device)
 * Outputs (device; only `cost` is required, others may be NULL):
 *   cost     : double [P]          <P, C> by Prop. 2, reduced in FP64
 *   row_marg : float  [P][d*d+1]   sum_y P_xy
 *   col_marg : float  [P][d*d+1]   sum_x P_xy
 *   f, g     : double [P][d*d+1]   potentials; entries whose kernel sum underflows are +inf
 *   iters    : int32  [P]          iterations run
 *   err      : float  [P]          last err_t (relative)
 *   status   : int32  [P]          PD_OK, PD_NOT_CONVERGED or PD_ERR_RANGE.  The linear-domain
 *                                  engines (PD_FP32_DENSE, PD_FP32_PLAIN) check every pair they
 *                                  report PD_OK: the exact log-domain marginals of its final plan
 *                                  must be within max(10 tol, 1e-5) of (a, b) (relative L1, both
 *                                  sides), else the pair is PD_ERR_RANGE (its representation
 *                                  dropped terms that matter, e.g. at small gamma)
 * Synchronises `stream` (the iteration loop checks convergence on the host).
 * Errors: PD_ERR_INVALID (bad params / NULL cost / P < 0), PD_ERR_OOM, PD_ERR_CUDA.
 */
pd_status pd_sinkhorn_batch(pd_ctx* ctx, const uint32_t* histA, const uint32_t* massA,
                            const uint32_t* histB, const uint32_t* massB, const int32_t* pairs, int P,
                            const pd_sinkhorn_params* params, const double* g_init,
                            double* cost, float* row_marg, float* col_marg, double* f, double* g,
                            int32_t* iters, float* err, int32_t* status, pd_stream stream);


/*
 * pd_sinkhorn_batch_groups -- pd_sinkhorn_batch over pairs of several grid
 * sizes at once: group g holds P pairs of d x d histograms (its own inputs and
 * outputs, laid out as in pd_sinkhorn_batch at that d), and the PD_FP32
 * iterations of every pair of every group run in one persistent launch (each
 * pair in its own CTA with its own grid size; CTAs handed out largest support
 * first over all groups).  Each pair's results are those pd_sinkhorn_batch
 * gives for it (bitwise: a pair's CTA does the same arithmetic whatever else is
 * in the launch).  A library feature for mixed workloads (e.g. serving several
 * grid sizes); the paper batches one grid size.
 *   ngroups   : 1..127; each group's P < 2^24
 *   params    : host pointer; params->d is ignored (each group has its own d);
 *               precision must be PD_FP32 and eps_stages 0
 * Synchronises `stream`.  Errors: as pd_sinkhorn_batch.
 */
typedef struct {
    int d;                                    /* grid size of the group, 2..256 */
    int P;                                    /* number of pairs (>= 0) */
    const uint32_t *histA, *massA, *histB, *massB;   /* [N][d][d], [N] (device) */
    const int32_t* pairs;                     /* [P][2] or NULL (pair p = (p, p)) (device) */
    const double* g_init;                     /* [P][d*d+1] or NULL (device) */
    double* cost;                             /* [P] (device, required) */
    float *row_marg, *col_marg;               /* [P][d*d+1] or NULL (device) */
    double *f, *g;                            /* [P][d*d+1] or NULL (device) */
    int32_t* iters;                           /* [P] or NULL (device) */
    float* err;                               /* [P] or NULL (device) */
    int32_t* status;                          /* [P] or NULL (device) */
} pd_sinkhorn_group;
pd_status pd_sinkhorn_batch_groups(pd_ctx* ctx, int ngroups, const pd_sinkhorn_group* groups_host,
                                   const pd_sinkhorn_params* params, pd_stream stream);

/*
 * pd_sinkhorn_bounds -- Sec. 3 "Upper and Lower Bounds": the PD_FP32 solve of
 * pd_sinkhorn_batch (same inputs, parameters and cost / iters / err / status
 * outputs), then for each pair, from its final iterate, the bounds
 *   lower[p] = m_t = <alpha^cc, a> + <alpha^c, b>  <=  L_C(a, b)  <=  upper[p] = M_t = <R, C>
 * on the exact (unregularised) transport cost L_C:
 *   - m_t: alpha = gamma log u (u = a exp(f/gamma)), its C-transform
 *     alpha^c(y) = min_x C(x,y) - alpha(x) and the C^T-transform
 *     alpha^cc(x) = min_y C(x,y) - alpha^c(y), over the supports (weak duality);
 *     evaluated exactly in FP64 as two separable (min, +) stages;
 *   - M_t (Prop. 3): the rounding algorithm of the supplementary (after
 *     Altschuler et al.) maps P to R in Pi(a, b) by X = min(a / r(P), 1),
 *     Y = min(b / c(diag(X) P), 1), R = diag(X) P diag(Y) + e_r e_c^T / |e_c|_1,
 *     with e_r, e_c the marginal errors of the rescaled plan; R is feasible,
 *     and <R, C> is computed without forming R (Prop. 2 on the rescaled
 *     potentials plus the rank-one term through the separable cost).
 *   lower, upper : double [P] (device, output; either may be NULL)
 * Synchronises `stream`.  Errors: as pd_sinkhorn_batch; precision must be
 * PD_FP32.  A pair whose status is not PD_OK / PD_NOT_CONVERGED gets NaN.
 */
pd_status pd_sinkhorn_bounds(pd_ctx* ctx, const uint32_t* histA, const uint32_t* massA, const uint32_t* histB,
                             const uint32_t* massB, const int32_t* pairs, int P, const pd_sinkhorn_params* params,
                             const double* g_init, double* cost, double* lower, double* upper, int32_t* iters,
                             float* err, int32_t* status, pd_stream stream);

/*
 * pd_sinkhorn_tune -- autotuner of the PD_FP32 iteration kernel for a batch
 * profile.  Library feature (the paper has no counterpart).  It runs the
 * batch's pairs (same arguments as pd_sinkhorn_batch; params->precision must
 * be PD_FP32) cold-started, each pair until params->tol or trial_iters
 * iterations, once per candidate width of the CTA that runs one pair (128
 * threads when d <= 128, 256, 512; one launch each, timed with CUDA events),
 * and records the fastest
 * in the context's tuning table under the key (d, support bucket), the
 * bucket being floor(2 log2(mean support cells per side + 1)).  From then on a
 * pd_sinkhorn_batch (or bounds / barycenter / k-means solve) on this context
 * whose batch falls in that key starts with the tuned width (cta_threads = 0),
 * still handing its last pairs to wider CTAs where the built-in rule does.  Results never depend on the
 * width (fixed-order sums), so tuning changes speed only.
 *   trial_iters   : iteration cap of each trial (>= 1); params->max_iter makes
 *                   every trial a full solve, which includes the end of the
 *                   solve where few pairs are left (a short cold trial of all
 *                   pairs at once can favour a width that is slower there)
 *   threads_host  : int (host) or NULL: the chosen width
 *   trial_ms_host : double[4] (host) or NULL: kernel time of the trials at
 *                   128, 256, 512, 1024 threads (NaN where not tried)
 * Synchronises `stream`.  Errors: PD_ERR_INVALID (bad arguments, or gamma
 * below the base-2 kernel's range), PD_ERR_OOM, PD_ERR_CUDA.
 */
pd_status pd_sinkhorn_tune(pd_ctx* ctx, const uint32_t* histA, const uint32_t* massA, const uint32_t* histB,
                           const uint32_t* massB, const int32_t* pairs, int P, const pd_sinkhorn_params* params,
                           int trial_iters, int* threads_host, double* trial_ms_host, pd_stream stream);
/* Write the context's tuning table to a text file (one "d bucket threads" line
 * per entry) / replace it by the table of such a file.  PD_ERR_INVALID if the
 * file cannot be written / read or holds a bad entry (the table is then
 * unchanged). */
pd_status pd_tune_save(pd_ctx* ctx, const char* path_host);
pd_status pd_tune_load(pd_ctx* ctx, const char* path_host);

/*
 * pd_workspace_query -- device workspace bytes a context holds for one call of
 * operation `op` with these parameters (n = P pairs for PD_OP_SINKHORN and
 * PD_OP_BOUNDS, N diagrams for the others; k = measures or centroids, read by
 * the k-means operations only).  The figure is the largest the call needs
 * (with the optional caller arrays of pd_barycenter_grad / pd_kmeans_assign
 * NULL).  A context allocates this itself (grow-only, kept until
 * pd_ctx_destroy), or the caller supplies it with pd_ctx_set_workspace.
 * Library feature for memory planning; no counterpart in the paper.
 * Errors: PD_ERR_INVALID (unknown op, NULL bytes/params, bad d, n or k).
 */
enum { PD_OP_SINKHORN = 0, PD_OP_BOUNDS = 1, PD_OP_BARYCENTER = 2, PD_OP_BARY_GRAD = 3,
       PD_OP_KMEANS_ASSIGN = 4, PD_OP_KMEANS = 5 };
pd_status pd_workspace_query(int op, const pd_sinkhorn_params* params, int n, int k, size_t* bytes);

/*
 * pd_ctx_set_workspace -- make `ws` (device memory of `bytes` bytes, 256-byte
 * aligned, owned by the caller) the context's workspace: from then on the
 * context allocates no workspace of its own (it frees what it held), and a
 * call whose need (pd_workspace_query) exceeds `bytes` returns PD_ERR_OOM
 * without running.  ws = NULL returns to library-allocated workspace.  The
 * buffer must stay valid until the next pd_ctx_set_workspace or
 * pd_ctx_destroy; calls on this context overwrite it.  Synchronises the
 * device.  (The serving pools of pd_serve_create are sized by their own
 * configuration.)  Errors: PD_ERR_INVALID (misaligned ws), PD_ERR_CUDA.
 */
pd_status pd_ctx_set_workspace(pd_ctx* ctx, void* ws, size_t bytes);

/*
 * pd_barycenter -- Alg. 2 (smoothed barycenter).  z starts as z_init, or, when
 * z_init is NULL, as the uniform measure above the diagonal (every cell j >= i
 * gets mean_i |D_i| / (d(d+1)/2)).  Each of the outer_iters steps solves the N
 * pairs (z + R a_i, a_i + R z) with the PD_FP32 engine (warm-started from the
 * previous step's g_i, the first step cold) and applies the multiplicative
 * update z <- z exp(-lambda grad) where z > 0, with the gradient of the
 * smoothed energy (the gradient proposition of Sec. 4) averaged over i:
 *   grad(x) = mean_i [ gamma log z(x) + f_i(x) + gamma log|z| + g_i(Delta) ].
 *   hist, mass  : uint32 [N][d][d], uint32 [N] (device)
 *   params      : inner Sinkhorn parameters (precision must be PD_FP32)
 *   lambda      : step size (> 0); outer_iters >= 0
 *   z_init      : double [d*d] or NULL (device); z_out: double [d*d] (device)
 *   rel_energy_tol : the stop of the barycenter experiment (Sec. 5): after step
 *                 t >= 1, stop when |E_t / E_{t-1} - 1| < rel_energy_tol, E_t the
 *                 energy of z_t below (the update of step t is applied first);
 *                 0 runs all outer_iters steps
 *   energy      : double [outer_iters] or NULL: mean transport cost of step t's
 *                 plans, (1/N) sum_i <P_i, C> (the energy of z_t) (device);
 *                 entries past the steps run are not written
 *   steps_host  : int (host) or NULL: number of steps run
 * Synchronises `stream` (once per step when rel_energy_tol > 0, to read E_t).
 * Errors: PD_ERR_INVALID, PD_ERR_OOM, PD_ERR_CUDA.
 */
pd_status pd_barycenter(pd_ctx* ctx, const uint32_t* hist, const uint32_t* mass, int N,
                        const pd_sinkhorn_params* params, double lambda, int outer_iters,
                        double rel_energy_tol, const double* z_init, double* z_out, double* energy,
                        int* steps_host, pd_stream stream);

/*
 * pd_barycenter_grad / pd_barycenter_apply -- one Alg. 2 step split at its only
 * exchange: the gradient of the smoothed energy (gradient proposition of
 * Sec. 4) is a sum over the diagrams, so a batch of diagrams sharded across
 * processes (one GPU each) computes per-shard sums, adds them across the
 * shards (an all-reduce of k*d*d + 2k doubles), and applies the same update
 * everywhere.  With one shard the two calls give bitwise the step of
 * pd_barycenter (k = 1) or of pd_kmeans' centroid update.
 *
 * pd_barycenter_grad solves this shard's N pairs (z_c + R a_n, a_n + R z_c),
 * c = owner[n], with the PD_FP32 engine and writes, for every measure c and
 * cell x:
 *   gsum[c][x] = sum over the shard's n with owner[n] = c of f_n(x) + g_n(Delta)
 *                (in diagram order; 0 where z_c(x) <= 0),
 *   count[c]   = the number of those n,
 *   cost_sum[c]= the sum of their transport costs <P_n, C>.
 *   hist, mass : uint32 [N][d][d], uint32 [N] (device): this shard's diagrams
 *   k, z       : number of measures; double [k][d*d] (device, read only)
 *   owner      : int32 [N] (device) or NULL (every n belongs to measure 0);
 *                a value outside [0, k) gives PD_ERR_INVALID (checked on the device first)
 *   g_warm     : double [N][d*d+1] (device) or NULL: the pairs' potentials g,
 *                written on return; read as the warm start when warm != 0
 *   gsum       : double [k][d*d]; count, cost_sum: double [k] (device, output)
 *   params     : as pd_barycenter (PD_FP32; bary_sharpen must be 0)
 * pd_barycenter_apply updates z in place with the summed values:
 *   z_c(x) <- z_c(x) exp(-lambda (gamma log z_c(x) + gamma log|z_c| + gsum[c][x] / count[c]))
 * where z_c(x) > 0 and count[c] > 0 (measures with count 0 are unchanged).
 * Both synchronise `stream`.  Errors: PD_ERR_INVALID, PD_ERR_OOM, PD_ERR_CUDA.
 */
pd_status pd_barycenter_grad(pd_ctx* ctx, const uint32_t* hist, const uint32_t* mass, int N, int k,
                             const pd_sinkhorn_params* params, const double* z, const int32_t* owner,
                             double* g_warm, int warm, double* gsum, double* count, double* cost_sum,
                             pd_stream stream);
pd_status pd_barycenter_apply(pd_ctx* ctx, double* z, int k, int d, const double* gsum, const double* count,
                              double gamma, double lambda, pd_stream stream);

/*
 * pd_kmeans_assign -- the assignment half of a k-means round (Sec. 5) against
 * given real-valued centroids: cold-started PD_FP32 solves of the N x k pairs
 * (a_n + R z_c, z_c + R a_n), assign[n] = argmin_c <P, C> (ties to the lowest
 * c), objective = sum_n min_c <P, C> (diagram order).  With
 * pd_barycenter_grad / pd_barycenter_apply (k measures, owner = assign) it
 * makes the k-means round of pd_kmeans for diagrams sharded across processes.
 *   hist, mass : uint32 [N][d][d], uint32 [N] (device); centroids: double [k][d*d] (device)
 *   assign     : int32 [N] (device, output)
 *   cost       : double [N][k] or NULL (device, output: every pair's cost)
 *   objective  : double [1] or NULL (device, output)
 * Synchronises `stream`.  Errors: PD_ERR_INVALID, PD_ERR_OOM, PD_ERR_CUDA.
 */
pd_status pd_kmeans_assign(pd_ctx* ctx, const uint32_t* hist, const uint32_t* mass, int N, int k,
                           const pd_sinkhorn_params* params, const double* centroids, int32_t* assign,
                           double* cost, double* objective, pd_stream stream);

/*
 * pd_kmeans -- k-means on persistence diagrams (Sec. 5): centroids start as k
 * distinct input histograms drawn by splitmix64(seed) (draw r mod N, repeats
 * skipped).  Each round assigns every diagram n to argmin_c <P, C> of the pair
 * (a_n + R z_c, z_c + R a_n) (cold-started PD_FP32 solves; ties go to the lowest
 * c), then moves every non-empty cluster's centroid by bary_steps steps of
 * Alg. 2 over its members (the first step cold, the others warm-started); an
 * empty cluster keeps its centroid.
 *   hist, mass : uint32 [N][d][d], uint32 [N] (device); 1 <= k <= N
 *   assign     : int32 [N] (device, output: assignment of the last round)
 *   centroids  : double [k][d*d] (device, output)
 *   objective  : double [rounds] or NULL (device): sum_n min_c cost at each round
 * Synchronises `stream`.  Errors: PD_ERR_INVALID, PD_ERR_OOM, PD_ERR_CUDA.
 */
pd_status pd_kmeans(pd_ctx* ctx, const uint32_t* hist, const uint32_t* mass, int N, int k,
                    const pd_sinkhorn_params* params, double lambda, int rounds, int bary_steps,
                    uint64_t seed, int32_t* assign, double* centroids, double* objective, pd_stream stream);

/*
 * Serving (pd_serve_*): a request loop with continuous batching for
 * distance and nearest-centroid queries.  The paper has no serving component;
 * the queries are the uses of the distance that Sec. 5 makes (pairwise
 * distances between diagrams, assignment of a diagram to the nearest of k
 * centroids), each answered by a PD_FP32 solve of Alg. 1.
 *
 * A server owns one pool of pair slots per grid size d in {32, 64, 128, 256};
 * a slot is the device workspace of one Sinkhorn pair.  A worker thread runs
 * scheduling rounds: it admits queued queries in FIFO order (per d) while their
 * pairs fit in free slots (distance: 1 pair, nearest: one pair per resident
 * centroid of that d), rasterises and sets them up, runs inner_iters
 * iterations of every active pair of every pool (one launch per pool, pools on
 * their own streams, so the work of all admitted queries overlaps on the
 * device), then finalises the pairs that stopped and releases their slots.
 * Queries that arrive while others are on the GPU join at the next round.
 * Centroids stay resident in device memory; with warm_start, the solve of a
 * query against centroid c starts from the centroid-side potential g of the
 * last finished solve against c (its support entries and Delta).  Each
 * half-step takes the pairwise form while it has at most twice the separable
 * form's terms (the batch calls allow 5 times): a pool's launch carries pairs
 * of every size, the largest sets its shared memory, and the pairwise form
 * loses where few CTAs fit on an SM.
 *
 * All entry points are thread-safe.  Points are host arrays, copied at submit.
 */
typedef struct pd_server pd_server;

typedef struct {
    double gamma;          /* entropic regularisation of every solve (> 0) */
    double tol;            /* relative marginal tolerance of every solve (>= 0) */
    int max_iter;          /* iterations per solve at most (>= 1) */
    int inner_iters;       /* iterations per scheduling round (<= 0: 64) */
    int slots[4];          /* pair slots for d = 32, 64, 128, 256; 0: from max_hbm_bytes;
                              < 0: no pool for that d (its queries are refused) */
    size_t max_hbm_bytes;  /* device memory shared equally by the pools whose slots[] is 0
                              (0: half of the free device memory at creation) */
    int queue_capacity;    /* queries submitted and not yet polled at most (<= 0: 65536) */
    int warm_start;        /* 1: nearest-centroid solves start from the last g of that centroid */
} pd_serve_config;

enum { PD_Q_DISTANCE = 0, PD_Q_NEAREST = 1 };

typedef struct {
    int kind;                  /* PD_Q_DISTANCE or PD_Q_NEAREST */
    int d;                     /* 32, 64, 128 or 256 */
    const double* birth_a_host;/* diagram A: n_a points (host, copied at submit) */
    const double* death_a_host;
    int n_a;
    const double* birth_b_host;/* diagram B (PD_Q_DISTANCE only) */
    const double* death_b_host;
    int n_b;
} pd_query;

typedef struct {
    pd_status status;    /* PD_OK; PD_NOT_CONVERGED if a solve hit max_iter; PD_ERR_* on failure */
    double cost;         /* distance: <P, C> of (A, B); nearest: <P, C> to the nearest centroid */
    int centroid;        /* nearest: index of the nearest centroid (ties: lowest); distance: -1 */
    int iters;           /* largest iteration count over the query's solves */
    double latency_ms;   /* submit to completion, host steady clock */
} pd_result;

/* Default configuration: gamma 5e-3, tol 1e-4, max_iter 5000, inner_iters 64,
 * slots from half the free memory, queue_capacity 65536, warm_start 1. */
void pd_serve_default_config(pd_serve_config* cfg);
/* Create a server on ctx's device (ctx must outlive the server; the server
 * does not use ctx's workspace).  Allocates the slot pools.
 * Errors: PD_ERR_INVALID (bad config), PD_ERR_OOM, PD_ERR_CUDA. */
pd_status pd_serve_create(pd_ctx* ctx, const pd_serve_config* cfg, pd_server** out);
/* Make z (double [k][d*d], device, non-negative weights) the resident centroids
 * of grid size d (copied; replaces earlier ones and their warm potentials).
 * Errors: PD_ERR_INVALID if d is not a pool size, k < 1, k exceeds the pool's
 * slots, or a query of size d is in flight; PD_ERR_OOM; PD_ERR_CUDA. */
pd_status pd_serve_load_centroids(pd_server* sv, int d, const double* z, int k);
/* Queue a query; *ticket identifies it.  Points must be finite with
 * 0 <= birth <= death <= 1 (checked here).  Errors: PD_ERR_INVALID (bad query,
 * no centroids loaded for a nearest query), PD_ERR_QUEUE_FULL, PD_ERR_CUDA (the
 * server stopped after a device error). */
pd_status pd_serve_submit(pd_server* sv, const pd_query* q, uint64_t* ticket);
/* Result of a ticket: PD_PENDING while it runs; otherwise the query's status,
 * with *out filled, and the ticket is released.  PD_ERR_INVALID for an unknown
 * ticket. */
pd_status pd_serve_poll(pd_server* sv, uint64_t ticket, pd_result* out);
/* As pd_serve_poll, but waits up to timeout_ms (< 0: without limit) for the
 * result; PD_PENDING if it is still running then. */
pd_status pd_serve_wait(pd_server* sv, uint64_t ticket, pd_result* out, double timeout_ms);
/* Host-side fault injection for tests: the next scheduling round fails as if
 * a CUDA call had failed, without touching the device.  The server then
 * fails every admitted and queued query with PD_ERR_CUDA and refuses new ones. */
pd_status pd_serve_inject_failure(pd_server* sv);
/* Stop the worker, drop unfinished queries, release the pools.  Safe on NULL. */
void pd_serve_destroy(pd_server* sv);

/* Kernel classes recorded by the launch profiler. */
enum {
    PD_K_RASTER = 0,   /* rasteriser */
    PD_K_SETUP = 1,    /* per-pair set-up of a Sinkhorn batch */
    PD_K_LOGSTEP = 2,  /* exact log-domain first iteration */
    PD_K_ABSORB = 3,   /* absorption / re-centring */
    PD_K_ITER = 4,     /* linear-domain Sinkhorn iterations (the GEMM kernel) */
    PD_K_FINALIZE = 5, /* transport cost (Prop. 2), marginals, potentials */
    PD_K_TC = 6,       /* tensor-core (tcgen05) iterations of the PD_BF16 engine */
    PD_K_COUNT = 16
};

/*
 * pd_profile_enable -- start (enable != 0) or stop recording a pair of CUDA
 * events around every kernel launch the library makes on ctx, on the stream
 * the kernel is launched on; starting clears earlier records.  Library
 * feature for tracing; no counterpart in the paper.
 */
pd_status pd_profile_enable(pd_ctx* ctx, int enable);

/*
 * pd_profile_read -- synchronise the recorded events and report, per kernel
 * class k < PD_K_COUNT: ms_host[k] = summed launch durations (milliseconds),
 * launches_host[k] = number of launches.  Host pointers of PD_K_COUNT
 * entries; either may be NULL.
 */
pd_status pd_profile_read(pd_ctx* ctx, double* ms_host, int64_t* launches_host);

/*
 * pd_sinkhorn_batch_noalloc -- the PD_FP32 solve of pd_sinkhorn_batch without
 * any device memory allocation.  (A library feature; the paper has no
 * counterpart.)
 *
 * For callers that must not allocate device memory: applications that hand
 * all device memory to their own pool allocator and forbid libraries from
 * calling cudaMalloc / cudaFree (which also synchronise the whole device and
 * can fail once the pool holds the memory), and latency-critical serving
 * threads that cannot afford an allocation's implicit device-wide
 * synchronisation.  It takes no pd_ctx (a context allocates) and calls no
 * cudaMalloc, cudaFree or other device-allocating routine.
 *
 * Its workspace is a fixed 16 MiB array in device memory that every GPU that
 * loads this library holds until the process exits.  That bounds the batch: the
 * pairs must fit in 16 MiB of workspace, about 9 pairs at d = 100..128 and 35
 * pairs at d <= 64; a larger P returns PD_ERR_INVALID.  params->precision must
 * be PD_FP32, params->p must be 2 and params->eps_stages must be 0 (the
 * gamma-continuation is not run here; other values return PD_ERR_INVALID).
 * Arguments, outputs and results are those of pd_sinkhorn_batch, computed on
 * the current CUDA device.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the one array and it keeps the last call's contents (each
 * call initialises everything it reads), so calls whose GPU work overlaps --
 * on two streams, or from two host threads -- race and corrupt each other's
 * results; serialise them.  Like pd_sinkhorn_batch, the call reads per-pair
 * counters back to the host between its launches and synchronises `stream`
 * before it returns.
 * Errors: PD_ERR_INVALID (bad params, NULL input/cost, P too large for the
 * array), PD_ERR_CUDA.
 */
pd_status pd_sinkhorn_batch_noalloc(const uint32_t* histA, const uint32_t* massA,
                                    const uint32_t* histB, const uint32_t* massB, const int32_t* pairs, int P,
                                    const pd_sinkhorn_params* params, const double* g_init,
                                    double* cost, float* row_marg, float* col_marg, double* f, double* g,
                                    int32_t* iters, float* err, int32_t* status, pd_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* PD_OT_H */
