// api.cu -- host implementation of the C ABI declared in include/pd_ot.h.
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>
#include <cmath>
#include <atomic>
#include <map>
#include <utility>

#include "pd_internal.h"
#include "../../include/pd_ot.h"


struct pd_ctx {
    int device = 0;
    std::string err;
    void* ws = nullptr;        // Sinkhorn workspace
    size_t ws_bytes = 0;
    void* ws2 = nullptr;       // outer-loop buffers (barycenter, k-means)
    size_t ws2_bytes = 0;
    int* dflag = nullptr;      // small device scratch (error flags, counters)
    int* hflag = nullptr;      // pinned host mirror
    double* hval = nullptr;    // pinned host doubles (per-step energies)
    // caller-supplied workspace (pd_ctx_set_workspace): when set, ws is carved
    // from its start and ws2 from its end, and nothing is allocated
    char* ext = nullptr;
    size_t ext_bytes = 0;
    size_t ws2_live = 0;       // bytes of ext used by ws2 in the current call
    // tuning table: (d, support-size bucket) -> first CTA width of the base-2 kernel
    std::map<std::pair<int, int>, int> tune;
    // launch profiler
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;   // free events
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> recs;
};

// RAII helper: records events around one kernel launch when profiling is on.
struct ProfScope {
    pd_ctx* c; int kind; cudaStream_t s; cudaEvent_t a = nullptr, b = nullptr;
    static cudaEvent_t get(pd_ctx* c) {
        if (!c->ev_pool.empty()) { cudaEvent_t e = c->ev_pool.back(); c->ev_pool.pop_back(); return e; }
        cudaEvent_t e; cudaEventCreate(&e); return e;
    }
    ProfScope(pd_ctx* c_, int k, cudaStream_t s_) : c(c_), kind(k), s(s_) {
        if (c && c->prof) { a = get(c); b = get(c); cudaEventRecord(a, s); }
    }
    ~ProfScope() {
        if (c && c->prof) { cudaEventRecord(b, s); c->recs.push_back({kind, a, b}); }
    }
};

int pd_ctx_device(const pd_ctx* c) { return c ? c->device : 0; }

static pd_status fail(pd_ctx* c, pd_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}
#define CUDA_TRY(ctx, expr)                                                                   \
    do {                                                                                      \
        cudaError_t _e = (expr);                                                              \
        if (_e != cudaSuccess)                                                                \
            return fail(ctx, PD_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(_e));    \
    } while (0)

// Start of every entry point that takes a context: clear the message and the
// per-call use of a caller-supplied workspace.
static void call_begin(pd_ctx* c) {
    c->err.clear();
    c->ws2_live = 0;
}

extern "C" int pd_abi_version(void) { return 3; }

extern "C" pd_status pd_ctx_create(int device, pd_ctx** out) {
    if (!out) return PD_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return PD_ERR_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return PD_ERR_CUDA;
    pd_ctx* c = new pd_ctx();
    c->device = device;
    if (cudaMalloc(&c->dflag, 64 * sizeof(int)) != cudaSuccess) { delete c; return PD_ERR_OOM; }
    if (cudaMallocHost(&c->hflag, 64 * sizeof(int)) != cudaSuccess) { cudaFree(c->dflag); delete c; return PD_ERR_OOM; }
    if (cudaMallocHost(&c->hval, 8 * sizeof(double)) != cudaSuccess) {
        cudaFree(c->dflag); cudaFreeHost(c->hflag); delete c; return PD_ERR_OOM;
    }
    *out = c;
    return PD_OK;
}

extern "C" void pd_ctx_destroy(pd_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto& r : c->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (!c->ext) {
        if (c->ws) cudaFree(c->ws);
        if (c->ws2) cudaFree(c->ws2);
    }
    if (c->dflag) cudaFree(c->dflag);
    if (c->hflag) cudaFreeHost(c->hflag);
    if (c->hval) cudaFreeHost(c->hval);
    delete c;
}

extern "C" const char* pd_last_error(const pd_ctx* c) { return c ? c->err.c_str() : "null context"; }

extern "C" pd_status pd_profile_enable(pd_ctx* c, int enable) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    if (enable) {
        if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, PD_ERR_CUDA, "cudaSetDevice failed");
        for (auto& r : c->recs) { c->ev_pool.push_back(r.a); c->ev_pool.push_back(r.b); }
        c->recs.clear();
    }
    c->prof = enable != 0;
    return PD_OK;
}

extern "C" pd_status pd_profile_read(pd_ctx* c, double* ms, int64_t* launches) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    if (ms) for (int k = 0; k < PD_K_COUNT; ++k) ms[k] = 0.0;
    if (launches) for (int k = 0; k < PD_K_COUNT; ++k) launches[k] = 0;
    for (auto& r : c->recs) {
        CUDA_TRY(c, cudaEventSynchronize(r.b));
        float t = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&t, r.a, r.b));
        if (r.kind >= 0 && r.kind < PD_K_COUNT) {
            if (ms) ms[r.kind] += t;
            if (launches) launches[r.kind] += 1;
        }
    }
    return PD_OK;
}

extern "C" pd_status pd_rasterize(pd_ctx* c, const double* birth, const double* death, const int64_t* offsets,
                                  int B, int d, uint32_t* hist, uint32_t* mass, pd_stream stream) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    if (B < 0 || d < 2 || d > 256) return fail(c, PD_ERR_INVALID, "pd_rasterize: need B >= 0 and 2 <= d <= 256");
    if (B == 0) return PD_OK;
    if (!offsets || !hist || !mass) return fail(c, PD_ERR_INVALID, "pd_rasterize: NULL pointer");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(c, cudaSetDevice(c->device));
    int64_t npts = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&npts, offsets + B, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaMemsetAsync(c->dflag, 0, sizeof(int), s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (npts < 0) return fail(c, PD_ERR_INVALID, "pd_rasterize: offsets[B] < 0");
    if (npts > 0 && (!birth || !death)) return fail(c, PD_ERR_INVALID, "pd_rasterize: NULL points");
    { ProfScope ps(c, PD_K_RASTER, s);
      CUDA_TRY(c, pd_launch_raster(birth, death, offsets, B, d, npts, hist, mass, c->dflag, s)); }
    CUDA_TRY(c, cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (c->hflag[0]) return fail(c, PD_ERR_INVALID, "pd_rasterize: a point is not a finite point of [0,1]^2 with birth <= death");
    return PD_OK;
}

extern "C" void pd_sinkhorn_default_params(pd_sinkhorn_params* p, double gamma, int d) {
    if (!p) return;
    p->gamma = gamma;
    p->d = d;
    p->max_iter = 20000;
    p->tol = 1e-6;
    p->precision = PD_FP32;
    p->refine_iters = 0;
    p->absorb_tau = 20.0;
    p->absorb_every = 64;
    p->rel_log_thresh = 0.0;
    p->eps_stages = 0;
    p->p = 2.0;
    p->bary_sharpen = 0;
    p->cta_threads = 0;
    p->kernel_tier = 0;
    p->max_inner = 0;
    p->diag_tc_timeout = 0;
    p->lse_form = 0;
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Carve the workspace for P pairs at padded size dp; returns bytes needed when
// base == nullptr.
size_t pd_carve_ws(char* base, int P, int d, int dp, double gamma, SkWS* w, int** counter) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* { char* r = base ? base + off : nullptr; off += align256(bytes); return r; };
    const size_t M = (size_t)dp * dp, n = M + 1;
    SkWS t{};
    t.d = d; t.dp = dp; t.n = (int)n; t.P = P; t.gamma = gamma; t.p = 2.0;
    float** fm[] = {&t.K1u, &t.K2u, &t.K1v, &t.K2v, &t.ut, &t.vt, &t.Wt, &t.Rt, &t.KDu, &t.KDv, &t.am, &t.bm};
    for (auto f : fm) *f = (float*)take(sizeof(float) * M * P);
    float** fv[] = {&t.rs_u, &t.cf_u, &t.rs_v, &t.cf_v};
    for (auto f : fv) *f = (float*)take(sizeof(float) * dp * P);
    double** dv[] = {&t.ap, &t.bp, &t.al, &t.be, &t.Au, &t.Bu, &t.Av, &t.Bv};
    for (auto f : dv) *f = (double*)take(sizeof(double) * dp * P);
    t.phi = (double*)take(sizeof(double) * n * P);
    t.psi = (double*)take(sizeof(double) * n * P);
    t.sc = (double*)take(sizeof(double) * SC_N * P);
    t.sa = (int*)take(sizeof(int) * M * P);
    t.sb = (int*)take(sizeof(int) * M * P);
    t.ic = (int*)take(sizeof(int) * IC_N * P);
    t.L64 = (double*)take(sizeof(double) * 2 * M * P);
    t.la = (double*)take(sizeof(double) * M * P);
    t.lb = (double*)take(sizeof(double) * M * P);
    t.rpa = (int*)take(sizeof(int) * (dp + 1) * P);
    t.rpb = (int*)take(sizeof(int) * (dp + 1) * P);
    t.cpa = (int*)take(sizeof(int) * (dp + 1) * P);
    t.cpb = (int*)take(sizeof(int) * (dp + 1) * P);
    t.cia = (int*)take(sizeof(int) * M * P);
    t.cib = (int*)take(sizeof(int) * M * P);
    t.ctab = (float*)take(sizeof(float) * 5 * dp);
    t.order_buf = (int*)take(sizeof(int) * P);
    t.order = nullptr;
    t.groups = (SkWS*)take(sizeof(SkWS));
    t.ngroups = 1;
    *counter = (int*)take(sizeof(int) * 8);
    if (w) *w = t;
    return off;
}


// Cost tables for m = 0..dp-1 (physical units, z = m/d): c_m/gamma = z^2/gamma and
// cD_m/gamma = z^2/(2 gamma), each split into FP32 hi + lo words; log c_m = 2 log z.
cudaError_t pd_upload_cost_tables(const SkWS& w, double gamma, cudaStream_t s) {
    const int dp = w.dp, d = w.d;
    std::vector<float> tab(5 * dp);
    const double pw = w.p;
    for (int m = 0; m < dp; ++m) {
        double z = (double)m / d;
        double v = pw == 2.0 ? z * z / gamma : std::pow(z, pw) / gamma;
        double v2 = pw == 2.0 ? 0.5 * z * z / gamma : 2.0 * std::pow(0.5 * z, pw) / gamma;
        float hi = (float)v, hi2 = (float)v2;
        tab[m] = hi;
        tab[dp + m] = (float)(v - (double)hi);
        tab[2 * dp + m] = hi2;
        tab[3 * dp + m] = (float)(v2 - (double)hi2);
        tab[4 * dp + m] = m == 0 ? -INFINITY : (float)(pw * std::log(z));
    }
    return cudaMemcpyAsync(w.ctab, tab.data(), sizeof(float) * 5 * dp, cudaMemcpyHostToDevice, s);
}

// Host-side view of pair p of a workspace as a one-pair workspace (the same
// per-pair offsets as the device-side pair_ptrs); used by the one-pair-per-
// launch engine.  Inputs and the pair list are not offset: only kernels that
// read per-pair state may be given a view.
static SkWS ws_view(const SkWS& w, int p) {
    SkWS v = w;
    const size_t M = (size_t)w.dp * w.dp, V = (size_t)w.dp, N = (size_t)w.n;
    float** fm[] = {&v.K1u, &v.K2u, &v.K1v, &v.K2v, &v.ut, &v.vt, &v.Wt, &v.Rt, &v.KDu, &v.KDv, &v.am, &v.bm};
    for (auto f : fm) *f += p * M;
    float** fv[] = {&v.rs_u, &v.cf_u, &v.rs_v, &v.cf_v};
    for (auto f : fv) *f += p * V;
    double** dv[] = {&v.ap, &v.bp, &v.al, &v.be, &v.Au, &v.Bu, &v.Av, &v.Bv};
    for (auto f : dv) *f += p * V;
    v.phi += p * N; v.psi += p * N; v.sc += (size_t)p * SC_N;
    v.sa += p * M; v.sb += p * M; v.ic += (size_t)p * IC_N;
    v.L64 += 2 * p * M; v.la += p * M; v.lb += p * M;
    v.rpa += p * (V + 1); v.rpb += p * (V + 1); v.cpa += p * (V + 1); v.cpb += p * (V + 1);
    v.cia += p * M; v.cib += p * M;
    v.P = 1;
    v.order = nullptr;
    v.histA = v.histB = nullptr; v.massA = v.massB = nullptr; v.wA = v.wB = nullptr; v.pairs = nullptr;
    return v;
}

static SkRun make_run(const pd_sinkhorn_params* prm) {
    SkRun r{};
    r.max_iter = prm->max_iter;
    r.tol = prm->tol;
    r.tau = prm->absorb_tau > 0 ? prm->absorb_tau : 20.0;
    r.absorb_every = prm->absorb_every > 0 ? prm->absorb_every : 64;
    r.rel_thresh = prm->rel_log_thresh < 0 ? prm->rel_log_thresh : (prm->precision == PD_BF16 ? -14.0 : -21.0);
    r.pot_support_only = 0;
    r.eps_stages = (prm->precision == PD_FP32 && prm->eps_stages > 0) ? std::min(prm->eps_stages, 16) : 0;
    r.cta_threads = prm->cta_threads;
    r.tier = prm->kernel_tier;
    r.max_inner = prm->max_inner > 0 ? prm->max_inner : 0;
    r.diag_tc_timeout = prm->precision == PD_BF16 && prm->diag_tc_timeout != 0;
    r.form = prm->lse_form;
    return r;
}

// Grow-only device buffer owned by the context, or, with a caller-supplied
// workspace, a range of it: the Sinkhorn workspace (ws) at its start, the
// outer-loop buffers (ws2, always taken first within a call) at its end.
static pd_status ensure_buffer(pd_ctx* c, void** buf, size_t* have, size_t need, cudaStream_t s) {
    if (c->ext) {
        const bool is_ws2 = (buf == &c->ws2);
        const size_t n = align256(need);
        if (is_ws2 ? n > c->ext_bytes : n + c->ws2_live > c->ext_bytes)
            return fail(c, PD_ERR_OOM, "caller-supplied workspace of %zu bytes is too small (%zu more needed)",
                        c->ext_bytes, n + (is_ws2 ? 0 : c->ws2_live) - c->ext_bytes);
        if (is_ws2) {
            *buf = c->ext + (c->ext_bytes - n);
            c->ws2_live = n;
        } else {
            *buf = c->ext;
        }
        *have = n;
        return PD_OK;
    }
    if (need <= *have) return PD_OK;
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    if (cudaMalloc(buf, need) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PD_ERR_OOM, "cannot allocate %zu bytes of workspace", need);
    }
    *have = need;
    return PD_OK;
}

// The PD_FP32 (log-domain) solve of the pairs described by w, on stream s:
// set-up, iteration rounds until every pair stops, finalize.  Synchronises s
// once per round (convergence check).
static pd_status lse_iterate(pd_ctx* c, SkWS& w, SkRun r, double* cost, float* row_marg, float* col_marg,
                             double* f, double* g, int32_t* iters, float* err, int32_t* status, int* counter,
                             cudaStream_t s);

// Iteration rounds of the log-domain engine: each round runs up to 64
// iterations of every active pair in the on-chip kernel (base-2 kernel when
// gamma allows a grid, else the double-float one), then its global-memory
// variant for the pairs whose supports do not fit on chip, then the FP64
// global-memory kernel for the pairs too large for that or whose potentials
// left the base-2 range, until
// no pair is active.  counter: 8 device ints; hbuf: 4 host ints; c (may be
// NULL) receives the per-launch profile records.
// Support-size profile of a batch for the tuning table: half-octave bucket of
// the mean number of support cells per side.
static int support_bucket(double mean_cells) { return (int)std::floor(2.0 * std::log2(mean_cells + 1.0)); }

// gs: the workspaces of the launch (one per grid size; gs[0] alone for a
// single batch); dev_groups: device array of gs.size() descriptors (filled
// here); order_buf: device ints for all pairs of all workspaces.
static cudaError_t lse_rounds_groups(pd_ctx* c, std::vector<SkWS>& gs, SkWS* dev_groups, int* order_buf, SkRun r,
                                     int* counter, int* hbuf, cudaStream_t s) {
    cudaError_t e;
    const int G = (int)gs.size();
    int Ptot = 0, dmax = 0;
    for (auto& g : gs) { Ptot += g.P; dmax = std::max(dmax, g.d); }
    if (Ptot == 0) return cudaSuccess;
    // Every pair runs to its stop inside one launch (its CTA iterates until
    // convergence or max_iter), so no round barrier idles the SMs; CTAs are
    // handed out largest support first, which keeps the long solves from
    // starting last (makespan).  r.max_inner caps the iterations per launch.
    int n_inner = r.max_iter;
    if (r.max_inner > 0 && r.max_inner < n_inner) n_inner = r.max_inner;
    const int* order = nullptr;
    if ((Ptot > 1 || G > 1) && order_buf) {
        std::vector<int> code, size;
        code.reserve(Ptot); size.reserve(Ptot);
        for (int gi = 0; gi < G; ++gi) {
            std::vector<int> ic((size_t)gs[gi].P * IC_N);
            if (gs[gi].P == 0) continue;
            if ((e = cudaMemcpyAsync(ic.data(), gs[gi].ic, ic.size() * sizeof(int), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            for (int p = 0; p < gs[gi].P; ++p) {
                code.push_back((gi << 24) | p);
                size.push_back(ic[(size_t)p * IC_N + IC_NA] + ic[(size_t)p * IC_N + IC_NB]);
            }
        }
        std::vector<int> ord(Ptot);
        for (int k = 0; k < Ptot; ++k) ord[k] = k;
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return size[a] > size[b]; });
        std::vector<int> codes(Ptot);
        for (int k = 0; k < Ptot; ++k) codes[k] = code[ord[k]];
        if (c && r.cta_threads == 0 && r.base_threads == 0 && !c->tune.empty()) {
            double tot = 0;
            for (int k = 0; k < Ptot; ++k) tot += size[k];
            auto it = c->tune.find({dmax, support_bucket(tot / (2.0 * Ptot))});
            if (it != c->tune.end()) r.base_threads = it->second;
        }
        if ((e = cudaMemcpyAsync(order_buf, codes.data(), sizeof(int) * Ptot, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        order = order_buf;
    }
    // device descriptors: every workspace with its own pointers (no order)
    for (int gi = 0; gi < G; ++gi) {
        SkWS d = gs[gi];
        d.order = nullptr;
        d.groups = dev_groups + gi;
        d.ngroups = 1;
        gs[gi].groups = dev_groups + gi;
        gs[gi].ngroups = 1;
        if ((e = cudaMemcpyAsync(dev_groups + gi, &d, sizeof(SkWS), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    }
    // the launch over all pairs of all workspaces
    SkWS wall = gs[0];
    wall.P = Ptot;
    wall.order = order;
    wall.groups = dev_groups;
    wall.ngroups = G;
    wall.d = dmax;
    // a pair can spend one round in each of the two hand-overs between kernels
    // and one in each of the two widenings below
    const int max_rounds = r.max_iter / n_inner + 6;
    const int gbits = sk_lse2_grid_bits(gs[0].gamma);
    size_t smem = 0;
    bool pw_all = false;   // every on-chip pair pairwise in both half-steps
    if (gbits >= 0) {
        if ((e = cudaMemsetAsync(counter + 2, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
        for (int gi = 0; gi < G; ++gi)
            if ((e = sk_launch_lse2_need(gs[gi], counter + 2, r.form, s)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(hbuf + 2, counter + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        smem = (size_t)hbuf[2];
        pw_all = hbuf[3] == 0;
        if (r.batch_form && r.form == 0 && smem > 0) {
            // the launch's shared memory is the largest pair's: where records
            // push it past a CTA-per-SM step (at most 3 count), the pairwise
            // half-steps run latency-bound in few warps; the whole call then
            // takes the separable form (dense barycenter sides at d = 64)
            if ((e = cudaMemsetAsync(counter + 2, 0, 2 * sizeof(int), s)) != cudaSuccess) return e;
            for (int gi = 0; gi < G; ++gi)
                if ((e = sk_launch_lse2_need(gs[gi], counter + 2, 1, s)) != cudaSuccess) return e;
            if ((e = cudaMemcpyAsync(hbuf + 2, counter + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost, s)) !=
                cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            const size_t smem1 = (size_t)hbuf[2];
            int dv = 0, per_sm = 0;
            cudaGetDevice(&dv);
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dv);
            auto ctas = [&](size_t b) { return std::min(3, (int)((size_t)per_sm / (b + 2048))); };
            if (ctas(smem1) > ctas(smem)) {
                r.form = 1;
                smem = smem1;
                pw_all = false;
            }
        }
    }
    // CTA width of the base-2 kernel: 256 threads while there are several pairs
    // per SM, wider CTAs (more warps on one pair) once fewer pairs than SMs
    // remain.  r.cta_threads fixes it.
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // on-chip CTAs per SM that the largest pair's shared memory allows (dynamic
    // part + the kernel's static part + the runtime's 1 KB per CTA)
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int fit_per_sm = smem > 0 ? (int)((size_t)smem_sm / (smem + 2048)) : 3;
    int fixed_threads = 0;
    if (r.cta_threads == 128 || r.cta_threads == 256 || r.cta_threads == 512 || r.cta_threads == 1024)
        fixed_threads = r.cta_threads;
    if (fixed_threads == 128 && dmax > 128) fixed_threads = 256;
    // tier 1 runs every pair in the global-memory variant, tier 2 in the FP64
    // global-memory kernel (checks of the tiers against each other)
    size_t gcap = (size_t)-1;
    if (r.tier == 1) smem = 0;
    if (r.tier == 2) { smem = 0; gcap = 0; }
    int active = Ptot;
    bool any_gm = false, any_old = false;
    for (int round = 0; round < max_rounds; ++round) {
        if ((e = cudaMemsetAsync(counter, 0, 8 * sizeof(int), s)) != cudaSuccess) return e;
        {
            ProfScope ps(c, PD_K_ITER, s);
            // 256 threads while several pairs share an SM; wider CTAs once fewer
            // pairs than 2 (1) per SM remain, or when the largest pair's shared
            // memory lets only 2 (1) CTAs onto an SM (e.g. a dense barycenter
            // side), so that the SM still runs 16-32 warps; the first width
            // comes from the tuning table (base_threads) or is 256
            const int base = (r.base_threads == 128 && dmax <= 128) || r.base_threads == 512 ? r.base_threads : 256;
            // (pairwise form only: a pair keeps its width; one pair nearly
            // fills an SM's issue slots in that form, a wider CTA was measured
            // no faster, and each hand-over costs a reload)
            const int by_active =
                pw_all || active > 2 * nsm ? base : (active > nsm ? std::max(base, 512) : 1024);
            const int by_smem = fit_per_sm <= 1 ? 1024 : (fit_per_sm == 2 ? 512 : 128);
            const int threads = fixed_threads ? fixed_threads : (by_active > by_smem ? by_active : by_smem);
            // Widening: a pair alone on an SM iterates ~2x faster in a
            // 512/1024-thread CTA than in a 256-thread CTA sharing the SM, so
            // once no more than 2 (1) pairs per SM are left the launch hands
            // them over to 512 (1024)-thread CTAs.
            SkRun rl = r;
            rl.exit_at = 0;
            if (!fixed_threads && !pw_all && gbits >= 0 && n_inner == r.max_iter) {
                if (threads <= 256) rl.exit_at = active - 2 * nsm;
                else if (threads == 512) rl.exit_at = active - nsm;
            }
            if (gbits >= 0) {
                e = sk_launch_lse2(wall, rl, n_inner, counter, smem, gbits, threads, s);
            } else {
                for (int gi = 0; gi < G && e == cudaSuccess; ++gi)
                    e = sk_launch_lse_smem(gs[gi], r, n_inner, counter, counter + 1, s);
            }
            if (e != cudaSuccess) return e;
        }
        if (gbits >= 0 && any_gm) {   // pairs whose supports do not fit on chip
            ProfScope ps(c, PD_K_ITER, s);
            for (int gi = 0; gi < G; ++gi)
                if ((e = sk_launch_lse2_gm(gs[gi], r, n_inner, counter, gbits, gcap, s)) != cudaSuccess) return e;
        }
        if (any_old) {                // the FP64 global-memory kernel
            ProfScope ps(c, PD_K_ITER, s);
            for (int gi = 0; gi < G; ++gi)
                if ((e = sk_launch_lse_iter(gs[gi], r, n_inner, counter, gbits >= 0 ? 2 : 1, s)) != cudaSuccess)
                    return e;
        }
        if ((e = cudaMemcpyAsync(hbuf, counter, 4 * sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        // pairs handed on by this round's launches run from the next round on
        if (gbits >= 0) {
            if (hbuf[1] > 0) any_gm = true;
            if (hbuf[3] > 0) any_old = true;
        } else if (hbuf[1] > 0) {
            any_old = true;
        }
        if (hbuf[0] == 0) break;
        active = hbuf[0];
    }
    return cudaSuccess;
}

// Iteration rounds of the log-domain engine for one workspace (see
// lse_rounds_groups).
static cudaError_t lse_rounds(pd_ctx* c, SkWS& w, SkRun r, int* counter, int* hbuf, cudaStream_t s) {
    std::vector<SkWS> gs{w};
    cudaError_t e = lse_rounds_groups(c, gs, w.groups, w.order_buf, r, counter, hbuf, s);
    w.groups = gs[0].groups;
    w.ngroups = 1;
    return e;
}
static pd_status lse_solve(pd_ctx* c, SkWS& w, SkRun r, const double* g_init, double* cost, float* row_marg,
                           float* col_marg, double* f, double* g, int32_t* iters, float* err, int32_t* status,
                           int* counter, cudaStream_t s) {
    { ProfScope ps(c, PD_K_SETUP, s); CUDA_TRY(c, sk_launch_setup(w, g_init, s)); }
    if (r.eps_stages > 0 && sk_lse2_grid_bits(w.gamma) >= 0) {
        // gamma-continuation inside the iteration kernel: every pair starts at
        // gamma * 4^K and moves to the next stage on its own once its error is
        // <= max(tol, 1e-4) (no batch-wide barrier between stages); warm-start
        // potentials are brought to the first stage's units
        CUDA_TRY(c, sk_launch_set_stage(w, r.eps_stages, s));
        CUDA_TRY(c, sk_launch_regamma(w, std::ldexp(1.0, -2 * r.eps_stages), r.max_iter, s));
        r.kstages = r.eps_stages;
        r.stage_tol = std::max(r.tol, 1e-4);
        return lse_iterate(c, w, r, cost, row_marg, col_marg, f, g, iters, err, status, counter, s);
    }
    if (r.eps_stages > 0) {
        // gamma below the base-2 kernel's range: stages run one after the other
        // (batch-wide), at gamma * 4^k, k = eps_stages..1, each to
        // err <= max(tol, 1e-4), carrying f and g (phi = f / gamma is rescaled)
        const double g_target = w.gamma;
        double g_prev = g_target;
        for (int k = r.eps_stages; k >= 1; --k) {
            const double gk = g_target * std::ldexp(1.0, 2 * k);
            CUDA_TRY(c, sk_launch_regamma(w, g_prev / gk, r.max_iter, s));
            w.gamma = gk;
            CUDA_TRY(c, pd_upload_cost_tables(w, gk, s));
            SkRun rk = r;
            rk.tol = std::max(r.tol, 1e-4);
            CUDA_TRY(c, lse_rounds(c, w, rk, counter, c->hflag, s));
            g_prev = gk;
        }
        CUDA_TRY(c, sk_launch_regamma(w, g_prev / g_target, r.max_iter, s));
        w.gamma = g_target;
        CUDA_TRY(c, pd_upload_cost_tables(w, g_target, s));
    }
    return lse_iterate(c, w, r, cost, row_marg, col_marg, f, g, iters, err, status, counter, s);
}

// Iteration rounds of the log-domain engine from the current potentials until
// every pair stops, then finalize.
static pd_status lse_iterate(pd_ctx* c, SkWS& w, SkRun r, double* cost, float* row_marg, float* col_marg,
                             double* f, double* g, int32_t* iters, float* err, int32_t* status, int* counter,
                             cudaStream_t s) {
    CUDA_TRY(c, lse_rounds(c, w, r, counter, c->hflag, s));
    { ProfScope ps(c, PD_K_FINALIZE, s);
      CUDA_TRY(c, sk_launch_lse_finalize(w, cost, row_marg, col_marg, f, g, iters, err, status, r.pot_support_only, s)); }
    return PD_OK;
}

// Range check of the linear-domain engines after their finalize: the exact
// log-domain marginals of each pair's final plan (potentials rebuilt from the
// residual representation) are compared with a and b; a pair reported PD_OK
// whose exact marginal error exceeds max(10 tol, 1e-5) gets PD_ERR_RANGE.
static pd_status linear_range_check(pd_ctx* c, SkWS& w, double tol, int32_t* status, float* err, cudaStream_t s) {
    if (!status) return PD_OK;
    CUDA_TRY(c, sk_launch_rebuild_potentials(w, s));
    // scratch for the exact marginals, [P][d*d+1] rows then columns: the
    // consecutive arrays K1v, K2v, ut, vt (4 P dp^2 floats), which the exact
    // finalize never touches (its stage buffers are Wt, Rt, K1u, K2u and the
    // FP64 scratch) and which are free once the potentials are rebuilt
    const size_t M = (size_t)w.dp * w.dp, n_out = (size_t)w.d * w.d + 1;
    if (w.K2v != w.K1v + w.P * M || w.ut != w.K2v + w.P * M || w.vt != w.ut + w.P * M)
        return fail(c, PD_ERR_CUDA, "range check: workspace layout changed");
    float* row = w.K1v;
    float* col = row + (size_t)w.P * n_out;
    double* cost_scratch = w.Au;                             // P doubles of scratch
    { ProfScope ps(c, PD_K_FINALIZE, s);
      CUDA_TRY(c, sk_launch_lse_finalize(w, cost_scratch, row, col, nullptr, nullptr, nullptr, nullptr, nullptr, 0, s)); }
    CUDA_TRY(c, sk_launch_range_check(w, row, col, status, err, std::max(10.0 * tol, 1e-5), s));
    return PD_OK;
}

extern "C" pd_status pd_sinkhorn_batch(pd_ctx* c, const uint32_t* histA, const uint32_t* massA, const uint32_t* histB,
                                       const uint32_t* massB, const int32_t* pairs, int P,
                                       const pd_sinkhorn_params* prm, const double* g_init, double* cost,
                                       float* row_marg, float* col_marg, double* f, double* g, int32_t* iters,
                                       float* err, int32_t* status, pd_stream stream) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    if (!prm) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: NULL params");
    const int d = prm->d;
    if (d < 2 || d > 256) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: d must be in [2,256]");
    if (!(prm->gamma > 0) || !std::isfinite(prm->gamma)) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: gamma must be > 0");
    if (prm->max_iter < 1) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: max_iter must be >= 1");
    if (!(prm->tol >= 0)) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: tol must be >= 0");
    if (prm->precision != PD_FP32 && prm->precision != PD_FP32_DENSE && prm->precision != PD_BF16 &&
        prm->precision != PD_FP32_PLAIN)
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: unknown precision %d", prm->precision);
    if (prm->precision == PD_BF16 && d > 128)
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: PD_BF16 supports d <= 128");
    if (!(prm->p >= 1.0 && prm->p <= 8.0)) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: p must be in [1, 8]");
    if (prm->p != 2.0 && prm->precision != PD_FP32)
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: p != 2 needs the PD_FP32 engine");
    if (prm->eps_stages > 0 && prm->precision != PD_FP32)
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: eps_stages needs the PD_FP32 engine");
    if (prm->cta_threads != 0 && prm->cta_threads != 128 && prm->cta_threads != 256 && prm->cta_threads != 512 &&
        prm->cta_threads != 1024)
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: cta_threads must be 0, 128, 256, 512 or 1024");
    if (prm->kernel_tier < 0 || prm->kernel_tier > 2 || prm->max_inner < 0 || prm->lse_form < 0 || prm->lse_form > 2)
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: kernel_tier and lse_form must be 0..2, max_inner >= 0");
    if (P < 0) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: P < 0");
    if (P == 0) return PD_OK;
    if (!cost || !histA || !histB || !massA || !massB) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: NULL input/cost");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int dp = ((d + 63) / 64) * 64;
    SkWS w;
    int* counter;
    size_t need = pd_carve_ws(nullptr, P, d, dp, prm->gamma, nullptr, &counter);
    {
        pd_status st0 = ensure_buffer(c, &c->ws, &c->ws_bytes, need, s);
        if (st0 != PD_OK) return st0;
    }
    pd_carve_ws((char*)c->ws, P, d, dp, prm->gamma, &w, &counter);
    w.histA = histA; w.histB = histB; w.massA = massA; w.massB = massB; w.pairs = pairs;
    w.p = prm->p;
    CUDA_TRY(c, pd_upload_cost_tables(w, prm->gamma, s));
    SkRun r = make_run(prm);
    if (prm->precision == PD_FP32) {
        pd_status st = lse_solve(c, w, r, g_init, cost, row_marg, col_marg, f, g, iters, err, status, counter, s);
        if (st != PD_OK) return st;
        CUDA_TRY(c, cudaStreamSynchronize(s));
        return PD_OK;
    }
    { ProfScope ps(c, PD_K_SETUP, s); CUDA_TRY(c, sk_launch_setup(w, g_init, s)); }
    if (prm->precision == PD_BF16) {
        // tensor-core phase to err <= max(tol, 1e-4) when refining, then exact FP32 refinement
        const bool refine = prm->refine_iters > 0;
        const bool x2 = sk_bf16x2_applies(w);
        SkRun rb = r;
        // the split-operand kernel (d <= 64) reaches the tolerance itself (a pair
        // whose error stalls leaves for the refinement); the single-rounding
        // kernel stops at 1e-4, its floor being near it
        if (refine) rb.tol = x2 ? prm->tol : std::max(prm->tol, 1e-4);
        // the split operands keep precision between absorptions (a pair whose
        // scalings leave the range is absorbed at once), so the two-pair kernel
        // re-absorbs every 512 iterations at most: fewer host rounds
        if (x2) rb.absorb_every = std::max(rb.absorb_every, 512);
        { ProfScope ps(c, PD_K_LOGSTEP, s); CUDA_TRY(c, sk_launch_logstep(w, rb, s)); }
        CUDA_TRY(c, cudaMemsetAsync(c->dflag, 0, sizeof(int), s));
        int nsm = 152;
        {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        }
        if (x2 && P > 2) {
            // two pairs per CTA: pair the batch largest support first, so that
            // the two pairs of a CTA run for similar numbers of iterations
            std::vector<int> ic((size_t)P * IC_N);
            CUDA_TRY(c, cudaMemcpyAsync(ic.data(), w.ic, ic.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(c, cudaStreamSynchronize(s));
            std::vector<int> ord(P);
            for (int p = 0; p < P; ++p) ord[p] = p;
            auto sz = [&](int p) { return ic[(size_t)p * IC_N + IC_NA] + ic[(size_t)p * IC_N + IC_NB]; };
            std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sz(a) > sz(b); });
            CUDA_TRY(c, cudaMemcpyAsync(w.order_buf, ord.data(), sizeof(int) * P, cudaMemcpyHostToDevice, s));
            CUDA_TRY(c, cudaStreamSynchronize(s));
            w.order = w.order_buf;
        }
        const int max_rounds_b = prm->max_iter + 8;
        for (int round = 0; round < max_rounds_b; ++round) {
            { ProfScope ps(c, PD_K_ABSORB, s); CUDA_TRY(c, sk_launch_absorb(w, rb, s)); }
            CUDA_TRY(c, cudaMemsetAsync(counter, 0, sizeof(int), s));
            { ProfScope ps(c, PD_K_TC, s);
              CUDA_TRY(c, x2 ? sk_launch_iter_bf16x2(w, rb, rb.absorb_every, counter, c->dflag, s)
                             : sk_launch_iter_bf16(w, rb, rb.absorb_every, counter, c->dflag, s)); }
            CUDA_TRY(c, cudaMemcpyAsync(c->hflag, counter, sizeof(int), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(c, cudaStreamSynchronize(s));
            if (c->hflag[0] == 0) break;
            // the two-pair kernel's tail: once at most two pairs per SM still
            // iterate, the exact engine (one pair per wide CTA, faster per
            // iteration for a lone pair) finishes them from their current state
            if (x2 && refine && c->hflag[0] <= 2 * nsm) break;
        }
        CUDA_TRY(c, cudaMemcpyAsync(c->hflag + 1, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if (c->hflag[1]) return fail(c, PD_ERR_TIMEOUT, "pd_sinkhorn_batch: a tensor-core wait timed out");
        w.order = nullptr;
        // every pair (including ones that hit the range limit) continues in the exact engine
        { ProfScope ps(c, PD_K_ABSORB, s); CUDA_TRY(c, sk_launch_refine_prep(w, s)); }
        SkRun rr = r;
        rr.tol = prm->tol;
        if (refine) rr.max_iter = prm->max_iter;   // total count: BF16 phase + refinement, capped at max_iter
        pd_status st = lse_iterate(c, w, rr, cost, row_marg, col_marg, f, g, iters, err, status, counter, s);
        if (st != PD_OK) return st;
        CUDA_TRY(c, cudaStreamSynchronize(s));
        return PD_OK;
    }
    if (prm->precision == PD_FP32_PLAIN) {
        // the plain form: every launch of the solve carries one pair (the
        // support set-up above is one launch for the batch), pairs one after
        // the other on the stream, the host reading each pair's state between
        // its iteration launches
        const size_t n = (size_t)d * d + 1;   // caller's per-pair output length
        for (int p = 0; p < P; ++p) {
            SkWS v = ws_view(w, p);
            { ProfScope ps(c, PD_K_LOGSTEP, s); CUDA_TRY(c, sk_launch_logstep(v, r, s)); }
            for (int round = 0; round < prm->max_iter + 8; ++round) {
                { ProfScope ps(c, PD_K_ABSORB, s); CUDA_TRY(c, sk_launch_absorb(v, r, s)); }
                CUDA_TRY(c, cudaMemsetAsync(counter, 0, sizeof(int), s));
                { ProfScope ps(c, PD_K_ITER, s); CUDA_TRY(c, sk_launch_iter_fp32(v, r, r.absorb_every, counter, s)); }
                CUDA_TRY(c, cudaMemcpyAsync(c->hflag, counter, sizeof(int), cudaMemcpyDeviceToHost, s));
                CUDA_TRY(c, cudaStreamSynchronize(s));
                if (c->hflag[0] == 0) break;
            }
            { ProfScope ps(c, PD_K_ABSORB, s); CUDA_TRY(c, sk_launch_absorb(v, r, s)); }
            { ProfScope ps(c, PD_K_FINALIZE, s);
              CUDA_TRY(c, sk_launch_finalize(v, cost + p, row_marg ? row_marg + p * n : nullptr,
                                             col_marg ? col_marg + p * n : nullptr, f ? f + p * n : nullptr,
                                             g ? g + p * n : nullptr, iters ? iters + p : nullptr,
                                             err ? err + p : nullptr, status ? status + p : nullptr, s)); }
        }
        pd_status stc = linear_range_check(c, w, prm->tol, status, err, s);
        if (stc != PD_OK) return stc;
        CUDA_TRY(c, cudaStreamSynchronize(s));
        return PD_OK;
    }
    { ProfScope ps(c, PD_K_LOGSTEP, s); CUDA_TRY(c, sk_launch_logstep(w, r, s)); }
    const int max_rounds = prm->max_iter + 8;
    for (int round = 0; round < max_rounds; ++round) {
        { ProfScope ps(c, PD_K_ABSORB, s); CUDA_TRY(c, sk_launch_absorb(w, r, s)); }
        CUDA_TRY(c, cudaMemsetAsync(counter, 0, sizeof(int), s));
        { ProfScope ps(c, PD_K_ITER, s); CUDA_TRY(c, sk_launch_iter_fp32(w, r, r.absorb_every, counter, s)); }
        CUDA_TRY(c, cudaMemcpyAsync(c->hflag, counter, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if (c->hflag[0] == 0) break;
    }
    { ProfScope ps(c, PD_K_ABSORB, s); CUDA_TRY(c, sk_launch_absorb(w, r, s)); }   // pairs that finished inside the log step
    { ProfScope ps(c, PD_K_FINALIZE, s); CUDA_TRY(c, sk_launch_finalize(w, cost, row_marg, col_marg, f, g, iters, err, status, s)); }
    pd_status stc = linear_range_check(c, w, prm->tol, status, err, s);
    if (stc != PD_OK) return stc;
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return PD_OK;
}


// ---------------------------------------------------------------------------
// Several grid sizes in one batch: one workspace per group, every pair of
// every group in one persistent launch of the iteration kernel.

extern "C" pd_status pd_sinkhorn_batch_groups(pd_ctx* c, int ngroups, const pd_sinkhorn_group* grp,
                                              const pd_sinkhorn_params* prm, pd_stream stream) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    if (!prm || !grp || ngroups < 1 || ngroups > 127)
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch_groups: need params, groups and 1 <= ngroups <= 127");
    if (!(prm->gamma > 0) || !std::isfinite(prm->gamma) || prm->max_iter < 1 || !(prm->tol >= 0) ||
        prm->precision != PD_FP32 || !(prm->p >= 1.0 && prm->p <= 8.0) || prm->eps_stages != 0 ||
        (prm->cta_threads != 0 && prm->cta_threads != 128 && prm->cta_threads != 256 && prm->cta_threads != 512 &&
         prm->cta_threads != 1024) || prm->kernel_tier < 0 || prm->kernel_tier > 2 || prm->max_inner < 0 ||
        prm->lse_form < 0 || prm->lse_form > 2)
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch_groups: bad params (PD_FP32 only, no eps_stages)");
    for (int gi = 0; gi < ngroups; ++gi) {
        const pd_sinkhorn_group& G = grp[gi];
        if (G.d < 2 || G.d > 256 || G.P < 0 || G.P >= (1 << 24))
            return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch_groups: group %d: need 2 <= d <= 256, 0 <= P < 2^24", gi);
        if (G.P > 0 && (!G.cost || !G.histA || !G.histB || !G.massA || !G.massB))
            return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch_groups: group %d: NULL input/cost", gi);
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(c, cudaSetDevice(c->device));
    // layout: the groups' workspaces, then the descriptor array and the order
    std::vector<size_t> off(ngroups);
    size_t need = 0;
    int Ptot = 0;
    int* dummy = nullptr;
    for (int gi = 0; gi < ngroups; ++gi) {
        const int d = grp[gi].d, dp = ((d + 63) / 64) * 64;
        off[gi] = need;
        need += align256(pd_carve_ws(nullptr, std::max(grp[gi].P, 1), d, dp, prm->gamma, nullptr, &dummy));
        Ptot += grp[gi].P;
    }
    const size_t off_desc = need;
    need += align256(sizeof(SkWS) * ngroups);
    const size_t off_order = need;
    need += align256(sizeof(int) * (size_t)std::max(Ptot, 1));
    if (Ptot == 0) return PD_OK;
    pd_status st = ensure_buffer(c, &c->ws, &c->ws_bytes, need, s);
    if (st != PD_OK) return st;
    char* base = (char*)c->ws;
    std::vector<SkWS> gs;
    int* counter = nullptr;
    int* counter0 = nullptr;
    for (int gi = 0; gi < ngroups; ++gi) {
        const pd_sinkhorn_group& G = grp[gi];
        const int d = G.d, dp = ((d + 63) / 64) * 64;
        SkWS w;
        pd_carve_ws(base + off[gi], std::max(G.P, 1), d, dp, prm->gamma, &w, &counter);
        if (!counter0) counter0 = counter;
        w.P = G.P;
        w.histA = G.histA; w.histB = G.histB; w.massA = G.massA; w.massB = G.massB; w.pairs = G.pairs;
        w.p = prm->p;
        CUDA_TRY(c, pd_upload_cost_tables(w, prm->gamma, s));
        { ProfScope ps(c, PD_K_SETUP, s); CUDA_TRY(c, sk_launch_setup(w, G.g_init, s)); }
        gs.push_back(w);
    }
    SkRun r = make_run(prm);
    CUDA_TRY(c, lse_rounds_groups(c, gs, (SkWS*)(base + off_desc), (int*)(base + off_order), r, counter0, c->hflag, s));
    for (int gi = 0; gi < ngroups; ++gi) {
        const pd_sinkhorn_group& G = grp[gi];
        if (G.P == 0) continue;
        ProfScope ps(c, PD_K_FINALIZE, s);
        CUDA_TRY(c, sk_launch_lse_finalize(gs[gi], G.cost, G.row_marg, G.col_marg, G.f, G.g, G.iters, G.err, G.status,
                                           r.pot_support_only, s));
    }
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return PD_OK;
}

// ---------------------------------------------------------------------------
// Outer loops: barycenter (Alg. 2) and k-means (Sec. 5).

static pd_status check_params(pd_ctx* c, const pd_sinkhorn_params* prm, const char* who) {
    if (!prm) return fail(c, PD_ERR_INVALID, "%s: NULL params", who);
    if (prm->d < 2 || prm->d > 256) return fail(c, PD_ERR_INVALID, "%s: d must be in [2,256]", who);
    if (!(prm->gamma > 0) || !std::isfinite(prm->gamma)) return fail(c, PD_ERR_INVALID, "%s: gamma must be > 0", who);
    if (prm->max_iter < 1) return fail(c, PD_ERR_INVALID, "%s: max_iter must be >= 1", who);
    if (!(prm->tol >= 0)) return fail(c, PD_ERR_INVALID, "%s: tol must be >= 0", who);
    if (prm->precision != PD_FP32) return fail(c, PD_ERR_INVALID, "%s: only PD_FP32 is supported", who);
    if (prm->p != 2.0) return fail(c, PD_ERR_INVALID, "%s: only p = 2 is supported", who);
    return PD_OK;
}

// Carve a Sinkhorn workspace for P pairs in c->ws.
static pd_status sinkhorn_ws(pd_ctx* c, int P, const pd_sinkhorn_params* prm, SkWS* w, int** counter,
                             cudaStream_t s) {
    const int d = prm->d, dp = ((d + 63) / 64) * 64;
    size_t need = pd_carve_ws(nullptr, P, d, dp, prm->gamma, nullptr, counter);
    pd_status st = ensure_buffer(c, &c->ws, &c->ws_bytes, need, s);
    if (st != PD_OK) return st;
    pd_carve_ws((char*)c->ws, P, d, dp, prm->gamma, w, counter);
    CUDA_TRY(c, pd_upload_cost_tables(*w, prm->gamma, s));
    return PD_OK;
}

// Sec. 3 "Upper and Lower Bounds": the PD_FP32 solve of pd_sinkhorn_batch, then
// the C-transform lower bound m_t and the rounded plan's cost M_t (Prop. 3).
extern "C" pd_status pd_sinkhorn_bounds(pd_ctx* c, const uint32_t* histA, const uint32_t* massA,
                                        const uint32_t* histB, const uint32_t* massB, const int32_t* pairs, int P,
                                        const pd_sinkhorn_params* prm, const double* g_init, double* cost,
                                        double* lower, double* upper, int32_t* iters, float* err, int32_t* status,
                                        pd_stream stream) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    if (!prm) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_bounds: NULL params");
    const int d = prm->d;
    if (d < 2 || d > 256) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_bounds: d must be in [2,256]");
    if (!(prm->gamma > 0) || !std::isfinite(prm->gamma))
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_bounds: gamma must be > 0");
    if (prm->max_iter < 1) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_bounds: max_iter must be >= 1");
    if (!(prm->tol >= 0)) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_bounds: tol must be >= 0");
    if (prm->precision != PD_FP32) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_bounds: only PD_FP32 is supported");
    if (prm->p != 2.0) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_bounds: only p = 2 is supported");
    if (P < 0) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_bounds: P < 0");
    if (P == 0) return PD_OK;
    if (!cost || !histA || !histB || !massA || !massB)
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_bounds: NULL input/cost");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(c, cudaSetDevice(c->device));
    SkWS w;
    int* counter;
    pd_status st = sinkhorn_ws(c, P, prm, &w, &counter, s);
    if (st != PD_OK) return st;
    w.histA = histA; w.histB = histB; w.massA = massA; w.massB = massB; w.pairs = pairs;
    SkRun r = make_run(prm);
    st = lse_solve(c, w, r, g_init, cost, nullptr, nullptr, nullptr, nullptr, iters, err, status, counter, s);
    if (st != PD_OK) return st;
    // the lower bound reads the final potentials; the upper bound then rescales them in place
    if (lower) { ProfScope ps(c, PD_K_FINALIZE, s); CUDA_TRY(c, sk_launch_ctransform(w, lower, s)); }
    if (upper) {
        { ProfScope ps(c, PD_K_FINALIZE, s); CUDA_TRY(c, sk_launch_round_bound(w, s)); }
        { ProfScope ps(c, PD_K_FINALIZE, s);
          CUDA_TRY(c, sk_launch_lse_finalize(w, upper, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, s)); }
        CUDA_TRY(c, sk_launch_add_corr(w, upper, s));
    }
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return PD_OK;
}

// Sub-allocator over c->ws2.
struct Arena {
    char* base; size_t off;
    template <class T> T* take(size_t n) { T* r = (T*)(base ? base + off : nullptr); off += (n * sizeof(T) + 255) & ~size_t(255); return r; }
};

// Outer-loop buffers of pd_barycenter in ws2 (base == nullptr: sizes only).
struct BaryBufs {
    double *z, *zmass, *f, *g, *cost, *ebuf;
    int32_t *pairs, *iters, *status;
    float* err;
    unsigned long long* H0bits;
};
static size_t bary_layout(char* base, int N, int d, BaryBufs* o) {
    const int D = d * d, n1 = D + 1;
    Arena a{base, 0};
    BaryBufs t;
    t.z = a.take<double>(D); t.zmass = a.take<double>(1); t.f = a.take<double>((size_t)N * n1);
    t.g = a.take<double>((size_t)N * n1); t.cost = a.take<double>(N); t.pairs = a.take<int32_t>(2 * (size_t)N);
    t.iters = a.take<int32_t>(N); t.err = a.take<float>(N); t.status = a.take<int32_t>(N);
    t.H0bits = a.take<unsigned long long>(1); t.ebuf = a.take<double>(1);
    if (o) *o = t;
    return a.off;
}

extern "C" pd_status pd_barycenter(pd_ctx* c, const uint32_t* hist, const uint32_t* mass, int N,
                                   const pd_sinkhorn_params* prm, double lambda, int outer_iters,
                                   double rel_energy_tol, const double* z_init, double* z_out, double* energy,
                                   int* steps_host, pd_stream stream) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    if (steps_host) *steps_host = 0;
    pd_status st = check_params(c, prm, "pd_barycenter");
    if (st != PD_OK) return st;
    if (N < 1 || !hist || !mass || !z_out) return fail(c, PD_ERR_INVALID, "pd_barycenter: need N >= 1, hist, mass, z_out");
    if (!(lambda > 0) || outer_iters < 0) return fail(c, PD_ERR_INVALID, "pd_barycenter: need lambda > 0, outer_iters >= 0");
    if (!(rel_energy_tol >= 0) || !std::isfinite(rel_energy_tol))
        return fail(c, PD_ERR_INVALID, "pd_barycenter: rel_energy_tol must be finite and >= 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int d = prm->d, D = d * d;
    st = ensure_buffer(c, &c->ws2, &c->ws2_bytes, bary_layout(nullptr, N, d, nullptr), s);
    if (st != PD_OK) return st;
    BaryBufs B;
    bary_layout((char*)c->ws2, N, d, &B);
    double* z = B.z;
    SkWS w;
    int* counter;
    st = sinkhorn_ws(c, N, prm, &w, &counter, s);
    if (st != PD_OK) return st;
    if (prm->bary_sharpen) CUDA_TRY(c, outer_input_entropy(hist, N, d, B.H0bits, s));
    if (z_init) CUDA_TRY(c, cudaMemcpyAsync(z, z_init, sizeof(double) * D, cudaMemcpyDeviceToDevice, s));
    else CUDA_TRY(c, outer_bary_init_uniform(z, mass, N, d, s));
    CUDA_TRY(c, outer_owner_pairs(nullptr, N, B.pairs, s));
    SkRun r = make_run(prm);
    r.pot_support_only = 1;
    r.batch_form = 1;
    const bool stop_rule = rel_energy_tol > 0;
    double e_prev = 0.0;
    int steps = 0;
    for (int t = 0; t < outer_iters; ++t) {
        CUDA_TRY(c, outer_measure_mass(z, 1, d, B.zmass, s));
        w.histA = nullptr; w.massA = nullptr; w.wA = z;            // a side: z + R a_i
        w.histB = hist; w.massB = mass; w.wB = nullptr;            // b side: a_i + R z
        w.pairs = B.pairs;
        st = lse_solve(c, w, r, t > 0 ? B.g : nullptr, B.cost, nullptr, nullptr, B.f, B.g, B.iters, B.err, B.status,
                       counter, s);
        if (st != PD_OK) return st;
        double* et = energy ? energy + t : B.ebuf;
        if (energy || stop_rule) CUDA_TRY(c, outer_mean(B.cost, N, et, s));
        CUDA_TRY(c, outer_bary_step(z, B.zmass, B.f, B.g, nullptr, N, 1, d, prm->gamma, lambda, s));
        if (prm->bary_sharpen) CUDA_TRY(c, outer_sharpen(z, 1, d, B.H0bits, s));
        steps = t + 1;
        if (stop_rule) {
            // the barycenter experiment's stop (Sec. 5): |E_t / E_{t-1} - 1| < rel_energy_tol
            CUDA_TRY(c, cudaMemcpyAsync(c->hval, et, sizeof(double), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(c, cudaStreamSynchronize(s));
            const double e_t = c->hval[0];
            if (t >= 1 && std::fabs(e_t / e_prev - 1.0) < rel_energy_tol) break;
            e_prev = e_t;
        }
    }
    CUDA_TRY(c, cudaMemcpyAsync(z_out, z, sizeof(double) * D, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    if (steps_host) *steps_host = steps;
    return PD_OK;
}

// Buffers of pd_barycenter_grad in ws2 (own_g: g is not the caller's g_warm).
static size_t grad_layout(char* base, int N, int d, bool own_g, double** f, double** g, double** cost,
                          int32_t** pairs, int32_t** iters, float** err, int32_t** status) {
    const size_t n1 = (size_t)d * d + 1;
    Arena ar{base, 0};
    *f = ar.take<double>((size_t)N * n1); *g = ar.take<double>(own_g ? (size_t)N * n1 : 0);
    *cost = ar.take<double>(N); *pairs = ar.take<int32_t>(2 * (size_t)N); *iters = ar.take<int32_t>(N);
    *err = ar.take<float>(N); *status = ar.take<int32_t>(N);
    return ar.off;
}

// Buffers of pd_kmeans_assign in ws2 (own_cost: the caller passed no cost array).
static size_t assign_layout(char* base, size_t NK, bool own_cost, double** cst, int32_t** pairs, int32_t** iters,
                            float** err, int32_t** status) {
    Arena ar{base, 0};
    *cst = ar.take<double>(own_cost ? NK : 0); *pairs = ar.take<int32_t>(2 * NK); *iters = ar.take<int32_t>(NK);
    *err = ar.take<float>(NK); *status = ar.take<int32_t>(NK);
    return ar.off;
}

// Buffers of pd_kmeans in ws2.
static size_t kmeans_layout(char* base, int N, int k, int d, double** zmass, double** f, double** g, double** cost,
                            int32_t** pairs, int32_t** iters, float** err, int32_t** status, int32_t** idx) {
    const size_t n1 = (size_t)d * d + 1, NK = (size_t)N * k;
    Arena ar{base, 0};
    *zmass = ar.take<double>(k); *f = ar.take<double>((size_t)N * n1); *g = ar.take<double>((size_t)N * n1);
    *cost = ar.take<double>(NK); *pairs = ar.take<int32_t>(2 * NK); *iters = ar.take<int32_t>(NK);
    *err = ar.take<float>(NK); *status = ar.take<int32_t>(NK); *idx = ar.take<int32_t>(k);
    return ar.off;
}

// Sharded Alg. 2 step, first half: solve this shard's pairs
// (z_owner[n] + R a_n, a_n + R z_owner[n]) and sum their gradient terms per
// measure (the caller adds the sums of all shards, then calls
// pd_barycenter_apply).
extern "C" pd_status pd_barycenter_grad(pd_ctx* c, const uint32_t* hist, const uint32_t* mass, int N, int k,
                                        const pd_sinkhorn_params* prm, const double* z, const int32_t* owner,
                                        double* g_warm, int warm, double* gsum, double* count, double* cost_sum,
                                        pd_stream stream) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    pd_status st = check_params(c, prm, "pd_barycenter_grad");
    if (st == PD_OK && prm->bary_sharpen)
        return fail(c, PD_ERR_INVALID, "pd_barycenter_grad: bary_sharpen is not supported (sharpening is not part of the sharded step)");
    if (st != PD_OK) return st;
    if (N < 1 || k < 1 || !hist || !mass || !z || !gsum || !count || !cost_sum || (warm && !g_warm))
        return fail(c, PD_ERR_INVALID, "pd_barycenter_grad: need N >= 1, k >= 1, non-NULL hist, mass, z, gsum, count, "
                                       "cost_sum, and g_warm when warm");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(c, cudaSetDevice(c->device));
    if (owner) {
        // an owner outside [0, k) would index past z: refuse it before any solve
        CUDA_TRY(c, cudaMemsetAsync(c->dflag, 0, sizeof(int), s));
        CUDA_TRY(c, outer_check_owner(owner, N, k, c->dflag, s));
        CUDA_TRY(c, cudaMemcpyAsync(c->hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if (c->hflag[0]) return fail(c, PD_ERR_INVALID, "pd_barycenter_grad: owner values must lie in [0, k)");
    }
    const int d = prm->d;
    double *f, *g, *cost; int32_t *pairs, *iters, *status; float* err;
    st = ensure_buffer(c, &c->ws2, &c->ws2_bytes,
                       grad_layout(nullptr, N, d, g_warm == nullptr, &f, &g, &cost, &pairs, &iters, &err, &status), s);
    if (st != PD_OK) return st;
    grad_layout((char*)c->ws2, N, d, g_warm == nullptr, &f, &g, &cost, &pairs, &iters, &err, &status);
    if (g_warm) g = g_warm;
    SkWS w;
    int* counter;
    st = sinkhorn_ws(c, N, prm, &w, &counter, s);
    if (st != PD_OK) return st;
    CUDA_TRY(c, outer_owner_pairs(owner, N, pairs, s));
    w.histA = nullptr; w.massA = nullptr; w.wA = z;            // a side: z_c + R a_n
    w.histB = hist; w.massB = mass; w.wB = nullptr;            // b side: a_n + R z_c
    w.pairs = pairs;
    SkRun r = make_run(prm);
    r.pot_support_only = 1;
    r.batch_form = 1;
    st = lse_solve(c, w, r, warm ? g : nullptr, cost, nullptr, nullptr, f, g, iters, err, status, counter, s);
    if (st != PD_OK) return st;
    CUDA_TRY(c, outer_bary_grad(z, f, g, owner, N, k, d, gsum, count, s));
    CUDA_TRY(c, outer_cost_sum(cost, owner, N, k, cost_sum, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return PD_OK;
}

// k-means assignment (Sec. 5) of N diagrams to k real-valued centroids:
// cold-started solves of (a_n + R z_c, z_c + R a_n) for every n, c, then
// argmin_c (ties to the lowest c) and sum_n min_c cost.
extern "C" pd_status pd_kmeans_assign(pd_ctx* c, const uint32_t* hist, const uint32_t* mass, int N, int k,
                                      const pd_sinkhorn_params* prm, const double* centroids, int32_t* assign,
                                      double* cost, double* objective, pd_stream stream) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    pd_status st = check_params(c, prm, "pd_kmeans_assign");
    if (st != PD_OK) return st;
    if (N < 1 || k < 1 || !hist || !mass || !centroids || !assign)
        return fail(c, PD_ERR_INVALID, "pd_kmeans_assign: need N >= 1, k >= 1, non-NULL hist, mass, centroids, assign");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(c, cudaSetDevice(c->device));
    const size_t NK = (size_t)N * k;
    if (NK > (size_t)INT32_MAX) return fail(c, PD_ERR_INVALID, "pd_kmeans_assign: N * k too large");
    double* cst; int32_t *pairs, *iters, *status; float* err;
    st = ensure_buffer(c, &c->ws2, &c->ws2_bytes, assign_layout(nullptr, NK, cost == nullptr, &cst, &pairs, &iters, &err,
                                                                &status), s);
    if (st != PD_OK) return st;
    assign_layout((char*)c->ws2, NK, cost == nullptr, &cst, &pairs, &iters, &err, &status);
    if (cost) cst = cost;
    SkWS w;
    int* counter;
    st = sinkhorn_ws(c, (int)NK, prm, &w, &counter, s);
    if (st != PD_OK) return st;
    CUDA_TRY(c, outer_km_pairs(N, k, pairs, s));
    w.histA = hist; w.massA = mass; w.wA = nullptr;
    w.histB = nullptr; w.massB = nullptr; w.wB = centroids;
    w.pairs = pairs;
    SkRun r = make_run(prm);
    r.batch_form = 1;
    r.pot_support_only = 0;
    st = lse_solve(c, w, r, nullptr, cst, nullptr, nullptr, nullptr, nullptr, iters, err, status, counter, s);
    if (st != PD_OK) return st;
    CUDA_TRY(c, outer_km_assign(cst, N, k, assign, objective, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return PD_OK;
}

// Sharded Alg. 2 step, second half: z_c <- z_c exp(-lambda grad_c) from the
// summed per-shard values.
extern "C" pd_status pd_barycenter_apply(pd_ctx* c, double* z, int k, int d, const double* gsum, const double* count,
                                         double gamma, double lambda, pd_stream stream) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    if (!z || !gsum || !count || k < 1 || d < 2 || d > 256 || !(gamma > 0) || !(lambda > 0))
        return fail(c, PD_ERR_INVALID, "pd_barycenter_apply: need z, gsum, count, k >= 1, 2 <= d <= 256, "
                                       "gamma > 0, lambda > 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, outer_bary_apply(z, gsum, count, k, d, gamma, lambda, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return PD_OK;
}

// splitmix64 (Steele, Lea & Flood, OOPSLA 2014).
static uint64_t splitmix64_next(uint64_t* st) {
    uint64_t z = (*st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" pd_status pd_kmeans(pd_ctx* c, const uint32_t* hist, const uint32_t* mass, int N, int k,
                               const pd_sinkhorn_params* prm, double lambda, int rounds, int bary_steps,
                               uint64_t seed, int32_t* assign, double* centroids, double* objective,
                               pd_stream stream) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    pd_status st = check_params(c, prm, "pd_kmeans");
    if (st == PD_OK && prm->bary_sharpen) return fail(c, PD_ERR_INVALID, "pd_kmeans: bary_sharpen is not supported");
    if (st != PD_OK) return st;
    if (N < 1 || k < 1 || k > N || !hist || !mass || !assign || !centroids)
        return fail(c, PD_ERR_INVALID, "pd_kmeans: need 1 <= k <= N and non-NULL hist, mass, assign, centroids");
    if (!(lambda > 0) || rounds < 0 || bary_steps < 0)
        return fail(c, PD_ERR_INVALID, "pd_kmeans: need lambda > 0, rounds >= 0, bary_steps >= 0");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int d = prm->d;
    const size_t NK = (size_t)N * k;
    double *zmass, *f, *g, *cost; int32_t *pairs, *iters, *status, *idx; float* err;
    st = ensure_buffer(c, &c->ws2, &c->ws2_bytes,
                       kmeans_layout(nullptr, N, k, d, &zmass, &f, &g, &cost, &pairs, &iters, &err, &status, &idx), s);
    if (st != PD_OK) return st;
    kmeans_layout((char*)c->ws2, N, k, d, &zmass, &f, &g, &cost, &pairs, &iters, &err, &status, &idx);
    // seeding: k distinct histograms drawn by splitmix64(seed), draw r mod N, repeats skipped
    std::vector<int32_t> chosen;
    uint64_t stt = seed;
    while ((int)chosen.size() < k) {
        int r0 = (int)(splitmix64_next(&stt) % (uint64_t)N);
        if (std::find(chosen.begin(), chosen.end(), r0) == chosen.end()) chosen.push_back(r0);
    }
    CUDA_TRY(c, cudaMemcpyAsync(idx, chosen.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, outer_km_seed(hist, idx, k, d, centroids, s));
    SkWS w;
    int* counter;
    st = sinkhorn_ws(c, (int)std::max(NK, (size_t)N), prm, &w, &counter, s);
    if (st != PD_OK) return st;
    SkRun r = make_run(prm);
    r.batch_form = 1;
    for (int rd = 0; rd < rounds; ++rd) {
        // assignment: pairs (a_n + R z_c, z_c + R a_n) for every n, c
        CUDA_TRY(c, outer_km_pairs(N, k, pairs, s));
        SkWS wa = w;
        wa.P = (int)NK;
        wa.histA = hist; wa.massA = mass; wa.wA = nullptr;
        wa.histB = nullptr; wa.massB = nullptr; wa.wB = centroids;
        wa.pairs = pairs;
        r.pot_support_only = 0;
        st = lse_solve(c, wa, r, nullptr, cost, nullptr, nullptr, nullptr, nullptr, iters, err, status, counter, s);
        if (st != PD_OK) return st;
        CUDA_TRY(c, outer_km_assign(cost, N, k, assign, objective ? objective + rd : nullptr, s));
        // centroid update: bary_steps steps of Alg. 2 per cluster, all clusters batched
        CUDA_TRY(c, outer_owner_pairs(assign, N, pairs, s));
        SkWS wb = w;
        wb.P = N;
        wb.histA = nullptr; wb.massA = nullptr; wb.wA = centroids;
        wb.histB = hist; wb.massB = mass; wb.wB = nullptr;
        wb.pairs = pairs;
        r.pot_support_only = 1;
        for (int st2 = 0; st2 < bary_steps; ++st2) {
            CUDA_TRY(c, outer_measure_mass(centroids, k, d, zmass, s));
            st = lse_solve(c, wb, r, st2 > 0 ? g : nullptr, cost, nullptr, nullptr, f, g, iters, err, status, counter, s);
            if (st != PD_OK) return st;
            CUDA_TRY(c, outer_bary_step(centroids, zmass, f, g, assign, N, k, d, prm->gamma, lambda, s));
        }
    }
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return PD_OK;
}

// ---------------------------------------------------------------------------
// Autotuner of the base-2 iteration kernel's CTA width.

extern "C" pd_status pd_sinkhorn_tune(pd_ctx* c, const uint32_t* histA, const uint32_t* massA,
                                      const uint32_t* histB, const uint32_t* massB, const int32_t* pairs, int P,
                                      const pd_sinkhorn_params* prm, int trial_iters, int* threads_host,
                                      double* trial_ms_host, pd_stream stream) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    if (!prm || prm->precision != PD_FP32 || prm->d < 2 || prm->d > 256 || !(prm->gamma > 0) ||
        !std::isfinite(prm->gamma) || !(prm->p >= 1.0 && prm->p <= 8.0) || P < 1 || trial_iters < 1 ||
        !histA || !histB || !massA || !massB)
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_tune: need PD_FP32 params, P >= 1, trial_iters >= 1, inputs");
    if (sk_lse2_grid_bits(prm->gamma) < 0)
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_tune: gamma below the base-2 kernel's range (nothing to tune)");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(c, cudaSetDevice(c->device));
    SkWS w;
    int* counter;
    pd_status st = sinkhorn_ws(c, P, prm, &w, &counter, s);
    if (st != PD_OK) return st;
    w.histA = histA; w.histB = histB; w.massA = massA; w.massB = massB; w.pairs = pairs;
    w.p = prm->p;
    CUDA_TRY(c, pd_upload_cost_tables(w, prm->gamma, s));
    SkRun r = make_run(prm);
    r.max_iter = trial_iters;
    r.max_inner = trial_iters;
    const int cands[4] = {128, 256, 512, 1024};
    double ms[4] = {NAN, NAN, NAN, NAN};
    const bool prof_was = c->prof;
    int best = 256;
    double best_ms = INFINITY;
    double mean_cells = 0.0;
    for (int k = 0; k < 3; ++k) {   // 1024 serves only the drain
        if (cands[k] == 128 && prm->d > 128) continue;
        // identical trials: the same cold start, each pair to tol or trial_iters, one launch of one width
        CUDA_TRY(c, sk_launch_setup(w, nullptr, s));
        r.cta_threads = cands[k];
        for (auto& rc : c->recs) { c->ev_pool.push_back(rc.a); c->ev_pool.push_back(rc.b); }
        c->recs.clear();
        c->prof = true;
        cudaError_t e = lse_rounds(c, w, r, counter, c->hflag, s);
        c->prof = prof_was;
        CUDA_TRY(c, e);
        double t = 0.0;
        for (auto& rc : c->recs) {
            if (rc.kind != PD_K_ITER) continue;
            float x = 0.f;
            CUDA_TRY(c, cudaEventSynchronize(rc.b));
            CUDA_TRY(c, cudaEventElapsedTime(&x, rc.a, rc.b));
            t += x;
        }
        for (auto& rc : c->recs) { c->ev_pool.push_back(rc.a); c->ev_pool.push_back(rc.b); }
        c->recs.clear();
        ms[k] = t;
        if (t < best_ms) { best_ms = t; best = cands[k]; }
    }
    {
        std::vector<int> ic((size_t)P * IC_N);
        CUDA_TRY(c, cudaMemcpyAsync(ic.data(), w.ic, ic.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        for (int p = 0; p < P; ++p) mean_cells += ic[(size_t)p * IC_N + IC_NA] + ic[(size_t)p * IC_N + IC_NB];
        mean_cells /= 2.0 * P;
    }
    c->tune[{prm->d, support_bucket(mean_cells)}] = best;
    if (threads_host) *threads_host = best;
    if (trial_ms_host) for (int k = 0; k < 4; ++k) trial_ms_host[k] = ms[k];
    return PD_OK;
}

extern "C" pd_status pd_tune_save(pd_ctx* c, const char* path) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    if (!path) return fail(c, PD_ERR_INVALID, "pd_tune_save: NULL path");
    FILE* fh = std::fopen(path, "w");
    if (!fh) return fail(c, PD_ERR_INVALID, "pd_tune_save: cannot write %s", path);
    std::fprintf(fh, "# pd_ot tuning table: d support_bucket cta_threads\n");
    for (auto& kv : c->tune) std::fprintf(fh, "%d %d %d\n", kv.first.first, kv.first.second, kv.second);
    std::fclose(fh);
    return PD_OK;
}

extern "C" pd_status pd_tune_load(pd_ctx* c, const char* path) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    if (!path) return fail(c, PD_ERR_INVALID, "pd_tune_load: NULL path");
    FILE* fh = std::fopen(path, "r");
    if (!fh) return fail(c, PD_ERR_INVALID, "pd_tune_load: cannot read %s", path);
    std::map<std::pair<int, int>, int> t;
    char line[256];
    int lineno = 0;
    while (std::fgets(line, sizeof(line), fh)) {
        ++lineno;
        if (line[0] == '#' || line[0] == '\n') continue;
        int d = 0, b = 0, th = 0;
        if (std::sscanf(line, "%d %d %d", &d, &b, &th) != 3 || d < 2 || d > 256 ||
            (th != 128 && th != 256 && th != 512) || (th == 128 && d > 128)) {
            std::fclose(fh);
            return fail(c, PD_ERR_INVALID, "pd_tune_load: bad entry on line %d of %s", lineno, path);
        }
        t[{d, b}] = th;
    }
    std::fclose(fh);
    c->tune = t;
    return PD_OK;
}

// ---------------------------------------------------------------------------
// Workspace sizing and caller-supplied workspace.

extern "C" pd_status pd_workspace_query(int op, const pd_sinkhorn_params* prm, int n, int k, size_t* bytes) {
    if (!bytes || !prm || n < 0 || prm->d < 2 || prm->d > 256) return PD_ERR_INVALID;
    *bytes = 0;
    const int d = prm->d, dp = ((d + 63) / 64) * 64;
    int* counter = nullptr;
    auto sk = [&](size_t P) { return P == 0 ? (size_t)0 : align256(pd_carve_ws(nullptr, (int)P, d, dp, prm->gamma,
                                                                                 nullptr, &counter)); };
    double *f, *g, *cost, *zmass; int32_t *pairs, *iters, *status, *idx; float* err;
    switch (op) {
        case PD_OP_SINKHORN:
        case PD_OP_BOUNDS:
            *bytes = sk((size_t)n);
            return PD_OK;
        case PD_OP_BARYCENTER:
            if (n < 1) return PD_ERR_INVALID;
            *bytes = sk((size_t)n) + align256(bary_layout(nullptr, n, d, nullptr));
            return PD_OK;
        case PD_OP_BARY_GRAD:
            if (n < 1) return PD_ERR_INVALID;
            *bytes = sk((size_t)n) +
                     align256(grad_layout(nullptr, n, d, true, &f, &g, &cost, &pairs, &iters, &err, &status));
            return PD_OK;
        case PD_OP_KMEANS_ASSIGN:
            if (n < 1 || k < 1 || (size_t)n * k > (size_t)INT32_MAX) return PD_ERR_INVALID;
            *bytes = sk((size_t)n * k) +
                     align256(assign_layout(nullptr, (size_t)n * k, true, &cost, &pairs, &iters, &err, &status));
            return PD_OK;
        case PD_OP_KMEANS:
            if (n < 1 || k < 1 || k > n || (size_t)n * k > (size_t)INT32_MAX) return PD_ERR_INVALID;
            *bytes = sk(std::max((size_t)n * k, (size_t)n)) +
                     align256(kmeans_layout(nullptr, n, k, d, &zmass, &f, &g, &cost, &pairs, &iters, &err, &status,
                                            &idx));
            return PD_OK;
        default:
            return PD_ERR_INVALID;
    }
}

extern "C" pd_status pd_ctx_set_workspace(pd_ctx* c, void* ws, size_t bytes) {
    if (!c) return PD_ERR_INVALID;
    call_begin(c);
    if (ws && ((uintptr_t)ws & 255u)) return fail(c, PD_ERR_INVALID, "pd_ctx_set_workspace: ws must be 256-byte aligned");
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaDeviceSynchronize());   // no call of this context may still use the old workspace
    if (!c->ext) {
        if (c->ws) cudaFree(c->ws);
        if (c->ws2) cudaFree(c->ws2);
    }
    c->ws = c->ws2 = nullptr;
    c->ws_bytes = c->ws2_bytes = 0;
    c->ext = (char*)ws;
    c->ext_bytes = ws ? bytes : 0;
    return PD_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of pd_sinkhorn_batch (PD_FP32 engine only).
//
// Its workspace is the file-scope device array below instead of memory from
// cudaMalloc: every GPU that loads this library reserves it for the lifetime
// of the process.  Host code cannot use the array's name as a device address
// (in host code it names a host-side stand-in), so the device address is
// obtained once per device with cudaGetSymbolAddress and cached; the cache
// entries are atomics, so two host threads making their first call on one
// device at the same time both store the same address without a data race.
#define PD_NOALLOC_SCRATCH_BYTES (16u << 20)
#define PD_NOALLOC_MAX_DEVICES 64
static __device__ __align__(256) unsigned char g_noalloc_scratch[PD_NOALLOC_SCRATCH_BYTES];
static std::atomic<void*> g_noalloc_addr[PD_NOALLOC_MAX_DEVICES];

extern "C" pd_status pd_sinkhorn_batch_noalloc(const uint32_t* histA, const uint32_t* massA,
                                               const uint32_t* histB, const uint32_t* massB,
                                               const int32_t* pairs, int P, const pd_sinkhorn_params* prm,
                                               const double* g_init, double* cost, float* row_marg,
                                               float* col_marg, double* f, double* g, int32_t* iters,
                                               float* err, int32_t* status, pd_stream stream) {
    if (!prm) return PD_ERR_INVALID;
    const int d = prm->d;
    // gamma-continuation (eps_stages) is a pd_sinkhorn_batch feature this entry
    // point does not run: refused rather than silently ignored
    if (d < 2 || d > 256 || !(prm->gamma > 0) || !std::isfinite(prm->gamma) || prm->max_iter < 1 ||
        !(prm->tol >= 0) || prm->precision != PD_FP32 || prm->p != 2.0 || prm->eps_stages != 0 || P < 0)
        return PD_ERR_INVALID;
    if (P == 0) return PD_OK;
    if (!cost || !histA || !histB || !massA || !massB) return PD_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= PD_NOALLOC_MAX_DEVICES) return PD_ERR_CUDA;
    // one-time set-up on this device: device address of the static scratch array
    void* base = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (!base) {
        if (cudaGetSymbolAddress(&base, g_noalloc_scratch) != cudaSuccess || !base) return PD_ERR_CUDA;
        g_noalloc_addr[dev].store(base, std::memory_order_release);
    }
    const int dp = ((d + 63) / 64) * 64;
    int* counter = nullptr;
    if (pd_carve_ws(nullptr, P, d, dp, prm->gamma, nullptr, &counter) > PD_NOALLOC_SCRATCH_BYTES)
        return PD_ERR_INVALID;   // this many pairs at this d do not fit in the static scratch
    SkWS w;
    pd_carve_ws((char*)base, P, d, dp, prm->gamma, &w, &counter);
    w.histA = histA; w.histB = histB; w.massA = massA; w.massB = massB; w.pairs = pairs;
    w.p = prm->p;
    if (pd_upload_cost_tables(w, prm->gamma, s) != cudaSuccess) return PD_ERR_CUDA;
    const SkRun r = make_run(prm);
    if (sk_launch_setup(w, g_init, s) != cudaSuccess) return PD_ERR_CUDA;
    int hcount[4] = {0, 0, 0, 0};
    if (lse_rounds(nullptr, w, r, counter, hcount, s) != cudaSuccess) return PD_ERR_CUDA;
    if (sk_launch_lse_finalize(w, cost, row_marg, col_marg, f, g, iters, err, status, 0, s) != cudaSuccess)
        return PD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PD_ERR_CUDA;
    return PD_OK;
}
