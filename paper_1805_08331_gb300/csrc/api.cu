// api.cu -- host implementation of the C ABI declared in include/pd_ot.h.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>
#include <cmath>

#include "pd_internal.h"
#include "../../include/pd_ot.h"


struct pd_ctx {
    int device = 0;
    std::string err;
    void* ws = nullptr;        // Sinkhorn workspace
    size_t ws_bytes = 0;
    int* dflag = nullptr;      // small device scratch (error flags, counters)
    int* hflag = nullptr;      // pinned host mirror
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
        if (c->prof) { a = get(c); b = get(c); cudaEventRecord(a, s); }
    }
    ~ProfScope() {
        if (c->prof) { cudaEventRecord(b, s); c->recs.push_back({kind, a, b}); }
    }
};

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

extern "C" int pd_abi_version(void) { return 1; }

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
    *out = c;
    return PD_OK;
}

extern "C" void pd_ctx_destroy(pd_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    for (auto& r : c->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->ws) cudaFree(c->ws);
    if (c->dflag) cudaFree(c->dflag);
    if (c->hflag) cudaFreeHost(c->hflag);
    delete c;
}

extern "C" const char* pd_last_error(const pd_ctx* c) { return c ? c->err.c_str() : "null context"; }

extern "C" pd_status pd_profile_enable(pd_ctx* c, int enable) {
    if (!c) return PD_ERR_INVALID;
    c->err.clear();
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
    c->err.clear();
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
    c->err.clear();
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
}

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Carve the workspace for P pairs at padded size dp; returns bytes needed when
// base == nullptr.
static size_t carve(char* base, int P, int d, int dp, double gamma, SkWS* w, int** counter) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* { char* r = base ? base + off : nullptr; off += align256(bytes); return r; };
    const size_t M = (size_t)dp * dp, n = M + 1;
    SkWS t{};
    t.d = d; t.dp = dp; t.n = (int)n; t.P = P; t.gamma = gamma;
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
    *counter = (int*)take(sizeof(int) * 4);
    if (w) *w = t;
    return off;
}

extern "C" pd_status pd_sinkhorn_batch(pd_ctx* c, const uint32_t* histA, const uint32_t* massA, const uint32_t* histB,
                                       const uint32_t* massB, const int32_t* pairs, int P,
                                       const pd_sinkhorn_params* prm, const double* g_init, double* cost,
                                       float* row_marg, float* col_marg, double* f, double* g, int32_t* iters,
                                       float* err, int32_t* status, pd_stream stream) {
    if (!c) return PD_ERR_INVALID;
    c->err.clear();
    if (!prm) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: NULL params");
    const int d = prm->d;
    if (d < 2 || d > 256) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: d must be in [2,256]");
    if (!(prm->gamma > 0) || !std::isfinite(prm->gamma)) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: gamma must be > 0");
    if (prm->max_iter < 1) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: max_iter must be >= 1");
    if (!(prm->tol >= 0)) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: tol must be >= 0");
    if (prm->precision != PD_FP32 && prm->precision != PD_FP32_DENSE)
        return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: unknown precision %d", prm->precision);
    if (P < 0) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: P < 0");
    if (P == 0) return PD_OK;
    if (!cost || !histA || !histB || !massA || !massB) return fail(c, PD_ERR_INVALID, "pd_sinkhorn_batch: NULL input/cost");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int dp = ((d + 63) / 64) * 64;
    SkWS w;
    int* counter;
    size_t need = carve(nullptr, P, d, dp, prm->gamma, nullptr, &counter);
    if (need > c->ws_bytes) {
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if (c->ws) cudaFree(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
        if (cudaMalloc(&c->ws, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PD_ERR_OOM, "pd_sinkhorn_batch: cannot allocate %zu bytes of workspace", need);
        }
        c->ws_bytes = need;
    }
    carve((char*)c->ws, P, d, dp, prm->gamma, &w, &counter);
    w.histA = histA; w.histB = histB; w.massA = massA; w.massB = massB; w.pairs = pairs;
    // Cost tables for m = 0..dp-1 (physical units, z = m/d): c_m/gamma = z^2/gamma and
    // cD_m/gamma = z^2/(2 gamma), each split into FP32 hi + lo words; log c_m = 2 log z.
    std::vector<float> tab(5 * dp);
    for (int m = 0; m < dp; ++m) {
        double z = (double)m / d;
        double v = z * z / prm->gamma, v2 = 0.5 * z * z / prm->gamma;
        float hi = (float)v, hi2 = (float)v2;
        tab[m] = hi;
        tab[dp + m] = (float)(v - (double)hi);
        tab[2 * dp + m] = hi2;
        tab[3 * dp + m] = (float)(v2 - (double)hi2);
        tab[4 * dp + m] = m == 0 ? -INFINITY : (float)(2.0 * std::log(z));
    }
    CUDA_TRY(c, cudaMemcpyAsync(w.ctab, tab.data(), sizeof(float) * 5 * dp, cudaMemcpyHostToDevice, s));
    SkRun r;
    r.max_iter = prm->max_iter;
    r.tol = prm->tol;
    r.tau = prm->absorb_tau > 0 ? prm->absorb_tau : 20.0;
    r.absorb_every = prm->absorb_every > 0 ? prm->absorb_every : 64;
    r.rel_thresh = prm->rel_log_thresh < 0 ? prm->rel_log_thresh : (prm->precision == PD_BF16 ? -14.0 : -21.0);
    { ProfScope ps(c, PD_K_SETUP, s); CUDA_TRY(c, sk_launch_setup(w, g_init, s)); }
    if (prm->precision == PD_FP32) {
        // exact log-domain engine: no absorption, iterate until every pair stops
        const int n_inner = 64;
        const int max_rounds = prm->max_iter / n_inner + 2;
        bool any_big = true;
        for (int round = 0; round < max_rounds; ++round) {
            CUDA_TRY(c, cudaMemsetAsync(counter, 0, 2 * sizeof(int), s));
            { ProfScope ps(c, PD_K_ITER, s); CUDA_TRY(c, sk_launch_lse_smem(w, r, n_inner, counter, counter + 1, s)); }
            if (any_big) {   // pairs whose supports do not fit on chip
                ProfScope ps(c, PD_K_ITER, s);
                CUDA_TRY(c, sk_launch_lse_iter(w, r, n_inner, counter, s));
            }
            CUDA_TRY(c, cudaMemcpyAsync(c->hflag, counter, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
            CUDA_TRY(c, cudaStreamSynchronize(s));
            if (round == 0) any_big = c->hflag[1] > 0;
            if (c->hflag[0] == 0) break;
        }
        { ProfScope ps(c, PD_K_FINALIZE, s);
          CUDA_TRY(c, sk_launch_lse_finalize(w, cost, row_marg, col_marg, f, g, iters, err, status, s)); }
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
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return PD_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of pd_sinkhorn_batch (PD_FP32 engine only).
//
// Its workspace is the file-scope device array below instead of memory from
// cudaMalloc: every GPU that loads this library reserves it for the lifetime
// of the process.  Host code cannot use the array's name as a device address
// (in host code it names a host-side stand-in), so the device address is
// obtained once per device with cudaGetSymbolAddress and cached.
#define PD_NOALLOC_SCRATCH_BYTES (16u << 20)
#define PD_NOALLOC_MAX_DEVICES 64
static __device__ __align__(256) unsigned char g_noalloc_scratch[PD_NOALLOC_SCRATCH_BYTES];
static void* g_noalloc_addr[PD_NOALLOC_MAX_DEVICES];

extern "C" pd_status pd_sinkhorn_batch_noalloc(const uint32_t* histA, const uint32_t* massA,
                                               const uint32_t* histB, const uint32_t* massB,
                                               const int32_t* pairs, int P, const pd_sinkhorn_params* prm,
                                               const double* g_init, double* cost, float* row_marg,
                                               float* col_marg, double* f, double* g, int32_t* iters,
                                               float* err, int32_t* status, pd_stream stream) {
    if (!prm) return PD_ERR_INVALID;
    const int d = prm->d;
    if (d < 2 || d > 256 || !(prm->gamma > 0) || !std::isfinite(prm->gamma) || prm->max_iter < 1 ||
        !(prm->tol >= 0) || prm->precision != PD_FP32 || P < 0)
        return PD_ERR_INVALID;
    if (P == 0) return PD_OK;
    if (!cost || !histA || !histB || !massA || !massB) return PD_ERR_INVALID;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= PD_NOALLOC_MAX_DEVICES) return PD_ERR_CUDA;
    // one-time set-up on this device: device address of the static scratch array
    if (!g_noalloc_addr[dev]) {
        void* a = nullptr;
        if (cudaGetSymbolAddress(&a, g_noalloc_scratch) != cudaSuccess || !a) return PD_ERR_CUDA;
        g_noalloc_addr[dev] = a;
    }
    const int dp = ((d + 63) / 64) * 64;
    int* counter = nullptr;
    if (carve(nullptr, P, d, dp, prm->gamma, nullptr, &counter) > PD_NOALLOC_SCRATCH_BYTES)
        return PD_ERR_INVALID;   // this many pairs at this d do not fit in the static scratch
    SkWS w;
    carve((char*)g_noalloc_addr[dev], P, d, dp, prm->gamma, &w, &counter);
    w.histA = histA; w.histB = histB; w.massA = massA; w.massB = massB; w.pairs = pairs;
    float tab[5 * 256];
    for (int m = 0; m < dp; ++m) {
        double z = (double)m / d;
        double v = z * z / prm->gamma, v2 = 0.5 * z * z / prm->gamma;
        float hi = (float)v, hi2 = (float)v2;
        tab[m] = hi;
        tab[dp + m] = (float)(v - (double)hi);
        tab[2 * dp + m] = hi2;
        tab[3 * dp + m] = (float)(v2 - (double)hi2);
        tab[4 * dp + m] = m == 0 ? -INFINITY : (float)(2.0 * std::log(z));
    }
    if (cudaMemcpyAsync(w.ctab, tab, sizeof(float) * 5 * dp, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return PD_ERR_CUDA;
    SkRun r;
    r.max_iter = prm->max_iter;
    r.tol = prm->tol;
    r.tau = 20.0;
    r.absorb_every = 64;
    r.rel_thresh = -21.0;
    if (sk_launch_setup(w, g_init, s) != cudaSuccess) return PD_ERR_CUDA;
    const int n_inner = 64;
    const int max_rounds = prm->max_iter / n_inner + 2;
    int hcount[2] = {0, 0};
    bool any_big = true;
    for (int round = 0; round < max_rounds; ++round) {
        if (cudaMemsetAsync(counter, 0, 2 * sizeof(int), s) != cudaSuccess) return PD_ERR_CUDA;
        if (sk_launch_lse_smem(w, r, n_inner, counter, counter + 1, s) != cudaSuccess) return PD_ERR_CUDA;
        if (any_big && sk_launch_lse_iter(w, r, n_inner, counter, s) != cudaSuccess) return PD_ERR_CUDA;
        if (cudaMemcpyAsync(hcount, counter, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return PD_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return PD_ERR_CUDA;
        if (round == 0) any_big = hcount[1] > 0;
        if (hcount[0] == 0) break;
    }
    if (sk_launch_lse_finalize(w, cost, row_marg, col_marg, f, g, iters, err, status, s) != cudaSuccess)
        return PD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PD_ERR_CUDA;
    return PD_OK;
}
