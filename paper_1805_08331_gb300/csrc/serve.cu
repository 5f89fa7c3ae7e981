// serve.cu -- pd_serve_*: a request loop with continuous batching for
// distance and nearest-centroid queries between persistence diagrams.
//
// The paper has no serving component; each query is answered by PD_FP32
// solves of Alg. 1 (the distance of Sec. 3 / the assignment step of the
// k-means of Sec. 5).  What this file adds is the scheduling around them:
//   - one pool of pair slots per grid size d (32, 64, 128, 256); a slot is the
//     device workspace of one Sinkhorn pair and the pool's size is fixed by a
//     device-memory budget at creation (admission by free memory = free slots);
//   - one worker thread per pool running scheduling rounds: admit queued
//     queries (FIFO) into free slots, rasterise + set them up, run
//     `inner_iters` iterations of every active pair of the pool, finalise the
//     pairs that stopped and release their slots.  Pools have their own
//     streams, so the launches of different grid sizes overlap on the device.  A query that arrives while others are on the
//     GPU joins at the next round boundary: iteration-level continuous batching;
//   - resident centroids per d and, with warm_start, the centroid-side
//     potential g of the last finished solve against each centroid, used as the
//     initial g of the next solve against it.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pd_common.cuh"
#include "pd_internal.h"
#include "../../include/pd_ot.h"

int pd_ctx_device(const pd_ctx* c);

namespace {

constexpr int kNumPools = 4;
constexpr int kPoolD[kNumPools] = {32, 64, 128, 256};
int pool_index(int d) {
    for (int i = 0; i < kNumPools; ++i)
        if (kPoolD[i] == d) return i;
    return -1;
}
double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Slot initialisation descriptor: side A from raster diagram srcA, side B
// from raster diagram srcB (distance) or centroid `centroid` (nearest).
struct SlotInit {
    int slot, srcA, srcB, centroid, warm;
};

__global__ void serve_gather_kernel(const SlotInit* __restrict__ si, const uint32_t* __restrict__ H,
                                    const double* __restrict__ Z, const double* __restrict__ warm, int d,
                                    double* __restrict__ WA, double* __restrict__ WB, double* __restrict__ ginit) {
    const SlotInit s = si[blockIdx.x];
    const int D = d * d, n1 = D + 1;
    double* wa = WA + (size_t)s.slot * D;
    double* wb = WB + (size_t)s.slot * D;
    double* gi = ginit + (size_t)s.slot * n1;
    for (int x = threadIdx.x; x < D; x += blockDim.x) {
        wa[x] = (double)H[(size_t)s.srcA * D + x];
        wb[x] = s.srcB >= 0 ? (double)H[(size_t)s.srcB * D + x] : Z[(size_t)s.centroid * D + x];
    }
    for (int x = threadIdx.x; x < n1; x += blockDim.x) gi[x] = s.warm ? warm[(size_t)s.centroid * n1 + x] : 0.0;
}

// status of every slot (IC_STATUS of the workspace)
__global__ void serve_status_kernel(const int* __restrict__ ic, int S, int* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < S) out[p] = ic[(size_t)p * IC_N + IC_STATUS];
}

// results of the finished slots, compacted: res[3*i] = cost, res[3*i+1] = iters, res[3*i+2] = status
__global__ void serve_collect_kernel(const int* __restrict__ list, int n, const double* __restrict__ cost,
                                     const int32_t* __restrict__ iters, const int32_t* __restrict__ status,
                                     double* __restrict__ res) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const int s = list[i];
        res[3 * i] = cost[s];
        res[3 * i + 1] = (double)iters[s];
        res[3 * i + 2] = (double)status[s];
    }
}

// warm[c] <- g of slot s on the centroid's support and Delta (0 elsewhere);
// list holds (slot, centroid) pairs.
__global__ void serve_warm_kernel(const int2* __restrict__ list, const double* __restrict__ gout,
                                  const double* __restrict__ Z, int d, double* __restrict__ warm) {
    const int2 sc = list[blockIdx.x];
    const int D = d * d, n1 = D + 1;
    const double* g = gout + (size_t)sc.x * n1;
    const double* z = Z + (size_t)sc.y * D;
    double* wv = warm + (size_t)sc.y * n1;
    for (int x = threadIdx.x; x < D; x += blockDim.x) {
        const double v = g[x];
        wv[x] = (z[x] > 0.0 && isfinite(v)) ? v : 0.0;
    }
    if (threadIdx.x == 0) wv[D] = isfinite(g[D]) ? g[D] : 0.0;
}

// Grow-only buffers (device or pinned host).  Growth happens only between
// rounds, after every stream using them has been synchronised.
struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= n) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        size_t want = std::max(bytes, (size_t)4096);
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) n = want;
        return e;
    }
    void release() { if (p) cudaFree(p); p = nullptr; n = 0; }
};
struct HostBuf {
    void* p = nullptr;
    size_t n = 0;
    cudaError_t ensure(size_t bytes) {
        if (bytes <= n) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        size_t want = std::max(bytes, (size_t)4096);
        cudaError_t e = cudaMallocHost(&p, want);
        if (e == cudaSuccess) n = want;
        return e;
    }
    void release() { if (p) cudaFreeHost(p); p = nullptr; n = 0; }
};

struct Req {
    uint64_t ticket = 0;
    int kind = 0, d = 0;
    std::vector<double> ba, da, bb, db;
    int npairs = 0, done = 0;
    double best = INFINITY;
    int best_c = -1;
    int max_iters = 0;
    pd_status st = PD_OK;   // aggregate of the solves
    bool finished = false;
    double t_submit = 0, t_done = 0;
};

struct Pool {
    int d = 0, dp = 0, S = 0;
    void* ws = nullptr;
    SkWS w{};
    int* counter = nullptr;            // 8 device ints inside ws
    double *WA = nullptr, *WB = nullptr, *ginit = nullptr, *gout = nullptr, *cost = nullptr;
    int32_t *iters = nullptr, *status = nullptr;
    float* err = nullptr;
    int* dstat = nullptr;              // [S] slot status mirror (device)
    int* dbad = nullptr;
    // resident centroids
    int k = 0;
    double* Z = nullptr;               // [k][d*d]
    double* warm = nullptr;            // [k][d*d+1]
    std::vector<char> warm_valid;
    // host bookkeeping
    std::vector<int> free_slots;
    std::vector<Req*> owner;           // [S]
    std::vector<int> owner_c;          // [S] centroid of a nearest pair, -1 for distance
    std::vector<int> active;           // slots in use
    bool any_gm = false, any_old = false;   // pairs in the global-memory tiers
    int gbits = -1;
    cudaStream_t stream = nullptr;
    // staging
    DevBuf d_pts, d_off, d_hist, d_mass, d_init, d_list, d_list2, d_res;
    HostBuf h_pts, h_off, h_init, h_list, h_list2, h_res, h_stat, h_cnt;
};

}  // namespace

struct pd_server {
    pd_ctx* ctx = nullptr;
    int device = 0;
    pd_serve_config cfg{};
    SkRun run{};
    Pool pools[kNumPools];
    std::thread workers[kNumPools];
    std::mutex mu;
    std::condition_variable cv_work[kNumPools], cv_done;
    std::deque<Req*> queue[kNumPools];             // submitted, not yet taken by the pool's worker
    std::unordered_map<uint64_t, Req*> live;       // every ticket not yet returned by poll
    uint64_t next_ticket = 1;
    int outstanding = 0;                           // live tickets
    bool stop = false;
    bool dead = false;                             // worker stopped after a failure
    bool inject = false;
    int inflight[kNumPools] = {0, 0, 0, 0};       // queries of that d submitted and not finished
    std::string err;
};

namespace {

// Complete a request (called with sv->mu held).
void complete_locked(pd_server* sv, Req* r, pd_status st) {
    if (r->finished) return;
    r->finished = true;
    if (st != PD_OK) r->st = st;
    r->t_done = now_ms();
    const int pi = pool_index(r->d);
    if (pi >= 0) sv->inflight[pi]--;
    sv->cv_done.notify_all();
}

cudaError_t pool_create(Pool& P, int d, int S, double gamma, bool want_g) {
    P.d = d;
    P.dp = ((d + 63) / 64) * 64;
    P.S = S;
    const size_t D = (size_t)d * d, n1 = D + 1;
    size_t wsb = pd_carve_ws(nullptr, S, d, P.dp, gamma, nullptr, &P.counter);
    cudaError_t e = cudaMalloc(&P.ws, wsb);
    if (e != cudaSuccess) return e;
    pd_carve_ws((char*)P.ws, S, d, P.dp, gamma, &P.w, &P.counter);
    auto dalloc = [&](void** p, size_t bytes) { return cudaMalloc(p, std::max(bytes, (size_t)256)); };
    if ((e = dalloc((void**)&P.WA, sizeof(double) * D * S)) != cudaSuccess) return e;
    if ((e = dalloc((void**)&P.WB, sizeof(double) * D * S)) != cudaSuccess) return e;
    if ((e = dalloc((void**)&P.ginit, sizeof(double) * n1 * S)) != cudaSuccess) return e;
    if (want_g && (e = dalloc((void**)&P.gout, sizeof(double) * n1 * S)) != cudaSuccess) return e;
    if ((e = dalloc((void**)&P.cost, sizeof(double) * S)) != cudaSuccess) return e;
    if ((e = dalloc((void**)&P.iters, sizeof(int32_t) * S)) != cudaSuccess) return e;
    if ((e = dalloc((void**)&P.status, sizeof(int32_t) * S)) != cudaSuccess) return e;
    if ((e = dalloc((void**)&P.err, sizeof(float) * S)) != cudaSuccess) return e;
    if ((e = dalloc((void**)&P.dstat, sizeof(int) * S)) != cudaSuccess) return e;
    if ((e = dalloc((void**)&P.dbad, sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking)) != cudaSuccess) return e;
    P.w.wA = P.WA;
    P.w.wB = P.WB;
    P.w.histA = P.w.histB = nullptr;
    P.w.massA = P.w.massB = nullptr;
    P.w.pairs = nullptr;
    if ((e = pd_upload_cost_tables(P.w, gamma, P.stream)) != cudaSuccess) return e;
    // the iteration kernel reads the pool's workspace descriptor from device memory
    if ((e = cudaMemcpyAsync(P.w.groups, &P.w, sizeof(SkWS), cudaMemcpyHostToDevice, P.stream)) != cudaSuccess)
        return e;
    // every slot starts stopped (status != ST_ACTIVE), so iteration launches skip it
    std::vector<int> ic((size_t)IC_N * S, 0);
    for (int s = 0; s < S; ++s) ic[(size_t)s * IC_N + IC_STATUS] = ST_CONVERGED;
    if ((e = cudaMemcpyAsync(P.w.ic, ic.data(), ic.size() * sizeof(int), cudaMemcpyHostToDevice, P.stream)) !=
        cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(P.stream)) != cudaSuccess) return e;
    P.free_slots.resize(S);
    for (int s = 0; s < S; ++s) P.free_slots[s] = S - 1 - s;   // pop_back hands out slot 0 first
    P.owner.assign(S, nullptr);
    P.owner_c.assign(S, -1);
    P.gbits = sk_lse2_grid_bits(gamma);
    return cudaSuccess;
}

void pool_destroy(Pool& P) {
    if (P.stream) cudaStreamSynchronize(P.stream);
    void* ptrs[] = {P.ws, P.WA, P.WB, P.ginit, P.gout, P.cost, P.iters, P.status, P.err, P.dstat, P.dbad, P.Z, P.warm};
    for (void* p : ptrs) if (p) cudaFree(p);
    DevBuf* db[] = {&P.d_pts, &P.d_off, &P.d_hist, &P.d_mass, &P.d_init, &P.d_list, &P.d_list2, &P.d_res};
    for (auto b : db) b->release();
    HostBuf* hb[] = {&P.h_pts, &P.h_off, &P.h_init, &P.h_list, &P.h_list2, &P.h_res, &P.h_stat, &P.h_cnt};
    for (auto b : hb) b->release();
    if (P.stream) cudaStreamDestroy(P.stream);
    P = Pool();
}

// Raster diagram of a round: request r, side 0 (A) or 1 (B).
struct RDiag { Req* r; int side; };

#define SV_TRY(expr)                                   \
    do {                                               \
        cudaError_t _e = (expr);                       \
        if (_e != cudaSuccess) return _e;              \
    } while (0)

// Admission work of one pool: rasterise the new diagrams, fill the new slots, set them up.
cudaError_t pool_admit(pd_server* sv, Pool& P, const std::vector<RDiag>& diags, const std::vector<SlotInit>& inits) {
    if (inits.empty()) return cudaSuccess;
    const int nd = (int)diags.size(), D = P.d * P.d;
    size_t npts = 0;
    for (auto& g : diags) npts += g.side == 0 ? g.r->ba.size() : g.r->bb.size();
    SV_TRY(P.h_pts.ensure(sizeof(double) * 2 * std::max(npts, (size_t)1)));
    SV_TRY(P.d_pts.ensure(sizeof(double) * 2 * std::max(npts, (size_t)1)));
    SV_TRY(P.h_off.ensure(sizeof(int64_t) * (nd + 1)));
    SV_TRY(P.d_off.ensure(sizeof(int64_t) * (nd + 1)));
    SV_TRY(P.d_hist.ensure(sizeof(uint32_t) * (size_t)nd * D));
    SV_TRY(P.d_mass.ensure(sizeof(uint32_t) * nd));
    SV_TRY(P.h_init.ensure(sizeof(SlotInit) * inits.size()));
    SV_TRY(P.d_init.ensure(sizeof(SlotInit) * inits.size()));
    SV_TRY(P.h_list.ensure(sizeof(int) * inits.size()));
    SV_TRY(P.d_list.ensure(sizeof(int) * inits.size()));
    double* hb = (double*)P.h_pts.p;
    double* ht = hb + npts;
    int64_t* ho = (int64_t*)P.h_off.p;
    size_t o = 0;
    for (int i = 0; i < nd; ++i) {
        const std::vector<double>& b = diags[i].side == 0 ? diags[i].r->ba : diags[i].r->bb;
        const std::vector<double>& t = diags[i].side == 0 ? diags[i].r->da : diags[i].r->db;
        ho[i] = (int64_t)o;
        std::memcpy(hb + o, b.data(), sizeof(double) * b.size());
        std::memcpy(ht + o, t.data(), sizeof(double) * t.size());
        o += b.size();
    }
    ho[nd] = (int64_t)o;
    std::memcpy(P.h_init.p, inits.data(), sizeof(SlotInit) * inits.size());
    int* hl = (int*)P.h_list.p;
    for (size_t i = 0; i < inits.size(); ++i) hl[i] = inits[i].slot;
    double* db = (double*)P.d_pts.p;
    SV_TRY(cudaMemcpyAsync(db, hb, sizeof(double) * 2 * npts, cudaMemcpyHostToDevice, P.stream));
    SV_TRY(cudaMemcpyAsync(P.d_off.p, ho, sizeof(int64_t) * (nd + 1), cudaMemcpyHostToDevice, P.stream));
    SV_TRY(cudaMemcpyAsync(P.d_init.p, P.h_init.p, sizeof(SlotInit) * inits.size(), cudaMemcpyHostToDevice,
                           P.stream));
    SV_TRY(cudaMemcpyAsync(P.d_list.p, hl, sizeof(int) * inits.size(), cudaMemcpyHostToDevice, P.stream));
    SV_TRY(pd_launch_raster(db, db + npts, (const int64_t*)P.d_off.p, nd, P.d, (int64_t)npts,
                            (uint32_t*)P.d_hist.p, (uint32_t*)P.d_mass.p, P.dbad, P.stream));
    serve_gather_kernel<<<(int)inits.size(), 256, 0, P.stream>>>((const SlotInit*)P.d_init.p,
                                                                 (const uint32_t*)P.d_hist.p, P.Z, P.warm, P.d,
                                                                 P.WA, P.WB, P.ginit);
    SV_TRY(cudaGetLastError());
    return sk_launch_setup_list(P.w, P.ginit, (const int*)P.d_list.p, (int)inits.size(), P.stream);
}

// One scheduling round of pool pi.  Returns a CUDA error (the caller then
// fails every query) or cudaSuccess.
cudaError_t serve_round(pd_server* sv, int pi, std::vector<Req*>& pending) {
    Pool& P = sv->pools[pi];
    // ---- 1. admission, FIFO; a query that does not fit blocks the later ones
    std::vector<RDiag> diags;
    std::vector<SlotInit> inits;
    size_t taken = 0;
    for (; taken < pending.size(); ++taken) {
        Req* r = pending[taken];
        const int need = r->kind == PD_Q_DISTANCE ? 1 : P.k;
        if ((int)P.free_slots.size() < need) break;
        const int ia = (int)diags.size();
        diags.push_back({r, 0});
        int ib = -1;
        if (r->kind == PD_Q_DISTANCE) {
            ib = ia + 1;
            diags.push_back({r, 1});
        }
        r->npairs = need;
        for (int c = 0; c < need; ++c) {
            const int slot = P.free_slots.back();
            P.free_slots.pop_back();
            const int cen = r->kind == PD_Q_NEAREST ? c : -1;
            P.owner[slot] = r;
            P.owner_c[slot] = cen;
            P.active.push_back(slot);
            const int warm = (cen >= 0 && sv->cfg.warm_start && P.warm_valid[cen]) ? 1 : 0;
            inits.push_back({slot, ia, ib, cen, warm});
        }
    }
    pending.erase(pending.begin(), pending.begin() + (long)taken);
    if (P.active.empty()) return cudaSuccess;
    // ---- 2. admission work and the shared-memory need of the active pairs
    SV_TRY(pool_admit(sv, P, diags, inits));
    SV_TRY(P.h_cnt.ensure(sizeof(int) * 4));
    SV_TRY(cudaMemsetAsync(P.counter, 0, sizeof(int) * 4, P.stream));
    if (P.gbits >= 0) SV_TRY(sk_launch_lse2_need(P.w, P.counter + 2, sv->run.form, P.stream));
    SV_TRY(cudaMemcpyAsync(P.h_cnt.p, P.counter, sizeof(int) * 4, cudaMemcpyDeviceToHost, P.stream));
    SV_TRY(cudaStreamSynchronize(P.stream));
    // ---- 3. one round of iterations, then the slots' status
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, sv->device);
    const int inner = sv->cfg.inner_iters > 0 ? sv->cfg.inner_iters : 64;
    const size_t smem = (size_t)((int*)P.h_cnt.p)[2];
    const int na = (int)P.active.size();
    // wider CTAs when few pairs are active, or when the largest pair's shared
    // memory lets only 2 (1) CTAs onto an SM (dynamic + static + 1 KB per CTA)
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, sv->device);
    const int fit_per_sm = smem > 0 ? (int)((size_t)smem_sm / (smem + 2048)) : 3;
    const bool pw_all = ((int*)P.h_cnt.p)[3] == 0;   // every pair pairwise: no widening
    const int by_active = pw_all || na > 2 * nsm ? 256 : (na > nsm ? 512 : 1024);
    const int by_smem = fit_per_sm <= 1 ? 1024 : (fit_per_sm == 2 ? 512 : 256);
    const int threads = by_active > by_smem ? by_active : by_smem;
    SV_TRY(cudaMemsetAsync(P.counter, 0, sizeof(int) * 4, P.stream));
    SV_TRY(P.gbits >= 0 ? sk_launch_lse2(P.w, sv->run, inner, P.counter, smem, P.gbits, threads, P.stream)
                        : sk_launch_lse_smem(P.w, sv->run, inner, P.counter, P.counter + 1, P.stream));
    if (P.gbits >= 0 && P.any_gm) SV_TRY(sk_launch_lse2_gm(P.w, sv->run, inner, P.counter, P.gbits, (size_t)-1, P.stream));
    if (P.any_old) SV_TRY(sk_launch_lse_iter(P.w, sv->run, inner, P.counter, P.gbits >= 0 ? 2 : 1, P.stream));
    serve_status_kernel<<<(P.S + 255) / 256, 256, 0, P.stream>>>(P.w.ic, P.S, P.dstat);
    SV_TRY(cudaGetLastError());
    SV_TRY(P.h_stat.ensure(sizeof(int) * P.S));
    SV_TRY(cudaMemcpyAsync(P.h_stat.p, P.dstat, sizeof(int) * P.S, cudaMemcpyDeviceToHost, P.stream));
    SV_TRY(cudaMemcpyAsync(P.h_cnt.p, P.counter, sizeof(int) * 4, cudaMemcpyDeviceToHost, P.stream));
    SV_TRY(cudaStreamSynchronize(P.stream));
    // ---- 4. finalise the pairs that stopped
    {
        // pairs handed on to the global-memory variant / the FP64 kernel run there from the next round on
        const int* hc = (const int*)P.h_cnt.p;
        if (P.gbits >= 0) {
            if (hc[1] > 0) P.any_gm = true;
            if (hc[3] > 0) P.any_old = true;
        } else if (hc[1] > 0) {
            P.any_old = true;
        }
    }
    std::vector<int> fin;
    const int* st = (const int*)P.h_stat.p;
    for (int s : P.active)
        if (st[s] != ST_ACTIVE) fin.push_back(s);
    if (fin.empty()) return cudaSuccess;
    const int nf = (int)fin.size();
    SV_TRY(P.h_list.ensure(sizeof(int) * nf));
    SV_TRY(P.d_list.ensure(sizeof(int) * nf));
    std::memcpy(P.h_list.p, fin.data(), sizeof(int) * nf);
    SV_TRY(cudaMemcpyAsync(P.d_list.p, P.h_list.p, sizeof(int) * nf, cudaMemcpyHostToDevice, P.stream));
    SV_TRY(sk_launch_lse_finalize_list(P.w, P.cost, nullptr, nullptr, nullptr, sv->cfg.warm_start ? P.gout : nullptr,
                                       P.iters, P.err, P.status, 1, (const int*)P.d_list.p, nf, P.stream));
    if (sv->cfg.warm_start) {
        std::vector<int2> wl;
        for (int s : fin)
            if (P.owner_c[s] >= 0) wl.push_back(make_int2(s, P.owner_c[s]));
        if (!wl.empty()) {
            SV_TRY(P.h_list2.ensure(sizeof(int2) * wl.size()));
            SV_TRY(P.d_list2.ensure(sizeof(int2) * wl.size()));
            std::memcpy(P.h_list2.p, wl.data(), sizeof(int2) * wl.size());
            SV_TRY(cudaMemcpyAsync(P.d_list2.p, P.h_list2.p, sizeof(int2) * wl.size(), cudaMemcpyHostToDevice,
                                   P.stream));
            serve_warm_kernel<<<(int)wl.size(), 256, 0, P.stream>>>((const int2*)P.d_list2.p, P.gout, P.Z, P.d,
                                                                   P.warm);
            SV_TRY(cudaGetLastError());
        }
    }
    SV_TRY(P.d_res.ensure(sizeof(double) * 3 * nf));
    SV_TRY(P.h_res.ensure(sizeof(double) * 3 * nf));
    serve_collect_kernel<<<(nf + 255) / 256, 256, 0, P.stream>>>((const int*)P.d_list.p, nf, P.cost, P.iters,
                                                                P.status, (double*)P.d_res.p);
    SV_TRY(cudaGetLastError());
    SV_TRY(cudaMemcpyAsync(P.h_res.p, P.d_res.p, sizeof(double) * 3 * nf, cudaMemcpyDeviceToHost, P.stream));
    SV_TRY(cudaStreamSynchronize(P.stream));
    // ---- 5. hand out results, release slots
    std::lock_guard<std::mutex> lk(sv->mu);
    const double* res = (const double*)P.h_res.p;
    for (size_t i = 0; i < fin.size(); ++i) {
        const int s = fin[i];
        Req* r = P.owner[s];
        const int c = P.owner_c[s];
        const double cost = res[3 * i];
        const int it = (int)res[3 * i + 1];
        const int stt = (int)res[3 * i + 2];
        if (stt == PD_NOT_CONVERGED && r->st == PD_OK) r->st = PD_NOT_CONVERGED;
        else if (stt != PD_OK && stt != PD_NOT_CONVERGED) r->st = stt;
        r->max_iters = std::max(r->max_iters, it);
        if (c < 0) {
            r->best = cost;
        } else {
            if (cost < r->best || (cost == r->best && c < r->best_c) || r->best_c < 0) {
                r->best = cost;
                r->best_c = c;
            }
            if (sv->cfg.warm_start && std::isfinite(cost)) P.warm_valid[c] = 1;
        }
        if (++r->done == r->npairs) complete_locked(sv, r, PD_OK);
        P.owner[s] = nullptr;
        P.owner_c[s] = -1;
        P.free_slots.push_back(s);
    }
    std::vector<int> keep;
    keep.reserve(P.active.size());
    for (int s : P.active)
        if (P.owner[s]) keep.push_back(s);
    P.active.swap(keep);
    return cudaSuccess;
}

// Fail the queries a worker holds (its pending list and its pool's slots)
// with PD_ERR_CUDA; called with sv->mu held.
void fail_own_locked(pd_server* sv, int pi, std::vector<Req*>& pending) {
    for (Req* r : pending) complete_locked(sv, r, PD_ERR_CUDA);
    pending.clear();
    for (Req* r : sv->queue[pi]) complete_locked(sv, r, PD_ERR_CUDA);
    sv->queue[pi].clear();
    Pool& P = sv->pools[pi];
    for (int s : P.active)
        if (P.owner[s]) complete_locked(sv, P.owner[s], PD_ERR_CUDA);
}

// Worker of pool pi: rounds while it has work, sleeps otherwise.  Each pool
// has its own worker and stream, so a slow grid size does not hold back the
// rounds of the others.  A failure (or an injected one) stops every worker.
void worker_main(pd_server* sv, int pi) {
    cudaSetDevice(sv->device);
    Pool& P = sv->pools[pi];
    std::vector<Req*> pending;
    while (true) {
        const bool active = !pending.empty() || !P.active.empty();
        bool inject = false;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            if (!active)
                sv->cv_work[pi].wait(lk, [&] { return sv->stop || sv->dead || !sv->queue[pi].empty() || sv->inject; });
            if (sv->stop) break;
            if (sv->dead) {
                fail_own_locked(sv, pi, pending);
                break;
            }
            while (!sv->queue[pi].empty()) {
                pending.push_back(sv->queue[pi].front());
                sv->queue[pi].pop_front();
            }
            inject = sv->inject;
            sv->inject = false;
        }
        const cudaError_t e = inject ? cudaErrorUnknown : serve_round(sv, pi, pending);
        if (e != cudaSuccess) {
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                sv->dead = true;
                sv->err = std::string("serving stopped: ") + cudaGetErrorString(e);
                fail_own_locked(sv, pi, pending);
            }
            for (auto& cv : sv->cv_work) cv.notify_all();
            break;
        }
    }
}

bool points_ok(const double* b, const double* t, int n) {
    if (n < 0 || (n > 0 && (!b || !t))) return false;
    for (int i = 0; i < n; ++i)
        if (!(b[i] >= 0.0 && b[i] <= 1.0 && t[i] >= 0.0 && t[i] <= 1.0 && b[i] <= t[i])) return false;
    return true;
}

}  // namespace

extern "C" void pd_serve_default_config(pd_serve_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->gamma = 5e-3;
    cfg->tol = 1e-4;
    cfg->max_iter = 5000;
    cfg->inner_iters = 64;
    cfg->max_hbm_bytes = 0;
    cfg->queue_capacity = 65536;
    cfg->warm_start = 1;
}

extern "C" pd_status pd_serve_create(pd_ctx* ctx, const pd_serve_config* cfg, pd_server** out) {
    if (!ctx || !cfg || !out) return PD_ERR_INVALID;
    *out = nullptr;
    if (!(cfg->gamma > 0) || !std::isfinite(cfg->gamma) || !(cfg->tol >= 0) || cfg->max_iter < 1) return PD_ERR_INVALID;
    const int dev = pd_ctx_device(ctx);
    if (cudaSetDevice(dev) != cudaSuccess) return PD_ERR_CUDA;
    pd_server* sv = new pd_server();
    sv->ctx = ctx;
    sv->device = dev;
    sv->cfg = *cfg;
    if (sv->cfg.queue_capacity <= 0) sv->cfg.queue_capacity = 65536;
    if (sv->cfg.inner_iters <= 0) sv->cfg.inner_iters = 64;
    sv->run.max_iter = cfg->max_iter;
    sv->run.tol = cfg->tol;
    sv->run.tau = 20.0;
    sv->run.absorb_every = 64;
    sv->run.rel_thresh = -21.0;
    sv->run.pot_support_only = 1;
    sv->run.form = SK_FORM_AUTO2;   // the pool's launch carries pairs of every size
    // slots per pool: explicit, or an equal share of the memory budget
    size_t budget = cfg->max_hbm_bytes;
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { delete sv; return PD_ERR_CUDA; }
        budget = fr / 2;
    }
    int nauto = 0;
    for (int i = 0; i < kNumPools; ++i) nauto += cfg->slots[i] == 0;
    for (int i = 0; i < kNumPools; ++i) {
        int S = cfg->slots[i] < 0 ? 0 : cfg->slots[i];
        if (cfg->slots[i] == 0) {
            const int d = kPoolD[i], dp = ((d + 63) / 64) * 64;
            int* dummy;
            const size_t per = pd_carve_ws(nullptr, 1, d, dp, cfg->gamma, nullptr, &dummy) +
                               sizeof(double) * ((size_t)d * d * 2 + ((size_t)d * d + 1) * 2) + 64;
            const size_t share = budget / (size_t)nauto;
            S = (int)std::min<size_t>(share / per, 8192);
        }
        if (S > 0) {
            cudaError_t e = pool_create(sv->pools[i], kPoolD[i], S, cfg->gamma, cfg->warm_start != 0);
            if (e != cudaSuccess) {
                for (auto& P : sv->pools) pool_destroy(P);
                cudaGetLastError();
                delete sv;
                return e == cudaErrorMemoryAllocation ? PD_ERR_OOM : PD_ERR_CUDA;
            }
        }
    }
    for (int i = 0; i < kNumPools; ++i)
        if (sv->pools[i].S > 0) sv->workers[i] = std::thread(worker_main, sv, i);
    *out = sv;
    return PD_OK;
}

extern "C" pd_status pd_serve_load_centroids(pd_server* sv, int d, const double* z, int k) {
    if (!sv || !z || k < 1) return PD_ERR_INVALID;
    const int pi = pool_index(d);
    if (pi < 0) return PD_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    Pool& P = sv->pools[pi];
    if (P.S == 0 || k > P.S || sv->inflight[pi] > 0 || sv->dead) return PD_ERR_INVALID;
    if (cudaSetDevice(sv->device) != cudaSuccess) return PD_ERR_CUDA;
    const size_t D = (size_t)d * d;
    if (P.Z) cudaFree(P.Z);
    if (P.warm) cudaFree(P.warm);
    P.Z = nullptr;
    P.warm = nullptr;
    P.k = 0;
    if (cudaMalloc(&P.Z, sizeof(double) * D * k) != cudaSuccess ||
        cudaMalloc(&P.warm, sizeof(double) * (D + 1) * k) != cudaSuccess) {
        cudaGetLastError();
        return PD_ERR_OOM;
    }
    if (cudaMemcpyAsync(P.Z, z, sizeof(double) * D * k, cudaMemcpyDeviceToDevice, P.stream) != cudaSuccess ||
        cudaMemsetAsync(P.warm, 0, sizeof(double) * (D + 1) * k, P.stream) != cudaSuccess ||
        cudaStreamSynchronize(P.stream) != cudaSuccess)
        return PD_ERR_CUDA;
    P.k = k;
    P.warm_valid.assign(k, 0);
    return PD_OK;
}

extern "C" pd_status pd_serve_submit(pd_server* sv, const pd_query* q, uint64_t* ticket) {
    if (!sv || !q || !ticket) return PD_ERR_INVALID;
    const int pi = pool_index(q->d);
    if (pi < 0 || (q->kind != PD_Q_DISTANCE && q->kind != PD_Q_NEAREST)) return PD_ERR_INVALID;
    if (!points_ok(q->birth_a_host, q->death_a_host, q->n_a)) return PD_ERR_INVALID;
    if (q->kind == PD_Q_DISTANCE && !points_ok(q->birth_b_host, q->death_b_host, q->n_b)) return PD_ERR_INVALID;
    Req* r = new Req();
    r->kind = q->kind;
    r->d = q->d;
    r->ba.assign(q->birth_a_host, q->birth_a_host + q->n_a);
    r->da.assign(q->death_a_host, q->death_a_host + q->n_a);
    if (q->kind == PD_Q_DISTANCE) {
        r->bb.assign(q->birth_b_host, q->birth_b_host + q->n_b);
        r->db.assign(q->death_b_host, q->death_b_host + q->n_b);
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        Pool& P = sv->pools[pi];
        pd_status bad = PD_OK;
        if (sv->dead) bad = PD_ERR_CUDA;
        else if (P.S == 0) bad = PD_ERR_INVALID;
        else if (q->kind == PD_Q_NEAREST && P.k == 0) bad = PD_ERR_INVALID;
        else if (sv->outstanding >= sv->cfg.queue_capacity) bad = PD_ERR_QUEUE_FULL;
        if (bad != PD_OK) {
            delete r;
            return bad;
        }
        r->ticket = sv->next_ticket++;
        r->t_submit = now_ms();
        sv->live[r->ticket] = r;
        sv->outstanding++;
        sv->inflight[pi]++;
        sv->queue[pi].push_back(r);
        *ticket = r->ticket;
    }
    sv->cv_work[pi].notify_one();
    return PD_OK;
}

static pd_status take_result_locked(pd_server* sv, Req* r, pd_result* out) {
    if (out) {
        out->status = r->st;
        out->cost = r->best;
        out->centroid = r->kind == PD_Q_NEAREST ? r->best_c : -1;
        out->iters = r->max_iters;
        out->latency_ms = r->t_done - r->t_submit;
    }
    const pd_status st = r->st;
    sv->live.erase(r->ticket);
    sv->outstanding--;
    delete r;
    return st;
}

extern "C" pd_status pd_serve_poll(pd_server* sv, uint64_t ticket, pd_result* out) {
    if (!sv) return PD_ERR_INVALID;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->live.find(ticket);
    if (it == sv->live.end()) return PD_ERR_INVALID;
    if (!it->second->finished) return PD_PENDING;
    return take_result_locked(sv, it->second, out);
}

extern "C" pd_status pd_serve_wait(pd_server* sv, uint64_t ticket, pd_result* out, double timeout_ms) {
    if (!sv) return PD_ERR_INVALID;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->live.find(ticket);
    if (it == sv->live.end()) return PD_ERR_INVALID;
    Req* r = it->second;
    auto ready = [&] { return r->finished; };
    if (timeout_ms < 0) sv->cv_done.wait(lk, ready);
    else sv->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready);
    if (!r->finished) return PD_PENDING;
    return take_result_locked(sv, r, out);
}

extern "C" pd_status pd_serve_inject_failure(pd_server* sv) {
    if (!sv) return PD_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->inject = true;
    }
    for (auto& cv : sv->cv_work) cv.notify_all();
    return PD_OK;
}

extern "C" void pd_serve_destroy(pd_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    for (auto& cv : sv->cv_work) cv.notify_all();
    for (auto& w : sv->workers)
        if (w.joinable()) w.join();
    cudaSetDevice(sv->device);
    for (auto& P : sv->pools) pool_destroy(P);
    for (auto& kv : sv->live) delete kv.second;
    delete sv;
}
