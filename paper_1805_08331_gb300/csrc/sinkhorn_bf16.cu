// sinkhorn_bf16.cu -- Sinkhorn iterations with the separable kernel applied by
// tcgen05 tensor-core GEMMs (BF16 operands, FP32 accumulation in TMEM).
//
// Same absorbed-potential representation as sinkhorn_fp32.cu (rank-one
// separable absorbed potentials keep the absorbed kernel a Kronecker product,
// residual scalings FP32 in global memory), with every product of Prop. 1
// written as a 128 x 128 x 128 GEMM on the tensor cores, each arranged so that
// the accumulator row a thread reads from TMEM is the contiguous K-major
// operand row of the next GEMM:
//   u-update:  Wt[j,k] = sum_l K1u[j,l] (rs_u[k] vt[k,l])      (A = K1u,  B = V')
//              R[i,j]  = sum_k K2u[i,k] Wt[j,k]                 (A = K2u,  B = Wt)
//              ut      = a / (cf_u[j] R + KDu vt_Delta)          on supp(a)
//   v-update:  Wv[l,i] = sum_j K1v[l,j] (rs_v[i] ut[i,j])      (A = K1v,  B = U')
//              S[k,l]  = sum_i K2v[k,i] Wv[l,i]                 (A = K2v,  B = Wv)
//              vt      = b / (cf_v[l] S + KDv ut_Delta)          on supp(b), with err_t
// One CTA (4 warps, warp w owns TMEM lanes 32w..32w+31) per pair; the four
// kernel factors stay in shared memory (4 x 32 KB BF16, 128B-swizzled K-major)
// for the whole launch, the B operand is rebuilt in place after each GEMM.
// Grids up to d = 128 (smaller d is zero-padded to 128).
#define T_CTA 256
#include "sk_common.cuh"
#include "tc_common.cuh"

#define BF_THREADS 128
#define TILE_BYTES (128 * 128 * 2)
#define BF_SMEM (5 * TILE_BYTES + 4 * 128 * 4 + 4 * 32 * 33 * 4 + 1024)

// Write row r of a K-major SW128 operand tile from 128 FP32 values given in
// chunks of 32 (chunk index ch), scaled by `scale` (BF16, saturating).
__device__ __forceinline__ void store_row_chunk(unsigned char* tile, int r, int ch, const float* v, float scale) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {   // four 16-byte pieces of 8 elements
        const int k0 = ch * 32 + q * 8;
        uint4 w;
        w.x = pack_bf16x2_sat(v[q * 8 + 0] * scale, v[q * 8 + 1] * scale);
        w.y = pack_bf16x2_sat(v[q * 8 + 2] * scale, v[q * 8 + 3] * scale);
        w.z = pack_bf16x2_sat(v[q * 8 + 4] * scale, v[q * 8 + 5] * scale);
        w.w = pack_bf16x2_sat(v[q * 8 + 6] * scale, v[q * 8 + 7] * scale);
        *reinterpret_cast<uint4*>(tile + sw128_offset(r, k0, 128)) = w;
    }
}
__device__ __forceinline__ void zero_row(unsigned char* tile, int r) {
#pragma unroll
    for (int k0 = 0; k0 < 128; k0 += 8) *reinterpret_cast<uint4*>(tile + sw128_offset(r, k0, 128)) = make_uint4(0, 0, 0, 0);
}
__device__ __forceinline__ void store_bf16(unsigned char* tile, int r, int k, float v) {
    *reinterpret_cast<unsigned short*>(tile + sw128_offset(r, k, 128)) = (unsigned short)(pack_bf16x2_sat(v, 0.f) & 0xFFFFu);
}

// Load one dp x dp FP32 kernel factor from global into a 128 x 128 BF16 tile
// (thread t converts row t; rows / columns beyond dp are zero).
__device__ void load_factor(unsigned char* tile, const float* __restrict__ src, int dp) {
    const int r = threadIdx.x;
    if (r >= dp) { zero_row(tile, r); return; }
    for (int ch = 0; ch < 4; ++ch) {
        float v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int k = ch * 32 + i;
            v[i] = k < dp ? src[(size_t)r * dp + k] : 0.f;
        }
        store_row_chunk(tile, r, ch, v, 1.f);
    }
}

struct BfShared {
    unsigned char *K1u, *K2u, *K1v, *K2v, *X;
    float *rs_u, *cf_u, *rs_v, *cf_v;
    float* stage;   // [4 warps][32][33] staging of TMEM chunks
};

// Issue one GEMM (thread 0) after making the operand writes visible, then wait
// for it; returns false on a timed-out wait.  diag (a check of the timeout
// path): the GEMM is not issued and the wait has a spin limit of 0, so it
// gives up at once with no tensor-core work in flight.
__device__ __forceinline__ bool run_gemm(uint32_t tmem, const unsigned char* A, const unsigned char* B, uint64_t* mbar,
                                         uint32_t& phase, bool diag) {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0 && !diag) gemm128_issue(tmem, smem_u32(A), smem_u32(B), mbar);
    const bool ok = __syncthreads_and(mbar_wait(mbar, phase, diag ? 0u : (1u << 26)) ? 1 : 0) != 0;   // same path for all
    phase ^= 1u;
    tc_fence_after();
    return ok;
}

// Dense epilogue: thread j copies its accumulator row into operand row j (BF16).
__device__ __forceinline__ void epi_dense(uint32_t tmem, unsigned char* X) {
    const int t = threadIdx.x, warp = t >> 5;
    for (int ch = 0; ch < 4; ++ch) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + ch * 32, v);
        store_row_chunk(X, t, ch, v, 1.f);
    }
}

__global__ void __launch_bounds__(BF_THREADS) sk_iter_bf16_kernel(SkWS w, SkRun r, int n_inner, int* active_count,
                                                                   int* error_flag) {
    extern __shared__ unsigned char smraw[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase;
    __shared__ int range_sh;
    __shared__ float shf[32];
    const int p = blockIdx.x, t = threadIdx.x, warp = t >> 5, lane = t & 31;
    PairPtrs q = pair_ptrs(w, p);
    if (q.ic[IC_STATUS] != ST_ACTIVE) return;
    if (q.ic[IC_ABSORB]) { if (t == 0) atomicAdd(active_count, 1); return; }
    const int d = w.d, dp = w.dp;
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    BfShared S;
    S.K1u = base; S.K2u = base + TILE_BYTES; S.K1v = base + 2 * TILE_BYTES; S.K2v = base + 3 * TILE_BYTES;
    S.X = base + 4 * TILE_BYTES;
    S.rs_u = reinterpret_cast<float*>(base + 5 * TILE_BYTES);
    S.cf_u = S.rs_u + 128; S.rs_v = S.cf_u + 128; S.cf_v = S.rs_v + 128;
    S.stage = S.cf_v + 128;
    // ---- prologue: kernel factors and vectors into shared memory, first B operand
    load_factor(S.K1u, q.K1u, dp);
    load_factor(S.K2u, q.K2u, dp);
    load_factor(S.K1v, q.K1v, dp);
    load_factor(S.K2v, q.K2v, dp);
    S.rs_u[t] = t < dp ? q.rs_u[t] : 0.f;
    S.cf_u[t] = t < dp ? q.cf_u[t] : 0.f;
    S.rs_v[t] = t < dp ? q.rs_v[t] : 0.f;
    S.cf_v[t] = t < dp ? q.cf_v[t] : 0.f;
    if (warp == 0) tmem_alloc(&tbase, 128);
    if (t == 0) { mbar_init(&mbar, 1); fence_mbar_init(); range_sh = 0; }
    __syncthreads();
    // V'[k, l] = rs_u[k] vt[k, l]: thread k builds row k
    zero_row(S.X, t);
    if (t < d) for (int e = q.rpb[t]; e < q.rpb[t + 1]; ++e) { int c = q.sb[e]; store_bf16(S.X, t, c % dp, S.rs_u[t] * q.vt[c]); }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = tbase;
    uint32_t phase = 0;
    const int na = q.ic[IC_NA], nb = q.ic[IC_NB];
    const float aD = (float)q.sc[SC_AD], bD = (float)q.sc[SC_BD], total = (float)q.sc[SC_TOTAL];
    const float DD = (float)q.sc[SC_DD], tau = (float)q.sc[SC_TAU];
    float utD = (float)q.sc[SC_UTD], vtD = (float)q.sc[SC_VTD];
    int iters = q.ic[IC_ITERS], since = q.ic[IC_SINCE];
    int status = ST_ACTIVE, absorb = 0, timeout = 0;
    float err = (float)q.sc[SC_ERR];
    float* stg = S.stage + warp * 32 * 33;
    for (int it = 0; it < n_inner; ++it) {
        // ================= u-update
        if (!run_gemm(tm, S.K1u, S.X, &mbar, phase, r.diag_tc_timeout != 0)) { timeout = 1; break; }
        epi_dense(tm, S.X);                                            // Wt rows j
        float sKv = 0.f;                                               // sum_y KDv vt (for ut_Delta)
        for (int e = t; e < nb; e += BF_THREADS) { int c = q.sb[e]; sKv += q.KDv[c] * q.vt[c]; }
        sKv = block_sum(sKv, shf);
        if (!run_gemm(tm, S.K2u, S.X, &mbar, phase, r.diag_tc_timeout != 0)) { timeout = 1; break; }
        // R rows i: ut on supp(a) row i, then U' row i = rs_v[i] ut[i, :]
        {
            const int i = t;
            const float rsv = S.rs_v[i];
            const int e0 = i < d ? q.rpa[i] : 0, e1 = i < d ? q.rpa[i + 1] : 0;
            zero_row(S.X, i);
            for (int ch = 0; ch < 4; ++ch) {
                float v[32];
                tmem_ld32(tm + ((uint32_t)(warp * 32) << 16) + ch * 32, v);
#pragma unroll
                for (int u = 0; u < 32; ++u) stg[lane * 33 + u] = v[u];
                __syncwarp();
                for (int e = e0; e < e1; ++e) {
                    const int c = q.sa[e], j = c % dp;
                    if ((j >> 5) != ch) continue;
                    const float den = S.cf_u[j] * stg[lane * 33 + (j & 31)] + q.KDu[c] * vtD;
                    const float uu = q.am[c] / den;
                    const float lr = logf(uu / q.am[c]), lo = logf(uu * rsv);
                    if (!(fabsf(lr) <= tau) || !(fabsf(lo) <= 85.f)) range_sh = 1;
                    q.ut[c] = uu;
                    store_bf16(S.X, i, j, uu * rsv);
                }
                __syncwarp();
            }
        }
        const float utD_new = (aD > 0.f) ? aD / (sKv + DD * vtD) : 0.f;
        if (aD > 0.f && !(fabsf(logf(utD_new / aD)) <= tau)) range_sh = 1;
        utD = utD_new;
        // ================= v-update
        if (!run_gemm(tm, S.K1v, S.X, &mbar, phase, r.diag_tc_timeout != 0)) { timeout = 1; break; }
        epi_dense(tm, S.X);                                            // Wv rows l
        float sKu = 0.f;                                               // sum_x KDu ut (for v_Delta)
        for (int e = t; e < na; e += BF_THREADS) { int c = q.sa[e]; sKu += q.KDu[c] * q.ut[c]; }
        sKu = block_sum(sKu, shf);
        if (!run_gemm(tm, S.K2v, S.X, &mbar, phase, r.diag_tc_timeout != 0)) { timeout = 1; break; }
        float e_loc = 0.f;
        {
            const int k = t;
            const float rsu = S.rs_u[k];
            const int e0 = k < d ? q.rpb[k] : 0, e1 = k < d ? q.rpb[k + 1] : 0;
            zero_row(S.X, k);
            for (int ch = 0; ch < 4; ++ch) {
                float v[32];
                tmem_ld32(tm + ((uint32_t)(warp * 32) << 16) + ch * 32, v);
#pragma unroll
                for (int u = 0; u < 32; ++u) stg[lane * 33 + u] = v[u];
                __syncwarp();
                for (int e = e0; e < e1; ++e) {
                    const int c = q.sb[e], l = c % dp;
                    if ((l >> 5) != ch) continue;
                    const float qv = S.cf_v[l] * stg[lane * 33 + (l & 31)] + q.KDv[c] * utD;
                    e_loc += fabsf(q.vt[c] * qv - q.bm[c]);
                    const float vv = q.bm[c] / qv;
                    if (!(fabsf(logf(vv / q.bm[c])) <= tau) || !(fabsf(logf(vv * rsu)) <= 85.f)) range_sh = 1;
                    q.vt[c] = vv;
                    store_bf16(S.X, k, l, vv * rsu);
                }
                __syncwarp();
            }
        }
        float errs = block_sum(e_loc, shf);
        const float qD = sKu + DD * utD;
        if (bD > 0.f) {
            errs += fabsf(vtD * qD - bD);
            const float vv = bD / qD;
            if (!(fabsf(logf(vv / bD)) <= tau)) range_sh = 1;
            vtD = vv;
        }
        err = errs / total;
        ++iters; ++since;
        __syncthreads();
        const int rng = range_sh;
        if (!isfinite(err)) { absorb = 1; break; }
        if (r.tol > 0 && err <= r.tol) { status = ST_CONVERGED; break; }
        if (iters >= r.max_iter) { status = ST_MAXITER; break; }
        if (rng || since >= r.absorb_every) { absorb = 1; break; }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tm, 128);
    if (t == 0) {
        if (timeout) { atomicExch(error_flag, 1); q.ic[IC_STATUS] = ST_RANGE; return; }
        q.sc[SC_UTD] = utD; q.sc[SC_VTD] = vtD; q.sc[SC_ERR] = err;
        q.ic[IC_ITERS] = iters; q.ic[IC_SINCE] = since;
        if (status != ST_ACTIVE) q.ic[IC_STATUS] = status;
        if (absorb) {
            if (range_sh && since == 1) q.ic[IC_RANGE] += 1; else q.ic[IC_RANGE] = 0;
            if (q.ic[IC_RANGE] >= 2 || !isfinite(err)) q.ic[IC_STATUS] = ST_RANGE;
            else q.ic[IC_ABSORB] = 1;
        }
        if (q.ic[IC_STATUS] == ST_ACTIVE) atomicAdd(active_count, 1);
    }
}

cudaError_t sk_launch_iter_bf16(const SkWS& w, SkRun r, int n_inner, int* active_count, int* error_flag,
                                cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(sk_iter_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, BF_SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    sk_iter_bf16_kernel<<<w.P, BF_THREADS, BF_SMEM, s>>>(w, r, n_inner, active_count, error_flag);
    return cudaGetLastError();
}

// Potentials from the residual representation (after a linear-domain phase):
// phi = Fb + log(ut / a), psi = Gb + log(vt / b) on the supports, in FP64, and
// every pair that did not fail is made active again (refinement).
__global__ void sk_rebuild_potentials_kernel(SkWS w) {
    const int p = blockIdx.x, t = threadIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    const int st = q.ic[IC_STATUS];
    if (st == ST_INVALID || (st == ST_CONVERGED && q.sc[SC_TOTAL] == 0)) return;
    if (q.ic[IC_ABSORB] && !q.ic[IC_FROMLIN]) return;   // potentials already current (log step only)
    const int dp = w.dp, na = q.ic[IC_NA], nb = q.ic[IC_NB];
    // a value that is not finite (a pair that left the range) keeps the
    // potential of the last absorption, which is always finite
    for (int e = t; e < na; e += blockDim.x) {
        int c = q.sa[e];
        double v = (q.ap[c / dp] + q.bp[c % dp]) + (double)logf(q.ut[c] / q.am[c]);
        if (isfinite(v)) q.phi[c] = v;
    }
    for (int e = t; e < nb; e += blockDim.x) {
        int c = q.sb[e];
        double v = (q.al[c / dp] + q.be[c % dp]) + (double)logf(q.vt[c] / q.bm[c]);
        if (isfinite(v)) q.psi[c] = v;
    }
    if (t == 0) {
        const double aD = q.sc[SC_AD], bD = q.sc[SC_BD];
        double v1 = aD > 0 ? q.sc[SC_FD] + log(q.sc[SC_UTD] / aD) : NAN;
        double v2 = bD > 0 ? q.sc[SC_GD] + log(q.sc[SC_VTD] / bD) : NAN;
        if (isfinite(v1)) q.phi[w.n - 1] = v1;
        if (isfinite(v2)) q.psi[w.n - 1] = v2;
    }
}

__global__ void sk_reactivate_kernel(SkWS w) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.P) return;
    int* ic = w.ic + (size_t)p * IC_N;
    const int st = ic[IC_STATUS];
    if (st == ST_INVALID) return;
    if (st == ST_CONVERGED && w.sc[(size_t)p * SC_N + SC_TOTAL] == 0) return;
    ic[IC_STATUS] = ST_ACTIVE;
    ic[IC_BIG] = 0;
}

cudaError_t sk_launch_rebuild_potentials(const SkWS& w, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_rebuild_potentials_kernel<<<w.P, 256, 0, s>>>(w);
    return cudaGetLastError();
}

// Range check of the linear-domain engines: row / col hold the exact
// (log-domain) marginals of every pair's final plan, [P][d*d+1] each; a pair
// reported PD_OK whose exact marginal error (both sides, relative to the total
// mass) exceeds thr is reported PD_ERR_RANGE instead (its representation
// dropped terms that matter).
__global__ void sk_range_check_kernel(SkWS w, const float* __restrict__ row, const float* __restrict__ col,
                                      int32_t* __restrict__ status, float* __restrict__ err, double thr) {
    __shared__ double sh[32];
    const int p = blockIdx.x;
    if (status[p] != 0) return;
    PairPtrs q = pair_ptrs(w, p);
    const int d = w.d, dp = w.dp, n = d * d + 1;   // marginal rows of d*d + 1 entries, Delta last
    const float* rp = row + (size_t)p * n;
    const float* cp = col + (size_t)p * n;
    double e = 0.0;
    for (int x = threadIdx.x; x < d * d; x += blockDim.x) {
        const int i = x / d, j = x - i * d;
        e += fabs((double)rp[x] - (double)q.am[i * dp + j]) + fabs((double)cp[x] - (double)q.bm[i * dp + j]);
    }
    if (threadIdx.x == 0) e += fabs((double)rp[n - 1] - q.sc[SC_AD]) + fabs((double)cp[n - 1] - q.sc[SC_BD]);
    e = block_sum(e, sh);
    if (threadIdx.x == 0 && q.sc[SC_TOTAL] > 0 && !(e / q.sc[SC_TOTAL] <= thr)) {
        status[p] = 8;   // PD_ERR_RANGE; err reports the exact marginal error found
        if (err) err[p] = (float)(e / q.sc[SC_TOTAL]);
    }
}

cudaError_t sk_launch_range_check(const SkWS& w, const float* row, const float* col, int32_t* status, float* err,
                                  double thr, cudaStream_t s) {
    if (w.P == 0 || !status) return cudaSuccess;
    sk_range_check_kernel<<<w.P, 256, 0, s>>>(w, row, col, status, err, thr);
    return cudaGetLastError();
}

cudaError_t sk_launch_refine_prep(const SkWS& w, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_rebuild_potentials_kernel<<<w.P, 256, 0, s>>>(w);
    sk_reactivate_kernel<<<(w.P + 255) / 256, 256, 0, s>>>(w);
    return cudaGetLastError();
}
