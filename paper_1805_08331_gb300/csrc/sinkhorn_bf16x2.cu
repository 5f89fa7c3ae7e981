// sinkhorn_bf16x2.cu -- PD_BF16 iterations for grids up to 64: two pairs per
// CTA on the tensor cores.
//
// The arithmetic is that of sinkhorn_bf16.cu (absorbed-potential linear-domain
// separable products of Prop. 1, residual scalings FP32 in global memory):
//   u-update:  Wt[j,k] = sum_l K1u[j,l] (rs_u[k] vt[k,l]),  R[i,j] = sum_k K2u[i,k] Wt[j,k],
//              ut = a / (cf_u[j] R + KDu vt_Delta) on supp(a)
//   v-update:  Wv[l,i] = sum_j K1v[l,j] (rs_v[i] ut[i,j]),  S[k,l] = sum_i K2v[k,i] Wv[l,i],
//              vt = b / (cf_v[l] S + KDv ut_Delta) on supp(b), with err_t
// but with dp = 64 the two pairs of a CTA share every MMA: the A operand
// stacks pair 0's 64 rows over pair 1's (M = 128), the B operand likewise
// (N = 128), K = 64; each pair's product is a diagonal 64 x 64 block of the
// 128 x 128 FP32 accumulator in TMEM (the off-diagonal blocks are not read).
// Thread t owns TMEM lane t, i.e. row t & 63 of pair slot t >> 6; warps 0-1
// serve slot 0, warps 2-3 slot 1.  The four kernel factors of both pairs
// arrive by TMA (BF16 copies written after every absorption, 128-byte
// swizzle, one 64 x 64 box per factor and pair); the B operand is rebuilt in
// shared memory by the epilogue, eight BF16 values per 16-byte store.
#define T_CTA 256
#include "sk_common.cuh"
#include "tc_common.cuh"
#include <cuda.h>
#include <cudaTypedefs.h>

#define X2_THREADS 128
#define X2_TILE (128 * 64 * 2)   // 128 rows x 64 K-elements BF16, K-major SW128: 16 KB
#define X2_SMEM (5 * X2_TILE + 4 * 32 * 33 * 4 + 8 * 64 * 4 + 1024)

// Row r (0..127) of a 128 x 64 K-major SW128 tile from 64 FP32 values given in
// chunks of 32 (chunk ch), times `scale`, eight BF16 values per 16-byte store.
__device__ __forceinline__ void x2_store_chunk(unsigned char* tile, int r, int ch, const float* v, float scale) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k0 = ch * 32 + q * 8;
        uint4 u;
        u.x = pack_bf16x2_sat(v[q * 8 + 0] * scale, v[q * 8 + 1] * scale);
        u.y = pack_bf16x2_sat(v[q * 8 + 2] * scale, v[q * 8 + 3] * scale);
        u.z = pack_bf16x2_sat(v[q * 8 + 4] * scale, v[q * 8 + 5] * scale);
        u.w = pack_bf16x2_sat(v[q * 8 + 6] * scale, v[q * 8 + 7] * scale);
        *reinterpret_cast<uint4*>(tile + sw128_offset(r, k0, 128)) = u;
    }
}
__device__ __forceinline__ void x2_zero_row(unsigned char* tile, int r) {
#pragma unroll
    for (int k0 = 0; k0 < 64; k0 += 8) *reinterpret_cast<uint4*>(tile + sw128_offset(r, k0, 128)) = make_uint4(0, 0, 0, 0);
}
__device__ __forceinline__ void x2_store_one(unsigned char* tile, int r, int k, float v) {
    *reinterpret_cast<unsigned short*>(tile + sw128_offset(r, k, 128)) = (unsigned short)(pack_bf16x2_sat(v, 0.f) & 0xFFFFu);
}

// D (TMEM, 128 lanes x 128 FP32 columns) = A (128 x 64) * B (128 x 64)^T, four
// MMAs of K = 16, issued by one thread, committed to mbar.
__device__ __forceinline__ void x2_gemm_issue(uint32_t tmem_d, uint32_t sa, uint32_t sb, uint64_t* mbar) {
    constexpr uint32_t idesc = idesc_bf16_f32(128, 128);
#pragma unroll
    for (int s = 0; s < 4; ++s)
        mma_bf16(tmem_d, sw128_desc(sa + s * 32), sw128_desc(sb + s * 32), idesc, s > 0 ? 1u : 0u);
    mma_commit(mbar);
}

// Make the operand writes visible to the tensor core, issue, wait (bounded);
// returns false on a timed-out wait.  diag: no issue and a spin limit of 0
// (check of the timeout path: the wait gives up with nothing in flight).
__device__ __forceinline__ bool x2_run(uint32_t tmem, const unsigned char* A, const unsigned char* B, uint64_t* mbar,
                                       uint32_t& phase, bool diag) {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0 && !diag) x2_gemm_issue(tmem, smem_u32(A), smem_u32(B), mbar);
    const bool ok = __syncthreads_and(mbar_wait(mbar, phase, diag ? 0u : (1u << 26)) ? 1 : 0) != 0;
    phase ^= 1u;
    tc_fence_after();
    return ok;
}

// Thread t's accumulator columns of its slot: 64 values in two chunks of 32.
__device__ __forceinline__ uint32_t x2_taddr(uint32_t tm, int ch) {
    const int t = threadIdx.x, warp = t >> 5, slot = t >> 6;
    return tm + ((uint32_t)(warp * 32) << 16) + (uint32_t)(slot * 64 + ch * 32);
}

// Sum over the 64 threads of a slot (warps 2 slot, 2 slot + 1); sh: 4 floats.
__device__ __forceinline__ float x2_slot_sum(float v, float* sh) {
    v = warp_sum(v);
    const int warp = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[warp] = v;
    __syncthreads();
    const int s = warp >> 1;
    return sh[2 * s] + sh[2 * s + 1];
}

// TMA: load box (64 x 64 BF16, 128-byte swizzle) of 4-D tensor map coordinate
// (0, 0, factor, pair) into shared memory, completing on mbar.
__device__ __forceinline__ void x2_tma_load(uint32_t dst, const CUtensorMap* map, int factor, int pair, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(0), "r"(factor), "r"(pair), "r"(smem_u32(mbar))
        : "memory");
}
__device__ __forceinline__ void x2_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

// Pair slot state, one copy per slot in shared memory.
struct X2Slot {
    int p;              // pair index, -1: none
    int live;           // still iterating in this launch
    int status, absorb, iters, since, range;
    float utD, vtD, err;
};

__global__ void __launch_bounds__(X2_THREADS, 2)
sk_iter_bf16x2_kernel(SkWS w, SkRun r, int n_inner, int* active_count, int* error_flag,
                      const __grid_constant__ CUtensorMap fmap) {
    extern __shared__ unsigned char smraw[];
    __shared__ uint64_t mbar, tbar;
    __shared__ uint32_t tbase;
    __shared__ X2Slot S[2];
    __shared__ float shf[4];
    __shared__ int any_live;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31, slot = t >> 6, row = t & 63;
    const bool diag = r.diag_tc_timeout != 0;
    // ---- pairs of this CTA (launch order: two consecutive entries)
    if (t < 2) {
        const int e = 2 * blockIdx.x + t;
        int p = -1;
        if (e < w.P) p = w.order ? w.order[e] : e;
        if (p >= 0) {
            const int* ic = w.ic + (size_t)p * IC_N;
            if (ic[IC_STATUS] != ST_ACTIVE) p = -1;
            else if (ic[IC_ABSORB]) { atomicAdd(active_count, 1); p = -1; }   // absorbed first by the host
        }
        S[t].p = p;
        S[t].live = p >= 0;
    }
    __syncthreads();
    if (S[0].p < 0 && S[1].p < 0) return;
    const int dp = w.dp, d = w.d;
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* K1u = base;
    unsigned char* K2u = base + X2_TILE;
    unsigned char* K1v = base + 2 * X2_TILE;
    unsigned char* K2v = base + 3 * X2_TILE;
    unsigned char* X = base + 4 * X2_TILE;
    float* stage = reinterpret_cast<float*>(base + 5 * X2_TILE);           // [4 warps][32][33]
    float* vec = stage + 4 * 32 * 33;                                       // rs_u, cf_u, rs_v, cf_v: [2][64] each
    float* rs_u = vec;
    float* cf_u = vec + 128;
    float* rs_v = vec + 256;
    float* cf_v = vec + 384;
    const int p = S[slot].p;
    PairPtrs q = pair_ptrs(w, p < 0 ? 0 : p);
    // ---- prologue: the factors of both pairs by TMA, vectors, first B operand
    if (t == 0) { mbar_init(&mbar, 1); mbar_init(&tbar, 1); fence_mbar_init(); }
    if (warp == 0) tmem_alloc(&tbase, 128);
    __syncthreads();
    if (t == 0) {
        uint32_t bytes = 0;
        for (int s = 0; s < 2; ++s) if (S[s].p >= 0) bytes += 4u * 64u * 64u * 2u;
        x2_expect_tx(&tbar, bytes);
        unsigned char* tiles[4] = {K1u, K2u, K1v, K2v};
        for (int s = 0; s < 2; ++s) {
            if (S[s].p < 0) continue;
            for (int f = 0; f < 4; ++f) x2_tma_load(smem_u32(tiles[f] + s * 64 * 128), &fmap, f, S[s].p, &tbar);
        }
    }
    if (p < 0) {   // an empty slot: zero its rows of the factor tiles (no TMA wrote them)
        x2_zero_row(K1u, t); x2_zero_row(K2u, t); x2_zero_row(K1v, t); x2_zero_row(K2v, t);
    }
    rs_u[t] = p >= 0 && row < dp ? q.rs_u[row] : 0.f;
    cf_u[t] = p >= 0 && row < dp ? q.cf_u[row] : 0.f;
    rs_v[t] = p >= 0 && row < dp ? q.rs_v[row] : 0.f;
    cf_v[t] = p >= 0 && row < dp ? q.cf_v[row] : 0.f;
    // V'[k, l] = rs_u[k] vt[k, l]: thread (slot, k) builds row k of its slot
    x2_zero_row(X, t);
    __syncthreads();
    if (p >= 0 && row < d)
        for (int e = q.rpb[row]; e < q.rpb[row + 1]; ++e) { const int c = q.sb[e]; x2_store_one(X, t, c % dp, rs_u[t] * q.vt[c]); }
    // the factor copies must have landed before anything else (also under the
    // diagnostic, which only shortens the waits for MMAs)
    int timeout = 0;
    if (!__syncthreads_and(mbar_wait(&tbar, 0) ? 1 : 0)) timeout = 1;
    if (t < 2 && S[t].p >= 0) {
        const double* sc = w.sc + (size_t)S[t].p * SC_N;
        const int* ic = w.ic + (size_t)S[t].p * IC_N;
        S[t].utD = (float)sc[SC_UTD]; S[t].vtD = (float)sc[SC_VTD]; S[t].err = (float)sc[SC_ERR];
        S[t].iters = ic[IC_ITERS]; S[t].since = ic[IC_SINCE];
        S[t].status = ST_ACTIVE; S[t].absorb = 0; S[t].range = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = tbase;
    uint32_t phase = 0;
    const int na = p >= 0 ? q.ic[IC_NA] : 0, nb = p >= 0 ? q.ic[IC_NB] : 0;
    const float aD = p >= 0 ? (float)q.sc[SC_AD] : 0.f, bD = p >= 0 ? (float)q.sc[SC_BD] : 0.f;
    const float total = p >= 0 ? (float)q.sc[SC_TOTAL] : 1.f;
    const float DD = p >= 0 ? (float)q.sc[SC_DD] : 0.f, tau = p >= 0 ? (float)q.sc[SC_TAU] : 0.f;
    float* stg = stage + warp * 32 * 33;
    const int st = slot * 64;   // first thread of this slot
    for (int it = 0; it < n_inner && !timeout; ++it) {
        const bool live = S[slot].live != 0;   // read before this iteration's writes (barrier-separated)
        const float vtD = S[slot].vtD;
        // ================= u-update
        if (!x2_run(tm, K1u, X, &mbar, phase, diag)) { timeout = 1; break; }
        for (int ch = 0; ch < 2; ++ch) {                                   // Wt rows j
            float v[32];
            tmem_ld32(x2_taddr(tm, ch), v);
            x2_store_chunk(X, t, ch, v, live ? 1.f : 0.f);
        }
        float sKv = 0.f;                                                   // sum_y KDv vt (ut_Delta)
        if (live) for (int e = row; e < nb; e += 64) { const int c = q.sb[e]; sKv += q.KDv[c] * q.vt[c]; }
        sKv = x2_slot_sum(sKv, shf);
        if (!x2_run(tm, K2u, X, &mbar, phase, diag)) { timeout = 1; break; }
        {
            const int i = row;
            const float rsv = rs_v[t];
            const int e0 = live && i < d ? q.rpa[i] : 0, e1 = live && i < d ? q.rpa[i + 1] : 0;
            x2_zero_row(X, t);
            bool rng = false;
            for (int ch = 0; ch < 2; ++ch) {
                float v[32];
                tmem_ld32(x2_taddr(tm, ch), v);
#pragma unroll
                for (int u = 0; u < 32; ++u) stg[lane * 33 + u] = v[u];
                __syncwarp();
                for (int e = e0; e < e1; ++e) {
                    const int c = q.sa[e], j = c % dp;
                    if ((j >> 5) != ch) continue;
                    const float den = cf_u[st + j] * stg[lane * 33 + (j & 31)] + q.KDu[c] * vtD;
                    const float uu = q.am[c] / den;
                    const float lr = logf(uu / q.am[c]), lo = logf(uu * rsv);
                    if (!(fabsf(lr) <= tau) || !(fabsf(lo) <= 85.f)) rng = true;
                    q.ut[c] = uu;
                    x2_store_one(X, t, j, uu * rsv);
                }
                __syncwarp();
            }
            if (rng) S[slot].range = 1;
        }
        if (live && t == st) {
            const float utD_new = (aD > 0.f) ? aD / (sKv + DD * vtD) : 0.f;
            if (aD > 0.f && !(fabsf(logf(utD_new / aD)) <= tau)) S[slot].range = 1;
            S[slot].utD = utD_new;
        }
        __syncthreads();
        const float utD = S[slot].utD;
        // ================= v-update
        if (!x2_run(tm, K1v, X, &mbar, phase, diag)) { timeout = 1; break; }
        for (int ch = 0; ch < 2; ++ch) {                                   // Wv rows l
            float v[32];
            tmem_ld32(x2_taddr(tm, ch), v);
            x2_store_chunk(X, t, ch, v, live ? 1.f : 0.f);
        }
        float sKu = 0.f;                                                   // sum_x KDu ut (v_Delta)
        if (live) for (int e = row; e < na; e += 64) { const int c = q.sa[e]; sKu += q.KDu[c] * q.ut[c]; }
        sKu = x2_slot_sum(sKu, shf);
        if (!x2_run(tm, K2v, X, &mbar, phase, diag)) { timeout = 1; break; }
        float e_loc = 0.f;
        {
            const int k = row;
            const float rsu = rs_u[t];
            const int e0 = live && k < d ? q.rpb[k] : 0, e1 = live && k < d ? q.rpb[k + 1] : 0;
            x2_zero_row(X, t);
            bool rng = false;
            for (int ch = 0; ch < 2; ++ch) {
                float v[32];
                tmem_ld32(x2_taddr(tm, ch), v);
#pragma unroll
                for (int u = 0; u < 32; ++u) stg[lane * 33 + u] = v[u];
                __syncwarp();
                for (int e = e0; e < e1; ++e) {
                    const int c = q.sb[e], l = c % dp;
                    if ((l >> 5) != ch) continue;
                    const float qv = cf_v[st + l] * stg[lane * 33 + (l & 31)] + q.KDv[c] * utD;
                    e_loc += fabsf(q.vt[c] * qv - q.bm[c]);
                    const float vv = q.bm[c] / qv;
                    if (!(fabsf(logf(vv / q.bm[c])) <= tau) || !(fabsf(logf(vv * rsu)) <= 85.f)) rng = true;
                    q.vt[c] = vv;
                    x2_store_one(X, t, l, vv * rsu);
                }
                __syncwarp();
            }
            if (rng) S[slot].range = 1;
        }
        const float errs = x2_slot_sum(e_loc, shf);
        if (live && t == st) {
            X2Slot& Z = S[slot];
            float ee = errs;
            const float qD = sKu + DD * utD;
            if (bD > 0.f) {
                ee += fabsf(vtD * qD - bD);
                const float vv = bD / qD;
                if (!(fabsf(logf(vv / bD)) <= tau)) Z.range = 1;
                Z.vtD = vv;
            }
            Z.err = ee / total;
            ++Z.iters; ++Z.since;
            if (!isfinite(Z.err)) { Z.absorb = 1; Z.live = 0; }
            else if (r.tol > 0 && Z.err <= r.tol) { Z.status = ST_CONVERGED; Z.live = 0; }
            else if (Z.iters >= r.max_iter) { Z.status = ST_MAXITER; Z.live = 0; }
            else if (Z.range || Z.since >= r.absorb_every) { Z.absorb = 1; Z.live = 0; }
        }
        if (t == 0) any_live = 0;
        __syncthreads();
        if (t < 2 && S[t].live) any_live = 1;
        __syncthreads();
        if (!any_live) break;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tm, 128);
    if (t < 2 && S[t].p >= 0) {
        X2Slot& Z = S[t];
        const int pp = Z.p;
        double* sc = w.sc + (size_t)pp * SC_N;
        int* ic = w.ic + (size_t)pp * IC_N;
        if (timeout) { atomicExch(error_flag, 1); ic[IC_STATUS] = ST_RANGE; return; }
        sc[SC_UTD] = Z.utD; sc[SC_VTD] = Z.vtD; sc[SC_ERR] = Z.err;
        ic[IC_ITERS] = Z.iters; ic[IC_SINCE] = Z.since;
        if (Z.status != ST_ACTIVE) ic[IC_STATUS] = Z.status;
        if (Z.absorb) {
            if (Z.range && Z.since == 1) ic[IC_RANGE] += 1; else ic[IC_RANGE] = 0;
            if (ic[IC_RANGE] >= 2 || !isfinite(Z.err)) ic[IC_STATUS] = ST_RANGE;
            else ic[IC_ABSORB] = 1;
        }
        if (ic[IC_STATUS] == ST_ACTIVE) atomicAdd(active_count, 1);
    }
}

// BF16 copies of the four absorbed kernel factors of every active pair, laid
// out for the tensor map: pair p's factor f (0..3: K1u, K2u, K1v, K2v) row r,
// column k at bf[p * (16 dp^2 / 2) + f * dp^2 + r * dp + k] (the pair's FP64
// scratch holds them; dp = 64).
__global__ void sk_factors_bf16_kernel(SkWS w, unsigned short* __restrict__ bf) {
    const int p = blockIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    if (q.ic[IC_STATUS] != ST_ACTIVE) return;
    const int M = w.dp * w.dp;
    unsigned short* o = bf + (size_t)p * 8 * M;
    const float* src[4] = {q.K1u, q.K2u, q.K1v, q.K2v};
    for (int f = 0; f < 4; ++f)
        for (int x = threadIdx.x * 2; x < M; x += blockDim.x * 2) {
            const uint32_t v = pack_bf16x2_sat(src[f][x], src[f][x + 1]);
            *reinterpret_cast<uint32_t*>(o + (size_t)f * M + x) = v;
        }
}

static PFN_cuTensorMapEncodeTiled_v12000 x2_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

// True when the two-pairs-per-CTA kernel serves this workspace (dp = 64).
bool sk_bf16x2_applies(const SkWS& w) { return w.dp == 64; }

cudaError_t sk_launch_iter_bf16x2(const SkWS& w, SkRun r, int n_inner, int* active_count, int* error_flag,
                                  cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    if (w.dp != 64) return cudaErrorInvalidValue;
    unsigned short* bf = reinterpret_cast<unsigned short*>(w.L64);
    sk_factors_bf16_kernel<<<w.P, 256, 0, s>>>(w, bf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    PFN_cuTensorMapEncodeTiled_v12000 enc = x2_encoder();
    if (!enc) return cudaErrorNotSupported;
    // 4-D view of the copies: (k, row, factor, pair), pair stride = the pair's
    // FP64 scratch (2 dp^2 doubles = 65536 bytes at dp = 64)
    CUtensorMap map;
    const cuuint64_t dims[4] = {64, 64, 4, (cuuint64_t)w.P};
    const cuuint64_t strides[3] = {64 * 2, 64 * 64 * 2, (cuuint64_t)2 * 64 * 64 * 8};
    const cuuint32_t box[4] = {64, 64, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, bf, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    static bool configured = false;
    if (!configured) {
        e = cudaFuncSetAttribute(sk_iter_bf16x2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, X2_SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    sk_iter_bf16x2_kernel<<<(w.P + 1) / 2, X2_THREADS, X2_SMEM, s>>>(w, r, n_inner, active_count, error_flag, map);
    return cudaGetLastError();
}
