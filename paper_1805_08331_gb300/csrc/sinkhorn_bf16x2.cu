// sinkhorn_bf16x2.cu -- PD_BF16 iterations for grids up to 64: two pairs per
// CTA on the tensor cores, operands split into BF16 hi + lo parts.
//
// The arithmetic is that of sinkhorn_bf16.cu (absorbed-potential linear-domain
// separable products of Prop. 1, residual scalings FP32 in global memory):
//   u-update:  Wt[j,k] = sum_l K1u[j,l] (rs_u[k] vt[k,l]),  R[i,j] = sum_k K2u[i,k] Wt[j,k],
//              ut = a / (cf_u[j] R + KDu vt_Delta) on supp(a)
//   v-update:  Wv[l,i] = sum_j K1v[l,j] (rs_v[i] ut[i,j]),  S[k,l] = sum_i K2v[k,i] Wv[l,i],
//              vt = b / (cf_v[l] S + KDv ut_Delta) on supp(b), with err_t
// with dp = 64 the two pairs of a CTA share every MMA: the A operand stacks
// pair 0's 64 rows over pair 1's (M = 128), the B operand likewise (N = 128),
// K = 64; each pair's product is a diagonal 64 x 64 block of the 128 x 128
// FP32 accumulator in TMEM (the off-diagonal blocks are not read).  Every
// operand is held as BF16 hi + lo (x = hi + lo to ~16 bits) and each product
// is Ah Bh + Ah Bl + Al Bh, accumulated in FP32: a single BF16 rounding of
// the operands leaves a marginal-error floor near 1e-4, the split form reaches
// the 1e-6 tolerance (host prototype against the FP64 oracle), and the MMA
// work it adds is small beside the epilogue.  TMEM lane l is row l & 63 of
// pair slot l >> 6; warps w and w + 4 read the same lanes, columns 0-31 and
// 32-63 of the slot.  The factors arrive by TMA (hi / lo BF16 copies written
// after every absorption, 128-byte swizzle, one 64 x 64 box per part and
// pair, this GPU's own memory, no multicast); the B operand is rebuilt in
// shared memory by the epilogue, eight BF16 values per 16-byte store.
#define T_CTA 256
#include "sk_common.cuh"
#include "tc_common.cuh"
#include <cuda.h>
#include <cudaTypedefs.h>

#define X2_THREADS 256
#define X2_TILE (128 * 64 * 2)   // 128 rows x 64 K-elements BF16, K-major SW128: 16 KB
// 8 factor tiles (hi, lo of four factors), 2 operand tiles (hi, lo), staging
// [8 warps][32][33] floats, vectors [4][128] floats, alignment slack
#define X2_SMEM (10 * X2_TILE + 8 * 32 * 33 * 4 + 4 * 128 * 4 + 1024)
// a pair leaves the tensor-core phase (for the exact refinement) once
// X2_STALL iterations have not lowered its marginal error by 5 %
#define X2_STALL 256

// hi + lo BF16 split of two FP32 values (hi = RN(x), lo = RN(x - hi)): the
// pair represents x to ~16 significant bits.
__device__ __forceinline__ void x2_split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    hi = pack_bf16x2_sat(a, b);
    const float ah = __uint_as_float(hi << 16), bh = __uint_as_float(hi & 0xFFFF0000u);
    lo = pack_bf16x2_sat(a - ah, b - bh);
}

// Chunk h (32 K-elements) of row r of the hi and lo operand tiles from 32 FP32
// values times `scale`, eight BF16 values per 16-byte store.
__device__ __forceinline__ void x2_store_chunk(unsigned char* thi, unsigned char* tlo, int r, int h, const float* v,
                                               float scale) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k0 = h * 32 + q * 8;
        uint4 uh, ul;
        x2_split2(v[q * 8 + 0] * scale, v[q * 8 + 1] * scale, uh.x, ul.x);
        x2_split2(v[q * 8 + 2] * scale, v[q * 8 + 3] * scale, uh.y, ul.y);
        x2_split2(v[q * 8 + 4] * scale, v[q * 8 + 5] * scale, uh.z, ul.z);
        x2_split2(v[q * 8 + 6] * scale, v[q * 8 + 7] * scale, uh.w, ul.w);
        *reinterpret_cast<uint4*>(thi + sw128_offset(r, k0, 128)) = uh;
        *reinterpret_cast<uint4*>(tlo + sw128_offset(r, k0, 128)) = ul;
    }
}
// zero chunk h of row r (both tiles); h = -1: the whole row
__device__ __forceinline__ void x2_zero(unsigned char* thi, unsigned char* tlo, int r, int h) {
    const int k_lo = h < 0 ? 0 : h * 32, k_hi = h < 0 ? 64 : h * 32 + 32;
    for (int k0 = k_lo; k0 < k_hi; k0 += 8) {
        *reinterpret_cast<uint4*>(thi + sw128_offset(r, k0, 128)) = make_uint4(0, 0, 0, 0);
        *reinterpret_cast<uint4*>(tlo + sw128_offset(r, k0, 128)) = make_uint4(0, 0, 0, 0);
    }
}
__device__ __forceinline__ void x2_store_one(unsigned char* thi, unsigned char* tlo, int r, int k, float v) {
    uint32_t hi, lo;
    x2_split2(v, 0.f, hi, lo);
    *reinterpret_cast<unsigned short*>(thi + sw128_offset(r, k, 128)) = (unsigned short)(hi & 0xFFFFu);
    *reinterpret_cast<unsigned short*>(tlo + sw128_offset(r, k, 128)) = (unsigned short)(lo & 0xFFFFu);
}

// D (TMEM, 128 lanes x 128 FP32 columns) = A (128 x 64) * B (128 x 64)^T with
// A = Ah + Al, B = Bh + Bl: Ah Bh + Ah Bl + Al Bh (the Al Bl term, ~2^-16 of
// the product, is dropped), 3 x 4 MMAs of K = 16 into one accumulator, issued
// by one thread, committed to mbar.
__device__ __forceinline__ void x2_gemm_issue(uint32_t tmem_d, uint32_t ah, uint32_t al, uint32_t bh, uint32_t bl,
                                              uint64_t* mbar) {
    constexpr uint32_t idesc = idesc_bf16_f32(128, 128);
    const uint32_t as[3] = {ah, ah, al}, bs[3] = {bh, bl, bh};
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
        for (int s = 0; s < 4; ++s)
            mma_bf16(tmem_d, sw128_desc(as[m] + s * 32), sw128_desc(bs[m] + s * 32), idesc, (m | s) ? 1u : 0u);
    mma_commit(mbar);
}

// Make the operand writes visible to the tensor core, issue, wait (bounded);
// returns false on a timed-out wait.  diag: no issue and a spin limit of 0
// (check of the timeout path: the wait gives up with nothing in flight).
__device__ __forceinline__ bool x2_run(uint32_t tmem, const unsigned char* const* A, const unsigned char* const* B,
                                       uint64_t* mbar, uint32_t& phase, bool diag) {
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0 && !diag)
        x2_gemm_issue(tmem, smem_u32(A[0]), smem_u32(A[1]), smem_u32(B[0]), smem_u32(B[1]), mbar);
    const bool ok = __syncthreads_and(mbar_wait(mbar, phase, diag ? 0u : (1u << 26)) ? 1 : 0) != 0;
    phase ^= 1u;
    tc_fence_after();
    return ok;
}

// TMEM address of thread t's accumulator chunk: its lane (t & 127), columns
// slot * 64 + half * 32 .. + 31 (warps w and w + 4 share lanes, one chunk each).
__device__ __forceinline__ uint32_t x2_taddr(uint32_t tm) {
    const int t = threadIdx.x, lr = t & 127, slot = lr >> 6, half = t >> 7;
    return tm + ((uint32_t)((lr >> 5) * 32) << 16) + (uint32_t)(slot * 64 + half * 32);
}

// Sum over the 128 threads of a slot (warps 2s, 2s + 1, 2s + 4, 2s + 5); sh: 8 floats.
__device__ __forceinline__ float x2_slot_sum(float v, float* sh) {
    v = warp_sum(v);
    const int warp = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[warp] = v;
    __syncthreads();
    const int s = (warp & 3) >> 1;
    return (sh[2 * s] + sh[2 * s + 1]) + (sh[2 * s + 4] + sh[2 * s + 5]);
}

// Two sums over the 128 threads of a slot at once; sh: 8 float2.
__device__ __forceinline__ float2 x2_slot_sum2(float a, float b, float2* sh) {
    a = warp_sum(a);
    b = warp_sum(b);
    const int warp = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[warp] = make_float2(a, b);
    __syncthreads();
    const int s = (warp & 3) >> 1;
    const float2 p0 = sh[2 * s], p1 = sh[2 * s + 1], p4 = sh[2 * s + 4], p5 = sh[2 * s + 5];
    return make_float2((p0.x + p1.x) + (p4.x + p5.x), (p0.y + p1.y) + (p4.y + p5.y));
}

// TMA: load box (64 x 64 BF16, 128-byte swizzle) of 4-D tensor map coordinate
// (0, 0, part, pair) into shared memory, completing on mbar.
__device__ __forceinline__ void x2_tma_load(uint32_t dst, const CUtensorMap* map, int part, int pair, uint64_t* mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(0), "r"(part), "r"(pair), "r"(smem_u32(mbar))
        : "memory");
}
__device__ __forceinline__ void x2_expect_tx(uint64_t* mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes) : "memory");
}

// First thread of a slot.
__device__ __forceinline__ int st0(int slot) { return slot * 64; }

// Pair slot state, one copy per slot in shared memory.
struct X2Slot {
    int p;              // pair index, -1: none
    int live;           // still iterating in this launch
    int status, absorb, iters, since, range, stall;
    float utD, vtD, err, best;
    float sKv, sKu;     // sum_y KDv vt and sum_x KDu ut of the current scalings (Delta updates)
};

// |log x| <= lim without a logarithm: e^-lim <= x <= e^lim (false for NaN)
__device__ __forceinline__ bool x2_in(float x, float elim, float einv) { return x >= einv && x <= elim; }

__global__ void __launch_bounds__(X2_THREADS, 1)
sk_iter_bf16x2_kernel(SkWS w, SkRun r, int n_inner, int* active_count, int* error_flag,
                      const __grid_constant__ CUtensorMap fmap) {
    extern __shared__ unsigned char smraw[];
    __shared__ uint64_t mbar, tbar;
    __shared__ uint32_t tbase;
    __shared__ X2Slot S[2];
    __shared__ float shf[8];
    __shared__ float2 shf2[8];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int lr = t & 127, slot = lr >> 6, row = lr & 63, half = t >> 7;
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
    // factor f (0..3: K1u, K2u, K1v, K2v), part h (0 hi, 1 lo) at base + (2 f + h) tiles
    unsigned char* F[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) F[k] = base + k * X2_TILE;
    unsigned char* X[2] = {base + 8 * X2_TILE, base + 9 * X2_TILE};
    float* stage = reinterpret_cast<float*>(base + 10 * X2_TILE);          // [8 warps][32][33]
    float* vec = stage + 8 * 32 * 33;                                       // rs_u, cf_u, rs_v, cf_v: [2][64] each
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
        for (int s = 0; s < 2; ++s) if (S[s].p >= 0) bytes += 8u * 64u * 64u * 2u;
        x2_expect_tx(&tbar, bytes);
        for (int s = 0; s < 2; ++s) {
            if (S[s].p < 0) continue;
            for (int k = 0; k < 8; ++k) x2_tma_load(smem_u32(F[k] + s * 64 * 128), &fmap, k, S[s].p, &tbar);
        }
    }
    if (p < 0 && half == 0)   // an empty slot: zero its rows of the factor tiles (no TMA wrote them)
        for (int k = 0; k < 8; k += 2) x2_zero(F[k], F[k + 1], lr, -1);
    if (half == 0) {
        rs_u[lr] = p >= 0 ? q.rs_u[row] : 0.f;
        cf_u[lr] = p >= 0 ? q.cf_u[row] : 0.f;
        rs_v[lr] = p >= 0 ? q.rs_v[row] : 0.f;
        cf_v[lr] = p >= 0 ? q.cf_v[row] : 0.f;
        x2_zero(X[0], X[1], lr, -1);
    }
    __syncthreads();
    // V'[k, l] = rs_u[k] vt[k, l]: thread (slot, k, half 0) builds row k of its slot
    if (p >= 0 && half == 0 && row < d)
        for (int e = q.rpb[row]; e < q.rpb[row + 1]; ++e) {
            const int c = q.sb[e];
            x2_store_one(X[0], X[1], lr, c % dp, rs_u[lr] * q.vt[c]);
        }
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
        S[t].best = INFINITY; S[t].stall = 0;
    }
    {   // sum_y KDv vt of the loaded scalings (later sums come from the epilogues)
        float v0 = 0.f;
        if (p >= 0) for (int e = row + 64 * half; e < q.ic[IC_NB]; e += 128) { const int c = q.sb[e]; v0 += q.KDv[c] * q.vt[c]; }
        v0 = x2_slot_sum(v0, shf);
        if (t == st0(slot)) S[slot].sKv = v0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = tbase;
    uint32_t phase = 0;
    const float aD = p >= 0 ? (float)q.sc[SC_AD] : 0.f, bD = p >= 0 ? (float)q.sc[SC_BD] : 0.f;
    const float total = p >= 0 ? (float)q.sc[SC_TOTAL] : 1.f;
    const float DD = p >= 0 ? (float)q.sc[SC_DD] : 0.f, tau = p >= 0 ? (float)q.sc[SC_TAU] : 0.f;
    const float etau = expf(tau), etaui = 1.f / etau, e85 = expf(85.f), e85i = expf(-85.f);
    float* stg = stage + warp * 32 * 33;
    const int st = slot * 64;   // first thread of this slot
    const unsigned char* A1u[2] = {F[0], F[1]};
    const unsigned char* A2u[2] = {F[2], F[3]};
    const unsigned char* A1v[2] = {F[4], F[5]};
    const unsigned char* A2v[2] = {F[6], F[7]};
    const unsigned char* BX[2] = {X[0], X[1]};
    int live_next = S[slot].live;   // thread st: its slot still iterates (the loop-top barrier ORs them)
    for (int it = 0; it < n_inner && !timeout; ++it) {
        if (!__syncthreads_or(t == st && live_next)) break;
        const bool live = S[slot].live != 0;   // written before the barrier above
        const float vtD = S[slot].vtD;
        const float sKv = S[slot].sKv;
        // ================= u-update
        if (!x2_run(tm, A1u, BX, &mbar, phase, diag)) { timeout = 1; break; }
        {                                                                  // Wt rows j
            float v[32];
            tmem_ld32(x2_taddr(tm), v);
            x2_store_chunk(X[0], X[1], lr, half, v, live ? 1.f : 0.f);
        }
        if (!x2_run(tm, A2u, BX, &mbar, phase, diag)) { timeout = 1; break; }
        float ku_loc = 0.f;                                                // sum_x KDu ut (v_Delta)
        {
            const int i = row;
            const float rsv = rs_v[lr];
            const int e0 = live && i < d ? q.rpa[i] : 0, e1 = live && i < d ? q.rpa[i + 1] : 0;
            x2_zero(X[0], X[1], lr, half);
            bool rng = false;
            float v[32];
            tmem_ld32(x2_taddr(tm), v);
#pragma unroll
            for (int u = 0; u < 32; ++u) stg[lane * 33 + u] = v[u];
            __syncwarp();
            for (int e = e0; e < e1; ++e) {
                const int c = q.sa[e], j = c % dp;
                if ((j >> 5) != half) continue;
                const float kdu = q.KDu[c];
                const float den = cf_u[st + j] * stg[lane * 33 + (j & 31)] + kdu * vtD;
                const float a = q.am[c];
                const float uu = a / den;
                if (!x2_in(uu / a, etau, etaui) || !x2_in(uu * rsv, e85, e85i)) rng = true;
                q.ut[c] = uu;
                ku_loc += kdu * uu;
                x2_store_one(X[0], X[1], lr, j, uu * rsv);
            }
            __syncwarp();
            if (rng) S[slot].range = 1;
        }
        const float sKu = x2_slot_sum(ku_loc, shf);
        const float utD = (aD > 0.f) ? aD / (sKv + DD * vtD) : 0.f;        // every thread of the slot
        if (live && t == st && aD > 0.f && !x2_in(utD / aD, etau, etaui)) S[slot].range = 1;
        // ================= v-update
        if (!x2_run(tm, A1v, BX, &mbar, phase, diag)) { timeout = 1; break; }
        {                                                                  // Wv rows l
            float v[32];
            tmem_ld32(x2_taddr(tm), v);
            x2_store_chunk(X[0], X[1], lr, half, v, live ? 1.f : 0.f);
        }
        if (!x2_run(tm, A2v, BX, &mbar, phase, diag)) { timeout = 1; break; }
        float e_loc = 0.f, kv_loc = 0.f;
        {
            const int k = row;
            const float rsu = rs_u[lr];
            const int e0 = live && k < d ? q.rpb[k] : 0, e1 = live && k < d ? q.rpb[k + 1] : 0;
            x2_zero(X[0], X[1], lr, half);
            bool rng = false;
            float v[32];
            tmem_ld32(x2_taddr(tm), v);
#pragma unroll
            for (int u = 0; u < 32; ++u) stg[lane * 33 + u] = v[u];
            __syncwarp();
            for (int e = e0; e < e1; ++e) {
                const int c = q.sb[e], l = c % dp;
                if ((l >> 5) != half) continue;
                const float kdv = q.KDv[c];
                const float qv = cf_v[st + l] * stg[lane * 33 + (l & 31)] + kdv * utD;
                const float b = q.bm[c];
                e_loc += fabsf(q.vt[c] * qv - b);
                const float vv = b / qv;
                if (!x2_in(vv / b, etau, etaui) || !x2_in(vv * rsu, e85, e85i)) rng = true;
                q.vt[c] = vv;
                kv_loc += kdv * vv;
                x2_store_one(X[0], X[1], lr, l, vv * rsu);
            }
            __syncwarp();
            if (rng) S[slot].range = 1;
        }
        const float2 ek = x2_slot_sum2(e_loc, kv_loc, shf2);
        if (live && t == st) {
            X2Slot& Z = S[slot];
            float ee = ek.x;
            const float qD = sKu + DD * utD;
            Z.utD = utD;
            Z.sKu = sKu;
            Z.sKv = ek.y;
            if (bD > 0.f) {
                ee += fabsf(vtD * qD - bD);
                const float vv = bD / qD;
                if (!x2_in(vv / bD, etau, etaui)) Z.range = 1;
                Z.vtD = vv;
            }
            Z.err = ee / total;
            ++Z.iters; ++Z.since;
            if (Z.err < 0.95f * Z.best) { Z.best = Z.err; Z.stall = 0; } else ++Z.stall;
            if (!isfinite(Z.err)) { Z.absorb = 1; Z.live = 0; }
            else if (r.tol > 0 && Z.err <= r.tol) { Z.status = ST_CONVERGED; Z.live = 0; }
            else if (Z.iters >= r.max_iter) { Z.status = ST_MAXITER; Z.live = 0; }
            else if (Z.stall >= X2_STALL) { Z.status = ST_MAXITER; Z.live = 0; }   // precision floor: refine
            else if (Z.range || Z.since >= r.absorb_every) { Z.absorb = 1; Z.live = 0; }
        }
        if (t == st) live_next = S[slot].live;
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

// hi + lo BF16 copies of the four absorbed kernel factors of every active pair,
// laid out for the tensor map: pair p's part k = 2 f + h (factor f: K1u, K2u,
// K1v, K2v; h: hi, lo) row r, column c at bf[p * 8 dp^2 + k dp^2 + r dp + c]
// (the pair's FP64 scratch, 16 dp^2 bytes, holds them; dp = 64).
__global__ void sk_factors_bf16_kernel(SkWS w, unsigned short* __restrict__ bf) {
    const int p = blockIdx.x;
    PairPtrs q = pair_ptrs(w, p);
    if (q.ic[IC_STATUS] != ST_ACTIVE) return;
    const int M = w.dp * w.dp;
    unsigned short* o = bf + (size_t)p * 8 * M;
    const float* src[4] = {q.K1u, q.K2u, q.K1v, q.K2v};
    for (int f = 0; f < 4; ++f)
        for (int x = threadIdx.x * 2; x < M; x += blockDim.x * 2) {
            uint32_t hi, lo;
            x2_split2(src[f][x], src[f][x + 1], hi, lo);
            *reinterpret_cast<uint32_t*>(o + (size_t)(2 * f) * M + x) = hi;
            *reinterpret_cast<uint32_t*>(o + (size_t)(2 * f + 1) * M + x) = lo;
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
    // 4-D view of the copies: (k, row, part, pair), pair stride = the pair's
    // FP64 scratch (2 dp^2 doubles = 65536 bytes at dp = 64)
    CUtensorMap map;
    const cuuint64_t dims[4] = {64, 64, 8, (cuuint64_t)w.P};
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
