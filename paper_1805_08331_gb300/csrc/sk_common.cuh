// sk_common.cuh -- per-pair workspace view and exact-evaluation helpers shared
// by the Sinkhorn engines.
#pragma once
#include "pd_common.cuh"
#include "pd_internal.h"

#ifndef T_CTA
#define T_CTA 256
#endif


// ---------------------------------------------------------------------------
// Exact-ish FP32 evaluation helpers.

// exp(arg) for an FP64 argument: arg = n + r with integer n and |r| <= 0.5
// evaluated as expf(r) * expf(n) (n exact in FP32); relative error ~2 ulp(FP32)
// whatever |arg|, where a plain expf((float)arg) would lose |arg| * 2^-24.
__device__ __forceinline__ float exp_split(double arg) {
    if (!(arg > -103.0)) return 0.0f;
    if (arg > 88.5) arg = 88.5;
    double n = rint(arg);
    float r = (float)(arg - n);
    return expf(r) * expf((float)n);
}

// TwoSum (Knuth): s + e == a + b exactly.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    float s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}
// exp(x + y - (zh + zl)) where x, y, zh are FP32 values of any size and zl is
// the low part of z: the sum is formed with TwoSum so its error is ulp-level of
// the (small) result.  Clamped to the finite FP32 range.
__device__ __forceinline__ float exp3(float x, float y, float zh, float zl) {
    float e1, e2;
    float s1 = two_sum(x, y, e1);
    float s2 = two_sum(s1, -zh, e2);
    float arg = s2 + ((e1 + e2) - zl);
    arg = fminf(arg, 88.5f);
    return arg < -104.0f ? 0.0f : expf(arg);
}

// Round an FP64 shift to an FP32-representable value (any shift is exact
// bookkeeping as long as the same value is used everywhere).
__device__ __forceinline__ double as_f32(double x) { return (double)(float)x; }

// ---------------------------------------------------------------------------
// Workspace accessors.
struct PairPtrs {
    float *K1u, *K2u, *K1v, *K2v, *ut, *vt, *Wt, *Rt, *KDu, *KDv, *am, *bm;
    float *rs_u, *cf_u, *rs_v, *cf_v;
    double *ap, *bp, *al, *be, *Au, *Bu, *Av, *Bv, *phi, *psi, *sc, *L64, *la, *lb;
    int *sa, *sb, *ic, *rpa, *rpb, *cpa, *cpb, *cia, *cib;
};
__device__ __forceinline__ PairPtrs pair_ptrs(const SkWS& w, int p) {
    PairPtrs q;
    const size_t M = (size_t)w.dp * w.dp, V = (size_t)w.dp, N = (size_t)w.n;
    q.K1u = w.K1u + p * M; q.K2u = w.K2u + p * M; q.K1v = w.K1v + p * M; q.K2v = w.K2v + p * M;
    q.ut = w.ut + p * M; q.vt = w.vt + p * M; q.Wt = w.Wt + p * M; q.Rt = w.Rt + p * M;
    q.KDu = w.KDu + p * M; q.KDv = w.KDv + p * M; q.am = w.am + p * M; q.bm = w.bm + p * M;
    q.rs_u = w.rs_u + p * V; q.cf_u = w.cf_u + p * V; q.rs_v = w.rs_v + p * V; q.cf_v = w.cf_v + p * V;
    q.ap = w.ap + p * V; q.bp = w.bp + p * V; q.al = w.al + p * V; q.be = w.be + p * V;
    q.Au = w.Au + p * V; q.Bu = w.Bu + p * V; q.Av = w.Av + p * V; q.Bv = w.Bv + p * V;
    q.phi = w.phi + p * N; q.psi = w.psi + p * N; q.sc = w.sc + (size_t)p * SC_N;
    q.sa = w.sa + p * M; q.sb = w.sb + p * M; q.ic = w.ic + (size_t)p * IC_N;
    q.L64 = w.L64 + 2 * p * M;
    q.la = w.la + p * M; q.lb = w.lb + p * M;
    q.rpa = w.rpa + p * (V + 1); q.rpb = w.rpb + p * (V + 1);
    q.cpa = w.cpa + p * (V + 1); q.cpb = w.cpb + p * (V + 1);
    q.cia = w.cia + p * M; q.cib = w.cib + p * M;
    return q;
}

