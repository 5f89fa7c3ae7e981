// sinkhorn_log2.cu -- on-chip log-domain Sinkhorn iterations in base 2 with
// exactly subtractable arguments (the default iteration kernel).
//
// Mathematics: Prop. 1's separable kernel application in the log semiring,
// restricted to the supports (zero-mass cells carry exp(-inf) = 0):
//   stage 1: L[k,j]   = LSE_{(k,l) in supp(in)} ( h_kl - c_jl/gamma )
//   stage 2: out_(i,j) = -LSE( LSE_k ( L[k,j] - c_ik/gamma ), h_D - cD_(i,j)/gamma )
//   Delta:   out_D     = -LSE( { h_y - cD_y/gamma : y in supp(in) } u { h_D } )
// with h = log(weight) + potential/gamma of the input side; the u-update
// (phi from psi) and the v-update (psi from phi) swap the two sides.  The
// v-update also yields err_t = sum_y w_y |exp(psi_old - psi_new) - 1| / mass,
// the column-marginal error of the plan after the u-update.
//
// Number format.  Every log-value x (log2 units) is a pair (xh, xl): xh is a
// multiple of 2^-G (G chosen from gamma on the host) and |xl| <= 2^-(G+1).
// Multiples of 2^-G below 2^(24-G) are exact FP32 numbers, so with the
// potentials kept below 2^(21-G) every sum or difference of xh words is exact,
// and an argument h - c is two plain additions (xh - ch exact,
// xl - cl to ~1e-11) and exp2 applies to it directly; no TwoSum, no FP64 in
// the loop.  Potentials that leave that range hand their pair to the FP64
// global-memory kernel.
//
// One pass per sum.  Stage 2 and the Delta output are shifted by the previous
// value of the potential they produce, so near convergence the shifted sum is
// close to 1 and its log2 is accurate to a few 1e-8 in absolute terms.  A sum
// outside [2^-100, 2^100] (the first iterations, or any jump) is recomputed
// with the exact maximum.  Stage 1 keeps (max, sum) un-logged, so a stage-2
// term is exp2(m - c) * S.
//
// Output columns are processed in chunks of 32: stage 1 for the chunk's
// columns, then stage 2 for the output cells in them, so the stage-1 buffer
// is (non-empty input rows) x 32 whatever the output support; several pairs
// fit on one SM.
#include "sk_common.cuh"
#include <atomic>
#include <cmath>

#define L2_CW 32          // output columns per chunk
#define L2_MAXCH (256 / L2_CW)   // chunks per side (d <= 256)
#define L2_MAXW 32        // warps per CTA at most

// Dynamic shared memory of the kernel; the per-side arrays are addressed by
// 32-bit byte offsets into it (shared-memory addressing, one register each).
extern __shared__ __align__(16) unsigned char l2_sm[];
template <typename T>
__device__ __forceinline__ T* smp(uint32_t off) { return reinterpret_cast<T*>(l2_sm + off); }
// Per-side arrays: in shared memory (GM = false), or in the pair's global
// workspace at gb (GM = true, pairs whose supports do not fit on chip); the
// cost tables and the stage-1 buffer are in shared memory in both variants.
template <typename T, bool GM>
__device__ __forceinline__ T* sdp(unsigned char* gb, uint32_t off) {
    if constexpr (GM) return reinterpret_cast<T*>(gb + off);
    else return reinterpret_cast<T*>(l2_sm + off);
}

struct L2Side {
    int n, nr, nc, nch;
    uint32_t lw;      // float2 [n] log2 weight (hi, lo)
    uint32_t pot;     // float2 [n] potential/gamma in log2 units (hi, lo)
    uint32_t hin;     // float2 [n] lw + pot, the side's h when it is the input
    uint32_t rec;     // pairwise records, two cells per 32 bytes (l2_rec_*): float4 [np] (A_2p, A_2p+1,
                      //        kap lo_2p, kap lo_2p+1), then float4 [np] (k_2p, k_2p+1, l_2p, l_2p+1),
                      //        np = ceil(n / 2); an odd n's last slot holds A = -inf (a zero term)
    uint32_t w;       // float  [n] weight (marginal error)
    uint32_t rp;      // int    [d+1] row pointers into the support while loading; then, per
                      //        non-empty row r: first cell | one-past-last cell << 16
    uint32_t row;     // short  [n]
    uint32_t col;     // short  [n]
    uint32_t chl;     // short  [n] support entries grouped by output chunk, row-major inside a chunk
    uint32_t rows;    // short  [nr] non-empty rows, longest first
    uint32_t cols;    // short  [nc] non-empty columns
    uint32_t colpos;  // short  [d] position of a column in cols, -1 if empty
    short chs[L2_MAXCH + 1];   // chunk starts in chl
    float2 lwD, potD, hinD;
    float wD;
};

__host__ __device__ __forceinline__ size_t l2_al(size_t x) { return (x + 15) & ~(size_t)15; }

// Bytes of the per-side arrays of a pair (rec: the pairwise form's records).
__host__ __device__ __forceinline__ size_t l2_side_bytes(int nA, int nB, int d, bool rec) {
    size_t b = 0;
    const int ns[2] = {nA, nB};
    for (int s = 0; s < 2; ++s) {
        const size_t n = (size_t)ns[s];
        b += l2_al(24 * n) + (rec ? l2_al(32 * ((n + 1) / 2)) : 0) + l2_al(4 * n) + l2_al(4 * (size_t)(d + 1)) + l2_al(6 * n) +
             l2_al(6 * (size_t)d);
    }
    return b;
}
// Bytes of the cost tables and the stage-1 buffer (nrmax non-empty input rows;
// none when no half-step of the pair takes the separable form).
__host__ __device__ __forceinline__ size_t l2_table_bytes(int nrmax, int d, bool sep = true) {
    return l2_al(8 * (size_t)(2 * d - 1)) + l2_al(8 * (size_t)d) + (sep ? l2_al(8 * (size_t)L2_CW * nrmax) : 0);
}

// Form of a half-step (in = input side, out = output side).  Separable: stage
// 1 has n_in x nc_out terms, stage 2 nr_in x n_out.  Pairwise (p = 2 only):
// n_in x n_out terms, each cheaper (no tables, no stage buffer, two barriers
// per half-step, one setup per output cell instead of one per stage-1 output),
// so it is taken while it has at most L2_PW_RATIO times the separable form's
// terms: 5, the measured break-even on batches of one support shape (random
// cells, d = 32 to 128, 40 to 2080 cells a side).  form: 0 automatic, 1
// separable only, 2 pairwise wherever p = 2, SK_FORM_AUTO2 automatic with the
// ratio 2 (the serving pools: pairs of every size share a launch there, whose
// shared memory the largest pair sets, and the pairwise form loses where few
// CTAs fit on an SM).
#define L2_PW_RATIO 5
__host__ __device__ __forceinline__ bool l2_pw_half(int n_in, int nr_in, int n_out, int nc_out, int form, bool p2) {
    if (!p2 || form == 1) return false;
    if (form == 2) return true;
    const long long direct = (long long)n_in * n_out;
    const long long sep = (long long)n_in * nc_out + (long long)nr_in * n_out;
    return direct <= (form == SK_FORM_AUTO2 ? 2 : L2_PW_RATIO) * sep;
}
// Shared-memory bytes of a pair in the on-chip variant (the host sizes the
// launch with the maximum over the pairs); pwU / pwV: the forms of its
// u- and v-updates.
// rec: the pair may take the pairwise form at some stage (records); sep: it
// may take the separable form at some stage (stage buffer).
__host__ __device__ __forceinline__ size_t l2_need(int nA, int nB, int nrA, int nrB, int d, bool rec, bool sep) {
    return l2_side_bytes(nA, nB, d, rec) + l2_table_bytes(nrA > nrB ? nrA : nrB, d, sep);
}

// Forms of a pair's half-steps.  rule*: the form rule says pairwise (with
// exact scaled units assumed); pw*: pairwise at the starting stage (scaled
// units exist at its gamma); rec: records are needed at some stage (scaled
// units at the target gamma: a smaller gamma only raises n1).
struct L2Forms {
    bool ruleU, ruleV, pwU, pwV, rec;
};
// cap: the shared memory a CTA may use; a pair that fits on chip only without
// the pairwise records (16 bytes per cell) takes the separable form rather
// than the global-memory tier.
__host__ __device__ inline L2Forms l2_forms(int nA, int nB, int nrA, int nrB, int ncA, int ncB, int d, int form,
                                           bool p2_start, bool p2_target, size_t cap) {
    L2Forms f;
    f.ruleU = l2_pw_half(nB, nrB, nA, ncA, form, p2_target);
    f.ruleV = l2_pw_half(nA, nrA, nB, ncB, form, p2_target);
    f.pwU = f.ruleU && p2_start;
    f.pwV = f.ruleV && p2_start;
    f.rec = f.ruleU || f.ruleV;
    if (f.rec && l2_need(nA, nB, nrA, nrB, d, true, !(f.pwU && f.pwV)) > cap &&
        l2_need(nA, nB, nrA, nrB, d, false, true) <= cap)
        f = L2Forms{false, false, false, false, false};
    return f;
}

// (hi, lo) split of an FP64 value on the 2^-G grid (gsc = 2^G).
__device__ __forceinline__ float2 l2_split(double x, double gsc) {
    if (!isfinite(x)) return make_float2((float)x, 0.f);
    const double h = rint(x * gsc) / gsc;
    return make_float2((float)h, (float)(x - h));
}
__device__ __forceinline__ float l2_round(float x, float gsc, float ginv) { return rintf(x * gsc) * ginv; }

// tot (normal, > 0) = 2^e * m with m in [0.75, 1.5); returns e and log2(m).
__device__ __forceinline__ float l2_log2(float tot, int& e) {
    const int b = __float_as_int(tot);
    e = ((b >> 23) & 0xff) - 127;
    float m = __int_as_float((b & 0x007fffff) | 0x3f800000);
    if (m >= 1.5f) { m *= 0.5f; e += 1; }
    return log2f(m);
}

// 2^x with the special-function unit (relative error below 1.5e-7 on the
// normal range, measured against FP64 exp2; results below 2^-126 flush to 0).
__device__ __forceinline__ float l2_ex2(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Non-empty rows (or columns) of a CSR pointer array, in increasing order;
// pos[i] = index in out or -1.  Needs blockDim.x >= d.
static __device__ void l2_compact(const int* __restrict__ ptr, int d, short* out, int* count, short* pos,
                                  int* warp_cnt) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int i = threadIdx.x;
    const bool f = (i < d) && (ptr[i + 1] > ptr[i]);
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_cnt[wid] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int q = 0; q < nw; ++q) { if (q < wid) off += warp_cnt[q]; tot += warp_cnt[q]; }
    const int idx = off + __popc(bal & ((1u << lane) - 1u));
    if (i < d) {
        if (f && out) out[idx] = (short)i;
        if (pos) pos[i] = f ? (short)idx : (short)-1;
    }
    if (threadIdx.x == 0) *count = tot;
    __syncthreads();
}

// Group the output cells of a side by chunk of L2_CW non-empty columns (warp w
// builds chunks w, w + warps, ...; the order inside a chunk stays row-major).
template <bool GM>
static __device__ void l2_chunks(L2Side& s, int* warp_cnt, unsigned char* gb) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nch = s.nch, n = s.n;
    const short* col = sdp<short, GM>(gb, s.col);
    const short* colpos = sdp<short, GM>(gb, s.colpos);
    short* chl = sdp<short, GM>(gb, s.chl);
    // counts per chunk (warp_cnt holds L2_MAXCH entries)
    for (int c = wid; c < nch; c += nw) {
        int cnt = 0;
        for (int b = 0; b < n; b += 32) {
            const int e = b + lane;
            const bool f = e < n && colpos[col[e]] / L2_CW == c;
            cnt += __popc(__ballot_sync(0xffffffffu, f));
        }
        if (lane == 0) warp_cnt[c] = cnt;
    }
    __syncthreads();
    for (int c = wid; c < nch; c += nw) {
        int off = 0;
        for (int q = 0; q < c; ++q) off += warp_cnt[q];
        if (lane == 0) s.chs[c] = (short)off;
        if (c == nch - 1 && lane == 0) s.chs[nch] = (short)(off + warp_cnt[c]);
        for (int b = 0; b < n; b += 32) {
            const int e = b + lane;
            const bool f = e < n && colpos[col[e]] / L2_CW == c;
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (f) chl[off + __popc(bal & ((1u << lane) - 1u))] = (short)e;
            off += __popc(bal);
        }
    }
    if (nch == 0 && threadIdx.x == 0) s.chs[0] = 0;
    __syncthreads();
}

// Reorder the non-empty rows longest first (ties by row index).  In full
// chunks the two half-warps of a warp run stage 1 on two consecutive rows, so
// rows of equal length side by side keep the half-warps in step; stage 2 sums
// over all rows whatever their order.  Needs blockDim.x >= nr.
static __device__ __forceinline__ void l2_sort_rows(short* rows, int nr, const int* rp) {
    const int e = threadIdx.x;
    int k = 0, rank = 0;
    if (e < nr) {
        k = rows[e];
        const int len = rp[k + 1] - rp[k];
        for (int f = 0; f < nr; ++f) {
            const int kf = rows[f], lf = rp[kf + 1] - rp[kf];
            rank += (lf > len) || (lf == len && f < e);
        }
    }
    __syncthreads();
    if (e < nr) rows[rank] = (short)k;
    __syncthreads();
}

// Cost tables in log2 units, (grid, rest) split: ct[m] = c_(m-(d-1))/gamma for
// the grid axis, cdt[m] = cD_m/gamma for the diagonal bin, at this gamma.
template <int NT>
__device__ void l2_tables(float2* ct, float2* cdt, int d, double gamma, double pw, double gsc) {
    const double LOG2E = 1.4426950408889634;
    const double sc2 = LOG2E / (gamma * (double)d * (double)d);
    const int t = threadIdx.x;
    for (int m = t; m < 2 * d - 1; m += NT) {
        const double z = (double)(m - (d - 1));
        ct[m] = l2_split(pw == 2.0 ? z * z * sc2 : pd_c1p(m, d - 1, d, pw) * (LOG2E / gamma), gsc);
    }
    for (int m = t; m < d; m += NT)
        cdt[m] = l2_split(pw == 2.0 ? 0.5 * (double)m * (double)m * sc2 : pd_cdiagp(0, m, d, pw) * (LOG2E / gamma), gsc);
}

struct L2Consts {
    uint32_t ct;     // float2 [2d-1] c_m/gamma in log2 units (hi, lo), m = (i - k) + d - 1
    uint32_t cdt;    // float2 [d] cD_m/gamma in log2 units, m = |j - i|
    uint32_t L1;     // float2 [nr][32] stage-1 (max, sum), swizzled columns
    int d;
    float gsc, ginv, lim;
    float escale;    // 2^40 / total mass (marginal-error terms in fixed point)
    // pairwise form (p = 2): c_xy/gamma in log2 units = s D, D = |x - y|^2 in
    // cells, s = log2(e) / (gamma d^2); it runs in units of kap log2 with
    // sp = s / kap = n1 2^-G on the grid (see l2_pw_consts)
    float sp, kap, rho_h, rho_l;   // sp; kap; 1/kap - 1 as a two-float sum
    bool pw_ok;      // the pairwise form is available at this gamma
    int form;        // 0 automatic, 1 separable only, 2 pairwise wherever pw_ok
};

// Pairwise-form constants at this gamma (p = 2).  The form sums in scaled
// units: a log2-unit value v is v' = v / kap, with kap = s / sp and sp = n1 2^-G
// the grid value nearest s (n1 >= 1, so kap lies in [1/2, 3/2]).  In those
// units a term's exponent is
//   kap ( (h'.hi - sp D - Ms') + h'.lo ),   D = (i-k)^2 + (j-l)^2,
// and h'.hi - sp D - Ms' = A_y + B_x + 2 sp (i k + j l) with A_y = h'.hi -
// sp (k^2 + l^2) per input cell and B_x = -sp (i^2 + j^2) - Ms' per output
// cell: every product and partial sum is a multiple of 2^-G below 2^(24-G)
// (checked here), hence exact in FP32, and kap multiplies only the small
// result.  pw_ok = false (the separable form runs) when no such n1 exists.
// Grid of the (hi, lo) words at the target gamma: 2^-G with 2^(23-G) >= 8
// (max cost/gamma + 64) in log2 units; -1 when G would fall below 4.
__host__ __device__ inline int l2_grid_bits(double gamma) {
    const double cmax = 2.0 / gamma * 1.4426950408889634 + 64.0;
    int e = 0;
    while (ldexp(1.0, e) < 8.0 * cmax && e < 64) ++e;
    const int g = 23 - e;
    return g >= 4 ? (g > 12 ? 12 : g) : -1;
}

struct L2PwC {
    double sp, kap, rho;
    bool ok;
};
__host__ __device__ inline L2PwC l2_pw_calc(double gamma, int d, int gbits, double pw) {
    L2PwC c{0.0, 1.0, 0.0, false};
    if (pw != 2.0 || gbits < 0) return c;
    const double s = 1.4426950408889634 / (gamma * (double)d * (double)d);
    const double n1 = rint(ldexp(s, gbits));
    if (n1 < 1.0) return c;
    c.sp = ldexp(n1, -gbits);
    c.kap = (double)(float)(s / c.sp);   // the FP32 value the kernel multiplies by
    c.rho = 1.0 / c.kap - 1.0;
    const double q = (double)(d - 1) * (double)(d - 1), dmax = 2.0 * q;
    // |h'| and |Ms'| (potentials below 2^(21-G), log2 weights below 64) plus the
    // cost words of every partial sum of A_y + B_x + 2 sp (j l) + 2 sp (i k)
    const double bound = (ldexp(1.0, 22 - gbits) + 128.0) * (1.0 + fabs(c.rho)) + 3.0 * c.sp * dmax;
    c.ok = bound < ldexp(1.0, 24 - gbits) && 2.0 * n1 * q < 16777216.0 && n1 * dmax < 16777216.0;
    return c;
}
__device__ __forceinline__ void l2_pw_consts(L2Consts& K, double gamma, int d, int gbits, double pw) {
    const L2PwC c = l2_pw_calc(gamma, d, gbits, pw);
    K.pw_ok = c.ok;
    K.sp = (float)c.sp;
    K.kap = (float)c.kap;
    K.rho_h = (float)c.rho;
    K.rho_l = (float)(c.rho - (double)(float)c.rho);
}

// The pairwise record of an input cell (row k, column l) from its h = (hi, lo)
// in log2 units: h' = h / kap = h (1 + rho) split into h'.hi on the grid and
// h'.lo (two-float products: hi rho = p + pe exactly), then
// (A = h'.hi - sp (k^2 + l^2), kap h'.lo).
__device__ __forceinline__ float2 l2_pw_record(float2 h, float k, float l, const L2Consts& K) {
    const float p = h.x * K.rho_h;
    const float pe = fmaf(h.x, K.rho_h, -p);
    const float ph = l2_round(p, K.gsc, K.ginv);
    const float hi = h.x + ph;
    const float lo = (p - ph) + (pe + fmaf(h.x, K.rho_l, fmaf(h.y, K.rho_h, h.y)));
    return make_float2(fmaf(-K.sp, fmaf(k, k, l * l), hi), K.kap * lo);
}

// Records of a side of n cells in pairs (the layout of L2Side::rec): cell e's
// (A, kap lo) and its (row, column) sit in lanes e & 1 of the pair records
// e >> 1, so that one packed f32x2 instruction works on two input cells.
__device__ __forceinline__ void l2_rec_put(uint32_t rec, int e, float2 Akl) {
    float* hi = smp<float>(rec + 16 * (e >> 1));
    hi[e & 1] = Akl.x;
    hi[2 + (e & 1)] = Akl.y;
}
__device__ __forceinline__ void l2_rec_coord(uint32_t rec, int n, int e, float k, float l) {
    float* co = smp<float>(rec + 16 * (((n + 1) >> 1) + (e >> 1)));
    co[e & 1] = k;
    co[2 + (e & 1)] = l;
}
__device__ __forceinline__ float2 l2_rec_xy(uint32_t rec, int n, int e) {
    const float* co = smp<float>(rec + 16 * (((n + 1) >> 1) + (e >> 1)));
    return make_float2(co[e & 1], co[2 + (e & 1)]);
}
__device__ __forceinline__ float4 l2_rec_get(uint32_t rec, int n, int e) {   // (A, kap lo, k, l)
    const float* hi = smp<float>(rec + 16 * (e >> 1));
    const float2 xy = l2_rec_xy(rec, n, e);
    return make_float4(hi[e & 1], hi[2 + (e & 1)], xy.x, xy.y);
}

// Packed FP32 pair arithmetic (two lanes of one 64-bit register pair).
__device__ __forceinline__ float2 f2_sub(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 ra, rb, rr;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rr, ra, rb;\n\tmov.b64 {%0, %1}, rr;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 f2_add(float2 a, float2 b) {
    float2 r;
    asm("{.reg .b64 ra, rb, rr;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rr, ra, rb;\n\tmov.b64 {%0, %1}, rr;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
__device__ __forceinline__ float2 f2_fma(float2 a, float2 b, float2 c) {
    float2 r;
    asm("{.reg .b64 ra, rb, rc, rr;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rr, ra, rb, rc;\n\tmov.b64 {%0, %1}, rr;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return r;
}

// Lanes of the Delta-output sum: a fixed partition (thread t < L2_DLANES sums
// the input cells t, t + L2_DLANES, ...), so the sum, like every other sum of
// the kernel, is the same for every CTA width.
#define L2_DLANES 256

// Lanes per output cell in stage 2 (NT / 4 cells per pass).  Wider groups
// measured slower: the per-cell epilogue runs on one lane of the group.
template <int NT> struct L2Lanes { static constexpr int G = 4; static constexpr int SW = 16 / G; };

// Stage-1 buffer index (float2 units): row r, chunk column cc.  Stage 2 reads
// rows r = g + G u together (g = lane in the cell's group); XOR-ing the column
// with g * SW puts those G reads in distinct 8-byte bank slots of a wavefront.
template <int NT>
__device__ __forceinline__ int l2_lidx(int r, int cc) {
    return r * L2_CW + (cc ^ ((r & (L2Lanes<NT>::G - 1)) * L2Lanes<NT>::SW));
}

// e^x - 1 for |x| <= 2^-5 ln 2 (the rest word of a potential, G >= 4): Taylor
// polynomial of degree 5 (relative error below x^5 / 720 < 7e-12).
__device__ __forceinline__ float l2_expm1_small(float x) {
    return x * fmaf(x, fmaf(x, fmaf(x, fmaf(x, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f), 0.5f), 1.f);
}

// New potential -(shift + log2 tot) as a (grid, rest) pair; err term
// w |exp(old - new) - 1| added when want_err, in units of 2^-40 of the total
// mass as a 64-bit integer: integer sums are exact, so err_t does not depend
// on which thread adds which cell (terms above 2^4 of the mass saturate, a
// non-finite term sets errbad).  Returns false if out of range.
__device__ __forceinline__ bool l2_update(float tot, float shift, float Ms, float2 po, float wgt, bool want_err,
                                          const L2Consts& K, long long& errq, bool& errbad, float2& pn) {
    if (!(tot > 0.f && isfinite(tot) && isfinite(shift))) return false;
    int ex;
    const float l = l2_log2(tot, ex);
    const float lr = l2_round(l, K.gsc, K.ginv);
    pn = make_float2(-((shift + (float)ex) + lr), -(l - lr));
    if (want_err) {
        // old - new = po.y + log2(tot) (+ po.x + shift, zero unless the exact path ran)
        const float ev = (shift == Ms) ? (tot - 1.f) + tot * l2_expm1_small(po.y * 0.69314718f)
                                       : tot * exp2f((po.x + shift) + po.y) - 1.f;
        const float term = wgt * fabsf(ev);
        const float v = term * K.escale;
        errbad |= !isfinite(term);
        errq += v <= 0x1p44f ? llrintf(v) : (1ll << 44);
    }
    return fabsf(pn.x) < K.lim;
}

// End of a Delta-output sum: tot = the input cells' terms shifted by the
// previous value MsD; adds the input Delta term, recomputes with the exact
// maximum when the sum left [2^-100, 2^100], and updates out.potD.
template <bool GM>
static __device__ __forceinline__ void l2_delta_finish(L2Side& in, L2Side& out, const L2Consts& K, float tot,
                                                       bool want_err, long long& errq, bool& errbad, int* range_flag,
                                                       unsigned char* gb) {
    const int in_n = in.n;
    const float2* in_hin = sdp<float2, GM>(gb, in.hin);
    const short* in_row = sdp<short, GM>(gb, in.row);
    const short* in_col = sdp<short, GM>(gb, in.col);
    const float2* cdt = smp<float2>(K.cdt);
    const float MsD = -out.potD.x;
    const float2 hD = in.hinD;
    if (hD.x > -INFINITY) tot += exp2f((hD.x - MsD) + hD.y);
    float shift = MsD;
    if (!(tot >= 0x1p-100f && tot <= 0x1p100f)) {
        float mx = hD.x;
        for (int q = 0; q < in_n; ++q)
            mx = fmaxf(mx, in_hin[q].x - cdt[abs((int)in_col[q] - (int)in_row[q])].x);
        shift = mx;
        tot = (hD.x > -INFINITY) ? exp2f((hD.x - shift) + hD.y) : 0.f;
        for (int q = 0; q < in_n; ++q) {
            const float2 h = in_hin[q];
            const float2 c = cdt[abs((int)in_col[q] - (int)in_row[q])];
            tot += exp2f(((h.x - c.x) - shift) + (h.y - c.y));
        }
    }
    float2 pn;
    if (l2_update(tot, shift, MsD, out.potD, out.wD, want_err, K, errq, errbad, pn)) {
        out.potD = pn;
        out.hinD = make_float2(out.lwD.x + pn.x, out.lwD.y + pn.y);
    } else {
        atomicOr(range_flag, 1);
    }
}

// Delta output of a half-step, shifted by its previous value: partial sums
// over a fixed L2_DLANES-lane partition of the input cells, one barrier, then
// thread `fin` finishes the sum and updates out.potD (the other threads go on).
template <int NT, bool GM>
static __device__ __forceinline__ void l2_delta_out(L2Side& in, L2Side& out, const L2Consts& K, bool want_err,
                                                    long long& errq, bool& errbad, float* redD, int* range_flag,
                                                    unsigned char* gb, int fin = 0) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int in_n = in.n;
    const float2* in_hin = sdp<float2, GM>(gb, in.hin);
    const short* in_row = sdp<short, GM>(gb, in.row);
    const short* in_col = sdp<short, GM>(gb, in.col);
    const float2* cdt = smp<float2>(K.cdt);
    const bool doD = out.wD > 0.f;
    const float MsD = -out.potD.x;
    // lane ln of the fixed L2_DLANES-lane partition is thread ln % NT (one pass
    // for NT >= L2_DLANES, two for 128 threads), so the per-warp partial sums
    // and their order are the same at every width
    if constexpr (NT >= L2_DLANES) {
        float sD = 0.f;
        if (doD && t < L2_DLANES) {
            for (int q = t; q < in_n; q += L2_DLANES) {
                const float2 h = in_hin[q];
                const float2 c = cdt[abs((int)in_col[q] - (int)in_row[q])];
                sD += l2_ex2(((h.x - c.x) - MsD) + (h.y - c.y));
            }
        }
        sD = warp_sum(sD);
        if (lane == 0 && wid < L2_DLANES / 32) redD[wid] = sD;
    } else {
#pragma unroll
        for (int base = 0; base < L2_DLANES; base += NT) {
            const int ln = base + t;
            float sD = 0.f;
            if (doD) {
                for (int q = ln; q < in_n; q += L2_DLANES) {
                    const float2 h = in_hin[q];
                    const float2 c = cdt[abs((int)in_col[q] - (int)in_row[q])];
                    sD += l2_ex2(((h.x - c.x) - MsD) + (h.y - c.y));
                }
            }
            sD = warp_sum(sD);
            if (lane == 0) redD[ln >> 5] = sD;
        }
    }
    __syncthreads();
    if (t == fin && doD) {
        float tot = 0.f;
        for (int q = 0; q < L2_DLANES / 32; ++q) tot += redD[q];
        l2_delta_finish<GM>(in, out, K, tot, want_err, errq, errbad, range_flag, gb);
    }
}

// Delta output of a pairwise half-step by one warp, with no block barrier:
// lane l sums the input cells l, l + 32, ... in order, a fixed shuffle tree
// adds the lanes, and lane 0 finishes.  The partition is the same whichever
// warp runs it and at every CTA width.  out.potD is read by the next
// half-step only, behind this half-step's closing barrier.
static __device__ __forceinline__ void l2_delta_warp(L2Side& in, L2Side& out, const L2Consts& K, bool want_err,
                                                     long long& errq, bool& errbad, int* range_flag) {
    if (!(out.wD > 0.f)) return;
    const int lane = threadIdx.x & 31, in_n = in.n;
    const float2* in_hin = smp<float2>(in.hin);
    const short* in_row = smp<short>(in.row);
    const short* in_col = smp<short>(in.col);
    const float2* cdt = smp<float2>(K.cdt);
    const float MsD = -out.potD.x;
    float sD = 0.f;
    for (int q = lane; q < in_n; q += 32) {
        const float2 h = in_hin[q];
        const float2 c = cdt[abs((int)in_col[q] - (int)in_row[q])];
        sD += l2_ex2(((h.x - c.x) - MsD) + (h.y - c.y));
    }
    sD = warp_sum(sD);
    if (lane == 0) l2_delta_finish<false>(in, out, K, sD, want_err, errq, errbad, range_flag, nullptr);
}

// One half-step: out.pot <- -LSE over the input side.  Adds the marginal-error
// terms of `out` to errq when want_err.  Sets *range_flag if a potential left
// the exact range (the pair then moves to the FP64 kernel).
template <int NT, bool GM>
static __device__ void l2_half(L2Side& in, L2Side& out, const L2Consts& K, bool want_err, long long& errq,
                               bool& errbad, float* redD, int* range_flag, unsigned char* gb) {
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int d = K.d;
    const int in_nr = in.nr;
    const float2* in_hin = sdp<float2, GM>(gb, in.hin);
    const short* in_col = sdp<short, GM>(gb, in.col);
    const short* in_rows = sdp<short, GM>(gb, in.rows);
    const int* in_rq = sdp<int, GM>(gb, in.rp);
    const float2* ct = smp<float2>(K.ct);
    const float2* cdt = smp<float2>(K.cdt);
    float2* L1 = smp<float2>(K.L1);
    l2_delta_out<NT, GM>(in, out, K, want_err, errq, errbad, redD, range_flag, gb);
    const float2 hD = in.hinD;   // input Delta term (not written in this half-step)
    constexpr int L2_G = L2Lanes<NT>::G;
    const unsigned gmask = ((1u << L2_G) - 1u) << (lane & ~(L2_G - 1));
    const int g = lane & (L2_G - 1);
    const int out_nch = out.nch, out_nc = out.nc;
    const short* out_cols = sdp<short, GM>(gb, out.cols);
    for (int ch = 0; ch < out_nch; ++ch) {
        const int c0 = ch * L2_CW;
        const int wc = min(L2_CW, out_nc - c0);
        // ---- stage 1 for the chunk's columns: element (r, cc), r over non-empty input rows
        if (wc == L2_CW) {
            // full chunk: lane handles columns cc and cc + 16 of one row, the two
            // half-warps two consecutive rows, so each input cell's (h, column)
            // is loaded once for two output columns
            const int cc = lane & 15;
            const float2* cta = ct + (out_cols[c0 + cc] + d - 1);
            const float2* ctb = ct + (out_cols[c0 + cc + 16] + d - 1);
            for (int r = 2 * wid + (lane >> 4); r < in_nr; r += 2 * (NT / 32)) {
                const int rq = in_rq[r];
                const int q0 = rq & 0xffff, q1 = rq >> 16;
                float2 h = in_hin[q0];
                int col = in_col[q0];
                float2 ca = cta[-col], cb = ctb[-col];
                float ma = h.x - ca.x, mb = h.x - cb.x;
                float Sa = l2_ex2(h.y - ca.y), Sb = l2_ex2(h.y - cb.y);
                for (int qq = q0 + 1; qq < q1; ++qq) {
                    h = in_hin[qq];
                    col = in_col[qq];
                    ca = cta[-col];
                    cb = ctb[-col];
                    const float aa = h.x - ca.x, ab = h.x - cb.x;
                    const float mna = fmaxf(ma, aa), mnb = fmaxf(mb, ab);
                    Sa = fmaf(Sa, l2_ex2(ma - mna), l2_ex2((aa - mna) + (h.y - ca.y)));
                    Sb = fmaf(Sb, l2_ex2(mb - mnb), l2_ex2((ab - mnb) + (h.y - cb.y)));
                    ma = mna;
                    mb = mnb;
                }
                L1[l2_lidx<NT>(r, cc)] = make_float2(ma, Sa);
                L1[l2_lidx<NT>(r, cc + 16)] = make_float2(mb, Sb);
            }
        } else {
            int r = t / wc, cc = t - r * wc;
            const int dr = NT / wc, dc = NT - dr * wc;
            while (r < in_nr) {
                const int j = out_cols[c0 + cc];
                const int rq = in_rq[r];
                const int q0 = rq & 0xffff, q1 = rq >> 16;
                const float2* ctj = ct + (j + d - 1);
                // online log-sum-exp over the row's cells: (m, S) with value m + log2 S
                float2 h = in_hin[q0];
                float2 c = ctj[-(int)in_col[q0]];
                float m = h.x - c.x;
                float S = l2_ex2(h.y - c.y);
                for (int qq = q0 + 1; qq < q1; ++qq) {
                    h = in_hin[qq];
                    c = ctj[-(int)in_col[qq]];
                    const float a = h.x - c.x;
                    const float mn = fmaxf(m, a);
                    S = fmaf(S, l2_ex2(m - mn), l2_ex2((a - mn) + (h.y - c.y)));
                    m = mn;
                }
                L1[l2_lidx<NT>(r, cc)] = make_float2(m, S);
                r += dr; cc += dc;
                if (cc >= wc) { cc -= wc; ++r; }
            }
        }
        __syncthreads();
        // ---- stage 2 for the chunk's output cells, L2_G lanes per cell
        {
            const int cs = out.chs[ch], ce = out.chs[ch + 1];
            const short* out_chl = sdp<short, GM>(gb, out.chl);
            const short* out_row = sdp<short, GM>(gb, out.row);
            const short* out_col = sdp<short, GM>(gb, out.col);
            const short* out_colpos = sdp<short, GM>(gb, out.colpos);
            float2* out_pot = sdp<float2, GM>(gb, out.pot);
            // every lane of a group runs the same trip count (the loop index is shared)
            for (int e0 = cs; e0 < ce; e0 += NT / L2_G) {
                const int e = e0 + (t / L2_G);
                const bool live = e < ce;
                int i = 0, j = 0, ccs = 0, qo = 0;
                float2 po = make_float2(0.f, 0.f);
                if (live) {
                    qo = out_chl[e];
                    i = out_row[qo]; j = out_col[qo];
                    ccs = (out_colpos[j] - c0) ^ (g * L2Lanes<NT>::SW);   // rows r = g + G u
                    po = out_pot[qo];
                }
                const float Ms = -po.x;
                const float2* cti = ct + (i + d - 1);
                float tot = 0.f;
                if (live) {
                    // two interleaved compensated sums (rows g + 2Gu and g + G + 2Gu)
                    float s0 = 0.f, c0s = 0.f, s1 = 0.f, c1s = 0.f;
                    int r2 = g;
                    for (; r2 + L2_G < in_nr; r2 += 2 * L2_G) {
                        const int ka = in_rows[r2], kb = in_rows[r2 + L2_G];
                        const float2 La = L1[r2 * L2_CW + ccs], Lb = L1[(r2 + L2_G) * L2_CW + ccs];
                        const float2 ca = cti[-ka], cb = cti[-kb];
                        kahan_add(s0, c0s, l2_ex2(((La.x - ca.x) - Ms) - ca.y) * La.y);
                        kahan_add(s1, c1s, l2_ex2(((Lb.x - cb.x) - Ms) - cb.y) * Lb.y);
                    }
                    if (r2 < in_nr) {
                        const int ka = in_rows[r2];
                        const float2 ca = cti[-ka];
                        const float2 La = L1[r2 * L2_CW + ccs];
                        kahan_add(s0, c0s, l2_ex2(((La.x - ca.x) - Ms) - ca.y) * La.y);
                    }
                    if (g == 0 && hD.x > -INFINITY) {
                        const float2 c = cdt[abs(j - i)];
                        kahan_add(s1, c1s, l2_ex2(((hD.x - c.x) - Ms) + (hD.y - c.y)));
                    }
                    tot = (s0 - c0s) + (s1 - c1s);
                }
#pragma unroll
                for (int o = 1; o < L2_G; o <<= 1) tot += __shfl_xor_sync(gmask, tot, o);
                float shift = Ms;
                if (live && !(tot >= 0x1p-100f && tot <= 0x1p100f)) {
                    // exact maximum of the group's terms; S_k <= 256 so shift = max + 8 bounds every term by 1
                    float mx = -INFINITY;
                    for (int r3 = g; r3 < in_nr; r3 += L2_G)
                        mx = fmaxf(mx, L1[r3 * L2_CW + ccs].x - cti[-(int)in_rows[r3]].x);
                    if (g == 0 && hD.x > -INFINITY) mx = fmaxf(mx, hD.x - cdt[abs(j - i)].x);
#pragma unroll
                    for (int o = 1; o < L2_G; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(gmask, mx, o));
                    shift = mx + 8.f;
                    float s = 0.f, cmp = 0.f;
                    for (int r3 = g; r3 < in_nr; r3 += L2_G) {
                        const float2 c = cti[-(int)in_rows[r3]];
                        const float2 La = L1[r3 * L2_CW + ccs];
                        kahan_add(s, cmp, l2_ex2(((La.x - c.x) - shift) - c.y) * La.y);
                    }
                    if (g == 0 && hD.x > -INFINITY) {
                        const float2 c = cdt[abs(j - i)];
                        kahan_add(s, cmp, l2_ex2(((hD.x - c.x) - shift) + (hD.y - c.y)));
                    }
                    tot = s - cmp;
#pragma unroll
                    for (int o = 1; o < L2_G; o <<= 1) tot += __shfl_xor_sync(gmask, tot, o);
                }
                if (live && g == 0) {
                    float2 pn;
                    if (l2_update(tot, shift, Ms, po, sdp<float, GM>(gb, out.w)[qo], want_err, K, errq, errbad,
                                  pn)) {
                        out_pot[qo] = pn;
                        const float2 lw = sdp<float2, GM>(gb, out.lw)[qo];
                        const float2 hn = make_float2(lw.x + pn.x, lw.y + pn.y);
                        sdp<float2, GM>(gb, out.hin)[qo] = hn;
                        if (!GM && K.pw_ok) l2_rec_put(out.rec, qo, l2_pw_record(hn, (float)i, (float)j, K));
                    } else {
                        atomicOr(range_flag, 1);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (out_nch == 0) __syncthreads();
}

// One pairwise term in the scaled units of l2_pw_consts: r = (A_y, kap h'.lo,
// k, l); B = B_x, a = 2 sp i, b = 2 sp j.  The hi word A_y + B_x + b l + a k
// is exact; kap multiplies it and adds kap h'.lo in one rounding.
__device__ __forceinline__ float l2_pw_term(const float4& r, float B, float a, float b, float kap) {
    return l2_ex2(fmaf(kap, fmaf(a, r.z, fmaf(b, r.w, r.x + B)), r.y));
}
// The same term for two input cells at once, from a pair record: hi = (A_0,
// A_1, kap lo_0, kap lo_1), co = (k_0, k_1, l_0, l_1); every step is one packed
// f32x2 instruction for both (each lane rounds as the scalar form does).
__device__ __forceinline__ float2 l2_pw_term2(const float4& hi, const float4& co, float2 B2, float2 a2, float2 b2,
                                              float2 k2) {
    float2 t = f2_add(make_float2(hi.x, hi.y), B2);
    t = f2_fma(b2, make_float2(co.z, co.w), t);
    t = f2_fma(a2, make_float2(co.x, co.y), t);
    t = f2_fma(k2, t, make_float2(hi.z, hi.w));
    return make_float2(l2_ex2(t.x), l2_ex2(t.y));
}

// Pairwise form of a half-step (p = 2, on chip): the same log-sum-exp as the
// separable form, summed over the input support directly,
//   out_x = -LSE( { h_y - s D_xy : y in supp(in) } u { h_D - cD_x/gamma } ),
// in the scaled units of l2_pw_consts: per output cell, Ms' = the grid value
// nearest Ms / kap (Ms = -(previous out_x)), B_x = -sp (i^2 + j^2) - Ms', and
// delta = kap Ms' - Ms; per term one shared record, FADD + 2 FFMA (the exact hi
// word), FFMA (kap hi + kap lo) and ex2: the terms are shifted by kap Ms' = Ms +
// delta, so tot = (their sum) 2^delta + (the Delta term shifted by Ms).  One
// lane per output cell runs over all input cells in order (every lane of a
// warp reads the same record: one broadcast load); it adds blocks of eight
// terms (then one of four), left to right, and sums the blocks compensated
// (Kahan), then the last records.  The partition does not depend on the CTA
// width, so neither does any result.  (Measured slower on the benchmark
// batch: several lanes per cell over strided parts of the input, 10 %; two
// cells per lane in packed arithmetic, 25 %: half the warps busy.)
template <int NT>
static __device__ void l2_half_pw(L2Side& in, L2Side& out, const L2Consts& K, bool want_err, long long& errq,
                                  bool& errbad, int* range_flag, bool end_sync) {
    const int t = threadIdx.x;
    const int n_in = in.n, m = out.n;
    // the Delta output: one warp, no block barrier; the first warp without an
    // output cell if there is one, else the last warp (fewest cells in the
    // last pass)
    const int idle = (m + 31) >> 5;
    if ((t >> 5) == (idle < NT / 32 ? idle : NT / 32 - 1))
        l2_delta_warp(in, out, K, want_err, errq, errbad, range_flag);
    const int np = (n_in + 1) >> 1;   // pair records of the input (an odd n's last slot is a zero term)
    const float4* rhi = smp<float4>(in.rec);
    const float4* rco = rhi + np;
    float2* out_pot = smp<float2>(out.pot);
    const float2* cdt = smp<float2>(K.cdt);
    const float2 hD = in.hinD;   // input Delta term (not written in this half-step)
    const float kap = K.kap, sp = K.sp;
    for (int e0 = 0; e0 < m; e0 += NT) {
        const int e = e0 + t;
        if (e >= m) continue;
        float sum, Mp;
        {
            // the sum over the records, shifted by kap Ms' (Ms' on the grid),
            // two input cells per packed instruction; only what the loop needs
            // is live across it
            const float2 xy = l2_rec_xy(out.rec, m, e);
            const float Ms = -out_pot[e].x;
            Mp = Ms + l2_round(Ms * K.rho_h, K.gsc, K.ginv);
            const float a = 2.f * sp * xy.x, b = 2.f * sp * xy.y;
            const float B = fmaf(-sp, fmaf(xy.x, xy.x, xy.y * xy.y), -Mp);
            const float2 B2 = make_float2(B, B), a2 = make_float2(a, a), b2 = make_float2(b, b),
                         k2 = make_float2(kap, kap);
            float sm = 0.f, cm = 0.f;
            int q = 0;
            for (; q + 3 < np; q += 4) {
                float2 ev[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) ev[u] = l2_pw_term2(rhi[q + u], rco[q + u], B2, a2, b2, k2);
                const float2 s2 = f2_add(f2_add(ev[0], ev[1]), f2_add(ev[2], ev[3]));
                kahan_add(sm, cm, s2.x + s2.y);
            }
            float2 rest = make_float2(0.f, 0.f);
#pragma unroll 1
            for (; q < np; ++q) rest = f2_add(rest, l2_pw_term2(rhi[q], rco[q], B2, a2, b2, k2));
            kahan_add(sm, cm, rest.x + rest.y);
            sum = sm - cm;
        }
        const float2 xy = l2_rec_xy(out.rec, m, e);
        const float xi = xy.x, xj = xy.y;
        const float2 po = out_pot[e];
        const float Ms = -po.x;
        const float2 cD = cdt[abs((int)xj - (int)xi)];
        // the records' terms are 2^(x - delta) (shift kap Ms' = Ms + delta, x the
        // exponent shifted by Ms): their sum times 2^delta, plus the Delta term
        float tot = fmaf(sum, exp2f(fmaf(kap, Mp, -Ms)),
                         hD.x > -INFINITY ? l2_ex2(((hD.x - cD.x) - Ms) + (hD.y - cD.y)) : 0.f);
        float shift = Ms;
        if (!(tot >= 0x1p-100f && tot <= 0x1p100f)) {
            // exact maximum of the terms (hi words, scaled units, shift 0); an
            // integer shift at or above kap times it keeps every term at most
            // about 1 and the largest near 1
            const float a = 2.f * sp * xi, b = 2.f * sp * xj;
            const float B0 = -sp * fmaf(xi, xi, xj * xj);
            float mx = -INFINITY;
#pragma unroll 1
            for (int y = 0; y < n_in; ++y) {
                const float4 r = l2_rec_get(in.rec, n_in, y);
                mx = fmaxf(mx, kap * fmaf(a, r.z, fmaf(b, r.w, r.x + B0)));
            }
            if (hD.x > -INFINITY) mx = fmaxf(mx, hD.x - cD.x);
            shift = ceilf(mx);
            const float Mf = shift + l2_round(shift * K.rho_h, K.gsc, K.ginv);
            const float B = fmaf(-sp, fmaf(xi, xi, xj * xj), -Mf);
            float sm = 0.f, cm = 0.f;
#pragma unroll 1
            for (int y = 0; y < n_in; ++y) kahan_add(sm, cm, l2_pw_term(l2_rec_get(in.rec, n_in, y), B, a, b, kap));
            tot = fmaf(sm - cm, exp2f(fmaf(kap, Mf, -shift)),
                       hD.x > -INFINITY ? l2_ex2(((hD.x - cD.x) - shift) + (hD.y - cD.y)) : 0.f);
        }
        float2 pn;
        if (l2_update(tot, shift, Ms, po, smp<float>(out.w)[e], want_err, K, errq, errbad, pn)) {
            out_pot[e] = pn;
            const float2 lw = smp<float2>(out.lw)[e];
            const float2 hn = make_float2(lw.x + pn.x, lw.y + pn.y);
            smp<float2>(out.hin)[e] = hn;
            l2_rec_put(out.rec, e, l2_pw_record(hn, xi, xj, K));
        } else {
            atomicOr(range_flag, 1);
        }
    }
    // the closing barrier (the caller's error reduction provides it after the
    // v-update)
    if (end_sync) __syncthreads();
}

// gamma-continuation step inside the launch: gamma -> gamma / 4.  Potentials
// in log2 units of the new gamma are 4x the old ones: 4 hi is exact on the grid,
// 4 lo is re-split; h = log2 weight + potential follows; the cost tables are
// rebuilt for the new gamma.  Sets *range_flag if a potential leaves the exact
// range (the pair then moves to the FP64 kernel).
template <int NT, bool GM>
static __device__ void l2_next_stage(L2Side* S, const L2Consts& K, double gamma_new, double pw, int d,
                                     int* range_flag, unsigned char* gb) {
    const int t = threadIdx.x;
    for (int s = 0; s < 2; ++s) {
        L2Side& X = S[s];
        float2* xpot = sdp<float2, GM>(gb, X.pot);
        float2* xhin = sdp<float2, GM>(gb, X.hin);
        const float2* xlw = sdp<float2, GM>(gb, X.lw);
        for (int e = t; e < X.n; e += NT) {
            const float2 po = xpot[e];
            const float v = po.y * 4.f, rv = l2_round(v, K.gsc, K.ginv);
            const float2 pn = make_float2(po.x * 4.f + rv, v - rv);
            if (!(fabsf(pn.x) < K.lim)) atomicOr(range_flag, 1);
            xpot[e] = pn;
            const float2 hn = make_float2(xlw[e].x + pn.x, xlw[e].y + pn.y);
            xhin[e] = hn;
            if (!GM && K.pw_ok)   // (records may not exist yet: the coordinates come from the cell lists)
                l2_rec_put(X.rec, e, l2_pw_record(hn, (float)smp<short>(X.row)[e], (float)smp<short>(X.col)[e], K));
        }
    }
    __syncthreads();   // every thread has read the sides' Delta state (hinD in the half-steps) before t == 0 writes it
    if (t == 0) {
        for (int s = 0; s < 2; ++s) {
            L2Side& X = S[s];
            const float v = X.potD.y * 4.f, rv = l2_round(v, K.gsc, K.ginv);
            X.potD = make_float2(X.potD.x * 4.f + rv, v - rv);
            if (!(fabsf(X.potD.x) < K.lim)) atomicOr(range_flag, 1);
            X.hinD = X.wD > 0.f ? make_float2(X.lwD.x + X.potD.x, X.lwD.y + X.potD.y) : make_float2(-INFINITY, 0.f);
        }
    }
    l2_tables<NT>(smp<float2>(K.ct), smp<float2>(K.cdt), d, gamma_new, pw, (double)K.gsc);
    __syncthreads();
}

// GM = false: pairs with IC_BIG == 0, everything on chip; a pair that does
// not fit moves to IC_BIG = 1.  GM = true: pairs with IC_BIG == 1, per-side
// arrays in the pair's FP64 scratch L64 (gcap bytes); a pair whose arrays
// exceed it moves to IC_BIG = 2 (the FP64 global-memory kernel), as does any
// pair whose potentials leave the exact range.  counter[0]: pairs still
// active; counter[1]: pairs moved to 1; counter[3]: pairs moved to 2;
// counter[4] (r.exit_at > 0, on-chip variant): pairs of this launch that
// stopped or moved.  Once it reaches r.exit_at, the pairs still iterating
// leave at their next 16-iteration check with their state saved (they stay
// active and the host runs them on in wider CTAs).
// The workspace descriptor of a CTA's pair: the kernel parameter itself (one
// workspace), or, in a launch over several workspaces, the pair's entry of
// w.groups copied once into shared memory (only that instantiation holds the
// copy).
template <bool MULTI> struct L2Desc {
    static __device__ __forceinline__ const SkWS& get(const SkWS& w, int) { return w; }
};
template <> struct L2Desc<true> {
    static __device__ __forceinline__ const SkWS& get(const SkWS& w, int code) {
        __shared__ SkWS Wsh;
        static_assert(sizeof(SkWS) % 4 == 0 && sizeof(SkWS) / 4 <= 128, "descriptor copy: one word per thread");
        const int* src = reinterpret_cast<const int*>(w.groups + (code >> 24));
        if ((int)threadIdx.x < (int)(sizeof(SkWS) / 4)) reinterpret_cast<int*>(&Wsh)[threadIdx.x] = src[threadIdx.x];
        __syncthreads();
        return Wsh;
    }
};

// MULTI = false: one workspace, its descriptor is the kernel parameter w
// (parameter-space reads, which the compiler can repeat instead of keeping
// the pair's pointers in registers); MULTI = true: a launch over several
// workspaces, the pair's descriptor copied from w.groups into shared memory.
template <int NT, bool GM, bool MULTI>
__global__ void __launch_bounds__(NT, (NT <= 128 ? 6 : (NT <= 256 ? 3 : (NT <= 512 ? 2 : 1))))
sk_lse2_kernel(SkWS w, SkRun r, int n_inner, int* counter, int smem_cap, size_t gcap, int gbits) {
    constexpr int NW = NT / 32;
    __shared__ L2Side S[2];
    __shared__ float redD[NW > L2_DLANES / 32 ? NW : L2_DLANES / 32];
    __shared__ long long redE[NW];
    __shared__ int wcnt[NW > L2_MAXCH ? NW : L2_MAXCH];
    __shared__ int cnt[4];
    __shared__ int range_flag, fits, leave;
    __shared__ L2Forms Fsh;   // the pair's forms (read at each half-step; not kept in registers)
    const bool can_leave = !GM && r.exit_at > 0;
    // the launch order maps this CTA to a pair, and, in a launch over several
    // workspaces (pairs of several grid sizes), to its workspace: code =
    // group << 24 | pair; the workspace descriptors are in device memory
    const int code = w.order ? w.order[blockIdx.x] : blockIdx.x, t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const SkWS& W = L2Desc<MULTI>::get(w, code);
    const int p = MULTI ? (code & 0xFFFFFF) : code;
    PairPtrs q = pair_ptrs(W, p);
    if (q.ic[IC_STATUS] != ST_ACTIVE || q.ic[IC_BIG] != (GM ? 1 : 0)) return;
    const int d = W.d, dp = W.dp, nA = q.ic[IC_NA], nB = q.ic[IC_NB];
    // gamma-continuation inside the launch: this pair's stage and gamma
    int stage = r.kstages > 0 ? q.ic[IC_STAGE] : 0;
    const double gamma_k = ldexp(W.gamma, 2 * stage);
    l2_compact(q.rpa, d, nullptr, &cnt[0], nullptr, wcnt);
    l2_compact(q.rpb, d, nullptr, &cnt[1], nullptr, wcnt);
    const int nrA = cnt[0], nrB = cnt[1];
    // the form of each half-step (the pairwise form runs on chip only)
    // (a pair that starts at a continuation stage without exact scaled units
    // takes the separable form there and switches at the first stage that has
    // them)
    L2Forms fm{false, false, false, false, false};
    if constexpr (!GM) {
        l2_compact(q.cpa, d, nullptr, &cnt[2], nullptr, wcnt);
        l2_compact(q.cpb, d, nullptr, &cnt[3], nullptr, wcnt);
        fm = l2_forms(nA, nB, nrA, nrB, cnt[2], cnt[3], d, r.form, l2_pw_calc(gamma_k, d, gbits, W.p).ok,
                      l2_pw_calc(W.gamma, d, gbits, W.p).ok, (size_t)smem_cap);
    }
    const bool pwU = fm.pwU, pwV = fm.pwV;   // at the starting stage (set-up only)
    if (t == 0) {
        Fsh = fm;
        if (GM)
            fits = l2_side_bytes(nA, nB, d, false) <= gcap &&
                   l2_table_bytes(nrA > nrB ? nrA : nrB, d) <= (size_t)smem_cap;
        else
            fits = l2_need(nA, nB, nrA, nrB, d, fm.rec, !(pwU && pwV)) <= (size_t)smem_cap;
        fits = fits && nA < 32768 && nB < 32768;   // cell indices are 16-bit (chl, packed row ranges)
    }
    __syncthreads();
    if (!fits) {
        if (GM && stage > 0) {
            // to the FP64 kernel, which runs the target gamma only: potentials
            // in the target's units (f / gamma = 4^stage f / gamma_k)
            const double sc = ldexp(1.0, 2 * stage);
            for (int e = t; e < nA; e += NT) q.phi[q.sa[e]] *= sc;
            for (int e = t; e < nB; e += NT) q.psi[q.sb[e]] *= sc;
            if (t == 0) { q.phi[W.n - 1] *= sc; q.psi[W.n - 1] *= sc; q.ic[IC_STAGE] = 0; }
        }
        if (t == 0) {
            q.ic[IC_BIG] = GM ? 2 : 1;
            atomicAdd(&counter[GM ? 3 : 1], 1);
            atomicAdd(&counter[0], 1);
            if (can_leave) atomicAdd(&counter[4], 1);
        }
        return;
    }
    unsigned char* gb = GM ? reinterpret_cast<unsigned char*>(q.L64) : nullptr;
    // ---- carve the per-side arrays, then the tables (byte offsets; in the GM
    // variant the side arrays start at gb and the tables at shared offset 0)
    uint32_t sp = 0;
    auto take = [&](size_t bytes) { const uint32_t r0 = sp; sp += (uint32_t)l2_al(bytes); return r0; };
    const int ns[2] = {nA, nB};
    for (int s = 0; s < 2; ++s) {
        const int n = ns[s];
        const uint32_t o_lw = take(24 * (size_t)n), o_rec = take(fm.rec ? 32 * (size_t)((n + 1) / 2) : 0),
                       o_w = take(4 * (size_t)n), o_rp = take(4 * (size_t)(d + 1));
        const uint32_t o_row = take(6 * (size_t)n), o_rows = take(6 * (size_t)d);
        if (t == 0) {
            L2Side& X = S[s];
            X.n = n;
            X.lw = o_lw; X.pot = o_lw + 8 * n; X.hin = o_lw + 16 * n; X.rec = o_rec;
            X.w = o_w; X.rp = o_rp;
            X.row = o_row; X.col = o_row + 2 * n; X.chl = o_row + 4 * n;
            X.rows = o_rows; X.cols = o_rows + 2 * d; X.colpos = o_rows + 4 * d;
        }
    }
    L2Consts K;
    if (GM) sp = 0;
    K.ct = take(8 * (size_t)(2 * d - 1));
    K.cdt = take(8 * (size_t)d);
    const int nrmax = nrA > nrB ? nrA : nrB;
    K.L1 = take((pwU && pwV) ? 0 : 8 * (size_t)L2_CW * nrmax);
    __syncthreads();
    const double gsc = ldexp(1.0, gbits);
    const double LOG2E = 1.4426950408889634;
    K.d = d;
    K.gsc = (float)gsc; K.ginv = (float)(1.0 / gsc);
    K.lim = (float)ldexp(1.0, 21 - gbits);   // |potential| bound keeping every sum of grid words exact
    K.escale = q.sc[SC_TOTAL] > 0 ? (float)(ldexp(1.0, 40) / q.sc[SC_TOTAL]) : 0.f;
    K.form = r.form;
    l2_pw_consts(K, gamma_k, d, gbits, W.p);
    K.pw_ok = K.pw_ok && (pwU || pwV);
    // ---- load
    {
        const int* lists[2] = {q.sa, q.sb};
        const double* lw[2] = {q.la, q.lb};
        const double* pot[2] = {q.phi, q.psi};
        const float* wt[2] = {q.am, q.bm};
        const int* rps[2] = {q.rpa, q.rpb};
        const int* cps[2] = {q.cpa, q.cpb};
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            L2Side& X = S[s];
            const int n = X.n;
            short* row = sdp<short, GM>(gb, X.row);
            short* col = sdp<short, GM>(gb, X.col);
            float2* xlw = sdp<float2, GM>(gb, X.lw);
            float2* xpot = sdp<float2, GM>(gb, X.pot);
            float2* xhin = sdp<float2, GM>(gb, X.hin);
            float* xw = sdp<float, GM>(gb, X.w);
            int* xrp = sdp<int, GM>(gb, X.rp);
            for (int e = t; e < n; e += NT) {
                const int c = lists[s][e];
                const int i = c / dp, j = c - i * dp;
                row[e] = (short)i; col[e] = (short)j;
                const float2 l2 = l2_split(lw[s][c] * LOG2E, gsc);
                const float2 p2 = l2_split(pot[s][c] * LOG2E, gsc);
                xlw[e] = l2; xpot[e] = p2;
                xhin[e] = make_float2(l2.x + p2.x, l2.y + p2.y);
                if (!GM && fm.rec) l2_rec_coord(X.rec, n, e, (float)i, (float)j);
                if (!GM && K.pw_ok)
                    l2_rec_put(X.rec, e, l2_pw_record(make_float2(l2.x + p2.x, l2.y + p2.y), (float)i, (float)j, K));
                xw[e] = wt[s][c];
            }
            if (!GM && fm.rec && (n & 1) && t == 0) {   // an odd side's last slot: a zero term
                l2_rec_put(X.rec, n, make_float2(-INFINITY, 0.f));
                l2_rec_coord(X.rec, n, n, 0.f, 0.f);
            }
            for (int i = t; i <= d; i += NT) xrp[i] = rps[s][i];
            l2_compact(rps[s], d, sdp<short, GM>(gb, X.rows), &cnt[2], nullptr, wcnt);
            l2_compact(cps[s], d, sdp<short, GM>(gb, X.cols), &cnt[3], sdp<short, GM>(gb, X.colpos), wcnt);
            l2_sort_rows(sdp<short, GM>(gb, X.rows), cnt[2], xrp);
            {
                // row pointers -> one word per non-empty row (stage 1 loads one value)
                const short* xrows = sdp<short, GM>(gb, X.rows);
                const int nr = cnt[2];
                int v = 0;
                if (t < nr) { const int k = xrows[t]; v = xrp[k] | (xrp[k + 1] << 16); }
                __syncthreads();
                if (t < nr) xrp[t] = v;
                __syncthreads();
            }
            if (t == 0) {
                X.nr = cnt[2]; X.nc = cnt[3]; X.nch = (cnt[3] + L2_CW - 1) / L2_CW;
                const double wD = q.sc[s == 0 ? SC_AD : SC_BD];
                X.wD = (float)wD;
                X.lwD = wD > 0 ? l2_split(log(wD) * LOG2E, gsc) : make_float2(-INFINITY, 0.f);
                X.potD = l2_split(pot[s][W.n - 1] * LOG2E, gsc);
                X.hinD = wD > 0 ? make_float2(X.lwD.x + X.potD.x, X.lwD.y + X.potD.y) : make_float2(-INFINITY, 0.f);
            }
            __syncthreads();
        }
    }
    l2_tables<NT>(smp<float2>(K.ct), smp<float2>(K.cdt), d, gamma_k, W.p, gsc);
    if (t == 0) range_flag = 0;
    __syncthreads();
    l2_chunks<GM>(S[0], wcnt, gb);
    l2_chunks<GM>(S[1], wcnt, gb);
    const float tolf = (float)r.tol, stage_tolf = (float)r.stage_tol;
    int iters = q.ic[IC_ITERS];
    float errf = (float)q.sc[SC_ERR];
    int status = ST_ACTIVE;
    bool moved = false;
    for (int it = 0; it < n_inner; ++it) {
        long long errq = 0;
        bool errbad = false;
        // u-update (phi from psi), then v-update (psi from phi, err_t): one copy
        // of the half-step code serves both (instruction cache)
#pragma unroll 1
        for (int hs = 0; hs < 2; ++hs) {
            if (!GM && K.pw_ok && (hs == 0 ? Fsh.pwU : Fsh.pwV))
                l2_half_pw<NT>(S[1 - hs], S[hs], K, hs == 1, errq, errbad, &range_flag, hs == 0);
            else
                l2_half<NT, GM>(S[1 - hs], S[hs], K, hs == 1, errq, errbad, redD, &range_flag, gb);
        }
        errq = warp_sum(errq);
        if (lane == 0) redE[wid] = errq;
        // written next to redE and read after the same barrier (the next write
        // is behind the barriers of the next iteration's half-steps); the
        // barrier also closes a pairwise v-update, whose results the next
        // iteration reads
        if (t == 0) leave = can_leave && (it & 15) == 15 && *(volatile int*)&counter[4] >= r.exit_at;
        const int bad = __syncthreads_or(errbad);
        long long e = 0;
        for (int k = 0; k < NW; ++k) e += redE[k];
        errf = bad ? INFINITY : (float)((double)e * 0x1p-40);
        ++iters;
        if (range_flag) { moved = true; break; }
        // a coarse stage that reached its tolerance moves on (never "converged")
        const bool stage_done = stage > 0 && errf <= stage_tolf;
        if (!stage_done && r.tol > 0 && errf <= tolf) { status = ST_CONVERGED; break; }
        if (iters >= r.max_iter) { status = ST_MAXITER; break; }
        if (!isfinite(errf)) { status = ST_RANGE; break; }
        if (stage_done) {
            --stage;
            {
                // the pairwise constants of the new gamma first: the stage step
                // rebuilds the records with them.  A pair takes the pairwise
                // form from the first stage with exact scaled units on (a
                // smaller gamma only raises n1, so it never turns off)
                const bool was = K.pw_ok;
                const L2Forms f = Fsh;
                l2_pw_consts(K, ldexp(W.gamma, 2 * stage), d, gbits, W.p);
                K.pw_ok = K.pw_ok && f.rec;
                __syncthreads();   // every thread has read Fsh
                if (t == 0) {
                    if (was && !K.pw_ok) range_flag = 1;   // not reached; the FP64 kernel would take over
                    Fsh.pwU = f.ruleU && K.pw_ok;
                    Fsh.pwV = f.ruleV && K.pw_ok;
                }
            }
            l2_next_stage<NT, GM>(S, K, ldexp(W.gamma, 2 * stage), W.p, d, &range_flag, gb);
            if (range_flag) { moved = true; break; }
        }
        if (leave) break;   // status stays ST_ACTIVE: relaunched in a wider CTA
    }
    // ---- store the potentials (FP64, natural units); the pair's arrays come
    // anew from the shared descriptor (not kept in registers across the loop)
    const double LN2 = 0.6931471805599453;
    const size_t Nn = (size_t)W.n, Mm = (size_t)W.dp * W.dp;
    double* s_phi = W.phi + p * Nn;
    double* s_psi = W.psi + p * Nn;
    const int* s_sa = W.sa + p * Mm;
    const int* s_sb = W.sb + p * Mm;
    double* s_sc = W.sc + (size_t)p * SC_N;
    int* s_ic = W.ic + (size_t)p * IC_N;
    // a pair handed on to a wider CTA keeps its stage; one that stops (or moves
    // to the FP64 kernel) is stored in the target gamma's units
    const bool keep_stage = status == ST_ACTIVE && !moved;
    const double units = LN2 * (keep_stage ? 1.0 : ldexp(1.0, 2 * stage));
    for (int s = 0; s < 2; ++s) {
        const L2Side& X = S[s];
        double* pot = s == 0 ? s_phi : s_psi;
        const int* list = s == 0 ? s_sa : s_sb;
        const float2* xpot = sdp<float2, GM>(gb, X.pot);
        for (int e = t; e < X.n; e += NT) pot[list[e]] = ((double)xpot[e].x + (double)xpot[e].y) * units;
        if (t == 0) pot[Nn - 1] = ((double)X.potD.x + (double)X.potD.y) * units;
    }
    if (t == 0 && r.kstages > 0) s_ic[IC_STAGE] = keep_stage ? stage : 0;
    if (t == 0) {
        s_sc[SC_ERR] = (double)errf;
        s_ic[IC_ITERS] = iters;
        if (moved) {
            // the exact-range guard tripped: the FP64 global-memory kernel takes the pair over
            s_ic[IC_BIG] = 2;
            atomicAdd(&counter[3], 1);
            atomicAdd(&counter[0], 1);
        } else {
            s_ic[IC_STATUS] = status;
            if (status == ST_ACTIVE) atomicAdd(&counter[0], 1);
        }
        if (can_leave && (moved || status != ST_ACTIVE)) atomicAdd(&counter[4], 1);
    }
}

// gamma-continuation inside the iteration kernel: every pair starts at stage K.
__global__ void sk_set_stage_kernel(SkWS w, int K) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < w.P) w.ic[(size_t)p * IC_N + IC_STAGE] = K;
}

cudaError_t sk_launch_set_stage(const SkWS& w, int K, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_set_stage_kernel<<<(w.P + 255) / 256, 256, 0, s>>>(w, K);
    return cudaGetLastError();
}

// Maximum shared-memory need over the active on-chip pairs (one thread per pair).
__global__ void sk_lse2_need_kernel(SkWS w, int* max_need, int form, size_t cap) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= w.P) return;
    PairPtrs q = pair_ptrs(w, p);
    if (q.ic[IC_STATUS] != ST_ACTIVE || q.ic[IC_BIG]) return;
    int nrA = 0, nrB = 0, ncA = 0, ncB = 0;
    for (int i = 0; i < w.d; ++i) {
        nrA += q.rpa[i + 1] > q.rpa[i];
        nrB += q.rpb[i + 1] > q.rpb[i];
        ncA += q.cpa[i + 1] > q.cpa[i];
        ncB += q.cpb[i + 1] > q.cpb[i];
    }
    const int nA = q.ic[IC_NA], nB = q.ic[IC_NB];
    const int gb = l2_grid_bits(w.gamma);
    const L2Forms fm = l2_forms(nA, nB, nrA, nrB, ncA, ncB, w.d, form,
                                l2_pw_calc(ldexp(w.gamma, 2 * q.ic[IC_STAGE]), w.d, gb, w.p).ok,
                                l2_pw_calc(w.gamma, w.d, gb, w.p).ok, cap);
    const size_t need = l2_need(nA, nB, nrA, nrB, w.d, fm.rec, !(fm.pwU && fm.pwV));
    atomicMax(max_need, (int)(need > 0x7fffffff ? 0x7fffffff : need));
    if (!(fm.pwU && fm.pwV)) atomicAdd(max_need + 1, 1);
}

size_t sk_lse2_smem_cap();
cudaError_t sk_launch_lse2_need(const SkWS& w, int* max_need, int form, cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    sk_lse2_need_kernel<<<(w.P + 255) / 256, 256, 0, s>>>(w, max_need, form, sk_lse2_smem_cap());
    return cudaGetLastError();
}

// Grid exponent G for a gamma.  Multiples of 2^-G below 2^(24-G) are exact in
// FP32, so a difference of two grid words is exact whenever its result is
// below that.  Potentials are kept below 2^(21-G) (the kernel's guard) and
// 2^(23-G) covers eight times the largest cost/gamma in log2 units plus a
// margin for log-weights, which bounds every argument the kernel forms.
// Returns -1 when gamma is too small for a grid of at least 2^-4 (the caller
// then uses the FP64-argument kernels).
int sk_lse2_grid_bits(double gamma) { return l2_grid_bits(gamma); }

size_t sk_lse2_smem_cap() {
    int dev = 0, cap = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return (size_t)cap - 1024;   // the widest kernel's static shared memory (<= 1 KB)
}

// Dynamic shared memory an instantiation may request: the per-block opt-in
// limit less its own static shared memory.
template <class F>
static size_t lse2_dyn_cap(F* kernel) {
    int dev = 0, cap = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return sk_lse2_smem_cap();
    return (size_t)cap - fa.sharedSizeBytes;
}

template <int NT, bool GM, bool MULTI>
static cudaError_t launch_lse2_v(const SkWS& w, SkRun r, int n_inner, int* counter, size_t smem, size_t gcap,
                                 int gbits, cudaStream_t s) {
    static std::atomic<size_t> configured{0};
    const size_t cap = lse2_dyn_cap(sk_lse2_kernel<NT, GM, MULTI>);
    if (configured != cap) {
        cudaError_t e = cudaFuncSetAttribute(sk_lse2_kernel<NT, GM, MULTI>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
        if (e != cudaSuccess) return e;
        configured = cap;
    }
    if (smem > cap) smem = cap;
    sk_lse2_kernel<NT, GM, MULTI><<<w.P, NT, smem, s>>>(w, r, n_inner, counter, (int)smem, gcap, gbits);
    return cudaGetLastError();
}
template <int NT, bool GM>
static cudaError_t launch_lse2(const SkWS& w, SkRun r, int n_inner, int* counter, size_t smem, size_t gcap, int gbits,
                               cudaStream_t s) {
    if (!GM && w.ngroups > 1) return launch_lse2_v<NT, false, true>(w, r, n_inner, counter, smem, gcap, gbits, s);
    return launch_lse2_v<NT, GM, false>(w, r, n_inner, counter, smem, gcap, gbits, s);
}

cudaError_t sk_launch_lse2(const SkWS& w, SkRun r, int n_inner, int* counter, size_t smem, int gbits, int threads,
                           cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    switch (threads) {
        case 128:   // needs d <= 128 (one thread per grid row while loading)
            if (w.d > 128) return cudaErrorInvalidValue;
            return launch_lse2<128, false>(w, r, n_inner, counter, smem, 0, gbits, s);
        case 256: return launch_lse2<256, false>(w, r, n_inner, counter, smem, 0, gbits, s);
        case 512: return launch_lse2<512, false>(w, r, n_inner, counter, smem, 0, gbits, s);
        case 1024: return launch_lse2<1024, false>(w, r, n_inner, counter, smem, 0, gbits, s);
        default: return cudaErrorInvalidValue;
    }
}

// Global-memory variant for the pairs with IC_BIG == 1 (512 threads); the
// side arrays of a pair may use up to `gcap` bytes of its L64 scratch
// (SIZE_MAX: all of it).
cudaError_t sk_launch_lse2_gm(const SkWS& w, SkRun r, int n_inner, int* counter, int gbits, size_t gcap,
                              cudaStream_t s) {
    if (w.P == 0) return cudaSuccess;
    const size_t l64 = sizeof(double) * 2 * (size_t)w.dp * w.dp;
    return launch_lse2<512, true>(w, r, n_inner, counter, l2_table_bytes(w.d, w.d), gcap < l64 ? gcap : l64, gbits,
                                  s);
}
