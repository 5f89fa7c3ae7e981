// outer.cu -- kernels of the barycenter (Alg. 2) and k-means (Sec. 5) loops.
//
// Both loops run batched Sinkhorn solves (Alg. 1) between a real-valued
// measure z (barycenter / centroid) and integer histograms a_i, as the pairs
// (z + R a_i, a_i + R z) of Alg. 2, and then apply the gradient of the
// smoothed energy (the gradient proposition of Sec. 4):
//     grad(x) = gamma log u_i(x) + gamma log v_i(Delta),  summed over i,
// where u_i = z exp(f_i/gamma) on the z side and v_i(Delta) = |z| exp(g_i(Delta)/gamma)
// (R^T maps the Delta value to a constant on the grid), so
//     gamma log u_i(x) + gamma log v_i(Delta) = gamma log z(x) + f_i(x) + gamma log|z| + g_i(Delta).
// The gradient is averaged over the diagrams (the energy is the mean) and the
// multiplicative update of Alg. 2, z <- z exp(-lambda grad), is applied where
// z > 0.  Sums over diagrams are FP64 in a fixed order (deterministic).
#include "pd_common.cuh"
#include <stdint.h>

// z = uniform measure above the diagonal: every cell with j >= i gets
// (mean histogram mass) / (d (d+1) / 2).
__global__ void bary_init_uniform_kernel(double* __restrict__ z, const uint32_t* __restrict__ mass, int N, int d) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s += (double)mass[i];
    s = block_sum(s, sh);
    const double per = (s / N) / (d * (d + 1) / 2.0);
    for (int x = threadIdx.x; x < d * d; x += blockDim.x) z[x] = ((x % d) >= (x / d)) ? per : 0.0;
}

// |z_c| for every measure c (one block per measure).
__global__ void measure_mass_kernel(const double* __restrict__ z, int d, double* __restrict__ out) {
    __shared__ double sh[32];
    const double* zc = z + (size_t)blockIdx.x * d * d;
    double s = 0.0;
    for (int x = threadIdx.x; x < d * d; x += blockDim.x) s += zc[x];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// Gradient of measure c at cell x, split as
//     mean_i grad_i(x) = gamma log z_c(x) + gamma log|z_c| + (sum_i (f_i(x) + g_i(Delta))) / m,
// the sum over the m diagrams i owned by c taken in diagram order.  The one-GPU
// step and the sharded form (per-shard sums added across ranks, then applied)
// use these same two helpers.
__device__ __forceinline__ double bary_fg_sum(const double* __restrict__ f, const double* __restrict__ g,
                                              const int32_t* __restrict__ owner, int N, int c, int x, int D,
                                              int& m) {
    const int n1 = D + 1;
    double s = 0.0;
    m = 0;
    for (int i = 0; i < N; ++i) {
        if (owner && owner[i] != c) continue;
        s += f[(size_t)i * n1 + x] + g[(size_t)i * n1 + D];
        ++m;
    }
    return s;
}
__device__ __forceinline__ double bary_update(double zx, double zmass, double fgsum, double m, double gamma,
                                              double lambda) {
    return zx * exp(-lambda * ((gamma * log(zx) + gamma * log(zmass)) + fgsum / m));
}

// Multiplicative gradient step for k measures at once.  Diagram n belongs to
// measure owner[n] (owner == NULL: all to measure 0); f, g are the potentials of
// the pair (z_owner[n] + R a_n, a_n + R z_owner[n]) with n = d*d+1 entries per pair.
// One thread per (measure c, cell x).
__global__ void bary_step_kernel(double* __restrict__ z, const double* __restrict__ zmass,
                                 const double* __restrict__ f, const double* __restrict__ g,
                                 const int32_t* __restrict__ owner, int N, int k, int d, double gamma,
                                 double lambda) {
    const int D = d * d;
    const int64_t tot = (int64_t)k * D;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / D), x = (int)(e % D);
        double* zc = z + (size_t)c * D;
        const double zx = zc[x];
        if (!(zx > 0.0)) continue;
        int m;
        const double s = bary_fg_sum(f, g, owner, N, c, x, D, m);
        if (m > 0) zc[x] = bary_update(zx, zmass[c], s, (double)m, gamma, lambda);
    }
}

// Sharded form, first half: gsum[c][x] = sum over this shard's diagrams owned
// by c of f_i(x) + g_i(Delta) (0 where z_c(x) <= 0), count[c] = their number.
__global__ void bary_grad_kernel(const double* __restrict__ z, const double* __restrict__ f,
                                 const double* __restrict__ g, const int32_t* __restrict__ owner, int N, int k,
                                 int d, double* __restrict__ gsum, double* __restrict__ count) {
    const int D = d * d;
    const int64_t tot = (int64_t)k * D;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / D), x = (int)(e % D);
        int m;
        const double sum = z[e] > 0.0 ? bary_fg_sum(f, g, owner, N, c, x, D, m) : 0.0;
        gsum[e] = sum;
        if (x == 0) {
            int mc = 0;
            for (int i = 0; i < N; ++i) mc += (!owner || owner[i] == c);
            count[c] = (double)mc;
        }
    }
}

// Sharded form, second half (one block of 512 threads per measure): |z_c| in
// the same order as measure_mass_kernel, then the multiplicative update from
// the summed gsum and count.
__global__ void bary_apply_kernel(double* __restrict__ z, const double* __restrict__ gsum,
                                  const double* __restrict__ count, int d, double gamma, double lambda) {
    __shared__ double sh[32];
    const int D = d * d, c = blockIdx.x;
    double* zc = z + (size_t)c * D;
    double s = 0.0;
    for (int x = threadIdx.x; x < D; x += blockDim.x) s += zc[x];
    const double zmass = block_sum(s, sh);
    const double m = count[c];
    if (!(m > 0.0)) return;
    for (int x = threadIdx.x; x < D; x += blockDim.x) {
        const double zx = zc[x];
        if (zx > 0.0) zc[x] = bary_update(zx, zmass, gsum[(size_t)c * D + x], m, gamma, lambda);
    }
}

// cost_sum[c] = sum of cost[n] over the diagrams n owned by c (diagram order).
__global__ void cost_sum_kernel(const double* __restrict__ cost, const int32_t* __restrict__ owner, int N, int k,
                                double* __restrict__ out) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < N; ++i)
            if (!owner || owner[i] == c) s += cost[i];
        out[c] = s;
    }
}

// energy[slot] = mean of cost[0..N)  (one block, fixed order).
__global__ void mean_kernel(const double* __restrict__ cost, int N, double* __restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s += cost[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = s / N;
}

// k-means assignment: assign[n] = argmin_c cost[n*k + c] (ties -> lowest c);
// objective = sum_n min_c cost (one block, fixed order).
__global__ void km_assign_kernel(const double* __restrict__ cost, int N, int k, int32_t* __restrict__ assign,
                                 double* __restrict__ objective) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        int best = 0;
        double bv = cost[(size_t)n * k];
        for (int c = 1; c < k; ++c) {
            double v = cost[(size_t)n * k + c];
            if (v < bv) { bv = v; best = c; }
        }
        assign[n] = best;
        s += bv;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0 && objective) *objective = s;
}

// centroid c <- histogram idx[c] as real weights.
__global__ void km_seed_kernel(const uint32_t* __restrict__ hist, const int32_t* __restrict__ idx, int k, int d,
                               double* __restrict__ z) {
    const int D = d * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)k * D;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / D), x = (int)(e % D);
        z[e] = (double)hist[(size_t)idx[c] * D + x];
    }
}

// pairs for the assignment batch: p = n*k + c -> (n, c)
__global__ void km_pairs_kernel(int N, int k, int32_t* __restrict__ pairs) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < (int64_t)N * k;
         p += (int64_t)gridDim.x * blockDim.x) {
        pairs[2 * p] = (int32_t)(p / k);
        pairs[2 * p + 1] = (int32_t)(p % k);
    }
}

// flag = 1 if some owner[n] is outside [0, k)
__global__ void check_owner_kernel(const int32_t* __restrict__ owner, int N, int k, int* __restrict__ flag) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x)
        if (owner[n] < 0 || owner[n] >= k) atomicOr(flag, 1);
}

// pairs for the centroid batch: p = n -> (owner[n], n)   (owner NULL: (0, n))
__global__ void owner_pairs_kernel(const int32_t* __restrict__ owner, int N, int32_t* __restrict__ pairs) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N; p += gridDim.x * blockDim.x) {
        pairs[2 * p] = owner ? owner[p] : 0;
        pairs[2 * p + 1] = p;
    }
}

// ---------------------------------------------------------------------------
cudaError_t outer_bary_init_uniform(double* z, const uint32_t* mass, int N, int d, cudaStream_t s) {
    bary_init_uniform_kernel<<<1, 1024, 0, s>>>(z, mass, N, d);
    return cudaGetLastError();
}
cudaError_t outer_measure_mass(const double* z, int k, int d, double* out, cudaStream_t s) {
    measure_mass_kernel<<<k, 512, 0, s>>>(z, d, out);
    return cudaGetLastError();
}
cudaError_t outer_bary_step(double* z, const double* zmass, const double* f, const double* g, const int32_t* owner,
                            int N, int k, int d, double gamma, double lambda, cudaStream_t s) {
    int64_t tot = (int64_t)k * d * d;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    bary_step_kernel<<<blocks, 256, 0, s>>>(z, zmass, f, g, owner, N, k, d, gamma, lambda);
    return cudaGetLastError();
}
cudaError_t outer_bary_grad(const double* z, const double* f, const double* g, const int32_t* owner, int N, int k,
                            int d, double* gsum, double* count, cudaStream_t s) {
    int64_t tot = (int64_t)k * d * d;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    bary_grad_kernel<<<blocks, 256, 0, s>>>(z, f, g, owner, N, k, d, gsum, count);
    return cudaGetLastError();
}
cudaError_t outer_bary_apply(double* z, const double* gsum, const double* count, int k, int d, double gamma,
                             double lambda, cudaStream_t s) {
    bary_apply_kernel<<<k, 512, 0, s>>>(z, gsum, count, d, gamma, lambda);
    return cudaGetLastError();
}
cudaError_t outer_cost_sum(const double* cost, const int32_t* owner, int N, int k, double* out, cudaStream_t s) {
    cost_sum_kernel<<<(k + 127) / 128, 128, 0, s>>>(cost, owner, N, k, out);
    return cudaGetLastError();
}
cudaError_t outer_mean(const double* cost, int N, double* out, cudaStream_t s) {
    mean_kernel<<<1, 1024, 0, s>>>(cost, N, out);
    return cudaGetLastError();
}
cudaError_t outer_km_assign(const double* cost, int N, int k, int32_t* assign, double* objective, cudaStream_t s) {
    km_assign_kernel<<<1, 1024, 0, s>>>(cost, N, k, assign, objective);
    return cudaGetLastError();
}
cudaError_t outer_km_seed(const uint32_t* hist, const int32_t* idx, int k, int d, double* z, cudaStream_t s) {
    km_seed_kernel<<<152, 256, 0, s>>>(hist, idx, k, d, z);
    return cudaGetLastError();
}
cudaError_t outer_km_pairs(int N, int k, int32_t* pairs, cudaStream_t s) {
    km_pairs_kernel<<<152, 256, 0, s>>>(N, k, pairs);
    return cudaGetLastError();
}
cudaError_t outer_check_owner(const int32_t* owner, int N, int k, int* flag, cudaStream_t s) {
    int blocks = (N + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    check_owner_kernel<<<blocks, 256, 0, s>>>(owner, N, k, flag);
    return cudaGetLastError();
}
cudaError_t outer_owner_pairs(const int32_t* owner, int N, int32_t* pairs, cudaStream_t s) {
    owner_pairs_kernel<<<(N + 255) / 256, 256, 0, s>>>(owner, N, pairs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Entropic sharpening (Solomon et al.; the paper's Sec. 4 names it as the way
// to spikier barycenters).  The target entropy H0 is the largest entropy of
// the normalised input histograms; a measure z whose normalised entropy exceeds
// H0 becomes |z| w^beta / sum w^beta (w = z / |z|) with the beta >= 1 at which
// that entropy equals H0 (it decreases with beta; bisection, FP64).

// H0 = max over the input histograms of log m - (sum h log h) / m  (one block per diagram)
__global__ void input_entropy_kernel(const uint32_t* __restrict__ hist, int d, unsigned long long* __restrict__ H0bits) {
    __shared__ double sh[32];
    const int D = d * d;
    const uint32_t* h = hist + (size_t)blockIdx.x * D;
    double m = 0.0, s = 0.0;
    for (int x = threadIdx.x; x < D; x += blockDim.x) {
        const double v = (double)h[x];
        if (v > 0) { m += v; s += v * log(v); }
    }
    m = block_sum(m, sh);
    s = block_sum(s, sh);
    if (threadIdx.x == 0 && m > 0) {
        const double H = fmax(log(m) - s / m, 0.0);   // >= 0, so its bits order like the values
        atomicMax(H0bits, (unsigned long long)__double_as_longlong(H));
    }
}

// entropy of w^beta / sum w^beta with w = z / |z|, from the powers of v = z / zmax
// (the same normalised measure; the largest term is 1, so the sum cannot
// underflow for large beta).  Block reduction; every thread gets the value.
__device__ double sharp_entropy(const double* z, int D, double zmax, double beta, double* sh) {
    double S = 0.0, T = 0.0;
    for (int x = threadIdx.x; x < D; x += blockDim.x) {
        if (!(z[x] > 0)) continue;
        const double lv = log(z[x] / zmax);
        const double vb = exp(beta * lv);
        S += vb;
        T += vb * lv;
    }
    S = block_sum(S, sh);
    T = block_sum(T, sh);
    return log(S) - beta * T / S;
}

// one block per measure c: sharpen z_c in place when its entropy exceeds H0
__global__ void sharpen_kernel(double* __restrict__ z, int d, const unsigned long long* __restrict__ H0bits) {
    __shared__ double sh[32];
    const int D = d * d;
    double* zc = z + (size_t)blockIdx.x * D;
    const double H0 = __longlong_as_double((long long)*H0bits);
    double zm = 0.0, zmax = 0.0;
    for (int x = threadIdx.x; x < D; x += blockDim.x) { zm += zc[x]; zmax = fmax(zmax, zc[x]); }
    zm = block_sum(zm, sh);
    zmax = block_max(zmax, sh, 0.0);
    if (!(zm > 0) || !(sharp_entropy(zc, D, zmax, 1.0, sh) > H0)) return;
    double lo = 1.0, hi = 2.0;
    while (sharp_entropy(zc, D, zmax, hi, sh) > H0 && hi < 1e6) { lo = hi; hi *= 2.0; }
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sharp_entropy(zc, D, zmax, mid, sh) > H0) lo = mid; else hi = mid;
    }
    const double beta = 0.5 * (lo + hi);
    double S = 0.0;
    for (int x = threadIdx.x; x < D; x += blockDim.x)
        if (zc[x] > 0) S += exp(beta * log(zc[x] / zmax));
    S = block_sum(S, sh);
    for (int x = threadIdx.x; x < D; x += blockDim.x)
        if (zc[x] > 0) zc[x] = zm * exp(beta * log(zc[x] / zmax)) / S;
}

cudaError_t outer_input_entropy(const uint32_t* hist, int N, int d, unsigned long long* H0bits, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(H0bits, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    input_entropy_kernel<<<N, 256, 0, s>>>(hist, d, H0bits);
    return cudaGetLastError();
}
cudaError_t outer_sharpen(double* z, int k, int d, const unsigned long long* H0bits, cudaStream_t s) {
    sharpen_kernel<<<k, 256, 0, s>>>(z, d, H0bits);
    return cudaGetLastError();
}
