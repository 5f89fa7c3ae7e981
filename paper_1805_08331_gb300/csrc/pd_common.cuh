// pd_common.cuh -- device helpers shared by the library's kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#ifndef PD_CTA_THREADS
#define PD_CTA_THREADS 256
#endif

// Grid cost of Sec. 3 "Convolutions" with p = 2 in physical units on [0,1]^2:
// the 1-D factor c_ik = ((i-k)/d)^2, so that C((i,j),(k,l)) = c_ik + c_jl.
__device__ __forceinline__ double pd_c1(int i, int k, int d) {
    double t = (double)(i - k) / (double)d;
    return t * t;
}
// Cost of grid cell (i,j) to the diagonal bin: squared distance of (i/d, j/d)
// to its orthogonal projection on the diagonal, (j-i)^2 / (2 d^2) (Prop. 1).
__device__ __forceinline__ double pd_cdiag(int i, int j, int d) {
    double t = (double)(j - i) / (double)d;
    return 0.5 * t * t;
}

// The same costs for a ground cost ||.||_p^p (p >= 1): c_ik = |i-k|^p / d^p,
// and the cell-to-diagonal cost ||x - pi(x)||_p^p = 2 |(j-i) / (2d)|^p with pi
// the orthogonal projection onto the diagonal.  p = 2 is pd_c1 / pd_cdiag.
__device__ __forceinline__ double pd_c1p(int i, int k, int d, double p) {
    if (p == 2.0) return pd_c1(i, k, d);
    return pow(fabs((double)(i - k)) / (double)d, p);
}
__device__ __forceinline__ double pd_cdiagp(int i, int j, int d, double p) {
    if (p == 2.0) return pd_cdiag(i, j, d);
    return 2.0 * pow(fabs((double)(j - i)) / (2.0 * (double)d), p);
}

// exp of an FP64 exponent evaluated in FP32 after clamping to the finite FP32
// range; entries below ~1e-38 become 0 and large ones saturate (never inf).
__device__ __forceinline__ float pd_exp_clamped(double arg) {
    float a = (float)fmin(arg, 88.0);
    return (a < -104.0f) ? 0.0f : expf(a);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum (all threads receive the result).  `sh` needs 32 slots.
template <typename T>
__device__ T block_sum(T v, T* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
    if (wid == 0) r = warp_sum(r);
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}
template <typename T>
__device__ T block_max(T v, T* sh, T lowest) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T r = (threadIdx.x < nw) ? sh[threadIdx.x] : lowest;
    if (wid == 0) r = warp_max(r);
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}
