// raster.cu -- Sec. 3 "Discretization": bin diagram points into d x d grid
// cells with integer counts.  The cell of (birth, death) is (floor(birth*d),
// floor(death*d)) computed in IEEE FP64 and clamped to d-1, so the closed edge
// at 1 belongs to the last cell (supplementary "Error control due to
// discretization" snaps points to (floor(xd)/d, floor(yd)/d)).
#include "pd_common.cuh"
#include "pd_internal.h"

// One thread per point; the owning diagram is found by binary search over the
// CSR offsets.  Counts are integers, so atomic accumulation order does not
// matter and the result is bit-exact.
__global__ void pd_raster_kernel(const double* __restrict__ birth, const double* __restrict__ death,
                                 const int64_t* __restrict__ offsets, int B, int d, int64_t npts,
                                 uint32_t* __restrict__ hist, int* __restrict__ bad) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npts;
         p += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = B - 1;
        while (lo < hi) {  // largest b with offsets[b] <= p
            int mid = (lo + hi + 1) >> 1;
            if (offsets[mid] <= p) lo = mid; else hi = mid - 1;
        }
        const double s = birth[p], t = death[p];
        if (!(s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0 && s <= t)) {
            atomicExch(bad, 1);
            continue;
        }
        long i = (long)floor(s * (double)d), j = (long)floor(t * (double)d);
        if (i > d - 1) i = d - 1;
        if (j > d - 1) j = d - 1;
        atomicAdd(&hist[(size_t)lo * d * d + (size_t)i * d + j], 1u);
    }
}

__global__ void pd_mass_kernel(const int64_t* __restrict__ offsets, int B, uint32_t* __restrict__ mass,
                               int* __restrict__ bad) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        int64_t n = offsets[b + 1] - offsets[b];
        if (n < 0 || n > 0xffffffffLL) atomicExch(bad, 1);
        mass[b] = (uint32_t)n;
    }
}

cudaError_t pd_launch_raster(const double* birth, const double* death, const int64_t* offsets, int B,
                             int d, int64_t npts, uint32_t* hist, uint32_t* mass, int* bad,
                             cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)B * d * d, s);
    if (e != cudaSuccess) return e;
    if (B > 0) {
        pd_mass_kernel<<<(B + 255) / 256, 256, 0, s>>>(offsets, B, mass, bad);
        if (npts > 0) {
            int64_t blocks = (npts + 255) / 256;
            if (blocks > 152 * 32) blocks = 152 * 32;
            pd_raster_kernel<<<(int)blocks, 256, 0, s>>>(birth, death, offsets, B, d, npts, hist, bad);
        }
    }
    return cudaGetLastError();
}
