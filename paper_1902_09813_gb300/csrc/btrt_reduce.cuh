// btrt_reduce.cuh -- the library's one fixed-order FP64 sum of a pitched array.
//
// btrt_mass, the steady-state residual, the D3Q19 mass and btrt_phi_sum_static
// all sum with these two kernels, so their results agree bitwise for the same
// values: block b of a kRedBlocks grid owns rows b, b + kRedBlocks, ...; its
// threads stride over the first nx values of each row and meet in a fixed
// shared-memory tree; one block then sums the kRedBlocks partials the same way.
#pragma once

#include <cuda_runtime.h>

namespace btrt {

constexpr int kRedBlocks = 1024;     // fixed grid of the FP64 reductions (deterministic order)
constexpr int kRedThreads = 256;

// Per-block partial sums of the first nx values of `rows` rows, `pitch` elements apart.
template <typename Real>
__global__ void __launch_bounds__(kRedThreads)
rows_sum_partials(const Real *__restrict__ a, int nx, long long rows, long long pitch, double *partials) {
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x)
        for (int x = threadIdx.x; x < nx; x += blockDim.x) acc += static_cast<double>(a[r * pitch + x]);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kRedThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// Sum of n partials into *out (one block of kRedThreads threads).  A template so
// that every translation unit that launches it may define it.
template <int NT>
__global__ void __launch_bounds__(NT) sum_partials(const double *partials, int n, double *out) {
    __shared__ double sh[NT];
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partials[k];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// Enqueue both kernels: partials[0 .. kRedBlocks) are overwritten, the sum lands in *out.
template <typename Real>
inline cudaError_t enqueue_rows_sum(const Real *a, int nx, long long rows, long long pitch, double *partials,
                                    double *out, cudaStream_t s) {
    rows_sum_partials<Real><<<kRedBlocks, kRedThreads, 0, s>>>(a, nx, rows, pitch, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    sum_partials<kRedThreads><<<1, kRedThreads, 0, s>>>(partials, kRedBlocks, out);
    return cudaGetLastError();
}

}  // namespace btrt
