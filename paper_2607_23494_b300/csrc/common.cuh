// Shared device helpers for the field-window estimator kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hermes {

// Size of the shared twiddle table e^{-2 pi i j / TW}; every transform length
// used here divides TW.
constexpr int TW = 2048;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Signed frequency of FFT index k on an N-point axis: 0..N/2-1, -N/2..-1.
__device__ __forceinline__ int signed_freq(int k, int N) { return k < (N >> 1) ? k : k - N; }

// Warp + block reduction of one double per thread; result valid in thread 0.
// `red` must hold at least blockDim.x/32 doubles.  Contains __syncthreads.
__device__ __forceinline__ double block_sum_double(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int i = 0; i < nw; ++i) s += red[i];
    }
    return s;
}

}  // namespace hermes
