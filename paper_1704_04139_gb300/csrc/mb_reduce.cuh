// mb_reduce.cuh -- deterministic FP64 reductions: a fixed grid of RED_BLOCKS
// blocks, per-thread FP64 partials, warp-shuffle and shared-memory block
// reduction into per-block partials, then one block per result.
#pragma once
#include "mb_internal.h"

namespace mb {

// Entry of a kernel that may be launched with programmatic dependent launch
// (programmatic stream serialization): such a launch can be scheduled before
// its predecessor in the stream has finished, so the kernel first waits until
// that predecessor has completed and its writes are visible, and only then
// lets its own successor be scheduled.  Called before any memory access; in a
// plain launch both instructions return at once.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <int K, bool MAX>
__device__ inline void block_reduce_store(double (&acc)[K], double* partials) {
    __shared__ double sh[K][RED_THREADS / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double a = acc[k];
        for (int o = 16; o > 0; o >>= 1) {
            double b = __shfl_down_sync(0xffffffffu, a, o);
            a = MAX ? fmax(a, b) : a + b;
        }
        if (lane == 0) sh[k][wid] = a;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        int k = threadIdx.x;
        double a = sh[k][0];
        for (int w = 1; w < RED_THREADS / 32; ++w) a = MAX ? fmax(a, sh[k][w]) : a + sh[k][w];
        partials[k * RED_BLOCKS + blockIdx.x] = a;
    }
}

// Sums of FP32 per-thread partials: FP32 within a warp (32 terms), FP64
// across the block's warps and blocks, so that per-element work stays off the
// FP64 pipe.
template <int K>
__device__ inline void block_reduce_store_f32(float (&acc)[K], double* partials) {
    __shared__ double sh[K][RED_THREADS / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float a = acc[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sh[k][wid] = (double)a;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        int k = threadIdx.x;
        double a = sh[k][0];
        for (int w = 1; w < RED_THREADS / 32; ++w) a += sh[k][w];
        partials[k * RED_BLOCKS + blockIdx.x] = a;
    }
}

// one block (RED_THREADS threads) per result k; out[k] = reduction of partials[k][*]
template <bool MAX>
__global__ void k_reduce_final(const double* __restrict__ partials, int K, double* __restrict__ out) {
    pdl_entry();
    __shared__ double sh[RED_THREADS];
    int k = blockIdx.x;
    double a = MAX ? -1.0 : 0.0;
    for (int i = threadIdx.x; i < RED_BLOCKS; i += blockDim.x) {
        double b = partials[k * RED_BLOCKS + i];
        a = MAX ? fmax(a, b) : a + b;
    }
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            sh[threadIdx.x] = MAX ? fmax(sh[threadIdx.x], sh[threadIdx.x + s]) : sh[threadIdx.x] + sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
}

}  // namespace mb
