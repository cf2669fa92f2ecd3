// Fixed-order block reductions for the streaming passes.  Each block writes
// its partials; the last block to finish (atomic ticket) combines all
// partials in block order.  Given the grid size, the result is bit-identical
// from run to run (no floating-point atomics).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rec {

// Sum K values over the block (fixed shuffle tree, then warps in order).
// Result valid in thread 0.
template <int K, int NT>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
  __shared__ double sm[NT / 32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
  }
  __syncthreads();  // sm may still be read by a previous call
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sm[warp][k] = v[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = sm[0][k];
      for (int w = 1; w < NT / 32; ++w) s += sm[w][k];
      v[k] = s;
    }
  }
}

template <int NT>
__device__ __forceinline__ double block_max(double v) {
  __shared__ double sm[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  __syncthreads();
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NT / 32; ++w) v = fmax(v, sm[w]);
    v = fmax(v, sm[0]);
  }
  return v;
}

// True in every thread of the last block of the grid (or of nblk blocks
// sharing the counter) to arrive.  The caller
// has written its partials before calling; the fence makes them visible.
__device__ __forceinline__ bool last_block_done(uint32_t* counter, uint32_t nblk) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == nblk - 1);
  __syncthreads();
  return am_last;
}
__device__ __forceinline__ bool last_block_done(uint32_t* counter) { return last_block_done(counter, gridDim.x); }

// In the last block: combine K partial sums of nblk blocks (layout
// part[b*stride + k]) in a fixed order.  Result valid in thread 0.
template <int K, int NT>
__device__ __forceinline__ void combine_partials(const double* part, int nblk, int stride, double (&out)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) out[k] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += NT) {
#pragma unroll
    for (int k = 0; k < K; ++k) out[k] += __ldcg(part + (size_t)b * stride + k);
  }
  block_sum<K, NT>(out);
}

template <int NT>
__device__ __forceinline__ double combine_max(const double* part, int nblk, int stride, int slot) {
  double m = 0.0;
  for (int b = threadIdx.x; b < nblk; b += NT) m = fmax(m, __ldcg(part + (size_t)b * stride + slot));
  return block_max<NT>(m);
}

// Compensated (two-sum) accumulation in binary32: the running error term
// keeps per-thread partial sums accurate to about 1e-14 relative.
struct Kahan32 {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

}  // namespace rec
