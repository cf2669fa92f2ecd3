// Fixed-order block reductions for the streaming passes.  Each block writes
// its partials; the last block to finish (atomic ticket) combines all
// partials in block order.  Given the grid size, the result is bit-identical
// from run to run (no floating-point atomics).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rec_df.cuh"

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

// The first K entries of a longer array.
template <int K, int NT, int N>
__device__ __forceinline__ void block_sum_first(double (&v)[N]) {
  static_assert(K <= N, "block_sum_first: K exceeds the array");
  block_sum<K, NT>(*reinterpret_cast<double(*)[K]>(&v[0]));
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
__device__ __forceinline__ void combine_partials(const double* part, int nblk, int stride, double (&out)[K]);
// Combined into the first K entries of a longer array (the rest set to zero).
template <int K, int NT, int N>
__device__ __forceinline__ void combine_partials_first(const double* part, int nblk, int stride, double (&out)[N]) {
  static_assert(K <= N, "combine_partials_first: K exceeds the array");
#pragma unroll
  for (int k = K; k < N; ++k) out[k] = 0.0;
  combine_partials<K, NT>(part, nblk, stride, *reinterpret_cast<double(*)[K]>(&out[0]));
}

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

// Block sum of K compensated binary32 accumulators into binary64 (result in
// thread 0).  The warp tree adds the (s, -c) pairs in double-float arithmetic
// (binary32 operations only); lane 0 of each warp widens its pair once, and
// thread 0 adds the warps in order in binary64.  On GB300 the binary64 pipe
// is slow, so this keeps the per-thread reduction off it.
template <int K, int NT, int N>
__device__ __forceinline__ void block_sum_kahan(const Kahan32 (&acc)[K], double (&out)[N]) {
  static_assert(K <= N, "block_sum_kahan: K exceeds the output");
  __shared__ double sm[NT / 32][K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float hi[K], lo[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const dfloat p = df_fast_two_sum(acc[k].s, -acc[k].c);
    hi[k] = p.hi;
    lo[k] = p.lo;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float h2 = __shfl_down_sync(0xffffffffu, hi[k], off);
      const float l2 = __shfl_down_sync(0xffffffffu, lo[k], off);
      const dfloat r = df_add(dfloat{hi[k], lo[k]}, dfloat{h2, l2});
      hi[k] = r.hi;
      lo[k] = r.lo;
    }
  }
  __syncthreads();  // sm may still be read by a previous call
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sm[warp][k] = (double)hi[k] + (double)lo[k];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double t = sm[0][k];
      for (int w = 1; w < NT / 32; ++w) t += sm[w][k];
      out[k] = t;
    }
  }
}

}  // namespace rec
