// Grid-wide barrier of a persistent cooperative launch, with a bounded wait.
//
// The batched step runs its phases (allocation, emission; the Newton passes
// and the final pass) as phases of one persistent launch each.  Between two
// phases every block arrives at this barrier: thread 0 of a block adds itself
// to the arrival count; the last block to arrive resets the count and opens the
// barrier by advancing its generation; the others poll the generation, each
// poll bounded (at most `limit` polls, about a second at the default), and
// give up when the limit runs out or when another block has already recorded
// an expiry.  A block that gives up records bit 3 in the flags word and
// returns false; the kernel then returns, so no block ever waits unboundedly
// (a cooperative launch also guarantees that every block of the grid is
// resident, so the barrier completes in normal operation).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rec {

struct GridBarrier {
  unsigned int arrived;  // blocks arrived at the open barrier
  unsigned int gen;      // generation: advanced by the last block to arrive
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Returns true in every thread of the block once all blocks of the grid have
// arrived; false (in every thread) if the wait expired here or elsewhere.
__device__ __forceinline__ bool grid_barrier(GridBarrier* g, int* flags, uint32_t limit) {
  __shared__ int s_ok;
  __syncthreads();  // the block's work of this phase is done
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int gen = ld_acquire_u32(&g->gen);
    __threadfence();  // this block's writes before its arrival
    const unsigned int a = atomicAdd(&g->arrived, 1u);
    if (a == gridDim.x - 1) {
      g->arrived = 0;  // reset before the barrier opens: nobody arrives again before that
      __threadfence();
      atomicAdd(&g->gen, 1u);
    } else {
      uint32_t polls = 0;
      while (ld_acquire_u32(&g->gen) == gen) {
        if ((ld_relaxed_i32(flags) & 8) || polls >= limit) {
          atomicOr(flags, 8);
          ok = 0;
          break;
        }
        ++polls;
        __nanosleep(256);
      }
    }
    __threadfence();  // the other blocks' writes are visible to this block's threads
    if (ok && (ld_relaxed_i32(flags) & 8)) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace rec
