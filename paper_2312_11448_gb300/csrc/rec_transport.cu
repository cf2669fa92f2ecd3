// Ly-alpha packet transport on the GPU.
//
// Method (arXiv:2312.11448, Sec. III.B and Appendix A): packets are emitted
// per cell in proportion to the local recombination rate alpha_e n_e^2 (the
// integrand of the global loss-rate Monte Carlo), injected at a random point
// of the cell (step (1)), streamed in a straight line while the expansion
// redshifts them by dx = -H dl / v_th (step (4)), with the gas-frame frequency
// shifted by the bulk flow, omega_r = omega (1 - U_par).  A packet is absorbed
// into the integer tally of the first cell in which it comes back into line
// resonance.
//
// Kernels (one lya_transport call):
//   k_alloc_max     r_max over the emission weights (and a validity check)
//   k_alloc_sum     Q_i = floor(2^31 r_i / r_max); block sums; last block scans
//                   them and draws the systematic-sampling offset u
//   k_alloc_prefix  packet prefix P_i = floor((N prefixQ_i + u) / sum Q), exact
//                   integer arithmetic; cell of every 32nd packet; packets per
//                   32^3 super-tile
//   k_bucket_offsets  queue bucket offsets (capacities) per super-tile
//   k_emit          one packet per thread: warp-cooperative cell lookup in P,
//                   Philox draws, emission, resonance test in the home cell
//                   (warp-aggregated tally); the others step once and are queued
//                   in their home super-tile's bucket
//   k_bucket_scan   prefix of the queued counts (bucket order of the march)
//   k_march         persistent warps march the queued packets (Amanatides-Woo),
//                   refilling idle lanes from the queue; tally atomics
//   k_transport_end counters to the statistics record
// The march is written operation by operation with round-to-nearest
// intrinsics (never contracted into FMA), in binary32 for the mixed form and
// binary64 for the FP64 form, so its integer results are reproducible.

#include <cmath>
#include <cstring>

#include "rec_internal.cuh"
#include "rec_reduce.cuh"

namespace rec {
namespace {

constexpr int TT = 256;  // transport block size
constexpr int AT = kAllocThreads;

// ---- Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) ----------------------
struct U4 {
  uint32_t a, b, c, d;
};

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                            uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // 32 x 32 -> 64-bit products (low and high words from one wide multiply)
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// The keys of the ten rounds, (k0 + r W0, k1 + r W1), formed once on the host.
// Kernels read them from their parameters, so every round takes its key as a
// constant operand instead of adding the Weyl increments per packet.
struct Keys {
  uint32_t a[10], b[10];
};
inline Keys key_schedule(uint32_t k0, uint32_t k1) {
  Keys K;
  for (int r = 0; r < 10; ++r) {
    K.a[r] = k0;
    K.b[r] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return K;
}
__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const Keys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ K.a[r];
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.b[r];
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
  }
  return U4{c0, c1, c2, c3};
}

// Streams: key (seed_lo, seed_hi ^ step), counter (cell, packet-in-cell, block, box).
struct Stream {
  uint32_t k0, k1, box;
};
__device__ __forceinline__ U4 draw(const Stream& s, uint32_t cell, uint32_t j, uint32_t block) {
  return philox4x32_10(cell, j, block, s.box, s.k0, s.k1);
}
// The same draw with the keys from a schedule (emission).
struct KStream {
  const Keys& K;
  uint32_t box;
};
__device__ __forceinline__ U4 draw(const KStream& s, uint32_t cell, uint32_t j, uint32_t block) {
  return philox4x32_10(cell, j, block, s.box, s.K);
}
constexpr uint32_t kAllocBlock = 0x000A110Cu;  // counter block of the allocation offset

// Uniform deviates strictly inside (0,1), exactly representable.
// Binary32: the float 1 + m 2^-23 with m the top 23 bits of r, minus 1 - 2^-24,
// is exactly (2m + 1) 2^-24 (Sterbenz: the operands are within a factor of
// two), with no integer-to-float conversion.
__device__ __forceinline__ float u01f(uint32_t r) {
  return __fsub_rn(__uint_as_float(0x3f800000u | (r >> 9)), 0x1.fffffep-1f);
}
__device__ __forceinline__ double u01d(uint32_t lo, uint32_t hi) {
  uint64_t w = ((uint64_t)hi << 32) | lo;
  return __ull2double_rn((w >> 11) | 1ull) * 0x1p-53;
}

// ---- explicitly rounded arithmetic -----------------------------------------------
template <class R> struct Ar;
template <> struct Ar<float> {
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
  static __device__ __forceinline__ float rcp(float a) { return __frcp_rn(a); }  // correctly rounded 1/a
  static __device__ __forceinline__ float sqr(float a) { return __fsqrt_rn(a); }
  static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
  static __device__ __forceinline__ int trunc(float a) { return __float2int_rz(a); }
};
template <> struct Ar<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ double rcp(double a) { return __drcp_rn(a); }  // correctly rounded 1/a
  static __device__ __forceinline__ double sqr(double a) { return __dsqrt_rn(a); }
  static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
  static __device__ __forceinline__ int trunc(double a) { return __double2int_rz(a); }
};

template <class R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = double4_32a; };

// Per-precision draw layout.
template <class R> struct Draws;
template <> struct Draws<float> {
  // block 0: three cell offsets and the frequency quantile; blocks 1..16: two
  // direction pairs each
  static constexpr int kPairs = 2;
  template <class S>
  static __device__ __forceinline__ void position(const S& s, uint32_t c, uint32_t j, float f[3], float* uq) {
    U4 r = draw(s, c, j, 0u);
    f[0] = u01f(r.a); f[1] = u01f(r.b); f[2] = u01f(r.c); *uq = u01f(r.d);
  }
  using Block = U4;
  static __device__ __forceinline__ bool first_of_block(int t) { return (t & 1) == 0; }
  template <class S>
  static __device__ __forceinline__ U4 block(const S& s, uint32_t c, uint32_t j, int t) {
    return draw(s, c, j, 1u + (uint32_t)(t >> 1));
  }
  static __device__ __forceinline__ void pair_from(const U4& r, int t, float* a, float* b) {
    if (t & 1) { *a = u01f(r.c); *b = u01f(r.d); }
    else { *a = u01f(r.a); *b = u01f(r.b); }
  }
};
template <> struct Draws<double> {
  // blocks 0, 1: three cell offsets and the quantile (two words per deviate);
  // blocks 2..33: one direction pair each
  static constexpr int kPairs = 1;
  template <class S>
  static __device__ __forceinline__ void position(const S& s, uint32_t c, uint32_t j, double f[3], double* uq) {
    U4 r = draw(s, c, j, 0u), q = draw(s, c, j, 1u);
    f[0] = u01d(r.a, r.b); f[1] = u01d(r.c, r.d); f[2] = u01d(q.a, q.b); *uq = u01d(q.c, q.d);
  }
  using Block = U4;
  static __device__ __forceinline__ bool first_of_block(int) { return true; }
  template <class S>
  static __device__ __forceinline__ U4 block(const S& s, uint32_t c, uint32_t j, int t) {
    return draw(s, c, j, 2u + (uint32_t)t);
  }
  static __device__ __forceinline__ void pair_from(const U4& r, int, double* a, double* b) {
    *a = u01d(r.a, r.b); *b = u01d(r.c, r.d);
  }
};

// ---- allocation -------------------------------------------------------------------
// The maximum is taken in the working precision (exact for any precision), so
// the binary32 form issues no binary64 instruction per cell.
template <class R>
__global__ void __launch_bounds__(kPassThreads) k_alloc_max(const R* emis, int64_t n3, DevScalars* sc, double* part) {
  R m = (R)0;
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * kPassThreads + threadIdx.x; i < n3; i += (int64_t)gridDim.x * kPassThreads) {
    const R r = emis[i];
    if (!(r >= (R)0) || isinf(r)) bad = 1;
    else m = fmax(m, r);
  }
  bad = __syncthreads_or(bad);
  double bm = block_max<kPassThreads>((double)m);
  if (threadIdx.x == 0) {
    part[(size_t)blockIdx.x * kMaxSums + 0] = bm;
    part[(size_t)blockIdx.x * kMaxSums + 1] = bad ? 1.0 : 0.0;
  }
  if (!last_block_done(&sc->counter)) return;
  double mx = combine_max<kPassThreads>(part, gridDim.x, kMaxSums, 0);
  double anybad = combine_max<kPassThreads>(part, gridDim.x, kMaxSums, 1);
  if (threadIdx.x == 0) {
    sc->rmax = anybad > 0.0 ? 0.0 : mx;  // invalid weights: emit nothing
    sc->flags &= ~(2 | 4 | 16);          // transport flags describe this call only
    if (anybad > 0.0) sc->flags |= 4;
    sc->counter = 0;
  }
}

template <class R>
__device__ __forceinline__ uint64_t quantised(R r, R rmax) {
  // Q = floor(2^31 r / r_max), the ratio rounded once in the working precision.
  // Q <= 2^31 fits 32 bits: the 32-bit truncation gives the same integer as a
  // 64-bit one without the 64-bit conversion (a binary64-pipe instruction).
  return (uint64_t)(uint32_t)Ar<R>::mul(Ar<R>::div(r, rmax), (R)2147483648.0);
}

// Inclusive block scan of 64-bit counts (thread order); returns the block total.
__device__ __forceinline__ uint64_t block_scan_incl(uint64_t v, uint64_t* incl) {
  __shared__ uint64_t wsum[AT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    uint64_t t = __shfl_up_sync(0xffffffffu, v, off);
    if (lane >= off) v += t;
  }
  __syncthreads();
  if (lane == 31) wsum[warp] = v;
  __syncthreads();
  uint64_t before = 0, total = 0;
  for (int w = 0; w < AT / 32; ++w) {
    uint64_t s = wsum[w];
    if (w < warp) before += s;
    total += s;
  }
  *incl = v + before;
  return total;
}

// Super-tiles of 2^tlg cells per side group the march queue: packets are queued in
// the bucket of their home super-tile, and the march takes the buckets in
// order, so the rays in flight at any time start in a compact region.

// Cell coordinates: shifts and masks for power-of-two sides, otherwise the
// quotients by n and n^2 from 64-bit multiply-high with precomputed
// multipliers ceil(2^64 / d), exact for every 32-bit dividend (Lemire, Kaser &
// Kurz 2019, "Faster remainder by direct computation").
struct Tiles {
  uint32_t n, nt, lg;  // box side, super-tiles per axis, log2 n (power-of-two sides)
  uint64_t mn, mn2;    // multipliers for the division by n and by n^2 (unused when n = 1: cell = 0)
  uint32_t tlg;        // log2 of the super-tile side
  template <bool P2>
  __device__ __forceinline__ void coords(uint32_t cell, uint32_t* ix, uint32_t* iy, uint32_t* iz) const {
    if (P2) {
      const uint32_t m = n - 1u;
      *ix = cell & m; *iy = (cell >> lg) & m; *iz = cell >> (2u * lg);
    } else {
      const uint32_t q = (uint32_t)__umul64hi(mn, (uint64_t)cell);   // cell / n
      const uint32_t z = (uint32_t)__umul64hi(mn2, (uint64_t)cell);  // cell / n^2
      *ix = cell - q * n; *iy = q - z * n; *iz = z;
    }
  }
  template <bool P2>
  __device__ __forceinline__ uint32_t at(uint32_t cell) const {
    uint32_t ix, iy, iz;
    coords<P2>(cell, &ix, &iy, &iz);
    return ((iz >> tlg) * nt + (iy >> tlg)) * nt + (ix >> tlg);
  }
  __device__ __forceinline__ uint32_t of(uint32_t cell) const { return at<false>(cell); }
};

// Multiplier ceil(2^64 / d) of the exact 32-bit division by d >= 2.
inline uint64_t fastdiv_multiplier(uint64_t d) { return d >= 2 ? UINT64_MAX / d + 1 : 0; }
inline uint32_t log2_of(uint32_t v) {
  uint32_t l = 0;
  while ((1u << l) < v) ++l;
  return l;
}
inline Tiles make_tiles(int n, int tile) {
  Tiles t;
  t.n = (uint32_t)n;
  t.tlg = log2_of((uint32_t)tile);
  t.nt = (uint32_t)((n + tile - 1) / tile);
  t.lg = 0;
  if ((n & (n - 1)) == 0)
    while ((1 << t.lg) < n) ++t.lg;
  t.mn = fastdiv_multiplier((uint64_t)n);
  t.mn2 = fastdiv_multiplier((uint64_t)n * (uint64_t)n);
  return t;
}

// The allocation kernels give each thread kAllocItems consecutive cells.
template <class R>
__device__ __forceinline__ void load_items(const R* p, int64_t c0, int64_t n3, R (&v)[kAllocItems]) {
  if (c0 + kAllocItems <= n3 && (reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
    if (sizeof(R) == 4) {
      const float4* q = reinterpret_cast<const float4*>(p + c0);
#pragma unroll
      for (int k = 0; k < kAllocItems / 4; ++k) {
        float4 t = q[k];
        v[4 * k] = (R)t.x; v[4 * k + 1] = (R)t.y; v[4 * k + 2] = (R)t.z; v[4 * k + 3] = (R)t.w;
      }
    } else {
      const double2* q = reinterpret_cast<const double2*>(p + c0);
#pragma unroll
      for (int k = 0; k < kAllocItems / 2; ++k) {
        double2 t = q[k];
        v[2 * k] = (R)t.x; v[2 * k + 1] = (R)t.y;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < kAllocItems; ++k) v[k] = (c0 + k < n3) ? p[c0 + k] : (R)0;
  }
}

template <class R>
__global__ void __launch_bounds__(AT) k_alloc_sum(const R* emis, int64_t n3, uint64_t n_packets, Stream strm,
                                                  DevScalars* sc, unsigned long long* partQ, uint32_t* P) {
  const R rmax = (R)sc->rmax;
  uint64_t acc = 0;
  if (rmax > (R)0) {
    R v[kAllocItems];
    load_items<R>(emis, (int64_t)blockIdx.x * kAllocChunk + (int64_t)threadIdx.x * kAllocItems, n3, v);
#pragma unroll
    for (int k = 0; k < kAllocItems; ++k) acc += quantised<R>(v[k], rmax);
  }
  uint64_t incl;
  uint64_t tot = block_scan_incl(acc, &incl);
  if (threadIdx.x == 0) partQ[blockIdx.x] = tot;
  if (!last_block_done(&sc->alloc_counter)) return;
  // exclusive scan of the block sums, in block order
  const int nb = gridDim.x;
  const int per = (nb + AT - 1) / AT;
  uint64_t seg = 0;
  for (int b = threadIdx.x * per; b < min(nb, (threadIdx.x + 1) * per); ++b) seg += __ldcg(&partQ[b]);
  uint64_t sincl;
  uint64_t sumQ = block_scan_incl(seg, &sincl);
  uint64_t run = sincl - seg;
  for (int b = threadIdx.x * per; b < min(nb, (threadIdx.x + 1) * per); ++b) {
    uint64_t q = __ldcg(&partQ[b]);
    partQ[b] = run;
    run += q;
  }
  if (threadIdx.x == 0) {
    U4 r = draw(strm, 0u, 0u, kAllocBlock);
    uint64_t w = ((uint64_t)r.b << 32) | r.a;
    uint64_t npk = (sumQ > 0) ? n_packets : 0;
    sc->sumQ = sumQ;
    sc->alloc_u = sumQ > 0 ? w % sumQ : 0;
    P[n3] = (uint32_t)npk;
    sc->emitted = npk;
    sc->absorbed = 0;
    sc->capped = 0;
    sc->crossings = 0;
    sc->qtail = 0;
    sc->alloc_counter = 0;
    if (sumQ == 0 && n_packets > 0) sc->flags |= 4;
  }
}

// floor((N * pre + u) / S) and the remainder, for N < 2^32, pre <= S < 2^64,
// u < S: a binary64 estimate corrected with exact 128-bit products.
__device__ __forceinline__ uint32_t sys_floor(uint64_t N, uint64_t pre, uint64_t u, uint64_t S, uint64_t* rem) {
  uint64_t lo = N * pre, hi = __umul64hi(N, pre);
  uint64_t lo2 = lo + u;
  hi += (lo2 < lo);
  lo = lo2;
  double est = ((double)hi * 18446744073709551616.0 + (double)lo) / (double)S;
  uint64_t q = (uint64_t)est;
  if (q > N) q = N;
  for (;;) {  // q S > X ?
    uint64_t plo = q * S, phi = __umul64hi(q, S);
    if (phi > hi || (phi == hi && plo > lo)) { --q; continue; }
    // X - q S >= S ?
    uint64_t rlo = lo - plo, rhi = hi - phi - (lo < plo);
    if (rhi > 0 || rlo >= S) { ++q; continue; }
    *rem = rlo;
    break;
  }
  return (uint32_t)q;
}

// floor(t / S) and t mod S for t < 2^64, given m = floor((2^64 - 1) / S): the
// multiply-high estimate is short by at most 2, then corrected exactly
// (replaces a 64-bit division per cell).
__device__ __forceinline__ uint64_t div_small(uint64_t t, uint64_t S, uint64_t m, uint64_t* r) {
  uint64_t q = __umul64hi(t, m);
  uint64_t rr = t - q * S;
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (rr >= S) { ++q; rr -= S; }
  *r = rr;
  return q;
}

// Packet prefix P_i = floor((N prefixQ_i + u) / S) of the thread's consecutive
// cells: one 128-bit division for the first, then exact 64-bit remainder
// updates, (R + N Q_i) / S.  The same pass writes the coarse index first[w] =
// cell of packet 32 w (each cell writes the multiples of 32 in its packet
// range, so a warp of 32 consecutive packets finds its first cell with one
// load) and the packets per super-tile (the capacity of its march-queue bucket).
template <class R>
__device__ __forceinline__ void alloc_prefix_block(const R* emis, int64_t n3, uint64_t n_packets, uint64_t S,
                                                   uint64_t u, R rmax, uint64_t pre_block, int64_t c0, uint32_t* P,
                                                   uint32_t* first, const Tiles& tl, uint32_t bk0,
                                                   unsigned long long* bcap) {
  uint64_t Q[kAllocItems];
  uint64_t acc = 0;
  {
    R v[kAllocItems];
    load_items<R>(emis, c0, n3, v);
#pragma unroll
    for (int k = 0; k < kAllocItems; ++k) {
      Q[k] = (rmax > (R)0 && c0 + k < n3) ? quantised<R>(v[k], rmax) : 0;
      acc += Q[k];
    }
  }
  uint64_t incl;
  block_scan_incl(acc, &incl);
  if (c0 >= n3) return;
  uint32_t out[kAllocItems];
  if (S == 0) {
#pragma unroll
    for (int k = 0; k < kAllocItems; ++k) out[k] = 0u;
  } else {
    uint64_t rem;
    uint32_t pk = sys_floor(n_packets, pre_block + incl - acc, u, S, &rem);
    uint32_t bk = 0xffffffffu, bcount = 0;
    const uint64_t minv = ~0ull / S;
#pragma unroll
    for (int k = 0; k < kAllocItems; ++k) {
      out[k] = pk;
      const uint64_t t = rem + n_packets * Q[k];  // < S + 2^63 <= 2^64
      const uint64_t dq = div_small(t, S, minv, &rem);
      const uint32_t p1 = pk + (uint32_t)dq;
      if (p1 > pk && c0 + k < n3) {
        for (uint32_t w = (pk + 31u) >> 5; 32ull * w < p1; ++w) first[w] = (uint32_t)(c0 + k);
        const uint32_t b = bk0 + tl.of((uint32_t)(c0 + k));
        if (b != bk) {
          if (bcount) atomicAdd(&bcap[bk], (unsigned long long)bcount);
          bk = b;
          bcount = 0;
        }
        bcount += p1 - pk;
      }
      pk = p1;
    }
    if (bcount) atomicAdd(&bcap[bk], (unsigned long long)bcount);
  }
  if (c0 + kAllocItems <= n3 && (reinterpret_cast<uintptr_t>(P + c0) & 15u) == 0) {
    uint4* q = reinterpret_cast<uint4*>(P + c0);
#pragma unroll
    for (int k = 0; k < kAllocItems / 4; ++k) q[k] = make_uint4(out[4 * k], out[4 * k + 1], out[4 * k + 2], out[4 * k + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < kAllocItems; ++k)
      if (c0 + k < n3) P[c0 + k] = out[k];
  }
}

template <class R>
__global__ void __launch_bounds__(AT) k_alloc_prefix(const R* emis, int64_t n3, uint64_t n_packets, DevScalars* sc,
                                                     const unsigned long long* partQ, uint32_t* P, uint32_t* first,
                                                     Tiles tl, unsigned long long* bcap) {
  const int64_t c0 = (int64_t)blockIdx.x * kAllocChunk + (int64_t)threadIdx.x * kAllocItems;
  alloc_prefix_block<R>(emis, n3, n_packets, sc->sumQ, sc->alloc_u, (R)sc->rmax, partQ[blockIdx.x], c0, P, first, tl,
                        0u, bcap);
}

// One block: bucket capacities -> offsets (in place); fill counters cleared.
template <int NTH>
__device__ __forceinline__ void bucket_offsets_block(unsigned long long* bcap, unsigned long long* bfill, int nb) {
  __shared__ unsigned long long part[NTH];
  const int per = (nb + NTH - 1) / NTH;
  unsigned long long s = 0;
  for (int b = threadIdx.x * per; b < min(nb, (threadIdx.x + 1) * per); ++b) s += __ldcg(&bcap[b]);
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0;
    for (int t = 0; t < NTH; ++t) { unsigned long long v = part[t]; part[t] = run; run += v; }
  }
  __syncthreads();
  unsigned long long run = part[threadIdx.x];
  for (int b = threadIdx.x * per; b < min(nb, (threadIdx.x + 1) * per); ++b) {
    unsigned long long v = __ldcg(&bcap[b]);
    bcap[b] = run;
    run += v;
    bfill[b] = 0;
  }
}
__global__ void __launch_bounds__(1024) k_bucket_offsets(unsigned long long* bcap, unsigned long long* bfill, int nb) {
  bucket_offsets_block<1024>(bcap, bfill, nb);
}

// One block: the march works through the queue in chunks of `chunk` packets
// that never straddle a bucket; cpre[b] = first chunk of bucket b, cpre[nb] =
// all chunks.  Also the total queued.
template <int NTH>
__device__ __forceinline__ void bucket_scan_block(const unsigned long long* bfill, unsigned long long* cpre, int nb,
                                                  DevScalars* sc, uint32_t chunk) {
  __shared__ unsigned long long part[NTH], qpart[NTH];
  const int per = (nb + NTH - 1) / NTH;
  unsigned long long s = 0, q = 0;
  for (int b = threadIdx.x * per; b < min(nb, (threadIdx.x + 1) * per); ++b) {
    const unsigned long long f = __ldcg(&bfill[b]);
    s += (f + chunk - 1) / chunk;
    q += f;
  }
  part[threadIdx.x] = s;
  qpart[threadIdx.x] = q;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0, qt = 0;
    for (int t = 0; t < NTH; ++t) { unsigned long long v = part[t]; part[t] = run; run += v; qt += qpart[t]; }
    cpre[nb] = run;
    sc->qtail = qt;
    sc->march_next = 0;
    sc->requeued = 0;
  }
  __syncthreads();
  unsigned long long run = part[threadIdx.x];
  for (int b = threadIdx.x * per; b < min(nb, (threadIdx.x + 1) * per); ++b) {
    cpre[b] = run;
    run += (__ldcg(&bfill[b]) + chunk - 1) / chunk;
  }
}
__global__ void __launch_bounds__(1024) k_bucket_scan(const unsigned long long* bfill, unsigned long long* cpre, int nb,
                                                      DevScalars* sc, uint32_t chunk) {
  bucket_scan_block<1024>(bfill, cpre, nb, sc, chunk);
}

// ---- transport ----------------------------------------------------------------------
// A queued packet: the march state right after it left its home cell.
// Binary32 form (two float4):
//   q0 = {cell bits, tMax_x, tMax_y, tMax_z},  q1 = {n_x, n_y, n_z, u0};
// the march recomputes tDelta = 1/|n| and kappa n with the same rounded
// operations as the emission, so it continues bit for bit.
// Binary64 form (three double4): q0 as above, q1 = {tDelta (sign = step
// direction), u0}, q2 = {kappa n, -}: recomputing them would cost three
// correctly rounded binary64 reciprocals per packet on the slow binary64 pipe.
template <class R> struct QueueVecs { static constexpr int value = sizeof(R) == 4 ? 2 : 3; };
template <class R>
struct TransportArgs {
  const uint32_t* P;
  const uint32_t* first;  // cell of packet 32 w
  int64_t n3;
  int n;
  const typename Vec4<R>::T* vel;
  const R* T;
  const R* quant;
  int M;
  R kappa, cth;
  Stream strm;
  Keys ks;  // round keys of strm (emission)
  uint32_t* tally;
  DevScalars* sc;
  typename Vec4<R>::T* queue;  // 3 entries per queued packet
  Tiles tl;
  int nb;                          // buckets (super-tiles)
  unsigned long long* boff;        // bucket start in the queue (capacity prefix)
  unsigned long long* bfill;       // packets queued per bucket
  const unsigned long long* cpre;  // first march chunk of each bucket [nb + 1]
  uint32_t chunk;                  // queued packets per march chunk
  int refill;                      // idle lanes of a warp that trigger a refill
  // region sweeps (single box, power-of-two side)
  typename Vec4<R>::T* rq;         // second queue: full traversal states, 3 vectors per entry
  unsigned long long* rcount;      // entries per bucket appended to the second queue
  unsigned long long* rqn;         // entries appended per part of the second queue [kRqParts]
  uint64_t rq_part;                // entries one part holds
  uint32_t halo;                   // region of a bucket: its super-tile and halo cells around it; 0: no limit
  int resumed;                     // the queue holds full states of an earlier sweep (3 vectors per entry)
};

// Loads of the packet prefix and coarse index: the read-only path, or through
// L2 (FRESH) when they were written earlier in the same launch.
template <bool FRESH>
__device__ __forceinline__ uint32_t ld_index(const uint32_t* p) {
  return FRESH ? __ldcg(p) : __ldg(p);
}

// First index k in [lo, hi] with P[k] > key (P[hi] > key holds).
template <bool FRESH = false>
__device__ __forceinline__ uint32_t upper_bound(const uint32_t* P, uint32_t lo, uint32_t hi, uint32_t key) {
  while (lo < hi) {
    uint32_t mid = lo + ((hi - lo) >> 1);
    if (ld_index<FRESH>(P + mid) > key) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

template <class R> __device__ __forceinline__ R bits_to(uint32_t v);
template <> __device__ __forceinline__ float bits_to<float>(uint32_t v) { return __uint_as_float(v); }
template <> __device__ __forceinline__ double bits_to<double>(uint32_t v) { return __longlong_as_double((long long)v); }
template <class R> __device__ __forceinline__ uint32_t to_bits(R v);
template <> __device__ __forceinline__ uint32_t to_bits<float>(float v) { return __float_as_uint(v); }
template <> __device__ __forceinline__ uint32_t to_bits<double>(double v) { return (uint32_t)__double_as_longlong(v); }

// Lower table node of the frequency quantile: k = min(trunc(tq), M - 2) (0 <= tq
// < M - 1) and k as a value of R.  Binary32: adding 2^23 rounded toward zero
// leaves 2^23 + trunc(tq) exactly, whose bits give k without a conversion.
template <class R>
__device__ __forceinline__ R quant_node(R tq, int M, int* k) {
  int kk = Ar<R>::trunc(tq);
  if (kk > M - 2) kk = M - 2;
  *k = kk;
  return (R)kk;
}
template <>
__device__ __forceinline__ float quant_node<float>(float tq, int M, int* k) {
  const float t = __fadd_rz(tq, 0x1p23f);
  int kk = __float_as_int(t) - 0x4b000000;
  float kf = __fsub_rn(t, 0x1p23f);
  if (kk > M - 2) { kk = M - 2; kf = (float)(M - 2); }
  *k = kk;
  return kf;
}

// Traversal state of one packet.
template <class R>
struct Ray {
  uint32_t ix, iy, iz, kc;
  R tMx, tMy, tMz, tDx, tDy, tDz, knx, kny, knz, u0;
  int sx, sy, sz;
};

// tDelta and step of one axis from the direction cosine (Amanatides-Woo).
template <class R>
// Written without branches: 1/|n_d| correctly rounded (the same value as the
// division 1/|n_d|) is +inf for n_d = 0, which is the tDelta of an axis never
// crossed.
__device__ __forceinline__ void axis_setup(R nd, R* tD, int* st) {
  using A = Ar<R>;
  *st = (nd > (R)0) - (nd < (R)0);
  *tD = A::rcp(fabs(nd));
}

// One cell of the march: resonance test in the current cell, then a step
// across the nearest face (ties x < y < z, periodic wrap).  Returns 1 when
// absorbed in the current cell, 2 when the crossing cap is hit, 0 otherwise.
// The step is written with selects rather than branches so that the lanes of
// a warp stepping along different axes do not serialise.
// Periodic neighbour index along one axis; a mask when the side is a power of two.
template <bool P2>
__device__ __forceinline__ uint32_t wrap_step(uint32_t i, int s, uint32_t n) {
  if (P2) return (i + (uint32_t)s) & (n - 1u);
  return s > 0 ? (i + 1 == n ? 0 : i + 1) : (i == 0 ? n - 1 : i - 1);
}

// Path length along the ray at which the packet leaves its current cell: the
// nearest face, ties broken x < y < z.
template <class R>
__device__ __forceinline__ R dda_exit(const Ray<R>& r, bool* ax0, bool* ax1, bool* ax2) {
  *ax0 = r.tMx <= r.tMy && r.tMx <= r.tMz;
  *ax1 = !*ax0 && r.tMy <= r.tMz;
  *ax2 = !*ax0 && !*ax1;
  return *ax0 ? r.tMx : (*ax1 ? r.tMy : r.tMz);
}

// Gas-frame resonance distance offset kappa n.U_c of a cell.
template <class R, class V>
__device__ __forceinline__ R doppler(const Ray<R>& r, const V& U) {
  using A = Ar<R>;
  return A::add(A::add(A::mul(r.knx, U.x), A::mul(r.kny, U.y)), A::mul(r.knz, U.z));
}

template <class R, bool P2>
__device__ __forceinline__ void dda_advance(Ray<R>& r, bool ax0, bool ax1, bool ax2, R s_exit, uint32_t n);

template <class R, bool P2 = false, class V>
__device__ __forceinline__ int march_cell(Ray<R>& r, const V& Uc, uint32_t n) {
  using A = Ar<R>;
  R dc = doppler(r, Uc);
  bool ax0, ax1, ax2;
  const R s_exit = dda_exit(r, &ax0, &ax1, &ax2);
  // resonance in this cell at path length u0 - kappa n.U_c: absorb unless beyond the exit
  if (A::sub(r.u0, dc) <= s_exit) return 1;
  if (r.kc >= kMaxCrossings) return 2;
  dda_advance<R, P2>(r, ax0, ax1, ax2, s_exit, n);
  return 0;
}

// The step across the exit face: periodic neighbour along the exit axis and
// its next face distance.
template <class R, bool P2>
__device__ __forceinline__ void dda_advance(Ray<R>& r, bool ax0, bool ax1, bool ax2, R s_exit, uint32_t n) {
  using A = Ar<R>;
  const uint32_t wx = wrap_step<P2>(r.ix, r.sx, n);
  const uint32_t wy = wrap_step<P2>(r.iy, r.sy, n);
  const uint32_t wz = wrap_step<P2>(r.iz, r.sz, n);
  r.ix = ax0 ? wx : r.ix;
  r.iy = ax1 ? wy : r.iy;
  r.iz = ax2 ? wz : r.iz;
  const R tD = ax0 ? r.tDx : (ax1 ? r.tDy : r.tDz);
  const R tn = A::add(s_exit, tD);
  r.tMx = ax0 ? tn : r.tMx;
  r.tMy = ax1 ? tn : r.tMy;
  r.tMz = ax2 ? tn : r.tMz;
  ++r.kc;
}

__device__ __forceinline__ void add_counters(DevScalars* sc, uint64_t ab, uint64_t cap, uint64_t cross) {
  __shared__ unsigned long long s_abs, s_cap, s_cross;
  if (threadIdx.x == 0) { s_abs = 0; s_cap = 0; s_cross = 0; }
  __syncthreads();
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ab += __shfl_down_sync(0xffffffffu, ab, off);
    cap += __shfl_down_sync(0xffffffffu, cap, off);
    cross += __shfl_down_sync(0xffffffffu, cross, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s_abs, (unsigned long long)ab);
    atomicAdd(&s_cap, (unsigned long long)cap);
    atomicAdd(&s_cross, (unsigned long long)cross);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_abs) atomicAdd(&sc->absorbed, s_abs);
    if (s_cap) atomicAdd(&sc->capped, s_cap);
    if (s_cross) atomicAdd(&sc->crossings, s_cross);
  }
}

// Batched contexts: per-box event counters of one block in shared memory
// (absorbed, capped, crossings), added to the boxes' scalars at the block's end.
struct BoxCounters {
  unsigned long long v[3][kMaxBoxes];
};
__device__ __forceinline__ void box_counters_clear(BoxCounters& c, int B) {
  for (int i = threadIdx.x; i < 3 * kMaxBoxes; i += blockDim.x) c.v[i / kMaxBoxes][i % kMaxBoxes] = 0ull;
  __syncthreads();
}
__device__ __forceinline__ void box_counters_add(BoxCounters& c, int b, uint64_t ab, uint64_t cap, uint64_t cross) {
  if (ab) atomicAdd(&c.v[0][b], (unsigned long long)ab);
  if (cap) atomicAdd(&c.v[1][b], (unsigned long long)cap);
  if (cross) atomicAdd(&c.v[2][b], (unsigned long long)cross);
}
__device__ __forceinline__ void box_counters_flush(BoxCounters& c, const BoxDev* bxs, int B) {
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    DevScalars* sc = bxs[b].sc;
    if (c.v[0][b]) atomicAdd(&sc->absorbed, c.v[0][b]);
    if (c.v[1][b]) atomicAdd(&sc->capped, c.v[1][b]);
    if (c.v[2][b]) atomicAdd(&sc->crossings, c.v[2][b]);
  }
}

// Last index i in [0, B) with key(i) <= v (key non-decreasing, key(0) <= v).
template <class F>
__device__ __forceinline__ int last_le(int B, uint64_t v, F key) {
  int lo = 0, hi = B;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if ((uint64_t)key(mid) <= v) lo = mid;
    else hi = mid;
  }
  return lo;
}

// One box as the emission sees it: its fields, packet prefix and coarse index,
// transport scalars, random stream, super-tiles and first queue bucket.
template <class R>
struct EmitBox {
  const uint32_t* P;
  const uint32_t* first;
  uint32_t n3, n;
  const typename Vec4<R>::T* vel;
  const R* T;
  uint32_t* tally;
  R kappa, cth;
  uint32_t box;  // fourth Philox counter word
  Tiles tl;
  uint32_t bk0;
};

// Emission of one packet, in three parts: the cell of each of a warp's 32
// packets (warp-collective), the packet's first Philox block, frequency and
// thermal speed (per lane), and the rest (warp-collective): direction, the
// resonance test in the home cell, the home tally or the queue entry.

// Cell and index within the cell of packet base + lane (< N): the coarse index
// gives the cell of the warp's first packet, then a 32-cell window of the
// packet prefix resolves the rest with shuffles.
template <class R, bool FRESH>
__device__ __forceinline__ bool emit_locate(const EmitBox<R>& e, uint32_t base, uint32_t N, uint32_t* cell_out,
                                            uint32_t* j_out) {
  const int lane = threadIdx.x & 31;
  const uint32_t n3 = e.n3;
  const uint32_t p = base + lane;
  const bool act = p < N;
  const uint32_t c0 = ld_index<FRESH>(e.first + (base >> 5));
  const uint32_t Pc0 = ld_index<FRESH>(e.P + c0);
  const uint32_t widx = c0 + 1u + lane;
  const uint32_t wv = (widx <= n3) ? ld_index<FRESH>(e.P + widx) : 0xffffffffu;
  // off = number of window entries <= p (the window is sorted): binary search
  // over the 32 lane values with shuffles
  uint32_t off = 0;
#pragma unroll
  for (uint32_t step = 16; step > 0; step >>= 1) {
    const uint32_t probe = __shfl_sync(0xffffffffu, wv, (off + step - 1u) & 31u);
    if (probe <= p) off += step;
  }
  const uint32_t w31 = __shfl_sync(0xffffffffu, wv, 31);  // every lane takes part
  if (off == 31u && w31 <= p) off = 32u;
  const uint32_t prev = __shfl_sync(0xffffffffu, wv, (off > 0 ? off - 1u : 0u) & 31u);
  uint32_t cell = c0 + off, Pc = (off == 0) ? Pc0 : prev;
  if (act && off >= 32) {
    cell = upper_bound<FRESH>(e.P, c0 + 32u, n3, p) - 1u;
    Pc = ld_index<FRESH>(e.P + cell);
  }
  *cell_out = cell;
  *j_out = p - Pc;
  return act;
}

// (1) injection point uniform in the cell (Philox block 0, which also holds the
// frequency quantile), the emission frequency from the tabulated inverse CDF
// and the thermal speed in cells.
template <class R>
__device__ __forceinline__ void emit_draw0(const TransportArgs<R>& a, const EmitBox<R>& e, uint32_t cell, uint32_t j,
                                           R f[3], R* xi, R* vt) {
  using A = Ar<R>;
  R uq;
  Draws<R>::position(KStream{a.ks, e.box}, cell, j, f, &uq);
  R tq = A::mul(uq, (R)(a.M - 1));
  int k;
  const R fr = A::sub(tq, quant_node<R>(tq, a.M, &k));
  R q0 = __ldg(a.quant + k), q1 = __ldg(a.quant + k + 1);
  *xi = A::add(q0, A::mul(fr, A::sub(q1, q0)));
  *vt = A::sqr(A::mul(__ldg(e.T + cell), e.cth));
}

// The rest of a packet's emission (all lanes of the warp call it; lanes with
// act false take no part): isotropic direction (Philox blocks 1, 2, ...),
// u0, the Amanatides-Woo set-up and the resonance test in the home cell;
// packets resonant at home are tallied (warp-aggregated), the others take
// their first step and are queued in their home super-tile's bucket.
template <class R, bool P2>
__device__ __forceinline__ void emit_rest(const TransportArgs<R>& a, const EmitBox<R>& e, bool act, uint32_t cell,
                                          uint32_t j, const R f[3], R xi, R vt, uint64_t& my_abs,
                                          uint64_t& my_cross) {
  using A = Ar<R>;
  using V = typename Vec4<R>::T;
  const int lane = threadIdx.x & 31;
  const uint32_t n = e.n;
  const R one = (R)1, two = (R)2, zero = (R)0;
  bool home = false, queued = false;
  Ray<R> r;
  R nx = zero, ny = zero, nz = one;
  if (act) {
    const KStream ks{a.ks, e.box};
    // isotropic direction (Marsaglia 1972): the first accepted of the candidate
    // pairs t = 0, 1, ... (each Philox block is computed once for the pairs it
    // holds).  The pairs of the first block are tested side by side; the loop
    // over later blocks runs for the few packets that reject all of them.
    {
      typename Draws<R>::Block blk = Draws<R>::block(ks, cell, j, 0);
      R ua, ub;
      Draws<R>::pair_from(blk, 0, &ua, &ub);
      R v1 = A::sub(A::mul(two, ua), one), v2 = A::sub(A::mul(two, ub), one);
      R s = A::add(A::mul(v1, v1), A::mul(v2, v2));
      bool ok = s < one && s > zero;
      int t = 1;
      if (Draws<R>::kPairs == 2) {  // the block's second pair
        Draws<R>::pair_from(blk, 1, &ua, &ub);
        const R w1 = A::sub(A::mul(two, ua), one), w2 = A::sub(A::mul(two, ub), one);
        const R sw = A::add(A::mul(w1, w1), A::mul(w2, w2));
        if (!ok && sw < one && sw > zero) { v1 = w1; v2 = w2; s = sw; ok = true; }
        t = 2;
      }
      for (; !ok && t < 32; ++t) {
        if (Draws<R>::first_of_block(t)) blk = Draws<R>::block(ks, cell, j, t);
        Draws<R>::pair_from(blk, t, &ua, &ub);
        v1 = A::sub(A::mul(two, ua), one);
        v2 = A::sub(A::mul(two, ub), one);
        s = A::add(A::mul(v1, v1), A::mul(v2, v2));
        ok = s < one && s > zero;
      }
      if (ok) {
        R fac = A::mul(two, A::sqr(A::sub(one, s)));
        nx = A::mul(v1, fac); ny = A::mul(v2, fac); nz = A::sub(one, A::mul(two, s));
      }
    }
    r.knx = A::mul(e.kappa, nx); r.kny = A::mul(e.kappa, ny); r.knz = A::mul(e.kappa, nz);
    V Uh = e.vel[cell];
    R dh = A::add(A::add(A::mul(r.knx, Uh.x), A::mul(r.kny, Uh.y)), A::mul(r.knz, Uh.z));
    r.u0 = A::add(A::mul(xi, vt), dh);
    e.tl.template coords<P2>(cell, &r.ix, &r.iy, &r.iz);
    axis_setup<R>(nx, &r.tDx, &r.sx);
    axis_setup<R>(ny, &r.tDy, &r.sy);
    axis_setup<R>(nz, &r.tDz, &r.sz);
    // distance to the first face along each axis (f in (0,1): an axis with
    // tDelta = inf gets tMax = inf)
    r.tMx = A::mul(r.sx < 0 ? f[0] : A::sub(one, f[0]), r.tDx);
    r.tMy = A::mul(r.sy < 0 ? f[1] : A::sub(one, f[1]), r.tDy);
    r.tMz = A::mul(r.sz < 0 ? f[2] : A::sub(one, f[2]), r.tDz);
    r.kc = 0;
    int res = march_cell<R, P2>(r, Uh, n);  // home cell (res == 2 impossible with kc = 0)
    home = res == 1;
    queued = res == 0;
    my_cross += r.kc;
    if (home) ++my_abs;
  }
  // warp-aggregated tally of the packets resonant at home (mostly one cell per warp)
  const uint32_t key = home ? cell : 0xffffffffu;
  const unsigned m = __match_any_sync(0xffffffffu, key);
  if (home && lane == __ffs(m) - 1) atomicAdd(e.tally + cell, (uint32_t)__popc(m));
  // queue the others after their first step, in their home super-tile's bucket
  const unsigned qm = __ballot_sync(0xffffffffu, queued);
  if (qm) {
    const uint32_t bk = queued ? e.bk0 + e.tl.template at<P2>(cell) : 0xffffffffu;
    const unsigned gm = __match_any_sync(0xffffffffu, bk) & qm;
    unsigned long long qb = 0;
    const int leader = __ffs(gm) - 1;
    if (queued && lane == leader) qb = atomicAdd(&a.bfill[bk], (unsigned long long)__popc(gm));
    qb = __shfl_sync(0xffffffffu, qb, leader < 0 ? 0 : leader);
    if (queued) {
      uint64_t slot = a.boff[bk] + qb + __popc(gm & ((1u << lane) - 1u));
      uint32_t c1 = P2 ? (((r.iz << e.tl.lg) | r.iy) << e.tl.lg) | r.ix : (r.iz * n + r.iy) * n + r.ix;
      constexpr int QV = QueueVecs<R>::value;
      V q0v, q1v;
      q0v.x = bits_to<R>(c1); q0v.y = r.tMx; q0v.z = r.tMy; q0v.w = r.tMz;
      if (QV == 2) {
        q1v.x = nx; q1v.y = ny; q1v.z = nz; q1v.w = r.u0;
      } else {
        q1v.x = r.sx < 0 ? -r.tDx : r.tDx; q1v.y = r.sy < 0 ? -r.tDy : r.tDy; q1v.z = r.sz < 0 ? -r.tDz : r.tDz;
        q1v.w = r.u0;
        V q2v;
        q2v.x = r.knx; q2v.y = r.kny; q2v.z = r.knz; q2v.w = zero;
        a.queue[QV * slot + 2] = q2v;
      }
      a.queue[QV * slot] = q0v;
      a.queue[QV * slot + 1] = q1v;
    }
  }
}

// One warp emits the packets base .. base + 31 of one box (N packets).
template <class R, bool P2, bool FRESH = false>
__device__ __forceinline__ void emit_warp(const TransportArgs<R>& a, const EmitBox<R>& e, uint32_t base, uint32_t N,
                                          uint64_t& my_abs, uint64_t& my_cross) {
  uint32_t cell, j;
  const bool act = emit_locate<R, FRESH>(e, base, N, &cell, &j);
  R f[3] = {(R)0, (R)0, (R)0}, xi = (R)0, vt = (R)0;
  if (act) emit_draw0<R>(a, e, cell, j, f, &xi, &vt);
  emit_rest<R, P2>(a, e, act, cell, j, f, xi, vt, my_abs, my_cross);
}

// A packet emitted at or below the line centre (xi <= 0) is resonant in its
// home cell whatever its direction: u0 - kappa n.U_home = (xi v_t + d) - d
// with d = kappa n.U_home is <= 0 by the monotonicity of rounding, and the
// exit distance is >= 0.  This holds exactly when xi v_t is not NaN (v_t
// finite) and d is finite (|U| components <= 1e30 keep kappa n.U far from
// overflow); such packets need no direction and are tallied at once.
template <class R>
__device__ __forceinline__ bool home_without_direction(R xi, R vt, const typename Vec4<R>::T& U) {
  const R big = (R)1e30, vmax = sizeof(R) == 4 ? (R)3.4028234e38f : (R)1.7976931348623157e308;
  return xi <= (R)0 && vt <= vmax && fabs(U.x) <= big && fabs(U.y) <= big && fabs(U.z) <= big;
}

// Emission in 64-packet windows.  The first Philox block of every packet
// gives its frequency; the packets with xi <= 0 (about half) are absorbed at
// home without a direction.  The others wait in a per-warp ring in shared
// memory and are finished 32 at a time, so the warp's lanes stay busy in the
// costly part (direction, ray set-up, home test); leftovers carry over to the
// next window and are flushed at the end (and, in batches, at a change of box).
constexpr uint32_t kStash = 96;  // < 32 left over + 64 new
template <class R>
struct EmitStash {
  uint32_t cell[kStash], j[kStash];
  R f0[kStash], f1[kStash], f2[kStash], xi[kStash], vt[kStash];
};

// Finish up to 32 packets from the head of the ring (head, count: warp-uniform).
template <class R, bool P2>
__device__ __forceinline__ void emit_finish32(const TransportArgs<R>& a, const EmitBox<R>& e, EmitStash<R>& st,
                                              uint32_t& head, uint32_t& count, uint64_t& my_abs,
                                              uint64_t& my_cross) {
  const int lane = threadIdx.x & 31;
  const uint32_t take = count < 32u ? count : 32u;
  const bool act = (uint32_t)lane < take;
  uint32_t k = head + lane;
  if (k >= kStash) k -= kStash;
  uint32_t cell = 0, j = 0;
  R f[3] = {(R)0, (R)0, (R)0}, xi = (R)0, vt = (R)0;
  if (act) {
    cell = st.cell[k]; j = st.j[k];
    f[0] = st.f0[k]; f[1] = st.f1[k]; f[2] = st.f2[k];
    xi = st.xi[k]; vt = st.vt[k];
  }
  __syncwarp();  // read before the slots are reused
  head += take;
  if (head >= kStash) head -= kStash;
  count -= take;
  emit_rest<R, P2>(a, e, act, cell, j, f, xi, vt, my_abs, my_cross);
}

template <class R, bool P2>
__device__ __forceinline__ void emit_flush(const TransportArgs<R>& a, const EmitBox<R>& e, EmitStash<R>& st,
                                           uint32_t& head, uint32_t& count, uint64_t& my_abs, uint64_t& my_cross) {
  while (count > 0) emit_finish32<R, P2>(a, e, st, head, count, my_abs, my_cross);
}

template <class R, bool P2, bool FRESH = false>
__device__ __forceinline__ void emit_window64(const TransportArgs<R>& a, const EmitBox<R>& e, EmitStash<R>& st,
                                              uint32_t base, uint32_t N, uint32_t& head, uint32_t& count,
                                              uint64_t& my_abs, uint64_t& my_cross) {
  using V = typename Vec4<R>::T;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t cell, j;
    const bool act = emit_locate<R, FRESH>(e, base + 32u * h, N, &cell, &j);
    R f[3] = {(R)0, (R)0, (R)0}, xi = (R)0, vt = (R)0;
    bool early = false;
    if (act) {
      emit_draw0<R>(a, e, cell, j, f, &xi, &vt);
      const V Uh = e.vel[cell];
      early = home_without_direction<R>(xi, vt, Uh);
    }
    // home tally of the early packets (warp-aggregated)
    const uint32_t key = early ? cell : 0xffffffffu;
    const unsigned m = __match_any_sync(0xffffffffu, key);
    if (early && lane == __ffs(m) - 1) atomicAdd(e.tally + cell, (uint32_t)__popc(m));
    if (early) ++my_abs;
    // the others to the ring, in lane order after the waiting ones
    const bool pend = act && !early;
    const unsigned pm = __ballot_sync(0xffffffffu, pend);
    if (pend) {
      uint32_t k = head + count + __popc(pm & lt);
      if (k >= kStash) k -= kStash;
      st.cell[k] = cell; st.j[k] = j;
      st.f0[k] = f[0]; st.f1[k] = f[1]; st.f2[k] = f[2];
      st.xi[k] = xi; st.vt[k] = vt;
    }
    count += __popc(pm);
  }
  __syncwarp();
  while (count >= 32u) emit_finish32<R, P2>(a, e, st, head, count, my_abs, my_cross);
}

// The same window for batches, whose consecutive windows may belong to
// different boxes: every waiting packet is finished before it returns (one
// call site of the costly part keeps the batch kernels' register budget).
template <class R, bool P2, bool FRESH = false>
__device__ __forceinline__ void emit_window64_drain(const TransportArgs<R>& a, const EmitBox<R>& e, EmitStash<R>& st,
                                              uint32_t base, uint32_t N, uint64_t& my_abs, uint64_t& my_cross) {
  using V = typename Vec4<R>::T;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  uint32_t npend = 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t cell, j;
    const bool act = emit_locate<R, FRESH>(e, base + 32u * h, N, &cell, &j);
    R f[3] = {(R)0, (R)0, (R)0}, xi = (R)0, vt = (R)0;
    bool early = false;
    if (act) {
      emit_draw0<R>(a, e, cell, j, f, &xi, &vt);
      const V Uh = e.vel[cell];
      early = home_without_direction<R>(xi, vt, Uh);
    }
    // home tally of the early packets (warp-aggregated)
    const uint32_t key = early ? cell : 0xffffffffu;
    const unsigned m = __match_any_sync(0xffffffffu, key);
    if (early && lane == __ffs(m) - 1) atomicAdd(e.tally + cell, (uint32_t)__popc(m));
    if (early) ++my_abs;
    // the others to the stash, in lane order after the pending ones
    const bool pend = act && !early;
    const unsigned pm = __ballot_sync(0xffffffffu, pend);
    if (pend) {
      const uint32_t k = npend + __popc(pm & lt);
      st.cell[k] = cell; st.j[k] = j;
      st.f0[k] = f[0]; st.f1[k] = f[1]; st.f2[k] = f[2];
      st.xi[k] = xi; st.vt[k] = vt;
    }
    npend += __popc(pm);
  }
  __syncwarp();
  for (uint32_t r0 = 0; r0 < npend; r0 += 32) {
    const uint32_t k = r0 + lane;
    const bool act = k < npend;
    uint32_t cell = 0, j = 0;
    R f[3] = {(R)0, (R)0, (R)0}, xi = (R)0, vt = (R)0;
    if (act) {
      cell = st.cell[k]; j = st.j[k];
      f[0] = st.f0[k]; f[1] = st.f1[k]; f[2] = st.f2[k];
      xi = st.xi[k]; vt = st.vt[k];
    }
    emit_rest<R, P2>(a, e, act, cell, j, f, xi, vt, my_abs, my_cross);
  }
  __syncwarp();  // the stash is reused by the next window
}

// Resident blocks per SM of the emission (registers and the shared-memory ring:
// with the ring a sixth block measured slower, 1.83 against 1.74 ms at 256^3).
template <class R> constexpr int emit_occupancy() { return sizeof(R) == 4 ? 5 : 4; }

template <class R, bool P2>
__global__ void __launch_bounds__(TT, emit_occupancy<R>()) k_emit(TransportArgs<R> a) {
  const EmitBox<R> e{a.P, a.first, (uint32_t)a.n3, (uint32_t)a.n, a.vel, a.T, a.tally, a.kappa, a.cth, 0u, a.tl, 0u};
  const uint32_t N = __ldg(a.P + a.n3);  // packets actually allocated
  __shared__ EmitStash<R> stash[TT / 32];
  EmitStash<R>& st = stash[threadIdx.x >> 5];
  uint64_t my_abs = 0, my_cross = 0;
  uint32_t head = 0, count = 0;
  const uint64_t warps_total = (uint64_t)gridDim.x * (TT / 32);
  for (uint64_t base = ((uint64_t)blockIdx.x * (TT / 32) + (threadIdx.x >> 5)) * 64; base < N;
       base += warps_total * 64)
    emit_window64<R, P2>(a, e, st, (uint32_t)base, N, head, count, my_abs, my_cross);
  emit_flush<R, P2>(a, e, st, head, count, my_abs, my_cross);
  add_counters(a.sc, my_abs, 0, my_cross);
}

// March of the queued packets.  Persistent warps take chunks of a.chunk queued
// packets (never straddling a bucket) from a shared counter in queue order, so
// the warps advance through the super-tile buckets together and the cells
// they touch stay close in memory; each warp refills its idle lanes from its
// current chunk, so that lanes stay busy whatever the spread of path lengths.
// Cells a lane marches per round between two votes of its warp.  The walk of
// the traversal does not depend on the velocities, so a round first steps the
// traversal through its cells and gathers their velocities together, then runs
// the resonance tests in order: the lane waits on memory once per round rather
// than once per cell.  The arithmetic of every cell is the same as one cell at
// a time; only the order of the loads changes.
#ifndef REC_MARCH_AHEAD
#define REC_MARCH_AHEAD 4
#endif
template <class R> struct MarchAhead { static constexpr int value = sizeof(R) == 4 ? REC_MARCH_AHEAD : 2; };

// Resident blocks per SM of the march (register budget per thread; a batch
// keeps the box of each lane's packet in registers).
template <class R, bool MB, bool RS = false> constexpr int march_occupancy() {
  return RS ? (sizeof(R) == 4 ? 3 : 2)
            : (MB ? 3 : (sizeof(R) == 4 ? (MarchAhead<R>::value > 4 ? 3 : MarchAhead<R>::value > 2 ? 4 : 5) : 3));
}

__device__ __forceinline__ void transport_end_batch(const BoxDev* bxs, int B, const unsigned long long* bfill,
                                                    rec_stats* st);

// P2: the box side is a power of two (cell index by shifts and masks).
// MB: batched context; the lanes of a warp may hold packets of different boxes.
template <class R, bool P2, bool MB, bool RS = false>
__global__ void __launch_bounds__(TT, (march_occupancy<R, MB, RS>())) k_march(TransportArgs<R> a, const BoxDev* bxs,
                                                                              int B, const BoxStep* bst,
                                                                              rec_stats* st) {
  static_assert(!RS || (P2 && !MB), "region sweeps: single box of power-of-two side");
  using V = typename Vec4<R>::T;
  const int lane = threadIdx.x & 31;
  const uint32_t n = (uint32_t)a.n;
  const uint32_t lg = P2 ? (uint32_t)(__ffs((int)n) - 1) : 0u;
  // region sweeps: bucket of the open chunk and of the lane's packet (its
  // super-tile), 0xffffffff for a packet that marches without a limit
  uint32_t cbk = 0, lbk = 0;
  bool rqp = false;  // the lane's packet leaves its region: queue it again
  __shared__ BoxCounters cnt;
  if (MB) box_counters_clear(cnt, B);
  // box of the lane's packet (batch) and of the open chunk
  const V* lvel = a.vel;
  uint32_t* ltally = a.tally;
  uint32_t ln = n;
  R lkappa = a.kappa;
  int lbox = -1, cbox = 0;
  const V* cvel = a.vel;
  uint32_t* ctally = a.tally;
  uint32_t cn = n;
  R ckappa = a.kappa;
  const uint64_t n_chunks = a.cpre[a.nb];
  uint64_t chunk = 0;
  uint64_t pos = 0, end = 0;  // queue slots [pos, end) left in the current chunk
  bool have = false;          // a chunk is open
  bool more = n_chunks > 0;
  bool active = false;
  uint32_t cell = 0;
  Ray<R> r;
  r.kc = 0;
  V Uc;
  uint64_t my_abs = 0, my_cap = 0, my_cross = 0;
  for (;;) {
    unsigned idle = __ballot_sync(0xffffffffu, !active);
    if (more && __popc(idle) >= a.refill) {
      // refill idle lanes in lane order from the warp's chunks
      while (idle && more) {
        if (!have || pos >= end) {
          // next chunk in queue order, shared by all warps: the warps in flight
          // stay on neighbouring chunks, so their rays start close together
          unsigned long long nc = 0;
          if (lane == 0) nc = atomicAdd(&a.sc->march_next, 1ull);
          chunk = __shfl_sync(0xffffffffu, nc, 0);
          if (chunk >= n_chunks) { more = false; break; }
          // bucket of this chunk: last b with cpre[b] <= chunk (uniform over the warp)
          uint32_t lo = 0, hi = (uint32_t)a.nb;
          while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (__ldg(a.cpre + mid) <= chunk) lo = mid;
            else hi = mid;
          }
          const uint64_t k0 = (chunk - __ldg(a.cpre + lo)) * a.chunk;
          pos = a.boff[lo] + k0;
          end = pos + min((uint64_t)a.chunk, (uint64_t)(a.bfill[lo] - k0));
          have = true;
          if (RS) cbk = lo;
          if (MB) {  // box of this bucket: last b with bk0 <= lo
            cbox = last_le(B, lo, [&](int i) { return bxs[i].bk0; });
            cvel = (const V*)bxs[cbox].vel4;
            ctally = bxs[cbox].tally;
            cn = bxs[cbox].n;
            ckappa = (R)bst[cbox].kappa;
          }
        }
        const uint32_t take = (uint32_t)min((uint64_t)__popc(idle), end - pos);
        const uint32_t rank = __popc(idle & ((1u << lane) - 1u));
        if (((idle >> lane) & 1u) && rank < take) {
          const uint64_t slot = pos + rank;
          constexpr int QV = QueueVecs<R>::value;
          if (RS) lbk = cbk;
          if (RS && a.resumed) {
            // a full state queued again by an earlier sweep
            const V q0v = a.queue[3 * slot], q1v = a.queue[3 * slot + 1], q2v = a.queue[3 * slot + 2];
            cell = to_bits<R>(q0v.x);
            r.ix = cell & (n - 1u); r.iy = (cell >> lg) & (n - 1u); r.iz = cell >> (2u * lg);
            r.tMx = q0v.y; r.tMy = q0v.z; r.tMz = q0v.w;
            r.sx = q1v.x < (R)0 ? -1 : 1; r.tDx = fabs(q1v.x);
            r.sy = q1v.y < (R)0 ? -1 : 1; r.tDy = fabs(q1v.y);
            r.sz = q1v.z < (R)0 ? -1 : 1; r.tDz = fabs(q1v.z);
            r.u0 = q1v.w;
            r.knx = q2v.x; r.kny = q2v.y; r.knz = q2v.z;
            r.kc = to_bits<R>(q2v.w);
            Uc = lvel[cell];
            active = true;
          } else {
          const V q0v = a.queue[QV * slot], q1v = a.queue[QV * slot + 1];
          if (MB) {
            if (lbox != cbox) {  // counters of the previous box to shared memory
              if (lbox >= 0) box_counters_add(cnt, lbox, my_abs, my_cap, my_cross);
              my_abs = my_cap = my_cross = 0;
              lbox = cbox;
            }
            lvel = cvel;
            ltally = ctally;
            ln = cn;
            lkappa = ckappa;
          }
          cell = to_bits<R>(q0v.x);
          if (P2) {
            r.ix = cell & (n - 1u); r.iy = (cell >> lg) & (n - 1u); r.iz = cell >> (2u * lg);
          } else if (MB) {
            r.ix = cell % ln; r.iy = (cell / ln) % ln; r.iz = cell / (ln * ln);
          } else {
            a.tl.template coords<false>(cell, &r.ix, &r.iy, &r.iz);
          }
          r.tMx = q0v.y; r.tMy = q0v.z; r.tMz = q0v.w;
          r.u0 = q1v.w;
          if (QV == 2) {  // tDelta and kappa n exactly as the emission formed them
            axis_setup<R>(q1v.x, &r.tDx, &r.sx);
            axis_setup<R>(q1v.y, &r.tDy, &r.sy);
            axis_setup<R>(q1v.z, &r.tDz, &r.sz);
            r.knx = Ar<R>::mul(lkappa, q1v.x); r.kny = Ar<R>::mul(lkappa, q1v.y); r.knz = Ar<R>::mul(lkappa, q1v.z);
          } else {
            const V q2v = a.queue[QV * slot + 2];
            r.sx = q1v.x < (R)0 ? -1 : 1; r.tDx = fabs(q1v.x);
            r.sy = q1v.y < (R)0 ? -1 : 1; r.tDy = fabs(q1v.y);
            r.sz = q1v.z < (R)0 ? -1 : 1; r.tDz = fabs(q1v.z);
            r.knx = q2v.x; r.kny = q2v.y; r.knz = q2v.z;
          }
          r.kc = 1;  // the step out of the home cell
          Uc = lvel[cell];
          active = true;
          }
        }
        // lanes taken this round leave the idle set (the lowest `take` idle lanes)
        unsigned taken = 0, m = idle;
        for (uint32_t t = 0; t < take; ++t) { unsigned bb = m & (0u - m); taken |= bb; m ^= bb; }
        idle &= ~taken;
        pos += take;
      }
    }
    if (!__any_sync(0xffffffffu, active)) break;  // no packet left in the warp
    if (active) {
      // one round of kA cells: cell 0 is the current one (velocity in Uc); the
      // walk records each cell's exit distance and gathers the velocity of the
      // cell after it, then the cells are tested in order
      constexpr int kA = MarchAhead<R>::value;
      R se[kA];
      V Un[kA];
      uint32_t cl[kA + 1];
      cl[0] = cell;
      const uint32_t kc0 = r.kc;
#pragma unroll
      for (int k = 0; k < kA; ++k) {
        bool ax0, ax1, ax2;
        se[k] = dda_exit(r, &ax0, &ax1, &ax2);
        dda_advance<R, P2>(r, ax0, ax1, ax2, se[k], ln);
        cl[k + 1] = P2 ? (((r.iz << lg) | r.iy) << lg) | r.ix : (r.iz * ln + r.iy) * ln + r.ix;
        Un[k] = lvel[cl[k + 1]];
      }
      int res = 0;
      uint32_t kend = 0, cend = 0;
#pragma unroll
      for (int k = 0; k < kA; ++k) {
        const R dc = doppler(r, k == 0 ? Uc : Un[k - 1]);
        if (res == 0) {
          // resonance in cell k at path length u0 - kappa n.U: absorb unless beyond its exit
          if (Ar<R>::sub(r.u0, dc) <= se[k]) { res = 1; kend = (uint32_t)k; cend = cl[k]; }
          else if (kc0 + (uint32_t)k >= kMaxCrossings) { res = 2; kend = (uint32_t)k; }
        }
      }
      if (res == 0) {
        cell = cl[kA];
        Uc = Un[kA - 1];
        if (RS && a.halo && lbk != 0xffffffffu) {
          // still inside the super-tile of its bucket widened by the halo?
          // (periodic: offsets from the region's low corner modulo n)
          const uint32_t tlg = a.tl.tlg, ntl = lg - tlg, ntm = (1u << ntl) - 1u, m = n - 1u;
          const uint32_t span = (1u << tlg) + 2u * a.halo;
          const uint32_t ox = (((lbk & ntm) << tlg) - a.halo) & m;
          const uint32_t oy = ((((lbk >> ntl) & ntm) << tlg) - a.halo) & m;
          const uint32_t oz = (((lbk >> (2u * ntl)) << tlg) - a.halo) & m;
          if (((r.ix - ox) & m) >= span || ((r.iy - oy) & m) >= span || ((r.iz - oz) & m) >= span) {
            rqp = true;
            active = false;
          }
        }
      } else {
        active = false;
        my_cross += kc0 + kend - 1;  // crossings up to the last cell; the first was counted at emission
        if (res == 1) { atomicAdd(ltally + cend, 1u); ++my_abs; }
        else ++my_cap;
      }
    }
    if (RS) {
      // packets that left their region: appended to the second queue as full
      // states (the current cell is the next to test), counted in the bucket
      // of the super-tile they have reached
      const unsigned rm = __ballot_sync(0xffffffffu, rqp);
      if (rm) {
        // the warp's part of the second queue
        const uint32_t part = (blockIdx.x * (TT / 32) + (threadIdx.x >> 5)) & (uint32_t)(kRqParts - 1);
        unsigned long long qb = 0;
        const int leader = __ffs(rm) - 1;
        if (lane == leader) qb = atomicAdd(&a.rqn[part], (unsigned long long)__popc(rm));
        qb = __shfl_sync(0xffffffffu, qb, leader);
        const uint64_t k = qb + __popc(rm & ((1u << lane) - 1u));
        const bool stored = rqp && k < a.rq_part;
        const uint64_t slot = (uint64_t)part * a.rq_part + k;
        if (stored) {
          V q0v, q1v, q2v;
          q0v.x = bits_to<R>(cell); q0v.y = r.tMx; q0v.z = r.tMy; q0v.w = r.tMz;
          q1v.x = r.sx < 0 ? -r.tDx : r.tDx; q1v.y = r.sy < 0 ? -r.tDy : r.tDy; q1v.z = r.sz < 0 ? -r.tDz : r.tDz;
          q1v.w = r.u0;
          q2v.x = r.knx; q2v.y = r.kny; q2v.z = r.knz; q2v.w = bits_to<R>(r.kc);
          a.rq[3 * slot] = q0v;
          a.rq[3 * slot + 1] = q1v;
          a.rq[3 * slot + 2] = q2v;
        }
        const unsigned sm = __ballot_sync(0xffffffffu, stored);
        const uint32_t bk = stored ? a.tl.template at<true>(cell) : 0xffffffffu;
        const unsigned gm = __match_any_sync(0xffffffffu, bk) & sm;
        if (stored && lane == __ffs(gm) - 1) atomicAdd(&a.rcount[bk], (unsigned long long)__popc(gm));
        if (rqp && !stored) {  // the second queue is full: this packet marches on without a limit
          active = true;
          lbk = 0xffffffffu;
        }
        if (__any_sync(0xffffffffu, rqp && !stored) && lane == 0) atomicOr(&a.sc->flags, 16);
        rqp = false;
      }
    }
  }
  if (MB) {
    if (lbox >= 0) box_counters_add(cnt, lbox, my_abs, my_cap, my_cross);
    box_counters_flush(cnt, bxs, B);
    // the last block to finish closes the call: queued counts, tally totals, statistics
    if (last_block_done(&a.sc->counter)) {
      transport_end_batch(bxs, B, a.bfill, st);
      if (threadIdx.x == 0) a.sc->counter = 0;
    }
  } else {
    add_counters(a.sc, my_abs, my_cap, my_cross);
  }
}

// Region sweeps, between two march launches (one block): the entries each
// bucket received in the second queue become the march queue of the next
// sweep: bucket offsets (exclusive prefix of the counts), fills, march-chunk
// prefix; the counts and the placement fills are reset.
__global__ void __launch_bounds__(1024) k_requeue_scan(unsigned long long* rcount, unsigned long long* boff,
                                                       unsigned long long* bfill, unsigned long long* cpre,
                                                       unsigned long long* scnt, unsigned long long* rqn, int nb,
                                                       DevScalars* sc, uint32_t chunk, uint64_t part_cap) {
  constexpr int NTH = 1024;
  static_assert(kRqParts <= NTH, "one thread per part");
  __shared__ unsigned long long pe[NTH], pc[NTH];
  __shared__ unsigned long long stored;
  if (threadIdx.x == 0) stored = 0;
  __syncthreads();
  if (threadIdx.x < kRqParts) {  // entries each part holds for the placement; append counters reset
    const unsigned long long m = rqn[threadIdx.x], c = m < part_cap ? m : part_cap;
    rqn[kRqParts + threadIdx.x] = c;
    rqn[threadIdx.x] = 0;
    atomicAdd(&stored, c);
  }
  const int per = (nb + NTH - 1) / NTH;
  const int b0 = threadIdx.x * per, b1 = min(nb, (int)(threadIdx.x + 1) * per);
  unsigned long long se = 0, sc_ = 0;
  for (int b = b0; b < b1; ++b) {
    const unsigned long long f = __ldcg(&rcount[b]);
    se += f;
    sc_ += (f + chunk - 1) / chunk;
  }
  pe[threadIdx.x] = se;
  pc[threadIdx.x] = sc_;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long re = 0, rc = 0;
    for (int t = 0; t < NTH; ++t) {
      const unsigned long long ve = pe[t], vc = pc[t];
      pe[t] = re; pc[t] = rc;
      re += ve; rc += vc;
    }
    cpre[nb] = rc;
    sc->requeued += stored;
    sc->march_next = 0;
  }
  __syncthreads();
  unsigned long long re = pe[threadIdx.x], rc = pc[threadIdx.x];
  for (int b = b0; b < b1; ++b) {
    const unsigned long long f = __ldcg(&rcount[b]);
    boff[b] = re;
    bfill[b] = f;
    cpre[b] = rc;
    re += f;
    rc += (f + chunk - 1) / chunk;
    rcount[b] = 0;
    scnt[b] = 0;
  }
}

// Region sweeps: every entry of the second queue to its bucket's range of the
// march queue (order within a bucket is free: the march of a packet does not
// depend on the others).
template <class R>
__global__ void __launch_bounds__(TT) k_requeue_place(TransportArgs<R> a, unsigned long long* scnt) {
  using V = typename Vec4<R>::T;
  const int lane = threadIdx.x & 31;
  for (int part = blockIdx.x; part < kRqParts; part += gridDim.x) {
  const uint64_t m = a.rqn[kRqParts + part], off = (uint64_t)part * a.rq_part;
  for (uint64_t base = (uint64_t)(threadIdx.x >> 5) * 32; base < m; base += TT) {
    const uint64_t i = base + lane;
    const bool act = i < m;
    V q0v, q1v, q2v;
    uint32_t bk = 0xffffffffu;
    if (act) {
      q0v = a.rq[3 * (off + i)]; q1v = a.rq[3 * (off + i) + 1]; q2v = a.rq[3 * (off + i) + 2];
      bk = a.tl.template at<true>(to_bits<R>(q0v.x));
    }
    const unsigned am = __ballot_sync(0xffffffffu, act);
    const unsigned gm = __match_any_sync(0xffffffffu, bk) & am;
    const int leader = __ffs(gm) - 1;
    unsigned long long qb = 0;
    if (act && lane == leader) qb = atomicAdd(&scnt[bk], (unsigned long long)__popc(gm));
    qb = __shfl_sync(0xffffffffu, qb, leader < 0 ? 0 : leader);
    if (act) {
      const uint64_t slot = a.boff[bk] + qb + __popc(gm & ((1u << lane) - 1u));
      a.queue[3 * slot] = q0v;
      a.queue[3 * slot + 1] = q1v;
      a.queue[3 * slot + 2] = q2v;
    }
  }
  }
}

__global__ void k_transport_end(DevScalars* sc, rec_stats* st) {
  if (threadIdx.x != 0) return;
  sc->tally_total += sc->absorbed;
  if (sc->capped) sc->flags |= 2;
  if (st) {
    st->emitted = sc->emitted;
    st->absorbed = sc->absorbed;
    st->capped = sc->capped;
    st->crossings = sc->crossings;
    st->queued = sc->qtail;
    st->requeued = sc->requeued;
    st->flags = sc->flags;
  }
}

template <class R>
cudaError_t run_transport(rec_ctx* c, int step, double z, rec_stats* st) {
  const rec_box& b = c->box;
  Stream s{(uint32_t)c->params.seed, (uint32_t)(c->params.seed >> 32) ^ (uint32_t)step, 0u};
  const bool p2 = (b.n & (b.n - 1)) == 0;
  const rec_tuning& tu = c->tune;
  const Tiles tl = make_tiles(b.n, tu.tile);
  const int nb = (int)(tl.nt * tl.nt * tl.nt);
  {
    GroupTimer t(c, kTAlloc, 4);
    k_alloc_max<R><<<c->grid, kPassThreads, 0, c->stream>>>((const R*)b.emis, c->n3, c->sc, c->part);
    k_alloc_sum<R><<<c->alloc_blocks, AT, 0, c->stream>>>((const R*)b.emis, c->n3, b.n_packets, s, c->sc,
                                                          c->partQ, c->P);
    cudaMemsetAsync(c->bcap, 0, sizeof(unsigned long long) * nb, c->stream);
    k_alloc_prefix<R><<<c->alloc_blocks, AT, 0, c->stream>>>((const R*)b.emis, c->n3, b.n_packets, c->sc,
                                                             c->partQ, c->P, c->first, tl, c->bcap);
    k_bucket_offsets<<<1, 1024, 0, c->stream>>>(c->bcap, c->bfill, nb);
  }
  double kappa, cth;
  transport_scalars(c->cosmo, b.n, z, &kappa, &cth);
  TransportArgs<R> a;
  a.P = c->P;
  a.first = c->first;
  a.n3 = c->n3;
  a.n = b.n;
  a.vel = (const typename Vec4<R>::T*)b.vel4;
  a.T = (const R*)b.T;
  a.quant = (const R*)c->quant;
  a.M = c->params.n_quantiles;
  a.kappa = (R)kappa;
  a.cth = (R)cth;
  a.strm = s;
  a.ks = key_schedule(s.k0, s.k1);
  a.tally = b.tally;
  a.sc = c->sc;
  a.queue = (typename Vec4<R>::T*)c->queue;
  a.tl = tl;
  a.nb = nb;
  a.boff = c->bcap;
  a.bfill = c->bfill;
  a.cpre = c->cpre;
  a.chunk = (uint32_t)tu.march_chunk;
  a.refill = tu.march_refill;
  a.rq = nullptr;
  a.rcount = nullptr;
  a.rqn = nullptr;
  a.rq_part = 0;
  a.halo = 0;
  a.resumed = 0;
  {
    GroupTimer t(c, kTEmit, 2);
    const int eb = c->sm_count * tu.emit_blocks_per_sm;
    if (p2) k_emit<R, true><<<eb, TT, 0, c->stream>>>(a);
    else k_emit<R, false><<<eb, TT, 0, c->stream>>>(a);
    k_bucket_scan<<<1, 1024, 0, c->stream>>>(c->bfill, c->cpre, nb, c->sc, a.chunk);
  }
  const uint32_t halo = (uint32_t)tu.march_halo;
  const bool sweeps = p2 && halo > 0 && c->rqueue && ((uint32_t)tu.tile + 2u * halo) < (uint32_t)b.n;
  if (!sweeps) {
    GroupTimer t(c, kTMarch, 1);
    const int mb = c->sm_count * tu.march_blocks_per_sm;
    if (p2) k_march<R, true, false><<<mb, TT, 0, c->stream>>>(a, nullptr, 1, nullptr, nullptr);
    else k_march<R, false, false><<<mb, TT, 0, c->stream>>>(a, nullptr, 1, nullptr, nullptr);
  } else {
    // region sweeps: each march leaves the packets that stray beyond the halo of
    // their bucket's super-tile in the second queue; those are placed by the
    // super-tile they reached and marched by the next sweep; the last sweep has
    // no limit, so every packet ends
    GroupTimer t(c, kTMarch, 3 * kMaxSweeps - 2);
    const int mb = c->sm_count * tu.march_blocks_per_sm;
    a.rq = (typename Vec4<R>::T*)c->rqueue;
    a.rcount = c->rcount;
    a.rqn = c->rqn;
    a.rq_part = c->rq_cap / kRqParts;
    cudaMemsetAsync(c->rqn, 0, sizeof(unsigned long long) * kRqParts, c->stream);
    for (int k = 0; k < kMaxSweeps; ++k) {
      if (k > 0) {
        k_requeue_scan<<<1, 1024, 0, c->stream>>>(c->rcount, c->bcap, c->bfill, c->cpre, c->scnt, c->rqn, nb, c->sc,
                                                  a.chunk, a.rq_part);
        k_requeue_place<R><<<kRqParts, TT, 0, c->stream>>>(a, c->scnt);
      }
      a.resumed = k > 0;
      a.halo = (k + 1 < kMaxSweeps) ? halo : 0u;
      k_march<R, true, false, true><<<mb, TT, 0, c->stream>>>(a, nullptr, 1, nullptr, nullptr);
    }
  }
  {
    GroupTimer t(c, kTEnd, 1);
    k_transport_end<<<1, 32, 0, c->stream>>>(c->sc, st);
  }
  return cudaGetLastError();
}

// ---- batched contexts: every phase is one launch over all boxes ------------------

// Allocation blocks: kAllocChunk cells of one box each; box of block g = last b
// with ablk0 <= g.
__device__ __forceinline__ int alloc_box(const BoxDev* bxs, int B, uint32_t g) {
  return last_le(B, g, [&](int i) { return bxs[i].ablk0; });
}

// Allocation phases of a batch as functions of the allocation block g of ng
// (blockIdx.x of a per-phase launch, or a virtual block of the persistent one).
template <class R>
__device__ __forceinline__ void alloc_max_batch(const BoxDev* bxs, int B, DevScalars* gsc, double* part, uint32_t g,
                                                uint32_t ng) {
  const int b = alloc_box(bxs, B, g);
  const BoxDev& d = bxs[b];
  const int64_t c0 = (int64_t)(g - d.ablk0) * kAllocChunk + (int64_t)threadIdx.x * kAllocItems;
  R v[kAllocItems];
  load_items<R>((const R*)d.emis, c0, d.n3, v);
  R m = (R)0;
  int bad = 0;
#pragma unroll
  for (int k = 0; k < kAllocItems; ++k) {
    if (c0 + k >= d.n3) continue;
    const R r = v[k];
    if (!(r >= (R)0) || isinf(r)) bad = 1;
    else m = fmax(m, r);
  }
  bad = __syncthreads_or(bad);
  double bm = block_max<AT>((double)m);
  if (threadIdx.x == 0) {
    part[(size_t)g * kMaxSums + 0] = bm;
    part[(size_t)g * kMaxSums + 1] = bad ? 1.0 : 0.0;
  }
  if (!last_block_done(&gsc->counter, ng)) return;
  // one warp per box: maximum over the box's blocks
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < B; i += AT / 32) {
    const uint32_t g0 = bxs[i].ablk0;
    const uint32_t g1 = (i + 1 < B) ? bxs[i + 1].ablk0 : ng;
    double mx = 0.0, anybad = 0.0;
    for (uint32_t g = g0 + lane; g < g1; g += 32) {
      mx = fmax(mx, __ldcg(part + (size_t)g * kMaxSums));
      anybad = fmax(anybad, __ldcg(part + (size_t)g * kMaxSums + 1));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      anybad = fmax(anybad, __shfl_xor_sync(0xffffffffu, anybad, o));
    }
    if (lane == 0) {
      DevScalars* sc = bxs[i].sc;
      sc->rmax = anybad > 0.0 ? 0.0 : mx;
      sc->flags &= ~(2 | 4 | 16);
      if (anybad > 0.0) sc->flags |= 4;
    }
  }
  if (threadIdx.x == 0) gsc->counter = 0;
}
template <class R>
__global__ void __launch_bounds__(AT) k_alloc_max_batch(const BoxDev* bxs, int B, DevScalars* gsc, double* part) {
  alloc_max_batch<R>(bxs, B, gsc, part, blockIdx.x, gridDim.x);
}

template <class R>
__device__ __forceinline__ void alloc_sum_batch(const BoxDev* bxs, int B, uint32_t k0, uint32_t k1, DevScalars* gsc,
                                                unsigned long long* partQ, uint32_t g, uint32_t ng) {
  const int b = alloc_box(bxs, B, g);
  const BoxDev& d = bxs[b];
  const R rmax = (R)__ldcg(&d.sc->rmax);
  uint64_t acc = 0;
  if (rmax > (R)0) {
    const int64_t c0 = (int64_t)(g - d.ablk0) * kAllocChunk + (int64_t)threadIdx.x * kAllocItems;
    R v[kAllocItems];
    load_items<R>((const R*)d.emis, c0, d.n3, v);
#pragma unroll
    for (int k = 0; k < kAllocItems; ++k) acc += quantised<R>(v[k], rmax);
  }
  uint64_t incl;
  uint64_t tot = block_scan_incl(acc, &incl);
  if (threadIdx.x == 0) partQ[g] = tot;
  if (!last_block_done(&gsc->alloc_counter, ng)) return;
  // one warp per box: exclusive scan of its block sums (in place), the
  // systematic-sampling offset and the box's packet total
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = warp; i < B; i += AT / 32) {
    const BoxDev& e = bxs[i];
    const uint32_t g0 = e.ablk0;
    const uint32_t g1 = (i + 1 < B) ? bxs[i + 1].ablk0 : ng;
    uint64_t run = 0;
    for (uint32_t gb = g0; gb < g1; gb += 32) {
      const uint32_t g = gb + lane;
      uint64_t q = g < g1 ? __ldcg(&partQ[g]) : 0ull, v = q;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      if (g < g1) partQ[g] = run + v - q;
      run += __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) {
      DevScalars* sc = e.sc;
      const uint64_t sumQ = run;
      U4 r = draw(Stream{k0, k1, (uint32_t)i}, 0u, 0u, kAllocBlock);
      uint64_t w = ((uint64_t)r.b << 32) | r.a;
      uint64_t npk = (sumQ > 0) ? e.npk : 0;
      sc->sumQ = sumQ;
      sc->alloc_u = sumQ > 0 ? w % sumQ : 0;
      e.P[e.n3] = (uint32_t)npk;
      sc->emitted = npk;
      sc->absorbed = 0;
      sc->capped = 0;
      sc->crossings = 0;
      sc->qtail = 0;
      if (sumQ == 0 && e.npk > 0) sc->flags |= 4;
    }
  }
  if (threadIdx.x == 0) gsc->alloc_counter = 0;
}
template <class R>
__global__ void __launch_bounds__(AT) k_alloc_sum_batch(const BoxDev* bxs, int B, uint32_t k0, uint32_t k1,
                                                        DevScalars* gsc, unsigned long long* partQ) {
  alloc_sum_batch<R>(bxs, B, k0, k1, gsc, partQ, blockIdx.x, gridDim.x);
}

template <class R>
__device__ __forceinline__ void alloc_prefix_batch(const BoxDev* bxs, int B, const unsigned long long* partQ,
                                                   unsigned long long* bcap, uint32_t g) {
  const int b = alloc_box(bxs, B, g);
  const BoxDev& d = bxs[b];
  const DevScalars* sc = d.sc;
  const int64_t c0 = (int64_t)(g - d.ablk0) * kAllocChunk + (int64_t)threadIdx.x * kAllocItems;
  alloc_prefix_block<R>((const R*)d.emis, d.n3, d.npk, __ldcg(&sc->sumQ), __ldcg(&sc->alloc_u), (R)__ldcg(&sc->rmax),
                        __ldcg(&partQ[g]), c0, d.P, d.first, Tiles{d.n, d.nt, d.lg, d.mn, d.mn2, d.tlg}, d.bk0, bcap);
}
template <class R>
__global__ void __launch_bounds__(AT) k_alloc_prefix_batch(const BoxDev* bxs, int B, const unsigned long long* partQ,
                                                           unsigned long long* bcap) {
  alloc_prefix_batch<R>(bxs, B, partQ, bcap, blockIdx.x);
}

// Emission over the batch packet space (each box padded to a multiple of 64,
// so a warp's 64-packet window belongs to one box).  FRESH: the packet prefixes and
// box scalars were written earlier in the same launch (read through L2).
template <class R, bool FRESH>
__device__ __forceinline__ void emit_batch_body_drain(const TransportArgs<R>& a, const BoxDev* bxs, const BoxStep* bst, int B,
                                                uint64_t tot_pk) {
  using V = typename Vec4<R>::T;
  __shared__ BoxCounters cnt;
  __shared__ EmitStash<R> stash[TT / 32];
  EmitStash<R>& st = stash[threadIdx.x >> 5];
  box_counters_clear(cnt, B);
  uint64_t my_abs = 0, my_cross = 0;
  int cur = -1;
  uint64_t lo_pk = 1, hi_pk = 0;  // packet range of box cur (empty before the first lookup)
  uint32_t N = 0;
  const uint64_t warps_total = (uint64_t)gridDim.x * (TT / 32);
  // 64-packet windows: every box's packet space is padded to a multiple of 64
  for (uint64_t gbase = ((uint64_t)blockIdx.x * (TT / 32) + (threadIdx.x >> 5)) * 64; gbase < tot_pk;
       gbase += warps_total * 64) {
    if (gbase < lo_pk || gbase >= hi_pk) {  // next box (uniform over the warp)
      const int b = last_le(B, gbase, [&](int i) { return bxs[i].pk0; });
      if (cur >= 0) box_counters_add(cnt, cur, my_abs, 0, my_cross);
      my_abs = my_cross = 0;
      cur = b;
      lo_pk = bxs[b].pk0;
      hi_pk = (b + 1 < B) ? bxs[b + 1].pk0 : tot_pk;
      N = ld_index<FRESH>(bxs[b].P + bxs[b].n3);  // packets actually allocated to this box
    }
    const uint64_t base = gbase - lo_pk;
    if (base >= N) continue;  // padding of the packet space
    const BoxDev& d = bxs[cur];
    const EmitBox<R> e{d.P, d.first, (uint32_t)d.n3, d.n, (const V*)d.vel4, (const R*)d.T, d.tally,
                       (R)__ldcg(&bst[cur].kappa), (R)__ldcg(&bst[cur].cth),
                       (uint32_t)cur, Tiles{d.n, d.nt, d.lg, d.mn, d.mn2, d.tlg}, d.bk0};
    // power-of-two sides take cell coordinates by shifts and the periodic wrap
    // by masks; other sides by exact multiply-high divisions (the binary64 form
    // keeps one path: both would not fit its register budget)
    if (sizeof(R) == 4 && d.p2) emit_window64_drain<R, true, FRESH>(a, e, st, (uint32_t)base, N, my_abs, my_cross);
    else emit_window64_drain<R, false, FRESH>(a, e, st, (uint32_t)base, N, my_abs, my_cross);
  }
  if (cur >= 0) box_counters_add(cnt, cur, my_abs, 0, my_cross);
  box_counters_flush(cnt, bxs, B);
}
// Binary32 batches: the ring carried over between windows (as the single-box
// emission), flushed at each change of box; one cell-coordinate path (exact
// multiply-high divisions) for every side keeps the kernel within its registers.
template <class R, bool FRESH>
__device__ __forceinline__ void emit_batch_body_ring(const TransportArgs<R>& a, const BoxDev* bxs, const BoxStep* bst,
                                                     int B, uint64_t tot_pk) {
  using V = typename Vec4<R>::T;
  __shared__ BoxCounters cnt;
  __shared__ EmitStash<R> stash[TT / 32];
  EmitStash<R>& st = stash[threadIdx.x >> 5];
  box_counters_clear(cnt, B);
  uint64_t my_abs = 0, my_cross = 0;
  int cur = -1;
  uint64_t lo_pk = 1, hi_pk = 0;  // packet range of box cur (empty before the first lookup)
  uint32_t N = 0;
  uint32_t head = 0, count = 0;   // the warp's ring of packets waiting for their direction
  auto box_of = [&](int b) {
    const BoxDev& d = bxs[b];
    return EmitBox<R>{d.P, d.first, (uint32_t)d.n3, d.n, (const V*)d.vel4, (const R*)d.T, d.tally,
                      (R)__ldcg(&bst[b].kappa), (R)__ldcg(&bst[b].cth),
                      (uint32_t)b, Tiles{d.n, d.nt, d.lg, d.mn, d.mn2, d.tlg}, d.bk0};
  };
  const uint64_t warps_total = (uint64_t)gridDim.x * (TT / 32);
  for (uint64_t gbase = ((uint64_t)blockIdx.x * (TT / 32) + (threadIdx.x >> 5)) * 64; gbase < tot_pk;
       gbase += warps_total * 64) {
    if (gbase < lo_pk || gbase >= hi_pk) {  // next box (uniform over the warp)
      if (count) emit_flush<R, false>(a, box_of(cur), st, head, count, my_abs, my_cross);
      const int b = last_le(B, gbase, [&](int i) { return bxs[i].pk0; });
      if (cur >= 0) box_counters_add(cnt, cur, my_abs, 0, my_cross);
      my_abs = my_cross = 0;
      cur = b;
      lo_pk = bxs[b].pk0;
      hi_pk = (b + 1 < B) ? bxs[b + 1].pk0 : tot_pk;
      N = ld_index<FRESH>(bxs[b].P + bxs[b].n3);  // packets actually allocated to this box
    }
    const uint64_t base = gbase - lo_pk;
    if (base >= N) continue;  // padding of the packet space
    emit_window64<R, false, FRESH>(a, box_of(cur), st, (uint32_t)base, N, head, count, my_abs, my_cross);
  }
  if (count) emit_flush<R, false>(a, box_of(cur), st, head, count, my_abs, my_cross);
  if (cur >= 0) box_counters_add(cnt, cur, my_abs, 0, my_cross);
  box_counters_flush(cnt, bxs, B);
}

template <class R, bool FRESH>
__device__ __forceinline__ void emit_batch_body(const TransportArgs<R>& a, const BoxDev* bxs, const BoxStep* bst, int B,
                                                uint64_t tot_pk) {
  if (sizeof(R) == 4) emit_batch_body_ring<R, FRESH>(a, bxs, bst, B, tot_pk);
  else emit_batch_body_drain<R, FRESH>(a, bxs, bst, B, tot_pk);
}

template <class R>
__global__ void __launch_bounds__(TT, 4) k_emit_batch(TransportArgs<R> a, const BoxDev* bxs, const BoxStep* bst,
                                                      int B, uint64_t tot_pk) {
  emit_batch_body<R, false>(a, bxs, bst, B, tot_pk);
}

struct BoxStepArgs {
  BoxStep s[kMaxBoxes];
};
__global__ void k_set_box_step(BoxStepArgs p, BoxStep* out, int B) {
  for (int b = threadIdx.x; b < B; b += blockDim.x) out[b] = p.s[b];
}

__device__ __forceinline__ void transport_end_batch(const BoxDev* bxs, int B, const unsigned long long* bfill,
                                                    rec_stats* st) {
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const BoxDev& d = bxs[b];
    DevScalars* sc = d.sc;
    unsigned long long q = 0;
    const uint32_t nb = d.nt * d.nt * d.nt;
    for (uint32_t k = 0; k < nb; ++k) q += __ldcg(&bfill[d.bk0 + k]);
    // the counters were added by other blocks' atomics: read them through L2
    const unsigned long long absorbed = __ldcg(&sc->absorbed), capped = __ldcg(&sc->capped);
    sc->qtail = q;
    sc->tally_total = __ldcg(&sc->tally_total) + absorbed;
    if (capped) atomicOr(&sc->flags, 2);
    if (st) {
      st[b].emitted = __ldcg(&sc->emitted);
      st[b].absorbed = absorbed;
      st[b].capped = capped;
      st[b].crossings = __ldcg(&sc->crossings);
      st[b].queued = q;
      st[b].requeued = 0;
      st[b].flags = __ldcg(&sc->flags);
    }
  }
}
__global__ void k_transport_end_batch(const BoxDev* bxs, int B, const unsigned long long* bfill, rec_stats* st) {
  transport_end_batch(bxs, B, bfill, st);
}

// The allocation and the emission of a batched transport call as phases of
// one persistent cooperative launch, separated by bounded grid barriers: box
// transport scalars, bucket capacities cleared and the allocation maxima;
// quantised sums and their scans; packet prefixes; bucket offsets; emission;
// march chunk prefix.  The allocation phases run the allocation blocks of the
// per-phase kernels as virtual blocks.  A barrier that gives up ends the launch
// (flags bit 3 of the batch record) and the march that follows finds no work.
template <class R>
__global__ void __launch_bounds__(AT, 4) k_batch_front(TransportArgs<R> a, const BoxDev* bxs, BoxStep* bst,
                                                       BoxStepArgs bs, int B, uint32_t k0, uint32_t k1,
                                                       DevScalars* gsc, double* part, unsigned long long* partQ,
                                                       unsigned long long* cpre, uint32_t n_ablk, uint64_t tot_pk,
                                                       uint32_t limit) {
  if (blockIdx.x == 0)
    for (int b = threadIdx.x; b < B; b += AT) bst[b] = bs.s[b];
  for (int i = blockIdx.x * AT + threadIdx.x; i < a.nb; i += gridDim.x * AT) a.boff[i] = 0ull;
  if (blockIdx.x == 0 && threadIdx.x == 0) gsc->march_next = ~0ull >> 1;  // no march work until the chunks exist
  for (uint32_t g = blockIdx.x; g < n_ablk; g += gridDim.x) alloc_max_batch<R>(bxs, B, gsc, part, g, n_ablk);
  if (!grid_barrier(&gsc->bar, &gsc->flags, limit)) return;
  for (uint32_t g = blockIdx.x; g < n_ablk; g += gridDim.x) alloc_sum_batch<R>(bxs, B, k0, k1, gsc, partQ, g, n_ablk);
  if (!grid_barrier(&gsc->bar, &gsc->flags, limit)) return;
  for (uint32_t g = blockIdx.x; g < n_ablk; g += gridDim.x) alloc_prefix_batch<R>(bxs, B, partQ, a.boff, g);
  if (!grid_barrier(&gsc->bar, &gsc->flags, limit)) return;
  if (blockIdx.x == 0) bucket_offsets_block<AT>(a.boff, a.bfill, a.nb);
  if (!grid_barrier(&gsc->bar, &gsc->flags, limit)) return;
  emit_batch_body<R, true>(a, bxs, bst, B, tot_pk);
  if (!grid_barrier(&gsc->bar, &gsc->flags, limit)) return;
  if (blockIdx.x == 0) bucket_scan_block<AT>(a.bfill, cpre, a.nb, gsc, a.chunk);
}

template <class R>
cudaError_t run_transport_batch(rec_ctx* c, int step, double z, rec_stats* st) {
  const int B = c->n_boxes;
  const uint32_t k0 = (uint32_t)c->params.seed, k1 = (uint32_t)(c->params.seed >> 32) ^ (uint32_t)step;
  const int nb = c->tot_buckets;
  BoxStepArgs bs;
  for (int b = 0; b < B; ++b) transport_scalars(c->cosmo, (int)c->hbx[b].n, z, &bs.s[b].kappa, &bs.s[b].cth);
  TransportArgs<R> a;
  std::memset(&a, 0, sizeof(a));
  a.quant = (const R*)c->quant;
  a.M = c->params.n_quantiles;
  a.strm = Stream{k0, k1, 0u};
  a.ks = key_schedule(k0, k1);
  a.sc = c->gsc;
  a.queue = (typename Vec4<R>::T*)c->queue;
  a.nb = nb;
  a.boff = c->bcap;
  a.bfill = c->bfill;
  a.cpre = c->cpre;
  a.chunk = (uint32_t)c->tune.march_chunk;
  a.refill = c->tune.march_refill;
  if (c->batch_front_grid == 0) {  // resident blocks of the persistent front (cooperative launch)
    int per_sm = 0, coop = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_front<R>, AT, 0);
    cudaGetLastError();
    c->batch_front_grid = (e == cudaSuccess && coop && per_sm > 0) ? per_sm * c->sm_count : -1;
  }
  if (c->batch_front_grid > 0) {
    // allocation + emission in one persistent launch, then the march (which closes the call)
    GroupTimer t(c, kTEmit, 1);
    const BoxDev* bxs = c->bx;
    BoxStep* bst = c->bstep;
    DevScalars* gsc = c->gsc;
    double* part = c->part;
    unsigned long long* partQ = c->partQ;
    unsigned long long* cpre = c->cpre;
    uint32_t n_ablk = (uint32_t)c->tot_ablk;
    uint64_t tot_pk = c->tot_pk;
    uint32_t limit = c->wait_limit;
    int Bv = B;
    uint32_t k0v = k0, k1v = k1;
    void* args[] = {&a, &bxs, &bst, &bs, &Bv, &k0v, &k1v, &gsc, &part, &partQ, &cpre, &n_ablk, &tot_pk, &limit};
    cudaError_t e = cudaLaunchCooperativeKernel((void*)k_batch_front<R>, c->batch_front_grid, AT, args, 0, c->stream);
    if (e != cudaSuccess) return e;
  } else {
    {
      GroupTimer t(c, kTAlloc, 5);
      k_set_box_step<<<1, kMaxBoxes, 0, c->stream>>>(bs, c->bstep, B);
      k_alloc_max_batch<R><<<c->tot_ablk, AT, 0, c->stream>>>(c->bx, B, c->gsc, c->part);
      k_alloc_sum_batch<R><<<c->tot_ablk, AT, 0, c->stream>>>(c->bx, B, k0, k1, c->gsc, c->partQ);
      cudaMemsetAsync(c->bcap, 0, sizeof(unsigned long long) * nb, c->stream);
      k_alloc_prefix_batch<R><<<c->tot_ablk, AT, 0, c->stream>>>(c->bx, B, c->partQ, c->bcap);
      k_bucket_offsets<<<1, 1024, 0, c->stream>>>(c->bcap, c->bfill, nb);
    }
    {
      GroupTimer t(c, kTEmit, 2);
      k_emit_batch<R><<<c->sm_count * c->tune.emit_blocks_per_sm, TT, 0, c->stream>>>(a, c->bx, c->bstep, B,
                                                                                      c->tot_pk);
      k_bucket_scan<<<1, 1024, 0, c->stream>>>(c->bfill, c->cpre, nb, c->gsc, a.chunk);
    }
  }
  {
    GroupTimer t(c, kTMarch, 1);
    k_march<R, false, true><<<c->sm_count * c->tune.march_blocks_per_sm, TT, 0, c->stream>>>(a, c->bx, B, c->bstep,
                                                                                             st);
  }
  return cudaGetLastError();
}

}  // namespace

// Largest resident blocks per SM of the emission and the march (their
// launch bounds), for the checks of rec_set_tuning.
int sweep_march_limit(bool mixed) {
  return mixed ? march_occupancy<float, false, true>() : march_occupancy<double, false, true>();
}

void transport_limits(bool mixed, bool batch, int* emit_max, int* march_max) {
  *emit_max = batch ? 4 : (mixed ? emit_occupancy<float>() : emit_occupancy<double>());
  *march_max = batch ? march_occupancy<float, true>()
                     : (mixed ? march_occupancy<float, false>() : march_occupancy<double, false>());
}

cudaError_t launch_transport(rec_ctx* c, int step, double z, rec_stats* st) {
  if (c->params.precision == REC_PREC_MIXED) return run_transport<float>(c, step, z, st);
  return run_transport<double>(c, step, z, st);
}

cudaError_t launch_transport_batch(rec_ctx* c, int step, double z, rec_stats* st) {
  if (c->params.precision == REC_PREC_MIXED) return run_transport_batch<float>(c, step, z, st);
  return run_transport_batch<double>(c, step, z, st);
}

}  // namespace rec
