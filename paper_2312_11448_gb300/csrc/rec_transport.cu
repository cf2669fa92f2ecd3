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
//                   128-bit integer arithmetic
//   k_transport     one packet per thread: warp-cooperative cell lookup in P,
//                   Philox draws, emission, Amanatides-Woo march, warp-aggregated
//                   tally atomics
//   k_transport_end counters to the statistics record
// The march is written operation by operation with round-to-nearest
// intrinsics (never contracted into FMA), in binary32 for the mixed form and
// binary64 for the FP64 form, so its integer results are reproducible.

#include <cmath>

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
    uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
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
constexpr uint32_t kAllocBlock = 0x000A110Cu;  // counter block of the allocation offset

// Uniform deviates strictly inside (0,1), exactly representable.
__device__ __forceinline__ float u01f(uint32_t r) { return __uint2float_rn((r >> 8) | 1u) * 0x1p-24f; }
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
  static __device__ __forceinline__ float sqr(float a) { return __fsqrt_rn(a); }
  static __device__ __forceinline__ float inf() { return __int_as_float(0x7f800000); }
  static __device__ __forceinline__ int trunc(float a) { return __float2int_rz(a); }
};
template <> struct Ar<double> {
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
  static __device__ __forceinline__ double sqr(double a) { return __dsqrt_rn(a); }
  static __device__ __forceinline__ double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
  static __device__ __forceinline__ int trunc(double a) { return __double2int_rz(a); }
};

template <class R> struct Vec4;
template <> struct Vec4<float> { using T = float4; };
template <> struct Vec4<double> { using T = double4; };

// Per-precision draw layout.
template <class R> struct Draws;
template <> struct Draws<float> {
  // block 0: three cell offsets and the frequency quantile; blocks 1..16: two
  // direction pairs each
  static __device__ __forceinline__ void position(const Stream& s, uint32_t c, uint32_t j, float f[3], float* uq) {
    U4 r = draw(s, c, j, 0u);
    f[0] = u01f(r.a); f[1] = u01f(r.b); f[2] = u01f(r.c); *uq = u01f(r.d);
  }
  static __device__ __forceinline__ void pair(const Stream& s, uint32_t c, uint32_t j, int t, float* a, float* b) {
    U4 r = draw(s, c, j, 1u + (uint32_t)(t >> 1));
    if (t & 1) { *a = u01f(r.c); *b = u01f(r.d); }
    else { *a = u01f(r.a); *b = u01f(r.b); }
  }
};
template <> struct Draws<double> {
  // blocks 0, 1: three cell offsets and the quantile (two words per deviate);
  // blocks 2..33: one direction pair each
  static __device__ __forceinline__ void position(const Stream& s, uint32_t c, uint32_t j, double f[3], double* uq) {
    U4 r = draw(s, c, j, 0u), q = draw(s, c, j, 1u);
    f[0] = u01d(r.a, r.b); f[1] = u01d(r.c, r.d); f[2] = u01d(q.a, q.b); *uq = u01d(q.c, q.d);
  }
  static __device__ __forceinline__ void pair(const Stream& s, uint32_t c, uint32_t j, int t, double* a, double* b) {
    U4 r = draw(s, c, j, 2u + (uint32_t)t);
    *a = u01d(r.a, r.b); *b = u01d(r.c, r.d);
  }
};

// ---- allocation -------------------------------------------------------------------
template <class R>
__global__ void __launch_bounds__(kPassThreads) k_alloc_max(const R* emis, int64_t n3, DevScalars* sc, double* part) {
  double m = 0.0;
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * kPassThreads + threadIdx.x; i < n3; i += (int64_t)gridDim.x * kPassThreads) {
    double r = (double)emis[i];
    if (!(r >= 0.0) || isinf(r)) bad = 1;
    else m = fmax(m, r);
  }
  bad = __syncthreads_or(bad);
  double bm = block_max<kPassThreads>(m);
  if (threadIdx.x == 0) {
    part[(size_t)blockIdx.x * kMaxSums + 0] = bm;
    part[(size_t)blockIdx.x * kMaxSums + 1] = bad ? 1.0 : 0.0;
  }
  if (!last_block_done(&sc->counter)) return;
  double mx = combine_max<kPassThreads>(part, gridDim.x, kMaxSums, 0);
  double anybad = combine_max<kPassThreads>(part, gridDim.x, kMaxSums, 1);
  if (threadIdx.x == 0) {
    sc->rmax = anybad > 0.0 ? 0.0 : mx;  // invalid weights: emit nothing
    sc->flags &= ~(2 | 4);               // transport flags describe this call only
    if (anybad > 0.0) sc->flags |= 4;
    sc->counter = 0;
  }
}

template <class R>
__device__ __forceinline__ uint64_t quantised(R r, R rmax) {
  // Q = floor(2^31 r / r_max), the ratio rounded once in the working precision
  return (uint64_t)Ar<R>::mul(Ar<R>::div(r, rmax), (R)2147483648.0);
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

template <class R>
__global__ void __launch_bounds__(AT) k_alloc_sum(const R* emis, int64_t n3, uint64_t n_packets, Stream strm,
                                                  DevScalars* sc, unsigned long long* partQ, uint32_t* P) {
  const R rmax = (R)sc->rmax;
  uint64_t acc = 0;
  if (rmax > (R)0) {
    for (int k = 0; k < kAllocItems; ++k) {
      int64_t i = (int64_t)blockIdx.x * kAllocChunk + (int64_t)k * AT + threadIdx.x;
      if (i < n3) acc += quantised<R>(emis[i], rmax);
    }
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
    sc->alloc_counter = 0;
    if (sumQ == 0 && n_packets > 0) sc->flags |= 4;
  }
}

// floor((N * pre + u) / S) for N < 2^32, pre <= S < 2^64, u < S: a binary64
// estimate corrected with exact 128-bit products.
__device__ __forceinline__ uint32_t sys_floor(uint64_t N, uint64_t pre, uint64_t u, uint64_t S) {
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
    break;
  }
  return (uint32_t)q;
}

template <class R>
__global__ void __launch_bounds__(AT) k_alloc_prefix(const R* emis, int64_t n3, uint64_t n_packets, DevScalars* sc,
                                                     const unsigned long long* partQ, uint32_t* P) {
  const R rmax = (R)sc->rmax;
  const uint64_t S = sc->sumQ, u = sc->alloc_u;
  uint64_t run = partQ[blockIdx.x];
  for (int k = 0; k < kAllocItems; ++k) {
    int64_t i = (int64_t)blockIdx.x * kAllocChunk + (int64_t)k * AT + threadIdx.x;
    uint64_t q = (i < n3 && rmax > (R)0) ? quantised<R>(emis[i], rmax) : 0;
    uint64_t incl;
    uint64_t tot = block_scan_incl(q, &incl);
    if (i < n3) P[i] = (S > 0) ? sys_floor(n_packets, run + incl - q, u, S) : 0u;
    run += tot;
  }
}

// ---- transport ----------------------------------------------------------------------
template <class R>
struct TransportArgs {
  const uint32_t* P;
  int64_t n3;
  int n;
  const typename Vec4<R>::T* vel;
  const R* T;
  const R* quant;
  int M;
  R kappa, cth;
  Stream strm;
  uint32_t* tally;
  DevScalars* sc;
};

// First index k in [lo, hi] with P[k] > key (P[hi] > key holds).
__device__ __forceinline__ uint32_t upper_bound(const uint32_t* P, uint32_t lo, uint32_t hi, uint32_t key) {
  while (lo < hi) {
    uint32_t mid = lo + ((hi - lo) >> 1);
    if (__ldg(P + mid) > key) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

template <class R>
__global__ void __launch_bounds__(TT) k_transport(TransportArgs<R> a) {
  using A = Ar<R>;
  using V = typename Vec4<R>::T;
  __shared__ unsigned long long s_abs, s_cap, s_cross;
  if (threadIdx.x == 0) { s_abs = 0; s_cap = 0; s_cross = 0; }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t N = __ldg(a.P + a.n3);  // packets actually allocated
  const uint32_t n = (uint32_t)a.n;
  const uint32_t n3 = (uint32_t)a.n3;
  const R one = (R)1, two = (R)2, zero = (R)0;
  uint64_t my_abs = 0, my_cap = 0, my_cross = 0;
  const uint64_t warps_total = (uint64_t)gridDim.x * (TT / 32);
  for (uint64_t base = ((uint64_t)blockIdx.x * (TT / 32) + (threadIdx.x >> 5)) * 32; base < N;
       base += warps_total * 32) {
    const uint32_t p = (uint32_t)base + lane;
    const bool act = p < N;
    // ---- cell of each packet: lane 0 searches for the warp's first packet,
    // then a 32-cell window of P resolves the rest with ballots
    uint32_t c0 = 0;
    if (lane == 0) c0 = upper_bound(a.P, 0u, n3, (uint32_t)base) - 1u;
    c0 = __shfl_sync(0xffffffffu, c0, 0);
    const uint32_t Pc0 = __ldg(a.P + c0);
    const uint32_t widx = c0 + 1u + lane;
    const uint32_t wv = (widx <= n3) ? __ldg(a.P + widx) : 0xffffffffu;
    uint32_t off = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      unsigned b = __ballot_sync(0xffffffffu, wv <= (uint32_t)base + (uint32_t)k);
      if (lane == k) off = __popc(b);
    }
    const uint32_t prev = __shfl_sync(0xffffffffu, wv, (off > 0 ? off - 1u : 0u) & 31u);
    uint32_t cell = c0 + off, Pc = (off == 0) ? Pc0 : prev;
    if (act && off >= 32) {
      cell = upper_bound(a.P, c0 + 32u, n3, p) - 1u;
      Pc = __ldg(a.P + cell);
    }
    bool done = false;
    uint32_t kc = 0;
    uint32_t acell = cell;
    if (act) {
      const uint32_t j = p - Pc;
      // (1) injection point uniform in the cell, frequency quantile
      R f[3], uq;
      Draws<R>::position(a.strm, cell, j, f, &uq);
      // isotropic direction (Marsaglia 1972)
      R nx = zero, ny = zero, nz = one;
      for (int t = 0; t < 32; ++t) {
        R ua, ub;
        Draws<R>::pair(a.strm, cell, j, t, &ua, &ub);
        R v1 = A::sub(A::mul(two, ua), one), v2 = A::sub(A::mul(two, ub), one);
        R s = A::add(A::mul(v1, v1), A::mul(v2, v2));
        if (s < one && s > zero) {
          R fac = A::mul(two, A::sqr(A::sub(one, s)));
          nx = A::mul(v1, fac); ny = A::mul(v2, fac); nz = A::sub(one, A::mul(two, s));
          break;
        }
      }
      // emission frequency from the tabulated inverse CDF
      R tq = A::mul(uq, (R)(a.M - 1));
      int k = A::trunc(tq);
      if (k > a.M - 2) k = a.M - 2;
      R fr = A::sub(tq, (R)k);
      R q0 = __ldg(a.quant + k), q1 = __ldg(a.quant + k + 1);
      R xi = A::add(q0, A::mul(fr, A::sub(q1, q0)));
      R vt = A::sqr(A::mul(__ldg(a.T + cell), a.cth));
      R knx = A::mul(a.kappa, nx), kny = A::mul(a.kappa, ny), knz = A::mul(a.kappa, nz);
      V Uh = a.vel[cell];
      R dh = A::add(A::add(A::mul(knx, Uh.x), A::mul(kny, Uh.y)), A::mul(knz, Uh.z));
      R u0 = A::add(A::mul(xi, vt), dh);
      // Amanatides-Woo traversal
      uint32_t ix = cell % n, iy = (cell / n) % n, iz = cell / (n * n);
      R tMx, tMy, tMz, tDx, tDy, tDz;
      int sx, sy, sz;
      if (nx > zero) { sx = 1; tDx = A::div(one, nx); tMx = A::mul(A::sub(one, f[0]), tDx); }
      else if (nx < zero) { sx = -1; tDx = A::div(one, -nx); tMx = A::mul(f[0], tDx); }
      else { sx = 0; tDx = A::inf(); tMx = A::inf(); }
      if (ny > zero) { sy = 1; tDy = A::div(one, ny); tMy = A::mul(A::sub(one, f[1]), tDy); }
      else if (ny < zero) { sy = -1; tDy = A::div(one, -ny); tMy = A::mul(f[1], tDy); }
      else { sy = 0; tDy = A::inf(); tMy = A::inf(); }
      if (nz > zero) { sz = 1; tDz = A::div(one, nz); tMz = A::mul(A::sub(one, f[2]), tDz); }
      else if (nz < zero) { sz = -1; tDz = A::div(one, -nz); tMz = A::mul(f[2], tDz); }
      else { sz = 0; tDz = A::inf(); tMz = A::inf(); }
      uint32_t c = cell;
      V Uc = Uh;
      for (;;) {
        R dc = A::add(A::add(A::mul(knx, Uc.x), A::mul(kny, Uc.y)), A::mul(knz, Uc.z));
        int ax;
        R s_exit;
        if (tMx <= tMy && tMx <= tMz) { ax = 0; s_exit = tMx; }
        else if (tMy <= tMz) { ax = 1; s_exit = tMy; }
        else { ax = 2; s_exit = tMz; }
        // resonance in this cell at path length u0 - kappa n.U_c: absorb if not beyond the exit
        if (A::sub(u0, dc) <= s_exit) { done = true; break; }
        if (kc >= kMaxCrossings) break;
        if (ax == 0) { ix = (sx > 0) ? (ix + 1 == n ? 0 : ix + 1) : (ix == 0 ? n - 1 : ix - 1); tMx = A::add(tMx, tDx); }
        else if (ax == 1) { iy = (sy > 0) ? (iy + 1 == n ? 0 : iy + 1) : (iy == 0 ? n - 1 : iy - 1); tMy = A::add(tMy, tDy); }
        else { iz = (sz > 0) ? (iz + 1 == n ? 0 : iz + 1) : (iz == 0 ? n - 1 : iz - 1); tMz = A::add(tMz, tDz); }
        ++kc;
        c = (iz * n + iy) * n + ix;
        Uc = a.vel[c];
      }
      acell = c;
      my_cross += kc;
      if (done) ++my_abs;
      else ++my_cap;
    }
    // warp-aggregated tally: one atomic per distinct absorbing cell in the warp
    const bool absd = act && done;
    const uint32_t key = absd ? acell : 0xffffffffu;
    const unsigned m = __match_any_sync(0xffffffffu, key);
    if (absd && lane == __ffs(m) - 1) atomicAdd(a.tally + acell, (uint32_t)__popc(m));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    my_abs += __shfl_down_sync(0xffffffffu, my_abs, off);
    my_cap += __shfl_down_sync(0xffffffffu, my_cap, off);
    my_cross += __shfl_down_sync(0xffffffffu, my_cross, off);
  }
  if (lane == 0) {
    atomicAdd(&s_abs, (unsigned long long)my_abs);
    atomicAdd(&s_cap, (unsigned long long)my_cap);
    atomicAdd(&s_cross, (unsigned long long)my_cross);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&a.sc->absorbed, s_abs);
    atomicAdd(&a.sc->capped, s_cap);
    atomicAdd(&a.sc->crossings, s_cross);
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
    st->flags = sc->flags;
  }
}

template <class R>
cudaError_t run_transport(rec_ctx* c, int step, double z, rec_stats* st) {
  const rec_box& b = c->box;
  Stream s{(uint32_t)c->params.seed, (uint32_t)(c->params.seed >> 32) ^ (uint32_t)step, 0u};
  k_alloc_max<R><<<c->grid, kPassThreads, 0, c->stream>>>((const R*)b.emis, c->n3, c->sc, c->part);
  k_alloc_sum<R><<<c->alloc_blocks, AT, 0, c->stream>>>((const R*)b.emis, c->n3, b.n_packets, s, c->sc, c->partQ,
                                                        c->P);
  k_alloc_prefix<R><<<c->alloc_blocks, AT, 0, c->stream>>>((const R*)b.emis, c->n3, b.n_packets, c->sc, c->partQ,
                                                           c->P);
  double kappa, cth;
  transport_scalars(c->cosmo, b.n, z, &kappa, &cth);
  TransportArgs<R> a;
  a.P = c->P;
  a.n3 = c->n3;
  a.n = b.n;
  a.vel = (const typename Vec4<R>::T*)b.vel4;
  a.T = (const R*)b.T;
  a.quant = (const R*)c->quant;
  a.M = c->params.n_quantiles;
  a.kappa = (R)kappa;
  a.cth = (R)cth;
  a.strm = s;
  a.tally = b.tally;
  a.sc = c->sc;
  k_transport<R><<<c->transport_blocks, TT, 0, c->stream>>>(a);
  k_transport_end<<<1, 32, 0, c->stream>>>(c->sc, st);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_transport(rec_ctx* c, int step, double z, rec_stats* st) {
  if (c->params.precision == REC_PREC_MIXED) return run_transport<float>(c, step, z, st);
  return run_transport<double>(c, step, z, st);
}

}  // namespace rec
