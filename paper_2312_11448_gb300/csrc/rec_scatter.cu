// Resonant-scattering Ly-alpha Monte Carlo (Appendix A of arXiv:2312.11448).
//
// A photon injected at line centre (gas frame) at a random point of its cell
// repeats: thermally averaged cross-section of Eq. MC and mean free path
// l = 1/(sigma n_1s) in the cell it is in (step (2)); advance eps l (step (3));
// redshift dx = -zeta H dl / v_th (step (4)); scatter with probability
// 1 - exp(-eps) (steps (5)-(6)).  A scattering ends the photon (photo-
// ionisation of the n = 2 atom or two-photon decay) or re-emits it with the
// frequency of Eq. inout and a new isotropic direction (steps (7)-(8)).
// Photons whose gas-frame offset falls below -x_lost are lost by redshifting.
//
// GPU organisation: a persistent kernel, one photon per lane, lanes refilled
// from a global counter as their photons end (photon lifetimes span orders of
// magnitude).  The step itself is a few dozen FP64 operations and a shared-
// memory lookup of the Voigt table; the redistribution is much longer, so a
// warp gathers the lanes that must scatter and runs the redistribution for
// them together once enough are waiting.  This translation unit is built
// without contraction into fused multiply-adds, so that every operation rounds
// as written.

#include <cmath>
#include <vector>

#include "rec_internal.cuh"

namespace rec {
namespace {

constexpr int ST = 256;                   // threads per block of the Monte-Carlo kernel
constexpr int kVoigtNodes = 1281;         // nodes y_k = k / 128 on [0, 10]
constexpr double kVoigtStep = 1.0 / 128.0;
constexpr double kVoigtYmax = 10.0;
constexpr double kPiD = 3.14159265358979323846;
constexpr double kSqrtPiD = 1.77245385090551602730;
constexpr int kMaxTries = 100000;         // rejection tries per atom-velocity draw
constexpr unsigned kFull = 0xffffffffu;

// ---- Voigt function on the host: table nodes ----------------------------------
// H(a, y) = Re w(y + i a), w the Faddeeva function.  |z| < 10: Weideman's
// rational expansion (SIAM J. Numer. Anal. 31, 1497 (1994)) with 64 terms,
// w = 2 sum_n c_n Z^(n-1) / (L - i z)^2 + 1 / (sqrt(pi) (L - i z)),
// Z = (L + i z)/(L - i z), L = sqrt(64 / sqrt 2), c_n the cosine coefficients of
// exp(-t^2)(L^2 + t^2), t = L tan(theta/2), on 256 points; |z| >= 10: the
// asymptotic series (i / sqrt pi) sum_k (2k-1)!! / (2^k z^(2k+1)), 12 terms.
struct Faddeeva64 {
  static constexpr int N = 64;
  double L;
  double c[N + 1];
  Faddeeva64() {
    const int M = 2 * N;
    L = std::sqrt((double)N / std::sqrt(2.0));
    double F[M];
    for (int k = 0; k < M; ++k) {
      const double t = L * std::tan(kPiD * k / (2.0 * M));
      F[k] = std::exp(-t * t) * (L * L + t * t);
    }
    for (int n = 1; n <= N; ++n) {
      double s = F[0];
      for (int k = 1; k < M; ++k) s += 2.0 * F[k] * std::cos(kPiD * (double)k * n / M);
      c[n] = s / (2.0 * M);
    }
  }
  // w(zr + i zi) -> (wr, wi), zi > 0
  void eval(double zr, double zi, double* wr, double* wi) const {
    if (std::hypot(zr, zi) >= 10.0) { asym(zr, zi, wr, wi); return; }
    // D = L - i z = (L + zi) - i zr;  Z = (L + i z) / D = ((L - zi) + i zr) / D
    const double dr = L + zi, di = -zr;
    const double dd = dr * dr + di * di;
    const double nr = L - zi, ni = zr;
    const double Zr = (nr * dr + ni * di) / dd, Zi = (ni * dr - nr * di) / dd;
    double pr = c[N], pi = 0.0;
    for (int n = N - 1; n >= 1; --n) {
      const double tr = pr * Zr - pi * Zi, ti = pr * Zi + pi * Zr;
      pr = tr + c[n];
      pi = ti;
    }
    // 1/D and 1/D^2
    const double ir = dr / dd, ii = -di / dd;
    const double i2r = ir * ir - ii * ii, i2i = 2.0 * ir * ii;
    *wr = 2.0 * (pr * i2r - pi * i2i) + ir / kSqrtPiD;
    *wi = 2.0 * (pr * i2i + pi * i2r) + ii / kSqrtPiD;
  }
  static void asym(double zr, double zi, double* wr, double* wi) {
    const double d = zr * zr + zi * zi;
    const double ir = zr / d, ii = -zi / d;
    const double qr = ir * ir - ii * ii, qi = 2.0 * ir * ii;
    double tr = ir, ti = ii, sr = ir, si = ii;
    for (int k = 1; k < 12; ++k) {
      const double f = 0.5 * (2.0 * k - 1.0);
      const double nr = (tr * qr - ti * qi) * f, ni = (tr * qi + ti * qr) * f;
      tr = nr; ti = ni; sr += tr; si += ti;
    }
    *wr = -si / kSqrtPiD;
    *wi = sr / kSqrtPiD;
  }
};

// Values H and slopes H' = -2 (y H - a Im w) at the table nodes.
void voigt_nodes(double a, double* H, double* dH) {
  static const Faddeeva64 fw;
  for (int k = 0; k < kVoigtNodes; ++k) {
    const double y = k * kVoigtStep;
    double wr, wi;
    fw.eval(y, a, &wr, &wi);
    H[k] = wr;
    dH[k] = -2.0 * (y * wr - a * wi);
  }
}

// ---- Voigt function on the device ------------------------------------------------
__host__ __device__ __forceinline__ double voigt_asym(double t, double a) {
  const double d = t * t + a * a;
  const double ir = t / d, ii = -a / d;
  const double qr = ir * ir - ii * ii, qi = 2.0 * ir * ii;
  double tr = ir, ti = ii, si = ii;
  for (int k = 1; k < 12; ++k) {
    const double f = 0.5 * (2.0 * k - 1.0);
    const double nr = (tr * qr - ti * qi) * f, ni = (tr * qi + ti * qr) * f;
    tr = nr; ti = ni; si += ti;
  }
  return -si / kSqrtPiD;
}

// Cubic Hermite interpolation of the nodes for |y| < 10, the asymptotic series beyond.
__host__ __device__ __forceinline__ double voigt_eval(const double* H, const double* dH, double y, double a) {
  const double t = fabs(y);
  if (!(t < kVoigtYmax)) return voigt_asym(t, a);
  const double q = t / kVoigtStep;
  int k = (int)q;
  if (k > kVoigtNodes - 2) k = kVoigtNodes - 2;
  const double s = q - k;
  const double s1 = 1.0 - s;
  const double h00 = (1.0 + 2.0 * s) * s1 * s1, h10 = s * s1 * s1;
  const double h01 = s * s * (3.0 - 2.0 * s), h11 = s * s * (s - 1.0);
  return h00 * H[k] + h10 * kVoigtStep * dH[k] + h01 * H[k + 1] + h11 * kVoigtStep * dH[k + 1];
}

// ---- random numbers ---------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).
__device__ __forceinline__ void philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1,
                                       uint32_t out[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

__device__ __forceinline__ double u01(uint32_t lo, uint32_t hi) {
  const uint64_t w = ((uint64_t)hi << 32) | lo;
  return __ull2double_rn((w >> 11) | 1ull) * 0x1p-53;
}

// One photon's stream: key (seed low word, seed high word ^ step), counter
// (cell, photon index in the cell, block, 2^31 | box); two binary64 deviates
// per block, used in order.
struct McRng {
  uint32_t cell, j, blk, tag, k0, k1;
  double spare;
  bool have;
  __device__ __forceinline__ void init(uint32_t c, uint32_t jj, uint32_t key0, uint32_t key1, uint32_t box) {
    cell = c; j = jj; blk = 0; tag = 0x80000000u | box; k0 = key0; k1 = key1; have = false;
  }
  __device__ __forceinline__ double next() {
    if (have) { have = false; return spare; }
    uint32_t r[4];
    philox(cell, j, blk, tag, k0, k1, r);
    ++blk;
    spare = u01(r[2], r[3]);
    have = true;
    return u01(r[0], r[1]);
  }
};

// Unit disk by rejection (at most 64 tries; the fallback point is never
// reached in practice).
__device__ __forceinline__ void disk(McRng& s, double& v1, double& v2, double& r2) {
  for (int it = 0; it < 64; ++it) {
    v1 = 2.0 * s.next() - 1.0;
    v2 = 2.0 * s.next() - 1.0;
    r2 = v1 * v1 + v2 * v2;
    if (r2 < 1.0) return;
  }
  v1 = 0.3; v2 = 0.4; r2 = 0.25;
}

// Cut between the normal and Lorentzian parts of the atom-velocity envelope.
__device__ __forceinline__ double cut_u0(double t, double a) {
  if (t < 1.2) return -0.7;
  if (t >= 10.0) return sqrt(log(t * t / a) + 4.0);
  const double kt[6] = {1.2, 2.0, 3.0, 4.0, 6.0, 10.0};
  const double ku[6] = {1.1, 1.8, 2.5, 2.95, 3.4, 3.8};
  int i = 0;
  while (t >= kt[i + 1]) ++i;
  return ku[i] + (ku[i + 1] - ku[i]) * (t - kt[i]) / (kt[i + 1] - kt[i]);
}

// Parallel velocity of the scattering atom: density exp(-p^2)/((y-p)^2 + a^2)
// by exact rejection from the envelope exp(-p^2)/((t-u0)^2 + a^2) for p <= u0
// (normal proposal of variance 1/2) and exp(-max(u0,0)^2)/((t-p)^2 + a^2) for
// p > u0 (Lorentzian proposal), t = |y|; the result takes the sign of y.
__device__ double sample_ppar(McRng& s, double y, double a, unsigned long long* caps) {
  const double t = fabs(y);
  const double u0 = cut_u0(t, a);
  const double d0 = t - u0;
  const double m0 = u0 > 0.0 ? u0 : 0.0;
  const double W1 = 0.5 * kSqrtPiD * (1.0 + erf(u0)) / (d0 * d0 + a * a);
  const double W2 = exp(-m0 * m0) * (0.5 * kPiD + atan(d0 / a)) / a;
  const double P1 = W1 / (W1 + W2);
  for (int it = 0; it < kMaxTries; ++it) {
    double p, v1, v2, r2;
    if (s.next() < P1) {
      disk(s, v1, v2, r2);
      p = v1 * sqrt(-log(r2) / r2);
      if (p > u0) continue;
      const double d = t - p;
      if (s.next() * (d * d + a * a) >= d0 * d0 + a * a) continue;
    } else {
      disk(s, v1, v2, r2);
      p = t + a * (v1 / v2);
      if (p <= u0) continue;
      if (s.next() >= exp(m0 * m0 - p * p)) continue;
    }
    return y < 0.0 ? -p : p;
  }
  ++*caps;
  return 0.0;
}

// Eq. inout for isotropic scattering; k is replaced by the outgoing direction.
__device__ double redistribute(McRng& s, double y, double a, double k[3], unsigned long long* caps) {
  const double p = sample_ppar(s, y, a, caps);
  const double r = sqrt(-log(s.next()));
  const double mu = 2.0 * s.next() - 1.0;
  double v1, v2, r2;
  disk(s, v1, v2, r2);
  const double cb = (v1 * v1 - v2 * v2) / r2;
  disk(s, v1, v2, r2);
  const double cphi = (v1 * v1 - v2 * v2) / r2, sphi = 2.0 * v1 * v2 / r2;
  const double sm = sqrt(1.0 - mu * mu);
  // orthonormal basis of the plane normal to k (Duff et al., JCGT 6(1), 2017)
  const double sg = copysign(1.0, k[2]);
  const double aa = -1.0 / (sg + k[2]);
  const double bb = k[0] * k[1] * aa;
  const double e1x = 1.0 + sg * k[0] * k[0] * aa, e1y = sg * bb, e1z = -sg * k[0];
  const double e2x = bb, e2y = sg + k[1] * k[1] * aa, e2z = -k[1];
  const double nx = mu * k[0] + sm * (cphi * e1x + sphi * e2x);
  const double ny = mu * k[1] + sm * (cphi * e1y + sphi * e2y);
  const double nz = mu * k[2] + sm * (cphi * e1z + sphi * e2z);
  const double norm = sqrt(nx * nx + ny * ny + nz * nz);
  k[0] = nx / norm; k[1] = ny / norm; k[2] = nz / norm;
  return y - p * (1.0 - mu) + r * sm * cb;
}

// ---- kernel -------------------------------------------------------------------------
struct McArgs {
  const uint32_t* P;        // photon prefix per cell [n3 + 1], or null: even allocation
  uint64_t N;               // photons
  int32_t n;
  int64_t n3;
  const void* delta;        // float | double [n3]
  const double* x;          // [n3]
  const void* vel;          // float4 | double4 [n3], km/s
  const double* tab;        // Voigt nodes: H [kVoigtNodes], then H'
  double nH, sig0, a, dxdl, cpm, ufac, eps, expm_eps, x_lost, p_ion, p_2g, kpc_cell;
  uint64_t max_steps;
  uint32_t k0, k1, box;
  int32_t pending;          // lanes waiting to scatter before a warp runs the redistribution
  // mixed-arithmetic form
  const float* tabf;        // Voigt nodes in binary32: H, then H'
  float af, Kfac, Kx, ufacf, x_lostf;  // a; eps cpm / sig0 (cells of path times n_1s H); dx per cell of path
  uint32_t thr_scatter;     // scatter when a 32-bit word is below it: (1 - exp(-eps)) 2^32
  uint64_t thr_ion, thr_end;// fates from a 64-bit word: below thr_ion ionised, below thr_end two-photon
  unsigned long long* next; // photon counter
  unsigned long long* cnt;  // [8]: fates 0..3, sampler caps, steps, scatterings, non-finite photons
  lya_mc_photon* out;       // per photon, or null
};

template <class R> struct Field;
template <> struct Field<float> {
  static __device__ __forceinline__ double delta(const void* p, int64_t c) { return (double)__ldg((const float*)p + c); }
  static __device__ __forceinline__ void vel(const void* p, int64_t c, double u[3]) {
    const float4 v = __ldg((const float4*)p + c);
    u[0] = v.x; u[1] = v.y; u[2] = v.z;
  }
};
template <> struct Field<double> {
  static __device__ __forceinline__ double delta(const void* p, int64_t c) { return __ldg((const double*)p + c); }
  static __device__ __forceinline__ void vel(const void* p, int64_t c, double u[3]) {
    const double2 v = __ldg((const double2*)p + 2 * c);
    u[0] = v.x; u[1] = v.y; u[2] = __ldg((const double*)p + 4 * c + 2);
  }
};

__device__ __forceinline__ int64_t cell_of(const double p[3], int n) {
  int64_t c[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    int64_t ci = (int64_t)floor(p[d]) % n;
    c[d] = ci < 0 ? ci + n : ci;
  }
  return (c[2] * n + c[1]) * n + c[0];
}

template <class R>
__device__ __forceinline__ double upar(const McArgs& A, int64_t c, const double k[3]) {
  double u[3];
  Field<R>::vel(A.vel, c, u);
  return (u[0] * k[0] + u[1] * k[1] + u[2] * k[2]) * A.ufac;
}

// Home cell of photon k: the last c with P[c] <= k.
__device__ __forceinline__ int64_t home_of(const McArgs& A, uint64_t k, uint64_t* first) {
  if (!A.P) {  // even allocation P_c = floor(c N / n3)
    const int64_t c = (int64_t)(((k + 1) * (uint64_t)A.n3 - 1) / A.N);
    *first = (uint64_t)c * A.N / (uint64_t)A.n3;
    return c;
  }
  int64_t lo = 0, hi = A.n3 - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if ((uint64_t)A.P[mid] <= k) lo = mid; else hi = mid - 1;
  }
  *first = A.P[lo];
  return lo;
}

template <class R>
__global__ void __launch_bounds__(ST) k_scatter(McArgs A) {
  __shared__ double sH[kVoigtNodes], sD[kVoigtNodes];
  for (int i = threadIdx.x; i < kVoigtNodes; i += blockDim.x) {
    sH[i] = A.tab[i];
    sD[i] = A.tab[kVoigtNodes + i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  bool active = false, retired = false, pend = false;
  uint64_t k = 0, steps = 0, nscat = 0;
  uint32_t home = 0, j = 0;
  double pos[3] = {0.0, 0.0, 0.0}, st[3] = {0.0, 0.0, 0.0}, kd[3] = {0.0, 0.0, 1.0}, xf = 0.0;
  McRng rng;
  rng.init(0, 0, 0, 0, 0);
  unsigned long long my_steps = 0, my_scat = 0, my_caps = 0, my_bad = 0;
  unsigned long long my_fate[4] = {0, 0, 0, 0};

  auto finish = [&](int fate) {
    my_fate[fate] += 1;
    my_steps += steps;
    my_scat += nscat;
    if (A.out) {
      const double dx = pos[0] - st[0], dy = pos[1] - st[1], dz = pos[2] - st[2];
      lya_mc_photon o;
      o.home = home;
      o.j = j;
      o.fate = fate;
      o.reserved = 0;
      o.n_scat = nscat;
      o.n_steps = steps;
      o.D_kpc = sqrt(dx * dx + dy * dy + dz * dz) * A.kpc_cell;
      o.x_end = xf;
      A.out[k] = o;
    }
    active = false;
  };

  for (;;) {
    // lanes without a photon take the next ones (one atomic per warp)
    const unsigned need = __ballot_sync(kFull, !active && !retired);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(A.next, (unsigned long long)__popc(need));
      base = __shfl_sync(kFull, base, leader);
      if (need & (1u << lane)) {
        k = base + (unsigned long long)__popc(need & ((1u << lane) - 1u));
        if (k < A.N) {
          uint64_t p0;
          const int64_t h = home_of(A, k, &p0);
          home = (uint32_t)h;
          j = (uint32_t)(k - p0);
          rng.init(home, j, A.k0, A.k1, A.box);
          const int n = A.n;
          const int ix = (int)(h % n), iy = (int)((h / n) % n), iz = (int)(h / ((int64_t)n * n));
          pos[0] = ix + rng.next();
          pos[1] = iy + rng.next();
          pos[2] = iz + rng.next();
          st[0] = pos[0]; st[1] = pos[1]; st[2] = pos[2];
          // isotropic direction (Marsaglia 1972)
          double v1, v2, r2;
          disk(rng, v1, v2, r2);
          const double q = 2.0 * sqrt(1.0 - r2);
          kd[0] = v1 * q; kd[1] = v2 * q; kd[2] = 1.0 - 2.0 * r2;
          xf = upar<R>(A, h, kd);  // line centre in the gas frame of the emitting cell
          steps = 0;
          nscat = 0;
          pend = false;
          active = true;
        } else {
          retired = true;
        }
      }
    }
    if (__ballot_sync(kFull, active) == 0) break;

    if (active && !pend) {
      const int64_t c = cell_of(pos, A.n);
      const double y = xf - upar<R>(A, c, kd);
      if (y < -A.x_lost) {
        finish(LYA_MC_LOST);
      } else {
        const double n1s = A.nH * Field<R>::delta(A.delta, c) * (1.0 - __ldg(A.x + c));
        const double l = 1.0 / (A.sig0 * voigt_eval(sH, sD, y, A.a) * n1s);
        const double dl = A.eps * l;
        const double dcell = dl * A.cpm;
        pos[0] += kd[0] * dcell;
        pos[1] += kd[1] * dcell;
        pos[2] += kd[2] * dcell;
        xf -= dl * A.dxdl;
        ++steps;
        if (!(dl < 1e300) || !(fabs(xf) < 1e300)) {  // non-finite state: end the photon, count it
          ++my_bad;
          finish(LYA_MC_CAPPED);
        } else if (rng.next() > A.expm_eps) {
          pend = true;
        } else if (steps >= A.max_steps) {
          finish(LYA_MC_CAPPED);
        }
      }
    }

    const unsigned waiting = __ballot_sync(kFull, pend);
    const unsigned stepping = __ballot_sync(kFull, active && !pend);
    if (waiting && (__popc(waiting) >= A.pending || stepping == 0)) {
      if (pend) {
        pend = false;
        ++nscat;
        const double uf = rng.next();
        if (uf < A.p_ion) {
          finish(LYA_MC_IONISED);
        } else if (uf < A.p_ion + A.p_2g) {
          finish(LYA_MC_TWO_PHOTON);
        } else {
          const int64_t c = cell_of(pos, A.n);
          const double y = xf - upar<R>(A, c, kd);
          const double yo = redistribute(rng, y, A.a, kd, &my_caps);
          xf = yo + upar<R>(A, c, kd);
          if (steps >= A.max_steps) finish(LYA_MC_CAPPED);
        }
      }
    }
  }
#pragma unroll
  for (int f = 0; f < 4; ++f)
    if (my_fate[f]) atomicAdd(A.cnt + f, my_fate[f]);
  if (my_caps) atomicAdd(A.cnt + 4, my_caps);
  if (my_steps) atomicAdd(A.cnt + 5, my_steps);
  if (my_scat) atomicAdd(A.cnt + 6, my_scat);
  if (my_bad) atomicAdd(A.cnt + 7, my_bad);
}

// ---- mixed-arithmetic form ------------------------------------------------------------
// The same steps in binary32, with two exceptions.  The position inside the
// current cell and the frequency are double-float pairs (hi + lo, Knuth's
// error-free sum), because a step in the line core moves a photon by ~1e-10
// cells and ~1e-10 Doppler widths.  The scattering and fate decisions compare
// 32- and 64-bit words with integer thresholds, exact to 2^-32 and 2^-64
// (p_ion is ~1e-7 at z ~ 1100).  The cell's n_1s and peculiar velocity are
// cached in registers until the photon changes cell.  Statistically equivalent
// to the binary64 form; not operation-for-operation equal to it.
__device__ __forceinline__ void df_add(float& hi, float& lo, float b) {
  const float s = hi + b;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (b - bb);
  const float t = e + lo;
  hi = s + t;
  lo = t - (hi - s);
}

// The mixed form's helpers below are host and device code: the host build
// runs the same redistribution (lya_mc_redistribution_host) for CPU checks.
__host__ __device__ __forceinline__ void philox_hd(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                   uint32_t k1, uint32_t out[4]) {
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

struct McRngF {
  uint32_t cell, j, blk, tag, k0, k1, w0, w1, w2, w3;
  int nw;
  __host__ __device__ __forceinline__ void init(uint32_t c, uint32_t jj, uint32_t key0, uint32_t key1, uint32_t box) {
    cell = c; j = jj; blk = 0; tag = 0x80000000u | box; k0 = key0; k1 = key1; nw = 0;
    w0 = w1 = w2 = w3 = 0;
  }
  __host__ __device__ __forceinline__ uint32_t word() {
    if (nw == 0) {
      uint32_t r[4];
      philox_hd(cell, j, blk, tag, k0, k1, r);
      ++blk;
      w0 = r[0]; w1 = r[1]; w2 = r[2]; w3 = r[3];
      nw = 4;
    }
    const uint32_t v = w0;
    w0 = w1; w1 = w2; w2 = w3;
    --nw;
    return v;
  }
  // (w >> 8) | 1 has at most 24 bits: the conversion to binary32 is exact
  __host__ __device__ __forceinline__ float u01() { return (float)((word() >> 8) | 1u) * 0x1p-24f; }
};

__host__ __device__ __forceinline__ void disk_f(McRngF& s, float& v1, float& v2, float& r2) {
  for (int it = 0; it < 64; ++it) {
    v1 = 2.0f * s.u01() - 1.0f;
    v2 = 2.0f * s.u01() - 1.0f;
    r2 = v1 * v1 + v2 * v2;
    if (r2 < 1.0f) return;
  }
  v1 = 0.3f; v2 = 0.4f; r2 = 0.25f;
}

// H(a, t) in binary32: cubic Hermite on the nodes for t < 10; beyond, the
// first-order-in-a wing series (a / sqrt(pi)) sum_k (2k+1)!! / (2^k t^(2k+2)),
// five terms (relative error below 1e-7 for t >= 10).
__host__ __device__ __forceinline__ float voigt_f(const float* H, const float* dH, float y, float a) {
  const float t = fabsf(y);
  if (!(t < 10.0f)) {
    const float q = 1.0f / (t * t);
    return a * 0.5641895835f * q * (1.0f + q * (1.5f + q * (3.75f + q * (13.125f + q * 59.0625f))));
  }
  const float qq = t * 128.0f;
  int k = (int)qq;
  if (k > kVoigtNodes - 2) k = kVoigtNodes - 2;
  const float s = qq - (float)k;
  const float s1 = 1.0f - s;
  const float h00 = (1.0f + 2.0f * s) * s1 * s1, h10 = s * s1 * s1;
  const float h01 = s * s * (3.0f - 2.0f * s), h11 = s * s * (s - 1.0f);
  const float st = (float)kVoigtStep;
  return h00 * H[k] + h10 * st * dH[k] + h01 * H[k + 1] + h11 * st * dH[k + 1];
}

__host__ __device__ __forceinline__ float cut_u0_f(float t, float a) {
  if (t < 1.2f) return -0.7f;
  if (t >= 10.0f) return sqrtf(logf(t * t / a) + 4.0f);
  if (t < 2.0f) return 1.1f + 0.875f * (t - 1.2f);
  if (t < 3.0f) return 1.8f + 0.7f * (t - 2.0f);
  if (t < 4.0f) return 2.5f + 0.45f * (t - 3.0f);
  if (t < 6.0f) return 2.95f + 0.225f * (t - 4.0f);
  return 3.4f + 0.1f * (t - 6.0f);
}

__host__ __device__ float sample_ppar_f(McRngF& s, float y, float a, unsigned long long* caps) {
  const float t = fabsf(y);
  const float u0 = cut_u0_f(t, a);
  const float d0 = t - u0;
  const float m0 = u0 > 0.0f ? u0 : 0.0f;
  const float W1 = 0.8862269255f * (1.0f + erff(u0)) / (d0 * d0 + a * a);
  const float W2 = expf(-m0 * m0) * (1.5707963268f + atanf(d0 / a)) / a;
  const float P1 = W1 / (W1 + W2);
  for (int it = 0; it < kMaxTries; ++it) {
    float p, v1, v2, r2;
    if (s.u01() < P1) {
      disk_f(s, v1, v2, r2);
      p = v1 * sqrtf(-logf(r2) / r2);
      if (p > u0) continue;
      const float d = t - p;
      if (s.u01() * (d * d + a * a) >= d0 * d0 + a * a) continue;
    } else {
      disk_f(s, v1, v2, r2);
      p = t + a * (v1 / v2);
      if (p <= u0) continue;
      if (s.u01() >= expf(m0 * m0 - p * p)) continue;
    }
    return y < 0.0f ? -p : p;
  }
  ++*caps;
  return 0.0f;
}

__host__ __device__ float redistribute_f(McRngF& s, float y, float a, float k[3], unsigned long long* caps,
                                         float* p_out = nullptr) {
  const float p = sample_ppar_f(s, y, a, caps);
  if (p_out) *p_out = p;
  const float r = sqrtf(-logf(s.u01()));
  const float mu = 2.0f * s.u01() - 1.0f;
  float v1, v2, r2;
  disk_f(s, v1, v2, r2);
  const float cb = (v1 * v1 - v2 * v2) / r2;
  disk_f(s, v1, v2, r2);
  const float cphi = (v1 * v1 - v2 * v2) / r2, sphi = 2.0f * v1 * v2 / r2;
  const float sm = sqrtf(fmaxf(1.0f - mu * mu, 0.0f));
  const float sg = copysignf(1.0f, k[2]);
  const float aa = -1.0f / (sg + k[2]);
  const float bb = k[0] * k[1] * aa;
  const float e1x = 1.0f + sg * k[0] * k[0] * aa, e1y = sg * bb, e1z = -sg * k[0];
  const float e2x = bb, e2y = sg + k[1] * k[1] * aa, e2z = -k[1];
  const float nx = mu * k[0] + sm * (cphi * e1x + sphi * e2x);
  const float ny = mu * k[1] + sm * (cphi * e1y + sphi * e2y);
  const float nz = mu * k[2] + sm * (cphi * e1z + sphi * e2z);
#ifdef __CUDA_ARCH__
  const float inv = rsqrtf(nx * nx + ny * ny + nz * nz);
#else
  const float inv = 1.0f / sqrtf(nx * nx + ny * ny + nz * nz);
#endif
  k[0] = nx * inv; k[1] = ny * inv; k[2] = nz * inv;
  return y - p * (1.0f - mu) + r * sm * cb;
}

template <class R>
__global__ void __launch_bounds__(ST) k_scatter_mixed(McArgs A) {
  __shared__ float sH[kVoigtNodes], sD[kVoigtNodes];
  for (int i = threadIdx.x; i < kVoigtNodes; i += blockDim.x) {
    sH[i] = A.tabf[i];
    sD[i] = A.tabf[kVoigtNodes + i];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int n = A.n;
  bool active = false, retired = false, pend = false;
  uint64_t k = 0, steps = 0, nscat = 0;
  uint32_t home = 0, j = 0;
  int ic[3] = {0, 0, 0}, is[3] = {0, 0, 0};
  float fh[3] = {0.f, 0.f, 0.f}, fl[3] = {0.f, 0.f, 0.f}, sf[3] = {0.f, 0.f, 0.f};
  float kd[3] = {0.f, 0.f, 1.f}, U[3] = {0.f, 0.f, 0.f};
  float xh = 0.f, xl = 0.f, up = 0.f, Kc = 0.f;
  McRngF rng;
  rng.init(0, 0, 0, 0, 0);
  unsigned long long my_steps = 0, my_scat = 0, my_caps = 0, my_bad = 0;
  unsigned long long f_lost = 0, f_2g = 0, f_ion = 0, f_cap = 0;

  // cached quantities of the cell the photon is in
  auto load_cell = [&]() {
    int w[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      int q = ic[d] % n;
      w[d] = q < 0 ? q + n : q;
    }
    const int64_t c = ((int64_t)w[2] * n + w[1]) * n + w[0];
    const double n1s = A.nH * Field<R>::delta(A.delta, c) * (1.0 - __ldg(A.x + c));
    Kc = (float)(A.Kfac / n1s);
    double u[3];
    Field<R>::vel(A.vel, c, u);
    U[0] = (float)u[0]; U[1] = (float)u[1]; U[2] = (float)u[2];
  };
  auto upar = [&]() { return (U[0] * kd[0] + U[1] * kd[1] + U[2] * kd[2]) * A.ufacf; };

  auto finish = [&](int fate) {
    if (fate == LYA_MC_LOST) ++f_lost;
    else if (fate == LYA_MC_TWO_PHOTON) ++f_2g;
    else if (fate == LYA_MC_IONISED) ++f_ion;
    else ++f_cap;
    my_steps += steps;
    my_scat += nscat;
    if (A.out) {
      double dd = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const double e = (double)(ic[d] - is[d]) + (((double)fh[d] + (double)fl[d]) - (double)sf[d]);
        dd += e * e;
      }
      lya_mc_photon o;
      o.home = home;
      o.j = j;
      o.fate = fate;
      o.reserved = 0;
      o.n_scat = nscat;
      o.n_steps = steps;
      o.D_kpc = sqrt(dd) * A.kpc_cell;
      o.x_end = (double)xh + (double)xl;
      A.out[k] = o;
    }
    active = false;
  };

  for (;;) {
    const unsigned need = __ballot_sync(kFull, !active && !retired);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(A.next, (unsigned long long)__popc(need));
      base = __shfl_sync(kFull, base, leader);
      if (need & (1u << lane)) {
        k = base + (unsigned long long)__popc(need & ((1u << lane) - 1u));
        if (k < A.N) {
          uint64_t p0;
          const int64_t h = home_of(A, k, &p0);
          home = (uint32_t)h;
          j = (uint32_t)(k - p0);
          rng.init(home, j, A.k0, A.k1, A.box);
          ic[0] = (int)(h % n); ic[1] = (int)((h / n) % n); ic[2] = (int)(h / ((int64_t)n * n));
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            is[d] = ic[d];
            fh[d] = rng.u01();
            fl[d] = 0.0f;
            sf[d] = fh[d];
          }
          float v1, v2, r2;
          disk_f(rng, v1, v2, r2);
          const float q = 2.0f * sqrtf(1.0f - r2);
          kd[0] = v1 * q; kd[1] = v2 * q; kd[2] = 1.0f - 2.0f * r2;
          load_cell();
          up = upar();
          xh = up;  // line centre in the gas frame of the emitting cell
          xl = 0.0f;
          steps = 0;
          nscat = 0;
          pend = false;
          active = true;
        } else {
          retired = true;
        }
      }
    }
    if (__ballot_sync(kFull, active) == 0) break;

    if (active && !pend) {
      const float y = (xh - up) + xl;
      if (y < -A.x_lostf) {
        finish(LYA_MC_LOST);
      } else {
        const float dcell = __fdividef(Kc, voigt_f(sH, sD, y, A.af));
#pragma unroll
        for (int d = 0; d < 3; ++d) df_add(fh[d], fl[d], kd[d] * dcell);
        df_add(xh, xl, -(A.Kx * dcell));
        ++steps;
        if (!(dcell < 1e30f) || !(fabsf(xh) < 1e30f)) {
          ++my_bad;
          finish(LYA_MC_CAPPED);
        } else {
          if (fh[0] < 0.0f || fh[0] >= 1.0f || fh[1] < 0.0f || fh[1] >= 1.0f || fh[2] < 0.0f || fh[2] >= 1.0f) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              const float m = floorf(fh[d]);
              if (m != 0.0f) {
                ic[d] += (int)m;
                fh[d] -= m;
                const float s2 = fh[d] + fl[d];  // renormalise the pair
                fl[d] = fl[d] - (s2 - fh[d]);
                fh[d] = s2;
              }
            }
            load_cell();
            up = upar();
          }
          if (rng.word() < A.thr_scatter) pend = true;
          else if (steps >= A.max_steps) finish(LYA_MC_CAPPED);
        }
      }
    }

    const unsigned waiting = __ballot_sync(kFull, pend);
    const unsigned stepping = __ballot_sync(kFull, active && !pend);
    if (waiting && (__popc(waiting) >= A.pending || stepping == 0)) {
      if (pend) {
        pend = false;
        ++nscat;
        const uint64_t hi = rng.word();
        const uint64_t uf = (hi << 32) | rng.word();
        if (uf < A.thr_ion) {
          finish(LYA_MC_IONISED);
        } else if (uf < A.thr_end) {
          finish(LYA_MC_TWO_PHOTON);
        } else {
          const float y = (xh - up) + xl;
          const float yo = redistribute_f(rng, y, A.af, kd, &my_caps);
          up = upar();
          const float s2 = yo + up;  // x = y_out + u_par as a double-float pair
          const float bb = s2 - yo;
          xl = (yo - (s2 - bb)) + (up - bb);
          xh = s2;
          if (steps >= A.max_steps) finish(LYA_MC_CAPPED);
        }
      }
    }
  }
  if (f_lost) atomicAdd(A.cnt + 0, f_lost);
  if (f_2g) atomicAdd(A.cnt + 1, f_2g);
  if (f_ion) atomicAdd(A.cnt + 2, f_ion);
  if (f_cap) atomicAdd(A.cnt + 3, f_cap);
  if (my_caps) atomicAdd(A.cnt + 4, my_caps);
  if (my_steps) atomicAdd(A.cnt + 5, my_steps);
  if (my_scat) atomicAdd(A.cnt + 6, my_scat);
  if (my_bad) atomicAdd(A.cnt + 7, my_bad);
}

__global__ void k_scatter_stats(const unsigned long long* cnt, lya_mc_stats* st) {
  if (threadIdx.x != 0 || !st) return;
  for (int f = 0; f < 4; ++f) st->count[f] = cnt[f];
  st->sampler_caps = cnt[4];
  st->steps = cnt[5];
  st->scatterings = cnt[6];
  st->nonfinite = cnt[7];
}

// ---- mixing fraction f_alpha(D) of Sec. III.B from the photon records ----------------
// Destroyed photons (two-photon decay or photo-ionisation) are the ones whose
// Ly-alpha energy leaves the line; f_alpha(D) is the share of them destroyed
// farther than D from where they were emitted.  Counts are integers
// (order-independent), so the fractions do not depend on the launch.
struct MfArgs {
  const lya_mc_photon* rec;
  uint64_t n;
  int32_t m;
  unsigned long long* cnt;  // [4 + m]: photons per fate, then destroyed photons with D > D_j
  double D[kMixFracMax];
};

__global__ void __launch_bounds__(ST) k_mix_fraction(MfArgs a) {
  __shared__ unsigned int s[4 + kMixFracMax];
  for (int i = threadIdx.x; i < 4 + a.m; i += ST) s[i] = 0u;
  __syncthreads();
  for (uint64_t k = (uint64_t)blockIdx.x * ST + threadIdx.x; k < a.n; k += (uint64_t)gridDim.x * ST) {
    const unsigned f = (unsigned)a.rec[k].fate;
    if (f < 4u) atomicAdd(&s[f], 1u);
    if (f == (unsigned)LYA_MC_TWO_PHOTON || f == (unsigned)LYA_MC_IONISED) {
      const double D = a.rec[k].D_kpc;
      for (int j = 0; j < a.m; ++j)
        if (D > a.D[j]) atomicAdd(&s[4 + j], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 4 + a.m; i += ST)
    if (s[i]) atomicAdd(a.cnt + i, (unsigned long long)s[i]);
}

// out[j] = B_j / N_d; out[m + j] = B_j / (N_d + N_c); out[2m + j] = (B_j + N_c) / (N_d + N_c),
// with B_j the destroyed photons beyond D_j, N_d the destroyed and N_c the capped ones.
__global__ void k_mix_fraction_final(const unsigned long long* cnt, int m, double* out, uint64_t* counts) {
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const double Nd = (double)(cnt[LYA_MC_TWO_PHOTON] + cnt[LYA_MC_IONISED]);
  const double Nc = (double)cnt[LYA_MC_CAPPED];
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double B = (double)cnt[4 + j];
    out[j] = Nd > 0.0 ? B / Nd : nan;
    out[m + j] = Nd + Nc > 0.0 ? B / (Nd + Nc) : nan;
    out[2 * m + j] = Nd + Nc > 0.0 ? (B + Nc) / (Nd + Nc) : nan;
  }
  if (counts && threadIdx.x < 4) counts[threadIdx.x] = cnt[threadIdx.x];
}

}  // namespace

// Scalars of one Monte-Carlo snapshot at redshift mp->z.  Branching of an
// n = 2 atom with 2s and 2p in statistical equilibrium (n_2p = 3 n_2s,
// Sec. III.A.1; rates per 2s atom): photo-ionisation beta_e, two-photon decay
// Lambda, Ly-alpha emission 3 A.  Eq. MC: <sigma> = sigma_0 4 a sqrt(pi) H(a, y),
// sigma_0 = 3 lambda_alpha^2 / (8 pi), a = A lambda_alpha / (4 pi c v_th).
bool scatter_setup(const Cosmo& c, const rec_params& p, int n, const lya_mc_params* mp, McSetup* S) {
  const double c_light = 2.99792458e8, k_boltz = 1.380649e-23;
  const double m_hyd = 1.00782503223 * 1.66053906660e-27;
  const double lambda_lya = 6.62607015e-34 * c_light / (0.75 * 13.598434 * 1.602176634e-19);
  const StepCoef k = step_coef(c, p, mp->z, mp->z, 1);
  S->Tg = k.Tg;
  S->nH = k.nH;
  S->Heff = mp->zeta * k.H;
  S->beta = k.beta;
  S->Lam = mp->lambda2g >= 0.0 ? mp->lambda2g : k.L2g;
  const double A = mp->A_alpha;
  const double tot = S->beta + S->Lam + 3.0 * A;
  S->p_ion = S->beta / tot;
  S->p_2g = S->Lam / tot;
  S->vth = std::sqrt(2.0 * k_boltz * S->Tg / m_hyd) / c_light;
  S->a = A * lambda_lya / (4.0 * kPiD * c_light * S->vth);
  S->sig0 = 3.0 * lambda_lya * lambda_lya / (8.0 * kPiD) * 4.0 * S->a * kSqrtPiD;
  S->dxdl = S->Heff / (c_light * S->vth);
  const double cell_m = c.L_m / n;
  S->cpm = (1.0 + mp->z) / cell_m;
  S->ufac = 1.0e3 / (c_light * S->vth);
  S->expm_eps = std::exp(-mp->eps);
  S->kpc_cell = p.L_box_kpc / n;
  return std::isfinite(S->a) && S->a > 0.0 && std::isfinite(S->sig0) && S->Heff > 0.0 && S->nH > 0.0;
}

// The mixed form's redistribution (Eq. inout) run on the host: m independent
// scatterings at gas-frame offset y along kin (streams (i, i >> 32) of seed).
// Returns the number of atom-velocity draws that hit the rejection cap.
uint64_t scatter_redistribution_mixed_host(double a, double y, const double* kin, uint64_t seed, int64_t m,
                                           double* ppar, double* dy, double* kout) {
  unsigned long long caps = 0;
  const double kn = std::sqrt(kin[0] * kin[0] + kin[1] * kin[1] + kin[2] * kin[2]);
  for (int64_t i = 0; i < m; ++i) {
    McRngF s;
    s.init((uint32_t)i, (uint32_t)(i >> 32), (uint32_t)seed, (uint32_t)(seed >> 32), 0);
    float k[3] = {(float)(kin[0] / kn), (float)(kin[1] / kn), (float)(kin[2] / kn)};
    float p = 0.0f;
    const float yo = redistribute_f(s, (float)y, (float)a, k, &caps, &p);
    if (ppar) ppar[i] = p;
    if (dy) dy[i] = (double)yo - (double)(float)y;
    if (kout) for (int d = 0; d < 3; ++d) kout[3 * i + d] = k[d];
  }
  return caps;
}

// The mixed form's binary32 Voigt evaluation (nodes rounded to binary32, the
// wing series beyond |y| = 10) on the host.
void scatter_voigt_mixed_host(double a, int64_t m, const double* y, double* H) {
  static thread_local double last_a = -1.0;
  static thread_local float tH[kVoigtNodes], tD[kVoigtNodes];
  if (a != last_a) {
    std::vector<double> h(2 * kVoigtNodes);
    voigt_nodes(a, h.data(), h.data() + kVoigtNodes);
    for (int i = 0; i < kVoigtNodes; ++i) { tH[i] = (float)h[i]; tD[i] = (float)h[kVoigtNodes + i]; }
    last_a = a;
  }
  for (int64_t i = 0; i < m; ++i) H[i] = voigt_f(tH, tD, (float)y[i], (float)a);
}

void scatter_voigt_host(double a, int64_t m, const double* y, double* H) {
  static thread_local double last_a = -1.0;
  static thread_local double tH[kVoigtNodes], tD[kVoigtNodes];
  if (a != last_a) {
    voigt_nodes(a, tH, tD);
    last_a = a;
  }
  for (int64_t i = 0; i < m; ++i) H[i] = voigt_eval(tH, tD, y[i], a);
}

cudaError_t run_scatter_mc(rec_ctx* c, const McSetup& S, const lya_mc_params* mp, const uint32_t* prefix,
                           lya_mc_photon* out, lya_mc_stats* st) {
  // Voigt nodes (binary64 and binary32) and counters in one scratch
  // allocation owned by the context
  const size_t tab_bytes = sizeof(double) * 2 * kVoigtNodes;
  const size_t tabf_bytes = sizeof(float) * 2 * kVoigtNodes;
  const size_t cnt_off = tab_bytes + ((tabf_bytes + 255) / 256) * 256;
  const size_t need = cnt_off + sizeof(unsigned long long) * 9;
  if (c->mc_bytes < need) {
    if (c->mc_scratch) cudaFree(c->mc_scratch);
    c->mc_scratch = nullptr;
    c->mc_bytes = 0;
    cudaError_t e = cudaMalloc(&c->mc_scratch, need);
    if (e != cudaSuccess) return e;
    c->mc_bytes = need;
  }
  double* tab = (double*)c->mc_scratch;
  float* tabf = (float*)((char*)c->mc_scratch + tab_bytes);
  unsigned long long* cnt = (unsigned long long*)((char*)c->mc_scratch + cnt_off);
  if (S.a != c->mc_a) {
    std::vector<double> h(2 * kVoigtNodes);
    voigt_nodes(S.a, h.data(), h.data() + kVoigtNodes);
    std::vector<float> hf(2 * kVoigtNodes);
    for (int i = 0; i < 2 * kVoigtNodes; ++i) hf[i] = (float)h[i];
    cudaError_t e = cudaMemcpyAsync(tab, h.data(), tab_bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(tabf, hf.data(), tabf_bytes, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(c->stream);  // the host buffer goes out of scope
    if (e != cudaSuccess) return e;
    c->mc_a = S.a;
  }
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 9, c->stream);
  if (e != cudaSuccess) return e;
  McArgs A;
  A.P = prefix;
  A.N = mp->n_photons;
  A.n = c->box.n;
  A.n3 = c->n3;
  A.delta = c->box.delta;
  A.x = c->box.x_e;
  A.vel = c->box.vel4;
  A.tab = tab;
  A.nH = S.nH;
  A.sig0 = S.sig0;
  A.a = S.a;
  A.dxdl = S.dxdl;
  A.cpm = S.cpm;
  A.ufac = S.ufac;
  A.eps = mp->eps;
  A.expm_eps = S.expm_eps;
  A.x_lost = mp->x_lost;
  A.p_ion = S.p_ion;
  A.p_2g = S.p_2g;
  A.kpc_cell = S.kpc_cell;
  A.max_steps = mp->max_steps;
  A.k0 = (uint32_t)c->params.seed;
  A.k1 = (uint32_t)(c->params.seed >> 32) ^ (uint32_t)mp->step;
  A.box = 0;
  A.pending = mp->pending > 0 ? mp->pending : 12;
  A.tabf = tabf;
  A.af = (float)S.a;
  A.Kfac = (float)(mp->eps * S.cpm / S.sig0);
  A.Kx = (float)(S.dxdl / S.cpm);
  A.ufacf = (float)S.ufac;
  A.x_lostf = (float)mp->x_lost;
  {
    const double ps = -std::expm1(-mp->eps);  // 1 - exp(-eps)
    const double t32 = std::floor(std::ldexp(ps, 32) + 0.5);
    A.thr_scatter = t32 >= 4294967295.0 ? 0xffffffffu : (uint32_t)t32;
    const double ti = std::ldexp(S.p_ion, 64), te = std::ldexp(S.p_ion + S.p_2g, 64);
    A.thr_ion = ti >= 18446744073709549568.0 ? ~0ull : (uint64_t)ti;
    A.thr_end = te >= 18446744073709549568.0 ? ~0ull : (uint64_t)te;
  }
  A.next = cnt + 8;
  A.cnt = cnt;
  A.out = out;
  // one persistent pass: blocks per SM limited by the kernel's resources
  int per_sm = 0;
  const bool fmix = c->params.precision == REC_PREC_MIXED, amix = mp->arith == LYA_MC_MIXED;
  if (amix)
    e = fmix ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter_mixed<float>, ST, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter_mixed<double>, ST, 0);
  else
    e = fmix ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter<float>, ST, 0)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter<double>, ST, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint64_t warps_needed = (mp->n_photons + 31) / 32;
  uint64_t blocks = (uint64_t)c->sm_count * per_sm;
  const uint64_t max_useful = (warps_needed + (ST / 32) - 1) / (ST / 32);
  if (blocks > max_useful) blocks = max_useful;
  if (blocks < 1) blocks = 1;
  {
    GroupTimer t(c, kTOther, 2);
    if (amix) {
      if (fmix) k_scatter_mixed<float><<<(unsigned)blocks, ST, 0, c->stream>>>(A);
      else k_scatter_mixed<double><<<(unsigned)blocks, ST, 0, c->stream>>>(A);
    } else {
      if (fmix) k_scatter<float><<<(unsigned)blocks, ST, 0, c->stream>>>(A);
      else k_scatter<double><<<(unsigned)blocks, ST, 0, c->stream>>>(A);
    }
    k_scatter_stats<<<1, 32, 0, c->stream>>>(cnt, st);
  }
  return cudaGetLastError();
}

cudaError_t run_mixing_fraction(rec_ctx* c, const lya_mc_photon* rec, uint64_t n, const double* D, int m,
                                double* out, uint64_t* counts) {
  if (!c->mf_cnt) {
    cudaError_t e = cudaMalloc(&c->mf_cnt, sizeof(unsigned long long) * (4 + kMixFracMax));
    if (e != cudaSuccess) { c->mf_cnt = nullptr; return e; }
  }
  cudaError_t e = cudaMemsetAsync(c->mf_cnt, 0, sizeof(unsigned long long) * (4 + m), c->stream);
  if (e != cudaSuccess) return e;
  MfArgs a;
  a.rec = rec;
  a.n = n;
  a.m = m;
  a.cnt = (unsigned long long*)c->mf_cnt;
  for (int j = 0; j < kMixFracMax; ++j) a.D[j] = j < m ? D[j] : 0.0;
  uint64_t blocks = (n + ST - 1) / ST;
  const uint64_t cap = (uint64_t)c->sm_count * 4;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  GroupTimer t(c, kTOther, 2);
  k_mix_fraction<<<(unsigned)blocks, ST, 0, c->stream>>>(a);
  k_mix_fraction_final<<<1, ST, 0, c->stream>>>(a.cnt, m, out, counts);
  return cudaGetLastError();
}

}  // namespace rec
