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

__global__ void k_scatter_stats(const unsigned long long* cnt, lya_mc_stats* st) {
  if (threadIdx.x != 0 || !st) return;
  for (int f = 0; f < 4; ++f) st->count[f] = cnt[f];
  st->sampler_caps = cnt[4];
  st->steps = cnt[5];
  st->scatterings = cnt[6];
  st->nonfinite = cnt[7];
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
  // Voigt nodes and counters in one scratch allocation owned by the context
  const size_t tab_bytes = sizeof(double) * 2 * kVoigtNodes;
  const size_t need = tab_bytes + sizeof(unsigned long long) * 9;
  if (c->mc_bytes < need) {
    if (c->mc_scratch) cudaFree(c->mc_scratch);
    c->mc_scratch = nullptr;
    c->mc_bytes = 0;
    cudaError_t e = cudaMalloc(&c->mc_scratch, need);
    if (e != cudaSuccess) return e;
    c->mc_bytes = need;
  }
  double* tab = (double*)c->mc_scratch;
  unsigned long long* cnt = (unsigned long long*)((char*)c->mc_scratch + tab_bytes);
  if (S.a != c->mc_a) {
    std::vector<double> h(2 * kVoigtNodes);
    voigt_nodes(S.a, h.data(), h.data() + kVoigtNodes);
    cudaError_t e = cudaMemcpyAsync(tab, h.data(), tab_bytes, cudaMemcpyHostToDevice, c->stream);
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
  A.next = cnt + 8;
  A.cnt = cnt;
  A.out = out;
  // one persistent pass: blocks per SM limited by the kernel's resources
  int per_sm = 0;
  if (c->params.precision == REC_PREC_MIXED)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter<float>, ST, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter<double>, ST, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const uint64_t warps_needed = (mp->n_photons + 31) / 32;
  uint64_t blocks = (uint64_t)c->sm_count * per_sm;
  const uint64_t max_useful = (warps_needed + (ST / 32) - 1) / (ST / 32);
  if (blocks > max_useful) blocks = max_useful;
  if (blocks < 1) blocks = 1;
  {
    GroupTimer t(c, kTOther, 2);
    if (c->params.precision == REC_PREC_MIXED)
      k_scatter<float><<<(unsigned)blocks, ST, 0, c->stream>>>(A);
    else
      k_scatter<double><<<(unsigned)blocks, ST, 0, c->stream>>>(A);
    k_scatter_stats<<<1, 32, 0, c->stream>>>(cnt, st);
  }
  return cudaGetLastError();
}

}  // namespace rec
