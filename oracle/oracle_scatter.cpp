// Oracle: the resonant-scattering Ly-alpha Monte Carlo of Appendix A of
// arXiv:2312.11448.  TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// A photon is injected at line centre in the gas frame at a random point of
// its emitting cell (step (1)).  Each step evaluates the thermally averaged
// cross-section (Eq. MC) and the mean free path l = 1 / (sigma n_1s) (step
// (2)), moves the photon by eps l (step (3)), redshifts it by
// dx = -H dl / v_th (step (4)) and scatters it with probability 1 - exp(-eps)
// (steps (5)-(6)).  A scattering ends the photon by photo-ionisation of the
// n = 2 atom or by two-photon decay, or re-emits it (step (7)); a re-emitted
// photon takes the frequency of Eq. inout from the scattering atom's velocity
// and the new direction (step (8)).  Photons that drift far enough onto the
// red wing are lost by redshifting.
//
// Plain FP64 with the C library's exp, log, erf, atan and sqrt.

#include "oracle.h"

#include <cmath>
#include <complex>
#include <vector>

namespace {

using cplx = std::complex<double>;

const double kPi = 3.14159265358979323846;
const double kSqrtPi = 1.77245385090551602730;
const double kC = 2.99792458e8;            // m/s
const double kHplanck = 6.62607015e-34;    // J s
const double kKB = 1.380649e-23;           // J/K
const double kAmu = 1.66053906660e-27;     // kg
const double kMH = 1.00782503223 * kAmu;   // hydrogen atom mass
const double kEalpha = 0.75 * 13.598434 * 1.602176634e-19;  // 10.2 eV (Sec. III.A.1)
const double kLambdaAlpha = kHplanck * kC / kEalpha;         // 121.57 nm
const double kMpcM = 3.0856775814913673e22;

// ---- Faddeeva function w(z), Im z > 0 ----------------------------------------
// The thermally averaged cross-section of Eq. MC is proportional to the Voigt
// function H(a, y) = Re w(y + i a), with a = Gamma_alpha / (2 omega_alpha v_th).
//
// |z| < 10: Weideman's rational expansion (J. A. C. Weideman, SIAM J. Numer.
// Anal. 31, 1497 (1994)) with N = 48 terms:
//   w(z) = 2 sum_{n=1}^{N} a_n Z^{n-1} / (L - i z)^2 + 1 / (sqrt(pi) (L - i z)),
//   Z = (L + i z) / (L - i z),  L = sqrt(N / sqrt 2),
// where a_n are the Fourier coefficients of F(theta) = exp(-t^2) (L^2 + t^2),
// t = L tan(theta / 2), taken at the 2M = 4N points theta_k = k pi / M:
//   a_n = [F_0 + 2 sum_{k=1}^{M-1} F_k cos(pi k n / M)] / (2 M).
// |z| >= 10: the asymptotic series w(z) ~ (i / sqrt pi) sum_k (2k-1)!! / (2^k z^{2k+1}).
struct Weideman {
  static const int N = 48;
  double L;
  double a[N + 1];
  Weideman() {
    const int M = 2 * N;
    L = std::sqrt(N / std::sqrt(2.0));
    std::vector<double> F(M);
    for (int k = 0; k < M; ++k) {
      double t = L * std::tan(0.5 * k * kPi / M);
      F[k] = std::exp(-t * t) * (L * L + t * t);
    }
    for (int n = 1; n <= N; ++n) {
      double s = F[0];
      for (int k = 1; k < M; ++k) s += 2.0 * F[k] * std::cos(kPi * k * n / M);
      a[n] = s / (2.0 * M);
    }
  }
  cplx eval(cplx z) const {
    const cplx I(0.0, 1.0);
    cplx den = L - I * z;
    cplx Z = (L + I * z) / den;
    cplx p = a[N];
    for (int n = N - 1; n >= 1; --n) p = p * Z + a[n];
    return 2.0 * p / (den * den) + 1.0 / (kSqrtPi * den);
  }
};

const Weideman& weideman() {
  static const Weideman w;
  return w;
}

cplx faddeeva_asym(cplx z) {
  cplx z2 = z * z;
  cplx term = 1.0 / z, sum = term;
  for (int k = 1; k < 12; ++k) {
    term *= (2.0 * k - 1.0) / (2.0 * z2);
    sum += term;
  }
  return cplx(0.0, 1.0 / kSqrtPi) * sum;
}

cplx faddeeva(double y, double a) {
  cplx z(y, a);
  if (std::abs(z) >= 10.0) return faddeeva_asym(z);
  return weideman().eval(z);
}

// ---- Voigt profile table -------------------------------------------------------
// H(a, y) for |y| < 10 from a cubic Hermite interpolant on nodes y_k = k/128
// (values and slopes H' = -2 (y H - a K), K = Im w, from the Faddeeva function
// above; interpolation error below 2e-8 relative for 1e-4 <= a <= 1e-2), and
// the asymptotic series beyond.
struct VoigtTable {
  static constexpr double kH = 1.0 / 128.0;
  static constexpr double kYmax = 10.0;
  static const int kNodes = 1281;
  double a;
  std::vector<double> H, dH;
  explicit VoigtTable(double a_) : a(a_), H(kNodes), dH(kNodes) {
    for (int k = 0; k < kNodes; ++k) {
      double y = k * kH;
      cplx w = faddeeva(y, a);
      H[k] = w.real();
      dH[k] = -2.0 * (y * w.real() - a * w.imag());
    }
  }
  double operator()(double y) const {
    double t = std::fabs(y);
    if (t >= kYmax) return faddeeva_asym(cplx(t, a)).real();
    double q = t / kH;
    int k = (int)q;
    double s = q - k;
    double s1 = 1.0 - s;
    double h00 = (1.0 + 2.0 * s) * s1 * s1, h10 = s * s1 * s1;
    double h01 = s * s * (3.0 - 2.0 * s), h11 = s * s * (s - 1.0);
    return h00 * H[k] + h10 * kH * dH[k] + h01 * H[k + 1] + h11 * kH * dH[k + 1];
  }
};

// ---- random stream ----------------------------------------------------------------
// One photon's deviates: Philox4x32-10 blocks with key (seed low word, seed
// high word XOR step) and counter (cell, photon index in the cell, block,
// 2^31 | box); each block gives two binary64 deviates (2 floor(w / 2^12) + 1) 2^-53
// from the 64-bit words (word1:word0) and (word3:word2), used in order.
struct Stream {
  uint32_t key[2], ctr[4], buf[4];
  int next_word;
  Stream(uint64_t seed, uint32_t step, uint32_t cell, uint32_t j, uint32_t box) {
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32) ^ step;
    ctr[0] = cell; ctr[1] = j; ctr[2] = 0; ctr[3] = 0x80000000u | box;
    next_word = 4;
  }
  double next() {
    if (next_word == 4) {
      orc_philox4x32_10(ctr, key, buf);
      ctr[2] += 1;
      next_word = 0;
    }
    uint64_t w = ((uint64_t)buf[next_word + 1] << 32) | buf[next_word];
    next_word += 2;
    return (double)((w >> 11) | 1u) * 0x1p-53;
  }
};

// A point uniform in the unit disk by rejection from the square (at most 64
// tries; the fallback point is never reached in practice).
void disk(Stream& s, double& v1, double& v2, double& r2) {
  for (int it = 0; it < 64; ++it) {
    v1 = 2.0 * s.next() - 1.0;
    v2 = 2.0 * s.next() - 1.0;
    r2 = v1 * v1 + v2 * v2;
    if (r2 < 1.0) return;
  }
  v1 = 0.3; v2 = 0.4; r2 = 0.25;
}

// Isotropic unit vector (Marsaglia 1972): from a disk point with r2 = s,
// n = (2 v1 sqrt(1-s), 2 v2 sqrt(1-s), 1 - 2 s).
void isotropic(Stream& s, double k[3]) {
  double v1, v2, r2;
  disk(s, v1, v2, r2);
  double q = 2.0 * std::sqrt(1.0 - r2);
  k[0] = v1 * q; k[1] = v2 * q; k[2] = 1.0 - 2.0 * r2;
}

// Normal deviate of variance 1/2 (density exp(-p^2)/sqrt(pi)), the Maxwellian
// component of the scaled atomic momentum in Eq. MC: polar method, one
// component per disk point.
double gauss_half(Stream& s) {
  double v1, v2, r2;
  disk(s, v1, v2, r2);
  return v1 * std::sqrt(-std::log(r2) / r2);
}

// Standard Cauchy deviate: ratio of the coordinates of a disk point (neither
// coordinate is ever zero: 2u - 1 is an odd multiple of 2^-52).
double cauchy(Stream& s) {
  double v1, v2, r2;
  disk(s, v1, v2, r2);
  return v1 / v2;
}

// ---- scattering atom's parallel velocity ---------------------------------------
// Density of the scaled parallel momentum p of the atom that scatters a
// photon at gas-frame frequency y (third factor of Eq. MC):
//   f(p) ~ exp(-p^2) / ((y - p)^2 + a^2).
// Exact rejection sampling for t = |y| (the result takes the sign of y) with
// a cut u0 < t and the envelope
//   p <= u0:  exp(-p^2) / ((t - u0)^2 + a^2)           (normal proposal),
//   p >  u0:  exp(-max(u0,0)^2) / ((t - p)^2 + a^2)    (Lorentzian proposal),
// of masses W1 = (sqrt(pi)/2)(1 + erf u0) / ((t-u0)^2 + a^2) and
// W2 = exp(-max(u0,0)^2) (pi/2 + atan((t-u0)/a)) / a.  Any u0 < t gives the
// exact density; the cut only sets the acceptance rate.
double cut_u0(double t, double a) {
  if (t < 1.2) return -0.7;
  if (t >= 10.0) return std::sqrt(std::log(t * t / a) + 4.0);
  static const double kt[6] = {1.2, 2.0, 3.0, 4.0, 6.0, 10.0};
  static const double ku[6] = {1.1, 1.8, 2.5, 2.95, 3.4, 3.8};
  int i = 0;
  while (t >= kt[i + 1]) ++i;
  return ku[i] + (ku[i + 1] - ku[i]) * (t - kt[i]) / (kt[i + 1] - kt[i]);
}

const int kMaxTries = 100000;

double sample_ppar(Stream& s, double y, double a, uint64_t* sampler_caps) {
  const double t = std::fabs(y);
  const double u0 = cut_u0(t, a);
  const double d0 = t - u0;
  const double m0 = u0 > 0.0 ? u0 : 0.0;
  const double W1 = 0.5 * kSqrtPi * (1.0 + std::erf(u0)) / (d0 * d0 + a * a);
  const double W2 = std::exp(-m0 * m0) * (0.5 * kPi + std::atan(d0 / a)) / a;
  const double P1 = W1 / (W1 + W2);
  for (int it = 0; it < kMaxTries; ++it) {
    double p;
    if (s.next() < P1) {
      p = gauss_half(s);
      if (p > u0) continue;
      double d = t - p;
      if (s.next() * (d * d + a * a) >= d0 * d0 + a * a) continue;
    } else {
      p = t + a * cauchy(s);
      if (p <= u0) continue;
      if (s.next() >= std::exp(m0 * m0 - p * p)) continue;
    }
    return y < 0.0 ? -p : p;
  }
  if (sampler_caps) ++*sampler_caps;
  return 0.0;
}

// ---- one scattering: Eq. inout --------------------------------------------------
// Isotropic scattering: mu = k_in . k_out uniform in [-1, 1], beta uniform.
// p_perp = sqrt(p1^2 + p2^2) of the two perpendicular momentum components of
// Eq. MC, drawn as sqrt(-ln u) (p1, p2 normal of variance 1/2).  The
// outgoing direction is mu k_in + sqrt(1-mu^2) (cos phi e1 + sin phi e2) in
// an orthonormal basis (e1, e2) of the plane normal to k_in (Duff et al.,
// JCGT 6(1), 2017); phi = beta + angle of p_perp is uniform and independent
// of beta.  Returns y_out = y - p_par (1 - mu) + p_perp sqrt(1 - mu^2) cos beta.
double scatter(Stream& s, double y, double a, double k[3], uint64_t* sampler_caps, double* ppar_out) {
  const double p = sample_ppar(s, y, a, sampler_caps);
  const double r = std::sqrt(-std::log(s.next()));
  const double mu = 2.0 * s.next() - 1.0;
  double v1, v2, r2;
  disk(s, v1, v2, r2);
  const double cb = (v1 * v1 - v2 * v2) / r2;
  disk(s, v1, v2, r2);
  const double cphi = (v1 * v1 - v2 * v2) / r2, sphi = 2.0 * v1 * v2 / r2;
  const double sm = std::sqrt(1.0 - mu * mu);
  const double sg = std::copysign(1.0, k[2]);
  const double aa = -1.0 / (sg + k[2]);
  const double bb = k[0] * k[1] * aa;
  const double e1[3] = {1.0 + sg * k[0] * k[0] * aa, sg * bb, -sg * k[0]};
  const double e2[3] = {bb, sg + k[1] * k[1] * aa, -k[1]};
  double kn[3];
  for (int d = 0; d < 3; ++d) kn[d] = mu * k[d] + sm * (cphi * e1[d] + sphi * e2[d]);
  const double norm = std::sqrt(kn[0] * kn[0] + kn[1] * kn[1] + kn[2] * kn[2]);
  for (int d = 0; d < 3; ++d) k[d] = kn[d] / norm;
  if (ppar_out) *ppar_out = p;
  return y - p * (1.0 - mu) + r * sm * cb;
}

// ---- scalars of one Monte-Carlo snapshot ---------------------------------------
struct McSetup {
  double a, vth, sig0, dxdl, com_per_m, p_ion, p_2g, beta, Lam, Heff, nH, Tg, expm_eps;
};

int mc_setup(const orc_cosmo* cp, const orc_mc_params* mp, int n, McSetup* S) {
  if (!cp || !mp || mp->eps <= 0.0 || !(mp->zeta > 0.0) || n <= 0) return -1;
  double bg[5], rt[6];
  if (orc_background(cp, mp->z, bg) != 0) return -1;
  const double Tg = bg[2];
  if (orc_rates(cp, mp->z, Tg, rt) != 0) return -1;
  S->Tg = Tg;
  S->nH = bg[1];
  S->Heff = mp->zeta * bg[0];
  S->beta = rt[1];
  S->Lam = mp->lambda2g >= 0.0 ? mp->lambda2g : rt[3];
  const double A = mp->A_alpha;
  // Branching of an n = 2 atom whose 2s and 2p sublevels are in statistical
  // equilibrium (n_2p = 3 n_2s, Sec. III.A.1; rates per 2s atom):
  // photo-ionisation beta_e, two-photon decay Lambda, Ly-alpha emission 3 A.
  const double tot = S->beta + S->Lam + 3.0 * A;
  S->p_ion = S->beta / tot;
  S->p_2g = S->Lam / tot;
  // v_th = sqrt(2 k T / m_H) in units of c; a = Gamma / (2 omega_alpha v_th).
  S->vth = std::sqrt(2.0 * kKB * Tg / kMH) / kC;
  S->a = A * kLambdaAlpha / (4.0 * kPi * kC * S->vth);
  // Eq. MC: <sigma> = sigma_0 (4 a sqrt(pi)) H(a, y), sigma_0 = 3 lambda^2 / (8 pi).
  S->sig0 = 3.0 * kLambdaAlpha * kLambdaAlpha / (8.0 * kPi) * 4.0 * S->a * kSqrtPi;
  // Step (4): dx = -H dl / v_th with dl the physical path (c = 1).
  S->dxdl = S->Heff / (kC * S->vth);
  // Physical metres to comoving cells.
  const double cell_m = cp->L_box_kpc * kMpcM * 1.0e-3 / n;
  S->com_per_m = (1.0 + mp->z) / cell_m;
  S->expm_eps = std::exp(-mp->eps);
  return 0;
}

}  // namespace

extern "C" {

int orc_faddeeva(double y, double a, double* w) {
  if (!w || !(a > 0.0)) return -1;
  cplx v = faddeeva(y, a);
  w[0] = v.real();
  w[1] = v.imag();
  return 0;
}

int orc_voigt_table(double a, int64_t m, const double* y, double* H) {
  if (!(a > 0.0) || m < 0 || !y || !H) return -1;
  VoigtTable tab(a);
  for (int64_t i = 0; i < m; ++i) H[i] = tab(y[i]);
  return 0;
}

int orc_mc_setup(const orc_cosmo* cp, const orc_mc_params* mp, int n, double* out) {
  McSetup S;
  if (!out || mc_setup(cp, mp, n, &S) != 0) return -1;
  out[0] = S.a; out[1] = S.vth; out[2] = S.sig0; out[3] = S.dxdl; out[4] = S.p_ion;
  out[5] = S.p_2g; out[6] = S.beta; out[7] = S.Lam; out[8] = S.Heff; out[9] = S.nH;
  out[10] = S.Tg; out[11] = S.com_per_m;
  return 0;
}

int orc_mc_redistribution(double a, double y, const double* kin, uint64_t seed, int64_t m, double* ppar,
                          double* dy, double* kout) {
  if (!(a > 0.0) || m < 0 || !kin) return -1;
  const double kn = std::sqrt(kin[0] * kin[0] + kin[1] * kin[1] + kin[2] * kin[2]);
  if (!(kn > 0.0)) return -1;
  uint64_t caps = 0;
  for (int64_t i = 0; i < m; ++i) {
    Stream s(seed, 0, (uint32_t)i, (uint32_t)(i >> 32), 0);
    double k[3] = {kin[0] / kn, kin[1] / kn, kin[2] / kn};
    double p = 0.0;
    double yo = scatter(s, y, a, k, &caps, &p);
    if (ppar) ppar[i] = p;
    if (dy) dy[i] = yo - y;
    if (kout) for (int d = 0; d < 3; ++d) kout[3 * i + d] = k[d];
  }
  return caps == 0 ? 0 : -2;
}

int orc_lya_mc(const orc_cosmo* cp, const orc_mc_params* mp, int n, const double* delta, const double* xe,
               const double* U, const uint32_t* P, uint64_t k0, uint64_t k1, orc_mc_photon* out,
               uint64_t* counters) {
  McSetup S;
  if (!delta || !xe || !P || !out || mc_setup(cp, mp, n, &S) != 0) return -1;
  const int64_t n3 = (int64_t)n * n * n;
  const uint64_t total = P[n3];
  if (k0 > k1 || k1 > total) return -1;
  std::vector<double> n1s(n3);
  for (int64_t c = 0; c < n3; ++c) {
    n1s[c] = S.nH * delta[c] * (1.0 - xe[c]);
    if (!(n1s[c] > 0.0)) return -1;
  }
  const VoigtTable voigt(S.a);
  // Peculiar velocity in Doppler units: u = U[km/s] * 1e3 / (c v_th).
  const double ufac = 1.0e3 / (kC * S.vth);
  const double kpc_per_cell = cp->L_box_kpc / n;
  uint64_t caps = 0;
  long long nphot = (long long)(k1 - k0);
#ifdef ORACLE_OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : caps)
#endif
  for (long long q = 0; q < nphot; ++q) {
    const uint64_t k = k0 + (uint64_t)q;
    // Emitting cell: the last c with P[c] <= k.
    int64_t lo = 0, hi = n3 - 1;
    while (lo < hi) {
      int64_t mid = (lo + hi + 1) / 2;
      if (P[mid] <= k) lo = mid; else hi = mid - 1;
    }
    const uint32_t home = (uint32_t)lo;
    const uint32_t j = (uint32_t)(k - P[lo]);
    Stream s(mp->seed, mp->step, home, j, mp->box);
    const int ix = (int)(home % n), iy = (int)((home / n) % n), iz = (int)(home / ((int64_t)n * n));
    double pos[3];
    pos[0] = ix + s.next();
    pos[1] = iy + s.next();
    pos[2] = iz + s.next();
    const double start[3] = {pos[0], pos[1], pos[2]};
    double kdir[3];
    isotropic(s, kdir);
    auto cell_of = [&](const double* p) {
      int64_t c3[3];
      for (int d = 0; d < 3; ++d) {
        int64_t ci = (int64_t)std::floor(p[d]) % n;
        c3[d] = ci < 0 ? ci + n : ci;
      }
      return (c3[2] * n + c3[1]) * n + c3[0];
    };
    auto upar = [&](int64_t c, const double* kk) {
      if (!U) return 0.0;
      const double* u = U + 3 * c;
      return (u[0] * kk[0] + u[1] * kk[1] + u[2] * kk[2]) * ufac;
    };
    // Step (1): line centre in the gas frame of the emitting cell; x is kept
    // in the frame without peculiar velocity, y = x - u_par in the gas frame.
    double x = upar(home, kdir);
    uint64_t steps = 0, nscat = 0;
    int fate = ORC_MC_CAPPED;
    while (steps < mp->max_steps) {
      int64_t c = cell_of(pos);
      double y = x - upar(c, kdir);
      if (y < -mp->x_lost) { fate = ORC_MC_LOST; break; }
      // (2) mean free path; (3) advance eps l; (4) redshift.
      double l = 1.0 / (S.sig0 * voigt(y) * n1s[c]);
      double dl = mp->eps * l;
      double dcell = dl * S.com_per_m;
      for (int d = 0; d < 3; ++d) pos[d] += kdir[d] * dcell;
      x -= dl * S.dxdl;
      ++steps;
      // (5)-(6) scatter with probability 1 - exp(-eps).
      if (s.next() <= S.expm_eps) continue;
      ++nscat;
      // (7) fate of the excited atom.
      double uf = s.next();
      if (uf < S.p_ion) { fate = ORC_MC_IONISED; break; }
      if (uf < S.p_ion + S.p_2g) { fate = ORC_MC_TWO_PHOTON; break; }
      // (8) re-emission at the scattering point (Eq. inout).
      c = cell_of(pos);
      y = x - upar(c, kdir);
      double yo = scatter(s, y, S.a, kdir, &caps, nullptr);
      x = yo + upar(c, kdir);
    }
    double dd = 0.0;
    for (int d = 0; d < 3; ++d) dd += (pos[d] - start[d]) * (pos[d] - start[d]);
    orc_mc_photon& o = out[q];
    o.home = home;
    o.j = j;
    o.fate = fate;
    o.n_scat = nscat;
    o.n_steps = steps;
    o.D_kpc = std::sqrt(dd) * kpc_per_cell;
    o.x_end = x;
  }
  if (counters) {
    for (int f = 0; f < 4; ++f) counters[f] = 0;
    counters[4] = caps;
    for (long long q = 0; q < nphot; ++q) counters[out[q].fate] += 1;
  }
  return 0;
}

}  // extern "C"
