// Oracle: background cosmology, three-level-atom rates, Saha initial state, the
// per-cell recombination step with full/tally Ly-alpha mixing, and trajectory
// objectives with a forward-mode tangent.  TEST INFRASTRUCTURE ONLY (see
// oracle.h).  Plain single-threaded FP64; the step code is a template so that
// the same lines run on double and on dual numbers for the tangent.
//
// Paper references are to Jedamzik, Abel & Ali-Haimoud, arXiv:2312.11448.

#include "oracle.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

// ---- physical constants, SI (CODATA 2018) ---------------------------------
const double kC = 2.99792458e8;            // speed of light [m/s]
const double kHplanck = 6.62607015e-34;    // Planck constant [J s]
const double kKB = 1.380649e-23;           // Boltzmann constant [J/K]
const double kMe = 9.1093837015e-31;       // electron mass [kg]
const double kSigmaT = 6.6524587321e-29;   // Thomson cross-section [m^2]
const double kSigmaSB = 5.670374419e-8;    // Stefan-Boltzmann [W/m^2/K^4]
const double kG = 6.67430e-11;             // Newton constant
const double kAmu = 1.66053906660e-27;     // atomic mass unit [kg]
const double kMH = 1.00782503223 * kAmu;   // hydrogen atom mass [kg]
const double kMHe = 4.00260325413 * kAmu;  // helium-4 atom mass [kg]
const double kEV = 1.602176634e-19;        // electron volt [J]
const double kMpc = 3.0856775814913673e22; // megaparsec [m]
const double kPi = 3.14159265358979323846;

// Radiation constant a_R = 4 sigma_SB / c.
const double kARad = 4.0 * kSigmaSB / kC;
// Hydrogen ground-state ionisation energy, 13.598434 eV (NIST; includes the
// relativistic and QED shifts of 1s that the reduced-mass Rydberg omits).
const double kEion = 13.598434 * 1.602176634e-19;
// Ly-alpha (1s-2p) energy: 3/4 of the ionisation energy (10.2 eV, Sec. III.A.1);
// the 2s binding energy is the remaining 1/4, so E_2s + E_alpha = E_ion.
const double kEalpha = 0.75 * kEion;
const double kE2s = 0.25 * kEion;
const double kLambdaAlpha = kHplanck * kC / kEalpha;  // 121.57 nm
// Two-photon 2s->1s decay rate, 8.22 /s (Sec. III.A.1).
const double kLambda2g = 8.22;
// Pequignot, Petitjean & Boisson (1991) case-B fit, cited in Sec. III.A.1:
// A_B = 1e-19 m^3/s * a t^b / (1 + c t^d), t = T / 1e4 K.
const double kPPB_a = 4.309, kPPB_b = -0.6166, kPPB_c = 0.6703, kPPB_d = 0.5300;

struct Cosmo {
  double H0, Om, Or, OL, nH0, T0, fHe, Yp, L_m, fudge, heat;
};

Cosmo make_cosmo(const orc_cosmo* p) {
  Cosmo c;
  c.H0 = p->h * 1.0e5 / kMpc;  // 100 h km/s/Mpc in 1/s
  double rho_crit = 3.0 * c.H0 * c.H0 / (8.0 * kPi * kG);
  double Ob = p->omega_b_h2 / (p->h * p->h);
  double Oc = p->omega_c_h2 / (p->h * p->h);
  c.Om = Ob + Oc;
  double T0 = p->T_cmb0;
  double Og = kARad * T0 * T0 * T0 * T0 / (kC * kC) / rho_crit;
  double Onu = p->N_eff * (7.0 / 8.0) * std::pow(4.0 / 11.0, 4.0 / 3.0) * Og;
  c.Or = Og + Onu;
  c.OL = 1.0 - c.Om - c.Or;
  c.nH0 = (1.0 - p->Y_p) * Ob * rho_crit / kMH;  // hydrogen nuclei per m^3 today
  c.T0 = T0;
  c.Yp = p->Y_p;
  c.fHe = p->Y_p * kMH / ((1.0 - p->Y_p) * kMHe);  // n_He / n_H, about 0.08 (Sec. II.A)
  c.L_m = p->L_box_kpc * kMpc * 1.0e-3;
  c.fudge = p->fudge;
  c.heat = p->heating;
  return c;
}

double hubble(const Cosmo& c, double z) {
  double a1 = 1.0 + z;
  return c.H0 * std::sqrt(c.Om * a1 * a1 * a1 + c.Or * a1 * a1 * a1 * a1 + c.OL);
}
double nH_bar(const Cosmo& c, double z) { double a1 = 1.0 + z; return c.nH0 * a1 * a1 * a1; }
double T_gamma(const Cosmo& c, double z) { return c.T0 * (1.0 + z); }

// Cosmic time between z_from and z_to: integral of d ln(1+z) / H, Simpson's
// rule in y = ln(1+z) on the (short) step interval.
double cosmic_dt(const Cosmo& c, double z_from, double z_to) {
  double ya = std::log1p(z_from), yb = std::log1p(z_to);
  double ym = 0.5 * (ya + yb);
  double zm = std::expm1(ym);
  return (ya - yb) / 6.0 * (1.0 / hubble(c, z_to) + 4.0 / hubble(c, zm) + 1.0 / hubble(c, z_from));
}

// ---- dual numbers for the forward-mode tangent ------------------------------
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
inline Dual pow(Dual a, double p) { double q = std::pow(a.v, p); return Dual(q, p * q / a.v * a.d); }
inline double val(Dual a) { return a.v; }
inline double val(double a) { return a; }
using std::exp;
using std::pow;
using std::sqrt;

// Case-B recombination coefficient times the fudge factor (Sec. III.A.1):
// alpha_e(T_b) = 1.14 A_B(T_b).
template <class R>
R alpha_e(const Cosmo& c, R T) {
  R t = T / 1.0e4;
  return c.fudge * 1.0e-19 * kPPB_a * pow(t, kPPB_b) / (1.0 + kPPB_c * pow(t, kPPB_d));
}

// (2 pi m_e k T / h^2)^{3/2}, the free-electron phase-space density factor.
double saha_phase(double T) {
  return std::pow(2.0 * kPi * kMe * kKB * T / (kHplanck * kHplanck), 1.5);
}

// Photo-ionisation rate per 2s atom by detailed balance with the CMB
// (Sec. III.A.1 and its footnote: rates are written per 2s atom):
// beta_e = alpha_e(T_gamma) (2 pi m_e k T_gamma/h^2)^{3/2} exp(-E_2s/k T_gamma).
double beta_e(const Cosmo& c, double Tg) {
  return alpha_e<double>(c, Tg) * saha_phase(Tg) * std::exp(-kE2s / (kKB * Tg));
}

// Physical divergence of the peculiar velocity per cell, 1/s: central
// differences of U (km/s, [n^3][3]) over the periodic grid, comoving cell side
// h = L / n, and 1/a = 1 + z from comoving to physical gradients.
void local_divergence(int n, const double* U, double L_m, double z, double* div) {
  const int64_t n3 = (int64_t)n * n * n;
  const double h = L_m / (double)n;  // m, comoving
  const double fac = (1.0 + z) * 1.0e3 / (2.0 * h);
  for (int64_t c = 0; c < n3; ++c) {
    const int ix = (int)(c % n), iy = (int)((c / n) % n), iz = (int)(c / ((int64_t)n * n));
    auto at = [&](int x, int y, int zz) {
      x = (x + n) % n; y = (y + n) % n; zz = (zz + n) % n;
      return ((int64_t)zz * n + y) * n + x;
    };
    const double dux = U[3 * at(ix + 1, iy, iz) + 0] - U[3 * at(ix - 1, iy, iz) + 0];
    const double duy = U[3 * at(ix, iy + 1, iz) + 1] - U[3 * at(ix, iy - 1, iz) + 1];
    const double duz = U[3 * at(ix, iy, iz + 1) + 2] - U[3 * at(ix, iy, iz - 1) + 2];
    div[c] = fac * (dux + duy + duz);
  }
}

// ---- one substep of the recombination update --------------------------------
template <class R>
struct SubStats {
  R lambda, C, Xe, S1s;
  int iters;
  double dt;
};

// Backward-Euler root for one cell.  The cell obeys
//   dx/dt = -alpha n_H x^2 + w G (1 - x),
// which is Eq. (dotne-mix) written per hydrogen atom with the 2s population
// n_2s = w n_1s <n_2s>/<n_1s> and beta <n_2s>/<n_1s> = G (Eq. n2s-sol on
// averages).  With A = dt alpha n_H and s = dt w the implicit update solves
// A x'^2 + (1 + sG) x' - (x + sG) = 0; this is its positive root, written
// without cancellation.  dxdG = d x'/d G.
template <class R>
R be_root(R A, R s, R G, R x_old, R* dxdG) {
  R B = 1.0 + s * G;
  R c = x_old + s * G;
  R D = B * B + 4.0 * A * c;
  R xr = 2.0 * c / (B + sqrt(D));
  if (dxdG) *dxdG = s * (1.0 - xr) / (2.0 * A * xr + B);
  return xr;
}

// One substep z_a -> z_b.  All coefficients are taken at the substep end z_b
// (backward Euler); the Peebles factor uses the substep-start <n_1s>.
//   delta: overdensity rho_b/<rho_b> (Sec. II.C), static.
//   afrac: absorbed-Ly-alpha fraction per cell (TALLY mode) or null.
template <class R>
void substep(const Cosmo& cm, int n, int64_t n3, int mixing, double fmix, double za, double zb, const R* delta, R* x,
             R* T, double* U, const R* afrac, R* emis, SubStats<R>* st) {
  if (mixing == 3 && !(fmix > 0.0)) mixing = 2;  // no full-mixing share: the local mode
  const double H = hubble(cm, zb);
  const double nH = nH_bar(cm, zb);
  const double Tg = T_gamma(cm, zb);
  const double dt = cosmic_dt(cm, za, zb);
  const double Tg4 = Tg * Tg * Tg * Tg;
  // Compton heating coefficient of Eq. (Tb-evolution): 8 sigma_T a_R T^4 / (3 m_e c),
  // times x n_H / n_tot per cell.
  const double kc = 8.0 * kSigmaT * kARad * Tg4 / (3.0 * kMe * kC);
  // Compton drag rate of Eq. (alpha-def): (4/3) n_e sigma_T rho_gamma / rho_b with
  // n_e / rho_b = x (1 - Y_p) / m_H; the density cancels.
  const double kd = 4.0 * kSigmaT * kARad * Tg4 * (1.0 - cm.Yp) / (3.0 * kC * kMH);
  // Heating term 2 Gamma / (3 n_tot k) with Gamma uniform; per cell it is
  // hq / (Delta (1 + f_He + x)).
  const double hq = 2.0 * cm.heat * kEV / (3.0 * kKB);
  const double beta = beta_e(cm, Tg);
  const double ea = std::exp(-kEalpha / (kKB * Tg));
  // R_alpha = 8 pi H / (lambda_alpha^3 n_1s), Eq. (R-alpha); with full mixing
  // R_alpha^mix uses <n_1s> (Sec. IV.A.2).
  const double KR = 8.0 * kPi * H / (kLambdaAlpha * kLambdaAlpha * kLambdaAlpha);

  R S = 0.0;
  for (int64_t i = 0; i < n3; ++i) S += delta[i] * (1.0 - x[i]);
  R n1s_mean = nH * S / (double)n3;
  R Rmix = KR / n1s_mean;
  // Peebles factor with R_alpha -> R_alpha^mix, Eq. (Cfactor).
  R C = (kLambda2g + Rmix) / (beta + kLambda2g + Rmix);

  std::vector<R> Tn(n3), al(n3), nn(n3), A(n3), s(n3);
  for (int64_t i = 0; i < n3; ++i) {
    R xi = x[i], d = delta[i];
    R g = kc * xi / (1.0 + cm.fHe + xi);
    R hh = hq / (d * (1.0 + cm.fHe + xi));
    // Eq. (Tb-evolution), backward Euler; the adiabatic term of a static comoving
    // field is -2 H T_b.
    Tn[i] = (T[i] + dt * (g * Tg + hh)) / (1.0 + dt * (2.0 * H + g));
    al[i] = alpha_e<R>(cm, Tn[i]);
    nn[i] = nH * d;
    A[i] = dt * al[i] * nn[i];
    R w = 1.0;
    if (mixing == 0 && afrac != nullptr) {
      // J_i / <J>: absorptions per neutral atom, normalised so that the
      // n_1s-weighted mean is one.
      R n1s_rel = d * (1.0 - xi);
      if (val(S) > 0.0 && val(n1s_rel) > 0.0) w = afrac[i] * S / n1s_rel;
    }
    s[i] = dt * w;
  }

  // Local Peebles factor of cell i (modes 2 and 3): R_alpha of Eq. (R-alpha) with
  // the cell's substep-start n_1s and H + div v / 3, zero below zero.
  std::vector<double> div;
  if (mixing == 2 || mixing == 3) {
    div.assign(n3, 0.0);
    if (U != nullptr) local_divergence(n, U, cm.L_m, zb, div.data());
  }
  const double KR0 = 8.0 * kPi / (kLambdaAlpha * kLambdaAlpha * kLambdaAlpha);
  auto local_C = [&](int64_t i) -> R {
    const double Heff = std::max(H + div[i] / 3.0, 0.0);
    const R n1s = nn[i] * (1.0 - x[i]);
    if (!(val(n1s) > 0.0)) return R(1.0);
    R Ri = KR0 * Heff / n1s;
    return (kLambda2g + Ri) / (beta + kLambda2g + Ri);
  };
  // Partial mixing (mode 3, fraction f of the full-mixing rate): the net rate is
  //   f [-alpha n_H x^2 + G (1 - x)] + (1 - f) C_i [-alpha n_H x^2 + beta e_alpha (1 - x)],
  // the same quadratic with A_i scaled by f + (1 - f) C_i, s = dt f and G offset
  // per cell by g_i = (1 - f)/f C_i beta e_alpha; lambda stays self-consistent.
  std::vector<R> gofs(n3, R(0.0));
  if (mixing == 3) {
    for (int64_t i = 0; i < n3; ++i) {
      const R Ci = local_C(i);
      A[i] = A[i] * (fmix + (1.0 - fmix) * Ci);
      s[i] = R(dt * fmix);
      gofs[i] = ((1.0 - fmix) / fmix) * Ci * (beta * ea);
    }
  }

  if (mixing == 2) {
    // No-mixing limit (Sec. III.A.2): recombination is local, Eq. (rec) with the
    // cell's own n_e and n_1s, and R_alpha of Eq. (R-alpha) with H -> H + div v / 3
    // (div v of the substep-start velocities).  Reading where the paper asks for
    // care: a flow converging faster than the expansion (H + div v/3 < 0) lets no
    // Ly-alpha photon escape, R_alpha = 0.  C per cell uses the substep-start n_1s
    // (as R_alpha^mix does with <n_1s>); no global lambda.
    R sx = 0.0, sd = 0.0, sC = 0.0, num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n3; ++i) {
      const R Ci = local_C(i);
      // dx/dt = -C (alpha n_H x^2 - beta e_alpha (1 - x)), backward Euler
      R xr = be_root<R>(dt * Ci * al[i] * nn[i], dt * Ci, R(beta * ea), x[i], nullptr);
      if (U != nullptr) {
        double damp = std::exp(-(kd * val(xr) + H) * dt);
        U[3 * i + 0] *= damp; U[3 * i + 1] *= damp; U[3 * i + 2] *= damp;
      }
      x[i] = xr;
      T[i] = Tn[i];
      if (emis) emis[i] = al[i] * (nn[i] * xr) * (nn[i] * xr);
      sx += delta[i] * xr;
      sd += delta[i];
      sC += Ci;
      num += al[i] * nn[i] * nn[i] * xr * xr;
      den += nn[i] * (1.0 - xr);
    }
    st->lambda = num / den;
    st->C = sC / (double)n3;  // volume mean of the local Peebles factors
    st->Xe = sx / sd;
    st->S1s = S;
    st->iters = 0;
    st->dt = dt;
    return;
  }

  const R CBe = C * beta * ea;
  const R omC = 1.0 - C;
  // lambda = <alpha n_e^2>/<n_1s> at the end state; start from the old x.
  R num = 0.0, den = 0.0;
  for (int64_t i = 0; i < n3; ++i) {
    num += al[i] * nn[i] * nn[i] * x[i] * x[i];
    den += nn[i] * (1.0 - x[i]);
  }
  R lam = num / den;
  int it = 0, extra = -1;
  for (it = 1; it <= 200; ++it) {
    R G = omC * lam + CBe;
    R F = 0.0, Fp = 0.0;
    for (int64_t i = 0; i < n3; ++i) {
      R dxdG;
      R xr = be_root<R>(A[i], s[i], G + gofs[i], x[i], &dxdG);
      R an2 = al[i] * nn[i] * nn[i];
      F += an2 * xr * xr - lam * nn[i] * (1.0 - xr);
      Fp += (2.0 * an2 * xr + lam * nn[i]) * dxdG * omC - nn[i] * (1.0 - xr);
    }
    R step = F / Fp;
    R lnew = lam - step;
    if (!(val(Fp) < 0.0) || !(val(lnew) > 0.0)) {
      // Safeguard for a start far from the root: F decreases with lambda, so
      // move by a factor two towards its zero.
      lnew = lam * (val(F) > 0.0 ? 2.0 : 0.5);
    }
    // Converged when the Newton step is below 1e-12 lambda (F is evaluated to
    // about 1e-13 relative); after many iterations accept the rounding floor.
    double as = std::fabs(val(step)), al0 = std::fabs(val(lam));
    bool conv = as <= 1e-12 * al0 || (it > 40 && as <= 1e-10 * al0);
    lam = lnew;
    if (extra < 0 && conv) extra = 2;  // two more passes settle the tangent part
    if (extra >= 0 && extra-- == 0) break;
  }

  R G = omC * lam + CBe;
  R sx = 0.0, sd = 0.0;
  for (int64_t i = 0; i < n3; ++i) {
    R xr = be_root<R>(A[i], s[i], G + gofs[i], x[i], nullptr);
    if (U != nullptr) {
      // Compton drag plus Hubble damping of peculiar velocity, Eq. (momentum):
      // d(a v)/dt = -alpha a v  =>  v' = v exp(-(alpha + H) dt), alpha at x'.
      double damp = std::exp(-(kd * val(xr) + H) * dt);
      U[3 * i + 0] *= damp; U[3 * i + 1] *= damp; U[3 * i + 2] *= damp;
    }
    x[i] = xr;
    T[i] = Tn[i];
    if (emis) emis[i] = al[i] * (nn[i] * xr) * (nn[i] * xr);
    sx += delta[i] * xr;
    sd += delta[i];
  }
  st->lambda = lam;
  st->C = C;
  st->Xe = sx / sd;  // X_e = <rho_b x_e>/<rho_b> (Sec. II.A)
  st->S1s = S;
  st->iters = it;
  st->dt = dt;
}

// ---- second-order substep: TR-BDF2 ------------------------------------------
// The same per-cell system as the backward-Euler substep (Eq. dotne-mix per
// hydrogen atom, dx/dt = -alpha(T) n_H x^2 + w G (1 - x) with
// G = (1 - C) lambda + C beta e_alpha, lambda = <alpha n_e^2>/<n_1s> and C the
// Peebles factor of Eq. Cfactor with R_alpha^mix from <n_1s>; Eq. Tb-evolution
// for T) advanced by TR-BDF2 (Bank et al., IEEE Trans. CAD 4, 436 (1985)):
// a trapezoidal stage to t + gamma h, gamma = 2 - sqrt 2, then a BDF2 stage to
// t + h.  Every coefficient is taken at the time it belongs to, and each stage
// end is fully implicit: x, T, lambda and C all at the stage end.

// Coefficients that depend only on the redshift.
struct Coef {
  double H, nH, Tg, kc, kd, hq, beta, ea, KR;
};

Coef coef_at(const Cosmo& cm, double z) {
  Coef k;
  k.H = hubble(cm, z);
  k.nH = nH_bar(cm, z);
  k.Tg = T_gamma(cm, z);
  const double Tg4 = k.Tg * k.Tg * k.Tg * k.Tg;
  k.kc = 8.0 * kSigmaT * kARad * Tg4 / (3.0 * kMe * kC);
  k.kd = 4.0 * kSigmaT * kARad * Tg4 * (1.0 - cm.Yp) / (3.0 * kC * kMH);
  k.hq = 2.0 * cm.heat * kEV / (3.0 * kKB);
  k.beta = beta_e(cm, k.Tg);
  k.ea = std::exp(-kEalpha / (kKB * k.Tg));
  k.KR = 8.0 * kPi * k.H / (kLambdaAlpha * kLambdaAlpha * kLambdaAlpha);
  return k;
}

// Peebles factor with R_alpha^mix at the state x (Eq. Cfactor, Sec. IV.A.2).
double peebles_mix(const Coef& k, int64_t n3, const double* delta, const double* x) {
  double S = 0.0;
  for (int64_t i = 0; i < n3; ++i) S += delta[i] * (1.0 - x[i]);
  const double Rmix = k.KR / (k.nH * S / (double)n3);
  return (kLambda2g + Rmix) / (k.beta + kLambda2g + Rmix);
}

// Time derivatives of x and T at a state, with lambda and C of that state.
void rates_at(const Cosmo& cm, const Coef& k, int64_t n3, const double* delta, const double* w, const double* x,
              const double* T, double* fx, double* fT) {
  const double C = peebles_mix(k, n3, delta, x);
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < n3; ++i) {
    const double nn = k.nH * delta[i];
    num += alpha_e<double>(cm, T[i]) * nn * nn * x[i] * x[i];
    den += nn * (1.0 - x[i]);
  }
  const double lam = num / den;
  const double G = (1.0 - C) * lam + C * k.beta * k.ea;
  for (int64_t i = 0; i < n3; ++i) {
    const double nn = k.nH * delta[i];
    fx[i] = -alpha_e<double>(cm, T[i]) * nn * x[i] * x[i] + w[i] * G * (1.0 - x[i]);
    const double g = k.kc * x[i] / (1.0 + cm.fHe + x[i]);
    const double hh = k.hq / (delta[i] * (1.0 + cm.fHe + x[i]));
    fT[i] = -2.0 * k.H * T[i] + g * (k.Tg - T[i]) + hh;
  }
}

// One implicit stage: find x, T (and lambda, C) at the stage end with
//   x_i = bx_i + h fx_i(x, T),   T_i = bT_i + h fT_i(x_i, T_i).
// T is linear given x; x is the positive root of the backward-Euler quadratic
// with x_old -> bx for a given G, and lambda solves its Newton equation as in the
// backward-Euler substep.  The outer iteration repeats T, alpha(T), C(x) and the
// lambda solve until x and T no longer change.  x, T hold the initial guess and
// receive the result.
// The quadratic of cell i has a positive root while c_i = bx_i + h w_i G > 0.  A
// stiff cell can have bx_i < 0 (its explicit part overshoots), so lambda is kept
// above lambda_min = max_i (-bx_i / (h w_i) - C beta e_alpha) / (1 - C): Newton
// iterates that fall below it are pulled back halfway.  Returns the Newton
// iterations, or -1 if the converged lambda leaves a cell without a positive
// root (the step is too long for the stage).
int stage_solve(const Cosmo& cm, const Coef& k, int64_t n3, const double* delta, const double* w, double h,
                const double* bx, const double* bT, double* x, double* T, double* lam_out, double* C_out) {
  std::vector<double> Tn(n3), al(n3), nn(n3), A(n3), sv(n3), xn(n3);
  int iters = 0;
  double lam = 0.0, C = 0.0;
  for (int outer = 0; outer < 200; ++outer) {
    C = peebles_mix(k, n3, delta, x);
    for (int64_t i = 0; i < n3; ++i) {
      const double g = k.kc * x[i] / (1.0 + cm.fHe + x[i]);
      const double hh = k.hq / (delta[i] * (1.0 + cm.fHe + x[i]));
      Tn[i] = (bT[i] + h * (g * k.Tg + hh)) / (1.0 + h * (2.0 * k.H + g));
      al[i] = alpha_e<double>(cm, Tn[i]);
      nn[i] = k.nH * delta[i];
      A[i] = h * al[i] * nn[i];
      sv[i] = h * w[i];
    }
    const double CBe = C * k.beta * k.ea, omC = 1.0 - C;
    double lam_min = -1e300;
    for (int64_t i = 0; i < n3; ++i) {
      if (sv[i] > 0.0) lam_min = std::max(lam_min, (-bx[i] / sv[i] - CBe) / omC);
      else if (!(bx[i] > 0.0)) return -1;  // no photo-ionisation term and no positive root
    }
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n3; ++i) {
      num += al[i] * nn[i] * nn[i] * x[i] * x[i];
      den += nn[i] * (1.0 - x[i]);
    }
    lam = num / den;
    const double lam_lo = std::max(lam_min, 0.0);  // lambda > 0 as well (G > 0)
    if (!(lam > lam_lo)) lam = lam_lo > 0.0 ? 2.0 * lam_lo : lam;
    for (int it = 1; it <= 200; ++it) {
      ++iters;
      const double G = omC * lam + CBe;
      double F = 0.0, Fp = 0.0;
      for (int64_t i = 0; i < n3; ++i) {
        double dxdG;
        const double xr = be_root<double>(A[i], sv[i], G, bx[i], &dxdG);
        const double an2 = al[i] * nn[i] * nn[i];
        F += an2 * xr * xr - lam * nn[i] * (1.0 - xr);
        Fp += (2.0 * an2 * xr + lam * nn[i]) * dxdG * omC - nn[i] * (1.0 - xr);
      }
      const double step = F / Fp;
      double lnew = lam - step;
      if (!(Fp < 0.0) || !(lnew > 0.0)) lnew = lam * (F > 0.0 ? 2.0 : 0.5);
      if (!(lnew > lam_lo)) lnew = 0.5 * (lam + lam_lo);
      const bool conv = std::fabs(lnew - lam) <= 1e-13 * std::fabs(lam);
      lam = lnew;
      if (conv) break;
    }
    if (!(lam > lam_lo)) return -1;
    const double G = omC * lam + CBe;
    double dmax = 0.0;
    for (int64_t i = 0; i < n3; ++i) {
      xn[i] = be_root<double>(A[i], sv[i], G, bx[i], nullptr);
      dmax = std::max(dmax, std::fabs(xn[i] - x[i]) / xn[i]);
      dmax = std::max(dmax, std::fabs(Tn[i] - T[i]) / Tn[i]);
    }
    for (int64_t i = 0; i < n3; ++i) { x[i] = xn[i]; T[i] = Tn[i]; }
    if (!(dmax < 1e300)) return -1;  // not finite
    if (dmax <= 1e-14) break;
  }
  *lam_out = lam;
  *C_out = C;
  return iters;
}

// Redshift z_g in [z_b, z_a] at which the cosmic time since z_a is tau.
double z_after(const Cosmo& cm, double za, double zb, double tau) {
  double lo = zb, hi = za;  // cosmic_dt(za, z) grows as z falls
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (cosmic_dt(cm, za, mid) < tau) hi = mid; else lo = mid;
    if (hi - lo <= 1e-13 * za) break;
  }
  return 0.5 * (lo + hi);
}

// One TR-BDF2 substep z_a -> z_b.  The cosmic times use the same Simpson rule
// as the backward-Euler substep.  Drag: U' = U exp(-int (alpha_C + H) dt) with
// the trapezoidal rule for the exponent.  Returns -1 as stage_solve does.
int substep_trbdf2(const Cosmo& cm, int64_t n3, double za, double zb, const double* delta, const double* w,
                   double* x, double* T, double* U, double* emis, SubStats<double>* st) {
  const double gam = 2.0 - std::sqrt(2.0);
  const double h = cosmic_dt(cm, za, zb);
  const double zg = z_after(cm, za, zb, gam * h);
  const Coef ka = coef_at(cm, za), kg = coef_at(cm, zg), kb = coef_at(cm, zb);
  std::vector<double> fx(n3), fT(n3), bx(n3), bT(n3), xg(x, x + n3), Tg(T, T + n3);
  rates_at(cm, ka, n3, delta, w, x, T, fx.data(), fT.data());
  // trapezoidal stage to t + gamma h
  const double h1 = 0.5 * gam * h;
  for (int64_t i = 0; i < n3; ++i) { bx[i] = x[i] + h1 * fx[i]; bT[i] = T[i] + h1 * fT[i]; }
  double lam, C;
  const int it1 = stage_solve(cm, kg, n3, delta, w, h1, bx.data(), bT.data(), xg.data(), Tg.data(), &lam, &C);
  if (it1 < 0) return -1;
  // BDF2 stage to t + h
  const double h2 = (1.0 - gam) / (2.0 - gam) * h;
  const double c1 = 1.0 / (gam * (2.0 - gam)), c0 = (1.0 - gam) * (1.0 - gam) / (gam * (2.0 - gam));
  std::vector<double> xb(xg), Tb(Tg);
  for (int64_t i = 0; i < n3; ++i) { bx[i] = c1 * xg[i] - c0 * x[i]; bT[i] = c1 * Tg[i] - c0 * T[i]; }
  const int it2 = stage_solve(cm, kb, n3, delta, w, h2, bx.data(), bT.data(), xb.data(), Tb.data(), &lam, &C);
  if (it2 < 0) return -1;
  double sx = 0.0, sd = 0.0, S = 0.0;
  for (int64_t i = 0; i < n3; ++i) {
    if (U != nullptr) {
      const double damp = std::exp(-0.5 * h * ((ka.kd * x[i] + ka.H) + (kb.kd * xb[i] + kb.H)));
      U[3 * i + 0] *= damp; U[3 * i + 1] *= damp; U[3 * i + 2] *= damp;
    }
    x[i] = xb[i];
    T[i] = Tb[i];
    const double nn = kb.nH * delta[i];
    if (emis) emis[i] = alpha_e<double>(cm, Tb[i]) * (nn * xb[i]) * (nn * xb[i]);
    sx += delta[i] * xb[i];
    sd += delta[i];
    S += delta[i] * (1.0 - xb[i]);
  }
  st->lambda = lam;
  st->C = C;
  st->Xe = sx / sd;
  st->S1s = S;
  st->iters = it1 + it2;
  st->dt = h;
  return 0;
}

// n_sub substeps uniform in ln(1+z) between z_from and z_to.
double sub_z(double z_from, double z_to, int k, int n_sub) {
  if (k == 0) return z_from;
  if (k == n_sub) return z_to;
  double ya = std::log1p(z_from), yb = std::log1p(z_to);
  return std::expm1(ya - (ya - yb) * (double)k / (double)n_sub);
}

template <class R>
void rec_step_t(const Cosmo& cm, int n, int mixing, double fmix, int n_sub, double z_from, double z_to,
                const R* delta, R* x, R* T, double* U, const R* afrac, R* emis, SubStats<R>* st) {
  const int64_t n3 = (int64_t)n * n * n;
  for (int k = 0; k < n_sub; ++k)
    substep<R>(cm, n, n3, mixing, fmix, sub_z(z_from, z_to, k, n_sub), sub_z(z_from, z_to, k + 1, n_sub), delta, x, T,
               U, afrac, emis, st);
}

// Objective over a trajectory (Sec. II.A for X_e; the visibility function is
// (d tau/dz) e^{-tau} with tau the Thomson optical depth, trapezoid on nodes).
template <class R>
R trajectory(const Cosmo& cm, int n, int mixing, int n_sub, int n_steps, const double* zs,
             const uint32_t* tallies, const R* delta, const R* x0, const R* T0, const R* a_pert, int objective,
             double z_star, double* Xe_hist) {
  int64_t n3 = (int64_t)n * n * n;
  std::vector<R> x(x0, x0 + n3), T(T0, T0 + n3), af(n3);
  std::vector<R> Xe(n_steps + 1);
  auto xe_of = [&](const std::vector<R>& xx) {
    R a = 0.0, b = 0.0;
    for (int64_t i = 0; i < n3; ++i) { a += delta[i] * xx[i]; b += delta[i]; }
    return a / b;
  };
  Xe[0] = xe_of(x);
  for (int s = 0; s < n_steps; ++s) {
    const R* afp = nullptr;
    if (mixing == 0 && tallies != nullptr) {
      const uint32_t* t = tallies + (int64_t)s * n3;
      uint64_t tot = 0;
      for (int64_t i = 0; i < n3; ++i) tot += t[i];
      if (tot > 0) {
        for (int64_t i = 0; i < n3; ++i) {
          af[i] = R((double)t[i] / (double)tot);
          if (a_pert) af[i] = af[i] + a_pert[i];
        }
        afp = af.data();
      }
    }
    SubStats<R> st;
    rec_step_t<R>(cm, n, mixing, 1.0, n_sub, zs[s], zs[s + 1], delta, x.data(), T.data(), nullptr, afp, nullptr,
                  &st);
    Xe[s + 1] = st.Xe;
  }
  if (Xe_hist)
    for (int k = 0; k <= n_steps; ++k) Xe_hist[k] = val(Xe[k]);
  int ks = 0;
  for (int k = 1; k <= n_steps; ++k)
    if (std::fabs(zs[k] - z_star) < std::fabs(zs[ks] - z_star)) ks = k;
  if (objective == 1) return Xe[ks];
  // d tau/dz = sigma_T c nbar_H X_e / ((1+z) H)
  auto f = [&](int k) { return Xe[k] * (kSigmaT * kC * nH_bar(cm, zs[k]) / ((1.0 + zs[k]) * hubble(cm, zs[k]))); };
  R tau = 0.0;
  for (int m = ks; m < n_steps; ++m) tau += 0.5 * (f(m) + f(m + 1)) * (zs[m] - zs[m + 1]);
  return f(ks) * exp(-tau);
}

}  // namespace

extern "C" {

int orc_background(const orc_cosmo* cp, double z, double* out) {
  if (!cp || !out) return -1;
  Cosmo c = make_cosmo(cp);
  out[0] = hubble(c, z);
  out[1] = nH_bar(c, z);
  out[2] = T_gamma(c, z);
  out[3] = c.Or;
  out[4] = c.OL;
  return 0;
}

double orc_dt(const orc_cosmo* cp, double z_from, double z_to) {
  Cosmo c = make_cosmo(cp);
  return cosmic_dt(c, z_from, z_to);
}

int orc_rates(const orc_cosmo* cp, double z, double T_b, double* out) {
  if (!cp || !out || !(T_b > 0)) return -1;
  Cosmo c = make_cosmo(cp);
  double Tg = T_gamma(c, z);
  out[0] = alpha_e<double>(c, T_b);
  out[1] = beta_e(c, Tg);
  out[2] = std::exp(-kEalpha / (kKB * Tg));
  out[3] = kLambda2g;
  out[4] = 8.0 * kPi * hubble(c, z) / (kLambdaAlpha * kLambdaAlpha * kLambdaAlpha);
  out[5] = saha_phase(T_b) * std::exp(-kEion / (kKB * T_b));
  return 0;
}

int orc_saha_xe(const orc_cosmo* cp, double z, int64_t n3, const double* delta, double* x_out) {
  if (!cp || !delta || !x_out || n3 < 0) return -1;
  Cosmo c = make_cosmo(cp);
  double Tg = T_gamma(c, z);
  double S = saha_phase(Tg) * std::exp(-kEion / (kKB * Tg));
  for (int64_t i = 0; i < n3; ++i) {
    // x^2/(1-x) = S / n_H  =>  x = 2 / (1 + sqrt(1 + 4 n_H / S))
    double nH = nH_bar(c, z) * delta[i];
    x_out[i] = 2.0 / (1.0 + std::sqrt(1.0 + 4.0 * nH / S));
  }
  return 0;
}

int orc_rec_step(const orc_cosmo* cp, int n, int mixing, int n_sub, double z_from, double z_to,
                 const double* delta, double* x, double* T, double* U, const uint32_t* tally, double* emis,
                 double* stats, double f_alpha) {
  if (!cp || n <= 0 || n_sub <= 0 || !delta || !x || !T || !(z_from > z_to) || mixing < 0 || mixing > 3)
    return -1;
  if (mixing == 3 && !(f_alpha >= 0.0 && f_alpha <= 1.0)) return -1;
  Cosmo c = make_cosmo(cp);
  int64_t n3 = (int64_t)n * n * n;
  std::vector<double> af;
  const double* afp = nullptr;
  if (mixing == 0 && tally != nullptr) {
    uint64_t tot = 0;
    for (int64_t i = 0; i < n3; ++i) tot += tally[i];
    if (tot > 0) {
      af.resize(n3);
      for (int64_t i = 0; i < n3; ++i) af[i] = (double)tally[i] / (double)tot;
      afp = af.data();
    }
  }
  SubStats<double> st;
  rec_step_t<double>(c, n, mixing, f_alpha, n_sub, z_from, z_to, delta, x, T, U, afp, emis, &st);
  if (stats) {
    stats[0] = st.lambda;
    stats[1] = st.C;
    stats[2] = st.Xe;
    stats[3] = st.iters;
    stats[4] = st.S1s;
    stats[5] = st.dt;
  }
  return 0;
}

int orc_rec_step_trbdf2(const orc_cosmo* cp, int n, int mixing, int n_sub, double z_from, double z_to,
                        const double* delta, double* x, double* T, double* U, const uint32_t* tally, double* emis,
                        double* stats) {
  if (!cp || n <= 0 || n_sub <= 0 || !delta || !x || !T || !(z_from > z_to) || (mixing != 0 && mixing != 1))
    return -1;
  Cosmo c = make_cosmo(cp);
  const int64_t n3 = (int64_t)n * n * n;
  // w_i = J_i / <J> from the absorbed-Ly-alpha fractions (TALLY), 1 otherwise; held
  // over the step as in the backward-Euler substep (it uses the step-start n_1s)
  std::vector<double> w(n3, 1.0);
  if (mixing == 0 && tally != nullptr) {
    uint64_t tot = 0;
    for (int64_t i = 0; i < n3; ++i) tot += tally[i];
    double S = 0.0;
    for (int64_t i = 0; i < n3; ++i) S += delta[i] * (1.0 - x[i]);
    if (tot > 0 && S > 0.0) {
      for (int64_t i = 0; i < n3; ++i) {
        const double n1s_rel = delta[i] * (1.0 - x[i]);
        if (n1s_rel > 0.0) w[i] = ((double)tally[i] / (double)tot) * S / n1s_rel;
      }
    }
  }
  SubStats<double> st;
  for (int k = 0; k < n_sub; ++k) {
    if (substep_trbdf2(c, n3, sub_z(z_from, z_to, k, n_sub), sub_z(z_from, z_to, k + 1, n_sub), delta, w.data(), x,
                       T, U, emis, &st) != 0)
      return -3;
  }
  if (stats) {
    stats[0] = st.lambda;
    stats[1] = st.C;
    stats[2] = st.Xe;
    stats[3] = st.iters;
    stats[4] = st.S1s;
    stats[5] = st.dt;
  }
  return 0;
}

int orc_divergence(const orc_cosmo* cp, int n, double z, const double* U, double* div) {
  if (!cp || n <= 0 || !U || !div) return -1;
  Cosmo c = make_cosmo(cp);
  local_divergence(n, U, c.L_m, z, div);
  return 0;
}

int orc_traj_objective(const orc_cosmo* cp, int n, int mixing, int n_sub, int n_steps, const double* zs,
                       const uint32_t* tallies, const double* delta, const double* x0, const double* T0,
                       const double* a_pert, int objective, double z_star, double* J, double* Xe_hist) {
  if (!cp || n <= 0 || n_steps <= 0 || !zs || !delta || !x0 || !T0 || !J || (objective != 1 && objective != 2))
    return -1;
  Cosmo c = make_cosmo(cp);
  J[0] = trajectory<double>(c, n, mixing, n_sub, n_steps, zs, tallies, delta, x0, T0, a_pert, objective, z_star,
                            Xe_hist);
  return 0;
}

int orc_traj_tangent(const orc_cosmo* cp, int n, int mixing, int n_sub, int n_steps, const double* zs,
                     const uint32_t* tallies, const double* delta, const double* x0, const double* T0,
                     const double* d_delta, const double* d_T0, const double* d_a, int objective, double z_star,
                     double* J) {
  if (!cp || n <= 0 || n_steps <= 0 || !zs || !delta || !x0 || !T0 || !J || (objective != 1 && objective != 2))
    return -1;
  Cosmo c = make_cosmo(cp);
  int64_t n3 = (int64_t)n * n * n;
  std::vector<Dual> dd(n3), xx(n3), tt(n3), aa(n3);
  for (int64_t i = 0; i < n3; ++i) {
    dd[i] = Dual(delta[i], d_delta ? d_delta[i] : 0.0);
    xx[i] = Dual(x0[i], 0.0);
    tt[i] = Dual(T0[i], d_T0 ? d_T0[i] : 0.0);
    aa[i] = Dual(0.0, d_a ? d_a[i] : 0.0);
  }
  Dual r = trajectory<Dual>(c, n, mixing, n_sub, n_steps, zs, tallies, dd.data(), xx.data(), tt.data(), aa.data(),
                            objective, z_star, nullptr);
  J[0] = r.v;
  J[1] = r.d;
  return 0;
}

}  // extern "C"
