// Host-side scalar physics of the recombination library: background
// cosmology, substep coefficients of the three-level atom and the transport
// scalars.  Everything here depends only on redshifts and parameters.
//
// References: Jedamzik, Abel & Ali-Haimoud, arXiv:2312.11448 -- Sec. II.A
// (Eq. alpha-def, Eq. Tb-evolution), Sec. III.A.1 (Eqs. rec0, n2s-sol,
// R-alpha, Cfactor), Sec. IV.B (Eq. dotne-mix), Appendix A (transport).

#include <cmath>

#include "rec_internal.cuh"

namespace rec {
namespace {

// SI constants (CODATA 2018)
constexpr double c_light = 2.99792458e8;
constexpr double h_planck = 6.62607015e-34;
constexpr double k_boltz = 1.380649e-23;
constexpr double m_elec = 9.1093837015e-31;
constexpr double sigma_thomson = 6.6524587321e-29;
constexpr double sigma_sb = 5.670374419e-8;
constexpr double G_newton = 6.67430e-11;
constexpr double amu = 1.66053906660e-27;
constexpr double m_hyd = 1.00782503223 * amu;
constexpr double m_hel = 4.00260325413 * amu;
constexpr double e_volt = 1.602176634e-19;
constexpr double megaparsec = 3.0856775814913673e22;
constexpr double pi = 3.14159265358979323846;

// Radiation constant 4 sigma_SB / c.
const double a_rad = 4.0 * sigma_sb / c_light;
// Ground-state ionisation energy of hydrogen (13.598434 eV).
const double E_ion = 13.598434 * e_volt;
// Ly-alpha energy (10.2 eV in Sec. III.A.1) and 2s binding energy: 3/4 and 1/4
// of E_ion, so that detailed balance reproduces the Saha equation exactly.
const double E_lya = 0.75 * E_ion;
const double E_2s = 0.25 * E_ion;
const double lambda_lya = h_planck * c_light / E_lya;
// Two-photon 2s->1s rate (Sec. III.A.1).
constexpr double Lambda_2g = 8.22;
// Case-B recombination fit of Pequignot, Petitjean & Boisson (1991), cited in
// Sec. III.A.1: A_B(T) = 1e-19 a t^b / (1 + c t^d) m^3/s, t = T / 1e4 K.
constexpr double ppb_a = 4.309, ppb_b = -0.6166, ppb_c = 0.6703, ppb_d = 0.5300;

double case_b(const Cosmo& c, double T) {
  double t = T / 1.0e4;
  return c.fudge * 1.0e-19 * ppb_a * std::pow(t, ppb_b) / (1.0 + ppb_c * std::pow(t, ppb_d));
}

double phase_space(double T) {
  return std::pow(2.0 * pi * m_elec * k_boltz * T / (h_planck * h_planck), 1.5);
}

}  // namespace

Cosmo make_cosmo(const rec_params& p) {
  Cosmo c;
  c.H0 = p.h * 1.0e5 / megaparsec;
  double rho_crit = 3.0 * c.H0 * c.H0 / (8.0 * pi * G_newton);
  double Ob = p.omega_b_h2 / (p.h * p.h);
  double Oc = p.omega_c_h2 / (p.h * p.h);
  c.Om = Ob + Oc;
  double T0 = p.T_cmb0;
  double Og = a_rad * T0 * T0 * T0 * T0 / (c_light * c_light) / rho_crit;
  double Onu = p.N_eff * (7.0 / 8.0) * std::pow(4.0 / 11.0, 4.0 / 3.0) * Og;
  c.Or = Og + Onu;
  c.OL = 1.0 - c.Om - c.Or;
  c.nH0 = (1.0 - p.Y_p) * Ob * rho_crit / m_hyd;
  c.T0 = T0;
  c.Yp = p.Y_p;
  c.fHe = p.Y_p * m_hyd / ((1.0 - p.Y_p) * m_hel);
  c.L_m = p.L_box_kpc * megaparsec * 1.0e-3;
  c.fudge = p.fudge;
  c.heat = p.heating;
  return c;
}

double hubble(const Cosmo& c, double z) {
  double a1 = 1.0 + z;
  return c.H0 * std::sqrt(c.Om * a1 * a1 * a1 + c.Or * a1 * a1 * a1 * a1 + c.OL);
}
double nH_bar(const Cosmo& c, double z) { double a1 = 1.0 + z; return c.nH0 * a1 * a1 * a1; }
double T_gamma(const Cosmo& c, double z) { return c.T0 * (1.0 + z); }

// Elapsed cosmic time: integral of d ln(1+z) / H (Simpson's rule on the step).
double cosmic_dt(const Cosmo& c, double z_from, double z_to) {
  double ya = std::log1p(z_from), yb = std::log1p(z_to);
  double zm = std::expm1(0.5 * (ya + yb));
  return (ya - yb) / 6.0 * (1.0 / hubble(c, z_to) + 4.0 / hubble(c, zm) + 1.0 / hubble(c, z_from));
}

// kappa: cells of Hubble drift per km/s of velocity, n / (H a L) with the
// proper box size a L; cth: kappa^2 times 2 k / m_H in (km/s)^2 per K.  The
// operation order is fixed (it defines the bits the transport consumes).
void transport_scalars(const Cosmo& c, int n, double z, double* kappa, double* cth) {
  double H = hubble(c, z);
  double a = 1.0 / (1.0 + z);
  double v_box = H * a * c.L_m * 1.0e-3;
  double k = (double)n / v_box;
  *kappa = k;
  *cth = k * k * (2.0 * k_boltz / m_hyd * 1.0e-6);
}

double thomson_sigma_c() { return sigma_thomson * c_light; }

double saha_S(double T) { return phase_space(T) * std::exp(-E_ion / (k_boltz * T)); }

StepCoef step_coef(const Cosmo& c, const rec_params& p, double z_from, double z_to, int last) {
  StepCoef s;
  s.dt = cosmic_dt(c, z_from, z_to);
  s.H = hubble(c, z_to);
  s.nH = nH_bar(c, z_to);
  s.Tg = T_gamma(c, z_to);
  double Tg4 = s.Tg * s.Tg * s.Tg * s.Tg;
  // Eq. Tb-evolution: Compton term 8 sigma_T x n_H rho_gamma / (3 m_e c n_tot).
  s.kc = 8.0 * sigma_thomson * a_rad * Tg4 / (3.0 * m_elec * c_light);
  // Eq. alpha-def: (4/3) n_e sigma_T rho_gamma / rho_b with n_e/rho_b = x (1-Y_p)/m_H.
  s.kd = 4.0 * sigma_thomson * a_rad * Tg4 * (1.0 - c.Yp) / (3.0 * c_light * m_hyd);
  // Uniform heating 2 Gamma / (3 n_tot k), Gamma = heating * nbar_H.
  s.hq = 2.0 * c.heat * e_volt / (3.0 * k_boltz);
  s.fHe = c.fHe;
  // beta_e by detailed balance at T_gamma, per 2s atom (Sec. III.A.1 footnote).
  s.beta = case_b(c, s.Tg) * phase_space(s.Tg) * std::exp(-E_2s / (k_boltz * s.Tg));
  s.ea = std::exp(-E_lya / (k_boltz * s.Tg));
  s.KR = 8.0 * pi * s.H / (lambda_lya * lambda_lya * lambda_lya);
  s.L2g = Lambda_2g;
  s.fa = c.fudge * 1.0e-19 * ppb_a;
  s.pb = ppb_b;
  s.pc = ppb_c;
  s.pd = ppb_d;
  s.mixing = p.mixing;
  s.last = last;
  return s;
}

}  // namespace rec
