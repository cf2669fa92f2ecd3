/*
 * Oracle for the recombination hot path of Jedamzik, Abel & Ali-Haimoud,
 * "Cosmic Recombination in the Presence of Primordial Magnetic Fields"
 * (arXiv:2312.11448).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64
 * restatement of what the GPU path computes, written from the paper.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header, constant table or helper with the CUDA
 * library; the two agree only because both follow the same definitions.
 *
 * Parity status of each function is stated beside it: "pinned by ..." names
 * the independent check in tests/ that would fail on a plausible mistake.
 *
 * Conventions
 *   - Cells are indexed c = (iz*n + iy)*n + ix of an n^3 periodic box.
 *   - Velocities are peculiar velocities in km/s; vel4 is [n^3][4] with the
 *     fourth slot unused.
 *   - Every function returns 0 on success and a negative code on bad input.
 */
#ifndef REC_ORACLE_H
#define REC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Cosmological and model parameters (Sec. II.C defaults: h=0.67,
 * Omega_b h^2=0.0224, Omega_c h^2=0.12, Y_p=0.24; box 24 kpc comoving). */
typedef struct {
  double h, omega_b_h2, omega_c_h2, Y_p;
  double T_cmb0;      /* K; not printed in the paper, 2.7255 taken */
  double N_eff;       /* not printed in the paper, 3.046 taken */
  double L_box_kpc;   /* comoving box side */
  double fudge;       /* 1.14 multiplying the case-B coefficient (Sec. III.A.1) */
  double heating;     /* uniform heating Gamma expressed per mean hydrogen atom, eV/s (Sec. VI) */
} orc_cosmo;

/* Background quantities at redshift z: out[0]=H [1/s], out[1]=nbar_H [1/m^3],
 * out[2]=T_gamma [K], out[3]=Omega_r, out[4]=Omega_Lambda.  Pinned by closed forms. */
int orc_background(const orc_cosmo* cp, double z, double* out);

/* Cosmic time elapsed from z_from down to z_to (z_from > z_to), seconds.
 * Pinned by the matter+radiation closed form. */
double orc_dt(const orc_cosmo* cp, double z_from, double z_to);

/* Rate coefficients of the effective three-level atom (Sec. III.A.1,
 * Eqs. rec0, n2s-sol, Cfactor): out[0]=alpha_e(T_b) [m^3/s],
 * out[1]=beta_e(T_gamma) [1/s per 2s atom], out[2]=exp(-E_alpha/kT_gamma),
 * out[3]=Lambda_2gamma, out[4]=8 pi H/lambda_alpha^3 [1/(m^3 s)]...per n_1s,
 * out[5]=Saha factor (2 pi m_e k T/h^2)^{3/2} exp(-E_ion/kT) [1/m^3].
 * Pinned by textbook case-B values and Saha equilibrium. */
int orc_rates(const orc_cosmo* cp, double z, double T_b, double* out);

/* Hydrogen Saha ionisation fraction per cell at redshift z (T_b = T_gamma). */
int orc_saha_xe(const orc_cosmo* cp, double z, int64_t n3, const double* delta, double* x_out);

/* One recombination step z_from -> z_to in n_sub substeps (Sec. IV, Eq.
 * dotne-mix; Eq. Tb-evolution; Eq. alpha-def).  mixing: 0 = TALLY (local 2s
 * population from the absorbed-Ly-alpha tallies), 1 = FULL (the paper's
 * full-mixing limit), 2 = LOCAL (the no-mixing limit of Sec. III.A.2: Eq. rec
 * per cell with H -> H + div v / 3 in Eq. R-alpha; div v from U, zero if U is
 * NULL; stats[1] = volume mean of the local C, stats[3] = 0), 3 = PARTIAL (the
 * fraction f_alpha in [0, 1] of the full-mixing rate plus 1 - f_alpha of the
 * local one; f_alpha is read in this mode only).  In/out: x (ionisation fraction), T (K), U ([n^3][3],
 * km/s, may be NULL).  tally may be NULL in FULL mode.  emis (may be NULL)
 * receives alpha_e n_e^2 at the end state.  stats[0]=lambda, [1]=C_mix,
 * [2]=X_e, [3]=Newton iterations of the last substep, [4]=S_1s used,
 * [5]=dt of the last substep.  Pinned by Saha, the standard TLA ODE, the
 * two-zone ODE system and the global-rate identity. */
int orc_rec_step(const orc_cosmo* cp, int n, int mixing, int n_sub, double z_from, double z_to,
                 const double* delta, double* x, double* T, double* U, const uint32_t* tally,
                 double* emis, double* stats, double f_alpha);

/* The same step as orc_rec_step (modes 0 = TALLY and 1 = FULL) advanced by the
 * second-order TR-BDF2 scheme per substep: a trapezoidal stage to t + gamma h
 * (gamma = 2 - sqrt 2) and a BDF2 stage to t + h, each stage end fully
 * implicit in x, T, lambda and the Peebles factor; drag with the trapezoidal
 * exponent.  Returns -3 where a stage has no positive root (step too long).
 * Pinned by second-order convergence to stiff ODE integrations of the
 * standard three-level atom and of the two-zone system. */
int orc_rec_step_trbdf2(const orc_cosmo* cp, int n, int mixing, int n_sub, double z_from, double z_to,
                        const double* delta, double* x, double* T, double* U, const uint32_t* tally, double* emis,
                        double* stats);

/* Physical divergence of the peculiar velocity U ([n^3][3], km/s) at redshift
 * z, 1/s: periodic central differences on the comoving grid of side L_box,
 * times 1 + z.  Pinned by the closed form for sinusoidal fields. */
int orc_divergence(const orc_cosmo* cp, int n, double z, const double* U, double* div);

/* Philox4x32-10 block (Salmon, Moraes, Dror, Shaw, SC'11).  Pinned word for
 * word against the cuRAND library's host Philox4_32_10 generator (random keys
 * and counters) and by statistical tests (uniformity, bit balance, avalanche). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Threads of the transport: 1 in the plain build; the OpenMP build (host-cores
 * timing baseline) sets its thread count to n (> 0) and returns it. */
int orc_threads(int n);

/* Transport scalars at redshift z for an n^3 box: out[0] = kappa, cells of
 * Hubble drift per km/s of velocity; out[1] = cth, so that the thermal
 * velocity in cells is sqrt(T * cth). */
int orc_transport_params(const orc_cosmo* cp, int n, double z, double* out);

/* Packet allocation (binary32 or binary64 emission weights): P[0..n^3] is
 * the exclusive prefix of packets per cell, P[n^3] = n_packets.  Pinned by
 * exact totals and the expected count per cell. */
int orc_allocate_f32(int n, const float* emis, uint64_t n_packets, uint64_t seed, uint32_t step,
                     uint32_t box, uint32_t* P);
int orc_allocate_f64(int n, const double* emis, uint64_t n_packets, uint64_t seed, uint32_t step,
                     uint32_t box, uint32_t* P);

/* One emitted packet, for the closed-form and brute-force checks. */
typedef struct {
  uint32_t home, j, absorb, crossings;
  double f[3];     /* offset of the emission point inside the home cell */
  double dir[3];   /* unit direction */
  double xi;       /* emission frequency offset, Doppler units */
  double u0;       /* resonance distance in cells of Hubble drift at emission */
} orc_packet;

/* Ballistic Ly-alpha packet transport (binary32 / binary64 arithmetic).
 * counters[0]=emitted, [1]=absorbed, [2]=packets stopped by the crossing cap,
 * [3]=total face crossings.  dump (may be NULL) receives up to dump_cap
 * packets in emission order.  Pinned by the closed-form resonance cell with
 * U = 0, conservation, and a brute-force crossing enumeration. */
int orc_transport_f32(const orc_cosmo* cp, int n, double z, uint64_t seed, uint32_t step, uint32_t box,
                      uint64_t n_packets, const float* emis, const float* vel4, const float* T,
                      const float* quant, int M, uint32_t* tally, uint64_t* counters,
                      orc_packet* dump, int64_t dump_cap);
int orc_transport_f64(const orc_cosmo* cp, int n, double z, uint64_t seed, uint32_t step, uint32_t box,
                      uint64_t n_packets, const double* emis, const double* vel4, const double* T,
                      const double* quant, int M, uint32_t* tally, uint64_t* counters,
                      orc_packet* dump, int64_t dump_cap);

/* Objective over a trajectory of n_steps steps through the node redshifts
 * zs[0..n_steps] with fixed per-step tallies ([n_steps][n^3], NULL in FULL
 * mode).  objective: 1 = volume-averaged X_e at the node nearest z_star,
 * 2 = visibility g = (d tau/dz) exp(-tau) at that node, tau integrated from
 * the last node.  a_pert (may be NULL) is added to every step's absorbed
 * fraction.  Xe_hist (may be NULL) receives X_e at every node. */
int orc_traj_objective(const orc_cosmo* cp, int n, int mixing, int n_sub, int n_steps, const double* zs,
                       const uint32_t* tallies, const double* delta, const double* x0, const double* T0,
                       const double* a_pert, int objective, double z_star, double* J, double* Xe_hist);

/* Forward-mode tangent of the same objective along the direction
 * (d_delta, d_T0, d_a): J[0] = objective, J[1] = its directional derivative. */
int orc_traj_tangent(const orc_cosmo* cp, int n, int mixing, int n_sub, int n_steps, const double* zs,
                     const uint32_t* tallies, const double* delta, const double* x0, const double* T0,
                     const double* d_delta, const double* d_T0, const double* d_a, int objective,
                     double z_star, double* J);

/* ---- Resonant-scattering Ly-alpha Monte Carlo (Appendix A) ----------------- */

/* Faddeeva function w(y + i a), a > 0: w[0] = H(a, y) (Voigt function),
 * w[1] = Im w.  Weideman's 48-term rational expansion for |z| < 10, the
 * asymptotic series beyond.  Pinned against the library Faddeeva function
 * and closed forms (H(a,0) = exp(a^2) erfc(a), H(0,y) = exp(-y^2),
 * normalisation sqrt(pi)). */
int orc_faddeeva(double y, double a, double* w);
/* The Voigt table the Monte Carlo uses (cubic Hermite on 1/128 nodes for
 * |y| < 10, asymptotic series beyond), at m points y. */
int orc_voigt_table(double a, int64_t m, const double* y, double* H);

typedef struct {
  double z;         /* redshift of the snapshot */
  double eps;       /* step (3): path of eps mean free paths per step */
  double x_lost;    /* photons whose gas-frame offset falls below -x_lost are lost by redshifting */
  double zeta;      /* expansion rate zeta H (1 normally; Fig. Cfact varies it) */
  double lambda2g;  /* two-photon rate, 1/s; negative: the paper's 8.22 */
  double A_alpha;   /* 2p -> 1s decay rate Gamma_alpha, 1/s */
  uint64_t seed;
  uint32_t step, box;
  uint64_t max_steps;  /* per photon; photons reaching it end as CAPPED */
} orc_mc_params;

enum { ORC_MC_LOST = 0, ORC_MC_TWO_PHOTON = 1, ORC_MC_IONISED = 2, ORC_MC_CAPPED = 3 };

typedef struct {
  uint32_t home, j;   /* emitting cell, photon index in the cell */
  int32_t fate;       /* ORC_MC_* */
  uint64_t n_scat, n_steps;
  double D_kpc;       /* comoving distance from injection to the end point */
  double x_end;       /* final frequency offset, Doppler units, frame without peculiar velocity */
} orc_mc_photon;

/* Derived scalars: out[0]=a, [1]=v_th/c, [2]=sig0 (m^2, <sigma> = sig0 H(a,y)),
 * [3]=dx per physical metre, [4]=p_ion, [5]=p_2gamma per scattering,
 * [6]=beta_e, [7]=Lambda, [8]=zeta H, [9]=nbar_H, [10]=T_gamma,
 * [11]=comoving cells per physical metre. */
int orc_mc_setup(const orc_cosmo* cp, const orc_mc_params* mp, int n, double* out);

/* m independent scatterings of a photon at gas-frame offset y travelling
 * along kin (Eq. inout, isotropic): ppar[i] = scattering atom's parallel
 * velocity, dy[i] = y_out - y, kout[3i..3i+2] = outgoing direction.  Any
 * output may be NULL. */
int orc_mc_redistribution(double a, double y, const double* kin, uint64_t seed, int64_t m, double* ppar,
                          double* dy, double* kout);

/* Photons k0..k1-1 of the allocation prefix P (n^3 + 1 entries, as from
 * orc_allocate_*) through steps (1)-(8) in an n^3 periodic box at redshift z
 * with overdensity delta, ionisation fraction xe and peculiar velocity U
 * ([n^3][3] km/s, may be NULL); T = T_gamma(z) throughout.  out[k - k0] per
 * photon; counters[0..3] = photons per fate, counters[4] = atom-velocity
 * draws that hit the rejection cap.  Pinned by the redistribution moments,
 * the first-flight distance law, Galilean invariance and the Sobolev
 * escape / C factor (Fig. Cfact). */
int orc_lya_mc(const orc_cosmo* cp, const orc_mc_params* mp, int n, const double* delta, const double* xe,
               const double* U, const uint32_t* P, uint64_t k0, uint64_t k1, orc_mc_photon* out,
               uint64_t* counters);

#ifdef __cplusplus
}
#endif
#endif
