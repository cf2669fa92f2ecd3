// Reverse (adjoint) of one recombination step, FP64, tallies held fixed.
//
// Forward substep per cell (see rec_step.cu): T' from Eq. (Tb-evolution),
// alpha = alpha_e(T'), A = dt alpha n_H, s = dt w, and x' the backward-Euler
// root of A x'^2 + (1 + sG) x' - (x + sG) = 0 with G = (1-C) lambda + C beta e_a;
// lambda solves F(lambda) = sum alpha n^2 x'^2 - lambda sum n (1 - x') = 0;
// C depends on S_1s = sum Delta (1 - x) through R_alpha^mix; U' = U exp(-(kd x' + H) dt).
//
// Reverse, by the implicit-function theorem for lambda (no differentiation
// through Newton iterations):
//   mu  = -(sum_i xbar'_i dx'_i/dlambda) / (dF/dlambda)
//   y_i = xbar'_i + mu (2 alpha n^2 x' + lambda n)        (effective adjoint of x'_i)
//   then the chain through A, s, w, alpha(T'), T', Delta, x and the global sums.
// Passes (all on the context stream):
//   k_adj_prep      sums of the pre-step state (S_1s, tally total, lambda guess)
//   k_substep_begin + k_newton   recompute lambda exactly as the forward step
//   k_adj_r1        mu numerator/denominator and X_e of the end state
//   k_adj_r2        per-cell adjoints; sums for the C and S_1s paths
//   k_adj_r3        the S_1s term applied to xbar and g_delta

#include <cmath>

#include "rec_internal.cuh"
#include "rec_reduce.cuh"

namespace rec {

namespace adj {

constexpr int NT = kPassThreads;

struct AdjArgs {
  int64_t n3;
  const double* delta;
  const double* x;
  const double* T;
  const double4_32a* U;
  const uint32_t* tally;
  double* xbar;
  double* Tbar;
  double4_32a* Ubar;
  double* g_delta;
  double* g_a;
  double Xe_bar;
  DevScalars* sc;
  double* part;
  StepCoef k;
};

struct Fwd {
  double opx, g, hh, den, Tn, al, n, A, w, s, a, xr, D, dxdG;
  bool wt;  // w from the tallies
};

__device__ __forceinline__ Fwd forward_cell(const StepCoef& k, double d, double x, double T, uint32_t tal, double tot,
                                            double S1s, double G) {
  Fwd f;
  f.opx = 1.0 + k.fHe + x;
  f.g = k.kc * x / f.opx;
  f.hh = k.hq / (d * f.opx);
  f.den = 1.0 + k.dt * (2.0 * k.H + f.g);
  f.Tn = (T + k.dt * (f.g * k.Tg + f.hh)) / f.den;
  double lt = log(f.Tn * 1.0e-4);
  f.al = k.fa * exp(k.pb * lt) / (1.0 + k.pc * exp(k.pd * lt));
  f.n = k.nH * d;
  f.A = k.dt * f.al * f.n;
  f.w = 1.0;
  f.wt = false;
  f.a = tot > 0.0 ? (double)tal / tot : 0.0;
  if (k.mixing == REC_MIX_TALLY && tot > 0.0) {
    double n1s_rel = d * (1.0 - x);
    if (S1s > 0.0 && n1s_rel > 0.0) { f.w = f.a * S1s / n1s_rel; f.wt = true; }
  }
  f.s = k.dt * f.w;
  double B = 1.0 + f.s * G;
  double cc = x + f.s * G;
  double sq = sqrt(B * B + 4.0 * f.A * cc);
  f.xr = 2.0 * cc / (B + sq);
  f.D = 2.0 * f.A * f.xr + B;
  f.dxdG = f.s * (1.0 - f.xr) / f.D;
  return f;
}

// Incoming adjoint of x' with the X_e seed and the drag term folded in.
__device__ __forceinline__ double xbar_out(const AdjArgs& a, int64_t i, const Fwd& f, double d, double Sd) {
  double xb = a.xbar[i] + a.Xe_bar * d / Sd;
  if (a.Ubar) {
    double4_32a ub = a.Ubar[i], u = a.U[i];
    double E = exp(-(a.k.kd * f.xr + a.k.H) * a.k.dt);
    double dot = (ub.x * u.x + ub.y * u.y + ub.z * u.z) * E;  // Ubar' . U'
    xb += -a.k.kd * a.k.dt * dot;
  }
  return xb;
}

// Sums of the pre-step state: S_1s, sum delta, tally total, lambda guess.
__global__ void __launch_bounds__(NT) k_adj_prep(AdjArgs a) {
  double v[5] = {0, 0, 0, 0, 0};
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += (int64_t)gridDim.x * NT) {
    double d = a.delta[i], x = a.x[i];
    v[0] += d * (1.0 - x);
    v[1] += d;
    v[2] += a.tally ? (double)a.tally[i] : 0.0;
    double lt = log(a.T[i] * 1.0e-4);
    double al = a.k.fa * exp(a.k.pb * lt) / (1.0 + a.k.pc * exp(a.k.pd * lt));
    double n = a.k.nH * d;
    v[3] += al * n * n * x * x;
    v[4] += n * (1.0 - x);
  }
  block_sum<5, NT>(v);
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) a.part[(size_t)blockIdx.x * kMaxSums + k] = v[k];
  if (!last_block_done(&a.sc->counter)) return;
  double S[5];
  combine_partials<5, NT>(a.part, gridDim.x, kMaxSums, S);
  if (threadIdx.x == 0) {
    a.sc->S1s = S[0];
    a.sc->Sd = S[1];
    a.sc->tally_total = (unsigned long long)(S[2] + 0.5);
    a.sc->lam_state = S[4] > 0.0 ? S[3] / S[4] : 0.0;
    a.sc->lam_prev = -1.0;
    a.sc->flags = 0;
    a.sc->counter = 0;
  }
}

// R1: numerator and denominator of mu, X_e of the end state.
__global__ void __launch_bounds__(NT) k_adj_r1(AdjArgs a) {
  DevScalars* sc = a.sc;
  const double lam = sc->lam, omC = sc->omC, G = omC * lam + sc->G0;
  const double tot = (double)sc->tally_total, S1s = sc->S1s, Sd = sc->Sd;
  double v[3] = {0, 0, 0};  // sum xbar' dx'/dlambda, dF/dlambda, sum delta x'
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += (int64_t)gridDim.x * NT) {
    double d = a.delta[i];
    Fwd f = forward_cell(a.k, d, a.x[i], a.T[i], a.tally ? a.tally[i] : 0u, tot, S1s, G);
    double xb = xbar_out(a, i, f, d, Sd);
    v[0] += xb * f.dxdG * omC;
    v[1] += (2.0 * f.al * f.n * f.n * f.xr + lam * f.n) * f.dxdG * omC - f.n * (1.0 - f.xr);
    v[2] += d * f.xr;
  }
  block_sum<3, NT>(v);
  if (threadIdx.x == 0)
    for (int k = 0; k < 3; ++k) a.part[(size_t)blockIdx.x * kMaxSums + k] = v[k];
  if (!last_block_done(&sc->counter)) return;
  double S[3];
  combine_partials<3, NT>(a.part, gridDim.x, kMaxSums, S);
  if (threadIdx.x == 0) {
    sc->last_step = -S[0] / S[1];  // mu
    sc->Sdx = S[2];
    sc->counter = 0;
  }
}

// R2: per-cell adjoints (before the S_1s term); sums for the C and S_1s paths.
__global__ void __launch_bounds__(NT) k_adj_r2(AdjArgs a) {
  DevScalars* sc = a.sc;
  const double lam = sc->lam, omC = sc->omC, G = omC * lam + sc->G0;
  const double tot = (double)sc->tally_total, S1s = sc->S1s, Sd = sc->Sd;
  const double mu = sc->last_step, Xe1 = sc->Sdx / Sd;
  const StepCoef& k = a.k;
  const double dGdC = k.beta * k.ea - lam;
  double v[2] = {0, 0};  // Cbar, direct S_1s adjoint through w
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += (int64_t)gridDim.x * NT) {
    const double d = a.delta[i], x = a.x[i];
    Fwd f = forward_cell(k, d, x, a.T[i], a.tally ? a.tally[i] : 0u, tot, S1s, G);
    double xb1 = xbar_out(a, i, f, d, Sd);
    double an2 = f.al * f.n * f.n;
    double y = xb1 + mu * (2.0 * an2 * f.xr + lam * f.n);
    // partials of x'
    double Ab = -y * f.xr * f.xr / f.D;
    double sb = y * G * (1.0 - f.xr) / f.D;
    double xbar = y / f.D;
    v[0] += y * f.dxdG * dGdC;
    // explicit dependence of F on alpha and n
    double alb = mu * f.n * f.n * f.xr * f.xr;
    double nb = mu * (2.0 * f.al * f.n * f.xr * f.xr - lam * (1.0 - f.xr));
    // A = dt alpha n
    alb += Ab * k.dt * f.n;
    nb += Ab * k.dt * f.al;
    // s = dt w
    double wb = sb * k.dt;
    double db = nb * k.nH;
    double ab = 0.0;
    if (f.wt) {
      double n1s_rel = d * (1.0 - x);
      ab = wb * S1s / n1s_rel;
      v[1] += wb * f.w / S1s;
      db += -wb * f.w / d;
      xbar += wb * f.w / (1.0 - x);
    }
    // alpha(T'): d alpha/dT' = (alpha/T') (pb - pc pd t^pd / (1 + pc t^pd))
    double tpd = exp(k.pd * log(f.Tn * 1.0e-4));
    double dal = f.al / f.Tn * (k.pb - k.pc * k.pd * tpd / (1.0 + k.pc * tpd));
    double Tnb = a.Tbar[i] + alb * dal;
    // T' = (T + dt (g Tg + hh)) / den
    double Tb = Tnb / f.den;
    double gb = Tnb * k.dt * (k.Tg - f.Tn) / f.den;
    double hhb = Tnb * k.dt / f.den;
    xbar += gb * k.kc * (1.0 + k.fHe) / (f.opx * f.opx);
    db += -hhb * f.hh / d;
    xbar += -hhb * f.hh / f.opx;
    // X_e of the end state: d/d delta_i of sum(delta x')/sum(delta)
    db += a.Xe_bar * (f.xr - Xe1) / Sd;
    if (a.Ubar) {
      double E = exp(-(k.kd * f.xr + k.H) * k.dt);
      double4_32a ub = a.Ubar[i];
      ub.x *= E; ub.y *= E; ub.z *= E;
      a.Ubar[i] = ub;
    }
    a.xbar[i] = xbar;
    a.Tbar[i] = Tb;
    a.g_delta[i] += db;
    if (a.g_a) a.g_a[i] += ab;
  }
  block_sum<2, NT>(v);
  if (threadIdx.x == 0)
    for (int q = 0; q < 2; ++q) a.part[(size_t)blockIdx.x * kMaxSums + q] = v[q];
  if (!last_block_done(&sc->counter)) return;
  double S[2];
  combine_partials<2, NT>(a.part, gridDim.x, kMaxSums, S);
  if (threadIdx.x == 0) {
    // C = (L + R)/(beta + L + R), R = KR n3 / (nH S_1s): dC/dS = beta/(beta+L+R)^2 * (-R/S)
    double R = k.KR * (double)a.n3 / (k.nH * S1s);
    double den = k.beta + k.L2g + R;
    double dCdS = k.beta / (den * den) * (-R / S1s);
    sc->Sdx = S[0] * dCdS + S[1];  // adjoint of S_1s
    sc->counter = 0;
  }
}

// R3: S_1s = sum delta (1 - x) pulls the S_1s adjoint back to x and delta.
__global__ void __launch_bounds__(NT) k_adj_r3(AdjArgs a) {
  const double Sb = a.sc->Sdx;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += (int64_t)gridDim.x * NT) {
    double d = a.delta[i], x = a.x[i];
    a.xbar[i] += -Sb * d;
    a.g_delta[i] += Sb * (1.0 - x);
  }
}

// X_e adjoint at a node: X_e = sum(delta x)/sum(delta).
__global__ void __launch_bounds__(NT) k_xe_sum(const double* delta, const double* x, int64_t n3, DevScalars* sc,
                                               double* part) {
  double v[2] = {0, 0};
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n3; i += (int64_t)gridDim.x * NT) {
    v[0] += delta[i] * x[i];
    v[1] += delta[i];
  }
  block_sum<2, NT>(v);
  if (threadIdx.x == 0)
    for (int q = 0; q < 2; ++q) part[(size_t)blockIdx.x * kMaxSums + q] = v[q];
  if (!last_block_done(&sc->counter)) return;
  double S[2];
  combine_partials<2, NT>(part, gridDim.x, kMaxSums, S);
  if (threadIdx.x == 0) {
    sc->Sdx = S[0];
    sc->Sd = S[1];
    sc->counter = 0;
  }
}

__global__ void __launch_bounds__(NT) k_xe_apply(const double* delta, const double* x, int64_t n3, DevScalars* sc,
                                                 double Xe_bar, double* xbar, double* g_delta) {
  const double Sd = sc->Sd, Xe = sc->Sdx / Sd;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n3; i += (int64_t)gridDim.x * NT) {
    xbar[i] += Xe_bar * delta[i] / Sd;
    g_delta[i] += Xe_bar * (x[i] - Xe) / Sd;
  }
}

}  // namespace adj

cudaError_t launch_rec_step_adjoint(rec_ctx* c, double z_from, double z_to, const double* x_in, const double* T_in,
                                    const double* vel4_in, const uint32_t* tally_in, double* xbar, double* Tbar,
                                    double* Ubar, double* g_delta, double* g_a, double Xe_bar_out) {
  StepCoef k = step_coef(c->cosmo, c->params, z_from, z_to, 1);
  adj::AdjArgs a;
  a.n3 = c->n3;
  a.delta = (const double*)c->box.delta;
  a.x = x_in;
  a.T = T_in;
  a.U = (const double4_32a*)vel4_in;
  a.tally = tally_in;
  a.xbar = xbar;
  a.Tbar = Tbar;
  a.Ubar = (double4_32a*)Ubar;
  a.g_delta = g_delta;
  a.g_a = g_a;
  a.Xe_bar = Xe_bar_out;
  a.sc = c->sc_adj;
  a.part = c->part;
  a.k = k;
  GroupTimer t(c, kTAdj, kNewtonMaxPasses + 5);
  adj::k_adj_prep<<<c->grid, adj::NT, 0, c->stream>>>(a);
  enqueue_newton_passes(c, c->sc_adj, k, x_in, T_in, tally_in);
  adj::k_adj_r1<<<c->grid, adj::NT, 0, c->stream>>>(a);
  adj::k_adj_r2<<<c->grid, adj::NT, 0, c->stream>>>(a);
  adj::k_adj_r3<<<c->grid, adj::NT, 0, c->stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_xe_adjoint(rec_ctx* c, const double* x, double Xe_bar, double* xbar, double* g_delta) {
  const double* delta = (const double*)c->box.delta;
  GroupTimer t(c, kTOther, 2);
  adj::k_xe_sum<<<c->grid, adj::NT, 0, c->stream>>>(delta, x, c->n3, c->sc_adj, c->part);
  adj::k_xe_apply<<<c->grid, adj::NT, 0, c->stream>>>(delta, x, c->n3, c->sc_adj, Xe_bar, xbar, g_delta);
  return cudaGetLastError();
}

}  // namespace rec
