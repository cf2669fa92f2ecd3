// Per-cell recombination step on the GPU: backward-Euler update of x_e with
// the full-mixing / tally-driven 2s population and a self-consistent global
// lambda = <alpha n_e^2>/<n_1s> (Newton over streaming passes), the T_b update
// and Compton drag.
//
// Physics (arXiv:2312.11448): the local rate of Eq. (dotne-mix),
//   n_dot_e = -C (alpha n_e^2 - beta n_1s e_a) - (1-C) alpha (n_e^2 - n_1s <n_e^2>/<n_1s>),
// is, per hydrogen atom, dx/dt = -alpha n_H x^2 + w G (1 - x) with
// G = (1-C) lambda + C beta e_a (Eq. n2s-sol on box averages) and w = 1 in the
// full-mixing limit; in tally mode w_i = a_i S_1s / (Delta_i (1-x_i)) follows the
// absorbed Ly-alpha packets.  C uses R_alpha^mix = 8 pi H/(lambda_a^3 <n_1s>)
// (Eq. R-alpha, Sec. IV.A.2).  T_b follows Eq. (Tb-evolution) and the velocity
// Eq. (momentum) with the drag rate of Eq. (alpha-def).
//
// Pass structure per substep (all on the context stream, no host sync):
//   k_substep_begin  (1 block)  C, G offset and the lambda guess from device sums
//   k_newton x N     streaming  F(lambda), F'(lambda); last block takes the Newton step;
//                               exits immediately once converged
//   k_final          streaming  writes x, T, U, emission weights, zeroes tallies,
//                               and the sums of the new state
// Two forms: FP64 (all binary64) and MIXED (binary32 per-cell coefficients and
// root, binary64 state x, net-rate residual correction and volume sums).

#include <cmath>

#include "rec_internal.cuh"
#include "rec_reduce.cuh"

namespace rec {
namespace {

constexpr int NT = kPassThreads;

struct PassArgs {
  int64_t n3;
  const void* delta;
  void* vel4;
  double* x;
  void* T;
  uint32_t* tally;
  void* emis;
  DevScalars* sc;
  double* part;
  StepCoef k;
  int64_t n3_total;
};

__device__ __forceinline__ int32_t ld_flag(const int32_t* p) { return *(volatile const int32_t*)p; }

// ---------------------------------------------------------------- FP64 cell
struct CellF64 {
  double Tn, al, n, A, s;
};

// Coefficients of one cell at the substep end (backward Euler, x_old in the
// Compton and heating terms).  w uses the substep-start neutral fraction.
__device__ __forceinline__ CellF64 cell_f64(const StepCoef& k, double d, double x, double T, uint32_t tal,
                                            double tot, double S1s) {
  CellF64 c;
  double opx = 1.0 + k.fHe + x;
  double g = k.kc * x / opx;
  double hh = k.hq / (d * opx);
  c.Tn = (T + k.dt * (g * k.Tg + hh)) / (1.0 + k.dt * (2.0 * k.H + g));
  double lt = log(c.Tn * 1.0e-4);
  c.al = k.fa * exp(k.pb * lt) / (1.0 + k.pc * exp(k.pd * lt));
  c.n = k.nH * d;
  c.A = k.dt * c.al * c.n;
  double w = 1.0;
  if (k.mixing == REC_MIX_TALLY && tot > 0.0) {
    double n1s_rel = d * (1.0 - x);
    if (S1s > 0.0 && n1s_rel > 0.0) w = ((double)tal / tot) * S1s / n1s_rel;
  }
  c.s = k.dt * w;
  return c;
}

// Positive root of A x'^2 + (1 + sG) x' - (x + sG) = 0 and d x'/dG.
__device__ __forceinline__ double root_f64(double A, double s, double G, double x, double* dxdG) {
  double B = 1.0 + s * G;
  double cc = x + s * G;
  double sq = sqrt(B * B + 4.0 * A * cc);
  double xr = 2.0 * cc / (B + sq);
  if (dxdG) *dxdG = s * (1.0 - xr) / (2.0 * A * xr + B);
  return xr;
}

// --------------------------------------------------------------- MIXED cell
struct CoefF32 {
  float dt, H2, nH, Tg, kc, opf, hq, fa, pb, pc, pd;
};
__device__ __forceinline__ CoefF32 coef_f32(const StepCoef& k) {
  CoefF32 f;
  f.dt = (float)k.dt; f.H2 = (float)(2.0 * k.H); f.nH = (float)k.nH; f.Tg = (float)k.Tg; f.kc = (float)k.kc;
  f.opf = (float)(1.0 + k.fHe); f.hq = (float)k.hq; f.fa = (float)k.fa; f.pb = (float)k.pb; f.pc = (float)k.pc;
  f.pd = (float)k.pd;
  return f;
}

struct CellF32 {
  float Tn, al, n, A, s, xf, yf;
};

// Binary32 coefficients; x and y = 1 - x both carried with full relative
// precision (y from the binary64 state).
__device__ __forceinline__ CellF32 cell_f32(const CoefF32& f, int mixing, float d, double x, float T, uint32_t tal,
                                            float wscale) {
  CellF32 c;
  c.xf = __double2float_rn(x);
  c.yf = __double2float_rn(1.0 - x);
  float opx = f.opf + c.xf;
  float g = f.kc * c.xf / opx;
  float hh = f.hq / (d * opx);
  c.Tn = (T + f.dt * (g * f.Tg + hh)) / (1.0f + f.dt * (f.H2 + g));
  float lt = __log2f(c.Tn * 1.0e-4f);
  c.al = f.fa * exp2f(f.pb * lt) / (1.0f + f.pc * exp2f(f.pd * lt));
  c.n = f.nH * d;
  c.A = f.dt * c.al * c.n;
  float w = 1.0f;
  if (mixing == REC_MIX_TALLY && wscale > 0.0f) {
    float n1s_rel = d * c.yf;
    if (n1s_rel > 0.0f) w = (float)tal * wscale / n1s_rel;
  }
  c.s = f.dt * w;
  return c;
}

// Roots in both forms: x' = 2c/(B + sqrt(D)) and y' = 1 - x' = 2(A + y)/(2A + B + sqrt(D)),
// D = B^2 + 4Ac; neither subtracts.
__device__ __forceinline__ void root_f32(float A, float s, float G, float x, float y, float* xr, float* yr,
                                         float* dxdG) {
  float sG = s * G;
  float B = 1.0f + sG;
  float cc = x + sG;
  float sq = sqrtf(B * B + 4.0f * A * cc);
  *xr = 2.0f * cc / (B + sq);
  *yr = 2.0f * (A + y) / (2.0f * A + B + sq);
  if (dxdG) *dxdG = s * (*yr) / (2.0f * A * (*xr) + B);
}

// -------------------------------------------------------------- kernels
// Substep prologue: C from the device sum S1s, Newton start.
__global__ void k_substep_begin(DevScalars* sc, StepCoef k, double n3) {
  if (threadIdx.x != 0) return;
  double n1s_mean = k.nH * sc->S1s / n3;
  double R = k.KR / n1s_mean;
  double C = (k.L2g + R) / (k.beta + k.L2g + R);
  sc->C = C;
  sc->omC = 1.0 - C;
  sc->G0 = C * k.beta * k.ea;
  double guess = sc->lam_state;
  if (sc->lam_prev > 0.0 && sc->lam_state > 0.0) guess = sc->lam_state * (sc->lam_state / sc->lam_prev);
  if (!(guess > 0.0)) guess = 1e-30;
  sc->lam = guess;
  sc->conv = 0;
  sc->passes = 0;
  sc->counter = 0;
  sc->last_step = 0.0;
}

// Newton step on the device scalars (last block, thread 0).
__device__ void newton_update(DevScalars* sc, double S0, double S1, double S2, double tol) {
  double lam = sc->lam;
  double F = S0 - lam * S1;
  double Fp = sc->omC * S2 - S1;
  double step = F / Fp;
  double lnew = lam - step;
  if (!(Fp < 0.0) || !(lnew > 0.0)) lnew = lam * (F > 0.0 ? 2.0 : 0.5);
  double rel = fabs(step) / lam;
  sc->lam = lnew;
  sc->passes += 1;
  sc->last_step = rel;
  // quadratic convergence: a step below tol leaves an error of order tol^2 in lnew
  if (rel <= tol && Fp < 0.0) sc->conv = 1;
  else if (sc->passes >= kNewtonMaxPasses) sc->flags |= 1;
}

template <bool MIXED>
__global__ void __launch_bounds__(NT) k_newton(PassArgs a) {
  DevScalars* sc = a.sc;
  if (ld_flag(&sc->conv)) return;
  const double lam = sc->lam;
  const double G = sc->omC * lam + sc->G0;
  const double tot = (double)sc->tally_total;
  const double S1s = sc->S1s;
  const int64_t stride = (int64_t)gridDim.x * NT;
  double v[3];
  if (!MIXED) {
    v[0] = v[1] = v[2] = 0.0;
    const double* delta = (const double*)a.delta;
    const double* T = (const double*)a.T;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += stride) {
      double d = delta[i], x = a.x[i];
      uint32_t tal = (a.k.mixing == REC_MIX_TALLY) ? a.tally[i] : 0u;
      CellF64 c = cell_f64(a.k, d, x, T[i], tal, tot, S1s);
      double dxdG;
      double xr = root_f64(c.A, c.s, G, x, &dxdG);
      double an2 = c.al * c.n * c.n;
      v[0] += an2 * xr * xr;
      v[1] += c.n * (1.0 - xr);
      v[2] += (2.0 * an2 * xr + lam * c.n) * dxdG;
    }
  } else {
    Kahan32 s0, s1, s2;
    const CoefF32 f = coef_f32(a.k);
    const float Gf = (float)G, lamf = (float)lam;
    const float wscale = tot > 0.0 ? (float)(S1s / tot) : 0.0f;
    const float* delta = (const float*)a.delta;
    const float* T = (const float*)a.T;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += stride) {
      uint32_t tal = (a.k.mixing == REC_MIX_TALLY) ? a.tally[i] : 0u;
      CellF32 c = cell_f32(f, a.k.mixing, delta[i], a.x[i], T[i], tal, wscale);
      float xr, yr, dxdG;
      root_f32(c.A, c.s, Gf, c.xf, c.yf, &xr, &yr, &dxdG);
      float an2 = c.al * c.n * c.n;
      s0.add(an2 * xr * xr);
      s1.add(c.n * yr);
      s2.add((2.0f * an2 * xr + lamf * c.n) * dxdG);
    }
    v[0] = s0.value(); v[1] = s1.value(); v[2] = s2.value();
  }
  block_sum<3, NT>(v);
  if (threadIdx.x == 0) {
    double* p = a.part + (size_t)blockIdx.x * kMaxSums;
    p[0] = v[0]; p[1] = v[1]; p[2] = v[2];
  }
  if (!last_block_done(&sc->counter)) return;
  double S[3];
  combine_partials<3, NT>(a.part, gridDim.x, kMaxSums, S);
  if (threadIdx.x == 0) {
    newton_update(sc, S[0], S[1], S[2], MIXED ? 1e-5 : 1e-8);
    sc->counter = 0;
  }
}

// Final pass: new state at the converged lambda, emission weights, sums.
template <bool MIXED>
__global__ void __launch_bounds__(NT) k_final(PassArgs a, rec_stats* st) {
  DevScalars* sc = a.sc;
  const double lam = sc->lam;
  const double G = sc->omC * lam + sc->G0;
  const double tot = (double)sc->tally_total;
  const double S1s = sc->S1s;
  const int64_t stride = (int64_t)gridDim.x * NT;
  const bool zero_tally = a.k.last != 0;
  double v[3];  // sum delta(1-x'), sum delta x', sum delta
  if (!MIXED) {
    v[0] = v[1] = v[2] = 0.0;
    const double* delta = (const double*)a.delta;
    double* T = (double*)a.T;
    double4* U = (double4*)a.vel4;
    double* emis = (double*)a.emis;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += stride) {
      double d = delta[i], x = a.x[i];
      uint32_t tal = a.tally[i];
      CellF64 c = cell_f64(a.k, d, x, T[i], tal, tot, S1s);
      double xr = root_f64(c.A, c.s, G, x, nullptr);
      double damp = exp(-(a.k.kd * xr + a.k.H) * a.k.dt);
      double4 u = U[i];
      u.x *= damp; u.y *= damp; u.z *= damp;
      U[i] = u;
      a.x[i] = xr;
      T[i] = c.Tn;
      double r = c.al * (c.n * xr) * (c.n * xr);
      emis[i] = r;
      if (zero_tally) a.tally[i] = 0u;
      v[0] += d * (1.0 - xr);
      v[1] += d * xr;
      v[2] += d;
    }
  } else {
    Kahan32 s0, s1, s2;
    const CoefF32 f = coef_f32(a.k);
    const float Gf = (float)G;
    const float wscale = tot > 0.0 ? (float)(S1s / tot) : 0.0f;
    const float* delta = (const float*)a.delta;
    float* T = (float*)a.T;
    float4* U = (float4*)a.vel4;
    float* emis = (float*)a.emis;
    const float kdf = (float)a.k.kd, Hf = (float)a.k.H, dtf = (float)a.k.dt;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += stride) {
      float d = delta[i];
      double x = a.x[i];
      uint32_t tal = a.tally[i];
      CellF32 c = cell_f32(f, a.k.mixing, d, x, T[i], tal, wscale);
      float xr, yr, dxdG;
      root_f32(c.A, c.s, Gf, c.xf, c.yf, &xr, &yr, &dxdG);
      // binary64 state: the binary32 root (x' or 1 - y', whichever is exact),
      // then one Newton correction of the backward-Euler residual
      //   q = (x' - x) + dt (alpha n_H x'^2 - w G (1 - x'))
      // whose rate difference (recombination minus photo-ionisation) is formed
      // in binary64.
      double xn = (yr < 0.5f) ? 1.0 - (double)yr : (double)xr;
      double sG = (double)c.s * G;
      double q = (xn - x) + (double)c.A * xn * xn - sG * (1.0 - xn);
      float Dq = 2.0f * c.A * xr + 1.0f + c.s * Gf;
      xn -= (double)(__double2float_rn(q) / Dq);
      float xnf = __double2float_rn(xn);
      float damp = __expf(-(kdf * xnf + Hf) * dtf);
      float4 u = U[i];
      u.x *= damp; u.y *= damp; u.z *= damp;
      U[i] = u;
      a.x[i] = xn;
      T[i] = c.Tn;
      float ne = c.n * xnf;
      float r = c.al * ne * ne;
      emis[i] = r;
      if (zero_tally) a.tally[i] = 0u;
      s0.add(d * __double2float_rn(1.0 - xn));
      s1.add(d * xnf);
      s2.add(d);
    }
    v[0] = s0.value(); v[1] = s1.value(); v[2] = s2.value();
  }
  block_sum<3, NT>(v);
  if (threadIdx.x == 0) {
    double* p = a.part + (size_t)blockIdx.x * kMaxSums;
    p[0] = v[0]; p[1] = v[1]; p[2] = v[2];
  }
  if (!last_block_done(&sc->counter)) return;
  double S[3];
  combine_partials<3, NT>(a.part, gridDim.x, kMaxSums, S);
  if (threadIdx.x == 0) {
    sc->S1s = S[0];
    sc->Sdx = S[1];
    sc->Sd = S[2];
    sc->lam_prev = sc->lam_state;
    sc->lam_state = lam;
    if (zero_tally) sc->tally_total = 0ull;
    sc->emis_valid = 1;
    sc->counter = 0;
    if (st) {
      st->X_e = S[1] / S[2];
      st->lambda = lam;
      st->C_mix = sc->C;
      st->S1s = S[0];
      st->newton_passes = sc->passes;
      st->flags = sc->flags;
    }
  }
}

// Emission weights and sums of the current state at redshift z (no update);
// also recounts the tallies.
template <bool MIXED>
__global__ void __launch_bounds__(NT) k_refresh(PassArgs a) {
  DevScalars* sc = a.sc;
  const int64_t stride = (int64_t)gridDim.x * NT;
  double v[6];  // S1s, Sdx, Sd, sum alpha n^2 x^2, sum n(1-x), tally count
  for (int k = 0; k < 6; ++k) v[k] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += stride) {
    double d, T;
    if (MIXED) { d = ((const float*)a.delta)[i]; T = ((const float*)a.T)[i]; }
    else { d = ((const double*)a.delta)[i]; T = ((const double*)a.T)[i]; }
    double x = a.x[i];
    double lt = log(T * 1.0e-4);
    double al = a.k.fa * exp(a.k.pb * lt) / (1.0 + a.k.pc * exp(a.k.pd * lt));
    double n = a.k.nH * d;
    double r = al * (n * x) * (n * x);
    if (MIXED) ((float*)a.emis)[i] = (float)r;
    else ((double*)a.emis)[i] = r;
    v[0] += d * (1.0 - x);
    v[1] += d * x;
    v[2] += d;
    v[3] += al * n * n * x * x;
    v[4] += n * (1.0 - x);
    v[5] += (double)a.tally[i];
  }
  block_sum<6, NT>(v);
  if (threadIdx.x == 0) {
    double* p = a.part + (size_t)blockIdx.x * kMaxSums;
    for (int k = 0; k < 6; ++k) p[k] = v[k];
  }
  if (!last_block_done(&sc->counter)) return;
  double S[6];
  combine_partials<6, NT>(a.part, gridDim.x, kMaxSums, S);
  if (threadIdx.x == 0) {
    sc->S1s = S[0];
    sc->Sdx = S[1];
    sc->Sd = S[2];
    sc->lam_state = S[4] > 0.0 ? S[3] / S[4] : 0.0;
    sc->lam_prev = -1.0;
    sc->tally_total = (unsigned long long)(S[5] + 0.5);
    sc->flags = 0;
    sc->emis_valid = 1;
    sc->counter = 0;
  }
}

// x_e from the hydrogen Saha equation and T = T_gamma (initial state).
template <bool MIXED>
__global__ void k_state_init(PassArgs a, double nH_over_S, double Tg) {
  const int64_t stride = (int64_t)gridDim.x * NT;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += stride) {
    double d = MIXED ? (double)((const float*)a.delta)[i] : ((const double*)a.delta)[i];
    // x^2/(1-x) = S/n_H  =>  x = 2/(1 + sqrt(1 + 4 n_H/S))
    a.x[i] = 2.0 / (1.0 + sqrt(1.0 + 4.0 * nH_over_S * d));
    if (MIXED) ((float*)a.T)[i] = (float)Tg;
    else ((double*)a.T)[i] = Tg;
  }
}

PassArgs pass_args(rec_ctx* c, const StepCoef& k) {
  PassArgs a;
  a.n3 = c->n3;
  a.delta = c->box.delta;
  a.vel4 = c->box.vel4;
  a.x = c->box.x_e;
  a.T = c->box.T;
  a.tally = c->box.tally;
  a.emis = c->box.emis;
  a.sc = c->sc;
  a.part = c->part;
  a.k = k;
  a.n3_total = c->n3;
  return a;
}

}  // namespace

void enqueue_newton_passes(rec_ctx* c, DevScalars* sc, const StepCoef& k, const double* x, const double* T,
                           const uint32_t* tally) {
  PassArgs a = pass_args(c, k);
  a.sc = sc;
  a.x = const_cast<double*>(x);
  a.T = const_cast<double*>(T);
  a.tally = const_cast<uint32_t*>(tally);
  k_substep_begin<<<1, 32, 0, c->stream>>>(sc, k, (double)c->n3);
  for (int it = 0; it < kNewtonMaxPasses; ++it) k_newton<false><<<c->grid, NT, 0, c->stream>>>(a);
}

cudaError_t launch_refresh(rec_ctx* c, double z) {
  StepCoef k = step_coef(c->cosmo, c->params, z + 1e-6 * (1.0 + z), z, 0);
  PassArgs a = pass_args(c, k);
  GroupTimer t(c, kTOther, 1);
  if (c->params.precision == REC_PREC_MIXED) k_refresh<true><<<c->grid, NT, 0, c->stream>>>(a);
  else k_refresh<false><<<c->grid, NT, 0, c->stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_state_init(rec_ctx* c, double z) {
  StepCoef k = step_coef(c->cosmo, c->params, z + 1e-6 * (1.0 + z), z, 0);
  PassArgs a = pass_args(c, k);
  double S = saha_S(k.Tg);
  GroupTimer t(c, kTOther, 1);
  if (c->params.precision == REC_PREC_MIXED) k_state_init<true><<<c->grid, NT, 0, c->stream>>>(a, k.nH / S, k.Tg);
  else k_state_init<false><<<c->grid, NT, 0, c->stream>>>(a, k.nH / S, k.Tg);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_refresh(c, z);
}

cudaError_t launch_rec_step(rec_ctx* c, double z_from, double z_to, rec_stats* st) {
  const int ns = c->params.n_sub;
  const bool mixed = c->params.precision == REC_PREC_MIXED;
  double ya = std::log1p(z_from), yb = std::log1p(z_to);
  GroupTimer t(c, kTStep, ns * (kNewtonMaxPasses + 2));
  for (int s = 0; s < ns; ++s) {
    double za = (s == 0) ? z_from : std::expm1(ya - (ya - yb) * (double)s / ns);
    double zb = (s == ns - 1) ? z_to : std::expm1(ya - (ya - yb) * (double)(s + 1) / ns);
    StepCoef k = step_coef(c->cosmo, c->params, za, zb, s == ns - 1);
    PassArgs a = pass_args(c, k);
    k_substep_begin<<<1, 32, 0, c->stream>>>(c->sc, k, (double)c->n3);
    for (int it = 0; it < kNewtonMaxPasses; ++it) {
      if (mixed) k_newton<true><<<c->grid, NT, 0, c->stream>>>(a);
      else k_newton<false><<<c->grid, NT, 0, c->stream>>>(a);
    }
    if (mixed) k_final<true><<<c->grid, NT, 0, c->stream>>>(a, st);
    else k_final<false><<<c->grid, NT, 0, c->stream>>>(a, st);
  }
  return cudaGetLastError();
}

}  // namespace rec
