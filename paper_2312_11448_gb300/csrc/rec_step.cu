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
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "rec_df.cuh"
#include "rec_internal.cuh"
#include "rec_reduce.cuh"

namespace rec {
namespace {

constexpr int NT = kPassThreads;

struct CoefF32 {
  float dt, H2, nH, Tg, kc, opf, hq, fa, pb, pc, pd;
  float kd, H;  // drag coefficient per unit x and H, for the final pass
};
// Binary32 coefficients of a substep, formed once on the host.
__host__ __device__ inline CoefF32 coef_f32(const StepCoef& k) {
  CoefF32 f;
  f.dt = (float)k.dt; f.H2 = (float)(2.0 * k.H); f.nH = (float)k.nH; f.Tg = (float)k.Tg; f.kc = (float)k.kc;
  f.opf = (float)(1.0 + k.fHe); f.hq = (float)k.hq; f.fa = (float)k.fa; f.pb = (float)k.pb; f.pc = (float)k.pc;
  f.pd = (float)k.pd;
  f.kd = (float)k.kd; f.H = (float)k.H;
  return f;
}

struct PassArgs {
  int64_t n3;
  const void* delta;
  void* vel4;
  double* x;
  float2* xy;  // mixed form: binary32 (x, 1 - x) of the state
  void* T;
  uint32_t* tally;
  void* emis;
  DevScalars* sc;
  double* part;
  StepCoef k;
  CoefF32 kf;       // k in binary32 (mixed form)
  const void* div;  // partial mixing: velocity divergence per cell (working precision)
  double fmix;      // partial mixing: share f of the full-mixing rate (0 < f <= 1)
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

struct CellF32 {
  float Tn, al, n, A, s, xf, yf;
};

// Binary32 arithmetic of the mixed form.  The per-cell coefficients only need
// a few ulp (the form's tolerance is 1e-4), so divisions, square roots and
// exponentials use the approximate hardware instructions.
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ float fexp2(float a) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

// Binary32 coefficients; x and y = 1 - x both carried with full relative
// precision (the binary32 cache of the binary64 state).
__device__ __forceinline__ CellF32 cell_f32(const CoefF32& f, int mixing, float d, float2 xy, float T, uint32_t tal,
                                            float wscale) {
  CellF32 c;
  c.xf = xy.x;
  c.yf = xy.y;
  float opx = f.opf + c.xf;
  float inv = fdiv(1.0f, d * opx);  // 1 / (Delta (1 + f_He + x))
  float g = f.kc * c.xf * d * inv;  // x / (1 + f_He + x)
  float hh = f.hq * inv;
  c.Tn = fdiv(T + f.dt * (g * f.Tg + hh), 1.0f + f.dt * (f.H2 + g));
  float lt = __log2f(c.Tn * 1.0e-4f);
  c.al = fdiv(f.fa * fexp2(f.pb * lt), 1.0f + f.pc * fexp2(f.pd * lt));
  c.n = f.nH * d;
  c.A = f.dt * c.al * c.n;
  float w = 1.0f;
  if (mixing == REC_MIX_TALLY && wscale > 0.0f) {
    float n1s_rel = d * c.yf;
    if (n1s_rel > 0.0f) w = fdiv((float)tal * wscale, n1s_rel);
  }
  c.s = f.dt * w;
  return c;
}

// Roots in both forms: x' = 2c/(B + sqrt(D)) and y' = 1 - x' = 2(A + y)/(2A + B + sqrt(D)),
// D = B^2 + 4Ac; neither subtracts.  d x'/dG = s (1 - x') / (2 A x' + B) = s y' / sqrt(D).
// They feed the sums whose difference F = S0 - lambda S1 is the lambda
// equation; in stiff cells (2 A x' + s lambda >> 1, early in recombination)
// its derivative (1 - C) S2 - S1 cancels to a small fraction of S1, so the
// square root and the quotients are correctly rounded.  With d2xdG2:
// d^2 x'/dG^2 = -2 x'_G (A x'_G + s) / sqrt(D) (the quadratic differentiated
// twice), for the Halley step of the mixed form.
__device__ __forceinline__ void root_f32(float A, float s, float G, float x, float y, float* xr, float* yr,
                                         float* dxdG, float* d2xdG2 = nullptr) {
  float sG = s * G;
  float B = 1.0f + sG;
  float cc = x + sG;
  float sq = __fsqrt_rn(B * B + 4.0f * A * cc);
  *xr = __fdiv_rn(2.0f * cc, B + sq);
  *yr = __fdiv_rn(2.0f * (A + y), 2.0f * A + B + sq);
  if (dxdG) *dxdG = __fdiv_rn(s * (*yr), sq);
  if (d2xdG2) *d2xdG2 = __fdiv_rn(-2.0f * (*dxdG) * (A * (*dxdG) + s), sq);
}

// -------------------------------------------------------------- kernels
// Binary32 copies of the iterate for the mixed form's passes (one thread).
__device__ __forceinline__ void set_mixed_scal(DevScalars* sc) {
  const double G = sc->omC * sc->lam + sc->G0;
  const dfloat Gd = df_from_double(G);
  sc->lamf = (float)sc->lam;
  sc->Gf = (float)G;
  sc->Ghi = Gd.hi;
  sc->Glo = Gd.lo;
  sc->wscale = sc->tally_total > 0 ? (float)(sc->S1s / (double)sc->tally_total) : 0.0f;
}

// The same as the mixed form's passes read them: through L2 when other blocks
// of the same launch may have written them.
struct MixedScal {
  float lamf, Gf, wscale;
  dfloat Gd;
};
__device__ __forceinline__ MixedScal mixed_scal(const DevScalars* sc, bool via_l2) {
  MixedScal m;
  if (via_l2) {
    m.lamf = __ldcg(&sc->lamf); m.Gf = __ldcg(&sc->Gf); m.wscale = __ldcg(&sc->wscale);
    m.Gd = dfloat{__ldcg(&sc->Ghi), __ldcg(&sc->Glo)};
  } else {
    m.lamf = sc->lamf; m.Gf = sc->Gf; m.wscale = sc->wscale;
    m.Gd = dfloat{sc->Ghi, sc->Glo};
  }
  return m;
}

// Substep prologue: C from the device sum S1s, Newton start.
__device__ void substep_begin(DevScalars* sc, const StepCoef& k, double n3) {
  double n1s_mean = k.nH * sc->S1s / n3;
  double R = k.KR / n1s_mean;
  double C = (k.L2g + R) / (k.beta + k.L2g + R);
  sc->C = C;
  sc->omC = 1.0 - C;
  sc->G0 = C * k.beta * k.ea;
  double guess = sc->lam_state;
  if (sc->lam_prev > 0.0 && sc->lam_state > 0.0)  // extrapolate the last substep's change (at most 2x)
    guess = sc->lam_state * fmin(2.0, fmax(0.5, sc->lam_state / sc->lam_prev));
  if (!(guess > 0.0)) guess = 1e-30;
  sc->lam = guess;
  set_mixed_scal(sc);
  sc->conv = 0;
  sc->passes = 0;
  sc->counter = 0;
  sc->last_step = 0.0;
}
__global__ void k_substep_begin(DevScalars* sc, StepCoef k, double n3) {
  if (threadIdx.x == 0) substep_begin(sc, k, n3);
}
__global__ void k_substep_begin_batch(const BoxDev* bxs, int B, StepCoef k) {
  for (int b = threadIdx.x; b < B; b += blockDim.x) substep_begin(bxs[b].sc, k, (double)bxs[b].n3);
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
  const double prev = sc->passes > 0 ? sc->last_step : HUGE_VAL;
  sc->lam = lnew;
  set_mixed_scal(sc);
  sc->passes += 1;
  sc->last_step = rel;
  // quadratic convergence: a step below tol leaves an error of order tol^2 in lnew;
  // a small step that no longer shrinks is the rounding floor of F
  if (Fp < 0.0 && (rel <= tol || (rel <= 1e-3 && rel >= 0.5 * prev))) sc->conv = 1;
  else if (sc->passes >= kNewtonMaxPasses) sc->flags |= 1;
}

// Halley step for the mixed form (last block, thread 0): with
// F = S0 - lambda S1, F' = (1 - C) S2 - S1 and F'' = (1 - C)^2 S3 + 2 (1 - C) S4,
// lambda' = lambda - 2 F F' / (2 F'^2 - F F'').  The error after a Halley step
// is of order the cube of the error before it, so a step below 2e-3 of lambda
// leaves an error of order 1e-8, far inside the form's 1e-4 tolerance: one
// evaluation pass usually suffices where the Newton step needs two.
__device__ void halley_update(DevScalars* sc, double S0, double S1, double S2, double S3, double S4) {
  const double lam = sc->lam, om = sc->omC;
  const double F = S0 - lam * S1;
  const double Fp = om * S2 - S1;
  const double Fpp = om * om * S3 + 2.0 * om * S4;
  const double den = 2.0 * Fp * Fp - F * Fpp;
  const double step = (den > 0.0) ? 2.0 * F * Fp / den : F / Fp;
  double lnew = lam - step;
  if (!(Fp < 0.0) || !(lnew > 0.0)) lnew = lam * (F > 0.0 ? 2.0 : 0.5);
  const double rel = fabs(step) / lam;
  sc->lam = lnew;
  set_mixed_scal(sc);
  sc->passes += 1;
  sc->last_step = rel;
  if (Fp < 0.0 && rel <= 2e-3) sc->conv = 1;
  else if (sc->passes >= kNewtonMaxPasses) sc->flags |= 1;
}

// Sums per Newton evaluation: three for the FP64 form (Newton), five for the
// mixed form (Halley).
template <bool MIXED> struct NSums { static constexpr int value = MIXED ? 5 : 3; };

// The update of either form from the combined sums.
template <bool MIXED>
__device__ __forceinline__ void lambda_update(DevScalars* sc, const double (&S)[5]) {
  if (MIXED) halley_update(sc, S[0], S[1], S[2], S[3], S[4]);
  else newton_update(sc, S[0], S[1], S[2], 1e-8);
}

// Local Peebles factor from the substep-start n_1s and H + div v / 3 (no
// escape when the flow converges faster than the expansion).
__device__ __forceinline__ double local_C(const StepCoef& k, double div, double n1s) {
  const double Heff = fmax(k.H + div / 3.0, 0.0);
  if (!(n1s > 0.0)) return 1.0;
  const double R = (k.KR / k.H) * Heff / n1s;
  return (k.L2g + R) / (k.beta + k.L2g + R);
}
__device__ __forceinline__ float local_C_f32(const StepCoef& k, float div, float n1s) {
  const float Heff = fmaxf((float)k.H + div / 3.0f, 0.0f);
  if (!(n1s > 0.0f)) return 1.0f;
  const float R = fdiv((float)(k.KR / k.H) * Heff, n1s);
  return fdiv((float)k.L2g + R, (float)(k.beta + k.L2g) + R);
}

// Per-block partial sums of one Newton evaluation at lambda (result in thread 0):
// v0 = sum alpha n^2 x'^2, v1 = sum n (1 - x'), v2 = sum (2 alpha n^2 x' + lambda n) dx'/dG;
// mixed form also v3 = sum [2 alpha n^2 (dx'/dG)^2 + (2 alpha n^2 x' + lambda n) d2x'/dG2],
// v4 = sum n dx'/dG (the second derivative of F for the Halley step).
// PART: partial mixing — per cell, A scaled by f + (1 - f) C_i, s = dt f and G
// offset by (1 - f)/f C_i beta e_alpha (C_i the local Peebles factor).
template <bool MIXED, bool PART = false>
__device__ __forceinline__ void newton_block_sums(const PassArgs& a, double lam, double G, double tot, double S1s,
                                                  const MixedScal& ms, int blk, int nblk, double (&v)[5]) {
  const int64_t stride = (int64_t)nblk * NT;
  v[3] = v[4] = 0.0;
  if (!MIXED) {
    v[0] = v[1] = v[2] = 0.0;
    const double* delta = (const double*)a.delta;
    const double* T = (const double*)a.T;
    for (int64_t i = (int64_t)blk * NT + threadIdx.x; i < a.n3; i += stride) {
      double d = delta[i], x = a.x[i];
      uint32_t tal = (a.k.mixing == REC_MIX_TALLY) ? a.tally[i] : 0u;
      CellF64 c = cell_f64(a.k, d, x, T[i], tal, tot, S1s);
      double Gc = G;
      if (PART) {
        const double Ci = local_C(a.k, ((const double*)a.div)[i], c.n * (1.0 - x));
        c.A *= a.fmix + (1.0 - a.fmix) * Ci;
        c.s = a.k.dt * a.fmix;
        Gc = G + ((1.0 - a.fmix) / a.fmix) * Ci * (a.k.beta * a.k.ea);
      }
      double dxdG;
      double xr = root_f64(c.A, c.s, Gc, x, &dxdG);
      double an2 = c.al * c.n * c.n;
      v[0] += an2 * xr * xr;
      v[1] += c.n * (1.0 - xr);
      v[2] += (2.0 * an2 * xr + lam * c.n) * dxdG;
    }
  } else {
    Kahan32 acc[5];
    const CoefF32& f = a.kf;
    const float Gf = ms.Gf, lamf = ms.lamf, wscale = ms.wscale;
    const float* delta = (const float*)a.delta;
    const float* T = (const float*)a.T;
    for (int64_t i = (int64_t)blk * NT + threadIdx.x; i < a.n3; i += stride) {
      uint32_t tal = (a.k.mixing == REC_MIX_TALLY) ? a.tally[i] : 0u;
      CellF32 c = cell_f32(f, a.k.mixing, delta[i], a.xy[i], T[i], tal, wscale);
      float Gc = Gf;
      if (PART) {
        const float fm = (float)a.fmix;
        const float Ci = local_C_f32(a.k, ((const float*)a.div)[i], c.n * c.yf);
        c.A *= fm + (1.0f - fm) * Ci;
        c.s = f.dt * fm;
        Gc = Gf + ((1.0f - fm) / fm) * Ci * (float)(a.k.beta * a.k.ea);
      }
      float xr, yr, dxdG, d2;
      root_f32(c.A, c.s, Gc, c.xf, c.yf, &xr, &yr, &dxdG, &d2);
      float an2 = c.al * c.n * c.n;
      const float q = 2.0f * an2 * xr + lamf * c.n;
      acc[0].add(an2 * xr * xr);
      acc[1].add(c.n * yr);
      acc[2].add(q * dxdG);
      acc[3].add(2.0f * an2 * dxdG * dxdG + q * d2);
      acc[4].add(c.n * dxdG);
    }
    block_sum_kahan<5, NT>(acc, v);
    return;
  }
  block_sum_first<NSums<MIXED>::value, NT>(v);
}

// Scalars of the mixed form's final pass at the converged lambda.
struct FinalMixed {
  CoefF32 f;
  float Gf, wscale, kdf, Hf, dtf;
  dfloat Gd;
};
__device__ __forceinline__ FinalMixed final_mixed_setup(const PassArgs& a, const MixedScal& ms) {
  FinalMixed m;
  m.f = a.kf;
  m.Gf = ms.Gf;
  m.wscale = ms.wscale;
  m.kdf = a.kf.kd;
  m.Hf = a.kf.H;
  m.dtf = a.kf.dt;
  m.Gd = ms.Gd;
  return m;
}

// One cell of the mixed form's final pass: x' (binary64 state by its
// increment), its binary32 cache (x', 1 - x'), T', the drag-damped velocity,
// the emission weight and the tally reset, from the cell's inputs d, x, T,
// tally and velocity; adds the cell to the sums of the new state.
template <bool PART>
__device__ __forceinline__ void final_cell_mixed(const PassArgs& a, const FinalMixed& m, bool zero_tally, int64_t i,
                                                 float d, double x, float Tin, uint32_t tal, float4 u,
                                                 Kahan32 (&acc)[3]) {
  const CoefF32& f = m.f;
  // the state and 1 - x as double-float pairs, from the bits of x
  const dfloat X = df_from_double(x);
  const dfloat Y = df_add(dfloat{1.0f, 0.0f}, df_neg(X));
  CellF32 c = cell_f32(f, a.k.mixing, d, make_float2(df_to_float(X), df_to_float(Y)), Tin,
                       (a.k.mixing == REC_MIX_TALLY) ? tal : 0u, m.wscale);
  float Gcf = m.Gf;
  dfloat Gc = m.Gd;
  if (PART) {
    const float fm = (float)a.fmix;
    const float Ci = local_C_f32(a.k, ((const float*)a.div)[i], c.n * c.yf);
    c.A *= fm + (1.0f - fm) * Ci;
    c.s = f.dt * fm;
    const float go = ((1.0f - fm) / fm) * Ci * (float)(a.k.beta * a.k.ea);
    Gcf = m.Gf + go;
    Gc = df_add(m.Gd, dfloat{go, 0.0f});
  }
  // binary32 roots x' and y' = 1 - x' (both without cancellation) and the
  // discriminant D = B^2 + 4 A c
  float sGf = c.s * Gcf;
  float B = 1.0f + sGf;
  float sq = __fsqrt_rn(B * B + 4.0f * c.A * (c.xf + sGf));
  float xr = __fdiv_rn(2.0f * (c.xf + sGf), B + sq);
  float yr = __fdiv_rn(2.0f * (c.A + c.yf), 2.0f * c.A + B + sq);
  // state update by its increment: with x' = x + dx the backward-Euler
  // equation reads A dx^2 + (2Ax + B) dx + r0 = 0, where
  //   r0 = A x^2 - sG (1 - x)
  // is dt times the net rate (recombination minus photo-ionisation) at the old
  // state.  Near Saha equilibrium the two terms cancel, so r0 is formed in
  // double-float arithmetic (about 48 bits) rather than in binary32; the
  // discriminant of this equation is D again.
  const dfloat r0 = df_add(df_mul_f(df_mul(X, X), c.A), df_neg(df_mul(df_mul_f(Gc, c.s), Y)));
  float dx = fdiv(-2.0f * r0.hi, 2.0f * c.A * c.xf + B + sq);
  double xn = add_small(x, dx);  // integer operations unless |dx| > x/4
  float damp = __expf(-(m.kdf * xr + m.Hf) * m.dtf);
  u.x *= damp; u.y *= damp; u.z *= damp;
  ((float4*)a.vel4)[i] = u;
  a.x[i] = xn;
  a.xy[i] = make_float2(xr, yr);
  ((float*)a.T)[i] = c.Tn;
  float ne = c.n * xr;
  ((float*)a.emis)[i] = c.al * ne * ne;
  if (zero_tally) a.tally[i] = 0u;
  acc[0].add(d * yr);
  acc[1].add(d * xr);
  acc[2].add(d);
}

// Per-block final update at the converged lambda: writes x, T, U, emission
// weights (zeroes the tallies on the last substep); partial sums (thread 0):
// v0 = sum delta (1 - x'), v1 = sum delta x', v2 = sum delta.
template <bool MIXED, bool PART = false>
__device__ __forceinline__ void final_block(const PassArgs& a, double G, double tot, double S1s, const MixedScal& ms,
                                            int blk, int nblk, double (&v)[3]) {
  const int64_t stride = (int64_t)nblk * NT;
  const bool zero_tally = a.k.last != 0;
  if (!MIXED) {
    v[0] = v[1] = v[2] = 0.0;
    const double* delta = (const double*)a.delta;
    double* T = (double*)a.T;
    double4_32a* U = (double4_32a*)a.vel4;
    double* emis = (double*)a.emis;
    for (int64_t i = (int64_t)blk * NT + threadIdx.x; i < a.n3; i += stride) {
      double d = delta[i], x = a.x[i];
      uint32_t tal = (a.k.mixing == REC_MIX_TALLY) ? a.tally[i] : 0u;
      CellF64 c = cell_f64(a.k, d, x, T[i], tal, tot, S1s);
      double Gc = G;
      if (PART) {
        const double Ci = local_C(a.k, ((const double*)a.div)[i], c.n * (1.0 - x));
        c.A *= a.fmix + (1.0 - a.fmix) * Ci;
        c.s = a.k.dt * a.fmix;
        Gc = G + ((1.0 - a.fmix) / a.fmix) * Ci * (a.k.beta * a.k.ea);
      }
      double xr = root_f64(c.A, c.s, Gc, x, nullptr);
      double damp = exp(-(a.k.kd * xr + a.k.H) * a.k.dt);
      double4_32a u = U[i];
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
    Kahan32 acc[3];
    const FinalMixed fm = final_mixed_setup(a, ms);
    const float* delta = (const float*)a.delta;
    const float* T = (const float*)a.T;
    const float4* U = (const float4*)a.vel4;
    for (int64_t i = (int64_t)blk * NT + threadIdx.x; i < a.n3; i += stride) {
      const uint32_t tal = (a.k.mixing == REC_MIX_TALLY) ? a.tally[i] : 0u;
      final_cell_mixed<PART>(a, fm, zero_tally, i, delta[i], a.x[i], T[i], tal, U[i], acc);
    }
    block_sum_kahan<3, NT>(acc, v);
    return;
  }
  block_sum<3, NT>(v);
}

// End-of-substep bookkeeping on the device scalars (one thread).
__device__ __forceinline__ void finish_substep(DevScalars* sc, const StepCoef& k, const double (&S)[3], double lam,
                                               rec_stats* st) {
  sc->S1s = S[0];
  sc->Sdx = S[1];
  sc->Sd = S[2];
  sc->lam_prev = sc->lam_state;
  sc->lam_state = lam;
  if (k.last) sc->tally_total = 0ull;
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

// Batched contexts (MB): the grid is the concatenation of every box's pass
// blocks; a block works on its box's cells with the box's own block count, and
// the last block of a box reduces that box's partials.  Single box: the whole grid.
// g: the block's index in the concatenated grid (blockIdx.x, or a virtual
// block of a persistent launch).
__device__ __forceinline__ void pass_view(PassArgs& a, const BoxDev* bxs, int B, int* blk, int* nblk, int* box,
                                          uint32_t g) {
  int lo = 0, hi = B;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (bxs[mid].pblk0 <= g) lo = mid;
    else hi = mid;
  }
  const BoxDev& d = bxs[lo];
  a.n3 = d.n3;
  a.delta = d.delta;
  a.vel4 = d.vel4;
  a.x = d.x;
  a.xy = (float2*)d.xy;
  a.T = d.T;
  a.tally = d.tally;
  a.emis = d.emis;
  a.sc = d.sc;
  a.part += (size_t)d.pblk0 * kMaxSums;
  *blk = (int)(g - d.pblk0);
  *nblk = (int)d.pblk;
  *box = lo;
}

template <bool MIXED, bool MB>
__global__ void __launch_bounds__(NT) k_newton(PassArgs a, const BoxDev* bxs, int B) {
  int blk = blockIdx.x, nblk = gridDim.x, box = 0;
  if (MB) pass_view(a, bxs, B, &blk, &nblk, &box, blockIdx.x);
  DevScalars* sc = a.sc;
  if (ld_flag(&sc->conv)) return;
  const double lam = sc->lam;
  constexpr int K = NSums<MIXED>::value;
  double v[5];
  newton_block_sums<MIXED>(a, lam, sc->omC * lam + sc->G0, (double)sc->tally_total, sc->S1s, mixed_scal(sc, false), blk,
                           nblk, v);
  if (threadIdx.x == 0) {
    double* p = a.part + (size_t)blk * kMaxSums;
    for (int j = 0; j < K; ++j) p[j] = v[j];
  }
  if (!last_block_done(&sc->counter, nblk)) return;
  double S[5];
  combine_partials_first<K, NT>(a.part, nblk, kMaxSums, S);
  if (threadIdx.x == 0) {
    lambda_update<MIXED>(sc, S);
    sc->counter = 0;
  }
}

// ---- Newton evaluation of the mixed form with TMA-staged tiles ----------------
// Persistent CTAs stream tiles of kTmaTile cells of the four per-cell inputs
// (Delta, the (x, 1 - x) cache, T, tallies) into a ring of kTmaStages shared-memory
// stages with bulk asynchronous copies (cp.async.bulk, completion counted in bytes
// on one mbarrier per stage); thread 0 keeps kTmaStages - 1 tiles in flight while
// the CTA evaluates the current one, so no warp waits on a global load.  Cells
// past the last whole tile are read directly.  Every wait on a stage barrier
// is bounded: past kTmaWaitLimit polls the CTA records bit 3 in the flags,
// waits (bounded) for the copies it issued and leaves without its partial sums.
constexpr int kTmaTile = 1024;
constexpr int kTmaStages = 3;
constexpr int kTmaThreads = 256;
constexpr uint32_t kTmaWaitLimit = 1u << 22;
constexpr int kTmaCtasPerSm = 3;  // resident CTAs per SM (shared-memory ring of each)

struct TmaStage {
  float delta[kTmaTile];
  float2 xy[kTmaTile];
  float T[kTmaTile];
  uint32_t tally[kTmaTile];
};
constexpr uint32_t kTmaStageBytes = kTmaTile * (4 + 8 + 4 + 4);
constexpr size_t kTmaSmem = sizeof(TmaStage) * kTmaStages + 8 * kTmaStages;
static_assert(sizeof(TmaStage) == kTmaStageBytes, "stage layout");

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for a stage: a non-blocking look, then at most `limit` blocking polls.
// limit 0 gives up without looking (the error path, for tests).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, uint32_t parity, uint32_t limit) {
  if (limit == 0) return false;
  if (mbar_test_wait(b, parity)) return true;
  for (uint32_t polls = 0; polls < limit; ++polls)
    if (mbar_try_wait(b, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(b))
               : "memory");
}

__global__ void __launch_bounds__(kTmaThreads) k_newton_tma(PassArgs a, uint32_t limit) {
  DevScalars* sc = a.sc;
  if (ld_flag(&sc->conv)) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TmaStage* stage = reinterpret_cast<TmaStage*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + sizeof(TmaStage) * kTmaStages);
  const MixedScal ms = mixed_scal(sc, false);
  const int64_t n_tiles = a.n3 / kTmaTile;  // whole tiles, copied in bulk
  const int64_t my_tiles = n_tiles > (int64_t)blockIdx.x ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const float* delta = (const float*)a.delta;
  const float* Tg = (const float*)a.T;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTmaStages; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int64_t it) {  // thread 0: tile `it` of this CTA into its stage
    const int s = (int)(it % kTmaStages);
    const int64_t c0 = ((int64_t)blockIdx.x + it * gridDim.x) * kTmaTile;
    mbar_expect_tx(&full[s], kTmaStageBytes);
    bulk_load(stage[s].delta, delta + c0, kTmaTile * 4, &full[s]);
    bulk_load(stage[s].xy, a.xy + c0, kTmaTile * 8, &full[s]);
    bulk_load(stage[s].T, Tg + c0, kTmaTile * 4, &full[s]);
    bulk_load(stage[s].tally, a.tally + c0, kTmaTile * 4, &full[s]);
  };
  if (threadIdx.x == 0)
    for (int64_t it = 0; it < my_tiles && it < kTmaStages - 1; ++it) issue(it);
  Kahan32 acc[5];
  const CoefF32& f = a.kf;
  const float Gf = ms.Gf, lamf = ms.lamf, wscale = ms.wscale;
  auto cell = [&](float d, float2 xy, float T, uint32_t tal) {
    CellF32 c = cell_f32(f, a.k.mixing, d, xy, T, (a.k.mixing == REC_MIX_TALLY) ? tal : 0u, wscale);
    float xr, yr, dxdG, d2;
    root_f32(c.A, c.s, Gf, c.xf, c.yf, &xr, &yr, &dxdG, &d2);
    float an2 = c.al * c.n * c.n;
    const float q = 2.0f * an2 * xr + lamf * c.n;
    acc[0].add(an2 * xr * xr);
    acc[1].add(c.n * yr);
    acc[2].add(q * dxdG);
    acc[3].add(2.0f * an2 * dxdG * dxdG + q * d2);
    acc[4].add(c.n * dxdG);
  };
  bool timed_out = false;
  int64_t it = 0;
  for (; it < my_tiles; ++it) {
    if (threadIdx.x == 0 && it + kTmaStages - 1 < my_tiles) {
      // the stage refilled here was read by every thread before the barrier that ended the last iteration
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(it + kTmaStages - 1);
    }
    const int s = (int)(it % kTmaStages);
    const uint32_t parity = (uint32_t)((it / kTmaStages) & 1);
    if (!mbar_wait_bounded(&full[s], parity, limit)) timed_out = true;
    if (!timed_out) {
      const TmaStage& t = stage[s];
      for (int k = threadIdx.x; k < kTmaTile; k += kTmaThreads) cell(t.delta[k], t.xy[k], t.T[k], t.tally[k]);
    }
    if (__syncthreads_or(timed_out)) { timed_out = true; break; }
  }
  if (timed_out) {
    if (threadIdx.x == 0) {
      atomicOr(&sc->flags, 8);
      // the copies issued for the tiles it .. it + kTmaStages - 2 may still be in flight
      for (int64_t j = it; j < my_tiles && j < it + kTmaStages - 1; ++j) {
        uint32_t polls = 0;
        while (!mbar_try_wait(&full[j % kTmaStages], (uint32_t)((j / kTmaStages) & 1)) && ++polls < kTmaWaitLimit) {
        }
      }
    }
    __syncthreads();
    return;
  }
  // cells after the last whole tile
  for (int64_t i = n_tiles * kTmaTile + (int64_t)blockIdx.x * kTmaThreads + threadIdx.x; i < a.n3;
       i += (int64_t)gridDim.x * kTmaThreads)
    cell(delta[i], a.xy[i], Tg[i], a.tally[i]);
  double v[5];
  block_sum_kahan<5, kTmaThreads>(acc, v);
  if (threadIdx.x == 0) {
    double* p = a.part + (size_t)blockIdx.x * kMaxSums;
    for (int j = 0; j < 5; ++j) p[j] = v[j];
  }
  if (!last_block_done(&sc->counter)) return;
  double S[5];
  combine_partials<5, kTmaThreads>(a.part, gridDim.x, kMaxSums, S);
  if (threadIdx.x == 0) {
    halley_update(sc, S[0], S[1], S[2], S[3], S[4]);
    sc->counter = 0;
  }
}

// Final pass: new state at the converged lambda, emission weights, sums.
// st: statistics record (one per box in a batch) or NULL.
template <bool MIXED, bool MB>
__global__ void __launch_bounds__(NT) k_final(PassArgs a, rec_stats* st, const BoxDev* bxs, int B) {
  int blk = blockIdx.x, nblk = gridDim.x, box = 0;
  if (MB) pass_view(a, bxs, B, &blk, &nblk, &box, blockIdx.x);
  DevScalars* sc = a.sc;
  const double lam = sc->lam;
  double v[3];
  final_block<MIXED>(a, sc->omC * lam + sc->G0, (double)sc->tally_total, sc->S1s, mixed_scal(sc, false), blk, nblk, v);
  if (threadIdx.x == 0) {
    double* p = a.part + (size_t)blk * kMaxSums;
    p[0] = v[0]; p[1] = v[1]; p[2] = v[2];
  }
  if (!last_block_done(&sc->counter, nblk)) return;
  double S[3];
  combine_partials<3, NT>(a.part, nblk, kMaxSums, S);
  if (threadIdx.x == 0) finish_substep(sc, a.k, S, lam, st ? st + box : nullptr);
}

// ---- batched substep as one persistent launch ------------------------------------
// A whole substep of a batched context in one cooperative launch: the Newton
// prologue of every box, then Newton evaluations (each box's pass blocks run
// as virtual blocks of the resident grid; the last virtual block of a box
// takes its Newton step) separated by bounded grid barriers until every box
// has converged, then the final pass.  Scalars that other blocks update within
// the launch are read through L2 (ld.cg).  A barrier that gives up ends the
// launch (flags bit 3 of the batch record; rec_sync reports it).
template <bool MIXED>
__global__ void __launch_bounds__(NT) k_batch_substep(PassArgs a0, rec_stats* st, const BoxDev* bxs, int B, int nvb,
                                                      DevScalars* gsc, uint32_t limit) {
  if (blockIdx.x == 0)
    for (int b = threadIdx.x; b < B; b += NT) substep_begin(bxs[b].sc, a0.k, (double)bxs[b].n3);
  if (!grid_barrier(&gsc->bar, &gsc->flags, limit)) return;
  for (int pass = 0; pass < kNewtonMaxPasses; ++pass) {
    for (int g = blockIdx.x; g < nvb; g += gridDim.x) {
      PassArgs a = a0;
      int blk, nblk, box;
      pass_view(a, bxs, B, &blk, &nblk, &box, (uint32_t)g);
      DevScalars* sc = a.sc;
      if (__ldcg(&sc->conv)) continue;  // the same for the whole block
      const double lam = __ldcg(&sc->lam);
      constexpr int K = NSums<MIXED>::value;
      double v[5];
      newton_block_sums<MIXED>(a, lam, __ldcg(&sc->omC) * lam + __ldcg(&sc->G0), (double)__ldcg(&sc->tally_total),
                               __ldcg(&sc->S1s), mixed_scal(sc, true), blk, nblk, v);
      if (threadIdx.x == 0) {
        double* p = a.part + (size_t)blk * kMaxSums;
        for (int j = 0; j < K; ++j) p[j] = v[j];
      }
      if (!last_block_done(&sc->counter, nblk)) continue;
      double S[5];
      combine_partials_first<K, NT>(a.part, nblk, kMaxSums, S);
      if (threadIdx.x == 0) {
        lambda_update<MIXED>(sc, S);
        sc->counter = 0;
      }
    }
    if (!grid_barrier(&gsc->bar, &gsc->flags, limit)) return;
    int open = 0;
    for (int b = threadIdx.x; b < B; b += NT) open |= __ldcg(&bxs[b].sc->conv) == 0;
    if (!__syncthreads_or(open)) break;
  }
  for (int g = blockIdx.x; g < nvb; g += gridDim.x) {
    PassArgs a = a0;
    int blk, nblk, box;
    pass_view(a, bxs, B, &blk, &nblk, &box, (uint32_t)g);
    DevScalars* sc = a.sc;
    const double lam = __ldcg(&sc->lam);
    double v[3];
    final_block<MIXED>(a, __ldcg(&sc->omC) * lam + __ldcg(&sc->G0), (double)__ldcg(&sc->tally_total), __ldcg(&sc->S1s),
                       mixed_scal(sc, true), blk, nblk, v);
    if (threadIdx.x == 0) {
      double* p = a.part + (size_t)blk * kMaxSums;
      p[0] = v[0]; p[1] = v[1]; p[2] = v[2];
    }
    if (!last_block_done(&sc->counter, nblk)) continue;
    double S[3];
    combine_partials<3, NT>(a.part, nblk, kMaxSums, S);
    if (threadIdx.x == 0) finish_substep(sc, a.k, S, lam, st ? st + box : nullptr);
  }
}

// ---- final pass of the mixed form with TMA-staged tiles ----------------------------
// The final pass streams five inputs per cell (Delta, x, T, tallies, velocity;
// 36 B) and writes six outputs.  As in the Newton evaluation, persistent CTAs
// bring tiles of kTmaTile cells of the inputs into a ring of shared-memory
// stages with bulk asynchronous copies, so that the loads are in flight while
// the previous tile is computed; the outputs are stored directly.  Waits are
// bounded as in k_newton_tma.
constexpr int kFinStages = 2;
constexpr int kFinCtasPerSm = 3;
struct FinStage {
  float delta[kTmaTile];
  double x[kTmaTile];
  float T[kTmaTile];
  uint32_t tally[kTmaTile];
  float4 U[kTmaTile];
};
constexpr size_t kFinSmem = sizeof(FinStage) * kFinStages + 8 * kFinStages;

__global__ void __launch_bounds__(kTmaThreads, kFinCtasPerSm) k_final_tma(PassArgs a, rec_stats* st, uint32_t limit) {
  DevScalars* sc = a.sc;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  FinStage* stage = reinterpret_cast<FinStage*>(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + sizeof(FinStage) * kFinStages);
  const double lam = sc->lam;
  const FinalMixed fm = final_mixed_setup(a, mixed_scal(sc, false));
  const bool zero_tally = a.k.last != 0;
  const bool tally_mode = a.k.mixing == REC_MIX_TALLY;
  const uint32_t stage_bytes = kTmaTile * (4 + 8 + 4 + 16) + (tally_mode ? kTmaTile * 4 : 0);
  const int64_t n_tiles = a.n3 / kTmaTile;
  const int64_t my_tiles = n_tiles > (int64_t)blockIdx.x ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const float* delta = (const float*)a.delta;
  const float* Tg = (const float*)a.T;
  const float4* Ug = (const float4*)a.vel4;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kFinStages; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int64_t it) {  // thread 0: tile `it` of this CTA into its stage
    const int s = (int)(it % kFinStages);
    const int64_t c0 = ((int64_t)blockIdx.x + it * gridDim.x) * kTmaTile;
    mbar_expect_tx(&full[s], stage_bytes);
    bulk_load(stage[s].delta, delta + c0, kTmaTile * 4, &full[s]);
    bulk_load(stage[s].x, a.x + c0, kTmaTile * 8, &full[s]);
    bulk_load(stage[s].T, Tg + c0, kTmaTile * 4, &full[s]);
    if (tally_mode) bulk_load(stage[s].tally, a.tally + c0, kTmaTile * 4, &full[s]);
    bulk_load(stage[s].U, Ug + c0, kTmaTile * 16, &full[s]);
  };
  if (threadIdx.x == 0)
    for (int64_t it = 0; it < my_tiles && it < kFinStages - 1; ++it) issue(it);
  Kahan32 acc[3];
  bool timed_out = false;
  int64_t it = 0;
  for (; it < my_tiles; ++it) {
    if (threadIdx.x == 0 && it + kFinStages - 1 < my_tiles) {
      // the stage refilled here was read by every thread before the barrier that ended the last iteration
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(it + kFinStages - 1);
    }
    const int s = (int)(it % kFinStages);
    const uint32_t parity = (uint32_t)((it / kFinStages) & 1);
    if (!mbar_wait_bounded(&full[s], parity, limit)) timed_out = true;
    if (!timed_out) {
      const FinStage& t = stage[s];
      const int64_t c0 = ((int64_t)blockIdx.x + it * gridDim.x) * kTmaTile;
      for (int k = threadIdx.x; k < kTmaTile; k += kTmaThreads)
        final_cell_mixed<false>(a, fm, zero_tally, c0 + k, t.delta[k], t.x[k], t.T[k], tally_mode ? t.tally[k] : 0u,
                                t.U[k], acc);
    }
    if (__syncthreads_or(timed_out)) { timed_out = true; break; }
  }
  if (timed_out) {
    if (threadIdx.x == 0) {
      atomicOr(&sc->flags, 8);
      // the copies issued for the tiles it .. it + kFinStages - 2 may still be in flight
      for (int64_t j = it; j < my_tiles && j < it + kFinStages - 1; ++j) {
        uint32_t polls = 0;
        while (!mbar_try_wait(&full[j % kFinStages], (uint32_t)((j / kFinStages) & 1)) && ++polls < kTmaWaitLimit) {
        }
      }
    }
    __syncthreads();
    return;
  }
  // cells after the last whole tile
  for (int64_t i = n_tiles * kTmaTile + (int64_t)blockIdx.x * kTmaThreads + threadIdx.x; i < a.n3;
       i += (int64_t)gridDim.x * kTmaThreads)
    final_cell_mixed<false>(a, fm, zero_tally, i, delta[i], a.x[i], Tg[i], tally_mode ? a.tally[i] : 0u, Ug[i], acc);
  double v[3];
  block_sum_kahan<3, kTmaThreads>(acc, v);
  if (threadIdx.x == 0) {
    double* p = a.part + (size_t)blockIdx.x * kMaxSums;
    p[0] = v[0]; p[1] = v[1]; p[2] = v[2];
  }
  if (!last_block_done(&sc->counter)) return;
  double S[3];
  combine_partials<3, kTmaThreads>(a.part, gridDim.x, kMaxSums, S);
  if (threadIdx.x == 0) finish_substep(sc, a.k, S, lam, st);
}

// Newton evaluation and final pass of partial mixing (single-box contexts).
template <bool MIXED>
__global__ void __launch_bounds__(NT) k_newton_part(PassArgs a) {
  DevScalars* sc = a.sc;
  if (ld_flag(&sc->conv)) return;
  const double lam = sc->lam;
  constexpr int K = NSums<MIXED>::value;
  double v[5];
  newton_block_sums<MIXED, true>(a, lam, sc->omC * lam + sc->G0, 0.0, sc->S1s, mixed_scal(sc, false), blockIdx.x,
                                 gridDim.x, v);
  if (threadIdx.x == 0) {
    double* p = a.part + (size_t)blockIdx.x * kMaxSums;
    for (int j = 0; j < K; ++j) p[j] = v[j];
  }
  if (!last_block_done(&sc->counter)) return;
  double S[5];
  combine_partials_first<K, NT>(a.part, gridDim.x, kMaxSums, S);
  if (threadIdx.x == 0) {
    lambda_update<MIXED>(sc, S);
    sc->counter = 0;
  }
}

template <bool MIXED>
__global__ void __launch_bounds__(NT) k_final_part(PassArgs a, rec_stats* st) {
  DevScalars* sc = a.sc;
  const double lam = sc->lam;
  double v[3];
  final_block<MIXED, true>(a, sc->omC * lam + sc->G0, 0.0, sc->S1s, mixed_scal(sc, false), blockIdx.x, gridDim.x, v);
  if (threadIdx.x == 0) {
    double* p = a.part + (size_t)blockIdx.x * kMaxSums;
    p[0] = v[0]; p[1] = v[1]; p[2] = v[2];
  }
  if (!last_block_done(&sc->counter)) return;
  double S[3];
  combine_partials<3, NT>(a.part, gridDim.x, kMaxSums, S);
  if (threadIdx.x == 0) finish_substep(sc, a.k, S, lam, st);
}

// ---------------------------------------------------------- no-mixing limit
// Sec. III.A.2: recombination local to each cell, Eq. (rec) with the cell's own
// n_e, n_1s and Eq. (R-alpha) at H + div v / 3.  k_divergence takes the
// physical divergence of the substep-start velocities (periodic central
// differences, fac = (1 + z) 1e3 / (2 h) with U in km/s and the comoving cell
// side h in m); k_local then updates every cell on its own (no global lambda).
template <bool MIXED>
__global__ void __launch_bounds__(NT) k_divergence(const void* vel4, int n, double fac, void* div) {
  const int64_t n3 = (int64_t)n * n * n;
  const int64_t stride = (int64_t)gridDim.x * NT;
  for (int64_t c = (int64_t)blockIdx.x * NT + threadIdx.x; c < n3; c += stride) {
    const int ix = (int)(c % n), iy = (int)((c / n) % n), iz = (int)(c / ((int64_t)n * n));
    const int xp = ix + 1 == n ? 0 : ix + 1, xm = ix == 0 ? n - 1 : ix - 1;
    const int yp = iy + 1 == n ? 0 : iy + 1, ym = iy == 0 ? n - 1 : iy - 1;
    const int zp = iz + 1 == n ? 0 : iz + 1, zm = iz == 0 ? n - 1 : iz - 1;
    const int64_t nn = (int64_t)n * n, row = (int64_t)iz * nn + (int64_t)iy * n;
    const int64_t cxp = row + xp, cxm = row + xm;
    const int64_t cyp = (int64_t)iz * nn + (int64_t)yp * n + ix, cym = (int64_t)iz * nn + (int64_t)ym * n + ix;
    const int64_t czp = (int64_t)zp * nn + (int64_t)iy * n + ix, czm = (int64_t)zm * nn + (int64_t)iy * n + ix;
    if (MIXED) {
      const float4* U = (const float4*)vel4;
      const float d = (U[cxp].x - U[cxm].x) + (U[cyp].y - U[cym].y) + (U[czp].z - U[czm].z);
      ((float*)div)[c] = (float)fac * d;
    } else {
      const double4_32a* U = (const double4_32a*)vel4;
      const double d = (U[cxp].x - U[cxm].x) + (U[cyp].y - U[cym].y) + (U[czp].z - U[czm].z);
      ((double*)div)[c] = fac * d;
    }
  }
}

// One local substep over all cells: x, T (and the (x, 1 - x) cache), Compton
// drag, emission weights, tally reset on the last substep; sums for the
// statistics (X_e, lambda of the end state, mean C).
template <bool MIXED>
__global__ void __launch_bounds__(NT) k_local(PassArgs a, const void* div, rec_stats* st) {
  DevScalars* sc = a.sc;
  const StepCoef& k = a.k;
  const int64_t stride = (int64_t)gridDim.x * NT;
  const bool zero_tally = k.last != 0;
  const double bea = k.beta * k.ea;
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // S1s, Sdx, Sd, sum alpha n^2 x^2, sum n (1-x), sum C
  if (!MIXED) {
    const double* delta = (const double*)a.delta;
    double* T = (double*)a.T;
    double4_32a* U = (double4_32a*)a.vel4;
    double* emis = (double*)a.emis;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += stride) {
      const double d = delta[i], x = a.x[i];
      CellF64 c = cell_f64(k, d, x, T[i], 0u, 0.0, 0.0);
      const double Ci = local_C(k, ((const double*)div)[i], c.n * (1.0 - x));
      // dx/dt = -C (alpha n_H x^2 - beta e_alpha (1 - x)), backward Euler
      const double xr = root_f64(c.A * Ci, c.s * Ci, bea, x, nullptr);
      const double damp = exp(-(k.kd * xr + k.H) * k.dt);
      double4_32a u = U[i];
      u.x *= damp; u.y *= damp; u.z *= damp;
      U[i] = u;
      a.x[i] = xr;
      T[i] = c.Tn;
      emis[i] = c.al * (c.n * xr) * (c.n * xr);
      if (zero_tally) a.tally[i] = 0u;
      v[0] += d * (1.0 - xr);
      v[1] += d * xr;
      v[2] += d;
      v[3] += c.al * c.n * c.n * xr * xr;
      v[4] += c.n * (1.0 - xr);
      v[5] += Ci;
    }
  } else {
    Kahan32 s0, s1, s2, s3, s4, s5;
    const CoefF32 f = coef_f32(k);
    const float* delta = (const float*)a.delta;
    float* T = (float*)a.T;
    float4* U = (float4*)a.vel4;
    float* emis = (float*)a.emis;
    const float kdf = (float)k.kd, Hf = (float)k.H, dtf = (float)k.dt, beaf = (float)bea;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += stride) {
      const float d = delta[i];
      const double x = a.x[i];
      CellF32 c = cell_f32(f, REC_MIX_FULL, d, a.xy[i], T[i], 0u, 0.0f);
      const float Ci = local_C_f32(k, ((const float*)div)[i], c.n * c.yf);
      const float A = c.A * Ci, sG = c.s * Ci * beaf;
      // binary32 roots and the binary64 increment of the state, as in k_final
      const float B = 1.0f + sG;
      const float sq = __fsqrt_rn(B * B + 4.0f * A * (c.xf + sG));
      const float xr = __fdiv_rn(2.0f * (c.xf + sG), B + sq);
      const float yr = __fdiv_rn(2.0f * (A + c.yf), 2.0f * A + B + sq);
      const double y = 1.0 - x;
      const double r0 = fma((double)A, x * x, -(double)sG * y);
      const float dx = fdiv(-2.0f * __double2float_rn(r0), 2.0f * A * c.xf + B + sq);
      const float damp = __expf(-(kdf * xr + Hf) * dtf);
      float4 u = U[i];
      u.x *= damp; u.y *= damp; u.z *= damp;
      U[i] = u;
      a.x[i] = x + (double)dx;
      a.xy[i] = make_float2(xr, yr);
      T[i] = c.Tn;
      const float ne = c.n * xr;
      emis[i] = c.al * ne * ne;
      if (zero_tally) a.tally[i] = 0u;
      s0.add(d * yr);
      s1.add(d * xr);
      s2.add(d);
      s3.add(c.al * ne * ne);
      s4.add(c.n * yr);
      s5.add(Ci);
    }
    v[0] = s0.value(); v[1] = s1.value(); v[2] = s2.value(); v[3] = s3.value(); v[4] = s4.value(); v[5] = s5.value();
  }
  block_sum<6, NT>(v);
  if (threadIdx.x == 0) {
    double* p = a.part + (size_t)blockIdx.x * kMaxSums;
    for (int j = 0; j < 6; ++j) p[j] = v[j];
  }
  if (!last_block_done(&sc->counter)) return;
  double S[6];
  combine_partials<6, NT>(a.part, gridDim.x, kMaxSums, S);
  if (threadIdx.x == 0) {
    const double lam = S[4] > 0.0 ? S[3] / S[4] : 0.0;
    sc->C = S[5] / (double)a.n3;
    sc->passes = 0;
    const double S3[3] = {S[0], S[1], S[2]};
    finish_substep(sc, k, S3, lam, st);
  }
}

// Emission weights and sums of the current state at redshift z (no update);
// also recounts the tallies.
template <bool MIXED, bool MB>
__global__ void __launch_bounds__(NT) k_refresh(PassArgs a, const BoxDev* bxs, int B) {
  int blk = blockIdx.x, nblk = gridDim.x, box = 0;
  if (MB) pass_view(a, bxs, B, &blk, &nblk, &box, blockIdx.x);
  DevScalars* sc = a.sc;
  const int64_t stride = (int64_t)nblk * NT;
  double v[6];  // S1s, Sdx, Sd, sum alpha n^2 x^2, sum n(1-x), tally count
  for (int k = 0; k < 6; ++k) v[k] = 0.0;
  for (int64_t i = (int64_t)blk * NT + threadIdx.x; i < a.n3; i += stride) {
    double d, T;
    if (MIXED) { d = ((const float*)a.delta)[i]; T = ((const float*)a.T)[i]; }
    else { d = ((const double*)a.delta)[i]; T = ((const double*)a.T)[i]; }
    double x = a.x[i];
    double lt = log(T * 1.0e-4);
    double al = a.k.fa * exp(a.k.pb * lt) / (1.0 + a.k.pc * exp(a.k.pd * lt));
    double n = a.k.nH * d;
    double r = al * (n * x) * (n * x);
    if (MIXED) {
      ((float*)a.emis)[i] = (float)r;
      a.xy[i] = make_float2(__double2float_rn(x), __double2float_rn(1.0 - x));
    } else {
      ((double*)a.emis)[i] = r;
    }
    v[0] += d * (1.0 - x);
    v[1] += d * x;
    v[2] += d;
    v[3] += al * n * n * x * x;
    v[4] += n * (1.0 - x);
    v[5] += (double)a.tally[i];
  }
  block_sum<6, NT>(v);
  if (threadIdx.x == 0) {
    double* p = a.part + (size_t)blk * kMaxSums;
    for (int k = 0; k < 6; ++k) p[k] = v[k];
  }
  if (!last_block_done(&sc->counter, nblk)) return;
  double S[6];
  combine_partials<6, NT>(a.part, nblk, kMaxSums, S);
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
template <bool MIXED, bool MB>
__global__ void k_state_init(PassArgs a, double nH_over_S, double Tg, const BoxDev* bxs, int B) {
  int blk = blockIdx.x, nblk = gridDim.x, box = 0;
  if (MB) pass_view(a, bxs, B, &blk, &nblk, &box, blockIdx.x);
  const int64_t stride = (int64_t)nblk * NT;
  for (int64_t i = (int64_t)blk * NT + threadIdx.x; i < a.n3; i += stride) {
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
  a.xy = (float2*)c->xy;
  a.T = c->box.T;
  a.tally = c->box.tally;
  a.emis = c->box.emis;
  a.sc = c->sc;
  a.part = c->part;
  a.k = k;
  a.kf = coef_f32(k);
  a.div = c->div;
  a.fmix = c->params.f_alpha;
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
  for (int it = 0; it < kNewtonMaxPasses; ++it) k_newton<false, false><<<c->grid, NT, 0, c->stream>>>(a, nullptr, 1);
}

cudaError_t launch_refresh(rec_ctx* c, double z) {
  StepCoef k = step_coef(c->cosmo, c->params, z + 1e-6 * (1.0 + z), z, 0);
  PassArgs a = pass_args(c, k);
  GroupTimer t(c, kTOther, 1);
  if (c->params.precision == REC_PREC_MIXED) k_refresh<true, false><<<c->grid, NT, 0, c->stream>>>(a, nullptr, 1);
  else k_refresh<false, false><<<c->grid, NT, 0, c->stream>>>(a, nullptr, 1);
  return cudaGetLastError();
}

cudaError_t launch_state_init(rec_ctx* c, double z) {
  StepCoef k = step_coef(c->cosmo, c->params, z + 1e-6 * (1.0 + z), z, 0);
  PassArgs a = pass_args(c, k);
  double S = saha_S(k.Tg);
  GroupTimer t(c, kTOther, 1);
  if (c->params.precision == REC_PREC_MIXED)
    k_state_init<true, false><<<c->grid, NT, 0, c->stream>>>(a, k.nH / S, k.Tg, nullptr, 1);
  else k_state_init<false, false><<<c->grid, NT, 0, c->stream>>>(a, k.nH / S, k.Tg, nullptr, 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_refresh(c, z);
}

// The TMA-staged Newton and final passes need 16-byte aligned streams (bulk
// copies) and their shared-memory rings; REC_NEWTON=plain selects the
// grid-stride kernels.
bool newton_tma_ok(rec_ctx* c, const PassArgs& a) {
  if (c->newton_tma == 0) {
    const char* sel = std::getenv("REC_NEWTON");
    bool ok = !(sel && std::strcmp(sel, "plain") == 0);
    ok = ok && cudaFuncSetAttribute(k_newton_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem) ==
                   cudaSuccess;
    ok = ok && cudaFuncSetAttribute(k_final_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFinSmem) ==
                   cudaSuccess;
    // their blocks fit the partials (2 x grid entries)
    ok = ok && kTmaCtasPerSm * c->sm_count <= 2 * c->grid && kFinCtasPerSm * c->sm_count <= 2 * c->grid;
    c->newton_tma = ok ? 1 : -1;
    cudaGetLastError();
  }
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  return c->newton_tma > 0 && al(a.delta) && al(a.xy) && al(a.T) && al(a.tally) && al(a.x) && al(a.vel4);
}

cudaError_t launch_rec_step(rec_ctx* c, double z_from, double z_to, rec_stats* st) {
  const int ns = c->params.n_sub;
  const bool mixed = c->params.precision == REC_PREC_MIXED;
  double ya = std::log1p(z_from), yb = std::log1p(z_to);
  const bool local_modes = c->params.mixing == REC_MIX_LOCAL || c->params.mixing == REC_MIX_PARTIAL;
  const bool one_pass = c->params.mixing == REC_MIX_LOCAL ||
                        (c->params.mixing == REC_MIX_PARTIAL && !(c->params.f_alpha > 0.0));
  GroupTimer t(c, kTStep, one_pass ? 2 * ns : ns * (kNewtonMaxPasses + 2 + (local_modes ? 1 : 0)));
  for (int s = 0; s < ns; ++s) {
    double za = (s == 0) ? z_from : std::expm1(ya - (ya - yb) * (double)s / ns);
    double zb = (s == ns - 1) ? z_to : std::expm1(ya - (ya - yb) * (double)(s + 1) / ns);
    StepCoef k = step_coef(c->cosmo, c->params, za, zb, s == ns - 1);
    PassArgs a = pass_args(c, k);
    const bool part = c->params.mixing == REC_MIX_PARTIAL && c->params.f_alpha > 0.0;
    if (c->params.mixing == REC_MIX_LOCAL || (c->params.mixing == REC_MIX_PARTIAL && !part)) {
      const double fac = (1.0 + zb) * 1.0e3 / (2.0 * c->cosmo.L_m / c->box.n);
      if (mixed) {
        k_divergence<true><<<c->grid, NT, 0, c->stream>>>(c->box.vel4, c->box.n, fac, c->div);
        k_local<true><<<c->grid, NT, 0, c->stream>>>(a, c->div, st);
      } else {
        k_divergence<false><<<c->grid, NT, 0, c->stream>>>(c->box.vel4, c->box.n, fac, c->div);
        k_local<false><<<c->grid, NT, 0, c->stream>>>(a, c->div, st);
      }
      continue;
    }
    if (part) {  // divergence, then the Newton passes and the final pass with the local shares
      const double fac = (1.0 + zb) * 1.0e3 / (2.0 * c->cosmo.L_m / c->box.n);
      if (mixed) k_divergence<true><<<c->grid, NT, 0, c->stream>>>(c->box.vel4, c->box.n, fac, c->div);
      else k_divergence<false><<<c->grid, NT, 0, c->stream>>>(c->box.vel4, c->box.n, fac, c->div);
      k_substep_begin<<<1, 32, 0, c->stream>>>(c->sc, k, (double)c->n3);
      for (int it = 0; it < kNewtonMaxPasses; ++it) {
        if (mixed) k_newton_part<true><<<c->grid, NT, 0, c->stream>>>(a);
        else k_newton_part<false><<<c->grid, NT, 0, c->stream>>>(a);
      }
      if (mixed) k_final_part<true><<<c->grid, NT, 0, c->stream>>>(a, st);
      else k_final_part<false><<<c->grid, NT, 0, c->stream>>>(a, st);
      continue;
    }
    k_substep_begin<<<1, 32, 0, c->stream>>>(c->sc, k, (double)c->n3);
    const bool tma = mixed && newton_tma_ok(c, a);
    for (int it = 0; it < kNewtonMaxPasses; ++it) {
      if (tma) k_newton_tma<<<c->sm_count * kTmaCtasPerSm, kTmaThreads, kTmaSmem, c->stream>>>(a, c->wait_limit);
      else if (mixed) k_newton<true, false><<<c->grid, NT, 0, c->stream>>>(a, nullptr, 1);
      else k_newton<false, false><<<c->grid, NT, 0, c->stream>>>(a, nullptr, 1);
    }
    if (tma) k_final_tma<<<c->sm_count * kFinCtasPerSm, kTmaThreads, kFinSmem, c->stream>>>(a, st, c->wait_limit);
    else if (mixed) k_final<true, false><<<c->grid, NT, 0, c->stream>>>(a, st, nullptr, 1);
    else k_final<false, false><<<c->grid, NT, 0, c->stream>>>(a, st, nullptr, 1);
  }
  return cudaGetLastError();
}


// ------------------------------------------------------- batched contexts
// One launch per pass over all boxes of the context (grid = the boxes' pass
// blocks); each box keeps its own sums, lambda, Newton state and statistics.
namespace {
PassArgs batch_args(rec_ctx* c, const StepCoef& k) {
  PassArgs a;
  std::memset(&a, 0, sizeof(a));
  a.part = c->part;
  a.k = k;
  a.kf = coef_f32(k);
  return a;
}
}  // namespace

// Volume statistics of the current state (sums of the last rec_state_init,
// rec_refresh or rec_step): X_e = sum delta x / sum delta (Sec. II.A).
__global__ void k_volume_stats(const DevScalars* sc, const BoxDev* bxs, int B, rec_stats* st) {
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const DevScalars* s = bxs ? bxs[b].sc : sc;
    st[b].X_e = s->Sdx / s->Sd;
    st[b].lambda = s->lam_state;
    st[b].S1s = s->S1s;
  }
}

cudaError_t launch_volume_stats(rec_ctx* c, rec_stats* st) {
  GroupTimer t(c, kTOther, 1);
  k_volume_stats<<<1, 128, 0, c->stream>>>(c->sc, c->n_boxes > 1 ? c->bx : nullptr, c->n_boxes, st);
  return cudaGetLastError();
}

// Expired bounded waits (flags bit 3) of every box: reported in *out and
// cleared, with the counters a pass that gave up may have left part-way.
__global__ void k_check_waits(DevScalars* sc, const BoxDev* bxs, int B, DevScalars* gsc, int* out) {
  if (threadIdx.x != 0) return;
  // a batch-wide expiry (a grid barrier gave up) may have left any box part-way
  const bool all = gsc && (gsc->flags & 8);
  int any = all ? 1 : 0;
  for (int b = 0; b < B; ++b) {
    DevScalars* s = bxs ? bxs[b].sc : sc;
    if (all || (s->flags & 8)) {
      any = 1;
      s->flags &= ~8;
      s->counter = 0;
      s->alloc_counter = 0;
    }
  }
  if (all) {
    gsc->flags &= ~8;
    gsc->counter = 0;
    gsc->alloc_counter = 0;
    gsc->bar.arrived = 0;
  }
  *out = any;
}

cudaError_t launch_check_waits(rec_ctx* c, int* timed_out) {
  int* d = reinterpret_cast<int*>(c->part);  // scratch word: no pass is in flight after the sync
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return e;
  k_check_waits<<<1, 32, 0, c->stream>>>(c->sc, c->n_boxes > 1 ? c->bx : nullptr, c->n_boxes,
                                         c->n_boxes > 1 ? c->gsc : nullptr, d);
  e = cudaMemcpyAsync(timed_out, d, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(c->stream);
}

cudaError_t launch_refresh_batch(rec_ctx* c, double z) {
  StepCoef k = step_coef(c->cosmo, c->params, z + 1e-6 * (1.0 + z), z, 0);
  PassArgs a = batch_args(c, k);
  GroupTimer t(c, kTOther, 1);
  if (c->params.precision == REC_PREC_MIXED) k_refresh<true, true><<<c->tot_pblk, NT, 0, c->stream>>>(a, c->bx, c->n_boxes);
  else k_refresh<false, true><<<c->tot_pblk, NT, 0, c->stream>>>(a, c->bx, c->n_boxes);
  return cudaGetLastError();
}

cudaError_t launch_state_init_batch(rec_ctx* c, double z) {
  StepCoef k = step_coef(c->cosmo, c->params, z + 1e-6 * (1.0 + z), z, 0);
  PassArgs a = batch_args(c, k);
  double S = saha_S(k.Tg);
  {
    GroupTimer t(c, kTOther, 1);
    if (c->params.precision == REC_PREC_MIXED)
      k_state_init<true, true><<<c->tot_pblk, NT, 0, c->stream>>>(a, k.nH / S, k.Tg, c->bx, c->n_boxes);
    else k_state_init<false, true><<<c->tot_pblk, NT, 0, c->stream>>>(a, k.nH / S, k.Tg, c->bx, c->n_boxes);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_refresh_batch(c, z);
}

// Resident blocks of the persistent batched substep (0: cooperative launch unavailable).
int batch_substep_grid(rec_ctx* c, bool mixed) {
  if (c->batch_step_grid == 0) {
    int per_sm = 0, coop = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaError_t e = mixed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_substep<true>, NT, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_substep<false>, NT, 0);
    cudaGetLastError();
    c->batch_step_grid = (e == cudaSuccess && coop && per_sm > 0) ? per_sm * c->sm_count : -1;
  }
  return c->batch_step_grid;
}

cudaError_t launch_rec_step_batch(rec_ctx* c, double z_from, double z_to, rec_stats* st) {
  const int ns = c->params.n_sub;
  const bool mixed = c->params.precision == REC_PREC_MIXED;
  const double ya = std::log1p(z_from), yb = std::log1p(z_to);
  const int pgrid = batch_substep_grid(c, mixed);
  if (pgrid > 0) {  // one persistent launch per substep
    GroupTimer t(c, kTStep, ns);
    for (int s = 0; s < ns; ++s) {
      double za = (s == 0) ? z_from : std::expm1(ya - (ya - yb) * (double)s / ns);
      double zb = (s == ns - 1) ? z_to : std::expm1(ya - (ya - yb) * (double)(s + 1) / ns);
      StepCoef k = step_coef(c->cosmo, c->params, za, zb, s == ns - 1);
      PassArgs a = batch_args(c, k);
      const BoxDev* bxs = c->bx;
      int B = c->n_boxes, nvb = c->tot_pblk;
      DevScalars* gsc = c->gsc;
      uint32_t limit = c->wait_limit;
      void* args[] = {&a, &st, &bxs, &B, &nvb, &gsc, &limit};
      cudaError_t e = cudaLaunchCooperativeKernel(mixed ? (void*)k_batch_substep<true> : (void*)k_batch_substep<false>,
                                                  pgrid, NT, args, 0, c->stream);
      if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
  }
  GroupTimer t(c, kTStep, ns * (kNewtonMaxPasses + 2));
  for (int s = 0; s < ns; ++s) {
    double za = (s == 0) ? z_from : std::expm1(ya - (ya - yb) * (double)s / ns);
    double zb = (s == ns - 1) ? z_to : std::expm1(ya - (ya - yb) * (double)(s + 1) / ns);
    StepCoef k = step_coef(c->cosmo, c->params, za, zb, s == ns - 1);
    PassArgs a = batch_args(c, k);
    k_substep_begin_batch<<<1, kMaxBoxes, 0, c->stream>>>(c->bx, c->n_boxes, k);
    for (int it = 0; it < kNewtonMaxPasses; ++it) {
      if (mixed) k_newton<true, true><<<c->tot_pblk, NT, 0, c->stream>>>(a, c->bx, c->n_boxes);
      else k_newton<false, true><<<c->tot_pblk, NT, 0, c->stream>>>(a, c->bx, c->n_boxes);
    }
    if (mixed) k_final<true, true><<<c->tot_pblk, NT, 0, c->stream>>>(a, st, c->bx, c->n_boxes);
    else k_final<false, true><<<c->tot_pblk, NT, 0, c->stream>>>(a, st, c->bx, c->n_boxes);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------- allocation-free step
// The same refresh + Newton + final passes as rec_refresh followed by rec_step
// (FP64 form), for callers that cannot allocate device memory at step time: a
// host code that hands all device memory to its own pool allocator at start-up
// (a cudaMalloc would then fail), or one stepping from a loop where the
// implicit device synchronisation of cudaMalloc/cudaFree would stall work on
// its other streams.  Its scratch, one DevScalars record and the per-block
// partial sums, lives in the file-scope array below instead of a context.
// Every call clears the record first (the last-block-done counter, the Newton
// state and the flags must start at zero); the partials are written before
// they are read.  All calls on a device share the array: calls that overlap in
// time on that device (other streams, other host threads) race on it.
namespace {

constexpr int kNoAllocMaxBlocks = 2048;
constexpr size_t kNoAllocScBytes = (sizeof(DevScalars) + 255) / 256 * 256;
constexpr size_t kNoAllocBytes = kNoAllocScBytes + sizeof(double) * kMaxSums * kNoAllocMaxBlocks;  // 130 KiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocDevice {
  unsigned char* scratch;  // device address of g_noalloc_scratch
  int sm_count;
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];

// Once per device, with that device current: the address of the scratch array
// and the SM count.  The first call on a device may load the module.
cudaError_t noalloc_device(int dev, NoAllocDevice* out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoAllocDevice& d = g_noalloc_dev[dev];
  if (!d.scratch) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int sm = 0;
    e = cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    d.sm_count = sm;
    d.scratch = (unsigned char*)ptr;
  }
  *out = d;
  return cudaSuccess;
}

}  // namespace

rec_status launch_rec_step_noalloc(const rec_params& p, const rec_box& b, double z_from, double z_to,
                                   cudaStream_t stream, rec_stats* st, std::string* why) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { *why = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return REC_ECUDA; }
  if (dev < 0 || dev >= kNoAllocMaxDevices) { *why = "device ordinal beyond the static set-up table"; return REC_EINVAL; }
  NoAllocDevice d;
  e = noalloc_device(dev, &d);
  if (e != cudaSuccess) { *why = std::string("scratch set-up: ") + cudaGetErrorString(e); return REC_ECUDA; }
  const int64_t n3 = (int64_t)b.n * b.n * b.n;
  // the grid of the context path, so that the sums are taken in the same order
  const int64_t want = (n3 + NT - 1) / NT;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)d.sm_count * 8));
  if (grid > kNoAllocMaxBlocks) {
    *why = "the step needs " + std::to_string(grid) + " blocks of partial sums; the static scratch holds " +
           std::to_string(kNoAllocMaxBlocks);
    return REC_EINVAL;
  }
  DevScalars* sc = (DevScalars*)d.scratch;
  double* part = (double*)(d.scratch + kNoAllocScBytes);
  const Cosmo cosmo = make_cosmo(p);
  PassArgs a;
  a.n3 = n3;
  a.delta = b.delta;
  a.vel4 = b.vel4;
  a.x = b.x_e;
  a.xy = nullptr;
  a.T = b.T;
  a.tally = b.tally;
  a.emis = b.emis;
  a.sc = sc;
  a.part = part;
  a.div = nullptr;
  a.fmix = 1.0;
  e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), stream);
  if (e != cudaSuccess) { *why = std::string("cudaMemsetAsync: ") + cudaGetErrorString(e); return REC_ECUDA; }
  // sums and emission weights of the incoming state at z_from (as rec_refresh)
  a.k = step_coef(cosmo, p, z_from + 1e-6 * (1.0 + z_from), z_from, 0);
  k_refresh<false, false><<<grid, NT, 0, stream>>>(a, nullptr, 1);
  const int ns = p.n_sub;
  const double ya = std::log1p(z_from), yb = std::log1p(z_to);
  for (int s = 0; s < ns; ++s) {
    double za = (s == 0) ? z_from : std::expm1(ya - (ya - yb) * (double)s / ns);
    double zb = (s == ns - 1) ? z_to : std::expm1(ya - (ya - yb) * (double)(s + 1) / ns);
    a.k = step_coef(cosmo, p, za, zb, s == ns - 1);
    k_substep_begin<<<1, 32, 0, stream>>>(sc, a.k, (double)n3);
    for (int it = 0; it < kNewtonMaxPasses; ++it) k_newton<false, false><<<grid, NT, 0, stream>>>(a, nullptr, 1);
    k_final<false, false><<<grid, NT, 0, stream>>>(a, st, nullptr, 1);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) { *why = std::string("launch: ") + cudaGetErrorString(e); return REC_ECUDA; }
  return REC_OK;
}

}  // namespace rec
