// Second-order recombination step: TR-BDF2 (Bank et al., IEEE Trans. CAD 4,
// 436 (1985)) per substep for the per-cell system of rec_step (Eq. dotne-mix
// per hydrogen atom with the self-consistent lambda = <alpha n_e^2>/<n_1s>,
// Eq. Tb-evolution for T_b, Compton drag of Eq. alpha-def).
//
// A trapezoidal stage to t + gamma h (gamma = 2 - sqrt 2), then a BDF2 stage
// to t + h.  Each stage end is fully implicit in x, T, lambda and the Peebles
// factor (R_alpha^mix from the stage-end <n_1s>): T is linear given x; x is the
// positive root of the backward-Euler quadratic with the stage's explicit part
// in place of x_old; lambda and the neutral sum S_1s (which sets C) solve their
// two equations by a 2x2 Newton iteration; an outer iteration repeats T and
// alpha(T) until x and T stop changing (relative change below 1e-12; the parity target is 1e-9).  Every
// coefficient is taken at its own time; drag uses the trapezoidal exponent.
// FP64 form, tally and full mixing.  (The oracle reaches the same stage end by
// a fixed point over T, alpha and C around a Newton iteration on lambda alone;
// the 2x2 iteration converges in a few passes where that fixed point is slow.)
//
// Launch organisation: the outer and Newton iterations are launched a fixed
// number of times per stage; once converged (device flags) the remaining
// launches return at once, so the host never synchronises.  Reductions are the
// library's fixed-order block sums (bit-reproducible for a given grid).

#include <cmath>

#include "rec_internal.cuh"
#include "rec_reduce.cuh"

namespace rec {
namespace {

constexpr int NT = kPassThreads;
constexpr int kOuterMax = 8;    // outer (T, alpha) iterations launched per stage
constexpr int kNewtonMax = 16;  // 2x2 Newton evaluations launched per outer iteration

struct TrbScal {
  double lam, S;             // current iterate: lambda and the neutral sum S_1s
  double M;                  // max_i (-bx_i / (h w_i)): lambda_min = (M - C beta e_alpha) / (1 - C)
  double Ga, Sa;             // G and S_1s of the substep-start state
  double C;                  // Peebles factor at the last S
  int32_t newton_conv, outer_done, bad, unconverged;
  int32_t passes;            // Newton evaluations of the current substep
  uint32_t counter;          // last-block-done ticket
};

struct TrbArgs {
  int64_t n3;
  const double* delta;
  double* x;
  double* T;
  double* vel;               // double4 layout [n3][4]
  uint32_t* tally;
  double* emis;
  double* bx; double* bT;    // explicit parts of the current stage
  double* xg; double* Tg;    // stage iterate (and result)
  double* Tn; double* al;    // T and alpha(T) of the current outer iteration
  double* w;                 // J_i / <J> (1 in full mixing)
  double* part;              // block partials [grid][kMaxSums]
  TrbScal* s;
  DevScalars* sc;
  int tally_mode;
};

// Block maximum of values that may be negative (block_max starts from 0).
__device__ __forceinline__ double block_max_signed(double v) {
  __shared__ double sm[NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  __syncthreads();
  if (lane == 0) sm[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < NT / 32; ++w) v = fmax(v, sm[w]);
  return v;
}

__device__ __forceinline__ double alpha_e(const StepCoef& k, double T) {
  const double lt = log(T * 1.0e-4);
  return k.fa * exp(k.pb * lt) / (1.0 + k.pc * exp(k.pd * lt));
}

__device__ __forceinline__ double peebles(const StepCoef& k, double S, double n3) {
  const double Rmix = k.KR / (k.nH * S / n3);
  return (k.L2g + Rmix) / (k.beta + k.L2g + Rmix);
}

// dC/dS_1s: R = K_R n3 / (nH S), dR/dS = -R/S, dC/dR = beta / (beta + Lambda + R)^2.
__device__ __forceinline__ double peebles_dS(const StepCoef& k, double S, double n3) {
  const double Rmix = k.KR / (k.nH * S / n3);
  const double den = k.beta + k.L2g + Rmix;
  return -k.beta * Rmix / (S * den * den);
}

// Lower bound on lambda for the current S: every cell keeps c_i = bx_i + h w_i G > 0.
__device__ __forceinline__ double lam_min(const StepCoef& k, const TrbScal* s, double C) {
  return (s->M - C * k.beta * k.ea) / (1.0 - C);
}

// Positive root of A x^2 + (1 + sG) x - (b + sG) = 0 and d x / d G.
__device__ __forceinline__ double root(double A, double s, double G, double b, double* dxdG) {
  const double B = 1.0 + s * G;
  const double c = b + s * G;
  const double xr = 2.0 * c / (B + sqrt(B * B + 4.0 * A * c));
  if (dxdG) *dxdG = s * (1.0 - xr) / (2.0 * A * xr + B);
  return xr;
}

// Sums of the substep-start state: S_1s, <alpha n_e^2> and <n_1s> numerators.
__global__ void __launch_bounds__(NT) k_trb_start(TrbArgs a, StepCoef k) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += (int64_t)gridDim.x * NT) {
    const double d = a.delta[i], x = a.x[i], n = k.nH * d;
    v[0] += d * (1.0 - x);
    v[1] += alpha_e(k, a.T[i]) * n * n * x * x;
    v[2] += n * (1.0 - x);
  }
  block_sum<3, NT>(v);
  if (threadIdx.x == 0)
    for (int j = 0; j < 3; ++j) a.part[(size_t)blockIdx.x * kMaxSums + j] = v[j];
  if (last_block_done(&a.s->counter)) {
    double S[3];
    combine_partials<3, NT>(a.part, gridDim.x, kMaxSums, S);
    if (threadIdx.x == 0) {
      const double C = peebles(k, S[0], (double)a.n3);
      const double lam = S[1] / S[2];
      a.s->Sa = S[0];
      a.s->Ga = (1.0 - C) * lam + C * k.beta * k.ea;
      a.s->passes = 0;
      a.s->counter = 0;
    }
  }
}

// Stage 1 explicit part x + (gamma h / 2) f(x_n), same for T; the iterate starts at the state.
// The weights w_i = J_i / <J> come from the tallies and the n_1s of the state at
// the start of the step (first substep) and are held over its substeps, as in
// the backward-Euler step.
__global__ void __launch_bounds__(NT) k_trb_explicit1(TrbArgs a, StepCoef k, double h1, int first_sub) {
  const double Ga = a.s->Ga, Sa = a.s->Sa;
  const double tot = (double)a.sc->tally_total;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += (int64_t)gridDim.x * NT) {
    const double d = a.delta[i], x = a.x[i], T = a.T[i], n = k.nH * d;
    double w = 1.0;
    if (!first_sub) {
      w = a.w[i];
    } else if (a.tally_mode && tot > 0.0 && Sa > 0.0) {
      const double n1s_rel = d * (1.0 - x);
      if (n1s_rel > 0.0) w = ((double)a.tally[i] / tot) * Sa / n1s_rel;
    }
    if (first_sub) a.w[i] = w;
    const double fx = -alpha_e(k, T) * n * x * x + w * Ga * (1.0 - x);
    const double g = k.kc * x / (1.0 + k.fHe + x);
    const double hh = k.hq / (d * (1.0 + k.fHe + x));
    const double fT = -2.0 * k.H * T + g * (k.Tg - T) + hh;
    a.bx[i] = x + h1 * fx;
    a.bT[i] = T + h1 * fT;
    a.xg[i] = x;
    a.Tg[i] = T;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.s->outer_done = 0;
}

// Stage 2 explicit part (x_g / gamma - (1-gamma)^2 x_n / gamma) / (2 - gamma), same for T.
__global__ void __launch_bounds__(NT) k_trb_explicit2(TrbArgs a, double c1, double c0) {
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += (int64_t)gridDim.x * NT) {
    a.bx[i] = c1 * a.xg[i] - c0 * a.x[i];
    a.bT[i] = c1 * a.Tg[i] - c0 * a.T[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.s->outer_done = 0;
}

// Outer iteration, first pass: T from the current x iterate (linear) and
// alpha(T); the bound M = max_i (-bx_i / (h w_i)); on the first outer pass of a
// stage also the starts lambda = <alpha n_e^2>/<n_1s> and S_1s of the iterate.
__global__ void __launch_bounds__(NT) k_trb_prep(TrbArgs a, StepCoef k, double h, int first) {
  if (a.s->outer_done) return;
  double v[3] = {0.0, 0.0, 0.0};
  double m = -1e300;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += (int64_t)gridDim.x * NT) {
    const double d = a.delta[i], x = a.xg[i], n = k.nH * d;
    const double g = k.kc * x / (1.0 + k.fHe + x);
    const double hh = k.hq / (d * (1.0 + k.fHe + x));
    const double Tn = (a.bT[i] + h * (g * k.Tg + hh)) / (1.0 + h * (2.0 * k.H + g));
    const double al = alpha_e(k, Tn);
    a.Tn[i] = Tn;
    a.al[i] = al;
    const double sw = h * a.w[i];
    if (sw > 0.0) m = fmax(m, -a.bx[i] / sw);
    else if (!(a.bx[i] > 0.0)) m = 1e300;  // no photo-ionisation term and no positive root
    v[0] += d * (1.0 - x);
    v[1] += al * n * n * x * x;
    v[2] += n * (1.0 - x);
  }
  block_sum<3, NT>(v);
  m = block_max_signed(m);
  if (threadIdx.x == 0) {
    for (int j = 0; j < 3; ++j) a.part[(size_t)blockIdx.x * kMaxSums + j] = v[j];
    a.part[(size_t)blockIdx.x * kMaxSums + 3] = m;
  }
  if (last_block_done(&a.s->counter)) {
    double S[3];
    combine_partials<3, NT>(a.part, gridDim.x, kMaxSums, S);
    double M = -1e300;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += NT) M = fmax(M, __ldcg(a.part + (size_t)b * kMaxSums + 3));
    M = block_max_signed(M);
    if (threadIdx.x == 0) {
      TrbScal* s = a.s;
      s->M = M;
      if (first) {
        s->lam = S[1] / S[2];
        s->S = S[0];
      }
      const double C = peebles(k, s->S, (double)a.n3);
      const double lmin = lam_min(k, s, C);
      if (!(s->lam > lmin)) s->lam = lmin + fmax(fabs(lmin), fabs(s->lam));
      s->newton_conv = 0;
      s->counter = 0;
    }
  }
}

// One 2x2 Newton evaluation for (lambda, S_1s):
//   F1 = sum alpha n^2 x^2 - lambda sum n (1 - x),   F2 = sum delta (1 - x) - S_1s,
// x_i the roots at G = (1 - C(S)) lambda + C(S) beta e_alpha.
__global__ void __launch_bounds__(NT) k_trb_newton(TrbArgs a, StepCoef k, double h) {
  if (a.s->outer_done || a.s->newton_conv) return;
  const double n3 = (double)a.n3;
  const double lam = a.s->lam, S = a.s->S;
  const double C = peebles(k, S, n3), omC = 1.0 - C, CBe = C * k.beta * k.ea;
  const double G = omC * lam + CBe;
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += (int64_t)gridDim.x * NT) {
    const double d = a.delta[i], n = k.nH * d, al = a.al[i];
    const double sw = h * a.w[i];
    const double b = a.bx[i];
    if (!(b + sw * G > 0.0)) v[5] += 1.0;  // no positive root at this G
    double dxdG;
    const double xr = root(h * al * n, sw, G, b, &dxdG);
    const double an2 = al * n * n;
    v[0] += an2 * xr * xr - lam * n * (1.0 - xr);
    v[1] += d * (1.0 - xr);
    v[2] += (2.0 * an2 * xr + lam * n) * dxdG;
    v[3] += n * (1.0 - xr);
    v[4] += d * dxdG;
  }
  block_sum<6, NT>(v);
  if (threadIdx.x == 0)
    for (int j = 0; j < 6; ++j) a.part[(size_t)blockIdx.x * kMaxSums + j] = v[j];
  if (last_block_done(&a.s->counter)) {
    double R[6];
    combine_partials<6, NT>(a.part, gridDim.x, kMaxSums, R);
    if (threadIdx.x == 0) {
      TrbScal* s = a.s;
      const double F1 = R[0], F2 = R[1] - S, P = R[2], Q = R[3], Dd = R[4];
      const double Gs = (k.beta * k.ea - lam) * peebles_dS(k, S, n3);
      const double J11 = P * omC - Q, J12 = P * Gs, J21 = -Dd * omC, J22 = -Dd * Gs - 1.0;
      const double det = J11 * J22 - J12 * J21;
      double ln = lam, Sn = S;
      if (det != 0.0 && isfinite(det)) {
        ln = lam - (F1 * J22 - J12 * F2) / det;
        Sn = S - (J11 * F2 - J21 * F1) / det;
      }
      // trust region: S within a factor 2 and lambda within a factor 4 per pass
      // (from a start far from the stage end the joint step can overshoot)
      if (!(Sn > 0.5 * S)) Sn = 0.5 * S;
      if (!(Sn < 2.0 * S)) Sn = 2.0 * S;
      if (!(ln < 4.0 * lam)) ln = 4.0 * lam;
      if (!(ln > 0.25 * lam)) ln = 0.25 * lam;
      const double lmin = lam_min(k, s, peebles(k, Sn, n3));
      if (!(ln > lmin)) ln = (lam > lmin) ? 0.5 * (lam + lmin) : lmin + fmax(fabs(lmin), fabs(lam));
      if (fabs(ln - lam) <= 1e-13 * fabs(lam) && fabs(Sn - S) <= 1e-13 * fabs(S)) s->newton_conv = 1;
      if (R[5] > 0.0 && s->newton_conv) s->bad = 1;  // converged with a cell left without a positive root
      s->lam = ln;
      s->S = Sn;
      s->passes += 1;
      s->counter = 0;
    }
  }
}

// Outer iteration, last pass: the roots at the converged (lambda, S_1s) become
// the iterate, with T; the stage is done when neither changed by more than 1e-12 (rounding keeps
// near-equilibrium cells changing at a few 1e-14).
__global__ void __launch_bounds__(NT) k_trb_update(TrbArgs a, StepCoef k, double h) {
  if (a.s->outer_done) return;
  const double C = peebles(k, a.s->S, (double)a.n3);
  const double G = (1.0 - C) * a.s->lam + C * k.beta * k.ea;
  double m = 0.0;
  double nbad[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += (int64_t)gridDim.x * NT) {
    const double n = k.nH * a.delta[i];
    const double xn = root(h * a.al[i] * n, h * a.w[i], G, a.bx[i], nullptr);
    const double Tn = a.Tn[i];
    if (!(xn > 0.0 && xn < 1e300) || !(Tn > 0.0 && Tn < 1e300)) nbad[0] += 1.0;  // fmax would hide a NaN
    m = fmax(m, fabs(xn - a.xg[i]) / xn);
    m = fmax(m, fabs(Tn - a.Tg[i]) / Tn);
    a.xg[i] = xn;
    a.Tg[i] = Tn;
  }
  m = block_max<NT>(m);
  block_sum<1, NT>(nbad);
  if (threadIdx.x == 0) {
    a.part[(size_t)blockIdx.x * kMaxSums] = m;
    a.part[(size_t)blockIdx.x * kMaxSums + 1] = nbad[0];
  }
  if (last_block_done(&a.s->counter)) {
    const double M = combine_max<NT>(a.part, gridDim.x, kMaxSums, 0);
    double B[1];
    combine_partials<1, NT>(a.part + 1, gridDim.x, kMaxSums, B);
    if (threadIdx.x == 0) {
      if (B[0] > 0.0) a.s->unconverged = 1;  // non-finite or non-positive stage end
      if (M <= 1e-12) a.s->outer_done = 1;
      a.s->C = C;
      a.s->counter = 0;
    }
  }
}

// Marks a stage whose outer iteration did not converge within the launches.
__global__ void k_trb_stage_end(TrbScal* s) {
  if (threadIdx.x == 0 && !s->outer_done) s->unconverged = 1;
}

// State <- stage-2 iterate; drag with the trapezoidal exponent; emission
// weights; tallies zeroed after the last substep; sums and statistics.
__global__ void __launch_bounds__(NT) k_trb_final(TrbArgs a, StepCoef ka, StepCoef kb, double h, rec_stats* st) {
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n3; i += (int64_t)gridDim.x * NT) {
    const double d = a.delta[i], x0 = a.x[i], x1 = a.xg[i], T1 = a.Tg[i];
    const double damp = exp(-0.5 * h * ((ka.kd * x0 + ka.H) + (kb.kd * x1 + kb.H)));
    double* u = a.vel + 4 * i;
    u[0] *= damp; u[1] *= damp; u[2] *= damp;
    a.x[i] = x1;
    a.T[i] = T1;
    const double ne = kb.nH * d * x1;
    a.emis[i] = alpha_e(kb, T1) * ne * ne;
    if (kb.last) a.tally[i] = 0u;
    v[0] += d * (1.0 - x1);
    v[1] += d * x1;
    v[2] += d;
  }
  block_sum<3, NT>(v);
  if (threadIdx.x == 0)
    for (int j = 0; j < 3; ++j) a.part[(size_t)blockIdx.x * kMaxSums + j] = v[j];
  if (last_block_done(&a.s->counter)) {
    double S[3];
    combine_partials<3, NT>(a.part, gridDim.x, kMaxSums, S);
    if (threadIdx.x == 0) {
      DevScalars* sc = a.sc;
      sc->S1s = S[0];
      sc->Sdx = S[1];
      sc->Sd = S[2];
      sc->lam_prev = sc->lam_state;
      sc->lam_state = a.s->lam;
      sc->C = a.s->C;
      sc->passes = a.s->passes;
      if (a.s->unconverged || a.s->bad) sc->flags |= 1;
      if (kb.last) sc->tally_total = 0ull;
      sc->emis_valid = 1;
      if (st) {
        st->X_e = S[1] / S[2];
        st->lambda = a.s->lam;
        st->C_mix = a.s->C;
        st->S1s = S[0];
        st->newton_passes = a.s->passes;
        st->flags = sc->flags;
      }
      a.s->counter = 0;
    }
  }
}

// Redshift at which the cosmic time since za is tau (bisection on the same
// Simpson-rule time integral as the substeps).
double z_after(const Cosmo& c, double za, double zb, double tau) {
  double lo = zb, hi = za;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (cosmic_dt(c, za, mid) < tau) hi = mid; else lo = mid;
    if (hi - lo <= 1e-13 * za) break;
  }
  return 0.5 * (lo + hi);
}

void stage(rec_ctx* c, const TrbArgs& a, const StepCoef& k, double h) {
  for (int outer = 0; outer < kOuterMax; ++outer) {
    k_trb_prep<<<c->grid, NT, 0, c->stream>>>(a, k, h, outer == 0 ? 1 : 0);
    for (int it = 0; it < kNewtonMax; ++it) k_trb_newton<<<c->grid, NT, 0, c->stream>>>(a, k, h);
    k_trb_update<<<c->grid, NT, 0, c->stream>>>(a, k, h);
  }
  k_trb_stage_end<<<1, 32, 0, c->stream>>>(a.s);
}

}  // namespace

cudaError_t launch_rec_step_trbdf2(rec_ctx* c, double z_from, double z_to, rec_stats* st) {
  const int64_t n3 = c->n3;
  const size_t arr = sizeof(double) * (size_t)n3;
  const size_t need = 7 * arr + 256;
  if (c->trb_bytes < need) {
    if (c->trb_scratch) cudaFree(c->trb_scratch);
    c->trb_scratch = nullptr;
    c->trb_bytes = 0;
    cudaError_t e = cudaMalloc(&c->trb_scratch, need);
    if (e != cudaSuccess) return e;
    c->trb_bytes = need;
  }
  char* base = (char*)c->trb_scratch;
  TrbArgs a;
  a.n3 = n3;
  a.delta = (const double*)c->box.delta;
  a.x = c->box.x_e;
  a.T = (double*)c->box.T;
  a.vel = (double*)c->box.vel4;
  a.tally = c->box.tally;
  a.emis = (double*)c->box.emis;
  a.bx = (double*)(base + 0 * arr);
  a.bT = (double*)(base + 1 * arr);
  a.xg = (double*)(base + 2 * arr);
  a.Tg = (double*)(base + 3 * arr);
  a.Tn = (double*)(base + 4 * arr);
  a.al = (double*)(base + 5 * arr);
  a.w = (double*)(base + 6 * arr);
  a.s = (TrbScal*)(base + 7 * arr);
  a.part = c->part;
  a.sc = c->sc;
  a.tally_mode = c->params.mixing == REC_MIX_TALLY ? 1 : 0;
  cudaError_t e = cudaMemsetAsync(a.s, 0, sizeof(TrbScal), c->stream);
  if (e != cudaSuccess) return e;
  const int ns = c->params.n_sub;
  const double ya = std::log1p(z_from), yb = std::log1p(z_to);
  const double gam = 2.0 - std::sqrt(2.0);
  const double c1 = 1.0 / (gam * (2.0 - gam)), c0 = (1.0 - gam) * (1.0 - gam) / (gam * (2.0 - gam));
  GroupTimer t(c, kTStep, ns * (4 + 2 * (kOuterMax * (kNewtonMax + 2) + 1)));
  for (int sidx = 0; sidx < ns; ++sidx) {
    const double za = (sidx == 0) ? z_from : std::expm1(ya - (ya - yb) * (double)sidx / ns);
    const double zb = (sidx == ns - 1) ? z_to : std::expm1(ya - (ya - yb) * (double)(sidx + 1) / ns);
    const double h = cosmic_dt(c->cosmo, za, zb);
    const double zg = z_after(c->cosmo, za, zb, gam * h);
    const StepCoef ka = step_coef(c->cosmo, c->params, za, za, 0);
    const StepCoef kg = step_coef(c->cosmo, c->params, zg, zg, 0);
    const StepCoef kb = step_coef(c->cosmo, c->params, zb, zb, sidx == ns - 1);
    k_trb_start<<<c->grid, NT, 0, c->stream>>>(a, ka);
    k_trb_explicit1<<<c->grid, NT, 0, c->stream>>>(a, ka, 0.5 * gam * h, sidx == 0 ? 1 : 0);
    stage(c, a, kg, 0.5 * gam * h);
    k_trb_explicit2<<<c->grid, NT, 0, c->stream>>>(a, c1, c0);
    stage(c, a, kb, (1.0 - gam) / (2.0 - gam) * h);
    k_trb_final<<<c->grid, NT, 0, c->stream>>>(a, ka, kb, h, st);
  }
  return cudaGetLastError();
}

}  // namespace rec
