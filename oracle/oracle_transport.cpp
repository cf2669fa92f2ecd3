// Oracle: counter-based random numbers, packet allocation and ballistic
// Ly-alpha packet transport.  TEST INFRASTRUCTURE ONLY (see oracle.h).
//
// The transport follows the Monte-Carlo description of Appendix A and
// Sec. III.B of arXiv:2312.11448 reduced to its ballistic part: a packet is
// injected at a random point of its emitting cell (step (1)), streams in a
// straight line while the Hubble expansion redshifts it by dx = -H dl / v_th
// (step (4)), and its frequency in the local gas frame includes the bulk-flow
// Doppler shift omega_r = omega (1 - U_par) (Eq. for omega_r).  It is absorbed
// in the first cell where it comes back into line resonance.
//
// The arithmetic is spelled out operation by operation (no fused multiply-add:
// build with -ffp-contract=off) in a real type R, float or double, so that a
// GPU kernel following the same sequence produces identical integer tallies.

#include "oracle.h"

#ifdef ORACLE_OPENMP
#include <omp.h>
#endif

#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

namespace {

// ---- Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) ----------------------
const uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
const uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

void philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)kPhiloxM0 * x0;
    uint64_t p1 = (uint64_t)kPhiloxM1 * x2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// Stream layout: key = (seed low word, seed high word XOR step);
// counter = (cell, packet index within the cell, block, box).
void draw(uint64_t seed, uint32_t step, uint32_t cell, uint32_t j, uint32_t block, uint32_t box, uint32_t out[4]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ step};
  uint32_t ctr[4] = {cell, j, block, box};
  philox(ctr, key, out);
}
// Block index reserved for the allocation offset.
const uint32_t kAllocBlock = 0x000A110Cu;

// Uniform deviates strictly inside (0,1), exactly representable:
//   binary32: (2 floor(r/2^9) + 1) 2^-24;  binary64 from a 64-bit word w:
//   (2 floor(w/2^12) + 1) 2^-53.
inline float u01f(uint32_t r) { return (float)((r >> 8) | 1u) * 0x1p-24f; }
inline double u01d(uint32_t lo, uint32_t hi) {
  uint64_t w = ((uint64_t)hi << 32) | lo;
  return (double)((w >> 11) | 1u) * 0x1p-53;
}

// ---- allocation ----------------------------------------------------------------
// Packets are emitted per cell in proportion to the local recombination rate
// r_i = alpha_e n_e^2 (the integrand of the global loss-rate Monte Carlo,
// Sec. III.B footnote).  Weights are quantised to Q_i = floor(2^31 r_i / r_max)
// and the n_packets packets are spread by systematic sampling with one random
// offset u in [0, sum Q): the exclusive packet prefix of cell i is
// P_i = floor((n_packets * prefixQ_i + u) / sum Q), in exact integer arithmetic.
template <class R>
int allocate(int n, const R* emis, uint64_t n_packets, uint64_t seed, uint32_t step, uint32_t box, uint32_t* P) {
  if (n <= 0 || !emis || !P) return -1;
  int64_t n3 = (int64_t)n * n * n;
  R rmax = 0;
  for (int64_t i = 0; i < n3; ++i) {
    if (!(emis[i] >= (R)0)) return -2;  // negative or NaN weight
    if (emis[i] > rmax) rmax = emis[i];
  }
  std::vector<uint64_t> Q(n3, 0);
  unsigned __int128 sumQ = 0;
  if (rmax > (R)0) {
    for (int64_t i = 0; i < n3; ++i) {
      R ratio = emis[i] / rmax;
      Q[i] = (uint64_t)(ratio * (R)2147483648.0);
      sumQ += Q[i];
    }
  }
  if (sumQ == 0 || n_packets == 0) {
    for (int64_t i = 0; i <= n3; ++i) P[i] = 0;
    return n_packets == 0 ? 0 : -3;
  }
  uint32_t r[4];
  draw(seed, step, 0u, 0u, kAllocBlock, box, r);
  uint64_t w = ((uint64_t)r[1] << 32) | r[0];
  unsigned __int128 u = (unsigned __int128)w % sumQ;
  unsigned __int128 pre = 0;
  for (int64_t i = 0; i <= n3; ++i) {
    P[i] = (uint32_t)(((unsigned __int128)n_packets * pre + u) / sumQ);
    if (i < n3) pre += Q[i];
  }
  return 0;
}

// ---- transport -------------------------------------------------------------------
const uint32_t kMaxCrossings = 1u << 20;

template <class R>
struct Rand;  // per-precision stream layout

template <>
struct Rand<float> {
  // block 0: cell offsets (3) and the frequency quantile; blocks 1..16: two
  // direction pairs each.
  static void position(uint64_t seed, uint32_t step, uint32_t c, uint32_t j, uint32_t box, float f[3], float* uq) {
    uint32_t r[4];
    draw(seed, step, c, j, 0u, box, r);
    f[0] = u01f(r[0]); f[1] = u01f(r[1]); f[2] = u01f(r[2]);
    *uq = u01f(r[3]);
  }
  static bool pair(uint64_t seed, uint32_t step, uint32_t c, uint32_t j, uint32_t box, int t, float* a, float* b) {
    if (t >= 32) return false;
    uint32_t r[4];
    draw(seed, step, c, j, 1u + (uint32_t)(t >> 1), box, r);
    int o = (t & 1) * 2;
    *a = u01f(r[o]); *b = u01f(r[o + 1]);
    return true;
  }
};

template <>
struct Rand<double> {
  // blocks 0,1: cell offsets (3) and the frequency quantile, two words per
  // deviate; blocks 2..33: one direction pair each.
  static void position(uint64_t seed, uint32_t step, uint32_t c, uint32_t j, uint32_t box, double f[3], double* uq) {
    uint32_t r[4], s[4];
    draw(seed, step, c, j, 0u, box, r);
    draw(seed, step, c, j, 1u, box, s);
    f[0] = u01d(r[0], r[1]); f[1] = u01d(r[2], r[3]); f[2] = u01d(s[0], s[1]);
    *uq = u01d(s[2], s[3]);
  }
  static bool pair(uint64_t seed, uint32_t step, uint32_t c, uint32_t j, uint32_t box, int t, double* a, double* b) {
    if (t >= 32) return false;
    uint32_t r[4];
    draw(seed, step, c, j, 2u + (uint32_t)t, box, r);
    *a = u01d(r[0], r[1]); *b = u01d(r[2], r[3]);
    return true;
  }
};

template <class R>
int transport(const orc_cosmo* cp, int n, double z, uint64_t seed, uint32_t step, uint32_t box, uint64_t n_packets,
              const R* emis, const R* vel4, const R* T, const R* quant, int M, uint32_t* tally, uint64_t* counters,
              orc_packet* dump, int64_t dump_cap) {
  if (!cp || n <= 0 || !emis || !vel4 || !T || !quant || M < 2 || !tally || !counters) return -1;
  int64_t n3 = (int64_t)n * n * n;
  if (n_packets > 0xFFFFFFFFull) return -1;
  double tp[2];
  if (orc_transport_params(cp, n, z, tp) != 0) return -1;
  const R kappa = (R)tp[0];
  const R cth = (R)tp[1];
  std::vector<uint32_t> P(n3 + 1);
  int rc = allocate<R>(n, emis, n_packets, seed, step, box, P.data());
  if (rc != 0) return rc;
  const R inf = std::numeric_limits<R>::infinity();
  const R one = (R)1, two = (R)2;
  uint64_t emitted = 0, absorbed = 0, capped = 0, crossings = 0;
  int64_t ndump = 0;
  // The OpenMP build of this file (host-cores timing baseline only) spreads the
  // emitting cells over threads; integer tallies and counters are the same in
  // any order.  The plain build ignores the pragmas.
#ifdef ORACLE_OPENMP
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : emitted, absorbed, capped, crossings) if (dump == nullptr)
#endif
  for (int64_t c = 0; c < n3; ++c) {
    uint32_t np = P[c + 1] - P[c];
    const int hx = (int)(c % n), hy = (int)((c / n) % n), hz = (int)(c / ((int64_t)n * n));
    for (uint32_t j = 0; j < np; ++j) {
      ++emitted;
      // (1) injection point, uniform in the emitting cell.
      R f[3], uq;
      Rand<R>::position(seed, step, (uint32_t)c, j, box, f, &uq);
      // Isotropic direction, Marsaglia (1972): accept (v1, v2) in the unit disc.
      R nx = 0, ny = 0, nz = 1;
      for (int t = 0;; ++t) {
        R a, b;
        if (!Rand<R>::pair(seed, step, (uint32_t)c, j, box, t, &a, &b)) break;  // fallback (0,0,1)
        R v1 = two * a - one, v2 = two * b - one;
        R s = v1 * v1 + v2 * v2;
        if (s < one && s > (R)0) {
          R fac = two * std::sqrt(one - s);
          nx = v1 * fac; ny = v2 * fac; nz = one - two * s;
          break;
        }
      }
      // Emission frequency offset from the tabulated inverse CDF of the profile.
      R tq = uq * (R)(M - 1);
      int k = (int)tq;
      if (k > M - 2) k = M - 2;
      R fr = tq - (R)k;
      R xi = quant[k] + fr * (quant[k + 1] - quant[k]);
      // Thermal velocity in cells: v_th kappa = sqrt(T cth).
      R vt = std::sqrt(T[c] * cth);
      R knx = kappa * nx, kny = kappa * ny, knz = kappa * nz;
      const R* Uh = vel4 + 4 * c;
      R dh = (knx * Uh[0] + kny * Uh[1]) + knz * Uh[2];
      // Resonance distance along the ray (cells) if the flow were uniform:
      // kappa (xi v_th + n.U_emit).
      R u0 = xi * vt + dh;
      // Amanatides-Woo traversal from the emission point.
      int ix = hx, iy = hy, iz = hz;
      R nd[3] = {nx, ny, nz};
      R tM[3], tD[3];
      int st[3];
      for (int a = 0; a < 3; ++a) {
        if (nd[a] > (R)0) { st[a] = 1; tD[a] = one / nd[a]; tM[a] = (one - f[a]) * tD[a]; }
        else if (nd[a] < (R)0) { st[a] = -1; tD[a] = one / (-nd[a]); tM[a] = f[a] * tD[a]; }
        else { st[a] = 0; tD[a] = inf; tM[a] = inf; }
      }
      uint32_t kc = 0;
      int64_t cell = c;
      bool done = false;
      for (;;) {
        cell = ((int64_t)iz * n + iy) * n + ix;
        const R* Uc = vel4 + 4 * cell;
        R dc = (knx * Uc[0] + kny * Uc[1]) + knz * Uc[2];
        int ax;
        R s_exit;
        if (tM[0] <= tM[1] && tM[0] <= tM[2]) { ax = 0; s_exit = tM[0]; }
        else if (tM[1] <= tM[2]) { ax = 1; s_exit = tM[1]; }
        else { ax = 2; s_exit = tM[2]; }
        // In cell `cell` the packet's gas-frame frequency reaches line centre at
        // path length u0 - kappa n.U_cell; absorb if that is before the exit.
        if (u0 - dc <= s_exit) { done = true; break; }
        if (kc >= kMaxCrossings) break;
        if (ax == 0) { ix += st[0]; if (ix == n) ix = 0; if (ix < 0) ix = n - 1; }
        else if (ax == 1) { iy += st[1]; if (iy == n) iy = 0; if (iy < 0) iy = n - 1; }
        else { iz += st[2]; if (iz == n) iz = 0; if (iz < 0) iz = n - 1; }
        tM[ax] = tM[ax] + tD[ax];
        ++kc;
      }
      crossings += kc;
      if (done) {
#ifdef ORACLE_OPENMP
#pragma omp atomic
#endif
        tally[cell] += 1u;
        ++absorbed;
      }
      else ++capped;
      if (dump && ndump < dump_cap) {
        orc_packet& p = dump[ndump++];
        p.home = (uint32_t)c; p.j = j; p.absorb = done ? (uint32_t)cell : 0xFFFFFFFFu; p.crossings = kc;
        p.f[0] = f[0]; p.f[1] = f[1]; p.f[2] = f[2];
        p.dir[0] = nx; p.dir[1] = ny; p.dir[2] = nz;
        p.xi = xi; p.u0 = u0;
      }
    }
  }
  counters[0] = emitted; counters[1] = absorbed; counters[2] = capped; counters[3] = crossings;
  return 0;
}

}  // namespace

extern "C" {

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) { philox(ctr, key, out); }

int orc_threads(int n) {
#ifdef ORACLE_OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

int orc_transport_params(const orc_cosmo* cp, int n, double z, double* out) {
  if (!cp || n <= 0 || !out) return -1;
  double bg[5];
  orc_background(cp, z, bg);
  const double kMpc_m = 3.0856775814913673e22;
  const double kB = 1.380649e-23, mH = 1.00782503223 * 1.66053906660e-27;
  double a = 1.0 / (1.0 + z);
  double L_m = cp->L_box_kpc * kMpc_m * 1.0e-3;
  // Proper Hubble velocity across the box, km/s; kappa = cells per km/s.
  double v_box = bg[0] * a * L_m * 1.0e-3;
  double kappa = (double)n / v_box;
  // v_th^2 = 2 k T / m_H in (km/s)^2 per K, times kappa^2.
  out[0] = kappa;
  out[1] = kappa * kappa * (2.0 * kB / mH * 1.0e-6);
  return 0;
}

int orc_allocate_f32(int n, const float* emis, uint64_t n_packets, uint64_t seed, uint32_t step, uint32_t box,
                     uint32_t* P) {
  return allocate<float>(n, emis, n_packets, seed, step, box, P);
}
int orc_allocate_f64(int n, const double* emis, uint64_t n_packets, uint64_t seed, uint32_t step, uint32_t box,
                     uint32_t* P) {
  return allocate<double>(n, emis, n_packets, seed, step, box, P);
}

int orc_transport_f32(const orc_cosmo* cp, int n, double z, uint64_t seed, uint32_t step, uint32_t box,
                      uint64_t n_packets, const float* emis, const float* vel4, const float* T, const float* quant,
                      int M, uint32_t* tally, uint64_t* counters, orc_packet* dump, int64_t dump_cap) {
  return transport<float>(cp, n, z, seed, step, box, n_packets, emis, vel4, T, quant, M, tally, counters, dump,
                          dump_cap);
}
int orc_transport_f64(const orc_cosmo* cp, int n, double z, uint64_t seed, uint32_t step, uint32_t box,
                      uint64_t n_packets, const double* emis, const double* vel4, const double* T,
                      const double* quant, int M, uint32_t* tally, uint64_t* counters, orc_packet* dump,
                      int64_t dump_cap) {
  return transport<double>(cp, n, z, seed, step, box, n_packets, emis, vel4, T, quant, M, tally, counters, dump,
                           dump_cap);
}

}  // extern "C"
