// Internal declarations of the GB300 recombination library (not part of the
// ABI).  Host-side scalar physics lives in rec_cosmo.h; kernels are in
// rec_transport.cu, rec_step.cu and rec_adjoint.cu; the C ABI in rec_capi.cu.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "rec.h"
#include "rec_grid.cuh"

namespace rec {

// Launch geometry of the streaming passes: a fixed grid so that the
// fixed-order reductions are bit-reproducible from run to run.
constexpr int kPassThreads = 256;
constexpr int kMaxSums = 8;            // block partials per reduction
constexpr int kNewtonMaxPasses = 10;   // Newton evaluations launched per substep
constexpr uint32_t kMaxCrossings = 1u << 20;  // per-packet cap on face crossings
constexpr int kAllocThreads = 256;
constexpr int kAllocItems = 16;        // consecutive cells per thread in the allocation scan
// Smallest side of the super-tiles whose buckets order the march queue (the
// bucket arrays are sized for it; the side in use is a tuning parameter).
constexpr uint32_t kMinTile = 8;
constexpr int kAllocChunk = kAllocThreads * kAllocItems;
// Polls of a bounded device-side wait before it gives up (about a second).
constexpr uint32_t kDefaultWaitLimit = 1u << 22;

// Device-resident scalars of one box.  Everything data-dependent stays on the
// device so that calls never synchronise with the host.
struct DevScalars {
  // sums of the current state (end of the last rec_step, or rec_refresh)
  double S1s;        // sum delta (1 - x)
  double Sdx;        // sum delta x
  double Sd;         // sum delta
  double lam_state;  // <alpha n_e^2>/<n_1s> of the current state
  double lam_prev;   // lambda of the previous step (<= 0: none)
  double rmax;       // largest emission weight
  // Newton iteration of the current substep
  double lam;        // current iterate
  double C;          // Peebles factor with R_alpha^mix
  double omC;        // 1 - C
  double G0;         // C beta e_alpha
  double last_step;  // |last Newton step| / lambda
  int32_t conv;      // 1 once converged
  int32_t passes;    // Newton evaluations so far
  int32_t flags;     // rec_stats.flags bits
  uint32_t counter;  // last-block-done counter of the streaming passes
  // transport
  unsigned long long emitted, absorbed, capped, crossings;
  unsigned long long tally_total;  // packets absorbed in the current tallies
  unsigned long long sumQ;         // sum of quantised emission weights
  unsigned long long alloc_u;      // systematic-sampling offset in [0, sumQ)
  unsigned long long qtail;        // packets queued for the march
  unsigned long long march_next;   // next queue chunk handed to a march warp
  unsigned long long requeued;     // region sweeps: packets queued again in this transport call
  uint32_t alloc_counter;
  int32_t emis_valid;
  GridBarrier bar;  // grid barrier of the persistent batched launches (batch-wide record)
  // binary32 copies of the current iterate for the mixed form's passes (set
  // with lam, so that no pass converts binary64 scalars per thread)
  float lamf;        // lambda
  float Gf;          // G = (1 - C) lambda + C beta e_alpha
  float Ghi, Glo;    // G as a double-float pair
  float wscale;      // S1s / tally_total (0 without tallies)
};

// Batched contexts (several boxes in one context, one launch per phase for
// all of them).  Each box has its own fields, scalars, packet count and random
// streams (box index in the Philox counter); the library scratch of all boxes
// is concatenated and every box is described by one record.
constexpr int kMaxBoxes = 128;
constexpr int kPassCellsPerThread = 32;  // streaming-pass blocks per box: ceil(n^3 / (256 * 32))

struct BoxDev {
  // caller fields
  const void* delta;
  void* vel4;
  double* x;
  void* T;
  uint32_t* tally;
  void* emis;
  // library scratch of this box
  void* xy;            // mixed form: (x, 1 - x) cache [n3]
  uint32_t* P;         // packet prefix [n3 + 1]
  uint32_t* first;     // cell of packet 32 w [npk / 32 + 2]
  DevScalars* sc;      // scalars of this box
  int64_t n3;
  uint32_t n, lg, nt, p2;  // side, log2 side (power of two), super-tiles per axis, side is a power of two
  uint64_t mn, mn2;        // multipliers ceil(2^64/n), ceil(2^64/n^2) of the exact divisions (n >= 2)
  uint32_t tlg;            // log2 of the super-tile side in use
  uint64_t npk;        // packets requested per transport
  uint64_t pk0;        // first packet of the box in the batch packet space (multiple of 64)
  uint32_t ablk0;      // first allocation block
  uint32_t bk0;        // first march-queue bucket
  uint32_t pblk0;      // first block of the streaming passes
  uint32_t pblk;       // blocks of the streaming passes
};

// Transport scalars of one box at the redshift of a transport call.
struct BoxStep {
  double kappa, cth;
};

// Per-substep coefficients, computed on the host from the redshifts (no
// data dependence), passed by value.
struct StepCoef {
  double dt;      // cosmic time of the substep, s
  double H;       // Hubble rate at the substep end, 1/s
  double nH;      // mean hydrogen density at the substep end, 1/m^3
  double Tg;      // photon temperature at the substep end, K
  double kc;      // Compton heating coefficient 8 sigma_T a_R T^4/(3 m_e c), 1/s
  double kd;      // Compton drag coefficient per unit x: 4 sigma_T a_R T^4 (1-Y_p)/(3 c m_H), 1/s
  double hq;      // heating term numerator 2 Gamma_per_H/(3k), K/s
  double fHe;     // n_He/n_H
  double beta;    // photo-ionisation rate per 2s atom at T_gamma, 1/s
  double ea;      // exp(-E_alpha/kT_gamma)
  double KR;      // 8 pi H / lambda_alpha^3 (R_alpha = KR / n_1s)
  double L2g;     // two-photon rate
  double fa;      // fudge * 1e-19 * a of the case-B fit (m^3/s)
  double pb, pc, pd;  // remaining case-B fit constants
  int32_t mixing;
  int32_t last;   // 1 on the last substep of a rec_step
};

// Host-side cosmology of one context.
struct Cosmo {
  double H0, Om, Or, OL, nH0, T0, fHe, Yp, L_m, fudge, heat;
};

}  // namespace rec

struct rec_ctx {
  rec_params params;
  rec_box box;
  cudaStream_t stream;
  int64_t n3;
  rec::Cosmo cosmo;
  // device scratch owned by the context
  rec::DevScalars* sc;       // device scalars of the forward sweep
  rec::DevScalars* sc_adj;   // device scalars of the reverse sweep
  double* part;              // block partials [grid * kMaxSums]
  uint32_t* P;               // packet prefix [n3 + 1]
  uint32_t* first;           // cell of every 32nd packet [n_packets/32 + 1]
  void* xy;                  // mixed form: binary32 (x, 1 - x) cache of the state [n3]
  void* div;                 // local mixing: velocity divergence per cell, 1/s (float | double) [n3]
  unsigned long long* bcap;  // march-queue bucket capacities / offsets [super-tiles]
  unsigned long long* bfill; // packets queued per bucket [super-tiles]
  unsigned long long* cpre;  // first march chunk of each bucket [super-tiles + 1]
  unsigned long long* partQ; // allocation block sums / offsets [alloc blocks]
  void* quant;               // emission-profile table (float or double) [n_quantiles]
  int grid;                  // blocks of the streaming passes
  int alloc_blocks;
  int newton_tma = 0;        // TMA-staged Newton pass usable (0: not yet queried, 1 / -1)
  int batch_step_grid = 0;   // resident blocks of the persistent batched substep (0: not queried, -1: none)
  int batch_front_grid = 0;  // resident blocks of the persistent batched transport front (same)
  void* queue;               // queued packets of the march (2 x 16 B binary32, 3 x 32 B binary64) [n_packets]
  // region sweeps (tuning.march_halo > 0): packets leaving their region are
  // appended to rqueue (48 B binary32, 96 B binary64 entries), counted per
  // bucket in rcount, and placed by bucket into queue for the next sweep (scnt:
  // per-bucket fill of that placement)
  void* rqueue = nullptr;
  size_t rq_cap = 0;
  unsigned long long* rcount = nullptr;
  unsigned long long* scnt = nullptr;
  unsigned long long* rqn = nullptr;  // [2 kRqParts]: entries appended per part; entries to place per part
  int sm_count;
  bool emis_ready;
  std::string err;
  // optional kernel timing (rec_timing / rec_kernel_times)
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[REC_T_COUNT];
  std::vector<cudaEvent_t> pool;
  int64_t launches[REC_T_COUNT] = {0, 0, 0, 0, 0, 0, 0};
  rec_tuning tune;  // transport launch and scheduling parameters
  // graph-captured steps (rec_graph_step): the executable graph, updated in place
  cudaGraphExec_t gexec = nullptr;
  bool capturing = false;  // no timing events while a step is captured
  // batched context (n_boxes > 1); unused for one box
  int n_boxes = 1;
  std::vector<rec_box> boxes;
  std::vector<rec::BoxDev> hbx;  // host copy of the box records
  rec::BoxDev* bx = nullptr;     // device box records [n_boxes]
  rec::BoxStep* bstep = nullptr; // device transport scalars [n_boxes]
  rec::DevScalars* gsc = nullptr;// batch-wide counters (last-block-done, march chunks)
  int tot_ablk = 0;              // allocation blocks of all boxes
  int tot_pblk = 0;              // streaming-pass blocks of all boxes
  int tot_buckets = 0;           // march-queue buckets of all boxes
  uint64_t tot_pk = 0;           // batch packet space (each box padded to 64)
  // resonant-scattering Monte Carlo (lya_scatter_mc): Voigt nodes and counters
  void* mc_scratch = nullptr;
  size_t mc_bytes = 0;
  double mc_a = -1.0;            // Voigt parameter of the nodes held in mc_scratch
  // second-order step (rec_step_trbdf2): stage arrays and scalars
  void* trb_scratch = nullptr;
  size_t trb_bytes = 0;
  // mixing fraction of Monte-Carlo records (lya_mc_mixing_fraction): counters
  void* mf_cnt = nullptr;
  // polls before a bounded device-side wait gives up (rec_set_wait_limit)
  uint32_t wait_limit = rec::kDefaultWaitLimit;
};

namespace rec {

enum TimerGroup { kTAlloc = 0, kTEmit = 1, kTMarch = 2, kTEnd = 3, kTStep = 4, kTAdj = 5, kTOther = 6 };

// Scoped timer of one kernel group: records an event pair on the context
// stream when timing is on and counts the launches of the group.
struct GroupTimer {
  rec_ctx* c;
  int g;
  cudaEvent_t e0 = nullptr;
  GroupTimer(rec_ctx* ctx, int group, int n_launches) : c(ctx), g(group) {
    c->launches[g] += n_launches;
    if (c->timing && !c->capturing) { e0 = take(); cudaEventRecord(e0, c->stream); }
  }
  ~GroupTimer() {
    if (e0) {
      cudaEvent_t e1 = take();
      cudaEventRecord(e1, c->stream);
      c->ev[g].emplace_back(e0, e1);
    }
  }
  cudaEvent_t take() {
    if (!c->pool.empty()) { cudaEvent_t e = c->pool.back(); c->pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};

// rec_cosmo.h
Cosmo make_cosmo(const rec_params& p);
double hubble(const Cosmo& c, double z);
double nH_bar(const Cosmo& c, double z);
double T_gamma(const Cosmo& c, double z);
double cosmic_dt(const Cosmo& c, double z_from, double z_to);
void transport_scalars(const Cosmo& c, int n, double z, double* kappa, double* cth);
StepCoef step_coef(const Cosmo& c, const rec_params& p, double z_from, double z_to, int last);
double saha_S(double T);  // (2 pi m_e k T/h^2)^{3/2} exp(-E_ion/kT), 1/m^3
double thomson_sigma_c(); // sigma_T c, m^3/s

// rec_step.cu
cudaError_t launch_state_init(rec_ctx* c, double z);
cudaError_t launch_refresh(rec_ctx* c, double z);
cudaError_t launch_rec_step(rec_ctx* c, double z_from, double z_to, rec_stats* st);
// X_e, lambda and S_1s of the current state of every box into st.
cudaError_t launch_volume_stats(rec_ctx* c, rec_stats* st);
// Synchronises the stream; *timed_out = 1 if a bounded device wait expired
// since the last check (flags bit 3 of any box), clearing it and the counters.
cudaError_t launch_check_waits(rec_ctx* c, int* timed_out);
// Context-free FP64 step on static device scratch; no device allocation.
rec_status launch_rec_step_noalloc(const rec_params& p, const rec_box& b, double z_from, double z_to,
                                   cudaStream_t stream, rec_stats* st, std::string* why);
// Newton passes for lambda of a substep on an arbitrary FP64 state (used by the adjoint).
void enqueue_newton_passes(rec_ctx* c, DevScalars* sc, const StepCoef& k, const double* x, const double* T,
                           const uint32_t* tally);

// rec_transport.cu
cudaError_t launch_transport(rec_ctx* c, int step, double z, rec_stats* st);
cudaError_t launch_transport_batch(rec_ctx* c, int step, double z, rec_stats* st);
void transport_limits(bool mixed, bool batch, int* emit_max, int* march_max);
// Largest march grid (blocks per SM) of the region-sweep march.
int sweep_march_limit(bool mixed);
constexpr int kMaxSweeps = 8;  // region sweeps per transport call (the last without a limit)
// The second queue is split into parts, each with its own append counter, so
// that the warps of the march do not all add to one address.
constexpr int kRqParts = 256;

// rec_step.cu, batched contexts
cudaError_t launch_state_init_batch(rec_ctx* c, double z);
cudaError_t launch_refresh_batch(rec_ctx* c, double z);
cudaError_t launch_rec_step_batch(rec_ctx* c, double z_from, double z_to, rec_stats* st);

// rec_scatter.cu: resonant-scattering Monte Carlo (Appendix A)
struct McSetup {
  double a;         // Voigt parameter Gamma / (2 omega_alpha v_th)
  double vth;       // sqrt(2 k T_gamma / m_H) / c
  double sig0;      // <sigma> = sig0 H(a, y), m^2
  double dxdl;      // frequency drift per physical metre, zeta H / (c v_th)
  double cpm;       // comoving cells per physical metre
  double ufac;      // Doppler units per km/s of peculiar velocity
  double p_ion, p_2g;  // fates per scattering
  double beta, Lam, Heff, nH, Tg;
  double expm_eps;  // exp(-eps)
  double kpc_cell;  // comoving kpc per cell
};
bool scatter_setup(const Cosmo& c, const rec_params& p, int n, const lya_mc_params* mp, McSetup* S);
void scatter_voigt_host(double a, int64_t m, const double* y, double* H);
void scatter_voigt_mixed_host(double a, int64_t m, const double* y, double* H);
uint64_t scatter_redistribution_mixed_host(double a, double y, const double* kin, uint64_t seed, int64_t m,
                                           double* ppar, double* dy, double* kout);
cudaError_t run_scatter_mc(rec_ctx* c, const McSetup& S, const lya_mc_params* mp, const uint32_t* prefix,
                           lya_mc_photon* out, lya_mc_stats* st);
constexpr int kMixFracMax = 256;  // distances per lya_mc_mixing_fraction call
cudaError_t run_mixing_fraction(rec_ctx* c, const lya_mc_photon* rec, uint64_t n, const double* D, int m,
                                double* out, uint64_t* counts);

// rec_trbdf2.cu: second-order (TR-BDF2) step, FP64 form, tally and full mixing
cudaError_t launch_rec_step_trbdf2(rec_ctx* c, double z_from, double z_to, rec_stats* st);

// rec_adjoint.cu
cudaError_t launch_rec_step_adjoint(rec_ctx* c, double z_from, double z_to, const double* x_in, const double* T_in,
                                    const double* vel4_in, const uint32_t* tally_in, double* xbar, double* Tbar,
                                    double* Ubar, double* g_delta, double* g_a, double Xe_bar_out);
cudaError_t launch_xe_adjoint(rec_ctx* c, const double* x, double Xe_bar, double* xbar, double* g_delta);

}  // namespace rec
