/*
 * rec.h -- C ABI of the GB300 recombination hot path.
 *
 * Implements, for a periodic box of n^3 cells, the two data-parallel parts of
 * the recombination step of Jedamzik, Abel & Ali-Haimoud, "Cosmic
 * Recombination in the Presence of Primordial Magnetic Fields"
 * (arXiv:2312.11448):
 *
 *   lya_transport  Monte-Carlo Ly-alpha packets emitted per cell in proportion
 *                  to the local recombination rate alpha_e n_e^2 (Sec. III.B and
 *                  its footnote on the global loss-rate integral), streamed along
 *                  isotropic directions while the Hubble expansion redshifts them
 *                  (Appendix A, step (4): dx = -H dl / v_th) with the bulk-flow
 *                  Doppler shift omega_r = omega (1 - U_par) (Appendix A), and
 *                  absorbed into integer per-cell tallies where they come back
 *                  into line resonance.
 *   rec_step       the per-cell effective three-level-atom update of x_e
 *                  (Eq. rec0 with the 2s population of Eq. n2s-sol; full-mixing
 *                  rate Eq. dotne-mix, Sec. IV.B) and of T_b (Eq. Tb-evolution),
 *                  plus Compton drag on the peculiar velocity (Eq. alpha-def in
 *                  Eq. momentum).
 *   rec_step_adjoint  the reverse (adjoint) of rec_step with the tallies held
 *                  fixed, for gradients of X_e (Sec. II.A) and of the visibility
 *                  function.
 *   lya_scatter_mc the paper's own resonant-scattering Monte Carlo (Appendix A):
 *                  single photons scattered on neutral hydrogen (Eq. MC, Eq. inout)
 *                  until they are lost by redshifting or destroyed, with their
 *                  travel distances.
 *
 * Conventions (all entry points)
 *   - Every call returns a rec_status; no C++ exception crosses the ABI.
 *     On failure, rec_last_error(ctx) describes the cause.
 *   - Field buffers are DEVICE pointers owned by the caller.  They must stay
 *     valid until rec_free.  The context owns its own scratch (packet prefix,
 *     reduction partials, device scalars, the emission-profile table).
 *   - Cells are indexed c = (iz*n + iy)*n + ix; the box is periodic.
 *   - All work is enqueued on the stream given to rec_init; calls return
 *     without synchronising (results are valid once the stream reaches them).
 *     Device-side counters and statistics go to a device rec_stats record.
 *   - Precision forms: REC_PREC_FP64 stores delta, vel4, T, emis in double and
 *     runs all arithmetic in binary64; REC_PREC_MIXED stores them in float,
 *     streams packets in binary32, and keeps x_e, the net
 *     recombination-minus-photoionisation difference and the volume sums in
 *     binary64.  x_e is double in both forms.
 */
#ifndef REC_H
#define REC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rec_ctx rec_ctx; /* opaque; created by rec_init, owned by the library */

typedef enum {
  REC_OK = 0,
  REC_EINVAL = 1,   /* invalid argument: NULL pointer, bad size or mode */
  REC_ENOMEM = 2,   /* device or host allocation failed */
  REC_ECUDA = 3,    /* a CUDA call failed; message in rec_last_error */
  REC_ETIMEOUT = 4, /* a bounded device-side wait expired */
  REC_ESTATE = 5    /* call out of order (e.g. transport before emission weights exist) */
} rec_status;

typedef enum { REC_PREC_FP64 = 0, REC_PREC_MIXED = 1 } rec_precision;

/* REC_MIX_TALLY: the local 2s population follows the Ly-alpha packets absorbed
 *   in each cell during this step's transport (J_i proportional to absorptions
 *   per neutral atom).  REC_MIX_FULL: the paper's full-mixing limit,
 *   Eq. dotne-mix (tallies unused).  REC_MIX_LOCAL: the no-mixing limit of
 *   Sec. III.A.2 — Eq. rec per cell with the cell's own n_e and n_1s and
 *   Eq. R-alpha with H -> H + div v / 3 (div v by periodic central differences
 *   of the substep-start velocities; no escape where H + div v / 3 < 0); tallies
 *   unused.  REC_MIX_PARTIAL: the share f_alpha of the full-mixing rate plus
 *   1 - f_alpha of the local one (the partial mixing of Sec. V with the mixing
 *   fraction of Sec. III.B, given here as a parameter); lambda stays
 *   self-consistent.  REC_MIX_LOCAL and REC_MIX_PARTIAL need a single-box
 *   context and have no adjoint. */
typedef enum { REC_MIX_TALLY = 0, REC_MIX_FULL = 1, REC_MIX_LOCAL = 2, REC_MIX_PARTIAL = 3 } rec_mixing;

typedef struct {
  /* Cosmology, Sec. II.C defaults: 0.67, 0.0224, 0.12, 0.24. */
  double h, omega_b_h2, omega_c_h2, Y_p;
  double T_cmb0;     /* K; not printed in the paper (2.7255 is the usual value) */
  double N_eff;      /* not printed in the paper (3.046) */
  double L_box_kpc;  /* comoving box side; 24 in Sec. II.C */
  double fudge;      /* 1.14, multiplies the case-B coefficient (Sec. III.A.1) */
  double heating;    /* uniform heating Gamma (Sec. VI) per mean hydrogen atom, eV/s; 0 = off */
  uint64_t seed;     /* Philox key for the packet streams */
  int32_t n_sub;     /* backward-Euler substeps per rec_step (>= 1) */
  int32_t precision; /* rec_precision */
  int32_t mixing;    /* rec_mixing */
  int32_t n_quantiles;               /* >= 2 */
  const double* emission_quantiles;  /* HOST array [n_quantiles]: inverse CDF of the
                                        emission-frequency profile in Doppler units at
                                        (k+1/2)/n_quantiles; copied at rec_init */
  double f_alpha;    /* REC_MIX_PARTIAL: share of the full-mixing rate, in [0, 1] (0 = local,
                        1 = full); read in that mode only */
} rec_params;

typedef struct {
  int32_t n;          /* cube side, 1 <= n <= 1024 */
  void* delta;        /* overdensity rho_b/<rho_b> [n^3]: float (MIXED) | double (FP64); read-only */
  void* vel4;         /* peculiar velocity {Ux,Uy,Uz,unused} km/s [n^3]: float4 | double4;
                         32-byte aligned (cudaMalloc's alignment; REC_EINVAL otherwise);
                         updated by rec_step (Compton drag) */
  double* x_e;        /* ionisation fraction n_e/n_H [n^3]; updated by rec_step */
  void* T;            /* baryon temperature K [n^3]: float | double; updated by rec_step */
  uint32_t* tally;    /* absorbed packets per cell [n^3]; lya_transport adds, rec_step zeroes */
  void* emis;         /* emission weight alpha_e n_e^2 [n^3]: float | double; written by
                         rec_state_init / rec_refresh / rec_step, read by lya_transport */
  uint64_t n_packets; /* packets emitted per lya_transport call, < 2^32 */
} rec_box;

/* Device-side statistics record (caller-owned device memory; one per box of a
 * batched context). */
typedef struct {
  uint64_t emitted, absorbed, capped, crossings; /* transport counters of the last call */
  uint64_t queued;  /* packets that left their home cell (marched by the second kernel) */
  double X_e;     /* <rho_b x_e>/<rho_b> after the last rec_step (Sec. II.A) */
  double lambda;  /* <alpha_e n_e^2>/<n_1s> at the end state, 1/s */
  double C_mix;   /* Peebles factor with R_alpha -> R_alpha^mix (Eq. Cfactor, Sec. IV.B);
                     REC_MIX_LOCAL: the volume mean of the cells' own factors */
  double S1s;     /* sum over cells of delta (1 - x_e) at the end state */
  int32_t newton_passes; /* Newton evaluations of the last substep */
  int32_t flags;         /* bit 0: Newton did not converge; bit 1: packets hit the crossing cap;
                            bit 2: non-finite or negative emission weight; bit 3: a bounded
                            device-side wait expired (copy pipeline of a Newton pass); bit 4:
                            region sweeps found their second queue full (the packets concerned
                            marched on without a region limit: results unchanged, speed only) */
  uint64_t requeued;     /* region sweeps (rec_tuning.march_halo > 0): packets queued again for a
                            later sweep in the last lya_transport call; 0 otherwise */
} rec_stats;

/* Launch and scheduling parameters of the transport: a library setting with
 * no counterpart in the paper.  They change only the speed: tallies, counters
 * and every other result are identical for any valid setting. */
typedef struct {
  int32_t emit_blocks_per_sm;  /* emission grid, blocks of 256 threads per SM: 1..5 (FP64 form and batch 1..4) */
  int32_t march_blocks_per_sm; /* march grid: 1..4 (FP64 form and batch 1..3); with march_halo > 0
                                  1..3 (FP64 form 1..2) */
  int32_t march_refill;        /* idle lanes of a warp that trigger a refill from the queue: 1..32 */
  int32_t march_chunk;         /* queued packets per unit of march work handed to a warp: 8..4096 */
  int32_t tile;                /* side of the super-tiles that order the march queue: 8, 16, 32 or 64 */
  int32_t march_halo;          /* region sweeps (single box, power-of-two side): 0 = off, every packet
                                  marches to its end in one launch; h in 1..256 = a packet marches only
                                  while it stays within h cells of the super-tile whose bucket it was
                                  taken from, then is queued again in the bucket of the super-tile it
                                  has reached, for the next of up to 8 sweeps (the last sweep has no
                                  limit).  Each sweep then touches a region that the L2 cache holds,
                                  which pays on boxes whose velocities are far larger than L2.  The
                                  first rec_set_tuning with h > 0 allocates the second queue
                                  (n_packets / 4 entries of 48 B, 96 B in the FP64 form); packets that
                                  find it full march on without a limit. */
} rec_tuning;

/* Create a context for n_boxes independent boxes (1 <= n_boxes <= 128), each
 * with its own side, fields and packet count; all share params (cosmology,
 * precision form, mixing mode, seed).  With n_boxes > 1 the work of all boxes
 * is done together: lya_transport is one persistent cooperative launch for the
 * allocation and the emission (its phases separated by grid barriers whose
 * waits are bounded, see rec_set_wait_limit) followed by the march, and
 * rec_step is one persistent cooperative launch per substep (the Newton
 * evaluations and the final pass as its phases), so a step is three launches;
 * box b draws its random numbers with box index b in the Philox counter
 * (box 0 therefore reproduces a single-box context bit for bit), keeps its own
 * sums, lambda and Newton state, and the dev_stats arguments of lya_transport
 * and rec_step point to n_boxes records, one per box.  The adjoint entry points
 * need a single-box context.
 * Validates params and buffers, copies the emission-profile table, allocates
 * scratch.  Does not touch the field buffers.
 * Errors: REC_EINVAL (message names the offending box), REC_ENOMEM, REC_ECUDA. */
rec_status rec_init(const rec_params* params, const rec_box* boxes, int32_t n_boxes, void* cuda_stream,
                    rec_ctx** out);

/* Initial state at redshift z: T = T_gamma(z) and x_e from the hydrogen Saha
 * equation per cell (T_b = T_gamma), then the emission weights as rec_refresh. */
rec_status rec_state_init(rec_ctx* ctx, double z);

/* Recompute the emission weights alpha_e(T) n_e^2 and the volume sums from the
 * current x_e, T at redshift z.  Needed once after the caller writes x_e or T
 * directly; rec_step keeps them current otherwise. */
rec_status rec_refresh(rec_ctx* ctx, double z);

/* Ly-alpha packet transport at redshift z for step index `step` (keys the
 * random streams): Sec. III.B (packets in proportion to alpha_e n_e^2),
 * Appendix A steps (1) and (4) and omega_r = omega (1 - U_par).  Emits
 * n_packets packets (allocation proportional to emis; emis, T and vel4 are read,
 * not written), marches each to its resonance cell and adds it to tally
 * (uint32, caller-owned; rec_step zeroes it).  The result does not depend on
 * rec_tuning.  Counters go to dev_stats (device pointer, may be NULL).
 * Errors: REC_ESTATE if emission weights were never computed; REC_ECUDA. */
rec_status lya_transport(rec_ctx* ctx, int32_t step, double z, rec_stats* dev_stats);

/* One recombination step z_from -> z_to (z_from > z_to) in n_sub backward-Euler
 * substeps, using the tallies of this step (TALLY mode); zeroes the tallies and
 * writes the emission weights for the next transport.  Statistics go to
 * dev_stats (device pointer, may be NULL).
 * Errors: REC_EINVAL (z order), REC_ESTATE, REC_ECUDA. */
rec_status rec_step(rec_ctx* ctx, int32_t step, double z_from, double z_to, rec_stats* dev_stats);

/* lya_transport(step, z_from) followed by rec_step(step, z_from, z_to), enqueued
 * as one CUDA graph: the call captures both on the context stream, updates the
 * executable graph it keeps from the previous call in place (the launch
 * sequence of a step never changes, only kernel parameters do) and launches
 * it.  Results are those of the two calls.  dev_stats receives the transport
 * counters and the rec_step statistics (n_boxes records for a batch).
 * Requires a context created on a non-default stream, kernel timing off, and
 * a stream that is not already being captured.
 * Errors: REC_EINVAL, REC_ESTATE, REC_ECUDA. */
rec_status rec_graph_step(rec_ctx* ctx, int32_t step, double z_from, double z_to, rec_stats* dev_stats);

/* Second-order variant of rec_step: each of the n_sub substeps is one TR-BDF2
 * step (Bank et al. 1985) of the same per-cell system (Eq. dotne-mix per
 * hydrogen atom, Eq. Tb-evolution, drag of Eq. alpha-def).  A trapezoidal
 * stage to t + gamma h (gamma = 2 - sqrt 2) is followed by a BDF2 stage to
 * t + h. Each stage end is fully implicit in x_e, T_b, lambda and the Peebles factor;
 * an outer fixed point over T_b, alpha(T_b) and C converges to 1e-14 relative.
 * Coefficients are taken at their own times, and the drag uses the trapezoidal
 * exponent.  Global error falls as the square of the step (backward Euler: linearly).  Same
 * outputs as rec_step: state, emission weights, tallies zeroed, statistics (flags bit 0: a stage did
 * not converge within its launches or had no positive root).  Single-box
 * context, FP64 form, tally or full mixing.  Scratch: 7 doubles per cell,
 * allocated on first use.  Meant for states near the quasi-equilibrium a run
 * reaches: with steps longer than the cells' relaxation time, a start far from
 * it can make the trapezoidal stage infeasible (it overshoots to about
 * 2 x_eq - x_n; flags bit 0 is set) or, far above ionisation equilibrium,
 * give stage equations with more than one solution.
 * Errors: REC_EINVAL, REC_ESTATE (no state yet), REC_ENOMEM, REC_ECUDA. */
rec_status rec_step_trbdf2(rec_ctx* ctx, int32_t step, double z_from, double z_to, rec_stats* dev_stats);

/* Partial mixing: set the share f_alpha of the full-mixing rate (REC_MIX_PARTIAL
 * contexts) for the following rec_step and rec_graph_step calls.  Sec. V takes
 * the share from the Monte-Carlo mixing fraction f_alpha(D) of Sec. III.B (the
 * fraction of Ly-alpha photons destroyed farther than D from where they were
 * emitted), which changes with redshift; lya_scatter_mc and
 * lya_mc_mixing_fraction give it.  f_alpha = 0 runs the local (no-mixing) limit
 * of REC_MIX_LOCAL and f_alpha = 1 full mixing.  The kernels a step launches
 * differ between f_alpha = 0 and f_alpha > 0, so the next rec_graph_step after
 * the share crosses zero re-instantiates its executable graph.  Host-side
 * only: takes effect from the next call enqueued.
 * Errors: REC_EINVAL (not a partial-mixing context, f_alpha outside [0, 1]). */
rec_status rec_set_f_alpha(rec_ctx* ctx, double f_alpha);

/* Current transport tuning of a context (defaults after rec_init). */
rec_status rec_get_tuning(const rec_ctx* ctx, rec_tuning* out);

/* Set the transport tuning; takes effect from the next lya_transport.
 * Synchronises the context stream (a set-up call, not for inside a step).
 * Errors: REC_EINVAL (a field out of range, march_halo > 0 on a batched context
 * or a box side that is not a power of two; nothing changed), REC_ENOMEM (the
 * second march queue of the region sweeps), REC_ECUDA. */
rec_status rec_set_tuning(rec_ctx* ctx, const rec_tuning* tuning);

/* Allocation-free step.  The paper has no counterpart: this is a library entry
 * point for callers that cannot allocate device memory while they step, such as
 * a host code whose own pool allocator has taken all device memory at start-up
 * (a cudaMalloc would fail) or one whose loop cannot afford the implicit device
 * synchronisation of cudaMalloc/cudaFree.  It needs no rec_ctx and performs the
 * same passes as rec_refresh(z_from) followed by rec_step(z_from, z_to) on a
 * context created for *box: the sums and emission weights of the incoming
 * state, then n_sub backward-Euler substeps of Eq. (dotne-mix) and the T_b /
 * drag update, in TALLY or FULL mixing.
 *   params: as for rec_init; precision must be REC_PREC_FP64 (the mixed form
 *     keeps a per-cell cache that a static array of modest size cannot hold).
 *   box: field buffers as for rec_init (n in [1, 1024]; n_packets unused);
 *     x_e, T, vel4, emis are updated in place, tallies zeroed at the end.
 *   cuda_stream: a stream of the current device (NULL: legacy default stream).
 *   dev_stats: device-visible rec_stats (may be NULL), written at the end.
 * Scratch: a static device array of 130 KiB per device (one scalar record and
 * per-block partial sums for at most 2048 blocks).  The step uses
 * min(ceil(n^3/256), 8 x SM count) blocks and is rejected with REC_EINVAL when
 * that exceeds 2048.  The first call on a device does the set-up (it looks up
 * the array's device address, which may load the module), so make it before
 * any stream capture.  Each call clears the scalar record on the stream first.
 * Calls that overlap in time on one device (several streams or host threads)
 * share the array and race: serialise them.  The array's device address is
 * looked up once per device and kept for the process: do not use this entry
 * point after a cudaDeviceReset of that device.
 * Errors: REC_EINVAL, REC_ECUDA; rec_last_error(NULL) gives the cause. */
rec_status rec_step_noalloc(const rec_params* params, const rec_box* box, double z_from, double z_to,
                            void* cuda_stream, rec_stats* dev_stats);

/* Reverse of rec_step (FP64 form only), tallies held fixed.
 *   x_in, T_in, vel4_in: the state BEFORE the step (device, FP64 layouts);
 *   tally_in: this step's tallies (device u32 [n^3], may be NULL in FULL mode).
 *   xbar, Tbar: in = adjoint of the state after the step, out = before (device f64 [n^3]);
 *   Ubar: adjoint of vel4 (device double4 [n^3], in/out) or NULL if zero;
 *   g_delta, g_a: accumulated (+=) gradients with respect to the overdensity and to
 *   the absorbed-Ly-alpha fraction a_i = tally_i / sum(tally) of this step
 *   (device f64 [n^3]);
 *   Xe_bar_out: adjoint of X_e at the step's end node (added before reversing).
 * Errors: REC_EINVAL (precision or z order), REC_ECUDA. */
rec_status rec_step_adjoint(rec_ctx* ctx, int32_t step, double z_from, double z_to, const double* x_in,
                            const double* T_in, const double* vel4_in, const uint32_t* tally_in, double* xbar,
                            double* Tbar, double* Ubar, double* g_delta, double* g_a, double Xe_bar_out);

/* Adds the adjoint of X_e = sum(delta x)/sum(delta) at a node to xbar and g_delta
 * (the start node of a trajectory; rec_step_adjoint handles its end node). */
rec_status rec_xe_adjoint(rec_ctx* ctx, const double* x, double Xe_bar, double* xbar, double* g_delta);

/* Statistics of the current state, for the start node of a trajectory: writes
 * X_e = sum delta x / sum delta (Sec. II.A), lambda = <alpha_e n_e^2>/<n_1s> and
 * S1s of each box (n_boxes records) from the sums of the last rec_state_init,
 * rec_refresh or rec_step; the other fields of the records are left as they are.
 * Errors: REC_EINVAL, REC_ESTATE (no sums yet), REC_ECUDA. */
rec_status rec_volume_stats(rec_ctx* ctx, rec_stats* dev_stats);

/* Bound of the device-side waits (no counterpart in the paper).  Every wait
 * inside a kernel is bounded: a bulk-copy stage of the per-cell passes is
 * looked at once without blocking, then polled at most `polls` times (default
 * 2^22, about a second); past that the block records the expiry (rec_stats
 * flags bit 3) and returns without finishing its share of the pass.  The wait
 * for its copies still in flight before such a return keeps the default bound.
 * The grid barriers between the phases of the persistent batched launches
 * (see rec_init) poll at most `polls` times as well.  0 makes every such wait
 * give up at once, which is how the error path is tested.  Host-side only: takes effect from the next call
 * enqueued.  Errors: REC_EINVAL (NULL context). */
rec_status rec_set_wait_limit(rec_ctx* ctx, uint32_t polls);

/* Waits for the context stream and reports the device-side failures of the
 * calls enqueued since the last rec_sync: REC_ETIMEOUT if a bounded wait
 * expired (see rec_set_wait_limit).  The state those calls left is then
 * incomplete: re-initialise it (zero the tallies; rec_state_init, or write x_e
 * and T and call rec_refresh) before stepping again; rec_sync clears the expiry and the
 * device counters a pass that gave up may have left part-way, so the context
 * stays usable.  Errors: REC_ETIMEOUT, REC_ECUDA. */
rec_status rec_sync(rec_ctx* ctx);

/* Objective on an X_e history over node redshifts zs[0..n_nodes-1] (decreasing),
 * host computation.  objective 1: X_e at the node nearest z_star.  objective 2:
 * the visibility function g = (d tau/dz) exp(-tau) at that node, with the Thomson
 * optical depth tau(z) = int sigma_T c nbar_H X_e / ((1+z) H) dz from the last
 * node (trapezoid on the nodes).  Writes J and dJ/dX_e at every node.
 * Errors: REC_EINVAL. */
rec_status rec_objective(const rec_params* params, const double* zs, const double* Xe, int32_t n_nodes,
                         int32_t objective, double z_star, double* J, double* dJ_dXe);

/* Transport scalars at redshift z for an n^3 box (host computation, no GPU
 * needed): out[0] = kappa = n / (H a L), cells of Hubble drift per km/s of
 * velocity; out[1] = cth = kappa^2 2 k_B / m_H, so that the thermal velocity
 * v_th = sqrt(2 k T / m_H) of Appendix A is sqrt(T cth) cells.
 * Errors: REC_EINVAL. */
rec_status rec_transport_params(const rec_params* params, int32_t n, double z, double* out);

/* Kernel timing, a measurement aid.  rec_timing(ctx, 1) clears the counters and
 * starts recording CUDA events on the context stream around each kernel group;
 * rec_timing(ctx, 0) stops.  rec_kernel_times synchronises the stream and
 * writes, per group, the summed device time in ms and the number of kernels
 * launched since the last clear (arrays of REC_T_COUNT).  Groups:
 *   0  packet allocation (3 kernels per lya_transport)
 *   1  packet emission and home-cell test (1 kernel)
 *   2  march of the queued packets (1 kernel)
 *   3  transport bookkeeping (1 kernel)
 *   4  rec_step passes (begin, Newton, final per substep)
 *   5  rec_step_adjoint passes
 *   6  rec_state_init / rec_refresh / rec_xe_adjoint */
#define REC_T_COUNT 7
rec_status rec_timing(rec_ctx* ctx, int32_t enable);
rec_status rec_kernel_times(rec_ctx* ctx, double* ms_out, int64_t* launches_out);

/* ---- Resonant-scattering Ly-alpha Monte Carlo (Appendix A) ------------------
 * Single photons followed through their scatterings on neutral hydrogen in
 * the box's density, ionisation and velocity fields at one redshift: steps
 * (1)-(8) of Appendix A.  A photon is injected at line centre in the gas frame
 * of its cell, at a uniform point of the cell, along an isotropic direction.
 * Each step evaluates the thermally averaged cross-section of Eq. MC,
 * <sigma> = (3 lambda_alpha^2 / 8 pi) 4 a sqrt(pi) H(a, y), in the cell the
 * photon is in (H the Voigt function, y the gas-frame offset in Doppler units
 * v_th = sqrt(2 k T_gamma / m_H), a = Gamma_alpha / (2 omega_alpha v_th)).
 * It advances eps mean free paths, redshifts by dx = -zeta H dl / v_th, and
 * scatters with probability 1 - exp(-eps).  At a scattering the n = 2 atom
 * (2s and 2p in statistical equilibrium, Sec. III.A.1) is photo-ionised,
 * decays by two photons or re-emits, with weights beta_e : Lambda : 3 A_alpha.
 * A re-emitted photon takes the frequency of Eq. inout (isotropic
 * scattering, the atom's velocity drawn from the third factor of Eq. MC).
 * A photon whose gas-frame offset falls below -x_lost is lost by redshifting.
 * T = T_gamma(z) throughout.  The arithmetic is set by lya_mc_params.arith
 * (binary64 by default) independently of the context's precision form; the
 * box's fields are read in their stored types. */
typedef struct {
  double z;          /* redshift of the snapshot (> 0) */
  double eps;        /* step (3): path of eps mean free paths per step, (0, 1] */
  double x_lost;     /* loss threshold on the red wing, Doppler units (> 0) */
  double zeta;       /* expansion rate zeta H (> 0; 1 for the true rate, Fig. Cfact varies it) */
  double lambda2g;   /* two-photon rate, 1/s (>= 0); negative: 8.22 (Sec. III.A.1) */
  double A_alpha;    /* 2p -> 1s decay rate Gamma_alpha, 1/s (> 0; about 6.3e8) */
  uint64_t n_photons;  /* photons, 1 .. 2^32 - 1 */
  uint64_t max_steps;  /* per photon (>= 1); a photon reaching it ends as LYA_MC_CAPPED */
  int32_t step;        /* keys the random streams (with rec_params.seed) */
  int32_t pending;     /* lanes of a warp waiting to scatter before the warp runs the
                          redistribution for them, 1..32; 0: 12.  Speed only: results
                          do not depend on it. */
  int32_t arith;       /* LYA_MC_FP64 (0): binary64 throughout, the oracle's operation
                          order.  LYA_MC_MIXED (1): binary32 with double-float pairs for
                          the position inside the cell and the frequency, and integer
                          thresholds for the scattering and fate decisions;
                          statistically equivalent, not operation-for-operation equal. */
  int32_t reserved;    /* 0 */
} lya_mc_params;

enum { LYA_MC_FP64 = 0, LYA_MC_MIXED = 1 };

enum { LYA_MC_LOST = 0, LYA_MC_TWO_PHOTON = 1, LYA_MC_IONISED = 2, LYA_MC_CAPPED = 3 };

typedef struct {
  uint32_t home, j;   /* emitting cell and index of the photon in that cell */
  int32_t fate;       /* LYA_MC_* */
  uint32_t reserved;
  uint64_t n_scat;    /* scatterings, the last one included */
  uint64_t n_steps;
  double D_kpc;       /* comoving distance from injection to the end point */
  double x_end;       /* final frequency offset, Doppler units, frame without peculiar velocity */
} lya_mc_photon;

typedef struct {
  uint64_t count[4];     /* photons per fate (LYA_MC_*) */
  uint64_t sampler_caps; /* atom-velocity draws that hit their rejection cap (0 in practice) */
  uint64_t steps, scatterings;
  uint64_t nonfinite;    /* photons ended because their state stopped being finite (counted as CAPPED) */
} lya_mc_stats;

/* Run mp->n_photons photons through the Monte Carlo in the fields of a
 * single-box context (delta, x_e, vel4 as they are when the stream reaches
 * the call).  Photon k belongs to the cell c with dev_prefix[c] <= k <
 * dev_prefix[c + 1] (device u32 [n^3 + 1], non-decreasing, dev_prefix[0] = 0,
 * dev_prefix[n^3] = n_photons), or, with dev_prefix NULL, to the even
 * allocation prefix_c = floor(c n_photons / n^3).  Photon (c, j) draws from the
 * Philox stream with key (seed low word, seed high word XOR step) and counter
 * (c, j, block, 2^31).  dev_photons (device, n_photons records, may be NULL)
 * receives one record per photon in photon order; dev_stats (device, may be
 * NULL) the totals.  Needs x_e < 1 and delta > 0 in the cells photons visit.
 * Errors: REC_EINVAL (argument out of range, batched context), REC_ENOMEM,
 * REC_ECUDA. */
rec_status lya_scatter_mc(rec_ctx* ctx, const lya_mc_params* mp, const uint32_t* dev_prefix,
                          lya_mc_photon* dev_photons, lya_mc_stats* dev_stats);

/* The mixing fraction f_alpha(D) of Sec. III.B (its Fig. MCtravel) from the
 * records of lya_scatter_mc: among the photons destroyed in the line
 * (two-photon decay or photo-ionisation of the n = 2 atom, the fates that end
 * a Ly-alpha photon's energy locally), the fraction whose comoving distance from
 * the emission point exceeds D.  Sec. V uses f_alpha at D = 3 kpc as the share of
 * full mixing (rec_set_f_alpha).  Photons lost by redshifting are not
 * destroyed and do not count.  Photons stopped by the step cap (LYA_MC_CAPPED)
 * would still be destroyed or lost later, so they are reported separately.
 *   dev_photons: device records [n_photons] of lya_scatter_mc (1 <= n_photons < 2^32).
 *   D_kpc: HOST array [m] of distances, comoving kpc, finite and >= 0, 1 <= m <= 256;
 *     read during the call.
 *   dev_out: DEVICE double [3 m]: dev_out[j] = B_j / N_d, with B_j the destroyed
 *     photons farther than D_j and N_d all destroyed photons (NaN if N_d = 0);
 *     dev_out[m + j] = B_j / (N_d + N_c) and dev_out[2 m + j] = (B_j + N_c) / (N_d + N_c),
 *     N_c the capped photons: the range f_alpha(D_j) can take whatever the capped
 *     photons' fates would have been.
 *   dev_counts: DEVICE uint64 [4] (may be NULL): photons per fate (LYA_MC_*).
 * Counts are integers, so the result does not depend on the launch.  Scratch:
 * 2 KiB of counters, allocated by the context on first use.
 * Errors: REC_EINVAL, REC_ENOMEM, REC_ECUDA. */
rec_status lya_mc_mixing_fraction(rec_ctx* ctx, const lya_mc_photon* dev_photons, uint64_t n_photons,
                                  const double* D_kpc, int32_t m, double* dev_out, uint64_t* dev_counts);

/* Scalars of a Monte-Carlo snapshot as lya_scatter_mc uses them (host
 * computation, no GPU needed): out[0] = a, out[1] = v_th / c,
 * out[2] = sig0 (m^2; <sigma> = sig0 H(a, y)), out[3] = frequency drift per
 * physical metre zeta H / (c v_th), out[4] = p_ion and out[5] = p_2gamma
 * (fates per scattering), out[6] = beta_e, out[7] = Lambda_2gamma,
 * out[8] = zeta H, out[9] = nbar_H (1/m^3), out[10] = T_gamma,
 * out[11] = comoving cells per physical metre of an n^3 box.
 * Errors: REC_EINVAL. */
rec_status lya_mc_scalars(const rec_params* params, const lya_mc_params* mp, int32_t n, double* out);

/* The redistribution of the LYA_MC_MIXED form (Eq. inout, isotropic; the
 * same source compiled for the host): m independent scatterings of a photon at
 * gas-frame offset y travelling along kin (host double[3], not normalised),
 * with the random streams of photon (i, i >> 32) of seed.  Outputs (host, may be NULL):
 * ppar[i] = scattering atom's parallel velocity, dy[i] = y_out - y,
 * kout[3i..3i+2] = outgoing direction; caps (may be NULL) = draws that hit the
 * rejection cap.  Host computation, for checking the kernel's sampler on a CPU.
 * Errors: REC_EINVAL. */
rec_status lya_mc_redistribution_host(double a, double y, const double* kin, uint64_t seed, int64_t m,
                                      double* ppar, double* dy, double* kout, uint64_t* caps);

/* The Voigt function H(a, y) as lya_scatter_mc evaluates it (cubic Hermite
 * interpolation of nodes spaced 1/128 for |y| < 10, the asymptotic series of
 * the Faddeeva function beyond), at m host points y; host computation.
 * Errors: REC_EINVAL. */
rec_status lya_voigt(double a, int64_t m, const double* y, double* H);

/* The same for the LYA_MC_MIXED form: binary32 nodes and interpolation for
 * |y| < 10, the first-order wing series (a / sqrt(pi)) sum_k (2k+1)!! /
 * (2^k y^(2k+2)) beyond; host computation.  Errors: REC_EINVAL. */
rec_status lya_voigt_mixed(double a, int64_t m, const double* y, double* H);

/* Release the context and its scratch (NULL-safe).  Synchronises the stream. */
void rec_free(rec_ctx* ctx);

/* Last error message of ctx, or of the last failed rec_init when ctx is NULL. */
const char* rec_last_error(const rec_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* REC_H */
