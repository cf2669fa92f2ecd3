// C ABI of the recombination library (declared in include/rec.h).
//
// Each entry point validates its arguments, enqueues kernels on the context
// stream and returns a rec_status; no exception crosses the boundary.  The
// context owns its scratch; field buffers belong to the caller.

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rec_internal.cuh"

namespace {

thread_local std::string g_init_error;

rec_status fail(rec_ctx* c, rec_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_init_error = msg;
  return s;
}

rec_status cuda_fail(rec_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(c, REC_ECUDA, m);
}

bool is_finite(double v) { return std::isfinite(v); }

rec_status check_params(const rec_params* p, std::string* why) {
  if (!p) { *why = "params is NULL"; return REC_EINVAL; }
  if (!(p->h > 0) || !(p->omega_b_h2 > 0) || !(p->omega_c_h2 >= 0) || !(p->Y_p >= 0 && p->Y_p < 1) ||
      !(p->T_cmb0 > 0) || !(p->N_eff >= 0) || !(p->L_box_kpc > 0) || !(p->fudge > 0) || !is_finite(p->heating) ||
      p->heating < 0) {
    *why = "cosmological parameters out of range";
    return REC_EINVAL;
  }
  if (p->n_sub < 1 || p->n_sub > 4096) { *why = "n_sub must be in [1, 4096]"; return REC_EINVAL; }
  if (p->precision != REC_PREC_FP64 && p->precision != REC_PREC_MIXED) { *why = "unknown precision"; return REC_EINVAL; }
  if (p->mixing != REC_MIX_TALLY && p->mixing != REC_MIX_FULL && p->mixing != REC_MIX_LOCAL &&
      p->mixing != REC_MIX_PARTIAL) {
    *why = "unknown mixing mode";
    return REC_EINVAL;
  }
  if (p->mixing == REC_MIX_PARTIAL && !(p->f_alpha >= 0.0 && p->f_alpha <= 1.0)) {
    *why = "f_alpha must be in [0, 1]";
    return REC_EINVAL;
  }
  if (p->n_quantiles < 2 || !p->emission_quantiles) { *why = "emission profile table missing"; return REC_EINVAL; }
  for (int i = 0; i < p->n_quantiles; ++i) {
    if (!is_finite(p->emission_quantiles[i]) || (i > 0 && p->emission_quantiles[i] < p->emission_quantiles[i - 1])) {
      *why = "emission profile table must be finite and non-decreasing";
      return REC_EINVAL;
    }
  }
  return REC_OK;
}

rec_status check_box(const rec_box& b, std::string* why) {
  if (b.n < 1 || b.n > 1024) { *why = "box side n must be in [1, 1024]"; return REC_EINVAL; }
  if (!b.delta || !b.vel4 || !b.x_e || !b.T || !b.tally || !b.emis) { *why = "a field buffer is NULL"; return REC_EINVAL; }
  if (b.n_packets >= (1ull << 32)) { *why = "n_packets must be below 2^32"; return REC_EINVAL; }
  // the FP64 form reads each velocity as one 32-byte vector; one rule for both forms
  if (reinterpret_cast<uintptr_t>(b.vel4) % 32 != 0) { *why = "vel4 must be 32-byte aligned"; return REC_EINVAL; }
  return REC_OK;
}

size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

rec_tuning default_tuning(bool mixed, bool batch) {
  rec_tuning t;
  rec::transport_limits(mixed, batch, &t.emit_blocks_per_sm, &t.march_blocks_per_sm);
  t.march_refill = 8;
  t.march_chunk = 64;
  t.tile = 32;
  t.march_halo = 0;
  return t;
}

uint32_t log2u(uint32_t v) {
  uint32_t l = 0;
  while ((1u << l) < v) ++l;
  return l;
}

// Super-tile layout of every box of a batch for the tile side in use.
void layout_buckets(rec_ctx* c) {
  c->tot_buckets = 0;
  for (auto& d : c->hbx) {
    d.nt = (d.n + (uint32_t)c->tune.tile - 1) / (uint32_t)c->tune.tile;
    d.tlg = log2u((uint32_t)c->tune.tile);
    d.bk0 = (uint32_t)c->tot_buckets;
    c->tot_buckets += (int)(d.nt * d.nt * d.nt);
  }
}

// Context of several boxes: per-box records and concatenated scratch.
rec_status init_batch(const rec_params* params, const rec_box* boxes, int32_t n_boxes, void* cuda_stream,
                      rec_ctx** out) {
  if (n_boxes > rec::kMaxBoxes) return fail(nullptr, REC_EINVAL, "at most 128 boxes per context");
  if (params->mixing == REC_MIX_LOCAL || params->mixing == REC_MIX_PARTIAL)
    return fail(nullptr, REC_EINVAL, "local and partial mixing need a single-box context");
  std::string why;
  for (int i = 0; i < n_boxes; ++i)
    if (check_box(boxes[i], &why) != REC_OK) return fail(nullptr, REC_EINVAL, "box " + std::to_string(i) + ": " + why);
  rec_ctx* c = new (std::nothrow) rec_ctx();
  if (!c) return fail(nullptr, REC_ENOMEM, "host allocation failed");
  c->params = *params;
  c->params.emission_quantiles = nullptr;
  c->box = boxes[0];
  c->boxes.assign(boxes, boxes + n_boxes);
  c->n_boxes = n_boxes;
  c->stream = (cudaStream_t)cuda_stream;
  c->cosmo = rec::make_cosmo(*params);
  c->sc = nullptr; c->sc_adj = nullptr; c->part = nullptr; c->P = nullptr; c->partQ = nullptr; c->quant = nullptr;
  c->queue = nullptr; c->first = nullptr; c->xy = nullptr; c->bcap = nullptr; c->bfill = nullptr; c->cpre = nullptr;
  c->emis_ready = false;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) { rec_status r = cuda_fail(nullptr, e, "device query"); delete c; return r; }
  // offsets of every box in the concatenated scratch
  const bool mixed = params->precision == REC_PREC_MIXED;
  size_t nP = 0, nfirst = 0, nxy = 0, npk_all = 0, nb_alloc = 0;
  c->hbx.resize(n_boxes);
  c->tune = default_tuning(mixed, true);
  int64_t n3_all = 0;
  for (int i = 0; i < n_boxes; ++i) {
    const rec_box& b = boxes[i];
    rec::BoxDev& d = c->hbx[i];
    std::memset(&d, 0, sizeof(d));
    d.n3 = (int64_t)b.n * b.n * b.n;
    d.n = (uint32_t)b.n;
    d.p2 = (b.n & (b.n - 1)) == 0 ? 1u : 0u;
    d.lg = 0;
    while (d.p2 && (1 << d.lg) < b.n) ++d.lg;
    d.mn = b.n >= 2 ? UINT64_MAX / (uint64_t)b.n + 1 : 0;
    d.mn2 = b.n >= 2 ? UINT64_MAX / ((uint64_t)b.n * b.n) + 1 : 0;
    d.npk = b.n_packets;
    d.pk0 = c->tot_pk;
    c->tot_pk += round_up(b.n_packets, 64);  // a 64-packet emission window never spans two boxes
    d.ablk0 = (uint32_t)c->tot_ablk;
    c->tot_ablk += (int)((d.n3 + rec::kAllocChunk - 1) / rec::kAllocChunk);
    d.pblk = (uint32_t)std::max<int64_t>(1, (d.n3 + rec::kPassThreads * rec::kPassCellsPerThread - 1) /
                                                (rec::kPassThreads * rec::kPassCellsPerThread));
    d.pblk0 = (uint32_t)c->tot_pblk;
    c->tot_pblk += (int)d.pblk;
    const size_t nt_min = (size_t)((b.n + rec::kMinTile - 1) / rec::kMinTile);
    nb_alloc += nt_min * nt_min * nt_min;
    // scratch offsets (element counts), kept in the pointer fields until the buffers exist
    d.P = (uint32_t*)(uintptr_t)nP;
    nP += round_up((size_t)d.n3 + 1, 4);
    d.first = (uint32_t*)(uintptr_t)nfirst;
    nfirst += (size_t)(b.n_packets / 32 + 2);
    d.xy = (void*)(uintptr_t)nxy;
    nxy += (size_t)d.n3;
    npk_all += b.n_packets;
    n3_all += d.n3;
  }
  c->n3 = n3_all;
  layout_buckets(c);
  c->grid = c->tot_pblk;
  c->alloc_blocks = c->tot_ablk;
  const size_t qbytes = (size_t)params->n_quantiles * (mixed ? 4 : 8);
  const size_t part_n = std::max<size_t>(2 * (size_t)rec::kMaxSums * c->tot_pblk, (size_t)rec::kMaxSums * c->tot_ablk);
  const size_t qentry = mixed ? 32 : 96;  // two float4 | three double4 per queued packet
  e = cudaMalloc(&c->sc, sizeof(rec::DevScalars) * n_boxes);
  if (e == cudaSuccess) e = cudaMalloc(&c->gsc, sizeof(rec::DevScalars));
  if (e == cudaSuccess) e = cudaMalloc(&c->sc_adj, sizeof(rec::DevScalars));
  if (e == cudaSuccess) e = cudaMalloc(&c->part, sizeof(double) * part_n);
  if (e == cudaSuccess) e = cudaMalloc(&c->P, sizeof(uint32_t) * nP);
  if (e == cudaSuccess) e = cudaMalloc(&c->partQ, sizeof(unsigned long long) * (size_t)c->tot_ablk);
  if (e == cudaSuccess) e = cudaMalloc(&c->first, sizeof(uint32_t) * nfirst);
  if (e == cudaSuccess && mixed) e = cudaMalloc(&c->xy, sizeof(float) * 2 * nxy);
  if (e == cudaSuccess) e = cudaMalloc(&c->bcap, sizeof(unsigned long long) * nb_alloc);
  if (e == cudaSuccess) e = cudaMalloc(&c->bfill, sizeof(unsigned long long) * nb_alloc);
  if (e == cudaSuccess) e = cudaMalloc(&c->cpre, sizeof(unsigned long long) * (nb_alloc + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->quant, qbytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->queue, qentry * std::max<size_t>(npk_all, 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->bx, sizeof(rec::BoxDev) * n_boxes);
  if (e == cudaSuccess) e = cudaMalloc(&c->bstep, sizeof(rec::BoxStep) * n_boxes);
  if (e != cudaSuccess) {
    rec_status r = (e == cudaErrorMemoryAllocation) ? fail(nullptr, REC_ENOMEM, "device allocation failed")
                                                    : cuda_fail(nullptr, e, "cudaMalloc");
    rec_free(c);
    return r;
  }
  for (int i = 0; i < n_boxes; ++i) {
    const rec_box& b = boxes[i];
    rec::BoxDev& d = c->hbx[i];
    d.delta = b.delta;
    d.vel4 = b.vel4;
    d.x = b.x_e;
    d.T = b.T;
    d.tally = b.tally;
    d.emis = b.emis;
    d.P = c->P + (size_t)(uintptr_t)d.P;
    d.first = c->first + (size_t)(uintptr_t)d.first;
    d.xy = mixed ? (void*)((float2*)c->xy + (size_t)(uintptr_t)d.xy) : nullptr;
    d.sc = c->sc + i;
  }
  std::vector<char> hq(qbytes);
  for (int i = 0; i < params->n_quantiles; ++i) {
    if (mixed) ((float*)hq.data())[i] = (float)params->emission_quantiles[i];
    else ((double*)hq.data())[i] = params->emission_quantiles[i];
  }
  std::vector<rec::DevScalars> zero(n_boxes);
  std::memset(zero.data(), 0, sizeof(rec::DevScalars) * n_boxes);
  for (auto& z : zero) z.lam_prev = -1.0;
  e = cudaMemcpyAsync(c->quant, hq.data(), qbytes, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->sc, zero.data(), sizeof(rec::DevScalars) * n_boxes, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->gsc, zero.data(), sizeof(rec::DevScalars), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->sc_adj, zero.data(), sizeof(rec::DevScalars), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->bx, c->hbx.data(), sizeof(rec::BoxDev) * n_boxes, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    rec_status r = cuda_fail(nullptr, e, "rec_init upload");
    rec_free(c);
    return r;
  }
  *out = c;
  return REC_OK;
}

}  // namespace

extern "C" {

rec_status rec_init(const rec_params* params, const rec_box* boxes, int32_t n_boxes, void* cuda_stream,
                    rec_ctx** out) {
  g_init_error.clear();
  if (!out) return fail(nullptr, REC_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  rec_status s = check_params(params, &why);
  if (s != REC_OK) return fail(nullptr, s, why);
  if (!boxes || n_boxes < 1) return fail(nullptr, REC_EINVAL, "need at least one box");
  if (n_boxes > 1) return init_batch(params, boxes, n_boxes, cuda_stream, out);
  const rec_box& b = boxes[0];
  if (check_box(b, &why) != REC_OK) return fail(nullptr, REC_EINVAL, why);

  rec_ctx* c = new (std::nothrow) rec_ctx();
  if (!c) return fail(nullptr, REC_ENOMEM, "host allocation failed");
  c->params = *params;
  c->params.emission_quantiles = nullptr;  // copied to the device below
  c->box = b;
  c->stream = (cudaStream_t)cuda_stream;
  c->n3 = (int64_t)b.n * b.n * b.n;
  c->cosmo = rec::make_cosmo(*params);
  c->sc = nullptr; c->sc_adj = nullptr; c->part = nullptr; c->P = nullptr; c->partQ = nullptr; c->quant = nullptr;
  c->queue = nullptr;
  c->first = nullptr;
  c->xy = nullptr;
  c->div = nullptr;
  c->bcap = nullptr; c->bfill = nullptr; c->cpre = nullptr;
  c->emis_ready = false;

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) { rec_status r = cuda_fail(nullptr, e, "device query"); delete c; return r; }
  // streaming passes: a fixed grid (several blocks per SM) for reproducible sums
  int64_t want = (c->n3 + rec::kPassThreads - 1) / rec::kPassThreads;
  c->grid = (int)std::min<int64_t>(want, (int64_t)c->sm_count * 8);
  if (c->grid < 1) c->grid = 1;
  c->alloc_blocks = (int)((c->n3 + rec::kAllocChunk - 1) / rec::kAllocChunk);
  c->tune = default_tuning(params->precision == REC_PREC_MIXED, false);

  size_t qbytes = (size_t)params->n_quantiles * (params->precision == REC_PREC_MIXED ? 4 : 8);
  e = cudaMalloc(&c->sc, sizeof(rec::DevScalars));
  if (e == cudaSuccess) e = cudaMalloc(&c->sc_adj, sizeof(rec::DevScalars));
  // block partials (two per block: the TMA-staged passes run more blocks than the grid)
  if (e == cudaSuccess) e = cudaMalloc(&c->part, 2 * sizeof(double) * rec::kMaxSums * (size_t)c->grid);
  if (e == cudaSuccess) e = cudaMalloc(&c->P, sizeof(uint32_t) * (size_t)(c->n3 + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->partQ, sizeof(unsigned long long) * (size_t)c->alloc_blocks);
  if (e == cudaSuccess) e = cudaMalloc(&c->first, sizeof(uint32_t) * (size_t)(b.n_packets / 32 + 2));
  if (e == cudaSuccess && params->precision == REC_PREC_MIXED) e = cudaMalloc(&c->xy, sizeof(float) * 2 * (size_t)c->n3);
  // local mixing: velocity divergence per cell (working precision)
  if (e == cudaSuccess && (params->mixing == REC_MIX_LOCAL || params->mixing == REC_MIX_PARTIAL))
    e = cudaMalloc(&c->div, (params->precision == REC_PREC_MIXED ? 4 : 8) * (size_t)c->n3);
  {
    // super-tiles of the march queue, sized for the smallest tile side
    size_t nt = (size_t)((b.n + rec::kMinTile - 1) / rec::kMinTile), nb = nt * nt * nt;
    if (e == cudaSuccess) e = cudaMalloc(&c->bcap, sizeof(unsigned long long) * nb);
    if (e == cudaSuccess) e = cudaMalloc(&c->bfill, sizeof(unsigned long long) * nb);
    if (e == cudaSuccess) e = cudaMalloc(&c->cpre, sizeof(unsigned long long) * (nb + 1));
  }
  if (e == cudaSuccess) e = cudaMalloc(&c->quant, qbytes);
  // march queue: two float4 (mixed) or three double4_32a (FP64) per packet, worst case all packets
  size_t qentry = params->precision == REC_PREC_MIXED ? 32 : 96;
  if (e == cudaSuccess) e = cudaMalloc(&c->queue, qentry * (size_t)std::max<uint64_t>(b.n_packets, 1));
  if (e != cudaSuccess) {
    rec_status r = (e == cudaErrorMemoryAllocation) ? fail(nullptr, REC_ENOMEM, "device allocation failed")
                                                    : cuda_fail(nullptr, e, "cudaMalloc");
    rec_free(c);
    return r;
  }
  // emission-profile table in the working precision of the transport
  std::vector<char> hq(qbytes);
  for (int i = 0; i < params->n_quantiles; ++i) {
    if (params->precision == REC_PREC_MIXED) ((float*)hq.data())[i] = (float)params->emission_quantiles[i];
    else ((double*)hq.data())[i] = params->emission_quantiles[i];
  }
  rec::DevScalars zero;
  std::memset(&zero, 0, sizeof(zero));
  zero.lam_prev = -1.0;
  e = cudaMemcpyAsync(c->quant, hq.data(), qbytes, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->sc, &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->sc_adj, &zero, sizeof(zero), cudaMemcpyHostToDevice, c->stream);
  // the host staging buffers go out of scope: wait for the copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    rec_status r = cuda_fail(nullptr, e, "rec_init upload");
    rec_free(c);
    return r;
  }
  *out = c;
  return REC_OK;
}

rec_status rec_state_init(rec_ctx* c, double z) {
  if (!c) return fail(nullptr, REC_EINVAL, "ctx is NULL");
  if (!(z > 0) || !is_finite(z)) return fail(c, REC_EINVAL, "z must be positive");
  cudaError_t e = c->n_boxes > 1 ? rec::launch_state_init_batch(c, z) : rec::launch_state_init(c, z);
  if (e != cudaSuccess) return cuda_fail(c, e, "rec_state_init");
  c->emis_ready = true;
  return REC_OK;
}

rec_status rec_refresh(rec_ctx* c, double z) {
  if (!c) return fail(nullptr, REC_EINVAL, "ctx is NULL");
  if (!(z > 0) || !is_finite(z)) return fail(c, REC_EINVAL, "z must be positive");
  cudaError_t e = c->n_boxes > 1 ? rec::launch_refresh_batch(c, z) : rec::launch_refresh(c, z);
  if (e != cudaSuccess) return cuda_fail(c, e, "rec_refresh");
  c->emis_ready = true;
  return REC_OK;
}

rec_status lya_transport(rec_ctx* c, int32_t step, double z, rec_stats* st) {
  if (!c) return fail(nullptr, REC_EINVAL, "ctx is NULL");
  if (!(z > 0) || !is_finite(z)) return fail(c, REC_EINVAL, "z must be positive");
  if (step < 0) return fail(c, REC_EINVAL, "step must be non-negative");
  cudaError_t e = c->n_boxes > 1 ? rec::launch_transport_batch(c, step, z, st) : rec::launch_transport(c, step, z, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "lya_transport");
  return REC_OK;
}

rec_status rec_step(rec_ctx* c, int32_t step, double z_from, double z_to, rec_stats* st) {
  if (!c) return fail(nullptr, REC_EINVAL, "ctx is NULL");
  (void)step;
  if (!(z_from > z_to) || !(z_to > 0) || !is_finite(z_from)) return fail(c, REC_EINVAL, "need z_from > z_to > 0");
  if (!c->emis_ready) return fail(c, REC_ESTATE, "state sums unknown: call rec_state_init or rec_refresh first");
  cudaError_t e = c->n_boxes > 1 ? rec::launch_rec_step_batch(c, z_from, z_to, st)
                                  : rec::launch_rec_step(c, z_from, z_to, st);
  if (e != cudaSuccess) return cuda_fail(c, e, "rec_step");
  return REC_OK;
}

rec_status rec_get_tuning(const rec_ctx* c, rec_tuning* out) {
  if (!c || !out) return fail(nullptr, REC_EINVAL, "ctx or out is NULL");
  *out = c->tune;
  return REC_OK;
}

rec_status rec_set_tuning(rec_ctx* c, const rec_tuning* t) {
  if (!c || !t) return fail(nullptr, REC_EINVAL, "ctx or tuning is NULL");
  int emax = 0, mmax = 0;
  rec::transport_limits(c->params.precision == REC_PREC_MIXED, c->n_boxes > 1, &emax, &mmax);
  if (t->emit_blocks_per_sm < 1 || t->emit_blocks_per_sm > emax)
    return fail(c, REC_EINVAL, "emit_blocks_per_sm must be in [1, " + std::to_string(emax) + "]");
  if (t->march_blocks_per_sm < 1 || t->march_blocks_per_sm > mmax)
    return fail(c, REC_EINVAL, "march_blocks_per_sm must be in [1, " + std::to_string(mmax) + "]");
  if (t->march_refill < 1 || t->march_refill > 32) return fail(c, REC_EINVAL, "march_refill must be in [1, 32]");
  if (t->march_chunk < 8 || t->march_chunk > 4096) return fail(c, REC_EINVAL, "march_chunk must be in [8, 4096]");
  if (t->tile != 8 && t->tile != 16 && t->tile != 32 && t->tile != 64)
    return fail(c, REC_EINVAL, "tile must be 8, 16, 32 or 64");
  if (t->march_halo < 0 || t->march_halo > 256) return fail(c, REC_EINVAL, "march_halo must be in [0, 256]");
  if (t->march_halo > 0) {
    if (c->n_boxes > 1) return fail(c, REC_EINVAL, "march_halo needs a single-box context");
    if ((c->box.n & (c->box.n - 1)) != 0) return fail(c, REC_EINVAL, "march_halo needs a power-of-two box side");
    const int smax = rec::sweep_march_limit(c->params.precision == REC_PREC_MIXED);
    if (t->march_blocks_per_sm > smax)
      return fail(c, REC_EINVAL, "with march_halo > 0, march_blocks_per_sm must be in [1, " + std::to_string(smax) + "]");
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);  // no transport of this context in flight
  if (e != cudaSuccess) return cuda_fail(c, e, "rec_set_tuning");
  if (t->march_halo > 0 && !c->rqueue) {
    // the second queue of the region sweeps and its per-bucket counters
    const size_t entry = c->params.precision == REC_PREC_MIXED ? 48 : 96;
    const size_t cap = (std::max<uint64_t>(c->box.n_packets / 4, 1) + rec::kRqParts - 1) / rec::kRqParts * rec::kRqParts;
    const size_t nt = (size_t)((c->box.n + rec::kMinTile - 1) / rec::kMinTile), nb = nt * nt * nt;
    e = cudaMalloc(&c->rqueue, entry * cap);
    if (e == cudaSuccess) e = cudaMalloc(&c->rcount, sizeof(unsigned long long) * nb);
    if (e == cudaSuccess) e = cudaMalloc(&c->scnt, sizeof(unsigned long long) * nb);
    if (e == cudaSuccess) e = cudaMalloc(&c->rqn, sizeof(unsigned long long) * 2 * rec::kRqParts);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->rcount, 0, sizeof(unsigned long long) * nb, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      cudaFree(c->rqueue); cudaFree(c->rcount); cudaFree(c->scnt); cudaFree(c->rqn);
      c->rqueue = nullptr; c->rcount = nullptr; c->scnt = nullptr; c->rqn = nullptr;
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? fail(c, REC_ENOMEM, "rec_set_tuning: second march queue")
                                            : cuda_fail(c, e, "rec_set_tuning: second march queue");
    }
    c->rq_cap = cap;
  }
  c->tune = *t;
  if (c->n_boxes > 1) {
    layout_buckets(c);
    e = cudaMemcpy(c->bx, c->hbx.data(), sizeof(rec::BoxDev) * c->n_boxes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "rec_set_tuning upload");
  }
  return REC_OK;
}

rec_status rec_graph_step(rec_ctx* c, int32_t step, double z_from, double z_to, rec_stats* st) {
  if (!c) return fail(nullptr, REC_EINVAL, "ctx is NULL");
  if (step < 0) return fail(c, REC_EINVAL, "step must be non-negative");
  if (!(z_from > z_to) || !(z_to > 0) || !is_finite(z_from)) return fail(c, REC_EINVAL, "need z_from > z_to > 0");
  if (!c->emis_ready) return fail(c, REC_ESTATE, "emission weights unknown: call rec_state_init or rec_refresh first");
  if (c->timing) return fail(c, REC_EINVAL, "kernel timing is off for graph steps (rec_timing(ctx, 0))");
  if (c->stream == nullptr) return fail(c, REC_EINVAL, "graph steps need a non-default stream");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(c->stream, &cs);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone) return fail(c, REC_EINVAL, "the context stream is already being captured");
  e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
  c->capturing = true;
  cudaError_t e1 = c->n_boxes > 1 ? rec::launch_transport_batch(c, step, z_from, st)
                                  : rec::launch_transport(c, step, z_from, st);
  cudaError_t e2 = (e1 == cudaSuccess) ? (c->n_boxes > 1 ? rec::launch_rec_step_batch(c, z_from, z_to, st)
                                                         : rec::launch_rec_step(c, z_from, z_to, st))
                                       : cudaSuccess;
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->stream, &g);
  c->capturing = false;
  if (e1 != cudaSuccess || e2 != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(c, e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e), "rec_graph_step capture");
  }
  // same topology every step: update the kernel parameters of the executable graph in place
  if (c->gexec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(c->gexec, g, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(c->gexec);
      c->gexec = nullptr;
    }
  }
  if (!c->gexec) e = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { c->gexec = nullptr; return cuda_fail(c, e, "cudaGraphInstantiate"); }
  e = cudaGraphLaunch(c->gexec, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphLaunch");
  return REC_OK;
}

rec_status rec_step_noalloc(const rec_params* params, const rec_box* box, double z_from, double z_to,
                            void* cuda_stream, rec_stats* dev_stats) {
  g_init_error.clear();
  std::string why;
  rec_status s = check_params(params, &why);
  if (s != REC_OK) return fail(nullptr, s, why);
  if (params->precision != REC_PREC_FP64)
    return fail(nullptr, REC_EINVAL, "rec_step_noalloc needs the FP64 form (the mixed form keeps a per-cell cache)");
  if (params->mixing == REC_MIX_LOCAL || params->mixing == REC_MIX_PARTIAL)
    return fail(nullptr, REC_EINVAL,
                "rec_step_noalloc covers tally and full mixing (local and partial mixing keep a per-cell field)");
  if (!box) return fail(nullptr, REC_EINVAL, "box is NULL");
  if (box->n < 1 || box->n > 1024) return fail(nullptr, REC_EINVAL, "box side n must be in [1, 1024]");
  if (!box->delta || !box->vel4 || !box->x_e || !box->T || !box->tally || !box->emis)
    return fail(nullptr, REC_EINVAL, "a field buffer is NULL");
  if (reinterpret_cast<uintptr_t>(box->vel4) % 32 != 0) return fail(nullptr, REC_EINVAL, "vel4 must be 32-byte aligned");
  if (!(z_from > z_to) || !(z_to > 0) || !is_finite(z_from)) return fail(nullptr, REC_EINVAL, "need z_from > z_to > 0");
  s = rec::launch_rec_step_noalloc(*params, *box, z_from, z_to, (cudaStream_t)cuda_stream, dev_stats, &why);
  if (s != REC_OK) return fail(nullptr, s, "rec_step_noalloc: " + why);
  return REC_OK;
}

rec_status rec_step_adjoint(rec_ctx* c, int32_t step, double z_from, double z_to, const double* x_in,
                            const double* T_in, const double* vel4_in, const uint32_t* tally_in, double* xbar,
                            double* Tbar, double* Ubar, double* g_delta, double* g_a, double Xe_bar_out) {
  if (!c) return fail(nullptr, REC_EINVAL, "ctx is NULL");
  (void)step;
  if (c->n_boxes > 1) return fail(c, REC_EINVAL, "the adjoint works on single-box contexts");
  if (c->params.mixing == REC_MIX_LOCAL || c->params.mixing == REC_MIX_PARTIAL)
    return fail(c, REC_EINVAL, "the adjoint covers tally and full mixing");
  if (c->params.precision != REC_PREC_FP64) return fail(c, REC_EINVAL, "the adjoint needs the FP64 form");
  if (c->params.n_sub != 1) return fail(c, REC_EINVAL, "the adjoint supports n_sub == 1");
  if (!(z_from > z_to) || !(z_to > 0)) return fail(c, REC_EINVAL, "need z_from > z_to > 0");
  if (!x_in || !T_in || !xbar || !Tbar || !g_delta) return fail(c, REC_EINVAL, "a required buffer is NULL");
  if (Ubar && !vel4_in) return fail(c, REC_EINVAL, "Ubar needs vel4_in");
  if (c->params.mixing == REC_MIX_TALLY && !tally_in) return fail(c, REC_EINVAL, "tally mode needs tally_in");
  cudaError_t e = rec::launch_rec_step_adjoint(c, z_from, z_to, x_in, T_in, vel4_in, tally_in, xbar, Tbar, Ubar,
                                               g_delta, g_a, Xe_bar_out);
  if (e != cudaSuccess) return cuda_fail(c, e, "rec_step_adjoint");
  return REC_OK;
}

rec_status rec_xe_adjoint(rec_ctx* c, const double* x, double Xe_bar, double* xbar, double* g_delta) {
  if (!c) return fail(nullptr, REC_EINVAL, "ctx is NULL");
  if (c->n_boxes > 1) return fail(c, REC_EINVAL, "the adjoint works on single-box contexts");
  if (c->params.mixing == REC_MIX_LOCAL || c->params.mixing == REC_MIX_PARTIAL)
    return fail(c, REC_EINVAL, "the adjoint covers tally and full mixing");
  if (c->params.precision != REC_PREC_FP64) return fail(c, REC_EINVAL, "the adjoint needs the FP64 form");
  if (!x || !xbar || !g_delta) return fail(c, REC_EINVAL, "a required buffer is NULL");
  cudaError_t e = rec::launch_xe_adjoint(c, x, Xe_bar, xbar, g_delta);
  if (e != cudaSuccess) return cuda_fail(c, e, "rec_xe_adjoint");
  return REC_OK;
}

rec_status rec_transport_params(const rec_params* p, int32_t n, double z, double* out) {
  std::string why;
  rec_status s = check_params(p, &why);
  if (s != REC_OK) return fail(nullptr, s, why);
  if (n < 1 || !out || !(z > 0)) return fail(nullptr, REC_EINVAL, "bad n, z or out");
  rec::Cosmo cm = rec::make_cosmo(*p);
  rec::transport_scalars(cm, n, z, &out[0], &out[1]);
  return REC_OK;
}

rec_status rec_objective(const rec_params* p, const double* zs, const double* Xe, int32_t n_nodes,
                         int32_t objective, double z_star, double* J, double* dJ) {
  std::string why;
  rec_status s = check_params(p, &why);
  if (s != REC_OK) return fail(nullptr, s, why);
  if (!zs || !Xe || !J || !dJ || n_nodes < 1 || (objective != 1 && objective != 2))
    return fail(nullptr, REC_EINVAL, "bad objective arguments");
  rec::Cosmo cm = rec::make_cosmo(*p);
  int ks = 0;
  for (int k = 1; k < n_nodes; ++k)
    if (std::fabs(zs[k] - z_star) < std::fabs(zs[ks] - z_star)) ks = k;
  for (int k = 0; k < n_nodes; ++k) dJ[k] = 0.0;
  if (objective == 1) {
    *J = Xe[ks];
    dJ[ks] = 1.0;
    return REC_OK;
  }
  // d tau/dz = c_k X_e,k with c_k = sigma_T c nbar_H / ((1+z) H)
  std::vector<double> ck(n_nodes);
  for (int k = 0; k < n_nodes; ++k)
    ck[k] = rec::thomson_sigma_c() * rec::nH_bar(cm, zs[k]) / ((1.0 + zs[k]) * rec::hubble(cm, zs[k]));
  double tau = 0.0;
  for (int m = ks; m < n_nodes - 1; ++m) tau += 0.5 * (ck[m] * Xe[m] + ck[m + 1] * Xe[m + 1]) * (zs[m] - zs[m + 1]);
  double e = std::exp(-tau);
  double g = ck[ks] * Xe[ks] * e;
  *J = g;
  dJ[ks] += ck[ks] * e;
  for (int m = ks; m < n_nodes - 1; ++m) {
    double h = 0.5 * (zs[m] - zs[m + 1]);
    dJ[m] -= g * h * ck[m];
    dJ[m + 1] -= g * h * ck[m + 1];
  }
  return REC_OK;
}

rec_status rec_timing(rec_ctx* c, int32_t enable) {
  if (!c) return fail(nullptr, REC_EINVAL, "ctx is NULL");
  if (enable) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "rec_timing");
    for (int g = 0; g < REC_T_COUNT; ++g) {
      for (auto& pr : c->ev[g]) { c->pool.push_back(pr.first); c->pool.push_back(pr.second); }
      c->ev[g].clear();
      c->launches[g] = 0;
    }
  }
  c->timing = enable != 0;
  return REC_OK;
}

rec_status rec_kernel_times(rec_ctx* c, double* ms_out, int64_t* launches_out) {
  if (!c || !ms_out) return fail(c, REC_EINVAL, "bad arguments");
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "rec_kernel_times");
  for (int g = 0; g < REC_T_COUNT; ++g) {
    double tot = 0.0;
    for (auto& pr : c->ev[g]) {
      float ms = 0.0f;
      e = cudaEventElapsedTime(&ms, pr.first, pr.second);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventElapsedTime");
      tot += ms;
    }
    ms_out[g] = tot;
    if (launches_out) launches_out[g] = c->launches[g];
  }
  return REC_OK;
}

void rec_free(rec_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (int g = 0; g < REC_T_COUNT; ++g)
    for (auto& pr : c->ev[g]) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  for (cudaEvent_t e : c->pool) cudaEventDestroy(e);
  cudaFree(c->sc);
  cudaFree(c->sc_adj);
  cudaFree(c->part);
  cudaFree(c->P);
  cudaFree(c->partQ);
  cudaFree(c->quant);
  cudaFree(c->queue);
  cudaFree(c->first);
  cudaFree(c->xy);
  cudaFree(c->bcap);
  cudaFree(c->bfill);
  cudaFree(c->cpre);
  cudaFree(c->rqueue);
  cudaFree(c->rcount);
  cudaFree(c->scnt);
  cudaFree(c->rqn);
  cudaFree(c->div);
  cudaFree(c->mc_scratch);
  cudaFree(c->trb_scratch);
  cudaFree(c->mf_cnt);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  cudaFree(c->bx);
  cudaFree(c->bstep);
  cudaFree(c->gsc);
  delete c;
}

rec_status rec_set_f_alpha(rec_ctx* c, double f_alpha) {
  if (!c) return fail(nullptr, REC_EINVAL, "context is NULL");
  if (c->params.mixing != REC_MIX_PARTIAL) return fail(c, REC_EINVAL, "f_alpha applies to partial mixing only");
  if (!(f_alpha >= 0.0 && f_alpha <= 1.0)) return fail(c, REC_EINVAL, "f_alpha must be in [0, 1]");
  c->params.f_alpha = f_alpha;
  return REC_OK;
}

rec_status rec_step_trbdf2(rec_ctx* c, int32_t step, double z_from, double z_to, rec_stats* st) {
  (void)step;
  if (!c) return fail(nullptr, REC_EINVAL, "context is NULL");
  if (c->n_boxes != 1) return fail(c, REC_EINVAL, "the TR-BDF2 step needs a single-box context");
  if (c->params.precision != REC_PREC_FP64) return fail(c, REC_EINVAL, "the TR-BDF2 step needs the FP64 form");
  if (c->params.mixing != REC_MIX_TALLY && c->params.mixing != REC_MIX_FULL)
    return fail(c, REC_EINVAL, "the TR-BDF2 step covers tally and full mixing");
  if (!(z_from > z_to) || !is_finite(z_from) || !(z_to > 0.0)) return fail(c, REC_EINVAL, "need z_from > z_to > 0");
  if (!c->emis_ready) return fail(c, REC_ESTATE, "rec_state_init or rec_refresh first");
  cudaError_t e = rec::launch_rec_step_trbdf2(c, z_from, z_to, st);
  if (e == cudaErrorMemoryAllocation) return fail(c, REC_ENOMEM, "TR-BDF2 scratch");
  if (e != cudaSuccess) return cuda_fail(c, e, "rec_step_trbdf2");
  return REC_OK;
}

rec_status lya_scatter_mc(rec_ctx* c, const lya_mc_params* mp, const uint32_t* dev_prefix,
                          lya_mc_photon* dev_photons, lya_mc_stats* dev_stats) {
  if (!c) return fail(nullptr, REC_EINVAL, "context is NULL");
  if (c->n_boxes != 1) return fail(c, REC_EINVAL, "the scattering Monte Carlo needs a single-box context");
  if (!mp) return fail(c, REC_EINVAL, "lya_mc_params is NULL");
  if (!(mp->z > 0.0) || !is_finite(mp->z)) return fail(c, REC_EINVAL, "z must be positive and finite");
  if (!(mp->eps > 0.0 && mp->eps <= 1.0)) return fail(c, REC_EINVAL, "eps must be in (0, 1]");
  if (!(mp->x_lost > 0.0) || !is_finite(mp->x_lost)) return fail(c, REC_EINVAL, "x_lost must be positive");
  if (!(mp->zeta > 0.0) || !is_finite(mp->zeta)) return fail(c, REC_EINVAL, "zeta must be positive");
  if (!is_finite(mp->lambda2g)) return fail(c, REC_EINVAL, "lambda2g must be finite");
  if (!(mp->A_alpha > 0.0) || !is_finite(mp->A_alpha)) return fail(c, REC_EINVAL, "A_alpha must be positive");
  if (mp->n_photons < 1 || mp->n_photons >= (1ull << 32))
    return fail(c, REC_EINVAL, "n_photons must be in [1, 2^32)");
  if (mp->max_steps < 1) return fail(c, REC_EINVAL, "max_steps must be at least 1");
  if (mp->pending < 0 || mp->pending > 32) return fail(c, REC_EINVAL, "pending must be in [0, 32]");
  if (mp->arith != LYA_MC_FP64 && mp->arith != LYA_MC_MIXED) return fail(c, REC_EINVAL, "unknown arith form");
  rec::McSetup S;
  if (!rec::scatter_setup(c->cosmo, c->params, c->box.n, mp, &S))
    return fail(c, REC_EINVAL, "Monte-Carlo scalars are not finite at this redshift");
  cudaError_t e = rec::run_scatter_mc(c, S, mp, dev_prefix, dev_photons, dev_stats);
  if (e == cudaErrorMemoryAllocation) return fail(c, REC_ENOMEM, "Monte-Carlo scratch");
  if (e != cudaSuccess) return cuda_fail(c, e, "lya_scatter_mc");
  return REC_OK;
}

rec_status lya_mc_mixing_fraction(rec_ctx* c, const lya_mc_photon* dev_photons, uint64_t n_photons,
                                  const double* D_kpc, int32_t m, double* dev_out, uint64_t* dev_counts) {
  if (!c) return fail(nullptr, REC_EINVAL, "context is NULL");
  if (!dev_photons || !dev_out || !D_kpc) return fail(c, REC_EINVAL, "lya_mc_mixing_fraction: a buffer is NULL");
  if (n_photons < 1 || n_photons >= (1ull << 32)) return fail(c, REC_EINVAL, "n_photons must be in [1, 2^32)");
  if (m < 1 || m > rec::kMixFracMax)
    return fail(c, REC_EINVAL, "m must be in [1, " + std::to_string(rec::kMixFracMax) + "]");
  for (int j = 0; j < m; ++j)
    if (!(D_kpc[j] >= 0.0) || !is_finite(D_kpc[j])) return fail(c, REC_EINVAL, "distances must be finite and >= 0");
  cudaError_t e = rec::run_mixing_fraction(c, dev_photons, n_photons, D_kpc, m, dev_out, dev_counts);
  if (e == cudaErrorMemoryAllocation) return fail(c, REC_ENOMEM, "mixing-fraction counters");
  if (e != cudaSuccess) return cuda_fail(c, e, "lya_mc_mixing_fraction");
  return REC_OK;
}

rec_status rec_set_wait_limit(rec_ctx* c, uint32_t polls) {
  if (!c) return fail(nullptr, REC_EINVAL, "context is NULL");
  c->wait_limit = polls;
  return REC_OK;
}

rec_status rec_sync(rec_ctx* c) {
  if (!c) return fail(nullptr, REC_EINVAL, "context is NULL");
  int timed_out = 0;
  cudaError_t e = rec::launch_check_waits(c, &timed_out);
  if (e != cudaSuccess) return cuda_fail(c, e, "rec_sync");
  if (timed_out)
    return fail(c, REC_ETIMEOUT,
                "a bounded device-side wait expired: the state of the calls since the last rec_sync is incomplete");
  return REC_OK;
}

rec_status rec_volume_stats(rec_ctx* c, rec_stats* dev_stats) {
  if (!c) return fail(nullptr, REC_EINVAL, "context is NULL");
  if (!dev_stats) return fail(c, REC_EINVAL, "dev_stats is NULL");
  if (!c->emis_ready) return fail(c, REC_ESTATE, "no state sums yet: call rec_state_init or rec_refresh first");
  cudaError_t e = rec::launch_volume_stats(c, dev_stats);
  if (e != cudaSuccess) return cuda_fail(c, e, "rec_volume_stats");
  return REC_OK;
}

rec_status lya_mc_scalars(const rec_params* p, const lya_mc_params* mp, int32_t n, double* out) {
  std::string why;
  rec_status st = check_params(p, &why);
  if (st != REC_OK) return fail(nullptr, st, why);
  if (!mp || !out || n < 1 || !(mp->z > 0.0) || !(mp->eps > 0.0 && mp->eps <= 1.0) || !(mp->zeta > 0.0) ||
      !(mp->A_alpha > 0.0))
    return fail(nullptr, REC_EINVAL, "lya_mc_scalars: bad arguments");
  rec::McSetup S;
  if (!rec::scatter_setup(rec::make_cosmo(*p), *p, n, mp, &S))
    return fail(nullptr, REC_EINVAL, "Monte-Carlo scalars are not finite at this redshift");
  out[0] = S.a; out[1] = S.vth; out[2] = S.sig0; out[3] = S.dxdl; out[4] = S.p_ion; out[5] = S.p_2g;
  out[6] = S.beta; out[7] = S.Lam; out[8] = S.Heff; out[9] = S.nH; out[10] = S.Tg; out[11] = S.cpm;
  return REC_OK;
}

rec_status lya_mc_redistribution_host(double a, double y, const double* kin, uint64_t seed, int64_t m,
                                      double* ppar, double* dy, double* kout, uint64_t* caps) {
  if (!(a > 0.0) || !is_finite(a) || !is_finite(y) || !kin || m < 0)
    return fail(nullptr, REC_EINVAL, "lya_mc_redistribution_host: bad arguments");
  const double kn = std::sqrt(kin[0] * kin[0] + kin[1] * kin[1] + kin[2] * kin[2]);
  if (!(kn > 0.0) || !is_finite(kn)) return fail(nullptr, REC_EINVAL, "lya_mc_redistribution_host: kin is zero");
  const uint64_t c = rec::scatter_redistribution_mixed_host(a, y, kin, seed, m, ppar, dy, kout);
  if (caps) *caps = c;
  return REC_OK;
}

rec_status lya_voigt(double a, int64_t m, const double* y, double* H) {
  if (!(a > 0.0) || !is_finite(a) || m < 0 || (m > 0 && (!y || !H)))
    return fail(nullptr, REC_EINVAL, "lya_voigt: a must be positive, y and H non-NULL");
  rec::scatter_voigt_host(a, m, y, H);
  return REC_OK;
}

rec_status lya_voigt_mixed(double a, int64_t m, const double* y, double* H) {
  if (!(a > 0.0) || !is_finite(a) || m < 0 || (m > 0 && (!y || !H)))
    return fail(nullptr, REC_EINVAL, "lya_voigt_mixed: a must be positive, y and H non-NULL");
  rec::scatter_voigt_mixed_host(a, m, y, H);
  return REC_OK;
}

const char* rec_last_error(const rec_ctx* c) {
  if (!c) return g_init_error.c_str();
  return c->err.c_str();
}

}  // extern "C"
