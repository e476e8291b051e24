// C ABI: argument checking, host-side tables, dispatch to the kernels.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "internal.h"

using namespace spin;

namespace {

int cuda_status(cudaError_t e) { return e == cudaSuccess ? SPIN_OK : SPIN_ECUDA; }

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// floor(p * 2^32), capped to [0, 2^32 - 1]
uint32_t prob_threshold(double p) {
  const double t = floor(p * 4294967296.0);
  if (t >= 4294967295.0) return 0xFFFFFFFFu;
  if (t <= 0.0) return 0u;
  return (uint32_t)t;
}

bool finite_nonneg(double b) { return isfinite(b) && b >= 0.0; }

// Metropolis thresholds per slot: row t = {float beta bits, thr(4), thr(8), thr(12)}.
// (Word 0 carries beta as a float for the Heisenberg kernel.)
int upload_thresholds(spin_lattice *h, const double *betas) {
  const int nt = h->g.n_temps;
  if (!betas) return SPIN_EINVAL;
  for (int t = 0; t < nt; ++t)
    if (!finite_nonneg(betas[t])) return SPIN_EINVAL;
  if (h->thr_valid && memcmp(h->betas_cached.data(), betas, sizeof(double) * nt) == 0) return SPIN_OK;
  std::vector<uint32_t> tab(4 * (size_t)nt);
  for (int t = 0; t < nt; ++t) {
    const float bf = (float)betas[t];
    uint32_t bits;
    memcpy(&bits, &bf, 4);
    tab[4 * t] = bits;
    for (int m = 1; m <= 3; ++m) tab[4 * t + m] = prob_threshold(exp(-betas[t] * (double)(4 * m)));
    if (h->d.model == SPIN_HEISENBERG) {
      // the fast-math acceptance tests u3 2^24 < 2^(24 - beta log2(e) dE)
      const float bl = (float)(betas[t] * 1.4426950408889634074);
      memcpy(&bits, &bl, 4);
      tab[4 * t + 1] = bits;
    }
  }
  cudaError_t e = cudaMemcpyAsync(h->d_thr, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return SPIN_ECUDA;
  e = cudaStreamSynchronize(h->stream);  // tab is a local staging copy
  if (e != cudaSuccess) return SPIN_ECUDA;
  h->betas_cached.assign(betas, betas + nt);
  h->thr_valid = 1;
  return SPIN_OK;
}

// Replica-exchange tables: for pair t, thr_t[m] = floor(exp(-|dbeta_t| 4m) 2^32)
// for m < len_t, where len_t is the first m whose threshold is 0 (all later
// ones are 0 too).  Energy differences on these lattices are multiples of 4.
int upload_pt_tables(spin_lattice *h, const double *betas) {
  const int nt = h->g.n_temps;
  for (int t = 0; t < nt; ++t)
    if (!finite_nonneg(betas[t])) return SPIN_EINVAL;
  if (!h->pt_betas_cached.empty() && memcmp(h->pt_betas_cached.data(), betas, sizeof(double) * nt) == 0)
    return SPIN_OK;
  const int64_t cap = 1 << 22;
  std::vector<uint32_t> tab;
  std::vector<int32_t> off(nt, 0), len(nt, 0);
  std::vector<double> db(nt, 0.0);
  for (int t = 0; t + 1 < nt; ++t) {
    db[t] = betas[t + 1] - betas[t];
    const double a = fabs(db[t]);
    off[t] = (int32_t)tab.size();
    int64_t m = 0;
    for (;; ++m) {
      const uint32_t v = prob_threshold(exp(-a * (double)(4 * m)));
      if (v == 0u) break;
      if (m >= cap) return SPIN_EINVAL;  // adjacent betas too close for the table
      tab.push_back(v);
      if (a == 0.0) break;  // Delta = 0: always accepted, table unused
    }
    len[t] = (int32_t)(tab.size() - off[t]);
  }
  if (tab.empty()) tab.push_back(0u);
  if (h->d_pt_thr) cudaFree(h->d_pt_thr);
  h->d_pt_thr = nullptr;
  if (cudaMalloc(&h->d_pt_thr, tab.size() * 4) != cudaSuccess) return SPIN_ENOMEM;
  cudaError_t e = cudaMemcpyAsync(h->d_pt_thr, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_pt_off, off.data(), nt * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_pt_len, len.data(), nt * 4, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_pt_dbeta, db.data(), nt * 8, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return SPIN_ECUDA;
  h->pt_betas_cached.assign(betas, betas + nt);
  return SPIN_OK;
}

int validate_desc(const spin_desc *d) {
  if (!d) return SPIN_EINVAL;
  if (d->L < 4 || (d->L & 1)) return SPIN_EINVAL;
  if (d->n_temps < 1 || d->n_temps > 4096 || d->n_sets < 1 || d->n_sets > 255 || d->n_real < 1)
    return SPIN_EINVAL;
  // per-lattice launches put the lattice index in grid.y (at most 65535)
  const int64_t n_lat = (int64_t)d->n_sets * d->n_temps * d->n_real;
  if (d->layout != SPIN_MSC1 && n_lat > 65535) return SPIN_EINVAL;
  // per-site kernels index sites (and 16-byte float4 words) with 32-bit integers
  int64_t N = 1;
  for (int k = 0; k < d->dim; ++k) N *= d->L;
  if (n_lat * N * (d->layout == SPIN_F32X4 ? 4 : 1) >= ((int64_t)1 << 32)) return SPIN_EINVAL;
  if (d->layout == SPIN_MSC1 && d->model == SPIN_ISING &&
      (n_lat > 65535 || n_lat * d->L * (d->L / 256) >= ((int64_t)1 << 31)))
    return SPIN_EINVAL;
  if (d->layout == SPIN_MSC1 && d->model == SPIN_EA &&
      (int64_t)d->n_sets * (d->n_real / 32) * d->n_temps > 65535)
    return SPIN_EINVAL;
  switch (d->model) {
    case SPIN_ISING:
      if (d->n_real > 4096) return SPIN_EINVAL;
      if (d->layout == SPIN_I8) return (d->dim == 2 || d->dim == 3) ? SPIN_OK : SPIN_EINVAL;
      if (d->layout == SPIN_MSC1) return (d->dim == 2 && d->L % 256 == 0) ? SPIN_OK : SPIN_EINVAL;
      return SPIN_EINVAL;
    case SPIN_EA:
      if (d->layout == SPIN_I8)
        return ((d->dim == 2 || d->dim == 3) && d->n_real <= 131072) ? SPIN_OK : SPIN_EINVAL;
      if (d->layout == SPIN_MSC1)
        return ((d->dim == 2 || d->dim == 3) && d->n_real % 32 == 0 && d->n_real / 32 < 4096) ? SPIN_OK
                                                                                               : SPIN_EINVAL;
      return SPIN_EINVAL;
    case SPIN_HEISENBERG:
      return ((d->dim == 2 || d->dim == 3) && d->layout == SPIN_F32X4 && d->n_real <= 4096) ? SPIN_OK
                                                                                              : SPIN_EINVAL;
    default:
      return SPIN_EINVAL;
  }
}

void free_workspaces(spin_lattice *h) {
  void *bufs[] = {h->d_thr,    h->d_pt_thr,      h->d_pt_off, h->d_pt_len,    h->d_pt_dbeta, h->d_energy,
                  h->d_scratch64, h->d_err, h->d_pingpong, h->d_ctr, h->d_bar,  h->d_escr, h->d_res_flags};
  for (void *b : bufs)
    if (b) cudaFree(b);
}

cudaError_t do_sweeps(spin_lattice *h, const void *J, int64_t n) {
  if (n <= 0) return cudaSuccess;
  switch (h->d.layout) {
    case SPIN_I8:
      return launch_sweeps_i8(h, (const int8_t *)J, n);
    case SPIN_MSC1:
      return launch_sweeps_msc(h, (const uint32_t *)J, n);
    default:
      return launch_sweeps_heis(h, n);
  }
}

bool ea(const spin_lattice *h) { return h->d.model == SPIN_EA; }

}  // namespace

namespace spin {
int upload_thresholds_for_batch(spin_lattice *h, const double *betas) { return upload_thresholds(h, betas); }
int upload_pt_tables_for_batch(spin_lattice *h, const double *betas) {
  if (!betas) return SPIN_EINVAL;
  return upload_pt_tables(h, betas);
}
// True when the tables for these betas are already on the device (nothing
// would be uploaded, so the call is safe inside a stream capture).
bool tables_cached_for_batch(const spin_lattice *h, const double *betas, bool pt) {
  const size_t nb = sizeof(double) * (size_t)h->g.n_temps;
  if (!betas || !h->thr_valid || memcmp(h->betas_cached.data(), betas, nb) != 0) return false;
  return !pt || (!h->pt_betas_cached.empty() && memcmp(h->pt_betas_cached.data(), betas, nb) == 0);
}
bool fused2d_supported(int L);
bool coded_i8_supported(const spin_lattice *h);
cudaError_t launch_init_msc2d(spin_lattice *h);
}

extern "C" {

int spin_init(spin_lattice **out, const spin_desc *desc, void *spins, void *couplings) {
  if (!out) return SPIN_EINVAL;
  *out = nullptr;
  int rc = validate_desc(desc);
  if (rc) return rc;
  if (!spins) return SPIN_EINVAL;
  if (!aligned16(spins) || (couplings && !aligned16(couplings))) return SPIN_EALIGN;
  if (desc->model == SPIN_EA && !couplings) return SPIN_EINVAL;
  spin_lattice *h = new (std::nothrow) spin_lattice();
  if (!h) return SPIN_ENOMEM;
  h->d = *desc;
  h->msc_width = 32;
  h->stream = (cudaStream_t)desc->stream;
  h->spins = spins;
  h->couplings = couplings;
  h->g.dim = desc->dim;
  h->g.L = desc->L;
  h->g.N = 1;
  for (int k = 0; k < desc->dim; ++k) h->g.N *= desc->L;
  h->g.n_real = desc->n_real;
  h->g.n_temps = desc->n_temps;
  h->g.n_sets = desc->n_sets;
  h->g.ea = desc->model == SPIN_EA;
  h->g.fL = make_fastdiv((uint32_t)desc->L);
  h->g.fHalfL = make_fastdiv((uint32_t)(desc->L / 2));
  h->g.fhalf = make_fastdiv((uint32_t)(h->g.N / 2));
  h->g.fquads = make_fastdiv((uint32_t)((h->g.N / 2 + 3) / 4));
  h->g.freal = make_fastdiv((uint32_t)desc->n_real);
  h->g.ftemps = make_fastdiv((uint32_t)desc->n_temps);
  h->g.fgrp = make_fastdiv((uint32_t)std::max(1, desc->n_real / 32));
  h->g.fgrp2 = make_fastdiv((uint32_t)std::max(1, desc->n_real / 64));
  h->n_lat = (int64_t)desc->n_sets * desc->n_temps * desc->n_real;
  const bool i8 = desc->model == SPIN_ISING && desc->layout == SPIN_I8, i8_2d = i8 && desc->dim == 2;
  h->variant = i8 && resident_supported(desc->dim, desc->L)
                   ? 3
                   : (i8_2d && coded_i8_supported(h) ? 4 : (i8_2d && fused2d_supported(desc->L) ? 1 : 0));
  const int nt = desc->n_temps;
  bool ok = cudaMalloc(&h->d_thr, 16 * (size_t)nt) == cudaSuccess &&
            cudaMalloc(&h->d_pt_off, 4 * (size_t)nt) == cudaSuccess &&
            cudaMalloc(&h->d_pt_len, 4 * (size_t)nt) == cudaSuccess &&
            cudaMalloc(&h->d_pt_dbeta, 8 * (size_t)nt) == cudaSuccess &&
            cudaMalloc(&h->d_energy, 8 * (size_t)(3 * h->n_lat + 2)) == cudaSuccess &&
            cudaMalloc(&h->d_scratch64, 8 * (size_t)(h->n_lat * 64 * 4 + 64)) == cudaSuccess &&
            cudaMalloc(&h->d_err, sizeof(int)) == cudaSuccess;
  if (!ok) {
    free_workspaces(h);
    delete h;
    cudaGetLastError();
    return SPIN_ENOMEM;
  }
  cudaError_t e = cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
  if (e == cudaSuccess) {
    if (desc->model == SPIN_HEISENBERG) {
      e = launch_init_heis(h);
    } else if (desc->layout == SPIN_I8) {
      e = launch_init_i8(h);
      if (e == cudaSuccess && ea(h)) e = launch_couplings_i8(h);
    } else if (desc->model == SPIN_EA) {
      e = launch_init_msc(h);
      if (e == cudaSuccess) e = launch_couplings_msc(h);
    } else {
      e = launch_init_msc2d(h);
    }
  }
  if (e != cudaSuccess) {
    free_workspaces(h);
    delete h;
    return SPIN_ECUDA;
  }
  *out = h;
  return SPIN_OK;
}

int spin_sweep(spin_lattice *h, const void *couplings, const double *betas, int64_t n_sweeps,
               uint64_t seed) {
  NvtxRange nvtx_range("spin_sweep");
  if (!h || n_sweeps < 0 || seed != h->d.seed) return SPIN_EINVAL;
  if (ea(h) && !couplings) return SPIN_EINVAL;
  if (couplings && !aligned16(couplings)) return SPIN_EALIGN;
  if (h->sweeps_done + n_sweeps > (int64_t)0xFFFFFFFFll) return SPIN_EINVAL;
  if (h->order != SPIN_ORDER_CHECKERBOARD &&
      (n_sweeps % h->order_hits != 0 || h->sweeps_done % h->order_hits != 0 || h->order_tile == 0))
    return SPIN_EINVAL;  // whole compound moves only, and a tile edge chosen
  int rc = upload_thresholds(h, betas);
  if (rc) return rc;
  cudaError_t e = h->order != SPIN_ORDER_CHECKERBOARD ? launch_sweeps_dcb(h, n_sweeps)
                                                      : do_sweeps(h, ea(h) ? couplings : nullptr, n_sweeps);
  if (e != cudaSuccess) return SPIN_ECUDA;
  h->sweeps_done += n_sweeps;
  return SPIN_OK;
}

int spin_measure(spin_lattice *h, const void *couplings, int64_t *E, int64_t *M, int64_t *Q,
                 double *Ef, double *Mf) {
  NvtxRange nvtx_range("spin_measure");
  if (!h) return SPIN_EINVAL;
  if (ea(h) && !couplings) return SPIN_EINVAL;
  if (couplings && !aligned16(couplings)) return SPIN_EALIGN;
  return cuda_status(launch_measure(h, ea(h) ? couplings : nullptr, E, M, Q, Ef, Mf));
}

namespace {
// One exchange step; `energies` (device, [n_lat]) are the lattices' current
// energies when the caller has just measured them, else NULL.
int pt_swap(spin_lattice *h, const void *couplings, const double *betas, uint64_t seed,
            int64_t *accepted, int32_t *labels, const int64_t *energies) {
  if (!h || seed != h->d.seed || !betas) return SPIN_EINVAL;
  if (h->d.model == SPIN_HEISENBERG) return SPIN_EINVAL;
  if (ea(h) && !couplings) return SPIN_EINVAL;
  int rc = upload_pt_tables(h, betas);
  if (rc) return rc;
  cudaError_t e = launch_pt_swap(h, ea(h) ? couplings : nullptr, accepted, labels, energies);
  if (e != cudaSuccess) return SPIN_ECUDA;
  h->pt_steps_done += 1;
  return SPIN_OK;
}
}  // namespace

int spin_pt_swap(spin_lattice *h, const void *couplings, const double *betas, uint64_t seed,
                 int64_t *accepted, int32_t *labels) {
  NvtxRange nvtx_range("spin_pt_swap");
  return pt_swap(h, couplings, betas, seed, accepted, labels, nullptr);
}

int spin_run(spin_lattice *h, const void *couplings, const double *betas, int64_t n_sweeps,
             int32_t measure_every, int32_t pt_every, int64_t *E_series, int64_t *M_series,
             int64_t *Q_series, double *Ef_series, double *Mf_series, int64_t *accepted,
             int32_t *labels) {
  NvtxRange nvtx_range("spin_run");
  if (!h || n_sweeps < 0) return SPIN_EINVAL;
  if (pt_every > 0 && h->d.model == SPIN_HEISENBERG) return SPIN_EINVAL;
  const bool measuring = measure_every > 0 && (E_series || M_series || Q_series || Ef_series || Mf_series);
  int64_t done = 0, k_meas = 0;
  // small int8 ferromagnets: the resident kernel measures E and M itself,
  // so a call is one launch per exchange interval
  const bool resident = measuring && h->d.model == SPIN_ISING && h->d.layout == SPIN_I8 && h->variant == 3 &&
                        resident_supported(h->d.dim, h->g.L) && h->order == SPIN_ORDER_CHECKERBOARD &&
                        !Q_series && !Ef_series && !Mf_series;
  while (resident && done < n_sweeps) {
    const int64_t cur = h->sweeps_done;
    int64_t next = n_sweeps - done;
    if (pt_every > 0) {
      const int64_t to = pt_every - (cur % pt_every);
      if (to < next) next = to;
    }
    if (cur + next > (int64_t)0xFFFFFFFFll) return SPIN_EINVAL;
    int rc = upload_thresholds(h, betas);
    if (rc) return rc;
    const int64_t nl = h->n_lat;
    const int first = (int)(measure_every - cur % measure_every);
    if (launch_resident(h, next, E_series ? E_series + k_meas * nl : nullptr,
                          M_series ? M_series + k_meas * nl : nullptr, measure_every, first) != cudaSuccess)
      return SPIN_ECUDA;
    h->sweeps_done += next;
    done += next;
    const int64_t now = h->sweeps_done;
    k_meas += now / measure_every - cur / measure_every;
    if (pt_every > 0 && now % pt_every == 0) {
      const int64_t *energies = E_series && now % measure_every == 0 ? E_series + (k_meas - 1) * nl : nullptr;
      rc = pt_swap(h, couplings, betas, h->d.seed, accepted, labels, energies);
      if (rc) return rc;
    }
  }
  while (done < n_sweeps) {
    // sweep up to the next measurement or exchange point
    const int64_t cur = h->sweeps_done;
    int64_t next = n_sweeps - done;
    if (measuring) {
      const int64_t to = measure_every - (cur % measure_every);
      if (to < next) next = to;
    }
    if (pt_every > 0) {
      const int64_t to = pt_every - (cur % pt_every);
      if (to < next) next = to;
    }
    int rc = spin_sweep(h, couplings, betas, next, h->d.seed);
    if (rc) return rc;
    done += next;
    const int64_t now = h->sweeps_done;
    const int64_t *energies = nullptr;  // energies measured at this sweep, if any
    if (measuring && now % measure_every == 0) {
      const int64_t nl = h->n_lat;
      const int64_t nq = (int64_t)h->g.n_temps * h->g.n_real;
      rc = spin_measure(h, couplings, E_series ? E_series + k_meas * nl : nullptr,
                        M_series ? M_series + k_meas * nl : nullptr,
                        Q_series ? Q_series + k_meas * nq : nullptr,
                        Ef_series ? Ef_series + k_meas * nl : nullptr,
                        Mf_series ? Mf_series + 3 * k_meas * nl : nullptr);
      if (rc) return rc;
      if (E_series) energies = E_series + k_meas * nl;
      ++k_meas;
    }
    if (pt_every > 0 && now % pt_every == 0) {
      rc = pt_swap(h, couplings, betas, h->d.seed, accepted, labels, energies);
      if (rc) return rc;
    }
  }
  return SPIN_OK;
}

int spin_unpack_i8(spin_lattice *h, int8_t *out) {
  if (!h || !out) return SPIN_EINVAL;
  if (h->d.layout == SPIN_I8)
    return cuda_status(cudaMemcpyAsync(out, h->spins, (size_t)(h->n_lat * h->g.N),
                                       cudaMemcpyDeviceToDevice, h->stream));
  if (h->d.layout != SPIN_MSC1) return SPIN_EINVAL;
  return cuda_status(launch_unpack_msc(h, out));
}

int spin_pack_i8(spin_lattice *h, const int8_t *in) {
  if (!h || !in) return SPIN_EINVAL;
  if (h->d.layout == SPIN_I8)
    return cuda_status(cudaMemcpyAsync(h->spins, in, (size_t)(h->n_lat * h->g.N),
                                       cudaMemcpyDeviceToDevice, h->stream));
  if (h->d.layout != SPIN_MSC1) return SPIN_EINVAL;
  return cuda_status(launch_pack_msc(h, in));
}

int spin_rng_fill(uint64_t seed, uint32_t tag, uint32_t colour, uint32_t extra,
                  uint32_t lattice_id, uint32_t sweep, uint64_t count, uint32_t *out,
                  void *stream) {
  if (tag > 15 || colour > 1 || extra >= (1u << 27) || (count && !out)) return SPIN_EINVAL;
  if (!aligned16(out)) return SPIN_EALIGN;
  if (count > (uint64_t)4 << 32) return SPIN_EINVAL;
  return cuda_status(launch_rng_fill(seed, ctr_w(tag, colour, extra), lattice_id, sweep, count,
                                     out, (cudaStream_t)stream));
}

int spin_rng_probe(uint64_t seed, uint32_t threads, uint32_t calls, uint32_t *out, void *stream) {
  if (threads && !out) return SPIN_EINVAL;
  if ((uint64_t)threads * calls > 0xFFFFFFFFull) return SPIN_EINVAL;  // counters stay distinct
  return cuda_status(launch_rng_probe(seed, threads, calls, out, (cudaStream_t)stream));
}

int spin_pipe_probe(int op, int32_t blocks_per_sm, uint32_t iters, int64_t *clocks, uint32_t *sink,
                    int32_t *sms, void *stream) {
  if (op < SPIN_PIPE_MUL_WIDE || op > SPIN_PIPE_MUFU_RSQ || blocks_per_sm < 1 || blocks_per_sm > 8 || !clocks ||
      !sink)
    return SPIN_EINVAL;
  return launch_pipe_probe(op, blocks_per_sm, iters, reinterpret_cast<long long *>(clocks), sink, sms,
                           (cudaStream_t)stream);
}

int spin_sync(spin_lattice *h) {
  if (!h) return SPIN_EINVAL;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return SPIN_ECUDA;
  if (cudaGetLastError() != cudaSuccess) return SPIN_ECUDA;
  int err = 0;
  if (cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SPIN_ECUDA;
  if (err) {
    cudaMemset(h->d_err, 0, sizeof(int));
    return SPIN_ETIMEOUT;
  }
  return SPIN_OK;
}

int64_t spin_sweeps_done(const spin_lattice *h) { return h ? h->sweeps_done : -1; }
int spin_describe(const spin_lattice *h, spin_desc *out) {
  if (!h || !out) return SPIN_EINVAL;
  *out = h->d;
  return SPIN_OK;
}
int64_t spin_pt_steps_done(const spin_lattice *h) { return h ? h->pt_steps_done : -1; }

int spin_set_counters(spin_lattice *h, int64_t sweeps_done, int64_t pt_steps_done) {
  if (!h || sweeps_done < 0 || pt_steps_done < 0 || sweeps_done > (int64_t)0xFFFFFFFFll)
    return SPIN_EINVAL;
  h->sweeps_done = sweeps_done;
  h->pt_steps_done = pt_steps_done;
  return spin::sync_device_counters(h, h->stream);
}

int spin_set_batch_options(spin_lattice *h, uint64_t timeout_ns, int32_t ctas_per_sm,
                           int32_t missing_arrivals) {
  if (!h || ctas_per_sm < 0 || ctas_per_sm > 8 || missing_arrivals < 0) return SPIN_EINVAL;
  h->batch_timeout_ns = timeout_ns;
  h->batch_ctas_per_sm = ctas_per_sm;
  h->batch_fault_extra = missing_arrivals;
  return SPIN_OK;
}

int spin_set_msc_width(spin_lattice *h, int32_t width) {
  if (!h || h->d.model != SPIN_EA || h->d.layout != SPIN_MSC1) return SPIN_EINVAL;
  if (width != 32 && !(width == 64 && h->g.n_real % 64 == 0)) return SPIN_EINVAL;
  h->msc_width = width;
  return SPIN_OK;
}

int spin_set_update_order(spin_lattice *h, int32_t order, int32_t tile, int32_t hits) {
  if (!h) return SPIN_EINVAL;
  if (order == SPIN_ORDER_CHECKERBOARD) {
    h->order = order;
    return SPIN_OK;
  }
  if ((order != SPIN_ORDER_DCB && order != SPIN_ORDER_DCB_SYMMETRIC) || hits < 1 || hits > (1 << 20))
    return SPIN_EINVAL;
  if (tile == 0) {  // chosen later by spin_tune: some tile edge must fit
    bool any = false;
    for (int t : {8, 16, 32, 64, 128}) any = any || spin::dcb_supported(h, t);
    if (!any) return SPIN_EINVAL;
  } else if (!spin::dcb_supported(h, tile)) {
    return SPIN_EINVAL;
  }
  h->order = order;
  h->order_tile = tile;
  h->order_hits = hits;
  return SPIN_OK;
}

int spin_set_variant(spin_lattice *h, int32_t variant) {
  if (!h || variant < 0 || variant > 4) return SPIN_EINVAL;
  const bool i8 = h->d.model == SPIN_ISING && h->d.layout == SPIN_I8, i8_2d = i8 && h->d.dim == 2;
  if (variant == 1 && !(i8_2d && fused2d_supported(h->g.L))) return SPIN_EINVAL;
  if (variant == 4 && !(coded_i8_supported(h) && fused2d_supported(h->g.L))) return SPIN_EINVAL;
  if (variant == 3 && !(i8 && resident_supported(h->d.dim, h->g.L))) return SPIN_EINVAL;
  if (variant == 2 && h->d.model != SPIN_HEISENBERG) return SPIN_EINVAL;
  h->variant = variant;
  return SPIN_OK;
}

const char *spin_strerror(int code) {
  switch (code) {
    case SPIN_OK: return "ok";
    case SPIN_EINVAL: return "invalid argument";
    case SPIN_EALIGN: return "device pointer not 16-byte aligned";
    case SPIN_ENOMEM: return "device workspace allocation failed";
    case SPIN_ECUDA: return "CUDA error";
    case SPIN_ETIMEOUT: return "device-side wait timed out";
    default: return "unknown error";
  }
}

void spin_destroy(spin_lattice *h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_workspaces(h);
  delete h;
}

}  // extern "C"
