// C ABI of the QED particle-step library (declared in include/qed.h).
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "qed_internal.h"

size_t qed_record_bytes(int prec);
size_t qed_pend_bytes(int prec);
size_t qed_step_const_bytes();
size_t qed_clock_bytes();
int qed_launch_count_live(qed_ctx *c, long long *d_live, cudaStream_t s);

namespace {

cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

template <typename T> int dalloc(T **p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return QED_OK;
  return cudaMalloc((void **)p, bytes) == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

size_t table_bytes(int prec) {
  return prec == 64 ? sizeof(double) * qed::Tab<double>::kSize : sizeof(float) * qed::Tab<float>::kSize;
}

void release(qed_ctx *c) {
  for (int sp = 0; sp < 4; ++sp)
    for (int b = 0; b < 2; ++b) {
      cudaFree(c->st[sp].pos[b]);
      cudaFree(c->st[sp].mom[b]);
      cudaFree(c->st[sp].id[b]);
    }
  cudaFree(c->pend[0]);
  cudaFree(c->pend[1]);
  cudaFree(c->d_count);
  cudaFree(c->d_nstart);
  cudaFree(c->d_pend_count);
  cudaFree(c->d_counters);
  cudaFree(c->d_spec);
  cudaFree(c->d_spec_e);
  cudaFree(c->d_status);
  cudaFree(c->d_barrier);
  cudaFree(c->d_tables);
  cudaFree(c->d_chi_star);
  cudaFree(c->d_eps_star);
  cudaFree(c->d_step_const);
  cudaFree(c->d_clock);
  cudaFree(c->d_blk_start);
  cudaFree(c->d_blk_cursor);
  cudaFree(c->d_tile);
  cudaFree(c->stage);
  cudaFree(c->d_ens);
  cudaFree(c->d_ens_h);
  cudaFree(c->d_std_cdf);
  cudaFree(c->d_grid_max);
  cudaFree(c->d_drift);
  cudaFree(c->d_grid_max_next);
  cudaFree(c->d_phot_start);
  cudaFree(c->d_std_lnw);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  cudaFree(c->d_ens_field);
  cudaFree(c->d_thin);
}

int read_counters(qed_ctx *c, unsigned long long *cnt, cudaStream_t s) {
  if (cudaMemcpyAsync(cnt, c->d_counters, sizeof(unsigned long long) * qed::kNumCounters, cudaMemcpyDeviceToHost,
                      s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return QED_ERR_CUDA;
  return QED_OK;
}

int check_tuning(const qed_ctx *c, const qed_tuning *t) {
  int maxp = 0, maxm = 0;
  if (qed_step_kernel_max_blocks(const_cast<qed_ctx *>(c), &maxp, &maxm) != QED_OK) return QED_ERR_CUDA;
  if (t->photon_blocks_per_sm < 1 || t->photon_blocks_per_sm > maxp) return QED_ERR_ARG;
  if (t->massive_blocks_per_sm < 1 || t->massive_blocks_per_sm > maxm) return QED_ERR_ARG;
  if (t->work_chunk < 0 || t->work_chunk % 256 != 0 || t->work_chunk > (1 << 24)) return QED_ERR_ARG;
  if (t->compact_interval < 1 || (t->sort_massive != 0 && t->sort_massive != 1)) return QED_ERR_ARG;
  if (t->concurrent != 0 && t->concurrent != 1) return QED_ERR_ARG;
  if (t->deposit_halo < 0 || t->deposit_halo > qed::kMaxDepositHalo) return QED_ERR_ARG;
  if (t->refill_lanes < 0 || t->refill_lanes > 32) return QED_ERR_ARG;
  return QED_OK;
}

// Classify a caller pointer: returns a device-usable alias, or nullptr when
// it is ordinary (pageable) host memory that must be staged.
const void *device_alias(const void *p) {
  if (!p) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
  if (at.type == cudaMemoryTypeHost) {
    void *dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, const_cast<void *>(p), 0) == cudaSuccess) return dp;
    cudaGetLastError();
  }
  return nullptr;
}

// p itself when it is device (or managed) memory, else NULL.
const void *device_memory(const void *p) {
  if (!p) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) ? p : nullptr;
}

int ensure_stage(qed_ctx *c, size_t bytes) {
  if (c->stage_bytes >= bytes) return QED_OK;
  cudaFree(c->stage);
  c->stage = nullptr;
  c->stage_bytes = 0;
  if (cudaMalloc(&c->stage, bytes) != cudaSuccess) return QED_ERR_CUDA;
  c->stage_bytes = bytes;
  return QED_OK;
}

int read_status(qed_ctx *c, cudaStream_t s) {
  int bits = 0;
  if (cudaMemcpyAsync(&bits, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return QED_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return QED_ERR_CUDA;
  return qed_latch_status(c, bits);
}

}  // namespace

extern "C" {

const char *qed_error_string(int status) {
  switch (status) {
    case QED_OK: return "ok";
    case QED_ERR_ARG: return "invalid argument";
    case QED_ERR_CUDA: return "CUDA runtime call failed";
    case QED_ERR_CAPACITY: return "particle or product buffer capacity exceeded";
    case QED_ERR_NONFINITE: return "non-finite field or momentum";
    case QED_ERR_TIMEOUT: return "bounded device wait gave up or products nested too deeply";
    case QED_ERR_PMGT1: return "event probability above one with pm_strict";
    case QED_ERR_STATE: return "context holds an earlier device error";
    case QED_ERR_COURANT: return "charged particle moved a cell or more in one step";
    default: return "unknown status";
  }
}

int qed_init(qed_ctx **out, const qed_grid_desc *g, const qed_species_desc *sp, const void *tables,
             size_t tables_bytes, const qed_params *p, void *stream) {
  if (!out) return QED_ERR_ARG;
  *out = nullptr;
  if (!g || !sp || !p) return QED_ERR_ARG;
  if (p->precision != 32 && p->precision != 64) return QED_ERR_ARG;
  long long ncell = 1;
  for (int k = 0; k < 3; ++k) {
    if (g->n[k] < 1 || !(g->d[k] > 0.0) || !std::isfinite(g->d[k]) || !std::isfinite(g->x0[k]))
      return QED_ERR_ARG;
    ncell *= g->n[k];
  }
  if (ncell >= (1ll << 31)) return QED_ERR_ARG;
  if (g->field_mode < QED_FIELD_GRID || g->field_mode > QED_FIELD_STANDING_WAVE || g->reserved != 0)
    return QED_ERR_ARG;
  if (g->field_mode == QED_FIELD_GRID) {
    for (int k = 0; k < 3; ++k)
      if (!g->periodic[k]) return QED_ERR_ARG;
    if (g->n[2] > 65535 || (g->n[1] + 7) / 8 > 65535) return QED_ERR_ARG;   // the FDTD launch shape
  }
  if (p->nsub_max < 1 || !(p->kappa > 0.0) || p->nbins < 0 || p->nbins > qed::kMaxBins)
    return QED_ERR_ARG;
  if (p->nbins > 0 && !(p->lg_hi > p->lg_lo)) return QED_ERR_ARG;
  if (p->pending_capacity < 0 || p->compact_interval < 0) return QED_ERR_ARG;
  if (p->ens_bits < 0 || p->ens_bits > QED_MAX_ENS_BITS || p->thin_interval < 0) return QED_ERR_ARG;
  if (!std::isfinite(p->emit_fg) || !std::isfinite(p->pair_fg) || p->emit_ng > 64 || p->pair_ng > 64)
    return QED_ERR_ARG;
  if (p->generator < QED_GEN_MODIFIED || p->generator > QED_GEN_STANDARD || p->reserved_gen != 0) return QED_ERR_ARG;
  if (p->generator != QED_GEN_MODIFIED && (p->emit_fg > 1.0 || p->emit_ng > 1)) return QED_ERR_ARG;
  if ((p->schwinger_on != 0 && p->schwinger_on != 1) || p->reserved_s != 0) return QED_ERR_ARG;
  if (p->schwinger_on && (!(p->schwinger_weight > 0.0) || !std::isfinite(p->schwinger_weight) ||
                          g->field_mode == QED_FIELD_ENSEMBLE))
    return QED_ERR_ARG;
  bool thinning = false;
  for (int k = 0; k < 4; ++k) {
    if (p->thin_limit[k] < 0) return QED_ERR_ARG;
    thinning |= p->thin_limit[k] > 0;
  }
  long long total_cap = 0, max_cap = 0;
  for (int k = 0; k < 4; ++k) {
    if (sp->capacity[k] < 0 || sp->capacity[k] > (1ll << 40)) return QED_ERR_ARG;
    if (k != QED_PHOTON && !(sp->mass[k] > 0.0)) return QED_ERR_ARG;
    total_cap += sp->capacity[k];
    max_cap = sp->capacity[k] > max_cap ? sp->capacity[k] : max_cap;
  }
  if (tables && tables_bytes != table_bytes(p->precision)) return QED_ERR_ARG;

  qed_ctx *c = new (std::nothrow) qed_ctx();
  if (!c) return QED_ERR_CUDA;
  c->prec = p->precision;
  c->grid = *g;
  c->species = *sp;
  c->par = *p;
  c->ext = g->field_mode == QED_FIELD_ENSEMBLE || p->emit_fg > 1.0 || p->pair_fg > 1.0 || p->emit_ng > 1 ||
           p->pair_ng > 1 || p->generator != QED_GEN_MODIFIED;
  cudaStream_t s = as_stream(stream);
  int rc = QED_OK;
  cudaDeviceProp prop;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return QED_ERR_CUDA;
  }
  c->num_sms = prop.multiProcessorCount;
  const size_t rec = qed_record_bytes(c->prec);  // pos + mom
  for (int k = 0; k < 4 && rc == QED_OK; ++k) {
    c->st[k].cap = sp->capacity[k];
    for (int b = 0; b < 2 && rc == QED_OK; ++b) {
      rc = dalloc(&c->st[k].pos[b], rec / 2 * sp->capacity[k]);
      if (rc == QED_OK) rc = dalloc(&c->st[k].mom[b], rec / 2 * sp->capacity[k]);
      if (rc == QED_OK) rc = dalloc(&c->st[k].id[b], sizeof(uint64_t) * sp->capacity[k]);
    }
  }
  c->pend_cap = p->pending_capacity > 0 ? p->pending_capacity
                                        : (total_cap / 8 > 65536 ? total_cap / 8 : 65536);
  if (rc == QED_OK) rc = dalloc(&c->pend[0], qed_pend_bytes(c->prec) * c->pend_cap);
  if (rc == QED_OK) rc = dalloc(&c->pend[1], qed_pend_bytes(c->prec) * c->pend_cap);
  if (rc == QED_OK) rc = dalloc(&c->d_count, 8 * sizeof(long long));   // [4 + 4]: sort totals
  if (rc == QED_OK) rc = dalloc(&c->d_nstart, 4 * sizeof(long long));
  // product counts per pass, then the work counters of the cell-block kernel
  if (rc == QED_OK) rc = dalloc(&c->d_pend_count, sizeof(unsigned long long) * (qed::kMaxPass + 5));
  if (g->field_mode == QED_FIELD_GRID) {
    long long nblk = 1;
    for (int k = 0; k < 3; ++k) {
      c->nb[k] = (g->n[k] + qed::kBlockCells - 1) / qed::kBlockCells;
      nblk *= c->nb[k];
    }
    c->nblk = (int)nblk;
    // records are sorted by cell, cell blocks in order and the cells of a
    // block in order, where the keys fit an int; else by cell block alone
    c->blk_keys = nblk * qed::kBlockVolume + 1 < (1ll << 31) ? qed::kBlockVolume : 1;
    const long long nkeys = nblk * c->blk_keys + 1;   // + 1: the photons that cannot pair
    if (rc == QED_OK) rc = dalloc(&c->d_blk_start, sizeof(unsigned) * 4 * (nblk + 1));
    // cursors (nkeys + 2), then the sums of the scan (one per 16384 keys; at
    // most one per 1024 allocated)
    if (rc == QED_OK) rc = dalloc(&c->d_blk_cursor, sizeof(unsigned) * (nkeys + 2 + (nkeys + 1024) / 1024 + 1));
    if (rc == QED_OK) rc = dalloc(&c->d_phot_start, sizeof(unsigned) * (nblk + 2));
    if (rc == QED_OK) rc = dalloc(&c->d_grid_max, sizeof(unsigned long long) * 6);
    if (c->par.deposit_on) {
      // the records that drift out of their block's current tile between
      // sorts: an eighth of the charged stores' capacity (more deposit directly)
      const long long charged = (long long)c->st[QED_ELECTRON].cap + c->st[QED_POSITRON].cap + c->st[QED_ION].cap;
      c->drift_cap = charged / 8 > (1ll << 20) ? charged / 8 : (1ll << 20);
      if (rc == QED_OK) rc = dalloc(&c->d_drift, sizeof(unsigned long long) * c->drift_cap);
    }
    if (rc == QED_OK) rc = dalloc(&c->d_grid_max_next, sizeof(unsigned long long) * 6 * qed::kMaxStripes);
  }
  if (g->field_mode == QED_FIELD_ENSEMBLE) {
    c->ens_cap = 1 << p->ens_bits;
    if (rc == QED_OK) rc = dalloc(&c->d_ens, sizeof(double) * QED_ENS_STRIDE * c->ens_cap);
    if (rc == QED_OK) rc = dalloc(&c->d_ens_h, sizeof(float) * c->ens_cap);
    if (rc == QED_OK)
      rc = dalloc(&c->d_ens_field, (c->prec == 64 ? sizeof(double) : sizeof(float)) * qed::kEnsFieldStride *
                                       c->ens_cap);
    {
      // counting sort of e-, e+ and ions by their estimated sub-interval count
      c->key_ensembles = 1;
      c->nblk = qed::kNsubKeys;
      if (rc == QED_OK) rc = dalloc(&c->d_blk_start, sizeof(unsigned) * 4 * (c->nblk + 1));
      if (rc == QED_OK) rc = dalloc(&c->d_blk_cursor, sizeof(unsigned) * (c->nblk + 2 + (c->nblk + 1024) / 1024 + 1));
    }
  }
  if (thinning) {
    c->thin_groups = (p->ens_bits > 0 && g->field_mode == QED_FIELD_ENSEMBLE) ? (1 << p->ens_bits) : 1;
    if (rc == QED_OK) rc = dalloc(&c->d_thin, (size_t)24 * c->thin_groups);
  }
  if (p->generator == QED_GEN_STANDARD) {
    const size_t r = c->prec == 64 ? sizeof(double) : sizeof(float);
    if (rc == QED_OK) rc = dalloc(&c->d_std_cdf, r * qed::kStdRows * qed::kStdCols);
    if (rc == QED_OK) rc = dalloc(&c->d_std_lnw, r * qed::kStdRows);
  }
  if (rc == QED_OK) rc = dalloc(&c->d_counters, sizeof(unsigned long long) * qed::kNumCounters);
  if (rc == QED_OK) rc = dalloc(&c->d_spec, sizeof(double) * (p->nbins > 0 ? p->nbins : 1));
  if (rc == QED_OK) rc = dalloc(&c->d_spec_e, sizeof(double) * (p->nbins > 0 ? p->nbins : 1));
  if (rc == QED_OK) rc = dalloc(&c->d_status, sizeof(int) * 4);
  if (rc == QED_OK) rc = dalloc(&c->d_barrier, sizeof(unsigned) * 4);
  c->tables_bytes = table_bytes(c->prec);
  if (rc == QED_OK) rc = dalloc(&c->d_tables, c->tables_bytes);
  if (rc == QED_OK) rc = dalloc(&c->d_chi_star, sizeof(double));
  if (rc == QED_OK) rc = dalloc(&c->d_eps_star, sizeof(double));
  if (rc == QED_OK) rc = dalloc(&c->d_step_const, qed_step_const_bytes());
  if (rc == QED_OK) rc = dalloc(&c->d_clock, qed_clock_bytes());
  c->tile_cap = 2 * ((max_cap + qed::kCompactTile - 1) / qed::kCompactTile + 2);   // two classes
  if (rc == QED_OK) rc = dalloc(&c->d_tile, sizeof(long long) * c->tile_cap);
  if (rc == QED_OK) {
    cudaMemsetAsync(c->d_count, 0, 8 * sizeof(long long), s);
    cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long) * qed::kNumCounters, s);
    cudaMemsetAsync(c->d_spec, 0, sizeof(double) * (p->nbins > 0 ? p->nbins : 1), s);
    cudaMemsetAsync(c->d_spec_e, 0, sizeof(double) * (p->nbins > 0 ? p->nbins : 1), s);
    cudaMemsetAsync(c->d_status, 0, sizeof(int) * 4, s);
    cudaMemsetAsync(c->d_barrier, 0, sizeof(unsigned) * 4, s);
    cudaMemsetAsync(c->d_clock, 0, qed_clock_bytes(), s);    // t = 0, step = 0
    if (tables)
      rc = cudaMemcpyAsync(c->d_tables, tables, c->tables_bytes, cudaMemcpyHostToDevice, s) == cudaSuccess
               ? QED_OK : QED_ERR_CUDA;
    else
      rc = qed_build_tables(c, s);
  }
  if (rc == QED_OK && p->generator == QED_GEN_STANDARD) rc = qed_build_standard_tables(c, s);
  if (rc == QED_OK) rc = qed_launch_chi_star(c, s);
  if (rc == QED_OK) rc = qed_step_kernel_blocks(c);
  if (rc == QED_OK) {
    int maxp = 0, maxm = 0;
    rc = qed_step_kernel_max_blocks(c, &maxp, &maxm);
    c->tune.photon_blocks_per_sm = maxp;
    c->tune.massive_blocks_per_sm = maxm;
    c->tune.work_chunk = 0;
    c->tune.compact_interval = p->compact_interval > 0 ? p->compact_interval : 8;
    c->tune.sort_massive = c->key_ensembles;
    // FP32: halo 3, four blocks per SM (measured on the 512^3 cascade:
    // 5.83 ms per step against 5.96 for halo 4 at three); FP64: halo 2
    c->tune.deposit_halo = c->prec == 64 ? 2 : 3;
  }
  if (rc == QED_OK && (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
                       cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                       cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess))
    rc = QED_ERR_CUDA;
  if (rc == QED_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = QED_ERR_CUDA;
  if (rc != QED_OK) {
    cudaGetLastError();
    release(c);
    delete c;
    return rc;
  }
  *out = c;
  return QED_OK;
}

int qed_tables_export(qed_ctx *c, void *host_buf, size_t bytes, size_t *needed) {
  if (!c) return QED_ERR_ARG;
  if (needed) *needed = c->tables_bytes;
  if (!host_buf) return QED_OK;
  if (bytes < c->tables_bytes) return QED_ERR_ARG;
  return cudaMemcpy(host_buf, c->d_tables, c->tables_bytes, cudaMemcpyDeviceToHost) == cudaSuccess
             ? QED_OK : QED_ERR_CUDA;
}

int qed_particles_set(qed_ctx *c, int sp, const double *x, const double *p, const double *w,
                      const uint64_t *id, int64_t n, void *stream) {
  if (!c || sp < 0 || sp >= QED_NSPECIES || n < 0 || n > c->st[sp].cap) return QED_ERR_ARG;
  if (n > 0 && (!x || !p || !w || !id)) return QED_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  const void *dx = device_alias(x), *dp = device_alias(p), *dw = device_alias(w), *di = device_alias(id);
  const size_t nn = (size_t)n;
  if (n > 0 && (!dx || !dp || !dw || !di)) {
    // stage pageable host arrays through device memory
    if (ensure_stage(c, 64 * nn) != QED_OK) return QED_ERR_CUDA;
    char *b = (char *)c->stage;
    if (cudaMemcpyAsync(b, x, 24 * nn, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaMemcpyAsync(b + 24 * nn, p, 24 * nn, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaMemcpyAsync(b + 48 * nn, w, 8 * nn, cudaMemcpyDefault, s) != cudaSuccess ||
        cudaMemcpyAsync(b + 56 * nn, id, 8 * nn, cudaMemcpyDefault, s) != cudaSuccess)
      return QED_ERR_CUDA;
    dx = b; dp = b + 24 * nn; dw = b + 48 * nn; di = b + 56 * nn;
  }
  c->sorted = 0;
  return qed_launch_set(c, sp, (const double *)dx, (const double *)dp, (const double *)dw,
                        (const uint64_t *)di, n, s);
}

int qed_particles_get(qed_ctx *c, int sp, double *x, double *p, double *w, uint64_t *id, int64_t max_n,
                      int64_t *n_out, void *stream) {
  if (!c || sp < 0 || sp >= QED_NSPECIES || !n_out || max_n < 0) return QED_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  int rc = qed_launch_compact(c, sp, false, s);
  if (rc != QED_OK) return rc;
  if (sp != QED_PHOTON) c->sorted = 0;   // compaction keeps the order but not the block starts
  long long n = 0;
  if (cudaMemcpyAsync(&n, c->d_count + sp, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return QED_ERR_CUDA;
  *n_out = n;
  if (n > max_n) return QED_ERR_ARG;
  if (n > 0) {
    if (!x || !p || !w || !id) return QED_ERR_ARG;
    // host buffers, page-locked or not, are filled from a device staging
    // buffer by the copy engines: kernel stores to host memory ran at a
    // third of their rate
    void *dx = (void *)device_memory(x), *dp = (void *)device_memory(p), *dw = (void *)device_memory(w),
         *di = (void *)device_memory(id);
    const size_t nn = (size_t)n;
    bool staged = !dx || !dp || !dw || !di;
    if (staged) {
      if (ensure_stage(c, 64 * nn) != QED_OK) return QED_ERR_CUDA;
      char *b = (char *)c->stage;
      dx = b; dp = b + 24 * nn; dw = b + 48 * nn; di = b + 56 * nn;
    }
    rc = qed_launch_get(c, sp, (double *)dx, (double *)dp, (double *)dw, (uint64_t *)di, n, s);
    if (rc != QED_OK) return rc;
    if (staged) {
      char *b = (char *)c->stage;
      if (cudaMemcpyAsync(x, b, 24 * nn, cudaMemcpyDefault, s) != cudaSuccess ||
          cudaMemcpyAsync(p, b + 24 * nn, 24 * nn, cudaMemcpyDefault, s) != cudaSuccess ||
          cudaMemcpyAsync(w, b + 48 * nn, 8 * nn, cudaMemcpyDefault, s) != cudaSuccess ||
          cudaMemcpyAsync(id, b + 56 * nn, 8 * nn, cudaMemcpyDefault, s) != cudaSuccess)
        return QED_ERR_CUDA;
    }
  }
  return read_status(c, s);
}

int qed_step(qed_ctx *c, const qed_fields *f, double dt, int32_t nsteps, void *stream) {
  if (!c) return QED_ERR_ARG;
  if (c->latched) return QED_ERR_STATE;
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0) return QED_ERR_ARG;
  const bool grid = c->grid.field_mode == QED_FIELD_GRID;
  if (grid) {
    if (!f) return QED_ERR_ARG;
    for (int k = 0; k < 3; ++k)
      if (!f->E[k] || !f->B[k] || (c->par.deposit_on && !f->J[k])) return QED_ERR_ARG;
  }
  if (c->grid.field_mode == QED_FIELD_ENSEMBLE && c->n_ens < 1) return QED_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  c->last_dt = dt;
  // the caller may have changed the fields since the last call
  c->grid_max_ready = 0;
  for (int n = 0; n < nsteps; ++n) {
    if (!c->ev_steps.empty()) {
      const size_t k = c->ev_steps.size() / QED_NSTAGES;
      for (int st = 0; st < QED_NSTAGES; ++st)
        c->ev_stage[st] = (size_t)n < k ? c->ev_steps[(size_t)n * QED_NSTAGES + st] : nullptr;
    }
    if (grid && c->nblk > 0 && !c->sorted) {
      // records in cell-block order let electrons, positrons and ions deposit
      // through shared-memory tiles
      for (int sp = 0; sp < 4; ++sp) {
        int rs = sp == QED_PHOTON ? QED_OK : qed_launch_sort(c, sp, s);
        if (rs != QED_OK) return rs;
      }
      c->sorted = 1;
      c->steps_since_compact = 0;
    }
    int rc = qed_launch_step(c, f, dt, s);
    if (rc == QED_OK && grid && c->par.deposit_on) rc = qed_launch_yee(c, f, dt, s);
    if (rc != QED_OK) return rc;
    qed_mark(c, QED_STAGE_FIELD, s);
    c->step += 1;
    if (c->par.thin_interval > 0 && c->step % c->par.thin_interval == 0)
      for (int sp = 0; sp < 4; ++sp)
        if ((rc = qed_launch_thin(c, sp, s)) != QED_OK) return rc;
    if (c->par.compact_interval > 0 && ++c->steps_since_compact >= c->par.compact_interval) {
      c->steps_since_compact = 0;
      for (int sp = 0; sp < 4; ++sp) {
        // grid mode: re-sort every species by cell block (photons that may
        // pair by block, the others after them); ensembles: optionally order
        // e-, e+ and ions by estimated sub-intervals; otherwise compaction
        const bool sort = c->nblk > 0 && (grid || (sp != QED_PHOTON && c->key_ensembles && c->tune.sort_massive));
        rc = sort ? qed_launch_sort(c, sp, s) : qed_launch_compact(c, sp, true, s);
        if (rc != QED_OK) return rc;
      }
    }
    qed_mark(c, QED_STAGE_END, s);
  }
  return QED_OK;
}

int qed_ensembles_set(qed_ctx *c, int32_t n_ens, const double *table, void *stream) {
  if (!c || c->grid.field_mode != QED_FIELD_ENSEMBLE || !table) return QED_ERR_ARG;
  if (n_ens < 1 || n_ens > c->ens_cap) return QED_ERR_ARG;
  double hmax = 0.0;
  float *hb = new (std::nothrow) float[n_ens];
  if (!hb) return QED_ERR_CUDA;
  for (long long e = 0; e < n_ens; ++e) {
    const double *q = table + e * QED_ENS_STRIDE;
    for (int k = 0; k < QED_ENS_STRIDE; ++k)
      if (!std::isfinite(q[k])) {
        delete[] hb;
        return QED_ERR_ARG;
      }
    // |E| + |B| <= |E0| + |Eu| + |Bu|
    const double h = std::fabs(q[0]) + std::sqrt(q[3] * q[3] + q[4] * q[4] + q[5] * q[5]) +
                     std::sqrt(q[6] * q[6] + q[7] * q[7] + q[8] * q[8]);
    hmax = h > hmax ? h : hmax;
    hb[e] = (float)h;
  }
  cudaStream_t s = as_stream(stream);
  const bool ok = cudaMemcpyAsync(c->d_ens, table, sizeof(double) * QED_ENS_STRIDE * n_ens,
                                  cudaMemcpyHostToDevice, s) == cudaSuccess &&
                  cudaMemcpyAsync(c->d_ens_h, hb, sizeof(float) * n_ens, cudaMemcpyHostToDevice, s) ==
                      cudaSuccess &&
                  cudaStreamSynchronize(s) == cudaSuccess;
  delete[] hb;
  if (!ok) return QED_ERR_CUDA;
  c->n_ens = n_ens;
  c->ens_hmax = hmax;
  int rc = qed_launch_chi_star(c, s);   // eps* = chi*/hmax changes with the fields
  if (rc != QED_OK) return rc;
  return cudaStreamSynchronize(s) == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

int qed_get_tuning(qed_ctx *c, qed_tuning *out) {
  if (!c || !out) return QED_ERR_ARG;
  *out = c->tune;
  return QED_OK;
}

int qed_set_tuning(qed_ctx *c, const qed_tuning *t) {
  if (!c || !t) return QED_ERR_ARG;
  int rc = check_tuning(c, t);
  if (rc != QED_OK) return rc;
  if (t->sort_massive && !c->key_ensembles) return QED_ERR_ARG;
  c->tune = *t;
  c->par.compact_interval = t->compact_interval;
  c->steps_since_compact = 0;   // the next compaction comes compact_interval steps later
  return QED_OK;
}

int qed_autotune(qed_ctx *c, const qed_fields *f, double dt, int32_t steps_per_trial, int64_t max_steps,
                 void *stream, qed_tuning *out, int64_t *steps_taken) {
  if (!c || steps_per_trial < 1 || !(dt > 0.0) || max_steps < 0) return QED_ERR_ARG;
  if (c->latched) return QED_ERR_STATE;
  cudaStream_t s = as_stream(stream);
  int maxp = 0, maxm = 0;
  int rc = qed_step_kernel_max_blocks(c, &maxp, &maxm);
  if (rc != QED_OK) return rc;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return QED_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return QED_ERR_CUDA;
  }
  int64_t taken = 0;
  qed_tuning best = c->tune;
  // the configured compaction interval bounds the candidates: the
  // capacities were sized for the dead records it lets accumulate
  const int ci_max = best.compact_interval;
  unsigned long long cnt[qed::kNumCounters];
  // time per particle-step of tuning t over whole compaction periods
  auto trial = [&](const qed_tuning &t, double *cost) -> int {
    c->tune = t;
    c->par.compact_interval = t.compact_interval;
    c->steps_since_compact = 0;
    const int n = steps_per_trial > t.compact_interval ? steps_per_trial : t.compact_interval;
    int r = read_counters(c, cnt, s);
    if (r != QED_OK) return r;
    unsigned long long ps0 = 0, ps1 = 0;
    for (int k = 0; k < 4; ++k) ps0 += cnt[qed::kCntSpeciesSteps + k];
    if (cudaEventRecord(e0, s) != cudaSuccess) return QED_ERR_CUDA;
    r = qed_step(c, f, dt, n, stream);
    if (r != QED_OK) return r;
    if (cudaEventRecord(e1, s) != cudaSuccess) return QED_ERR_CUDA;
    r = read_counters(c, cnt, s);
    if (r != QED_OK) return r;
    for (int k = 0; k < 4; ++k) ps1 += cnt[qed::kCntSpeciesSteps + k];
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return QED_ERR_CUDA;
    taken += n;
    *cost = ps1 > ps0 ? (double)ms / (double)(ps1 - ps0) : (double)ms;
    return read_status(c, s);
  };
  bool out_of_steps = false;
  // one field at a time; candidates in order, then reversed
  auto tune_field = [&](int32_t qed_tuning::*field, const int *cand, int nc) -> int {
    if (nc < 2 || out_of_steps) return QED_OK;
    // the whole search of this field must fit in the step budget
    int64_t need = 0;
    for (int j = 0; j < nc; ++j) {
      const int ci = field == &qed_tuning::compact_interval ? cand[j] : best.compact_interval;
      need += 2 * (steps_per_trial > ci ? steps_per_trial : ci);
    }
    if (taken + need > max_steps) {
      out_of_steps = true;
      return QED_OK;
    }
    double sum[16] = {0};
    for (int pass = 0; pass < 2; ++pass)
      for (int k = 0; k < nc; ++k) {
        const int j = pass == 0 ? k : nc - 1 - k;
        qed_tuning t = best;
        t.*field = cand[j];
        double cost = 0.0;
        int r = trial(t, &cost);
        if (r != QED_OK) return r;
        sum[j] += cost;
      }
    int jb = 0;
    for (int j = 1; j < nc; ++j)
      if (sum[j] < sum[jb]) jb = j;
    best.*field = cand[jb];
    return QED_OK;
  };
  int cand[16], nc = 0;
  for (int b = 1; b <= maxp && nc < 4; ++b) cand[nc++] = b;
  rc = tune_field(&qed_tuning::photon_blocks_per_sm, cand, nc);
  if (rc == QED_OK) {
    nc = 0;
    for (int b = 1; b <= maxm && nc < 4; ++b) cand[nc++] = b;
    rc = tune_field(&qed_tuning::massive_blocks_per_sm, cand, nc);
  }
  if (rc == QED_OK) {
    const int chunks[5] = {0, 256, 1024, 4096, 16384};
    rc = tune_field(&qed_tuning::work_chunk, chunks, 5);
  }
  if (rc == QED_OK) {
    nc = 0;
    for (int v = ci_max; v >= 1 && nc < 3; v /= 2) cand[nc++] = v;
    rc = tune_field(&qed_tuning::compact_interval, cand, nc);
  }
  if (rc == QED_OK && c->key_ensembles) {
    const int so[2] = {1, 0};
    rc = tune_field(&qed_tuning::sort_massive, so, 2);
  }
  if (rc == QED_OK && c->grid.field_mode == QED_FIELD_GRID && c->par.deposit_on) {
    // the deposit's current tiles: halo 4 .. 1, or global atomics only
    const int halos[5] = {4, 3, 2, 1, 0};
    rc = tune_field(&qed_tuning::deposit_halo, halos, 5);
  }
  if (rc == QED_OK && c->grid.field_mode == QED_FIELD_GRID) {
    // e-/e+ of the cell-block pass: whole batches, or lanes refilled in groups
    const int refill[3] = {0, 24, 16};
    rc = tune_field(&qed_tuning::refill_lanes, refill, 3);
  }
  if (rc == QED_OK) {
    // the two passes side by side: split the SM's blocks between them
    qed_tuning t = best;
    const int tot = maxp < maxm ? maxp : maxm;
    if (tot >= 2 && !out_of_steps) {
      t.concurrent = 1;
      t.photon_blocks_per_sm = tot - 1;
      t.massive_blocks_per_sm = 1;
      double c0 = 0.0, c1 = 0.0, x = 0.0;
      const int ci = best.compact_interval;
      const int64_t need = 4 * (steps_per_trial > ci ? steps_per_trial : ci);
      if (taken + need <= max_steps) {
        for (int pass = 0; pass < 2 && rc == QED_OK; ++pass) {
          rc = trial(pass == 0 ? best : t, &x);
          (pass == 0 ? c0 : c1) += x;
          if (rc == QED_OK) rc = trial(pass == 0 ? t : best, &x);
          (pass == 0 ? c1 : c0) += x;
        }
        if (rc == QED_OK && c1 < c0) best = t;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->tune = best;
  c->par.compact_interval = best.compact_interval;
  if (out) *out = best;
  if (steps_taken) *steps_taken = taken;
  return rc;
}

int qed_set_clock(qed_ctx *c, int64_t step, double time) {
  if (!c || step < 0 || !std::isfinite(time)) return QED_ERR_ARG;
  struct { double t; long long step; } clk = {time, (long long)step};
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(c->d_clock, &clk, sizeof(clk), cudaMemcpyHostToDevice) != cudaSuccess)
    return QED_ERR_CUDA;
  c->step = step;
  return QED_OK;
}

int qed_profile_events(qed_ctx *c, void *start, void *photon_done, void *stop) {
  if (!c || (start == nullptr) != (stop == nullptr) || (photon_done && !start)) return QED_ERR_ARG;
  c->ev_start = (cudaEvent_t)start;
  c->ev_photon = (cudaEvent_t)photon_done;
  c->ev_stop = (cudaEvent_t)stop;
  return QED_OK;
}

int qed_profile_stages(qed_ctx *c, void *const *events, int32_t n) {
  if (!c || n < 0 || (n > QED_NSTAGES && n % QED_NSTAGES) || (n > 0 && !events)) return QED_ERR_ARG;
  c->ev_steps.clear();
  if (n > QED_NSTAGES) {
    c->ev_steps.assign((cudaEvent_t *)events, (cudaEvent_t *)events + n);
    n = 0;   // set per step by qed_step
  }
  for (int k = 0; k < QED_NSTAGES; ++k) c->ev_stage[k] = k < n ? (cudaEvent_t)events[k] : nullptr;
  return QED_OK;
}

int qed_diagnostics(qed_ctx *c, qed_diag *out, void *stream) {
  if (!c || !out) return QED_ERR_ARG;
  if (out->nbins != 0 && out->nbins != c->par.nbins) return QED_ERR_ARG;
  cudaStream_t s = as_stream(stream);
  long long *d_live = (long long *)c->d_nstart;  // reused: only valid inside a step
  const int64_t launches = c->launches;           // before this call's own counting kernels
  int rc = qed_launch_count_live(c, d_live, s);
  if (rc != QED_OK) return rc;
  unsigned long long cnt[qed::kNumCounters];
  long long live[4];
  int bits = 0;
  struct { double t; long long step; } clk = {0.0, 0};
  if (cudaMemcpyAsync(cnt, c->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&clk, c->d_clock, sizeof(clk), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(live, d_live, sizeof(live), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&bits, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return QED_ERR_CUDA;
  if (out->nbins > 0) {
    if (out->spectrum &&
        cudaMemcpyAsync(out->spectrum, c->d_spec, sizeof(double) * out->nbins, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
      return QED_ERR_CUDA;
    if (out->spectrum_energy &&
        cudaMemcpyAsync(out->spectrum_energy, c->d_spec_e, sizeof(double) * out->nbins,
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
      return QED_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return QED_ERR_CUDA;
  for (int k = 0; k < 4; ++k) out->count[k] = live[k];
  out->emissions = (int64_t)cnt[qed::kCntEmissions];
  out->pairs = (int64_t)cnt[qed::kCntPairs];
  out->substeps_lepton = (int64_t)cnt[qed::kCntSubLepton];
  out->substeps_photon = (int64_t)cnt[qed::kCntSubPhoton];
  out->pm_gt1 = (int64_t)cnt[qed::kCntPmGt1];
  out->pp_gt1 = (int64_t)cnt[qed::kCntPpGt1];
  out->capped = (int64_t)cnt[qed::kCntCapped];
  out->absorbed = (int64_t)cnt[qed::kCntAbsorbed];
  out->overflow = (int64_t)cnt[qed::kCntOverflow];
  out->nonfinite = (int64_t)cnt[qed::kCntNonfinite];
  out->photons_created = (int64_t)cnt[qed::kCntPhotonsMade];
  out->pairs_created = (int64_t)cnt[qed::kCntPairsMade];
  out->thinned = (int64_t)cnt[qed::kCntThinned];
  out->schwinger_pairs = (int64_t)cnt[qed::kCntSchwinger];
  out->schwinger_gt1 = (int64_t)cnt[qed::kCntSchwingerGt1];
  out->block_steps = (int64_t)cnt[qed::kCntBlockSteps];
  out->tile_deposits = (int64_t)cnt[qed::kCntTileDeposits];
  out->particle_steps = 0;
  for (int k = 0; k < 4; ++k) {
    out->species_steps[k] = (int64_t)cnt[qed::kCntSpeciesSteps + k];
    out->particle_steps += out->species_steps[k];
  }
  out->kernel_launches = launches;
  out->step = clk.step;
  out->time = clk.t;
  const int st = qed_latch_status(c, bits);
  out->status = st;
  return st;
}

int qed_destroy(qed_ctx *c) {
  if (!c) return QED_OK;
  cudaDeviceSynchronize();
  release(c);
  delete c;
  return QED_OK;
}

}  // extern "C"
