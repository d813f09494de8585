// The particle step: field gather, Boris push, adaptive event generator with
// photon emission and pair creation, append of products, Esirkepov deposit.
//
// Three launches per step.  Pass 0 advances every particle alive at the
// start of the step by dt, with the fields taken once at its start position
// (Sec. IV.H: no re-interpolation inside the step): one kernel for photons
// (most of the particles in a cascade, and the lightest code path) and one
// for electrons, positrons and ions, each register-allocated for its own
// path.  Products created in sub-interval s of an N-interval loop carry the
// time left, (N-1-s) h, and the parent's frozen fields into a product buffer;
// a persistent cooperative kernel advances them for that time in passes
// 1, 2, ... separated by a bounded grid barrier, until no products are left.
// Finished products are appended to their species stores.  Dead particles
// keep their slot (cell = -1) until the next compaction.
#include "step_kernels.cuh"

namespace {
// chi* of the pair skip, and eps* = chi*/H_max: photons below eps* cannot
// pair anywhere in an analytic field whose effective field is bounded by
// H_max (|E| + |B|); zero on the grid, where no bound is known.
template <typename R>
__global__ void k_chi_star(const R *tab, double kappa, int mode, qed_grid_desc g, double ens_hmax, double *chi,
                           double *eps) {
  const double cs = qed::photon_chi_star(tab, kappa);
  *chi = cs;
  double hmax = 0.0;
  if (mode == qed::kFieldUniform)
    hmax = sqrt(g.fp[0] * g.fp[0] + g.fp[1] * g.fp[1] + g.fp[2] * g.fp[2]) +
           sqrt(g.fp[3] * g.fp[3] + g.fp[4] * g.fp[4] + g.fp[5] * g.fp[5]);
  else if (mode == qed::kFieldRotatingE || mode == qed::kFieldStandingWave)
    hmax = fabs(g.fp[0]);
  else if (mode == qed::kFieldGaussianLP)
    hmax = 2.0 * fabs(g.fp[0]);
  else if (mode == qed::kFieldEnsemble)
    hmax = ens_hmax;
  *eps = hmax > 0.0 ? 0.999 * cs / hmax : 0.0;
}

// Self-test of the bounded grid barrier of the product passes: every block
// of a cooperative launch but `absent` meets at the barrier; `passed` counts
// the blocks that got through it.
__global__ void k_barrier_check(unsigned *bar, int *status, int absent, long long limit, int *passed) {
  if ((int)blockIdx.x == absent) return;
  const bool ok = qed::grid_barrier(bar, status, limit);
  if (threadIdx.x == 0 && ok) atomicAdd(passed, 1);
}

}  // namespace

extern "C" int qed_selftest_barrier(qed_ctx *c, int32_t absent_block, int64_t spin_limit, void *stream) {
  if (!c || spin_limit < 1 || absent_block >= c->num_sms) return QED_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // spare words of the context: barrier [2..3], status [1], pass count [2]
  unsigned *bar = c->d_barrier + 2;
  int *status = c->d_status + 1, *passed = c->d_status + 2;
  if (cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(status, 0, 2 * sizeof(int), s) != cudaSuccess)
    return QED_ERR_CUDA;
  int absent = absent_block < 0 ? -1 : absent_block;
  long long limit = spin_limit;
  void *args[] = {(void *)&bar, (void *)&status, (void *)&absent, (void *)&limit, (void *)&passed};
  c->launches += 1;
  // one block of one warp per SM: every block is co-resident
  if (cudaLaunchCooperativeKernel((const void *)k_barrier_check, dim3(c->num_sms), dim3(32), args, 0, s) !=
      cudaSuccess)
    return QED_ERR_CUDA;
  int out[2] = {0, 0};
  if (cudaMemcpyAsync(out, status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return QED_ERR_CUDA;
  const int expect = absent < 0 ? c->num_sms : 0;
  if (out[0] & qed::kStTimeout) return out[1] == 0 ? QED_ERR_TIMEOUT : QED_ERR_CUDA;
  return out[1] == expect ? QED_OK : QED_ERR_CUDA;
}

int qed_step_kernel_blocks(qed_ctx *c) {
  if (c->ext) return qed_step_kernel_blocks_ext(c);
  return c->prec == 64 ? qed::step_blocks<double, false>(c) : qed::step_blocks<float, false>(c);
}

int qed_step_kernel_max_blocks(qed_ctx *c, int *photon, int *massive) {
  if (c->ext) return qed_step_kernel_max_blocks_ext(c, photon, massive);
  return c->prec == 64 ? qed::max_blocks<double, false>(photon, massive)
                       : qed::max_blocks<float, false>(photon, massive);
}

// Threshold of the photon pair skip for this context's kappa and table.
int qed_launch_chi_star(qed_ctx *c, cudaStream_t s) {
  c->launches += 1;
  if (c->prec == 64)
    k_chi_star<double><<<1, 1, 0, s>>>((const double *)c->d_tables, c->par.kappa, c->grid.field_mode, c->grid,
                                       c->ens_hmax, c->d_chi_star, c->d_eps_star);
  else
    k_chi_star<float><<<1, 1, 0, s>>>((const float *)c->d_tables, c->par.kappa, c->grid.field_mode, c->grid,
                                      c->ens_hmax, c->d_chi_star, c->d_eps_star);
  return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}

int qed_launch_step(qed_ctx *c, const qed_fields *f, double dt, cudaStream_t s) {
  if (c->ext) return qed_launch_step_ext(c, f, dt, s);
  return c->prec == 64 ? qed::launch<double, false>(c, f, dt, s) : qed::launch<float, false>(c, f, dt, s);
}

size_t qed_step_const_bytes() { return sizeof(qed::StepConst); }
size_t qed_clock_bytes() { return sizeof(qed::Clock); }

size_t qed_pend_bytes(int prec) {
  return prec == 64 ? sizeof(qed::Pend<double>) : sizeof(qed::Pend<float>);
}
