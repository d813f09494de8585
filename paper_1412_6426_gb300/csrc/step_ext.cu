// The particle step with independent ensembles or the generator factors of
// Sec. VI (the EXT variants of the kernels in step_kernels.cuh).
#include "step_kernels.cuh"

int qed_launch_step_ext(qed_ctx *c, const qed_fields *f, double dt, cudaStream_t s) {
  return c->prec == 64 ? qed::launch<double, true>(c, f, dt, s) : qed::launch<float, true>(c, f, dt, s);
}

int qed_step_kernel_blocks_ext(qed_ctx *c) {
  return c->prec == 64 ? qed::step_blocks<double, true>(c) : qed::step_blocks<float, true>(c);
}

int qed_step_kernel_max_blocks_ext(qed_ctx *c, int *photon, int *massive) {
  return c->prec == 64 ? qed::max_blocks<double, true>(photon, massive)
                       : qed::max_blocks<float, true>(photon, massive);
}
