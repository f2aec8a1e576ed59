// batch.cu -- a13: n_crit autotuner for batched ensembles.
//
// The forest solve (fmm_solve_batch) is timed with CUDA events on the
// context's stream for every candidate leaf size; the fastest is returned.
// The candidates change only the leaf size (a leaf holds at most n_crit
// bodies, Sec. 2); every candidate gives a valid solve of the same method.
#include "internal.cuh"

using namespace amfmm;

extern "C" int fmm_autotune_ncrit(fmm_ctx *c, const double *x, const double *y, const double *z,
                                  const double *m, const int64_t *offsets, int nsys, const int *candidates,
                                  int ncand, int reps, double *ax, double *ay, double *az, int *best,
                                  float *ms_out) {
  if (!c || !candidates || ncand < 1 || reps < 1 || !best) return FMM_EINVAL;
  for (int k = 0; k < ncand; ++k)
    if (candidates[k] < 1) return set_error(c, FMM_EINVAL, "candidate n_crit must be >= 1");
  const fmm_opts saved = c->opts;
  cudaEvent_t e0, e1;
  AMFMM_CUDA(c, cudaEventCreate(&e0));
  AMFMM_CUDA(c, cudaEventCreate(&e1));
  float best_ms = 0.f;
  int rc = FMM_OK;
  *best = candidates[0];
  for (int k = 0; k < ncand && rc == FMM_OK; ++k) {
    c->opts.n_crit = candidates[k];
    rc = fmm_solve_batch(c, x, y, z, m, offsets, nsys, ax, ay, az);  // warm-up and buffer growth
    float tot = 0.f;
    for (int r = 0; r < reps && rc == FMM_OK; ++r) {
      cudaError_t ce = cudaEventRecord(e0, c->stream);
      if (ce == cudaSuccess) rc = fmm_solve_batch(c, x, y, z, m, offsets, nsys, ax, ay, az);
      if (rc != FMM_OK) break;
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, c->stream);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float t = 0.f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
      // a repetition that cannot be timed fails the call: counting it as
      // zero would make the candidate look fast
      if (ce != cudaSuccess) rc = set_error(c, FMM_ECUDA, "timing candidate n_crit %d: %s", candidates[k],
                                            cudaGetErrorString(ce));
      tot += t;
    }
    const float ms = tot / reps;
    if (ms_out) ms_out[k] = ms;
    if (rc == FMM_OK && (k == 0 || ms < best_ms)) {
      best_ms = ms;
      *best = candidates[k];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->opts = saved;
  c->stage = kNone;
  return rc;
}
