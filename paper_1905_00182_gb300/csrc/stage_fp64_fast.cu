// Fast FP64 stage kernels: fused multiply-add, reciprocals and atomic spreading allowed.
#define IBFSA_STRICT 0
#define IBFSA_MODE_NS fast_ns
#include "stage_fp64.cuh"

namespace ibfsa {
cudaError_t fast_stage(const Plan &p, const StageArgs &s, cudaStream_t st) {
  return fast_ns::stage_impl(p, s, st);
}
cudaError_t fast_wavespeed(const Plan &p, const double *Q, cudaStream_t st) {
  return fast_ns::wavespeed_impl(p, Q, st);
}
cudaError_t fast_probe(const Plan &p, const double *Q, int np, const double *xp, double *out,
                        cudaStream_t st, Prof *pr) {
  return fast_ns::probe_impl(p, Q, np, xp, out, st, pr);
}
}  // namespace ibfsa
