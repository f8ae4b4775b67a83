// Strict FP64 stage kernels: compiled with --fmad=false so that every multiply and add is
// rounded on its own, in the order the formulas are written (bit-reproducible evaluation).
#define IBFSA_STRICT 1
#define IBFSA_MODE_NS strict_ns
#include "stage_fp64.cuh"

namespace ibfsa {
cudaError_t strict_stage(const Plan &p, const StageArgs &s, cudaStream_t st) {
  return strict_ns::stage_impl(p, s, st);
}
cudaError_t strict_wavespeed(const Plan &p, const double *Q, cudaStream_t st) {
  return strict_ns::wavespeed_impl(p, Q, st);
}
cudaError_t strict_probe(const Plan &p, const double *Q, int np, const double *xp, double *out,
                         cudaStream_t st, Prof *pr) {
  return strict_ns::probe_impl(p, Q, np, xp, out, st, pr);
}
}  // namespace ibfsa
