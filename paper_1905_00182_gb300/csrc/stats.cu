// stats.cu -- time statistics of probe signals.
//
// Sec. 3.2 defines the fluctuating pressure about its time mean, dp~ = dp - mean_t(dp), and
// Sec. 3.3 and 4 plot its root mean square on rings of probes.  The accumulator keeps, per
// probe, the sample count, the running mean and the running sum of squared deviations
// (Welford's update), which stays accurate when the mean is much larger than the fluctuation.
// Every operation is a separately rounded IEEE double operation (no fused multiply-add), in a
// fixed order.
#include <cuda_runtime.h>

#include "ibfsa_internal.h"

namespace ibfsa {
namespace {

__global__ void k_probe_fold(int np, const double *__restrict__ dp, double *__restrict__ acc) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  double n = __dadd_rn(acc[k], 1.0);
  double m = acc[np + k];
  double x = dp[k];
  double d = __dsub_rn(x, m);
  m = __dadd_rn(m, __ddiv_rn(d, n));
  double m2 = __dadd_rn(acc[2 * np + k], __dmul_rn(d, __dsub_rn(x, m)));
  acc[k] = n;
  acc[np + k] = m;
  acc[2 * np + k] = m2;
}

__global__ void k_probe_moments(int np, const double *__restrict__ acc, double *__restrict__ mean,
                                double *__restrict__ rms) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  double n = acc[k];
  bool any = n > 0.0;
  mean[k] = any ? acc[np + k] : 0.0;
  rms[k] = any ? __dsqrt_rn(__ddiv_rn(acc[2 * np + k], n)) : 0.0;
}

}  // namespace

cudaError_t probe_fold(int np, const double *dp, double *acc, cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  k_probe_fold<<<(np + 127) / 128, 128, 0, st>>>(np, dp, acc);
  return cudaGetLastError();
}

cudaError_t probe_moments(int np, const double *acc, double *mean, double *rms, cudaStream_t st) {
  if (np <= 0) return cudaSuccess;
  k_probe_moments<<<(np + 127) / 128, 128, 0, st>>>(np, acc, mean, rms);
  return cudaGetLastError();
}

}  // namespace ibfsa
