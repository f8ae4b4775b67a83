// mesh.cuh -- the non-uniform (stretched) Cartesian mesh of arXiv:1905.00182, Sec. 2: a mapping
// x(xi) per direction of a computational coordinate xi with unit spacing per cell.  Differences
// are taken in xi and divided by dx/dxi at the node where the derivative is taken; immersed-
// boundary markers and probes keep their four-point support where the spacing is constant (the
// paper keeps the body inside its uniform box) and take the delta with that spacing.  Device
// helpers shared by the stage kernels; a NULL array in the plan means a uniform direction, for
// which every helper returns what the uniform formulas give.
#pragma once

#include <math.h>

#include "ibfsa_internal.h"

namespace ibfsa {
namespace mesh {

// coordinate of node i (-NG <= i < n + NG) along direction a
__device__ __forceinline__ double node(const Plan &p, int a, int i) {
  return p.mx[a] ? p.mx[a][i + NG] : p.lo[a] + ((double)i + 0.5) * p.h[a];
}

// clamp a node index into the stored range -NG .. n+NG-1 (for points whose results are unused)
__device__ __forceinline__ int clamp_node(const Plan &p, int a, int i) {
  return i < -NG ? -NG : (i > p.n[a] + NG - 1 ? p.n[a] + NG - 1 : i);
}

// 1/(dx/dxi) and 1/(12 dx/dxi) at node i in FP32 (uniform: the plan's FP32 1/h, 1/(12 h))
__device__ __forceinline__ float inv32(const Plan &p, int a, int i) {
  return p.minv32[a] ? p.minv32[a][i + NG] : p.inv_h32[a];
}
__device__ __forceinline__ float inv12_32(const Plan &p, int a, int i) {
  return p.minv12_32[a] ? p.minv12_32[a][i + NG] : p.inv_h12_32[a];
}

// Four-point support along a stretched direction a of position x: the first support node j0,
// the position in node units *s = i + (x - x_i)/(dx/dxi)_i with x_i the last node at or left of
// x (the weights are lambda(*s - j) for j = j0 .. j0 + 3), and the local spacing *hl.  The
// support (and one node beyond each side) must lie where the metric is constant (relative
// 1e-12); otherwise, or when x lies outside the nodes, it returns -NG - 4, outside every
// interior, which the callers report as out of bounds.
__device__ __forceinline__ int support_stretched(const Plan &p, int a, double x, double *s_out,
                                                 double *hl) {
  const int n = p.n[a];
  const double *X = p.mx[a], *M = p.mm[a];
  if (!(x >= X[0]) || !(x < X[n + 2 * NG - 1])) return -NG - 4;
  int lo = 0, hi = n + 2 * NG - 2;  // storage indices: the largest k in [lo, hi] with X[k] <= x
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (X[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  const int i = lo - NG;
  const double m = M[lo];
  const double s = (double)i + (x - X[lo]) / m;
  const int j0 = (int)floor(s) - 1;
  for (int r = -1; r < 5; r++) {
    int jj = j0 + r;
    if (jj < -NG || jj > n + NG - 1) return -NG - 4;
    if (fabs(M[jj + NG] - m) > 1e-12 * m) return -NG - 4;
  }
  *s_out = s;
  *hl = m;
  return j0;
}

}  // namespace mesh
}  // namespace ibfsa
