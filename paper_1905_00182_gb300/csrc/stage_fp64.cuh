// stage_fp64.cuh -- FP64 kernels of one Runge-Kutta stage of the IB-WENO/TENO method
// (arXiv:1905.00182, Sec. 2).  Included twice: once with IBFSA_STRICT = 1 and --fmad=false
// (every operation rounded separately, in the order the formulas are written below, divisions
// kept, spreading summed in marker order), once with IBFSA_STRICT = 0 (fused multiply-add,
// reciprocals, atomic spreading).
//
// Per stage:  pad (ghosts + primitives + split speeds)  ->  IB interpolation and penalty force
//   (Eq. 7-8)  ->  convective flux differences x, y, z  ->  viscous fluxes and their divergence
//   (Eq. 2-5)  ->  IB spreading (Eq. 9)  ->  finish (sponge, IB source, RK combination).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ibfsa_internal.h"
#include "mesh.cuh"

#ifndef IBFSA_STRICT
#error "define IBFSA_STRICT to 0 or 1"
#endif

namespace ibfsa {
namespace IBFSA_MODE_NS {

constexpr bool STRICT = IBFSA_STRICT != 0;
constexpr int THREADS = 256;

// ------------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double divide(double x, double d, double inv_d) {
  if constexpr (STRICT) return x / d;
  else return x * inv_d;
}

// ghost rule of one direction: interior index, or -1 for a free-stream ghost
__device__ __forceinline__ int map_index(int i, int n, int rlo, int rhi) {
  if (i < 0) {
    if (rlo == IBFSA_BC_ZERO_GRAD || rlo == IBFSA_BC_CHARACTERISTIC) return 0;
    if (rlo == IBFSA_BC_PERIODIC) return n + i;
    return -1;
  }
  if (i >= n) {
    if (rhi == IBFSA_BC_ZERO_GRAD || rhi == IBFSA_BC_CHARACTERISTIC) return n - 1;
    if (rhi == IBFSA_BC_PERIODIC) return i - n;
    return -1;
  }
  return i;
}

// the boundary cell of a characteristic face along a (its normal term comes from k_char_face)
__device__ __forceinline__ bool char_cell(const Plan &p, int a, int i) {
  return (i == 0 && p.bc[a][0] == IBFSA_BC_CHARACTERISTIC) ||
         (i == p.n[a] - 1 && p.bc[a][1] == IBFSA_BC_CHARACTERISTIC);
}

__device__ __forceinline__ long long pad_index(const Plan &p, int i, int j, int k) {
  return ((long long)(k + p.g[2]) * p.P[1] + (j + p.g[1])) * (long long)p.P[0] + (i + p.g[0]);
}

__device__ __forceinline__ long long int_index(const Plan &p, int i, int j, int k) {
  return ((long long)k * p.n[1] + j) * (long long)p.n[0] + i;
}

__device__ __forceinline__ double load_alpha(const Plan &p, int a) {
  return __longlong_as_double((long long)p.alpha_bits[a]);
}

// Peskin's four-point kernel, Eq. 11
__device__ __forceinline__ double peskin(double r) {
  double a = fabs(r);
  if (a < 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
  if (a < 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
  return 0.0;
}

// first of the four support nodes of position x along direction a, and their weights
__device__ __forceinline__ int support(const Plan &p, int a, double x, double w[4]) {
  double s = divide(x - p.lo[a], p.h[a], p.inv_h[a]) - 0.5;
  int j0 = (int)floor(s) - 1;
#pragma unroll
  for (int r = 0; r < 4; r++) w[r] = peskin(s - (double)(j0 + r));
  return j0;
}

// ------------------------------------------------------------------------------------------
// fifth-order reconstruction at face i+1/2 from (f_{i-2}, ..., f_{i+2})
// ------------------------------------------------------------------------------------------
struct Cands {
  double q0, q1, q2, b0, b1, b2;
};

__device__ __forceinline__ Cands candidates(double a, double b, double c, double d, double e) {
  Cands r;
  // third-order candidates on {i-2..i}, {i-1..i+1}, {i..i+2}
  if constexpr (STRICT) {
    r.q0 = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
    r.q1 = (-b + 5.0 * c + 2.0 * d) / 6.0;
    r.q2 = (2.0 * c + 5.0 * d - e) / 6.0;
  } else {
    const double s6 = 1.0 / 6.0;
    r.q0 = (2.0 * a - 7.0 * b + 11.0 * c) * s6;
    r.q1 = (-b + 5.0 * c + 2.0 * d) * s6;
    r.q2 = (2.0 * c + 5.0 * d - e) * s6;
  }
  // Jiang-Shu smoothness indicators
  double t;
  t = a - 2.0 * b + c;       r.b0 = 13.0 / 12.0 * t * t;
  t = a - 4.0 * b + 3.0 * c; r.b0 += 0.25 * t * t;
  t = b - 2.0 * c + d;       r.b1 = 13.0 / 12.0 * t * t;
  t = b - d;                 r.b1 += 0.25 * t * t;
  t = c - 2.0 * d + e;       r.b2 = 13.0 / 12.0 * t * t;
  t = 3.0 * c - 4.0 * d + e; r.b2 += 0.25 * t * t;
  return r;
}

// WENO5-JS: alpha_k = d_k / (1e-6 + beta_k)^2, omega = alpha / sum alpha, d = (0.1, 0.6, 0.3)
__device__ __forceinline__ double weno5js(double a, double b, double c, double d, double e) {
  Cands k = candidates(a, b, c, d, e);
  const double eps = 1e-6;
  if constexpr (STRICT) {
    double al0 = 0.1 / ((eps + k.b0) * (eps + k.b0));
    double al1 = 0.6 / ((eps + k.b1) * (eps + k.b1));
    double al2 = 0.3 / ((eps + k.b2) * (eps + k.b2));
    double s = al0 + al1 + al2;
    return (al0 / s) * k.q0 + (al1 / s) * k.q1 + (al2 / s) * k.q2;
  } else {
    // common denominator: alpha_k proportional to d_k prod_{j != k} (eps + beta_j)^2
    double s0 = (eps + k.b0) * (eps + k.b0);
    double s1 = (eps + k.b1) * (eps + k.b1);
    double s2 = (eps + k.b2) * (eps + k.b2);
    double al0 = 0.1 * (s1 * s2), al1 = 0.6 * (s0 * s2), al2 = 0.3 * (s0 * s1);
    return (al0 * k.q0 + al1 * k.q1 + al2 * k.q2) / (al0 + al1 + al2);
  }
}

// TENO5: gamma_k = (1 + tau5/(beta_k + 1e-40))^6, tau5 = |beta_0 - beta_2|; stencil k kept when
// gamma_k / sum gamma >= 1e-5; omega = normalised linear weights of the kept stencils
__device__ __forceinline__ double teno5(const Plan &p, double a, double b, double c, double d,
                                        double e) {
  Cands k = candidates(a, b, c, d, e);
  const double eps = 1e-40, CT = 1e-5;
  double tau5 = fabs(k.b0 - k.b2);
  double g0, g1, g2;
  int mask;
  if constexpr (STRICT) {
    double x, x2;
    x = 1.0 + tau5 / (k.b0 + eps); x2 = x * x; g0 = x2 * x2 * x2;
    x = 1.0 + tau5 / (k.b1 + eps); x2 = x * x; g1 = x2 * x2 * x2;
    x = 1.0 + tau5 / (k.b2 + eps); x2 = x * x; g2 = x2 * x2 * x2;
    double s = g0 + g1 + g2;
    mask = ((g0 / s) >= CT ? 1 : 0) | ((g1 / s) >= CT ? 2 : 0) | ((g2 / s) >= CT ? 4 : 0);
  } else {
    double e0 = k.b0 + eps, e1 = k.b1 + eps, e2 = k.b2 + eps;
    double r = tau5 / (e0 * e1 * e2);
    double x, x2;
    x = 1.0 + r * (e1 * e2); x2 = x * x; g0 = x2 * x2 * x2;
    x = 1.0 + r * (e0 * e2); x2 = x * x; g1 = x2 * x2 * x2;
    x = 1.0 + r * (e0 * e1); x2 = x * x; g2 = x2 * x2 * x2;
    double th = CT * (g0 + g1 + g2);
    mask = (g0 >= th ? 1 : 0) | (g1 >= th ? 2 : 0) | (g2 >= th ? 4 : 0);
  }
  const double *w = p.teno_w[mask];
  return w[0] * k.q0 + w[1] * k.q1 + w[2] * k.q2;
}

// Fast arithmetic only: TENO5 keeps every stencil when tau5 <= 4 (min beta + eps) -- each
// gamma_k lies in [1, 5^6], so chi_k >= 1/(3 5^6) = 2.1e-5 > C_T -- and the reconstruction is
// the optimal linear combination (2a - 13b + 47c + 27d - 3e)/60 (the strict form evaluates
// every step as written).  Only this sufficient test is taken in FP32 (the FP64 pipe is the
// bound; a conversion issues at the FP64 rate): the four first differences in FP64, rounded to
// FP32, give t and u of every indicator (t0 = d2 - d1, u0 = 3 d2 - d1, t1 = d3 - d2,
// u1 = -(d2 + d3), t2 = d4 - d3, u2 = d4 - 3 d3), taken times 4, (13/3) t^2 + u^2, against
// 4 min + 1.6e-29.  Each indicator is a positive definite form of its two differences, so its
// relative error stays a few 1e-7 (where t or u cancels, the other term dominates) -- far
// inside the test's factor-2 margin in chi_k (2.1e-5 against C_T = 1e-5): a stencil the test
// keeps is one TENO5 keeps; where the test fails, the full FP64 TENO5 decides.  Differences
// below FP32's range flush to zero and pass the test; their stencils vary by less than 1e-17
// of the flux, whatever TENO5 would cut.
__device__ __forceinline__ double teno5_fast(const Plan &p, double a, double b, double c,
                                             double d, double e) {
  const double e1 = b - a, e2 = c - b, e3 = d - c, e4 = e - d;
  const float d1 = (float)e1, d2 = (float)e2, d3 = (float)e3, d4 = (float)e4;
  const float t0 = d2 - d1, u0 = fmaf(3.f, d2, -d1);
  const float t1 = d3 - d2, u1 = d2 + d3;
  const float t2 = d4 - d3, u2 = fmaf(-3.f, d3, d4);
  const float k13 = 13.f / 3.f;
  const float b0 = fmaf(k13 * t0, t0, u0 * u0);
  const float b1 = fmaf(k13 * t1, t1, u1 * u1);
  const float b2 = fmaf(k13 * t2, t2, u2 * u2);
  // the linear combination as c plus its differences, (-2 d1 + 11 d2 + 24 d3 - 3 d4)/60: four
  // fused multiply-adds, and a constant stencil gives c exactly
  if (fabsf(b0 - b2) <= fmaf(4.f, fminf(b0, fminf(b1, b2)), 1.6e-29f))
    return fma(-3.0 / 60.0, e4, fma(24.0 / 60.0, e3, fma(11.0 / 60.0, e2, fma(-2.0 / 60.0, e1, c))));
  return teno5(p, a, b, c, d, e);
}

template <int SCHEME>
__device__ __forceinline__ double recon(const Plan &p, double a, double b, double c, double d,
                                        double e) {
  if constexpr (SCHEME == IBFSA_TENO5) {
    if constexpr (STRICT) return teno5(p, a, b, c, d, e);
    else return teno5_fast(p, a, b, c, d, e);
  } else {
    return weno5js(a, b, c, d, e);
  }
}

// ------------------------------------------------------------------------------------------
// pad: ghost fill by index mapping, primitives on the padded grid, split speeds
// ------------------------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(THREADS) k_pad(Plan p, const double *__restrict__ Q) {
  constexpr int NV = DIM + 2;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double wmax[3] = {0.0, 0.0, 0.0};
  double c2 = 0.0, ua[3] = {0.0, 0.0, 0.0};  // fast form: c^2 and |u_a| of an interior cell
  bool have = false;
  if (t < p.NP) {
    int ix = (int)(t % p.P[0]);
    long long r = t / p.P[0];
    int iy = (int)(r % p.P[1]);
    int iz = (int)(r / p.P[1]);
    int I[3] = {ix - p.g[0], iy - p.g[1], iz - p.g[2]};
    bool free_ghost = false, interior = true;
    int S[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      if (a < DIM) {
        S[a] = map_index(I[a], p.n[a], p.bc[a][0], p.bc[a][1]);
        if (S[a] < 0) free_ghost = true;
        if (I[a] < 0 || I[a] >= p.n[a]) interior = false;
      } else {
        S[a] = 0;
      }
    }
    double q[NV];
    if (free_ghost) {
#pragma unroll
      for (int c = 0; c < NV; c++) q[c] = p.qinf[c];
    } else {
      long long o = int_index(p, S[0], S[1], S[2]);
#pragma unroll
      for (int c = 0; c < NV; c++) q[c] = Q[c * p.N + o];
    }
#pragma unroll
    for (int c = 0; c < NV; c++) p.Qp[c * p.NP + t] = q[c];
    double rho = q[0];
    double ke = 0.0, u[DIM];
    // strict: each division as the oracle writes it; fast: one reciprocal of rho
    const double inv_rho = STRICT ? 0.0 : 1.0 / rho;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      u[a] = STRICT ? q[1 + a] / rho : q[1 + a] * inv_rho;
      ke += q[1 + a] * u[a];
      p.Wp[a * p.NP + t] = u[a];
    }
    double pr = p.gm1 * (q[NV - 1] - 0.5 * ke);
    p.Wp[DIM * p.NP + t] = pr;
    if (interior) {
      if constexpr (STRICT) {
        const double c = sqrt(p.gamma * pr / rho);
#pragma unroll
        for (int a = 0; a < DIM; a++) wmax[a] = fabs(u[a]) + c;
      } else {
        c2 = p.gamma * pr * inv_rho;
#pragma unroll
        for (int a = 0; a < DIM; a++) ua[a] = fabs(u[a]);
        have = true;
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if constexpr (!STRICT) {
    // The block's maxima in FP32 first: the FP64 sound speed is taken only where |u| + c in
    // FP32 lies within 2e-6 of the block's FP32 maximum (their relative errors, and that of
    // the threshold, stay below 3e-7, so the cell of the exact maximum is among them); the
    // other cells give 0 -- the same FP64 maxima for a fraction of the square roots.
    __shared__ float red32[3][THREADS / 32];
    const float c32 = have ? sqrtf((float)c2) : 0.f;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      float v = have ? (float)ua[a] + c32 : 0.f;
      for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (lane == 0) red32[a][wid] = v;
    }
    __syncthreads();
    float m32[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < DIM; a++)
      for (int w = 0; w < THREADS / 32; w++) m32[a] = fmaxf(m32[a], red32[a][w]);
    bool near = false;
#pragma unroll
    for (int a = 0; a < DIM; a++)
      near |= have && !((float)ua[a] + c32 < m32[a] * (1.f - 2e-6f));  // NaN counts as near
    if (near) {
      const double c = sqrt(c2);
#pragma unroll
      for (int a = 0; a < DIM; a++) wmax[a] = ua[a] + c;
    }
  }
  // block max of the (non-negative) speeds on their bits (the order of non-negative doubles is
  // that of their bit patterns; a NaN's pattern exceeds every finite one), then one atomic per
  // block
  __shared__ unsigned long long red[3][THREADS / 32];
#pragma unroll
  for (int a = 0; a < DIM; a++) {
    unsigned long long v = (unsigned long long)__double_as_longlong(wmax[a]);
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    if (lane == 0) red[a][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < DIM) {
    unsigned long long b = 0;
    for (int w = 0; w < THREADS / 32; w++) b = red[threadIdx.x][w] > b ? red[threadIdx.x][w] : b;
    const double v = __longlong_as_double((long long)b);
    if (!(v <= 1e300)) atomicOr(p.status, IBFSA_STATUS_NONFINITE);
    else atomicMax(&p.alpha_bits[threadIdx.x], b);
  }
}

// ------------------------------------------------------------------------------------------
// convective term along direction A: split fluxes of a tile of lines staged in shared memory,
// one face per thread per pass, conservative difference into L
// ------------------------------------------------------------------------------------------
// ------------------------------------------------------------------------------------------
// characteristic-wise option: eigenvectors of the Euler flux Jacobian along A at the Roe
// average of the face's two cells (sqrt(rho)-weighted velocity and total enthalpy).  Right
// eigenvectors are the columns of R, left ones the rows of Lv, in the order u-c, entropy,
// shears (transverse directions in increasing order), u+c.  Written operation by operation in
// the order of the formulas, so that the strict form is reproducible.
// ------------------------------------------------------------------------------------------
template <int DIM, int A>
__device__ __forceinline__ void roe_eigen(const Plan &p, const double *Ql, const double *Qr,
                                          double R[DIM + 2][DIM + 2],
                                          double Lv[DIM + 2][DIM + 2]) {
  constexpr int NV = DIM + 2;
  const double gm1 = p.gm1;
  double sl = sqrt(Ql[0]), sr = sqrt(Qr[0]);
  double u[DIM], kel = 0.0, ker = 0.0;
#pragma unroll
  for (int b = 0; b < DIM; b++) {
    double ul = Ql[1 + b] / Ql[0], ur = Qr[1 + b] / Qr[0];
    u[b] = (sl * ul + sr * ur) / (sl + sr);
    kel = kel + Ql[1 + b] * ul;
    ker = ker + Qr[1 + b] * ur;
  }
  double pl = gm1 * (Ql[NV - 1] - 0.5 * kel);
  double pr = gm1 * (Qr[NV - 1] - 0.5 * ker);
  double Hl = (Ql[NV - 1] + pl) / Ql[0], Hr = (Qr[NV - 1] + pr) / Qr[0];
  double H = (sl * Hl + sr * Hr) / (sl + sr);
  double q2 = 0.0;
#pragma unroll
  for (int b = 0; b < DIM; b++) q2 = q2 + u[b] * u[b];
  double c2 = gm1 * (H - 0.5 * q2);
  double c = sqrt(c2);
  double b1 = gm1 / c2, b2 = 0.5 * q2 * b1;
  double ua = u[A];
#pragma unroll
  for (int i = 0; i < NV; i++)
#pragma unroll
    for (int j = 0; j < NV; j++) {
      R[i][j] = 0.0;
      Lv[i][j] = 0.0;
    }
  constexpr int km = 0, ke = 1, kp = NV - 1;
  R[0][km] = 1.0;
  R[0][ke] = 1.0;
  R[0][kp] = 1.0;
#pragma unroll
  for (int b = 0; b < DIM; b++) {
    R[1 + b][km] = u[b] - (b == A ? c : 0.0);
    R[1 + b][ke] = u[b];
    R[1 + b][kp] = u[b] + (b == A ? c : 0.0);
  }
  R[NV - 1][km] = H - ua * c;
  R[NV - 1][ke] = 0.5 * q2;
  R[NV - 1][kp] = H + ua * c;
  Lv[km][0] = 0.5 * (b2 + ua / c);
  Lv[kp][0] = 0.5 * (b2 - ua / c);
  Lv[ke][0] = 1.0 - b2;
#pragma unroll
  for (int b = 0; b < DIM; b++) {
    Lv[km][1 + b] = 0.5 * (-b1 * u[b] - (b == A ? 1.0 / c : 0.0));
    Lv[kp][1 + b] = 0.5 * (-b1 * u[b] + (b == A ? 1.0 / c : 0.0));
    Lv[ke][1 + b] = b1 * u[b];
  }
  Lv[km][NV - 1] = 0.5 * b1;
  Lv[kp][NV - 1] = 0.5 * b1;
  Lv[ke][NV - 1] = -b1;
  int t = 0;
#pragma unroll
  for (int b = 0; b < DIM; b++) {
    if (b == A) continue;
    R[1 + b][2 + t] = 1.0;
    R[NV - 1][2 + t] = u[b];
    Lv[2 + t][0] = -u[b];
    Lv[2 + t][1 + b] = 1.0;
    t++;
  }
}

template <int A>
struct ConvTile {
  // A == 0: 4 lines (y/z) of 63 cells; otherwise 32 lines (consecutive x) of 15 cells
  static constexpr int ROWS = A == 0 ? 4 : 32;
  static constexpr int SEG = A == 0 ? 63 : 15;
  static constexpr int LEN = SEG + 6;          // cells staged per line
  static constexpr int FACES = SEG + 1;        // faces per line
  static constexpr int PASSES = (ROWS * FACES + THREADS - 1) / THREADS;
};

template <int DIM, int A>
__host__ __device__ constexpr size_t conv_smem_bytes() {
  return sizeof(double) * 2 * (DIM + 2) * ConvTile<A>::ROWS * ConvTile<A>::LEN;
}

template <int DIM, int A, int SCHEME, bool CHAR>
__global__ void __launch_bounds__(THREADS) k_conv(Plan p, int first) {
  constexpr int NV = DIM + 2;
  // TENO5's weights depend on ratios of indicators only (its floors aside), so its fast
  // component-wise form can reconstruct F +- alpha q and halve once at the face; WENO5-JS's
  // eps = 1e-6 is not scale-free
  constexpr bool FOLD = !STRICT && !CHAR && SCHEME == IBFSA_TENO5;
  using T = ConvTile<A>;
  extern __shared__ double sm[];
  double *sfp = sm;                              // [NV][ROWS][LEN]
  double *sfm = sm + NV * T::ROWS * T::LEN;      // [NV][ROWS][LEN]
  const double alpha = load_alpha(p, A);

  // tile origin
  int seg0, line0, other;
  if constexpr (A == 0) {
    seg0 = blockIdx.x * T::SEG;
    line0 = blockIdx.y * T::ROWS;   // y of the first line
    other = blockIdx.z;             // z
  } else {
    int nseg = (p.n[A] + T::SEG - 1) / T::SEG;
    seg0 = (blockIdx.x % nseg) * T::SEG;
    line0 = (blockIdx.x / nseg) * T::ROWS;  // x of the first line
    other = blockIdx.y;                     // z for A = 1, y for A = 2
  }
  auto cell_of = [&](int row, int l, int I[3]) -> bool {
    // row-th line of the tile, position l along A (tile-relative, may be negative)
    if constexpr (A == 0) {
      int y = line0 + row;
      if (y >= p.n[1]) return false;
      I[0] = seg0 + l;
      I[1] = y;
      I[2] = other;
    } else {
      int x = line0 + row;
      if (x >= p.n[0]) return false;
      I[0] = x;
      I[A] = seg0 + l;
      I[A == 1 ? 2 : 1] = other;
    }
    return true;
  };

  // 1. split fluxes f+- = (F_A(Q) +- alpha Q)/2 of the staged cells
  for (int e = threadIdx.x; e < T::ROWS * T::LEN; e += THREADS) {
    int row, l;
    if constexpr (A == 0) { row = e / T::LEN; l = e % T::LEN; }
    else { row = e % T::ROWS; l = e / T::ROWS; }
    int I[3];
    bool ok = cell_of(row, l - 3, I);
    if (ok && I[A] > p.n[A] + 2) ok = false;
    if (ok) {
      long long s = pad_index(p, I[0], I[1], I[2]);
      double ua = p.Wp[A * p.NP + s];
      double pr = p.Wp[DIM * p.NP + s];
#pragma unroll
      for (int c = 0; c < NV; c++) {
        double q = p.Qp[c * p.NP + s];
        double F;
        if (c == 0) F = p.Qp[(1 + A) * p.NP + s];
        else if (c == NV - 1) F = (q + pr) * ua;
        else {
          F = q * ua;
          if (c - 1 == A) F += pr;
        }
        // fast component-wise TENO5: F +- alpha q, the halves taken once at the face
        sfp[(c * T::ROWS + row) * T::LEN + l] = FOLD ? fma(alpha, q, F) : 0.5 * (F + alpha * q);
        sfm[(c * T::ROWS + row) * T::LEN + l] = FOLD ? fma(-alpha, q, F) : 0.5 * (F - alpha * q);
      }
    } else {
#pragma unroll
      for (int c = 0; c < NV; c++) {
        sfp[(c * T::ROWS + row) * T::LEN + l] = 0.0;
        sfm[(c * T::ROWS + row) * T::LEN + l] = 0.0;
      }
    }
  }
  __syncthreads();

  // 2. faces m+1/2 for m = seg0-1 .. seg0+SEG-1 (tile-relative face index fi = m - seg0 + 1)
  double Fh[T::PASSES][NV];
#pragma unroll
  for (int ps = 0; ps < T::PASSES; ps++) {
    int e = threadIdx.x + ps * THREADS;
    if (e < T::ROWS * T::FACES) {
      int row, fi;
      if constexpr (A == 0) { row = e / T::FACES; fi = e % T::FACES; }
      else { row = e % T::ROWS; fi = e / T::ROWS; }
      // staged index of cell m is (m - seg0) + 3 = fi + 2
      int b = fi + 2;
      if constexpr (CHAR) {
        // characteristic fields of the stencil at the Roe average of cells m and m+1 (only
        // the faces -1/2 .. n-1/2 are used)
        int I[3];
        bool ok = cell_of(row, fi - 1, I) && I[A] <= p.n[A] - 1;
        if (ok) {
          long long sl = pad_index(p, I[0], I[1], I[2]);
          I[A] += 1;
          long long sr = pad_index(p, I[0], I[1], I[2]);
          double Ql[NV], Qr[NV];
#pragma unroll
          for (int c = 0; c < NV; c++) {
            Ql[c] = p.Qp[c * p.NP + sl];
            Qr[c] = p.Qp[c * p.NP + sr];
          }
          double R[NV][NV], Lv[NV][NV];
          roe_eigen<DIM, A>(p, Ql, Qr, R, Lv);
          double hk[NV];
#pragma unroll
          for (int k = 0; k < NV; k++) {
            double vp[5], vm[5];
#pragma unroll
            for (int r = 0; r < 5; r++) {
              double sp = 0.0, sn = 0.0;
#pragma unroll
              for (int c = 0; c < NV; c++) {
                const double *fp = sfp + (c * T::ROWS + row) * T::LEN;
                const double *fm = sfm + (c * T::ROWS + row) * T::LEN;
                sp = sp + Lv[k][c] * fp[b - 2 + r];
                sn = sn + Lv[k][c] * fm[b + 3 - r];
              }
              vp[r] = sp;
              vm[r] = sn;
            }
            hk[k] = recon<SCHEME>(p, vp[0], vp[1], vp[2], vp[3], vp[4]) +
                    recon<SCHEME>(p, vm[0], vm[1], vm[2], vm[3], vm[4]);
          }
#pragma unroll
          for (int c = 0; c < NV; c++) {
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < NV; k++) acc = acc + R[c][k] * hk[k];
            Fh[ps][c] = acc;
          }
        } else {
#pragma unroll
          for (int c = 0; c < NV; c++) Fh[ps][c] = 0.0;
        }
      } else {
#pragma unroll
        for (int c = 0; c < NV; c++) {
          const double *fp = sfp + (c * T::ROWS + row) * T::LEN;
          const double *fm = sfm + (c * T::ROWS + row) * T::LEN;
          const double h = recon<SCHEME>(p, fp[b - 2], fp[b - 1], fp[b], fp[b + 1], fp[b + 2]) +
                           recon<SCHEME>(p, fm[b + 3], fm[b + 2], fm[b + 1], fm[b], fm[b - 1]);
          Fh[ps][c] = FOLD ? 0.5 * h : h;
        }
      }
    }
  }
  __syncthreads();
  constexpr int FST = A == 0 ? T::FACES : T::FACES + 1;  // odd stride when lanes walk rows
  double *sh = sm;  // reuse: face fluxes [NV][ROWS][FST]
#pragma unroll
  for (int ps = 0; ps < T::PASSES; ps++) {
    int e = threadIdx.x + ps * THREADS;
    if (e < T::ROWS * T::FACES) {
      int row, fi;
      if constexpr (A == 0) { row = e / T::FACES; fi = e % T::FACES; }
      else { row = e % T::ROWS; fi = e / T::ROWS; }
#pragma unroll
      for (int c = 0; c < NV; c++) sh[(c * T::ROWS + row) * FST + fi] = Fh[ps][c];
    }
  }
  __syncthreads();

  // 3. L = L - (Fhat_{m+1/2} - Fhat_{m-1/2}) / h
  for (int e = threadIdx.x; e < T::ROWS * T::SEG; e += THREADS) {
    int row, l;
    if constexpr (A == 0) { row = e / T::SEG; l = e % T::SEG; }
    else { row = e % T::ROWS; l = e / T::ROWS; }
    int I[3];
    if (!cell_of(row, l, I) || I[A] >= p.n[A]) continue;
    long long o = int_index(p, I[0], I[1], I[2]);
#pragma unroll
    for (int c = 0; c < NV; c++) {
      const double *hh = sh + (c * T::ROWS + row) * FST;
      // dx/dxi at the cell (the spacing h on a uniform direction); the boundary cell of a
      // characteristic face takes its normal term from k_char_face instead
      double d = char_cell(p, A, I[A]) ? 0.0
                 : p.mm[A] ? divide(hh[l + 1] - hh[l], p.mm[A][I[A] + NG], p.minv[A][I[A] + NG])
                           : divide(hh[l + 1] - hh[l], p.h[A], p.inv_h[A]);
      double prev = first ? 0.0 : p.L[c * p.N + o];
      p.L[c * p.N + o] = prev - d;
    }
  }
}

// ------------------------------------------------------------------------------------------
// characteristic non-reflecting faces (Sec. 2, after Thompson): at the boundary cell the normal
// convective term is dF_a/dx_a in characteristic form, from fourth-order one-sided derivatives
// of the primitives with the entering waves' amplitudes set to zero
// ------------------------------------------------------------------------------------------
// fourth-order one-sided derivative into the domain (s = +1 from the low face, -1 from the high
// face) of the padded field phi at padded offset o, stride st along the direction;
// (-25 f0 + 48 f1 - 36 f2 + 16 f3 - 3 f4)/12 on the differences f_k - f0
__device__ __forceinline__ double one_sided(const double *phi, long long o, long long st, int s,
                                            double h12, double inv_h12) {
  const double f0 = phi[o];
  double acc = 0.0;
  acc = acc + 48.0 * (phi[o + s * st] - f0);
  acc = acc + -36.0 * (phi[o + 2 * s * st] - f0);
  acc = acc + 16.0 * (phi[o + 3 * s * st] - f0);
  acc = acc + -3.0 * (phi[o + 4 * s * st] - f0);
  return divide((double)s * acc, h12, inv_h12);
}

// one thread per cell of the face (a, side): L -= (dF_a/dx_a)_char, in the order the formulas
// are written (the strict form reproduces a sequential evaluation)
template <int DIM>
__global__ void k_char_face(Plan p, int a, int side) {
  constexpr int NV = DIM + 2;
  const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)p.n[b1] * p.n[b2]) return;
  int I[3];
  I[a] = side == 0 ? 0 : p.n[a] - 1;
  I[b1] = (int)(t % p.n[b1]);
  I[b2] = (int)(t / p.n[b1]);
  const int s = side == 0 ? 1 : -1;
  const long long o = pad_index(p, I[0], I[1], I[2]);
  const long long st = a == 0 ? 1 : a == 1 ? (long long)p.P[0] : (long long)p.P[0] * p.P[1];
  const double h12 = p.mm[a] ? 12.0 * p.mm[a][I[a] + NG] : p.h12[a];
  const double ih12 = p.mm[a] ? p.minv12[a][I[a] + NG] : p.inv_h12[a];
  const double r = p.Qp[o], pr = p.Wp[DIM * p.NP + o];
  const double c = sqrt(p.gamma * pr / r);
  const double ua = p.Wp[a * p.NP + o];
  const double rx = one_sided(p.Qp, o, st, s, h12, ih12);
  const double px = one_sided(p.Wp + DIM * p.NP, o, st, s, h12, ih12);
  const double uxa = one_sided(p.Wp + a * p.NP, o, st, s, h12, ih12);
  const double lam1 = ua - c, lam2 = ua, lam5 = ua + c;
  // a speed points into the domain when it has the sign of s
  const double L1 = (lam1 * (double)s > 0.0) ? 0.0 : lam1 * (px - r * c * uxa);
  const double L2 = (lam2 * (double)s > 0.0) ? 0.0 : lam2 * (c * c * rx - px);
  const double L5 = (lam5 * (double)s > 0.0) ? 0.0 : lam5 * (px + r * c * uxa);
  double dv[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int b = 0; b < DIM; b++) {
    if (b == a) continue;
    double utx = one_sided(p.Wp + b * p.NP, o, st, s, h12, ih12);
    dv[b] = (lam2 * (double)s > 0.0) ? 0.0 : lam2 * utx;
  }
  const double d1 = (L2 + 0.5 * (L5 + L1)) / (c * c);
  const double d2 = 0.5 * (L5 + L1);
  dv[a] = (L5 - L1) / (2.0 * r * c);
  double D[NV];
  double ke = 0.0, work = 0.0;
  D[0] = d1;
#pragma unroll
  for (int b = 0; b < DIM; b++) {
    double ub = p.Wp[b * p.NP + o];
    D[1 + b] = ub * d1 + r * dv[b];
    ke = ke + ub * ub;
    work = work + ub * dv[b];
  }
  D[NV - 1] = 0.5 * ke * d1 + d2 / p.gm1 + r * work;
  const long long oi = int_index(p, I[0], I[1], I[2]);
#pragma unroll
  for (int c2 = 0; c2 < NV; c2++) p.L[c2 * p.N + oi] = p.L[c2 * p.N + oi] - D[c2];
}

// ------------------------------------------------------------------------------------------
// viscous term (Eq. 2, 5): gradients of u by 4th-order central differences on the box
// [-2, n+2), tau_ij = du_i/dx_j + du_j/dx_i - 2/3 delta_ij div u, b_j = u_i tau_ij, then
// (1/Re) sum_a D4_a [0, tau_{.a}, b_a]
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double d4(double fm2, double fm1, double fp1, double fp2, double h12,
                                     double inv_h12) {
  return divide(8.0 * (fp1 - fm1) - (fp2 - fm2), h12, inv_h12);
}

template <int DIM>
__global__ void __launch_bounds__(THREADS) k_visc_flux(Plan p) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.NB) return;
  int bx = (int)(t % p.B[0]);
  long long r = t / p.B[0];
  int by = (int)(r % p.B[1]);
  int bz = (int)(r / p.B[1]);
  int I[3] = {bx - 2, DIM > 1 ? by - 2 : by, DIM > 2 ? bz - 2 : bz};
  long long s = pad_index(p, I[0], I[1], I[2]);
  long long stride[3] = {1, p.P[0], (long long)p.P[0] * p.P[1]};
  double g[DIM][DIM];
#pragma unroll
  for (int ci = 0; ci < DIM; ci++) {
    const double *u = p.Wp + ci * p.NP + s;
#pragma unroll
    for (int dj = 0; dj < DIM; dj++) {
      long long st = stride[dj];
      if (p.mm[dj]) {  // 12 dx/dxi at this node, rounded as 12 h is on a uniform direction
        int at = I[dj] + NG;
        g[ci][dj] = d4(u[-2 * st], u[-st], u[st], u[2 * st], 12.0 * p.mm[dj][at], p.minv12[dj][at]);
      } else {
        g[ci][dj] = d4(u[-2 * st], u[-st], u[st], u[2 * st], p.h12[dj], p.inv_h12[dj]);
      }
    }
  }
  double div = 0.0;
#pragma unroll
  for (int a = 0; a < DIM; a++) div += g[a][a];
#pragma unroll
  for (int a = 0; a < DIM; a++) {
    double b = 0.0;
#pragma unroll
    for (int ci = 0; ci < DIM; ci++) {
      double tau = g[ci][a] + g[a][ci];
      if (ci == a) tau -= 2.0 / 3.0 * div;
      p.V[(long long)(a * (DIM + 1) + ci) * p.NB + t] = tau;
      b += p.Wp[ci * p.NP + s] * tau;
    }
    p.V[(long long)(a * (DIM + 1) + DIM) * p.NB + t] = b;
  }
}

template <int DIM>
__global__ void __launch_bounds__(THREADS) k_visc_div(Plan p) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.N) return;
  int i = (int)(t % p.n[0]);
  long long r = t / p.n[0];
  int j = (int)(r % p.n[1]);
  int k = (int)(r / p.n[1]);
  long long b = ((long long)(DIM > 2 ? k + 2 : k) * p.B[1] + (DIM > 1 ? j + 2 : j)) * p.B[0] + (i + 2);
  long long stride[3] = {1, p.B[0], (long long)p.B[0] * p.B[1]};
#pragma unroll
  for (int fc = 0; fc <= DIM; fc++) {
    double sum = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      const double *F = p.V + (long long)(a * (DIM + 1) + fc) * p.NB + b;
      long long st = stride[a];
      if (p.mm[a]) {
        int at = (a == 0 ? i : a == 1 ? j : k) + NG;
        sum += d4(F[-2 * st], F[-st], F[st], F[2 * st], 12.0 * p.mm[a][at], p.minv12[a][at]);
      } else {
        sum += d4(F[-2 * st], F[-st], F[st], F[2 * st], p.h12[a], p.inv_h12[a]);
      }
    }
    long long o = (long long)(fc + 1) * p.N + t;
    p.L[o] = p.L[o] + divide(sum, p.Re, p.inv_Re);
  }
}

// ------------------------------------------------------------------------------------------
// immersed boundary (Eq. 7-9)
// ------------------------------------------------------------------------------------------
// the four-point supports of point k of X [dim][nm] in every direction (Eq. 10-11); *hprod
// (may be NULL) receives the product of the local spacings, h^d of the delta at the point
template <int DIM>
__device__ __forceinline__ bool marker_support(const Plan &p, const double *X, int nm, int k,
                                               int j0[3], double w[3][4],
                                               double *hprod = nullptr) {
  bool ok = true;
  double hp = 1.0;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (a < DIM) {
      if (p.mx[a]) {
        double s, hl;
        j0[a] = mesh::support_stretched(p, a, X[a * nm + k], &s, &hl);
#pragma unroll
        for (int r = 0; r < 4; r++) w[a][r] = peskin(s - (double)(j0[a] + r));
        hp *= hl;
      } else {
        j0[a] = support(p, a, X[a * nm + k], w[a]);
        hp *= p.h[a];
      }
      if (j0[a] < 0 || j0[a] + 3 > p.n[a] - 1) ok = false;
    } else {
      j0[a] = 0;
      w[a][0] = 1.0; w[a][1] = 0.0; w[a][2] = 0.0; w[a][3] = 0.0;
    }
  }
  if (hprod) *hprod = hp;
  return ok;
}

// U_ib = sum_j u_j prod lambda (Eq. 8), F = alpha xi + beta (U_ib - U) (Eq. 7), and the RK
// update of xi (xi' = U_ib - U) when the stage is advanced
template <int DIM>
__global__ void k_ib_interp(Plan p, const double *__restrict__ xis, const double *xin,
                            double *xio, double A, double Bc, double dt, int advance) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int nm = p.nm, M = p.max_markers;
  if (k >= nm) return;
  int j0[3];
  double w[3][4];
  if (!marker_support<DIM>(p, p.X, M, k, j0, w)) {
    atomicOr(p.status, IBFSA_STATUS_BOUNDS);
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      p.F[a * M + k] = 0.0;
      if (advance) xio[a * M + k] = xin[a * M + k];
    }
    return;
  }
  constexpr int C2 = DIM > 2 ? 4 : 1;
#pragma unroll
  for (int a = 0; a < DIM; a++) {
    const double *u = p.Wp + a * p.NP;
    double acc = 0.0;
    for (int r2 = 0; r2 < C2; r2++)
      for (int r1 = 0; r1 < 4; r1++)
#pragma unroll
        for (int r0 = 0; r0 < 4; r0++)
          acc += u[pad_index(p, j0[0] + r0, j0[1] + r1, j0[2] + r2)] *
                 (w[0][r0] * w[1][r1] * w[2][r2]);
    double slip = acc - p.U[a * M + k];
    p.F[a * M + k] = p.alpha_pen * xis[a * M + k] + p.beta_pen * slip;
    if (advance) xio[a * M + k] = A * xin[a * M + k] + Bc * (xis[a * M + k] + dt * slip);
  }
}

// strict spreading: one block walks the markers in order; its threads own the 4^DIM support
// cells of the current marker (distinct cells), so every cell sums its contributions in marker
// order: f_j = f_j - F_k w dS_k / prod h  (Eq. 9)
template <int DIM>
__global__ void k_spread_ordered(Plan p) {
  constexpr int C2 = DIM > 2 ? 4 : 1;
  int r = threadIdx.x;  // 0 .. 4^DIM - 1
  int r0 = r & 3, r1 = (r >> 2) & 3, r2 = DIM > 2 ? (r >> 4) : 0;
  int M = p.max_markers;
  for (int k = 0; k < p.nm; k++) {
    int j0[3];
    double w[3][4], hprod;
    bool ok = marker_support<DIM>(p, p.X, M, k, j0, w, &hprod);
    if (ok && r < 4 * 4 * C2) {
      double wt = w[0][r0] * w[1][r1] * w[2][r2];
      long long o = int_index(p, j0[0] + r0, j0[1] + r1, j0[2] + r2);
#pragma unroll
      for (int a = 0; a < DIM; a++)
        p.f[a * p.N + o] -= p.F[a * M + k] * wt * p.dS[k] / hprod;
    }
    __syncthreads();
  }
}

// fast spreading: one thread per (marker, support cell), atomics straight into L:
// momentum += f, energy += f.u
template <int DIM>
__global__ void k_spread_atomic(Plan p) {
  constexpr int S = DIM > 2 ? 64 : 16;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)p.nm * S) return;
  int k = (int)(t / S), r = (int)(t % S);
  int r0 = r & 3, r1 = (r >> 2) & 3, r2 = DIM > 2 ? (r >> 4) : 0;
  int M = p.max_markers;
  int j0[3];
  double w[3][4], hprod;
  if (!marker_support<DIM>(p, p.X, M, k, j0, w, &hprod)) return;
  double wt = w[0][r0] * w[1][r1] * w[2][r2];
  long long o = int_index(p, j0[0] + r0, j0[1] + r1, j0[2] + r2);
  long long s = pad_index(p, j0[0] + r0, j0[1] + r1, j0[2] + r2);
  double scale = wt * p.dS[k] / hprod;
  double pw = 0.0;
#pragma unroll
  for (int a = 0; a < DIM; a++) {
    double fa = -p.F[a * M + k] * scale;
    atomicAdd(&p.L[(1 + a) * p.N + o], fa);
    pw += fa * p.Wp[a * p.NP + s];
  }
  atomicAdd(&p.L[(DIM + 1) * p.N + o], pw);
}

// ------------------------------------------------------------------------------------------
// finish: sponge, strict-mode IB source, then RHS out or RK combination a Qn + b (Qs + dt L)
// ------------------------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(THREADS) k_finish(Plan p, const double *__restrict__ Qs,
                                                    const double *Qn, double *out, double A,
                                                    double Bc, double dt, int advance) {
  constexpr int NV = DIM + 2;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.N) return;
  int I[3];
  I[0] = (int)(t % p.n[0]);
  long long r = t / p.n[0];
  I[1] = (int)(r % p.n[1]);
  I[2] = (int)(r / p.n[1]);
  double Lc[NV];
#pragma unroll
  for (int c = 0; c < NV; c++) Lc[c] = p.L[c * p.N + t];
  if (p.sponge_cells > 0) {
    int S = p.sponge_cells;
    int nmin = 1 << 30;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      int e = I[a] < p.n[a] - 1 - I[a] ? I[a] : p.n[a] - 1 - I[a];
      if (e < nmin) nmin = e;
    }
    if (nmin < S) {
      double rr = (double)(S - nmin) / (double)S;
      double sig = p.sponge_sigma * rr * rr * rr;
#pragma unroll
      for (int c = 0; c < NV; c++) Lc[c] = Lc[c] - sig * (Qs[c * p.N + t] - p.qinf[c]);
    }
  }
  if (p.src_on) {  // periodic Gaussian pressure source (Sec. 3.6, Eq. 16), energy equation
    const double LN2 = 0.693147180559945309417;
    double r2 = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      double x = mesh::node(p, a, I[a]);
      r2 = r2 + (x - p.src_xc[a]) * (x - p.src_xc[a]);
    }
    Lc[NV - 1] = Lc[NV - 1] + exp(-(p.src_b * LN2) * r2) * p.src_scale;
  }
  if constexpr (STRICT) {
    if (p.nm > 0) {
      long long s = pad_index(p, I[0], I[1], I[2]);
      double pw = 0.0;
#pragma unroll
      for (int a = 0; a < DIM; a++) {
        double fa = p.f[a * p.N + t];
        Lc[1 + a] = Lc[1 + a] + fa;
        pw += fa * p.Wp[a * p.NP + s];
      }
      Lc[NV - 1] = Lc[NV - 1] + pw;
    }
  }
  if (!advance) {
#pragma unroll
    for (int c = 0; c < NV; c++) out[c * p.N + t] = Lc[c];
  } else {
    bool bad = false;
#pragma unroll
    for (int c = 0; c < NV; c++) {
      double v = A * Qn[c * p.N + t] + Bc * (Qs[c * p.N + t] + dt * Lc[c]);
      out[c * p.N + t] = v;
      bad |= !isfinite(v);
    }
    if (bad) atomicOr(p.status, IBFSA_STATUS_NONFINITE);
  }
}

// ------------------------------------------------------------------------------------------
// probes: dp = sum_j p_j prod lambda - p_inf
// ------------------------------------------------------------------------------------------
template <int DIM>
__global__ void k_probe(Plan p, int np, const double *__restrict__ xp, double *__restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  int j0[3];
  double w[3][4];
  if (!marker_support<DIM>(p, xp, np, k, j0, w)) {
    atomicOr(p.status, IBFSA_STATUS_BOUNDS);
    out[k] = 0.0;
    return;
  }
  constexpr int C2 = DIM > 2 ? 4 : 1;
  const double *pr = p.Wp + DIM * p.NP;
  double acc = 0.0;
  for (int r2 = 0; r2 < C2; r2++)
    for (int r1 = 0; r1 < 4; r1++)
#pragma unroll
      for (int r0 = 0; r0 < 4; r0++)
        acc += pr[pad_index(p, j0[0] + r0, j0[1] + r1, j0[2] + r2)] *
               (w[0][r0] * w[1][r1] * w[2][r2]);
  out[k] = acc - p.p_inf;
}

// ------------------------------------------------------------------------------------------
// host-side orchestration of one stage
// ------------------------------------------------------------------------------------------
inline unsigned blocks_for(long long n, int threads) {
  return (unsigned)((n + threads - 1) / threads);
}

template <int DIM, int A, int SCHEME>
cudaError_t launch_conv(const Plan &p, int first, cudaStream_t st) {
  using T = ConvTile<A>;
  constexpr size_t smem = conv_smem_bytes<DIM, A>();
  cudaError_t e = p.charwise
                      ? cudaFuncSetAttribute(k_conv<DIM, A, SCHEME, true>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                      : cudaFuncSetAttribute(k_conv<DIM, A, SCHEME, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid;
  if (A == 0) {
    grid = dim3((p.n[0] + T::SEG - 1) / T::SEG, (p.n[1] + T::ROWS - 1) / T::ROWS, p.n[2]);
  } else {
    int nseg = (p.n[A] + T::SEG - 1) / T::SEG;
    int nx = (p.n[0] + T::ROWS - 1) / T::ROWS;
    grid = dim3(nseg * nx, A == 1 ? p.n[2] : p.n[1]);
  }
  if (p.charwise) k_conv<DIM, A, SCHEME, true><<<grid, THREADS, smem, st>>>(p, first);
  else k_conv<DIM, A, SCHEME, false><<<grid, THREADS, smem, st>>>(p, first);
  return cudaGetLastError();
}

template <int DIM, int SCHEME>
cudaError_t run_stage(const Plan &p, const StageArgs &s, cudaStream_t st) {
  cudaError_t e;
  Prof *pr = s.prof;
  e = cudaMemsetAsync(p.alpha_bits, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  prof_begin(pr, st);
  k_pad<DIM><<<blocks_for(p.NP, THREADS), THREADS, 0, st>>>(p, s.Qs);
  prof_end(pr, K_PAD, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int advance = s.stage >= 0;
  if (p.nm > 0) {
    prof_begin(pr, st);
    k_ib_interp<DIM><<<blocks_for(p.nm, 128), 128, 0, st>>>(p, s.xis, s.xin, s.xio, s.a, s.b,
                                                           s.dt, advance);
    prof_end(pr, K_INTERP, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  prof_begin(pr, st);
  e = launch_conv<DIM, 0, SCHEME>(p, 1, st);
  prof_end(pr, K_CONV_X, st);
  if (e != cudaSuccess) return e;
  prof_begin(pr, st);
  e = launch_conv<DIM, 1, SCHEME>(p, 0, st);
  prof_end(pr, K_CONV_Y, st);
  if (e != cudaSuccess) return e;
  if constexpr (DIM == 3) {
    prof_begin(pr, st);
    e = launch_conv<DIM, 2, SCHEME>(p, 0, st);
    prof_end(pr, K_CONV_Z, st);
    if (e != cudaSuccess) return e;
  }
  // characteristic faces, direction by direction, low face first
  for (int a = 0; a < DIM; a++)
    for (int side = 0; side < 2; side++) {
      if (p.bc[a][side] != IBFSA_BC_CHARACTERISTIC) continue;
      long long cells = (long long)p.n[(a + 1) % 3] * p.n[(a + 2) % 3];
      prof_begin(pr, st);
      k_char_face<DIM><<<blocks_for(cells, THREADS), THREADS, 0, st>>>(p, a, side);
      prof_end(pr, K_CONV_X + a, st);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  if (p.Re > 0.0) {
    prof_begin(pr, st);
    k_visc_flux<DIM><<<blocks_for(p.NB, THREADS), THREADS, 0, st>>>(p);
    prof_end(pr, K_VISC_FLUX, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    prof_begin(pr, st);
    k_visc_div<DIM><<<blocks_for(p.N, THREADS), THREADS, 0, st>>>(p);
    prof_end(pr, K_VISC_DIV, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (p.nm > 0) {
    if constexpr (STRICT) {
      e = cudaMemsetAsync(p.f, 0, sizeof(double) * DIM * p.N, st);
      if (e != cudaSuccess) return e;
      prof_begin(pr, st);
      k_spread_ordered<DIM><<<1, DIM > 2 ? 64 : 16, 0, st>>>(p);
      prof_end(pr, K_SPREAD, st);
    } else {
      constexpr int S = DIM > 2 ? 64 : 16;
      prof_begin(pr, st);
      k_spread_atomic<DIM><<<blocks_for((long long)p.nm * S, THREADS), THREADS, 0, st>>>(p);
      prof_end(pr, K_SPREAD, st);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  double *out = advance ? s.Qo : s.Lout;
  prof_begin(pr, st);
  Plan q = p;
  q.src_scale = s.src_scale;
  k_finish<DIM><<<blocks_for(p.N, THREADS), THREADS, 0, st>>>(q, s.Qs, s.Qn, out, s.a, s.b, s.dt,
                                                             advance);
  prof_end(pr, K_FINISH, st);
  return cudaGetLastError();
}

inline cudaError_t stage_impl(const Plan &p, const StageArgs &s, cudaStream_t st) {
  if (p.dim == 2)
    return p.scheme == IBFSA_TENO5 ? run_stage<2, IBFSA_TENO5>(p, s, st)
                                   : run_stage<2, IBFSA_WENO5JS>(p, s, st);
  return p.scheme == IBFSA_TENO5 ? run_stage<3, IBFSA_TENO5>(p, s, st)
                                 : run_stage<3, IBFSA_WENO5JS>(p, s, st);
}

inline cudaError_t wavespeed_impl(const Plan &p, const double *Q, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(p.alpha_bits, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (p.dim == 2) k_pad<2><<<blocks_for(p.NP, THREADS), THREADS, 0, st>>>(p, Q);
  else k_pad<3><<<blocks_for(p.NP, THREADS), THREADS, 0, st>>>(p, Q);
  return cudaGetLastError();
}

inline cudaError_t probe_impl(const Plan &p, const double *Q, int np, const double *xp,
                              double *out, cudaStream_t st, Prof *pr) {
  prof_begin(pr, st);
  cudaError_t e = wavespeed_impl(p, Q, st);  // pad + primitives of the current state
  prof_end(pr, K_PAD, st);
  if (e != cudaSuccess) return e;
  prof_begin(pr, st);
  if (p.dim == 2) k_probe<2><<<blocks_for(np, 128), 128, 0, st>>>(p, np, xp, out);
  else k_probe<3><<<blocks_for(np, 128), 128, 0, st>>>(p, np, xp, out);
  prof_end(pr, K_PROBE, st);
  return cudaGetLastError();
}

}  // namespace IBFSA_MODE_NS
}  // namespace ibfsa
