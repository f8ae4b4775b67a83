// stage_fp32.cu -- the perturbation form of one Runge-Kutta stage (arXiv:1905.00182, Sec. 2):
// the stencil arithmetic in FP32 on q' = Q - q_inf and on primitive perturbations, expanded so
// that no O(1) free-stream term ever cancels, while the RK state and its combination, the IB
// markers (Eq. 7-9) and the probes stay FP64.
//
// Perturbation algebra (u = u_inf + u', m_inf = rho_inf u_inf, H_inf = E_inf + p_inf):
//   u'_a = (m'_a - rho' u_inf_a) / rho
//   p'   = (gamma - 1) (E' - (m' . u + m_inf . u') / 2)
//   F'_d = [m'_d,  m'_i u_d + m_inf_i u'_d + p' delta_id,  (E' + p') u_d + H_inf u'_d]
// The split f+-' = (F'_d +- alpha_d q')/2 differs from f+- by a constant, and both candidate
// polynomials and smoothness indicators are invariant under constant shifts, so the
// reconstructed flux differences are those of the full fluxes.  Gradients of u equal those of
// u', and b_j = (u_inf + u')_i tau_ij.
//
// Stage values inside a step are FP32 increments over the FP64 state: with a_s + b_s = 1,
//   Q^(s+1) - Qn = b_s (Q^(s) - Qn + dt L(Q^(s))),
// so d1 = dt L(Qn), d2 = (d1 + dt L(Q1))/4 and the step ends with Qn += 2/3 (d2 + dt L(Q2)),
// added in FP64 -- the only FP64 arithmetic of the bulk.  qn32 = (float)(Qn - q_inf) is
// refreshed from the FP64 state at the end of every step, so stencil inputs never drift.
//
// TENO5 in FP32: eps = 1e-40 is below the FP32 normal range, so eps = 1e-30 is used, and the
// cut-off is evaluated on gamma_k / gamma_max = ((1 + r_k)/(1 + r_max))^6 (r = tau5/(beta + eps)),
// which keeps every quantity in [0, 1] without changing the decision gamma_k >= C_T sum gamma.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ibfsa_internal.h"
#include "mesh.cuh"
#include "mlp_tile.cuh"
#include "tma.cuh"

namespace ibfsa {
namespace fp32_ns {

constexpr int THREADS = 256;

struct Free {
  float rho, p, H, gamma, gm1;
  float u[3], m[3];
};

__device__ __forceinline__ Free free_stream(const Plan &p) {
  Free f;
  f.rho = p.rho_inf32;
  f.p = p.p_inf32;
  f.H = p.H_inf32;
  f.gamma = p.gamma32;
  f.gm1 = p.gm1_32;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    f.u[a] = p.u_inf32[a];
    f.m[a] = p.m_inf32[a];
  }
  return f;
}

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

// the boundary cell of a characteristic face along a (its normal term comes from k_char_face32)
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

// Peskin's four-point kernel, Eq. 11 (FP64: the IB and the probes stay in double precision)
__device__ __forceinline__ double peskin(double r) {
  double a = fabs(r);
  if (a < 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) * 0.125;
  if (a < 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) * 0.125;
  return 0.0;
}

// four-point supports of point k of X [dim][stride] (Eq. 10-11); *hprod (may be NULL): the
// product of the local spacings
template <int DIM>
__device__ __forceinline__ bool point_support(const Plan &p, const double *X, int stride, int k,
                                              int j0[3], double w[3][4],
                                              double *hprod = nullptr) {
  bool ok = true;
  double hp = 1.0;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    if (a < DIM) {
      double s, hl;
      if (p.mx[a]) {
        j0[a] = mesh::support_stretched(p, a, X[a * stride + k], &s, &hl);
      } else {
        s = (X[a * stride + k] - p.lo[a]) * p.inv_h[a] - 0.5;
        j0[a] = (int)floor(s) - 1;
        hl = p.h[a];
      }
      hp *= hl;
#pragma unroll
      for (int r = 0; r < 4; r++) w[a][r] = peskin(s - (double)(j0[a] + r));
      if (j0[a] < 0 || j0[a] + 3 > p.n[a] - 1) ok = false;
    } else {
      j0[a] = 0;
      w[a][0] = 1.0; w[a][1] = 0.0; w[a][2] = 0.0; w[a][3] = 0.0;
    }
  }
  if (hprod) *hprod = hp;
  return ok;
}

// ------------------------------------------------------------------------------------------
// FP32 reconstructions at face i+1/2 from (f_{i-2}, ..., f_{i+2})
// ------------------------------------------------------------------------------------------
struct Cands {
  float q0, q1, q2, b0, b1, b2;
};

__device__ __forceinline__ Cands candidates(float a, float b, float c, float d, float e) {
  Cands r;
  const float s6 = 1.f / 6.f;
  r.q0 = (2.f * a - 7.f * b + 11.f * c) * s6;
  r.q1 = (-b + 5.f * c + 2.f * d) * s6;
  r.q2 = (2.f * c + 5.f * d - e) * s6;
  const float k13 = 13.f / 12.f;
  float t, u;
  t = a - 2.f * b + c; u = a - 4.f * b + 3.f * c; r.b0 = k13 * t * t + 0.25f * u * u;
  t = b - 2.f * c + d; u = b - d;                 r.b1 = k13 * t * t + 0.25f * u * u;
  t = c - 2.f * d + e; u = 3.f * c - 4.f * d + e; r.b2 = k13 * t * t + 0.25f * u * u;
  return r;
}

__device__ __forceinline__ float weno5js(float a, float b, float c, float d, float e) {
  Cands k = candidates(a, b, c, d, e);
  const float eps = 1e-6f;
  float s0 = (eps + k.b0) * (eps + k.b0);
  float s1 = (eps + k.b1) * (eps + k.b1);
  float s2 = (eps + k.b2) * (eps + k.b2);
  float al0 = 0.1f * (s1 * s2), al1 = 0.6f * (s0 * s2), al2 = 0.3f * (s0 * s1);
  return __fdividef(al0 * k.q0 + al1 * k.q1 + al2 * k.q2, al0 + al1 + al2);
}

__device__ __forceinline__ int teno_mask(const Cands &k) {
  const float eps = 1e-30f, CT = 1e-5f;
  float tau = fabsf(k.b0 - k.b2);
  float r0 = __fdividef(tau, k.b0 + eps);
  float r1 = __fdividef(tau, k.b1 + eps);
  float r2 = __fdividef(tau, k.b2 + eps);
  float inv = __fdividef(1.f, 1.f + fmaxf(r0, fmaxf(r1, r2)));
  float t, t2, g0, g1, g2;
  t = (1.f + r0) * inv; t2 = t * t; g0 = t2 * t2 * t2;
  t = (1.f + r1) * inv; t2 = t * t; g1 = t2 * t2 * t2;
  t = (1.f + r2) * inv; t2 = t * t; g2 = t2 * t2 * t2;
  float th = CT * (g0 + g1 + g2);
  return (g0 >= th ? 1 : 0) | (g1 >= th ? 2 : 0) | (g2 >= th ? 4 : 0);
}

__device__ __forceinline__ float teno5(const Plan &tw, float a, float b, float c, float d,
                                       float e) {
  Cands k = candidates(a, b, c, d, e);
  const float eps = 1e-30f, CT = 1e-5f;
  float tau = fabsf(k.b0 - k.b2);
  float r0 = __fdividef(tau, k.b0 + eps);
  float r1 = __fdividef(tau, k.b1 + eps);
  float r2 = __fdividef(tau, k.b2 + eps);
  float inv = __fdividef(1.f, 1.f + fmaxf(r0, fmaxf(r1, r2)));
  float t, t2, g0, g1, g2;
  t = (1.f + r0) * inv; t2 = t * t; g0 = t2 * t2 * t2;
  t = (1.f + r1) * inv; t2 = t * t; g1 = t2 * t2 * t2;
  t = (1.f + r2) * inv; t2 = t * t; g2 = t2 * t2 * t2;
  float th = CT * (g0 + g1 + g2);
  int mask = (g0 >= th ? 1 : 0) | (g1 >= th ? 2 : 0) | (g2 >= th ? 4 : 0);
  const float *w = tw.teno_w32[mask];
  return w[0] * k.q0 + w[1] * k.q1 + w[2] * k.q2;
}

// Smoothness indicators only (the candidates are not needed on the smooth path).
__device__ __forceinline__ void indicators(float a, float b, float c, float d, float e,
                                           float &b0, float &b1, float &b2) {
  const float k13 = 13.f / 12.f;
  float t, u;
  t = a - 2.f * b + c; u = a - 4.f * b + 3.f * c; b0 = k13 * t * t + 0.25f * u * u;
  t = b - 2.f * c + d; u = b - d;                 b1 = k13 * t * t + 0.25f * u * u;
  t = c - 2.f * d + e; u = 3.f * c - 4.f * d + e; b2 = k13 * t * t + 0.25f * u * u;
}

// TENO5 keeps every stencil when tau5 <= 4 (min beta + eps): then each gamma_k lies in
// [1, 5^6] and chi_k >= 1/(3 5^6) = 2.1e-5 > C_T = 1e-5.  The reconstruction is then the
// optimal linear combination (2a - 13b + 47c + 27d - 3e)/60, without divisions or powers.
__device__ __forceinline__ bool teno_all_kept(float b0, float b1, float b2) {
  return fabsf(b0 - b2) <= 4.f * (fminf(b0, fminf(b1, b2)) + 1e-30f);
}

__device__ __forceinline__ float linear5(float a, float b, float c, float d, float e) {
  return (2.f * a - 13.f * b + 47.f * c + 27.f * d - 3.f * e) * (1.f / 60.f);
}

__device__ __forceinline__ float teno5_fast(const Plan &tw, float a, float b, float c, float d,
                                            float e) {
  float b0, b1, b2;
  indicators(a, b, c, d, e, b0, b1, b2);
  if (teno_all_kept(b0, b1, b2)) return linear5(a, b, c, d, e);
  return teno5(tw, a, b, c, d, e);
}

// make_float2(v, v)
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// TENO5 at one face for both split fluxes on packed FP32x2 arithmetic, with a warp-uniform slow
// path: every lane of the warp must call it.  The input is the interleaved face stencil
// z_k = (f+ at staged cell i+k, f- at staged cell i+k+1), k = 0..4, of the face between staged
// cells i+2 and i+3: the .x lanes are the f+ stencil upwind to downwind, the .y lanes the f-
// stencil downwind to upwind, so one 8-byte load per k fetches both sides.  With the f- stencil
// reversed, the packed indicator of z0 z1 z2 is (beta_0+, beta_2-) and that of z2 z3 z4 is
// (beta_2+, beta_0-) (the second differences and the squared one-sided differences are
// symmetric under the reversal), so tau5 and the all-kept test are those of each side; the
// linear combination takes per-lane coefficient pairs.  The all-kept test is scale-invariant, so
// the indicators are taken times 4, (13/3) t^2 + u^2 (one multiplication fewer each), with the
// floor 4e-30.  The linear (all-kept) result is computed without branches; only when some lane
// of the warp has a side that cuts a stencil does the whole warp enter the full TENO5 (a uniform
// branch, no divergence to reconverge).
__device__ __forceinline__ float teno5_pz_warp(const Plan &tw, float2 z0, float2 z1, float2 z2,
                                               float2 z3, float2 z4) {
  float2 t0 = __fadd2_rn(__ffma2_rn(f2(-2.f), z1, z0), z2);
  float2 t1 = __fadd2_rn(__ffma2_rn(f2(-2.f), z2, z1), z3);
  float2 t2 = __fadd2_rn(__ffma2_rn(f2(-2.f), z3, z2), z4);
  float2 u0 = __ffma2_rn(f2(3.f), z2, __ffma2_rn(f2(-4.f), z1, z0));
  float2 u1 = __ffma2_rn(f2(-1.f), z3, z1);
  float2 u2 = __ffma2_rn(f2(3.f), z2, __ffma2_rn(f2(-4.f), z3, z4));
  const float2 k13 = f2(13.f / 3.f);
  float2 b0 = __ffma2_rn(__fmul2_rn(k13, t0), t0, __fmul2_rn(u0, u0));
  float2 b1 = __ffma2_rn(__fmul2_rn(k13, t1), t1, __fmul2_rn(u1, u1));
  float2 b2 = __ffma2_rn(__fmul2_rn(k13, t2), t2, __fmul2_rn(u2, u2));
  float2 tau = __ffma2_rn(f2(-1.f), b2, b0);
  const bool kx = fabsf(tau.x) <= fmaf(4.f, fminf(b0.x, fminf(b1.x, b2.x)), 1.6e-29f);
  const bool ky = fabsf(tau.y) <= fmaf(4.f, fminf(b0.y, fminf(b1.y, b2.y)), 1.6e-29f);
  float2 lin = __fmul2_rn(make_float2(2.f / 60.f, -3.f / 60.f), z0);
  lin = __ffma2_rn(make_float2(-13.f / 60.f, 27.f / 60.f), z1, lin);
  lin = __ffma2_rn(f2(47.f / 60.f), z2, lin);
  lin = __ffma2_rn(make_float2(27.f / 60.f, -13.f / 60.f), z3, lin);
  lin = __ffma2_rn(make_float2(-3.f / 60.f, 2.f / 60.f), z4, lin);
  float h = lin.x + lin.y;
  if (__any_sync(0xffffffffu, !(kx && ky))) {
    float hx = kx ? lin.x : teno5(tw, z0.x, z1.x, z2.x, z3.x, z4.x);
    float hy = ky ? lin.y : teno5(tw, z4.y, z3.y, z2.y, z1.y, z0.y);
    h = hx + hy;
  }
  return h;
}

// teno5_pz_warp per side: returns (h+, h-) and whether each side keeps all three stencils (by
// the all-kept test or, where that fails, by the full cut-off).  Every lane of the warp must call
// it.
__device__ __forceinline__ float2 teno5_pz_sides(const Plan &tw, float2 z0, float2 z1, float2 z2,
                                                 float2 z3, float2 z4, bool &kx, bool &ky) {
  float2 t0 = __fadd2_rn(__ffma2_rn(f2(-2.f), z1, z0), z2);
  float2 t1 = __fadd2_rn(__ffma2_rn(f2(-2.f), z2, z1), z3);
  float2 t2 = __fadd2_rn(__ffma2_rn(f2(-2.f), z3, z2), z4);
  float2 u0 = __ffma2_rn(f2(3.f), z2, __ffma2_rn(f2(-4.f), z1, z0));
  float2 u1 = __ffma2_rn(f2(-1.f), z3, z1);
  float2 u2 = __ffma2_rn(f2(3.f), z2, __ffma2_rn(f2(-4.f), z3, z4));
  const float2 k13 = f2(13.f / 3.f);
  float2 b0 = __ffma2_rn(__fmul2_rn(k13, t0), t0, __fmul2_rn(u0, u0));
  float2 b1 = __ffma2_rn(__fmul2_rn(k13, t1), t1, __fmul2_rn(u1, u1));
  float2 b2 = __ffma2_rn(__fmul2_rn(k13, t2), t2, __fmul2_rn(u2, u2));
  float2 tau = __ffma2_rn(f2(-1.f), b2, b0);
  kx = fabsf(tau.x) <= fmaf(4.f, fminf(b0.x, fminf(b1.x, b2.x)), 1.6e-29f);
  ky = fabsf(tau.y) <= fmaf(4.f, fminf(b0.y, fminf(b1.y, b2.y)), 1.6e-29f);
  float2 lin = __fmul2_rn(make_float2(2.f / 60.f, -3.f / 60.f), z0);
  lin = __ffma2_rn(make_float2(-13.f / 60.f, 27.f / 60.f), z1, lin);
  lin = __ffma2_rn(f2(47.f / 60.f), z2, lin);
  lin = __ffma2_rn(make_float2(27.f / 60.f, -13.f / 60.f), z3, lin);
  lin = __ffma2_rn(make_float2(-3.f / 60.f, 2.f / 60.f), z4, lin);
  if (__any_sync(0xffffffffu, !(kx && ky))) {
    if (!kx) {
      const Cands k = candidates(z0.x, z1.x, z2.x, z3.x, z4.x);
      const int mask = teno_mask(k);
      const float *w = tw.teno_w32[mask];
      lin.x = w[0] * k.q0 + w[1] * k.q1 + w[2] * k.q2;
      kx = mask == 7;
    }
    if (!ky) {
      const Cands k = candidates(z4.y, z3.y, z2.y, z1.y, z0.y);
      const int mask = teno_mask(k);
      const float *w = tw.teno_w32[mask];
      lin.y = w[0] * k.q0 + w[1] * k.q1 + w[2] * k.q2;
      ky = mask == 7;
    }
  }
  return lin;
}

// The learned weights' face loop, in two phases.  First, unrolled as the component-wise pass,
// packed TENO5 at every face and the eligibility of each side (TENO5 keeping all three stencils
// and an amplitude above the floor), one bit per (pass, component, side).  Then a rolled loop
// over (pass, component) with one call site of the warp-wide network (unrolled, the network's
// code was copied 2 x NV x MAXP times and the kernel ran out of the instruction cache) visits
// only the faces where some lane of the warp is eligible: a side with an eligible lane runs the
// network for all 32 lanes' stencils of that side, and its eligible lanes take the delta-form
// reconstruction with the network's weights.  zat(ps, c, valid) gives the interleaved stencil
// z_0 (z_k ZS float2 further) of this thread's face slot ps, component c, and whether the slot
// holds a face (an empty slot points at a valid stencil, its results unused).  Every lane of the
// warp must call it; used / seen accumulate this lane's counts.
template <int MAXP, int NV, int ZS, typename ZAt>
__device__ __forceinline__ void learned_faces(const Plan &p, const unsigned char *img,
                                              float (&Fh)[MAXP][NV], unsigned &used,
                                              unsigned &seen, ZAt zat) {
  static_assert(2 * MAXP * NV <= 32, "one eligibility bit per (pass, component, side)");
  unsigned emask = 0;
#pragma unroll
  for (int ps = 0; ps < MAXP; ps++) {
    bool valid = false;
#pragma unroll
    for (int c = 0; c < NV; c++) {
      const float2 *z = zat(ps, c, valid);
      const float2 z0 = z[0], z1 = z[ZS], z2 = z[2 * ZS], z3 = z[3 * ZS], z4 = z[4 * ZS];
      bool kx, ky;
      const float2 h = teno5_pz_sides(p, z0, z1, z2, z3, z4, kx, ky);
      Fh[ps][c] = h.x + h.y;
      // amplitude max_j |v_j - v_2| of each side (the same set of values in either order)
      const float2 d0 = __ffma2_rn(f2(-1.f), z2, z0), d1 = __ffma2_rn(f2(-1.f), z2, z1);
      const float2 d3 = __ffma2_rn(f2(-1.f), z2, z3), d4 = __ffma2_rn(f2(-1.f), z2, z4);
      const float ax = fmaxf(fmaxf(fabsf(d0.x), fabsf(d1.x)), fmaxf(fabsf(d3.x), fabsf(d4.x)));
      const float ay = fmaxf(fmaxf(fabsf(d0.y), fabsf(d1.y)), fmaxf(fabsf(d3.y), fabsf(d4.y)));
      const bool ex = valid && kx && ax > p.mlp_floor, ey = valid && ky && ay > p.mlp_floor;
      const int j = 2 * (ps * NV + c);
      emask |= (ex ? 1u << j : 0u) | (ey ? 2u << j : 0u);
    }
    seen += valid ? 2 * NV : 0;
  }
  used += __popc(emask);
#pragma unroll 1
  for (int it = 0; it < MAXP * NV; it++) {
    const unsigned bits = (emask >> (2 * it)) & 3u;
    const unsigned bx = __ballot_sync(0xffffffffu, bits & 1u);
    const unsigned by = __ballot_sync(0xffffffffu, bits & 2u);
    if ((bx | by) == 0u) continue;  // warp-uniform
    const int ps = it / NV, c = it % NV;
    bool valid;
    const float2 *z = zat(ps, c, valid);
    // phase 1's TENO5 values again, where some lane keeps one of them (a side it is not
    // eligible on): warp-uniform
    float2 h = make_float2(0.f, 0.f);
    if (__any_sync(0xffffffffu, bits != 3u)) {
      bool kx, ky;
      h = teno5_pz_sides(p, z[0], z[ZS], z[2 * ZS], z[3 * ZS], z[4 * ZS], kx, ky);
    }
#pragma unroll 1
    for (int sd = 0; sd < 2; sd++) {
      if ((sd ? by : bx) == 0u) continue;  // warp-uniform
      // this side's stencil upwind to downwind, re-read from shared memory (nothing of it stays
      // live across the network): f+ = z_0..z_4 .x, f- = z_4..z_0 .y
      const volatile float *f = reinterpret_cast<const volatile float *>(z) + sd;
      const int o = sd ? 8 * ZS : 0, st = sd ? -2 * ZS : 2 * ZS;
      float v[5];
#pragma unroll
      for (int k = 0; k < 5; k++) v[k] = f[o + k * st];
      float amp = 0.f;
#pragma unroll
      for (int k = 0; k < 5; k++) amp = fmaxf(amp, fabsf(v[k] - v[2]));
      const float inv = amp > 1e-30f ? __fdividef(1.f, amp) : 0.f;
      float x[5];
#pragma unroll
      for (int k = 0; k < 5; k++) x[k] = (v[k] - v[2]) * inv;
      float w[3];
      mlp::warp_weights2(img, x, w);
      if ((bits >> sd) & 1u) {
#pragma unroll
        for (int k = 0; k < 5; k++) v[k] = f[o + k * st];
        // delta form: constant stencils are reproduced exactly whatever the weights
        const Cands q = candidates(v[0], v[1], v[2], v[3], v[4]);
        const float hs = v[2] + w[0] * (q.q0 - v[2]) + w[1] * (q.q1 - v[2]) + w[2] * (q.q2 - v[2]);
        if (sd) h.y = hs;
        else h.x = hs;
      }
    }
    Fh[ps][c] = h.x + h.y;
  }
}

template <int SCHEME>
__device__ __forceinline__ float recon(const Plan &tw, float a, float b, float c, float d,
                                       float e) {
  if constexpr (SCHEME == IBFSA_TENO5) return teno5_fast(tw, a, b, c, d, e);
  else return weno5js(a, b, c, d, e);
}

// ------------------------------------------------------------------------------------------
// pad: q' = Q - q_inf (subtracted in FP64, then rounded to FP32), primitive perturbations,
// split speeds of the stage input
// ------------------------------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(THREADS) k_pad32(Plan p, const float *__restrict__ din) {
  constexpr int NV = DIM + 2;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float wmax[3] = {0.f, 0.f, 0.f};
  if (t < p.NP) {
    Free fs = free_stream(p);
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
    float q[NV];
    if (free_ghost) {
#pragma unroll
      for (int c = 0; c < NV; c++) q[c] = 0.f;
    } else {
      long long o = int_index(p, S[0], S[1], S[2]);
#pragma unroll
      for (int c = 0; c < NV; c++) q[c] = p.qn32[c * p.N + o] + (din ? din[c * p.N + o] : 0.f);
    }
#pragma unroll
    for (int c = 0; c < NV; c++) p.Qp32[c * p.NP + t] = q[c];
    float rho = fs.rho + q[0];
    float inv_rho = 1.f / rho;
    float ke2 = 0.f;  // m'.u + m_inf.u'
    float u[DIM];
#pragma unroll
    for (int a = 0; a < DIM; a++) {
      float up = (q[1 + a] - q[0] * fs.u[a]) * inv_rho;
      u[a] = fs.u[a] + up;
      ke2 += q[1 + a] * u[a] + fs.m[a] * up;
      p.Wp32[a * p.NP + t] = up;
    }
    float pp = fs.gm1 * (q[NV - 1] - 0.5f * ke2);
    p.Wp32[DIM * p.NP + t] = pp;
    if (interior) {
      float c = sqrtf(fs.gamma * (fs.p + pp) * inv_rho);
#pragma unroll
      for (int a = 0; a < DIM; a++) wmax[a] = fabsf(u[a]) + c;
    }
  }
  __shared__ float red[3][THREADS / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < DIM; a++) {
    float v = wmax[a];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[a][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < DIM) {
    float v = 0.f;
    for (int w = 0; w < THREADS / 32; w++) v = fmaxf(v, red[threadIdx.x][w]);
    if (!(v <= 1e30f)) atomicOr(p.status, IBFSA_STATUS_NONFINITE);
    else atomicMax(&p.alpha_bits[threadIdx.x], (unsigned long long)__double_as_longlong((double)v));
  }
}

// ------------------------------------------------------------------------------------------
// convective term along A: split flux perturbations of a tile of line segments in shared
// memory, faces of the tile (only those that exist), conservative difference into L
// ------------------------------------------------------------------------------------------
template <int A>
struct Tile {
  // A == 0: 8 lines (y) of 63 cells; otherwise 32 lines (consecutive x) of 15 cells -- two
  // faces per thread either way
  static constexpr int ROWS = A == 0 ? 8 : 32;
  static constexpr int SEG = A == 0 ? 63 : 15;
  static constexpr int LEN = SEG + 6;
  static constexpr int FACES = SEG + 1;
};

template <int DIM, int A>
constexpr size_t conv_smem() {
  return sizeof(float) * 2 * (DIM + 2) * Tile<A>::ROWS * Tile<A>::LEN;  // >= face-flux area
}

// split fluxes f+-' = (F' +- alpha q') / 2 along A of one staged cell, from q', u'_A and p';
// F' is the perturbation-expanded flux (no O(1) free-stream terms cancel)
template <int DIM, int A>
__device__ __forceinline__ void split_cell(const Free &fs, float alpha, const float q[DIM + 2],
                                           float up, float pp, float fpv[DIM + 2],
                                           float fmv[DIM + 2]) {
  constexpr int NV = DIM + 2;
  const float ua = fs.u[A] + up;
#pragma unroll
  for (int c = 0; c < NV; c++) {
    float F;
    if (c == 0) F = q[1 + A];
    else if (c == NV - 1) F = (q[c] + pp) * ua + fs.H * up;
    else {
      F = q[c] * ua + fs.m[c - 1] * up;
      if (c - 1 == A) F += pp;
    }
    const float aq = alpha * q[c];
    fpv[c] = 0.5f * (F + aq);
    fmv[c] = 0.5f * (F - aq);
  }
}

// Characteristic-wise option in the perturbation form: eigenvectors of the Euler flux Jacobian
// along A at the Roe average of the face's two cells, from their full primitive state
// (rho_inf + rho', u_inf + u', p_inf + p'), H = gamma p/((gamma - 1) rho) + |u|^2/2; right
// eigenvectors are the columns of R, left ones the rows of Lv, in the order u-c, entropy,
// shears, u+c.  The split-flux perturbations are projected on them: their constant free-stream
// part would pass through L and R unchanged and cancel in the face difference.
template <int DIM, int A>
__device__ __forceinline__ void roe_eigen32(const Free &fs, const float wl[DIM + 2],
                                            const float wr[DIM + 2], float R[DIM + 2][DIM + 2],
                                            float Lv[DIM + 2][DIM + 2]) {
  // w = [rho', u'_0 .. u'_{DIM-1}, p']
  constexpr int NV = DIM + 2;
  const float rl = fs.rho + wl[0], rr = fs.rho + wr[0];
  const float sl = sqrtf(rl), sr = sqrtf(rr), inv = 1.f / (sl + sr);
  const float kap = fs.gamma / fs.gm1;
  float u[DIM], kl = 0.f, kr = 0.f;
#pragma unroll
  for (int b = 0; b < DIM; b++) {
    float ul = fs.u[b] + wl[1 + b], ur = fs.u[b] + wr[1 + b];
    u[b] = (sl * ul + sr * ur) * inv;
    kl += ul * ul;
    kr += ur * ur;
  }
  const float Hl = kap * (fs.p + wl[NV - 1]) / rl + 0.5f * kl;
  const float Hr = kap * (fs.p + wr[NV - 1]) / rr + 0.5f * kr;
  const float H = (sl * Hl + sr * Hr) * inv;
  float q2 = 0.f;
#pragma unroll
  for (int b = 0; b < DIM; b++) q2 += u[b] * u[b];
  const float c2 = fs.gm1 * (H - 0.5f * q2);
  const float c = sqrtf(c2), ic = 1.f / c;
  const float b1 = fs.gm1 / c2, b2 = 0.5f * q2 * b1;
  const float ua = u[A];
#pragma unroll
  for (int i = 0; i < NV; i++)
#pragma unroll
    for (int j = 0; j < NV; j++) {
      R[i][j] = 0.f;
      Lv[i][j] = 0.f;
    }
  constexpr int km = 0, ke = 1, kp = NV - 1;
  R[0][km] = 1.f;
  R[0][ke] = 1.f;
  R[0][kp] = 1.f;
#pragma unroll
  for (int b = 0; b < DIM; b++) {
    R[1 + b][km] = u[b] - (b == A ? c : 0.f);
    R[1 + b][ke] = u[b];
    R[1 + b][kp] = u[b] + (b == A ? c : 0.f);
  }
  R[NV - 1][km] = H - ua * c;
  R[NV - 1][ke] = 0.5f * q2;
  R[NV - 1][kp] = H + ua * c;
  Lv[km][0] = 0.5f * (b2 + ua * ic);
  Lv[kp][0] = 0.5f * (b2 - ua * ic);
  Lv[ke][0] = 1.f - b2;
#pragma unroll
  for (int b = 0; b < DIM; b++) {
    Lv[km][1 + b] = 0.5f * (-b1 * u[b] - (b == A ? ic : 0.f));
    Lv[kp][1 + b] = 0.5f * (-b1 * u[b] + (b == A ? ic : 0.f));
    Lv[ke][1 + b] = b1 * u[b];
  }
  Lv[km][NV - 1] = 0.5f * b1;
  Lv[kp][NV - 1] = 0.5f * b1;
  Lv[ke][NV - 1] = -b1;
  int t = 0;
#pragma unroll
  for (int b = 0; b < DIM; b++) {
    if (b == A) continue;
    R[1 + b][2 + t] = 1.f;
    R[NV - 1][2 + t] = u[b];
    Lv[2 + t][0] = -u[b];
    Lv[2 + t][1 + b] = 1.f;
    t++;
  }
}

// eight blocks per SM (32 registers) for the fixed schemes, four (64 registers) for the
// learned form's warp-wide network tiles, one for the characteristic-wise option (its two
// eigen-systems per face take registers).  The x pass gives each warp one row of the tile.
template <int DIM, int A, int SCHEME, bool CHAR = false>
__global__ void __launch_bounds__(THREADS, SCHEME == IBFSA_MLP_TENO5 ? 4 : (CHAR ? 1 : 8))
    k_conv32(Plan p, int first) {
  constexpr int NV = DIM + 2;
  using T = Tile<A>;
  static_assert(A != 0 || T::ROWS * 32 == THREADS, "x pass: one warp per row");
  // face fluxes are stored with an odd row stride when a warp walks the rows (A != 0), so the
  // 32 lanes hit 32 different banks
  constexpr int FST = A == 0 ? T::FACES : T::FACES + 1;
  extern __shared__ float smf[];
  // component-wise TENO5 and the learned weights stage the interleaved face stencils
  // z_l = (f+ at l, f- at l+1), [NV][ROWS][LEN] float2 (teno5_pz_warp); the other schemes f+ and
  // f- apart, [NV][ROWS][LEN]
  constexpr bool ZL = (SCHEME == IBFSA_TENO5 || SCHEME == IBFSA_MLP_TENO5) && !CHAR;
  float *sfp = smf;
  float *sfm = smf + NV * T::ROWS * T::LEN;
  const float alpha = (float)__longlong_as_double((long long)p.alpha_bits[A]);
  Free fs = free_stream(p);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  int seg0, line0, other;
  if constexpr (A == 0) {
    seg0 = blockIdx.x * T::SEG;
    line0 = blockIdx.y * T::ROWS;
    other = blockIdx.z;
  } else {
    int nseg = (p.n[A] + T::SEG - 1) / T::SEG;
    seg0 = (blockIdx.x % nseg) * T::SEG;
    line0 = (blockIdx.x / nseg) * T::ROWS;
    other = blockIdx.y;
  }
  const int ncell = min(T::SEG, p.n[A] - seg0);   // cells of this tile along A
  const int nface = ncell + 1;
  const int nrow = A == 0 ? min(T::ROWS, p.n[1] - line0) : min(T::ROWS, p.n[0] - line0);
  // 32-bit offsets inside one component array: padded cell (row, l) and interior cell (row, l)
  const int PX = p.P[0], PXY = p.P[0] * p.P[1];
  const int NX = p.n[0], NXY = p.n[0] * p.n[1];
  int pbase, prs, pas, ibase, irs, ias;
  if constexpr (A == 0) {
    pbase = (other + p.g[2]) * PXY + (line0 + p.g[1]) * PX + (seg0 + p.g[0]);
    prs = PX; pas = 1;
    ibase = other * NXY + line0 * NX + seg0;
    irs = NX; ias = 1;
  } else {
    int y = A == 1 ? seg0 : other, z = A == 1 ? other : seg0;
    pbase = (z + p.g[2]) * PXY + (y + p.g[1]) * PX + (line0 + p.g[0]);
    prs = 1; pas = A == 1 ? PX : PXY;
    ibase = z * NXY + y * NX + line0;
    irs = 1; ias = A == 1 ? NX : NXY;
  }
  const float *Wa = p.Wp32 + (size_t)A * p.NP;
  const float *Wpr = p.Wp32 + (size_t)DIM * p.NP;

  if constexpr (SCHEME == IBFSA_MLP_TENO5) {
    mlp::stage_inference_image(reinterpret_cast<uint4 *>(smf + 2 * NV * T::ROWS * T::LEN),
                               reinterpret_cast<const uint4 *>(p.mlp_img), threadIdx.x, THREADS);
  }
  // 1. f+-' of the staged cells (seg0-3 .. seg0+ncell+2)
  constexpr int S1 = A == 0 ? (T::LEN + 31) / 32 : (T::ROWS * T::LEN + THREADS - 1) / THREADS;
#pragma unroll
  for (int k = 0; k < S1; k++) {
    int row, l;
    if constexpr (A == 0) {
      row = warp;
      l = lane + 32 * k;
      if (l >= T::LEN) break;
    } else {
      const int e = threadIdx.x + k * THREADS;
      if (e >= T::ROWS * T::LEN) break;
      row = e % T::ROWS;
      l = e / T::ROWS;
    }
    if (row >= nrow || l >= ncell + 6) continue;
    const int s = pbase + row * prs + (l - 3) * pas;
    float q[NV], fpv[NV], fmv[NV];
#pragma unroll
    for (int c = 0; c < NV; c++) q[c] = p.Qp32[(size_t)c * p.NP + s];
    split_cell<DIM, A>(fs, alpha, q, Wa[s], Wpr[s], fpv, fmv);
    if constexpr (ZL) {
#pragma unroll
      for (int c = 0; c < NV; c++) {
        float2 *zr = reinterpret_cast<float2 *>(smf) + (c * T::ROWS + row) * T::LEN;
        zr[l].x = fpv[c];
        if (l > 0) zr[l - 1].y = fmv[c];
      }
    } else {
#pragma unroll
      for (int c = 0; c < NV; c++) {
        sfp[(c * T::ROWS + row) * T::LEN + l] = fpv[c];
        sfm[(c * T::ROWS + row) * T::LEN + l] = fmv[c];
      }
    }
  }
  __syncthreads();

  // 2. faces m+1/2, m = seg0-1 .. seg0+ncell-1 (tile face index fi = m - seg0 + 1)
  constexpr int MAXP = (T::ROWS * T::FACES + THREADS - 1) / THREADS;
  float Fh[MAXP][NV];
  if constexpr (SCHEME == IBFSA_MLP_TENO5) {
    unsigned char *img = reinterpret_cast<unsigned char *>(smf + 2 * NV * T::ROWS * T::LEN);
    unsigned used = 0, seen = 0;
    const float2 *Z = reinterpret_cast<const float2 *>(smf);
    learned_faces<MAXP, NV, 1>(p, img, Fh, used, seen, [&](int ps, int c, bool &valid) {
      int e = threadIdx.x + ps * THREADS;
      int row, fi;
      if constexpr (A == 0) { row = e / T::FACES; fi = e % T::FACES; }
      else { row = e % T::ROWS; fi = e / T::ROWS; }
      valid = e < T::ROWS * T::FACES && row < nrow && fi < nface;
      if (!valid) { row = 0; fi = 0; }  // in-bounds reads; results discarded
      return Z + (c * T::ROWS + row) * T::LEN + fi;
    });
    used = __reduce_add_sync(0xffffffffu, used);  // warp totals
    seen = __reduce_add_sync(0xffffffffu, seen);
    if ((threadIdx.x & 31) == 0 && seen) {
      atomicAdd(&p.mlp_counts[0], (unsigned long long)used);
      atomicAdd(&p.mlp_counts[1], (unsigned long long)seen);
    }
  } else if constexpr (CHAR) {
    // characteristic-wise: per face the Roe-averaged eigen-system of cells m and m+1 (staged
    // cells fi + 2 and fi + 3), the stencils of each characteristic field, back-projection
#pragma unroll 1
    for (int ps = 0; ps < MAXP; ps++) {
      int e = threadIdx.x + ps * THREADS;
      int row, fi;
      if constexpr (A == 0) { row = e / T::FACES; fi = e % T::FACES; }
      else { row = e % T::ROWS; fi = e / T::ROWS; }
#pragma unroll
      for (int c = 0; c < NV; c++) Fh[ps][c] = 0.f;
      if (e < T::ROWS * T::FACES && row < nrow && fi < nface) {
        const int b = fi + 2;
        const int sl = pbase + row * prs + (b - 3) * pas, sr = sl + pas;
        float wl[NV], wr[NV];
        wl[0] = p.Qp32[sl];
        wr[0] = p.Qp32[sr];
#pragma unroll
        for (int k = 0; k <= DIM; k++) {
          wl[1 + k] = p.Wp32[(size_t)k * p.NP + sl];
          wr[1 + k] = p.Wp32[(size_t)k * p.NP + sr];
        }
        float Rm[NV][NV], Lv[NV][NV];
        roe_eigen32<DIM, A>(fs, wl, wr, Rm, Lv);
        float hk[NV];
#pragma unroll
        for (int k = 0; k < NV; k++) {
          float vp[5], vm[5];
#pragma unroll
          for (int r = 0; r < 5; r++) {
            float sp = 0.f, sn = 0.f;
#pragma unroll
            for (int c = 0; c < NV; c++) {
              sp = fmaf(Lv[k][c], sfp[(c * T::ROWS + row) * T::LEN + b - 2 + r], sp);
              sn = fmaf(Lv[k][c], sfm[(c * T::ROWS + row) * T::LEN + b + 3 - r], sn);
            }
            vp[r] = sp;
            vm[r] = sn;
          }
          hk[k] = recon<SCHEME>(p, vp[0], vp[1], vp[2], vp[3], vp[4]) +
                  recon<SCHEME>(p, vm[0], vm[1], vm[2], vm[3], vm[4]);
        }
#pragma unroll
        for (int c = 0; c < NV; c++) {
          float acc = 0.f;
#pragma unroll
          for (int k = 0; k < NV; k++) acc = fmaf(Rm[c][k], hk[k], acc);
          Fh[ps][c] = acc;
        }
      }
    }
  } else {
#pragma unroll
    for (int ps = 0; ps < MAXP; ps++) {
      int e = threadIdx.x + ps * THREADS;
      int row, fi;
      if constexpr (A == 0) { row = e / T::FACES; fi = e % T::FACES; }
      else { row = e % T::ROWS; fi = e / T::ROWS; }
      if constexpr (SCHEME == IBFSA_TENO5) {
        // every lane of the warp takes part (the slow path is warp-uniform): lanes without a
        // face evaluate a valid one of their row (or row 0) and store nothing
        const bool valid = e < T::ROWS * T::FACES && row < nrow && fi < nface;
        if (!valid) {
          fi = 0;
          if (row >= nrow) row = 0;
        }
        // face fi + 1/2 - 1 between staged cells fi + 2 and fi + 3: z_fi .. z_fi+4
#pragma unroll
        for (int c = 0; c < NV; c++) {
          const float2 *z = reinterpret_cast<const float2 *>(smf) + (c * T::ROWS + row) * T::LEN + fi;
          Fh[ps][c] = teno5_pz_warp(p, z[0], z[1], z[2], z[3], z[4]);
        }
      } else if (e < T::ROWS * T::FACES && row < nrow && fi < nface) {
        int b = fi + 2;
#pragma unroll
        for (int c = 0; c < NV; c++) {
          const float *fp = sfp + (c * T::ROWS + row) * T::LEN;
          const float *fm = sfm + (c * T::ROWS + row) * T::LEN;
          Fh[ps][c] = recon<SCHEME>(p, fp[b - 2], fp[b - 1], fp[b], fp[b + 1], fp[b + 2]) +
                      recon<SCHEME>(p, fm[b + 3], fm[b + 2], fm[b + 1], fm[b], fm[b - 1]);
        }
      }
    }
  }
  __syncthreads();
  float *sh = smf;
#pragma unroll
  for (int ps = 0; ps < MAXP; ps++) {
    int e = threadIdx.x + ps * THREADS;
    int row, fi;
    if constexpr (A == 0) { row = e / T::FACES; fi = e % T::FACES; }
    else { row = e % T::ROWS; fi = e / T::ROWS; }
    if (e < T::ROWS * T::FACES && row < nrow && fi < nface) {
#pragma unroll
      for (int c = 0; c < NV; c++) sh[(c * T::ROWS + row) * FST + fi] = Fh[ps][c];
    }
  }
  __syncthreads();

  // 3. L' = L' - (Fhat_{m+1/2} - Fhat_{m-1/2}) / (dx/dxi)
  constexpr int S3 = A == 0 ? (T::SEG + 31) / 32 : (T::ROWS * T::SEG + THREADS - 1) / THREADS;
#pragma unroll
  for (int k = 0; k < S3; k++) {
    int row, l;
    if constexpr (A == 0) {
      row = warp;
      l = lane + 32 * k;
      if (l >= T::SEG) break;
    } else {
      const int e = threadIdx.x + k * THREADS;
      if (e >= T::ROWS * T::SEG) break;
      row = e % T::ROWS;
      l = e / T::ROWS;
    }
    if (row >= nrow || l >= ncell) continue;
    int o = ibase + row * irs + l * ias;
    // the boundary cell of a characteristic face takes its normal term from k_char_face32
    const float inv_h = char_cell(p, A, seg0 + l) ? 0.f : mesh::inv32(p, A, seg0 + l);
#pragma unroll
    for (int c = 0; c < NV; c++) {
      const float *hh = sh + (c * T::ROWS + row) * FST;
      float d = (hh[l + 1] - hh[l]) * inv_h;
      float *Lc = p.L32 + (size_t)c * p.N;
      Lc[o] = (first ? 0.f : Lc[o]) - d;
    }
  }
}

// y and z passes of the fixed schemes with tensor copies (x extent a multiple of 4, so every
// stride of the copied tensors is a multiple of 16 bytes).  A tile is 32 consecutive x-lines by
// the staged cells along A; a warp covers the 32 lines of one position along A, so there is no
// index division and every shared-memory access of a warp falls in 32 banks.
//   shared memory: [ q' (NV) | u'_A | p' ] staged cells, [NV][LEN][32], reused for the block's
//   L' [NV][SEG][32] once the split fluxes are built; f+ at staged cells 0..LEN-2 and f- at
//   1..LEN-1 (the only ones the faces read), [NV][LEN-1][32] each, reused for the face fluxes;
//   one barrier.  44 KB in 3D: five blocks per SM.
// One thread issues the copies: the staged inputs (three copies) at entry, the block's L' after
// the split fluxes (its latency hides behind the reconstruction); L' is updated in shared
// memory and written back with a tensor store.  Waits are bounded: on expiry the block reports
// IBFSA_STATUS_TIMEOUT and ends.
template <int DIM, int A>
struct TmaTile {
  using T = Tile<A>;
  static constexpr int NV = DIM + 2, R = T::ROWS, LEN = T::LEN, SEG = T::SEG;
  static constexpr int IN = (NV + 2) * LEN * R;     // floats of the staged inputs
  static constexpr int LT = NV * SEG * R;           // floats of the L' tile
  static constexpr int SF = NV * (LEN - 1) * R;     // floats of f+ (and of f-)
  static constexpr size_t BYTES = sizeof(float) * (IN + 2 * SF) + 16;
  static_assert(LT <= IN, "the L' tile reuses the staged inputs");
  static_assert(R == 32, "one warp spans the x-lines of a tile");
};

// Wait (bounded) for phase `parity` of the block's barrier; every thread of the block calls it.
// On expiry the block reports IBFSA_STATUS_TIMEOUT, thread 0 waits once more (bounded) for
// copies still in flight, and the function returns false: the caller then returns.
__device__ __forceinline__ bool block_wait_or_report(const Plan &p, uint64_t *bar,
                                                     uint32_t parity) {
  if (__syncthreads_or(!tma::mbar_wait(bar, parity))) {
    if (threadIdx.x == 0) {
      atomicOr(p.status, IBFSA_STATUS_TIMEOUT);
      tma::mbar_wait(bar, parity);
    }
    return false;
  }
  return true;
}

template <int DIM, int A, int SCHEME>
__global__ void __launch_bounds__(THREADS, SCHEME == IBFSA_MLP_TENO5 ? 4 : 5)
    k_conv32_tma(Plan p, const __grid_constant__ CUtensorMap tq,
                 const __grid_constant__ CUtensorMap tw, const __grid_constant__ CUtensorMap tl) {
  using TT = TmaTile<DIM, A>;
  using T = Tile<A>;
  constexpr int NV = TT::NV, R = TT::R, LEN = TT::LEN, SEG = TT::SEG;
  constexpr int FST = T::FACES + 1;
  // TENO5 and the learned weights stage interleaved face stencils z_l = (f+ at l, f- at l+1)
  constexpr bool ZL = SCHEME == IBFSA_TENO5 || SCHEME == IBFSA_MLP_TENO5;
  extern __shared__ __align__(128) float smf[];
  float *in = smf;                         // [NV + 2][LEN][R], then L' [NV][SEG][R]
  float *sfp = smf + TT::IN;               // [NV][LEN - 1][R]: f+ at staged cells 0..LEN-2
  float *sfm = sfp + TT::SF;               // [NV][LEN - 1][R]: f- at staged cells 1..LEN-1
  uint64_t *bar = reinterpret_cast<uint64_t *>(sfm + TT::SF);
  // the learned weights' parameter image follows the barrier (16-byte aligned)
  unsigned char *img = reinterpret_cast<unsigned char *>(bar) + 16;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = THREADS / 32;
  static_assert((sizeof(float) * (TT::IN + 2 * TT::SF) + 16) % 16 == 0, "image alignment");

  const int nseg = (p.n[A] + SEG - 1) / SEG;
  const int seg0 = (blockIdx.x % nseg) * SEG;
  const int line0 = (blockIdx.x / nseg) * R;
  const int other = blockIdx.y;
  const int ncell = min(SEG, p.n[A] - seg0);
  const int nface = ncell + 1;
  const bool row_ok = lane < min(R, p.n[0] - line0);
  const int yi = A == 1 ? seg0 : other, zi = A == 1 ? other : seg0;  // first owned cell

  if (threadIdx.x == 0) tma::mbar_init(bar, 1);
  if constexpr (SCHEME == IBFSA_MLP_TENO5)
    mlp::stage_inference_image(reinterpret_cast<uint4 *>(img),
                               reinterpret_cast<const uint4 *>(p.mlp_img), threadIdx.x, THREADS);
  __syncthreads();
  if (threadIdx.x == 0) {
    tma::mbar_expect_tx(bar, (uint32_t)(sizeof(float) * TT::IN));
    const int px = line0 + p.g[0];
    const int py = (A == 1 ? yi - 3 : yi) + p.g[1], pz = (A == 2 ? zi - 3 : zi) + p.g[2];
    tma::load_4d(in, &tq, px, py, pz, 0, bar);
    tma::load_4d(in + NV * LEN * R, &tw, px, py, pz, A, bar);
    tma::load_4d(in + (NV + 1) * LEN * R, &tw, px, py, pz, DIM, bar);
  }
  if (!block_wait_or_report(p, bar, 0)) return;

  // 1. f+-' of the staged cells l = 0 .. ncell+5 (cells seg0-3 .. seg0+ncell+2)
  const float alpha = (float)__longlong_as_double((long long)p.alpha_bits[A]);
  {
    Free fs = free_stream(p);
    for (int l = warp; l < ncell + 6; l += NW) {
      float q[NV], fpv[NV], fmv[NV];
#pragma unroll
      for (int c = 0; c < NV; c++) q[c] = in[(c * LEN + l) * R + lane];
      split_cell<DIM, A>(fs, alpha, q, in[(NV * LEN + l) * R + lane],
                         in[((NV + 1) * LEN + l) * R + lane], fpv, fmv);
      if constexpr (ZL) {
        // interleaved face stencils z_l = (f+ at l, f- at l+1), [NV][LEN-1][R] float2
        float2 *Z = reinterpret_cast<float2 *>(sfp);
#pragma unroll
        for (int c = 0; c < NV; c++) {
          if (l < LEN - 1) Z[(c * (LEN - 1) + l) * R + lane].x = fpv[c];
          if (l > 0) Z[(c * (LEN - 1) + l - 1) * R + lane].y = fmv[c];
        }
      } else {
#pragma unroll
        for (int c = 0; c < NV; c++) {
          if (l < LEN - 1) sfp[(c * (LEN - 1) + l) * R + lane] = fpv[c];
          if (l > 0) sfm[(c * (LEN - 1) + l - 1) * R + lane] = fmv[c];
        }
      }
    }
  }
  __syncthreads();
  // the staged inputs are consumed: the block's L' comes into their place
  if (threadIdx.x == 0) {
    tma::mbar_expect_tx(bar, (uint32_t)(sizeof(float) * TT::LT));
    tma::load_4d(in, &tl, line0, yi, zi, 0, bar);
  }

  // 2. faces fi = warp, warp + NW (face m+1/2 with m = seg0-1+fi): f+ at staged cells
  //    fi .. fi+4, f- at fi+1 .. fi+5
  constexpr int MAXP = (T::FACES + NW - 1) / NW;
  float Fh[MAXP][NV];
  if constexpr (SCHEME == IBFSA_MLP_TENO5) {
    const float2 *Z = reinterpret_cast<const float2 *>(sfp);
    unsigned used = 0, seen = 0;
    learned_faces<MAXP, NV, R>(p, img, Fh, used, seen, [&](int ps, int c, bool &valid) {
      int fi = warp + ps * NW;
      valid = fi < nface && row_ok;
      if (fi >= nface) fi = 0;  // in-bounds reads; results discarded
      return Z + (c * (LEN - 1) + fi) * R + lane;
    });
    used = __reduce_add_sync(0xffffffffu, used);  // warp totals
    seen = __reduce_add_sync(0xffffffffu, seen);
    if (lane == 0 && seen) {
      atomicAdd(&p.mlp_counts[0], (unsigned long long)used);
      atomicAdd(&p.mlp_counts[1], (unsigned long long)seen);
    }
  } else {
#pragma unroll
  for (int ps = 0; ps < MAXP; ps++) {
    const int fi = warp + ps * NW;
    if (fi < nface) {
#pragma unroll
      for (int c = 0; c < NV; c++) {
        if constexpr (SCHEME == IBFSA_TENO5) {  // fi is the same for the whole warp
          const float2 *z = reinterpret_cast<const float2 *>(sfp) + (c * (LEN - 1) + fi) * R + lane;
          Fh[ps][c] = teno5_pz_warp(p, z[0], z[R], z[2 * R], z[3 * R], z[4 * R]);
        } else {
          const float *fp = sfp + (c * (LEN - 1) + fi) * R + lane;
          const float *fm = sfm + (c * (LEN - 1) + fi) * R + lane;   // f- of staged cell fi+1
          Fh[ps][c] = recon<SCHEME>(p, fp[0], fp[R], fp[2 * R], fp[3 * R], fp[4 * R]) +
                      recon<SCHEME>(p, fm[4 * R], fm[3 * R], fm[2 * R], fm[R], fm[0]);
        }
      }
    }
  }
  }
  __syncthreads();
  float *sh = sfp;  // face fluxes [NV][R][FST]
#pragma unroll
  for (int ps = 0; ps < MAXP; ps++) {
    const int fi = warp + ps * NW;
    if (fi < nface) {
#pragma unroll
      for (int c = 0; c < NV; c++) sh[(c * R + lane) * FST + fi] = Fh[ps][c];
    }
  }
  __syncthreads();
  if (!block_wait_or_report(p, bar, 1)) return;

  // 3. L' = L' - (Fhat_{m+1/2} - Fhat_{m-1/2}) / (dx/dxi) on the copied tile, then stored back
  if (row_ok) {
    for (int l = warp; l < ncell; l += NW) {
      const float inv_h = char_cell(p, A, seg0 + l) ? 0.f : mesh::inv32(p, A, seg0 + l);
#pragma unroll
      for (int c = 0; c < NV; c++) {
        const float *hh = sh + (c * R + lane) * FST;
        in[(c * SEG + l) * R + lane] -= (hh[l + 1] - hh[l]) * inv_h;
      }
    }
  }
  tma::fence_async_shared();
  __syncthreads();
  if (threadIdx.x == 0) tma::store_4d(&tl, line0, yi, zi, 0, in);
}

// ------------------------------------------------------------------------------------------
// characteristic non-reflecting faces (Sec. 2, after Thompson) on the perturbations: the
// one-sided derivatives of rho', u', p' are those of rho, u, p; the wave speeds and the map
// back to the conservative variables use the full state
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float one_sided32(const float *phi, long long o, long long st, int s,
                                             float inv12) {
  const float f0 = phi[o];
  float acc = 48.f * (phi[o + s * st] - f0);
  acc = fmaf(-36.f, phi[o + 2 * s * st] - f0, acc);
  acc = fmaf(16.f, phi[o + 3 * s * st] - f0, acc);
  acc = fmaf(-3.f, phi[o + 4 * s * st] - f0, acc);
  return (float)s * acc * inv12;
}

template <int DIM>
__global__ void k_char_face32(Plan p, int a, int side) {
  constexpr int NV = DIM + 2;
  const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)p.n[b1] * p.n[b2]) return;
  int I[3];
  I[a] = side == 0 ? 0 : p.n[a] - 1;
  I[b1] = (int)(t % p.n[b1]);
  I[b2] = (int)(t / p.n[b1]);
  const int s = side == 0 ? 1 : -1;
  const Free fs = free_stream(p);
  const long long o = pad_index(p, I[0], I[1], I[2]);
  const long long st = a == 0 ? 1 : a == 1 ? (long long)p.P[0] : (long long)p.P[0] * p.P[1];
  const float inv12 = mesh::inv12_32(p, a, I[a]);
  const float r = fs.rho + p.Qp32[o], pr = fs.p + p.Wp32[DIM * p.NP + o];
  const float c = sqrtf(fs.gamma * pr / r);
  const float ua = fs.u[a] + p.Wp32[a * p.NP + o];
  const float rx = one_sided32(p.Qp32, o, st, s, inv12);
  const float px = one_sided32(p.Wp32 + DIM * p.NP, o, st, s, inv12);
  const float uxa = one_sided32(p.Wp32 + a * p.NP, o, st, s, inv12);
  const float lam1 = ua - c, lam2 = ua, lam5 = ua + c, rc = r * c;
  const float L1 = (lam1 * (float)s > 0.f) ? 0.f : lam1 * (px - rc * uxa);
  const float L2 = (lam2 * (float)s > 0.f) ? 0.f : lam2 * (c * c * rx - px);
  const float L5 = (lam5 * (float)s > 0.f) ? 0.f : lam5 * (px + rc * uxa);
  float dv[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int b = 0; b < DIM; b++) {
    if (b == a) continue;
    float utx = one_sided32(p.Wp32 + b * p.NP, o, st, s, inv12);
    dv[b] = (lam2 * (float)s > 0.f) ? 0.f : lam2 * utx;
  }
  const float d1 = (L2 + 0.5f * (L5 + L1)) / (c * c);
  const float d2 = 0.5f * (L5 + L1);
  dv[a] = (L5 - L1) / (2.f * rc);
  float D[NV];
  float ke = 0.f, work = 0.f;
  D[0] = d1;
#pragma unroll
  for (int b = 0; b < DIM; b++) {
    float ub = fs.u[b] + p.Wp32[b * p.NP + o];
    D[1 + b] = ub * d1 + r * dv[b];
    ke += ub * ub;
    work += ub * dv[b];
  }
  D[NV - 1] = 0.5f * ke * d1 + d2 / fs.gm1 + r * work;
  const long long oi = int_index(p, I[0], I[1], I[2]);
#pragma unroll
  for (int c2 = 0; c2 < NV; c2++) p.L32[c2 * p.N + oi] -= D[c2];
}

// ------------------------------------------------------------------------------------------
// viscous term on the velocity perturbations
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float d4f(float fm2, float fm1, float fp1, float fp2, float inv_h12) {
  return (8.f * (fp1 - fm1) - (fp2 - fm2)) * inv_h12;
}

template <int DIM>
__global__ void __launch_bounds__(THREADS) k_visc_flux32(Plan p) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.NB) return;
  Free fs = free_stream(p);
  int bx = (int)(t % p.B[0]);
  long long r = t / p.B[0];
  int by = (int)(r % p.B[1]);
  int bz = (int)(r / p.B[1]);
  int I[3] = {bx - 2, DIM > 1 ? by - 2 : by, DIM > 2 ? bz - 2 : bz};
  long long s = pad_index(p, I[0], I[1], I[2]);
  long long stride[3] = {1, p.P[0], (long long)p.P[0] * p.P[1]};
  float g[DIM][DIM];
#pragma unroll
  for (int ci = 0; ci < DIM; ci++) {
    const float *u = p.Wp32 + ci * p.NP + s;
#pragma unroll
    for (int dj = 0; dj < DIM; dj++) {
      long long st = stride[dj];
      g[ci][dj] = d4f(u[-2 * st], u[-st], u[st], u[2 * st], mesh::inv12_32(p, dj, I[dj]));
    }
  }
  float div = 0.f;
#pragma unroll
  for (int a = 0; a < DIM; a++) div += g[a][a];
#pragma unroll
  for (int a = 0; a < DIM; a++) {
    float b = 0.f;
#pragma unroll
    for (int ci = 0; ci < DIM; ci++) {
      float tau = g[ci][a] + g[a][ci];
      if (ci == a) tau -= (2.f / 3.f) * div;
      p.V32[(long long)(a * (DIM + 1) + ci) * p.NB + t] = tau;
      b += (fs.u[ci] + p.Wp32[ci * p.NP + s]) * tau;
    }
    p.V32[(long long)(a * (DIM + 1) + DIM) * p.NB + t] = b;
  }
}

// ------------------------------------------------------------------------------------------
// immersed boundary in FP64 from the FP64 stage state
// ------------------------------------------------------------------------------------------
// FP64 value of component c of the stage state at interior cell o: Qn + increment
__device__ __forceinline__ double stage_q(const Plan &p, const double *__restrict__ Qn,
                                          const float *__restrict__ din, int c, long long o) {
  double v = Qn[c * p.N + o];
  return din ? v + (double)din[c * p.N + o] : v;
}

template <int DIM>
__global__ void k_ib_interp64(Plan p, const double *__restrict__ Qn, const float *__restrict__ din,
                              const double *__restrict__ xis, const double *xin, double *xio,
                              double A, double Bc, double dt, int advance) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int nm = p.nm, M = p.max_markers;
  if (k >= nm) return;
  int j0[3];
  double w[3][4];
  if (!point_support<DIM>(p, p.X, M, k, j0, w)) {
    atomicOr(p.status, IBFSA_STATUS_BOUNDS);
    for (int a = 0; a < DIM; a++) {
      p.F[a * M + k] = 0.0;
      if (advance) xio[a * M + k] = xin[a * M + k];
    }
    return;
  }
  constexpr int C2 = DIM > 2 ? 4 : 1;
  double acc[DIM];
#pragma unroll
  for (int a = 0; a < DIM; a++) acc[a] = 0.0;
  for (int r2 = 0; r2 < C2; r2++)
    for (int r1 = 0; r1 < 4; r1++)
      for (int r0 = 0; r0 < 4; r0++) {
        long long o = int_index(p, j0[0] + r0, j0[1] + r1, j0[2] + r2);
        double wt = w[0][r0] * w[1][r1] * w[2][r2];
        double inv_rho = 1.0 / stage_q(p, Qn, din, 0, o);
#pragma unroll
        for (int a = 0; a < DIM; a++) acc[a] += stage_q(p, Qn, din, 1 + a, o) * inv_rho * wt;
      }
#pragma unroll
  for (int a = 0; a < DIM; a++) {
    double slip = acc[a] - p.U[a * M + k];
    p.F[a * M + k] = p.alpha_pen * xis[a * M + k] + p.beta_pen * slip;
    if (advance) xio[a * M + k] = A * xin[a * M + k] + Bc * (xis[a * M + k] + dt * slip);
  }
}

// Spreading (Eq. 9) into the FP32 right-hand side: one group of S = 4^DIM threads per marker,
// one thread per support cell.  The marker's 4 DIM kernel weights (FP64, Eq. 11) are evaluated
// once, by the first 4 DIM threads of its group, and shared; the per-cell force, the fluid
// velocity of the power term f.u and the atomic additions are FP32, the precision of the
// right-hand side they enter.
template <int DIM>
__global__ void __launch_bounds__(128) k_spread32(Plan p, const double *__restrict__ Qn,
                                                  const float *__restrict__ din) {
  constexpr int S = DIM > 2 ? 64 : 16, MPB = 128 / S;
  __shared__ double sw[MPB][3][4];
  __shared__ int sj[MPB][3];
  __shared__ float sf[MPB][3];
  __shared__ int sok[MPB];
  const int lm = threadIdx.x / S, r = threadIdx.x % S;
  const int k = blockIdx.x * MPB + lm;
  const int M = p.max_markers;
  const bool live = k < p.nm;
  const bool stretched = p.mx[0] || p.mx[1] || p.mx[2];
  if (live && r < 4 * DIM && !stretched) {
    int a = r / 4, q = r % 4;
    double s = (p.X[a * M + k] - p.lo[a]) * p.inv_h[a] - 0.5;
    int j0 = (int)floor(s) - 1;
    sw[lm][a][q] = peskin(s - (double)(j0 + q));
    if (q == 0) sj[lm][a] = j0;
  }
  if (live && r == 0) {
    bool ok = true;
    double hprod = p.hprod;
    if (stretched) {  // one thread finds the marker's supports and its local spacings
      int j0[3];
      double w[3][4];
      ok = point_support<DIM>(p, p.X, M, k, j0, w, &hprod);
#pragma unroll
      for (int a = 0; a < DIM; a++) {
        sj[lm][a] = j0[a];
#pragma unroll
        for (int q = 0; q < 4; q++) sw[lm][a][q] = w[a][q];
      }
    } else {
#pragma unroll
      for (int a = 0; a < DIM; a++) {
        double s = (p.X[a * M + k] - p.lo[a]) * p.inv_h[a] - 0.5;
        int j0 = (int)floor(s) - 1;
        if (j0 < 0 || j0 + 3 > p.n[a] - 1) ok = false;
      }
    }
    sok[lm] = ok;
    double sc = p.dS[k] / hprod;
#pragma unroll
    for (int a = 0; a < 3; a++) sf[lm][a] = a < DIM ? (float)(-p.F[a * M + k] * sc) : 0.f;
    if (DIM < 3) {
      sw[lm][2][0] = 1.0;
      sw[lm][2][1] = sw[lm][2][2] = sw[lm][2][3] = 0.0;
      sj[lm][2] = 0;
    }
  }
  __syncthreads();
  if (!live || !sok[lm]) return;  // the interpolation kernel reports markers off the grid
  int r0 = r & 3, r1 = (r >> 2) & 3, r2 = DIM > 2 ? (r >> 4) : 0;
  float wt = (float)(sw[lm][0][r0] * sw[lm][1][r1] * sw[lm][2][r2]);
  long long o = int_index(p, sj[lm][0] + r0, sj[lm][1] + r1, sj[lm][2] + r2);
  Free fs = free_stream(p);
  float d0 = p.qn32[o] + (din ? din[o] : 0.f);
  float inv_rho = 1.f / (fs.rho + d0);
  float pw = 0.f;
#pragma unroll
  for (int a = 0; a < DIM; a++) {
    float da = p.qn32[(1 + a) * p.N + o] + (din ? din[(1 + a) * p.N + o] : 0.f);
    float fa = sf[lm][a] * wt;
    atomicAdd(&p.L32[(1 + a) * p.N + o], fa);
    pw += fa * ((fs.m[a] + da) * inv_rho);
  }
  atomicAdd(&p.L32[(DIM + 1) * p.N + o], pw);
}

// ------------------------------------------------------------------------------------------
// finish: sponge on the FP32 right-hand side, then
//   mode 0: L out (FP64 copy);  mode 1: dout = b (din + dt L);
//   mode 2: Qn += b (din + dt L) in FP64 and qn32 = (float)(Qn - q_inf)
// ------------------------------------------------------------------------------------------
// periodic Gaussian pressure source (Sec. 3.6, Eq. 16) of cell (i, j, k): energy-equation term
template <bool STRETCHED = true>
__device__ __forceinline__ float pressure_source32(const Plan &p, int dim, int i, int j, int k) {
  const int I[3] = {i, j, k};
  float r2 = 0.f;
  for (int a = 0; a < dim; a++) {
    double x = STRETCHED ? mesh::node(p, a, I[a]) : p.lo[a] + ((double)I[a] + 0.5) * p.h[a];
    float dx = (float)(x - p.src_xc[a]);
    r2 += dx * dx;
  }
  return expf(-(float)(p.src_b * 0.693147180559945309417) * r2) * (float)p.src_scale;
}

template <int DIM, bool VISC>
__global__ void __launch_bounds__(THREADS) k_finish32(Plan p, const float *__restrict__ din,
                                                      float *__restrict__ dout, double *Qn,
                                                      double *__restrict__ Lout, float Bc,
                                                      float dt, int mode) {
  constexpr int NV = DIM + 2;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.N) return;
  float Lc[NV];
#pragma unroll
  for (int c = 0; c < NV; c++) Lc[c] = p.L32[c * p.N + t];
  if constexpr (VISC) {
    // viscous divergence (1/Re) sum_a D4_a [0, tau_{.a}, b_a], fused here to save a pass over L
    int i = (int)(t % p.n[0]);
    long long r = t / p.n[0];
    int j = (int)(r % p.n[1]);
    int k = (int)(r / p.n[1]);
    long long bb = ((long long)(DIM > 2 ? k + 2 : k) * p.B[1] + (DIM > 1 ? j + 2 : j)) * p.B[0] + (i + 2);
    long long stride[3] = {1, p.B[0], (long long)p.B[0] * p.B[1]};
#pragma unroll
    for (int fc = 0; fc <= DIM; fc++) {
      float sum = 0.f;
#pragma unroll
      for (int a = 0; a < DIM; a++) {
        const float *F = p.V32 + (long long)(a * (DIM + 1) + fc) * p.NB + bb;
        long long st = stride[a];
        sum += d4f(F[-2 * st], F[-st], F[st], F[2 * st],
                   mesh::inv12_32(p, a, a == 0 ? i : a == 1 ? j : k));
      }
      Lc[fc + 1] += sum * p.inv_Re32;
    }
  }
  if (p.sponge_cells > 0) {
    int I[3];
    I[0] = (int)(t % p.n[0]);
    long long r = t / p.n[0];
    I[1] = (int)(r % p.n[1]);
    I[2] = (int)(r / p.n[1]);
    int S = p.sponge_cells, nmin = 1 << 30;
#pragma unroll
    for (int a = 0; a < DIM; a++) nmin = min(nmin, min(I[a], p.n[a] - 1 - I[a]));
    if (nmin < S) {
      float rr = (float)(S - nmin) / (float)S;
      float sig = (float)p.sponge_sigma * rr * rr * rr;
#pragma unroll
      for (int c = 0; c < NV; c++) {
        float qp = p.qn32[c * p.N + t] + (din ? din[c * p.N + t] : 0.f);
        Lc[c] -= sig * qp;
      }
    }
  }
  if (p.src_on) {
    int i = (int)(t % p.n[0]);
    long long r = t / p.n[0];
    Lc[NV - 1] += pressure_source32(p, DIM, i, (int)(r % p.n[1]), (int)(r / p.n[1]));
  }
  if (mode == 0) {
#pragma unroll
    for (int c = 0; c < NV; c++) Lout[c * p.N + t] = (double)Lc[c];
    return;
  }
  bool bad = false;
  float inc[NV];
#pragma unroll
  for (int c = 0; c < NV; c++) {
    inc[c] = Bc * ((din ? din[c * p.N + t] : 0.f) + dt * Lc[c]);
    bad |= !isfinite(inc[c]);
  }
  if (mode == 1) {
#pragma unroll
    for (int c = 0; c < NV; c++) dout[c * p.N + t] = inc[c];
  } else {
#pragma unroll
    for (int c = 0; c < NV; c++) {
      double q = Qn[c * p.N + t] + (double)inc[c];
      Qn[c * p.N + t] = q;
      p.qn32[c * p.N + t] = (float)(q - p.qinf[c]);
    }
  }
  if (bad) atomicOr(p.status, IBFSA_STATUS_NONFINITE);
}

// 3D viscous term + finish, marching along z.  A 32 x 8 block of threads owns 32 x 8 columns
// and walks a z-chunk: velocity perturbations of five planes (x, y halo 4) sit in a shared-
// memory ring, refilled from registers loaded one plane ahead; at each plane c the 9 gradients
// are evaluated at the block's cells and at the x/y halo points the x/y divergence needs,
// giving F_v,x and F_v,y (shared memory, divergence taken at once) and F_v,z, whose
// z-differences are accumulated per thread into the cells c-2 .. c+2 of its column; cell c-2
// is then complete: L += (1/Re) sum_a D4_a F_v,a, sponge, RK update.
#ifndef VM_MIN_BLOCKS
#define VM_MIN_BLOCKS 4
#endif
namespace vm {
constexpr int TX = 32, TY = 8, ZC = 64;        // block columns, z-chunk
constexpr int VT = TX * TY;                    // threads (one column each)
constexpr int SX = TX + 8, SY = TY + 8;        // staged plane (halo 4)
constexpr int PX = TX + 4, PY = TY + 4;        // flux points (halo 2)
constexpr size_t SMEM = sizeof(float) * (5 * 3 * SX * SY + 4 * PX * TY + 4 * TX * PY);
}  // namespace vm

// STRETCHED: some direction has a non-uniform mesh (per-point metrics); otherwise the uniform
// 1/(12 h) constants, with no per-point lookups
template <bool STRETCHED>
__global__ void __launch_bounds__(vm::VT, VM_MIN_BLOCKS) k_visc_march32(Plan p, const float *__restrict__ din,
                                                          float *__restrict__ dout, double *Qn,
                                                          double *__restrict__ Lout, float Bc,
                                                          float dt, int mode) {
  using namespace vm;
  extern __shared__ float smm[];
  float *ring = smm;                              // [5][3][SY][SX]
  float *fx = smm + 5 * 3 * SX * SY;              // F_v,x at [TY][PX], 4 components
  float *fy = fx + 4 * PX * TY;                   // F_v,y at [PY][TX], 4 components
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, zs = blockIdx.z * ZC;
  const int ze = min(zs + ZC, p.n[2]);
  const int X = x0 + tx, Y = y0 + ty;
  const bool own = X < p.n[0] && Y < p.n[1];
  Free fs = free_stream(p);
  const float ih[3] = {p.inv_h12_32[0], p.inv_h12_32[1], p.inv_h12_32[2]};
  const int PLANE = 3 * SX * SY;

  // plane z (ghost range -4 .. n+3) is read into registers one iteration before it enters
  // ring slot z mod 5, so its global-memory latency hides behind the gradients of a plane.
  // Per thread, the staged points it loads and their padded offsets within a plane are fixed:
  // computed once.
  constexpr int PER = (SX * SY + VT - 1) / VT;
  const int PXY = p.P[0] * p.P[1];
  const float *W0 = p.Wp32, *W1 = p.Wp32 + p.NP, *W2 = p.Wp32 + 2 * p.NP;
  int foff[PER];
#pragma unroll
  for (int j = 0; j < PER; j++) {
    int e = threadIdx.x + j * VT;
    int sx = e % SX, sy = e / SX;
    int gx = min(x0 - 4 + sx, p.n[0] + 3), gy = min(y0 - 4 + sy, p.n[1] + 3);
    foff[j] = (gy + p.g[1]) * p.P[0] + (gx + p.g[0]);
  }
  float R[PER][3];
  auto fetch = [&](int z) {
    const int zo = (z + p.g[2]) * PXY;
#pragma unroll
    for (int j = 0; j < PER; j++) {
      if (threadIdx.x + j * VT < SX * SY) {
        const int o = zo + foff[j];
        R[j][0] = W0[o];
        R[j][1] = W1[o];
        R[j][2] = W2[o];
      }
    }
  };
  auto put = [&](int slot) {
    float *dst = ring + slot * PLANE + threadIdx.x;
#pragma unroll
    for (int j = 0; j < PER; j++) {
      if (threadIdx.x + j * VT < SX * SY) {
#pragma unroll
        for (int c = 0; c < 3; c++) dst[c * SX * SY + j * VT] = R[j][c];
      }
    }
  };
  // 1/(12 dx/dxi) of node i along a (the plan's 1/(12 h) on a uniform direction); indices of
  // staged points beyond the box (their results are never used) are clamped into it
  auto ihat = [&](int a, int i) -> float {
    if constexpr (STRETCHED)
      return p.minv12_32[a] ? p.minv12_32[a][mesh::clamp_node(p, a, i) + NG] : ih[a];
    else
      return ih[a];
  };
  // gradients g[i][j] = du_i/dx_j at staged position (sx, sy) = offset e of plane c (ihx, ihy,
  // ihz: the metrics there)
  auto grads = [&](const float *const pl[5], int e, float ihx, float ihy, float ihz,
                   float g[3][3], float u[3]) {
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const float *m = pl[2] + i * SX * SY + e;
      u[i] = m[0];
      g[i][0] = d4f(m[-2], m[-1], m[1], m[2], ihx);
      g[i][1] = d4f(m[-2 * SX], m[-SX], m[SX], m[2 * SX], ihy);
      g[i][2] = d4f(pl[0][i * SX * SY + e], pl[1][i * SX * SY + e], pl[3][i * SX * SY + e],
                    pl[4][i * SX * SY + e], ihz);
    }
  };
  // viscous flux of direction a: [tau_0a, tau_1a, tau_2a, b_a]
  auto vflux = [&](int a, const float g[3][3], const float u[3], float f[4]) {
    float div = g[0][0] + g[1][1] + g[2][2];
    float b = 0.f;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      float tau = g[i][a] + g[a][i];
      if (i == a) tau -= (2.f / 3.f) * div;
      f[i] = tau;
      b += (fs.u[i] + u[i]) * tau;
    }
    f[3] = b;
  };

  // divergence of the viscous flux of this column's cells c-2 .. c+2, accumulated as the
  // fluxes arrive: F_v,z of plane c enters the z-differences of cells c-2, c-1, c+1, c+2
  // (weights -1, 8, -8, 1 over 12 dx/dxi of that cell), the x/y divergence of plane c enters
  // cell c
  float acc[5][4];
#pragma unroll
  for (int o = 0; o < 5; o++)
#pragma unroll
    for (int k = 0; k < 4; k++) acc[o][k] = 0.f;
  const float ihx_own = ihat(0, X), ihy_own = ihat(1, Y);
  // the halo point this thread evaluates each plane (threads below 4 TY + 4 TX): F_v,x at x
  // offsets -2, -1, TX, TX+1 of a row, or F_v,y at y offsets -2, -1, TY, TY+1 of a column; its
  // staged offset, its metrics and where its flux goes, fixed for the whole march
  const int hkind = threadIdx.x < 4 * TY ? 1 : (threadIdx.x < 4 * TY + 4 * TX ? 2 : 0);
  int he = 0, hout = 0;
  float hihx = ih[0], hihy = ih[1];
  if (hkind == 1) {
    int r = threadIdx.x / 4, h = threadIdx.x % 4, px = h < 2 ? h : TX + h;  // 0,1,TX+2,TX+3
    he = (r + 4) * SX + px + 2;
    hout = r * PX + px;
    hihx = ihat(0, x0 - 4 + px + 2);
    hihy = ihat(1, y0 + r);
  } else if (hkind == 2) {
    int e2 = threadIdx.x - 4 * TY, col = e2 % TX, h = e2 / TX, py = h < 2 ? h : TY + h;
    he = (py + 2) * SX + col + 4;
    hout = py * TX + col;
    hihx = ihat(0, x0 + col);
    hihy = ihat(1, y0 - 4 + py + 2);
  }
  const int eown = (ty + 4) * SX + tx + 4;
  // inputs of the cell finished next (L, stage increment), loaded one plane ahead
  const int NXY = p.n[0] * p.n[1];
  const int town = Y * p.n[0] + X;  // interior offset within a plane (own columns)
  float Lnext[5], Dnext[5];
  auto fetch_cell = [&](int d) {
    if (own && d >= zs && d < ze) {
      const long long t = (long long)d * NXY + town;
#pragma unroll
      for (int cc = 0; cc < 5; cc++) {
        Lnext[cc] = p.L32[cc * p.N + t];
        Dnext[cc] = din ? din[cc * p.N + t] : 0.f;
      }
    }
  };

  // ring slot of plane z: (z + 8) mod 5, advanced incrementally
  int slot = (zs - 4 + 8) % 5;
  for (int z = zs - 4; z <= zs; z++) {
    fetch(z);
    put(slot);
    slot = slot == 4 ? 0 : slot + 1;
  }
  fetch(zs + 1);
  // slot now belongs to plane zs + 1; planes c - 2 .. c + 2 for c = zs - 2 start at slot of
  // plane zs - 4
  int s0 = (zs - 4 + 8) % 5;
  __syncthreads();
  for (int c = zs - 2; c < ze + 2; c++) {
    // ring slots of planes c-2 .. c+2, once per plane
    const float *pl[5];
#pragma unroll
    for (int o = 0; o < 5; o++) {
      int so = s0 + o;
      pl[o] = ring + (so >= 5 ? so - 5 : so) * PLANE;
    }
    // own cell: all three fluxes; halo points: F_v,x (x offsets -2,-1,32,33) or F_v,y
    const float ihz = ihat(2, c);
    {
      float g[3][3], u[3], f[4];
      grads(pl, eown, ihx_own, ihy_own, ihz, g, u);
      vflux(0, g, u, f);
#pragma unroll
      for (int k = 0; k < 4; k++) fx[(k * TY + ty) * PX + tx + 2] = f[k];
      vflux(1, g, u, f);
#pragma unroll
      for (int k = 0; k < 4; k++) fy[(k * PY + ty + 2) * TX + tx] = f[k];
      vflux(2, g, u, f);
      const float zm2 = ihat(2, c - 2), zm1 = 8.f * ihat(2, c - 1);
      const float zp1 = 8.f * ihat(2, c + 1), zp2 = ihat(2, c + 2);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        acc[0][k] -= zm2 * f[k];
        acc[1][k] += zm1 * f[k];
        acc[3][k] -= zp1 * f[k];
        acc[4][k] += zp2 * f[k];
      }
    }
    static_assert(4 * TY + 4 * TX <= VT, "one halo point per thread at most");
    if (hkind) {
      float g[3][3], u[3], f[4];
      grads(pl, he, hihx, hihy, ihz, g, u);
      if (hkind == 1) {  // x-halo point
        vflux(0, g, u, f);
#pragma unroll
        for (int k = 0; k < 4; k++) fx[k * TY * PX + hout] = f[k];
      } else {           // y-halo point
        vflux(1, g, u, f);
#pragma unroll
        for (int k = 0; k < 4; k++) fy[k * PY * TX + hout] = f[k];
      }
    }
    __syncthreads();
    // x/y divergence at this column's cell of plane c
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const float *Fx = fx + (k * TY + ty) * PX + tx + 2;
      const float *Fy = fy + (k * PY + ty + 2) * TX + tx;
      acc[2][k] += d4f(Fx[-2], Fx[-1], Fx[1], Fx[2], ihx_own) +
                   d4f(Fy[-2 * TX], Fy[-TX], Fy[TX], Fy[2 * TX], ihy_own);
    }
    // plane d = c - 2 is complete: viscous term, sponge, RK update
    int d = c - 2;
    if (own && d >= zs && d < ze) {
      const long long t = (long long)d * NXY + town;
      float Lc[5];
#pragma unroll
      for (int cc = 0; cc < 5; cc++) Lc[cc] = Lnext[cc];
#pragma unroll
      for (int k = 0; k < 4; k++) Lc[k + 1] += acc[0][k] * p.inv_Re32;
      if (p.sponge_cells > 0) {
        int I[3] = {X, Y, d};
        int S = p.sponge_cells, nmin = 1 << 30;
#pragma unroll
        for (int a = 0; a < 3; a++) nmin = min(nmin, min(I[a], p.n[a] - 1 - I[a]));
        if (nmin < S) {
          float rr = (float)(S - nmin) / (float)S;
          float sig = (float)p.sponge_sigma * rr * rr * rr;
#pragma unroll
          for (int cc = 0; cc < 5; cc++) Lc[cc] -= sig * (p.qn32[cc * p.N + t] + Dnext[cc]);
        }
      }
      if (p.src_on) Lc[4] += pressure_source32<STRETCHED>(p, 3, X, Y, d);
      if (mode == 0) {
#pragma unroll
        for (int cc = 0; cc < 5; cc++) Lout[cc * p.N + t] = (double)Lc[cc];
      } else {
        bool bad = false;
        float inc[5];
#pragma unroll
        for (int cc = 0; cc < 5; cc++) {
          inc[cc] = Bc * (Dnext[cc] + dt * Lc[cc]);
          bad |= !isfinite(inc[cc]);
        }
        if (mode == 1) {
#pragma unroll
          for (int cc = 0; cc < 5; cc++) dout[cc * p.N + t] = inc[cc];
        } else {
#pragma unroll
          for (int cc = 0; cc < 5; cc++) {
            double qv = Qn[cc * p.N + t] + (double)inc[cc];
            Qn[cc * p.N + t] = qv;
            p.qn32[cc * p.N + t] = (float)(qv - p.qinf[cc]);
          }
        }
        if (bad) atomicOr(p.status, IBFSA_STATUS_NONFINITE);
      }
    }
    // plane c + 3 (needed from the next iteration on) replaces plane c - 2, whose gradients
    // were all taken before the barrier above; plane c + 4 starts loading
#pragma unroll
    for (int o = 0; o < 4; o++)
#pragma unroll
      for (int k = 0; k < 4; k++) acc[o][k] = acc[o + 1][k];
#pragma unroll
    for (int k = 0; k < 4; k++) acc[4][k] = 0.f;
    if (c + 1 < ze + 2) {
      put(s0);  // plane c + 3 takes the slot of plane c - 2
      if (c + 2 < ze + 2) fetch(c + 4);
      fetch_cell(c - 1);
    }
    s0 = s0 == 4 ? 0 : s0 + 1;
    __syncthreads();
  }
}

template <int DIM>
__global__ void __launch_bounds__(THREADS) k_refresh32(Plan p, const double *__restrict__ Q) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.N) return;
#pragma unroll
  for (int c = 0; c < DIM + 2; c++) p.qn32[c * p.N + t] = (float)(Q[c * p.N + t] - p.qinf[c]);
}

template <int DIM>
__global__ void k_probe64(Plan p, const double *__restrict__ Q, int np,
                          const double *__restrict__ xp, double *__restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  int j0[3];
  double w[3][4];
  if (!point_support<DIM>(p, xp, np, k, j0, w)) {
    atomicOr(p.status, IBFSA_STATUS_BOUNDS);
    out[k] = 0.0;
    return;
  }
  constexpr int C2 = DIM > 2 ? 4 : 1;
  double acc = 0.0;
  for (int r2 = 0; r2 < C2; r2++)
    for (int r1 = 0; r1 < 4; r1++)
      for (int r0 = 0; r0 < 4; r0++) {
        long long o = int_index(p, j0[0] + r0, j0[1] + r1, j0[2] + r2);
        double rho = Q[o], ke = 0.0;
        for (int a = 0; a < DIM; a++) {
          double m = Q[(1 + a) * p.N + o];
          ke += m * (m / rho);
        }
        double pr = p.gm1 * (Q[(DIM + 1) * p.N + o] - 0.5 * ke);
        acc += pr * (w[0][r0] * w[1][r1] * w[2][r2]);
      }
  out[k] = acc - p.p_inf;
}

// ------------------------------------------------------------------------------------------
inline unsigned blocks_for(long long n, int threads) {
  return (unsigned)((n + threads - 1) / threads);
}

// Tensor maps of the y/z tile copies: q' and the primitives over the padded box, L' over the
// interior, each as a rank-4 tensor (x, y, z, component) with boxes of 32 x-lines by the staged
// (or owned) cells along A.
template <int DIM, int A>
cudaError_t conv_tensor_maps(const Plan &p, CUtensorMap *tq, CUtensorMap *tw, CUtensorMap *tl) {
  using T = Tile<A>;
  const uint64_t P0 = p.P[0], P1 = p.P[1], P2 = p.P[2], n0 = p.n[0], n1 = p.n[1], n2 = p.n[2];
  const uint64_t ps[3] = {4 * P0, 4 * P0 * P1, 4 * (uint64_t)p.NP};
  const uint64_t is[3] = {4 * n0, 4 * n0 * n1, 4 * (uint64_t)p.N};
  const uint64_t dq[4] = {P0, P1, P2, (uint64_t)DIM + 2}, dw[4] = {P0, P1, P2, (uint64_t)DIM + 1};
  const uint64_t dl[4] = {n0, n1, n2, (uint64_t)DIM + 2};
  const uint32_t ly = A == 1 ? T::LEN : 1, lz = A == 2 ? T::LEN : 1;
  const uint32_t sy = A == 1 ? T::SEG : 1, sz = A == 2 ? T::SEG : 1;
  const uint32_t bq[4] = {T::ROWS, ly, lz, DIM + 2}, bw[4] = {T::ROWS, ly, lz, 1};
  const uint32_t bl[4] = {T::ROWS, sy, sz, DIM + 2};
  cudaError_t e;
  if ((e = tma::encode_f32_4d(tq, p.Qp32, dq, ps, bq)) != cudaSuccess) return e;
  if ((e = tma::encode_f32_4d(tw, p.Wp32, dw, ps, bw)) != cudaSuccess) return e;
  return tma::encode_f32_4d(tl, p.L32, dl, is, bl);
}

template <int DIM, int A, int SCHEME>
cudaError_t launch_conv(const Plan &p, int first, cudaStream_t st) {
  using T = Tile<A>;
  cudaError_t e;
  if constexpr (SCHEME != IBFSA_MLP_TENO5) {
    if (p.charwise) {  // the characteristic-wise option: generic tiles for every direction
      constexpr size_t smem = conv_smem<DIM, A>();
      e = cudaFuncSetAttribute(k_conv32<DIM, A, SCHEME, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      dim3 grid;
      if (A == 0) {
        grid = dim3((p.n[0] + T::SEG - 1) / T::SEG, (p.n[1] + T::ROWS - 1) / T::ROWS, p.n[2]);
      } else {
        int nseg = (p.n[A] + T::SEG - 1) / T::SEG;
        grid = dim3(nseg * ((p.n[0] + T::ROWS - 1) / T::ROWS), A == 1 ? p.n[2] : p.n[1]);
      }
      k_conv32<DIM, A, SCHEME, true><<<grid, THREADS, smem, st>>>(p, first);
      return cudaGetLastError();
    }
  }
  if constexpr (A != 0) {
    if (p.n[0] % 4 == 0 && !first) {
      using TT = TmaTile<DIM, A>;
      constexpr size_t smem =
          TT::BYTES + (SCHEME == IBFSA_MLP_TENO5 ? (size_t)mlp::PACKED_BYTES : 0);
      e = cudaFuncSetAttribute(k_conv32_tma<DIM, A, SCHEME>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      CUtensorMap tq, tw, tl;
      if ((e = conv_tensor_maps<DIM, A>(p, &tq, &tw, &tl)) != cudaSuccess) return e;
      int nseg = (p.n[A] + T::SEG - 1) / T::SEG;
      int nx = (p.n[0] + T::ROWS - 1) / T::ROWS;
      dim3 grid(nseg * nx, A == 1 ? p.n[2] : p.n[1]);
      k_conv32_tma<DIM, A, SCHEME><<<grid, THREADS, smem, st>>>(p, tq, tw, tl);
      return cudaGetLastError();
    }
  }
  constexpr size_t smem =
      conv_smem<DIM, A>() + (SCHEME == IBFSA_MLP_TENO5 ? (size_t)mlp::PACKED_BYTES : 0);
  e = cudaFuncSetAttribute(k_conv32<DIM, A, SCHEME>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid;
  if (A == 0) {
    grid = dim3((p.n[0] + T::SEG - 1) / T::SEG, (p.n[1] + T::ROWS - 1) / T::ROWS, p.n[2]);
  } else {
    int nseg = (p.n[A] + T::SEG - 1) / T::SEG;
    int nx = (p.n[0] + T::ROWS - 1) / T::ROWS;
    grid = dim3(nseg * nx, A == 1 ? p.n[2] : p.n[1]);
  }
  k_conv32<DIM, A, SCHEME><<<grid, THREADS, smem, st>>>(p, first);
  return cudaGetLastError();
}

template <int DIM, int SCHEME>
cudaError_t run_stage(const Plan &p, const StageArgs &s, cudaStream_t st) {
  cudaError_t e;
  Prof *pr = s.prof;
  e = cudaMemsetAsync(p.alpha_bits, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  // stage increments: none at the step start, d1 after stage 1, d2 after stage 2
  const float *din = s.stage == 1 ? p.d1 : s.stage == 2 ? p.d2 : nullptr;
  float *dout = s.stage == 0 ? p.d1 : s.stage == 1 ? p.d2 : nullptr;
  const double *Qn = s.Qn;
  prof_begin(pr, st);
  k_pad32<DIM><<<blocks_for(p.NP, THREADS), THREADS, 0, st>>>(p, din);
  prof_end(pr, K_PAD, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int advance = s.stage >= 0;
  if (p.nm > 0) {
    prof_begin(pr, st);
    k_ib_interp64<DIM><<<blocks_for(p.nm, 128), 128, 0, st>>>(p, Qn, din, s.xis, s.xin, s.xio,
                                                             s.a, s.b, s.dt, advance);
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
  for (int a = 0; a < DIM; a++)  // characteristic faces
    for (int side = 0; side < 2; side++) {
      if (p.bc[a][side] != IBFSA_BC_CHARACTERISTIC) continue;
      long long cells = (long long)p.n[(a + 1) % 3] * p.n[(a + 2) % 3];
      prof_begin(pr, st);
      k_char_face32<DIM><<<blocks_for(cells, THREADS), THREADS, 0, st>>>(p, a, side);
      prof_end(pr, K_CONV_X + a, st);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  if (p.Re > 0.0 && DIM == 2) {
    prof_begin(pr, st);
    k_visc_flux32<DIM><<<blocks_for(p.NB, THREADS), THREADS, 0, st>>>(p);
    prof_end(pr, K_VISC_FLUX, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (p.nm > 0) {
    constexpr int MPB = DIM > 2 ? 2 : 8;  // markers per 128-thread block
    prof_begin(pr, st);
    k_spread32<DIM><<<blocks_for(p.nm, MPB), 128, 0, st>>>(p, Qn, din);
    prof_end(pr, K_SPREAD, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  int mode = !advance ? 0 : (s.stage < 2 ? 1 : 2);
  Plan q = p;
  q.src_scale = s.src_scale;
  prof_begin(pr, st);
  if (p.Re > 0.0 && DIM == 3) {
    using namespace vm;
    const bool stretched = p.minv12_32[0] || p.minv12_32[1] || p.minv12_32[2];
    auto kern = stretched ? k_visc_march32<true> : k_visc_march32<false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((p.n[0] + TX - 1) / TX, (p.n[1] + TY - 1) / TY, (p.n[2] + ZC - 1) / ZC);
    kern<<<grid, VT, SMEM, st>>>(q, din, dout, const_cast<double *>(Qn), s.Lout, (float)s.b,
                                 (float)s.dt, mode);
  } else if (p.Re > 0.0)
    k_finish32<DIM, true><<<blocks_for(p.N, THREADS), THREADS, 0, st>>>(
        q, din, dout, const_cast<double *>(Qn), s.Lout, (float)s.b, (float)s.dt, mode);
  else
    k_finish32<DIM, false><<<blocks_for(p.N, THREADS), THREADS, 0, st>>>(
        q, din, dout, const_cast<double *>(Qn), s.Lout, (float)s.b, (float)s.dt, mode);
  prof_end(pr, K_FINISH, st);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------
// training stencils of the learned weights from the current state
// ------------------------------------------------------------------------------------------
struct Coef9 {
  float c[9];  // face value of the 9-point upwind-biased reconstruction from cells i-4 .. i+4
};

__device__ __forceinline__ unsigned long long splitmix(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

template <int DIM>
__global__ void k_mlp_sample(Plan p, int n_max, unsigned long long seed, int attempts, Coef9 cf,
                             float *__restrict__ S, float *__restrict__ T, int *count) {
  constexpr int NV = DIM + 2;
  long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  Free fs = free_stream(p);
  for (int att = 0; att < attempts; att++) {
    unsigned long long r = splitmix(seed ^ splitmix((unsigned long long)tid * attempts + att));
    int A = (int)(r % DIM);
    int c = (int)((r >> 8) % NV);
    int sign = (int)((r >> 16) & 1);
    unsigned long long r2 = splitmix(r);
    int I[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      unsigned span = a == A ? (unsigned)(p.n[a] - 1) : (unsigned)p.n[a];
      I[a] = a < DIM ? (int)((r2 >> (20 * a)) % (span ? span : 1u)) : 0;
    }
    if (p.n[A] < 2) continue;
    const float alpha = (float)__longlong_as_double((long long)p.alpha_bits[A]);
    float f[10];
#pragma unroll
    for (int o = 0; o < 10; o++) {
      int J[3] = {I[0], I[1], I[2]};
      J[A] += o - 4;
      long long sidx = ((long long)(J[2] + p.g[2]) * p.P[1] + (J[1] + p.g[1])) * p.P[0] + (J[0] + p.g[0]);
      float up = p.Wp32[A * p.NP + sidx];
      float pp = p.Wp32[DIM * p.NP + sidx];
      float ua = fs.u[A] + up;
      float q = p.Qp32[c * p.NP + sidx];
      float F;
      if (c == 0) F = p.Qp32[(1 + A) * p.NP + sidx];
      else if (c == NV - 1) F = (q + pp) * ua + fs.H * up;
      else {
        F = q * ua + fs.m[c - 1] * up;
        if (c - 1 == A) F += pp;
      }
      f[o] = 0.5f * (sign == 0 ? F + alpha * q : F - alpha * q);
    }
    float v[5];
    if (sign == 0) { v[0] = f[2]; v[1] = f[3]; v[2] = f[4]; v[3] = f[5]; v[4] = f[6]; }
    else { v[0] = f[7]; v[1] = f[6]; v[2] = f[5]; v[3] = f[4]; v[4] = f[3]; }
    Cands k = candidates(v[0], v[1], v[2], v[3], v[4]);
    float amp = 0.f;
#pragma unroll
    for (int j = 0; j < 5; j++) amp = fmaxf(amp, fabsf(v[j] - v[2]));
    if (teno_mask(k) != 7 || !(amp > p.mlp_floor)) continue;
    // upwind side of the face: cells i-4 .. i+4 for the right-going flux, the mirror image
    // (cells i+5 .. i-3) for the left-going one
    float tgt = 0.f;
#pragma unroll
    for (int o = 0; o < 9; o++) tgt += cf.c[o] * (sign == 0 ? f[o] : f[9 - o]);
    int idx = atomicAdd(count, 1);
    if (idx >= n_max) return;
#pragma unroll
    for (int j = 0; j < 5; j++) S[(size_t)idx * 5 + j] = v[j];
    T[idx] = tgt;
  }
}

}  // namespace fp32_ns

// coefficients c_o (o = -4..4) with sum_o c_o avg_o(h) = h(0) for polynomials h of degree <= 8,
// avg_o = mean over [o-1, o] (the cell left of the face is o = 0): the flux-reconstruction target
// of the ninth-order upwind-biased scheme
static void upwind9(float out[9]) {
  constexpr int K = 9;
  double M[K][K + 1];
  for (int pw = 0; pw < K; pw++) {
    for (int j = 0; j < K; j++) {
      double o = j - 4;
      M[pw][j] = (pow(o, pw + 1) - pow(o - 1.0, pw + 1)) / (pw + 1);
    }
    M[pw][K] = pw == 0 ? 1.0 : 0.0;
  }
  for (int col = 0; col < K; col++) {
    int piv = col;
    for (int r = col + 1; r < K; r++)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    for (int k = 0; k <= K; k++) {
      double tmp = M[col][k];
      M[col][k] = M[piv][k];
      M[piv][k] = tmp;
    }
    for (int r = 0; r < K; r++) {
      if (r == col) continue;
      double fct = M[r][col] / M[col][col];
      for (int k = col; k <= K; k++) M[r][k] -= fct * M[col][k];
    }
  }
  for (int j = 0; j < K; j++) out[j] = (float)(M[j][K] / M[j][j]);
}

cudaError_t fp32_mlp_sample(const Plan &p, const double *Q, int n_max, unsigned long long seed,
                            int attempts, float *stencils, float *targets, int *count,
                            cudaStream_t st) {
  using namespace fp32_ns;
  cudaError_t e = fp32_wavespeed(p, Q, st);  // qn32, padded perturbation and split speeds
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(count, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  Coef9 cf;
  upwind9(cf.c);
  int threads = 256, blocks = 152 * 8;
  if (p.dim == 2)
    k_mlp_sample<2><<<blocks, threads, 0, st>>>(p, n_max, seed, attempts, cf, stencils, targets,
                                               count);
  else
    k_mlp_sample<3><<<blocks, threads, 0, st>>>(p, n_max, seed, attempts, cf, stencils, targets,
                                               count);
  return cudaGetLastError();
}

// Self-test of the bounded wait: one block announces bytes on its barrier and issues no copy,
// so the phase never completes; the block must give up after the poll limit, report
// IBFSA_STATUS_TIMEOUT through the same path as the convective kernels, and end (nothing is in
// flight when it exits).
__global__ void __launch_bounds__(fp32_ns::THREADS) k_wait_selftest(Plan p) {
  __shared__ __align__(8) uint64_t bar[1];
  if (threadIdx.x == 0) tma::mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) tma::mbar_expect_tx(bar, 16);  // no copy will deliver these bytes
  if (!fp32_ns::block_wait_or_report(p, bar, 0)) return;
  if (threadIdx.x == 0) atomicOr(p.status, IBFSA_STATUS_NONFINITE);  // unreachable
}

cudaError_t wait_selftest(const Plan &p, cudaStream_t st) {
  k_wait_selftest<<<1, fp32_ns::THREADS, 0, st>>>(p);
  return cudaGetLastError();
}

// Force the fluid exerts on the body and the power it delivers, from the Lagrangian penalty
// forces of the last evaluated stage (Eq. 7): sum_k F_k dS_k and sum_k (F_k . U_k) dS_k, in
// FP64, summed by one block in a fixed order (reproducible).
__global__ void k_body_force(Plan p, const double *__restrict__ U, double *__restrict__ out) {
  __shared__ double red[4][256];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int M = p.max_markers;
  for (int k = threadIdx.x; k < p.nm; k += blockDim.x) {
    double pw = 0.0;
    for (int a = 0; a < p.dim; a++) {
      double fa = p.F[a * M + k] * p.dS[k];
      acc[a] += fa;
      pw += fa * U[a * M + k];
    }
    acc[3] += pw;
  }
  for (int c = 0; c < 4; c++) red[c][threadIdx.x] = acc[c];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int c = 0; c < 4; c++) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = red[threadIdx.x][0];
}

cudaError_t body_force(const Plan &p, const double *U, double *out, cudaStream_t st) {
  k_body_force<<<1, 256, 0, st>>>(p, U, out);
  return cudaGetLastError();
}

cudaError_t fp32_stage(const Plan &p, const StageArgs &s, cudaStream_t st) {
  using namespace fp32_ns;
  if (p.dim == 2) {
    if (p.scheme == IBFSA_MLP_TENO5) return run_stage<2, IBFSA_MLP_TENO5>(p, s, st);
    return p.scheme == IBFSA_TENO5 ? run_stage<2, IBFSA_TENO5>(p, s, st)
                                   : run_stage<2, IBFSA_WENO5JS>(p, s, st);
  }
  if (p.scheme == IBFSA_MLP_TENO5) return run_stage<3, IBFSA_MLP_TENO5>(p, s, st);
  return p.scheme == IBFSA_TENO5 ? run_stage<3, IBFSA_TENO5>(p, s, st)
                                 : run_stage<3, IBFSA_WENO5JS>(p, s, st);
}

cudaError_t fp32_refresh(const Plan &p, const double *Q, cudaStream_t st) {
  using namespace fp32_ns;
  if (p.dim == 2) k_refresh32<2><<<blocks_for(p.N, THREADS), THREADS, 0, st>>>(p, Q);
  else k_refresh32<3><<<blocks_for(p.N, THREADS), THREADS, 0, st>>>(p, Q);
  return cudaGetLastError();
}

cudaError_t fp32_wavespeed(const Plan &p, const double *Q, cudaStream_t st) {
  using namespace fp32_ns;
  cudaError_t e = fp32_refresh(p, Q, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(p.alpha_bits, 0, 3 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (p.dim == 2) k_pad32<2><<<blocks_for(p.NP, THREADS), THREADS, 0, st>>>(p, nullptr);
  else k_pad32<3><<<blocks_for(p.NP, THREADS), THREADS, 0, st>>>(p, nullptr);
  return cudaGetLastError();
}

cudaError_t fp32_probe(const Plan &p, const double *Q, int np, const double *xp, double *out,
                       cudaStream_t st, Prof *pr) {
  using namespace fp32_ns;
  prof_begin(pr, st);
  if (p.dim == 2) k_probe64<2><<<blocks_for(np, 128), 128, 0, st>>>(p, Q, np, xp, out);
  else k_probe64<3><<<blocks_for(np, 128), 128, 0, st>>>(p, Q, np, xp, out);
  prof_end(pr, K_PROBE, st);
  return cudaGetLastError();
}

}  // namespace ibfsa
