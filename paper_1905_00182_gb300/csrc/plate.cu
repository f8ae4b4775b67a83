// plate.cu -- the flexible plate of arXiv:1905.00182 (Sec. 2, Eq. 1) in the absolute nodal
// coordinate formulation, its clamp motion (Sec. 4.1, Eq. 17), and the two-way coupling with the
// fluid grid through the penalty forces (Eq. 7-9).
//
// Compiled with --fmad=false and host -ffp-contract=off: every FP64 operation is rounded on its
// own, in the order written, except the explicit fused multiply-adds (__fma_rn) of the element
// dot products and of the cyclic reduction, so every run gives the same bits.  Against an
// independent solve of the same Newton systems (Gaussian elimination in natural order) the
// result agrees to a few roundings of the residual times the Newton matrix's condition number.
//
// The structure solve is tiny (4 (n_el + 1) unknowns) and sequential by nature (Newton), so it
// runs in ONE thread block with all state in shared memory, and the host never waits on it:
// Gauss-point factors one thread per (element, point), element residual rows and Jacobian rows
// one thread per (element, row), assembly one thread per coordinate, and the Newton system --
// block tridiagonal in the nodes -- by block cyclic reduction: at each of ~log2(n_el) levels the
// eliminated 4 x 4 blocks are factorised by half-warps in parallel, so the dependent chain is a
// few levels long instead of one pivot per unknown.  On GB300 a warp's FP64 instruction holds its
// SM quarter's narrow FP64 pipe for tens of cycles however few lanes are active, which is what
// makes the length of that chain, not the amount of work, the cost.
//
// Discretisation (Eq. 1 read as the Euler-Lagrange equation of
// 1/2 int rho_s |r_t|^2 ds - 1/2 int [K_S (|r_s| - 1)^2 + K_B |r_ss|^2] ds):
//   node j: e_j = [x, y, x_s, y_s]; element k, xi = (s - k l)/l:
//   r = S0 r_k + S1 r_s,k + S2 r_k+1 + S3 r_s,k+1 (cubic Hermite);
//   consistent mass rho_s int S^T S, bending K_B int S''^T S'' (closed forms), stretching
//   int K_S (1 - 1/|r_s|) S'^T r_s by 5-point Gauss-Legendre quadrature;
//   implicit midpoint step: M (v_{n+1} - v_n) = dt [Q_f - Q_int(e_n + d/2)], d = e_{n+1} - e_n,
//   Newton on d with Jacobian M + dt^2/4 dQ_int/de (both scaled by dt/2);
//   clamp: node 0 position prescribed, slope = sigma t(t) with sigma free.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "ibfsa_internal.h"

namespace ibfsa {
namespace plate {

constexpr int BW = 7;  // half-bandwidth

__constant__ double c_gx[5] = {-0.90617984593866399280, -0.53846931010568309104, 0.0,
                               0.53846931010568309104, 0.90617984593866399280};
__constant__ double c_gw[5] = {0.23692688505618908751, 0.47862867049936646804,
                               0.56888888888888888889, 0.47862867049936646804,
                               0.23692688505618908751};

struct Params {
  int n_el, nd, nm, clamped, newton_max;
  double L, l, rho_s, K_S, K_B, tol;
};

// element coordinate of shape function i, component a
__device__ __forceinline__ int lc(int i, int a) { return 4 * (i / 2) + 2 * (i % 2) + a; }

__device__ __forceinline__ void shape_fn(double xi, double l, double S[4]) {
  double x2 = xi * xi, x3 = x2 * xi;
  S[0] = 1.0 - 3.0 * x2 + 2.0 * x3;
  S[1] = l * (xi - 2.0 * x2 + x3);
  S[2] = 3.0 * x2 - 2.0 * x3;
  S[3] = l * (x3 - x2);
}

__device__ __forceinline__ void shape_ds(double xi, double l, double D[4]) {
  double x2 = xi * xi;
  D[0] = (6.0 * x2 - 6.0 * xi) / l;
  D[1] = 1.0 - 4.0 * xi + 3.0 * x2;
  D[2] = (6.0 * xi - 6.0 * x2) / l;
  D[3] = 3.0 * x2 - 2.0 * xi;
}

// entry (i, j) of the element's consistent mass and bending matrices (per component)
__device__ __forceinline__ double mass_ij(const Params &P, int i, int j) {
  double l = P.l;
  double c = P.rho_s * l / 420.0;
  double m;
  switch (i * 4 + j) {
    case 0: m = 156.0; break;
    case 1: case 4: m = 22.0 * l; break;
    case 2: case 8: m = 54.0; break;
    case 3: case 12: m = -13.0 * l; break;
    case 5: m = 4.0 * l * l; break;
    case 6: case 9: m = 13.0 * l; break;
    case 7: case 13: m = -3.0 * l * l; break;
    case 10: m = 156.0; break;
    case 11: case 14: m = -22.0 * l; break;
    default: m = 4.0 * l * l; break;  // 15
  }
  return c * m;
}

__device__ __forceinline__ double bend_ij(const Params &P, int i, int j) {
  double l = P.l;
  double c = P.K_B / (l * l * l);
  double k;
  switch (i * 4 + j) {
    case 0: k = 12.0; break;
    case 1: case 4: k = 6.0 * l; break;
    case 2: case 8: k = -12.0; break;
    case 3: case 12: k = 6.0 * l; break;
    case 5: k = 4.0 * l * l; break;
    case 6: case 9: k = -6.0 * l; break;
    case 7: case 13: k = 2.0 * l * l; break;
    case 10: k = 12.0; break;
    case 11: case 14: k = -6.0 * l; break;
    default: k = 4.0 * l * l; break;  // 15
  }
  return c * k;
}

// marker k: element and local coordinate (s_k = (k + 1/2) L / n_m)
__device__ __forceinline__ int marker_site(const Params &P, int k, double *xi) {
  double s = ((double)k + 0.5) * P.L / (double)P.nm;
  int el = (int)(s / P.l);
  if (el > P.n_el - 1) el = P.n_el - 1;
  *xi = (s - (double)el * P.l) / P.l;
  return el;
}

__device__ int first_marker_of(const Params &P, int el) {
  double xi;
  int k = (int)((double)el * (double)P.nm / (double)P.n_el) - 2;
  if (k < 0) k = 0;
  if (k > P.nm) k = P.nm;
  while (k > 0 && marker_site(P, k - 1, &xi) >= el) k--;
  while (k < P.nm && marker_site(P, k, &xi) < el) k++;
  return k;
}

// ---- marker tables (built once per plate): element, shape values, first marker of each element
__global__ void k_tables(Params P, int *mk_el, double *mk_S, int *el_first) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < P.nm) {
    double xi, S[4];
    int el = marker_site(P, k, &xi);
    shape_fn(xi, P.l, S);
    mk_el[k] = el;
    for (int i = 0; i < 4; i++) mk_S[4 * k + i] = S[i];
  }
  if (k <= P.n_el) el_first[k] = k == P.n_el ? P.nm : first_marker_of(P, k);
}

// ---- markers from the plate: X, U [2][stride], dS ------------------------------------------
__global__ void k_markers(Params P, const double *__restrict__ e, const double *__restrict__ v,
                          const int *__restrict__ mk_el, const double *__restrict__ mk_S,
                          double *X, double *U, double *dS, int stride, double *U2) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.nm) return;
  int el = mk_el[k];
  double S[4];
  for (int i = 0; i < 4; i++) S[i] = mk_S[4 * k + i];
  for (int a = 0; a < 2; a++) {
    double x = 0.0, u = 0.0;
    for (int i = 0; i < 4; i++) {
      x = x + S[i] * e[4 * el + lc(i, a)];
      u = u + S[i] * v[4 * el + lc(i, a)];
    }
    X[a * stride + k] = x;
    U[a * stride + k] = u;
    if (U2) U2[a * P.nm + k] = u;  // the plate's own copy of the step's marker velocities
  }
  dS[k] = P.L / (double)P.nm;
}

// ---- force and power of the step's load (Eq. 19 numerators), summed in marker order ------
__global__ void k_force(Params P, const double *__restrict__ F, const double *__restrict__ U,
                        double *res) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int nm = P.nm;
  double dS = P.L / (double)nm;
  double fx = 0.0, fy = 0.0, pw = 0.0;
  for (int k = 0; k < nm; k++) {
    fx = fx + F[k] * dS;
    fy = fy + F[nm + k] * dS;
    pw = pw + (F[k] * U[k] + F[nm + k] * U[nm + k]) * dS;
  }
  res[0] = fx;
  res[1] = fy;
  res[2] = pw;
}

// ---- stage force average: Fbar = w F (first stage) or Fbar + w F ---------------------------
__global__ void k_force_average(int nm, const double *__restrict__ F, int stride, double *Fbar,
                                double w, int first) {
  int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= 2 * nm) return;
  int a = o / nm, k = o - a * nm;
  double f = F[a * stride + k];
  Fbar[o] = first ? w * f : Fbar[o] + w * f;
}

// ---- the structure step (one block) --------------------------------------------------------
struct StepArgs {
  double dt;
  double ep[4], vp[4];   // clamp coordinates and rates of node 0 at the new time
  double *e, *v;         // state, advanced in place
  const double *F;       // marker forces [2][nm]
  const double *mk_S;    // shape values of the markers [nm][4]
  const int *el_first;   // first marker of each element, [n_el + 1]
  int *status;
  int *max_iters;
};

// Shared-memory carve-up (doubles) for n_el elements.  Tables that depend only on l and the
// quadrature are built once per launch: D[g][i] = dS_i/ds at Gauss point g, PD[g][i][j] =
// (w_g l D_gi) D_gj (the first two factors of every tangent term), the element mass and bending
// matrices.  Per element and Gauss point: r_s, K_S (1 - 1/|r_s|) w l (times r_s) and the four
// tangent factors s_ab = c2 r_a r_b (+ c1 on the diagonal).
struct Smem {
  double *en, *vn, *d, *em, *g, *R, *Qf, *x;
  double (*Ag)[BW + 1];
  double (*Rel)[8];
  // element scratch (element rows, Gauss-point factors) and, after assembly, the node blocks of
  // the reduction share one region
  double (*Jel)[64];
  double (*gt)[5][2];   // per element, Gauss point: (w l c1) r_a
  double (*gs)[5][4];   // per element, Gauss point: s_ab, ab = 00, 01, 10, 11
  double (*BD)[16];     // per node block: D_j (factor after elimination)
  double (*BB)[16];     // Br_j, coupling to the next active block
  double (*BY)[16];     // D_i^-1 Br_i
  double (*BZ)[16];     // D_i^-1 Br_{i-s}^T
  double (*BT)[16];     // new couplings of a level
  double (*bb)[4], (*bx)[4], (*by)[4], (*br)[4];  // rhs, solution, D_i^-1 b_i, 1 / pivots
  double *D;            // [5][4]
  double *PD;           // [5][4][4]
  double *Ms, *Kb;      // [4][4]
  int *flags;
};

__host__ __device__ inline size_t union_doubles(int n_el) {
  size_t ne = (size_t)n_el, nb = ne + 1;
  size_t elem = 94 * ne, blocks = 96 * nb;
  return elem > blocks ? elem : blocks;
}

__host__ __device__ inline size_t smem_doubles(int n_el) {
  size_t nd = 4 * (size_t)(n_el + 1), ne = (size_t)n_el;
  return 8 * nd + 8 * nd + 8 * ne + union_doubles(n_el) + 20 + 80 + 32 + 4;
}

__device__ inline Smem carve(double *base, int n_el) {
  int nd = 4 * (n_el + 1), nb = n_el + 1;
  Smem s;
  double *p = base;
  s.en = p; p += nd;
  s.vn = p; p += nd;
  s.d = p; p += nd;
  s.em = p; p += nd;
  s.g = p; p += nd;
  s.R = p; p += nd;
  s.Qf = p; p += nd;
  s.x = p; p += nd;
  s.Ag = reinterpret_cast<double(*)[BW + 1]>(p); p += 8 * nd;
  s.Rel = reinterpret_cast<double(*)[8]>(p); p += 8 * n_el;
  double *u = p;
  s.Jel = reinterpret_cast<double(*)[64]>(u);
  s.gt = reinterpret_cast<double(*)[5][2]>(u + 64 * n_el);
  s.gs = reinterpret_cast<double(*)[5][4]>(u + 74 * n_el);
  s.BD = reinterpret_cast<double(*)[16]>(u);
  s.BB = reinterpret_cast<double(*)[16]>(u + 16 * nb);
  s.BY = reinterpret_cast<double(*)[16]>(u + 32 * nb);
  s.BZ = reinterpret_cast<double(*)[16]>(u + 48 * nb);
  s.BT = reinterpret_cast<double(*)[16]>(u + 64 * nb);
  s.bb = reinterpret_cast<double(*)[4]>(u + 80 * nb);
  s.bx = reinterpret_cast<double(*)[4]>(u + 84 * nb);
  s.by = reinterpret_cast<double(*)[4]>(u + 88 * nb);
  s.br = reinterpret_cast<double(*)[4]>(u + 92 * nb);
  p += union_doubles(n_el);
  s.D = p; p += 20;
  s.PD = p; p += 80;
  s.Ms = p; p += 16;
  s.Kb = p; p += 16;
  s.flags = reinterpret_cast<int *>(p);
  return s;
}

// v <- (L D L^T)^-1 v for one 4 x 4 block factored in place (M row-major, upper triangle)
__device__ __forceinline__ void solve4(const double *M, const double *rinv, double v[4]) {
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int k = 1; i + k < 4; k++) v[i + k] = __fma_rn(-M[i * 4 + i + k], v[i], v[i + k]);
#pragma unroll
  for (int i = 0; i < 4; i++) v[i] = v[i] * rinv[i];
#pragma unroll
  for (int i = 3; i >= 0; i--)
#pragma unroll
    for (int k = 1; i + k < 4; k++) v[i] = __fma_rn(-M[i * 4 + i + k], v[i + k], v[i]);
}

// Block cyclic reduction of the node-block system (S.BD, S.BB, S.bb) into S.bx, all threads of
// the block; returns false on a zero or non-finite pivot.  Per level: eliminated blocks
// i = s, 3s, ... one per half-warp (4 x 4 L D L^T with the pivot's updates in parallel lanes,
// then nine solves, one per lane); survivors k = 0, 2s, ... one item per thread for each
// entry of D_k, Br_k (new) and b_k; then back substitution from coarse to fine.
__device__ bool bcr_solve(const Smem &S, int nb, int *flag) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nt >> 5, half = lane >> 4, hl = lane & 15;
  // pivot pairs (k, m), 1 <= k <= m <= 3 - pi, for the 16 lanes of a half-warp
  if (tid == 0) *flag = 0;
  __syncthreads();
  int s;
  for (s = 1; s < nb; s *= 2) {
    const int nelim = (nb - 1 - s) / (2 * s) + 1;
    for (int base = 0; base < nelim; base += 2 * nwarps) {
      const int t = base + 2 * warp + half;
      const bool act = t < nelim;
      const int i = s + 2 * s * t;
      double *M = S.BD[act ? i : 0];
      bool bad = false;
#pragma unroll
      for (int pi = 0; pi < 4; pi++) {
        double dpiv = act ? M[pi * 4 + pi] : 1.0;
        bad = bad || !(dpiv != 0.0) || !isfinite(dpiv);
        double r = 1.0 / dpiv;
        int n = 3 - pi;  // entries right of the pivot
        // pair index hl -> (k, m) with 1 <= k <= m <= n
        int k = 0, m = 0, q = hl;
        for (int kk = 1; kk <= n; kk++) {
          if (k == 0 && q < n - kk + 1) { k = kk; m = kk + q; }
          else if (k == 0) q -= n - kk + 1;
        }
        double lk = 0.0;
        if (act && k > 0) {
          lk = M[pi * 4 + pi + k] * r;
          M[(pi + k) * 4 + pi + m] = __fma_rn(-lk, M[pi * 4 + pi + m], M[(pi + k) * 4 + pi + m]);
        }
        __syncwarp();
        if (act && k > 0 && m == k) M[pi * 4 + pi + k] = lk;
        if (act && hl == 0) S.br[i][pi] = r;
        __syncwarp();
      }
      if (act && bad && hl == 0) atomicOr(flag, 1);
      if (act && hl < 9) {
        double v[4];
        const bool right = i + s < nb;
#pragma unroll
        for (int q = 0; q < 4; q++) {
          if (hl < 4) v[q] = right ? S.BB[i][q * 4 + hl] : 0.0;
          else if (hl < 8) v[q] = S.BB[i - s][(hl - 4) * 4 + q];
          else v[q] = S.bb[i][q];
        }
        solve4(M, S.br[i], v);
#pragma unroll
        for (int q = 0; q < 4; q++) {
          if (hl < 4) S.BY[i][q * 4 + hl] = v[q];
          else if (hl < 8) S.BZ[i][q * 4 + hl - 4] = v[q];
          else S.by[i][q] = v[q];
        }
      }
    }
    __syncthreads();
    if (*flag) return false;
    // survivors: D_k, b_k in place (each item owns its entry), new couplings into BT
    const int nsurv = (nb - 1) / (2 * s) + 1;
    for (int it = tid; it < nsurv * 36; it += nt) {
      const int k = (it / 36) * 2 * s, e = it % 36;
      const int il = k - s, ir = k + s;
      const bool hl_ = il >= 0, hr = ir < nb, hn = hr && ir + s < nb;
      if (e < 16) {
        const int r = e / 4, c = e % 4;
        double v = S.BD[k][e];
        if (hl_)
#pragma unroll
          for (int q = 0; q < 4; q++) v = __fma_rn(-S.BB[il][q * 4 + r], S.BY[il][q * 4 + c], v);
        if (hr)
#pragma unroll
          for (int q = 0; q < 4; q++) v = __fma_rn(-S.BB[k][r * 4 + q], S.BZ[ir][q * 4 + c], v);
        S.BD[k][e] = v;
      } else if (e < 32) {
        const int r = (e - 16) / 4, c = (e - 16) % 4;
        double u = 0.0;
        if (hn)
#pragma unroll
          for (int q = 0; q < 4; q++) u = __fma_rn(-S.BB[k][r * 4 + q], S.BY[ir][q * 4 + c], u);
        S.BT[k][r * 4 + c] = u;
      } else {
        const int r = e - 32;
        double v = S.bb[k][r];
        if (hl_)
#pragma unroll
          for (int q = 0; q < 4; q++) v = __fma_rn(-S.BB[il][q * 4 + r], S.by[il][q], v);
        if (hr)
#pragma unroll
          for (int q = 0; q < 4; q++) v = __fma_rn(-S.BB[k][r * 4 + q], S.by[ir][q], v);
        S.bb[k][r] = v;
      }
    }
    __syncthreads();
    for (int it = tid; it < nsurv * 16; it += nt) {
      const int k = (it / 16) * 2 * s;
      S.BB[k][it % 16] = S.BT[k][it % 16];
    }
    __syncthreads();
  }
  // block 0 alone (one half-warp), then back substitution
  if (tid < 16) {
    double *M = S.BD[0];
    bool bad = false;
#pragma unroll
    for (int pi = 0; pi < 4; pi++) {
      double dpiv = M[pi * 4 + pi];
      bad = bad || !(dpiv != 0.0) || !isfinite(dpiv);
      double r = 1.0 / dpiv;
      int n = 3 - pi, k = 0, m = 0, q = tid;
      for (int kk = 1; kk <= n; kk++) {
        if (k == 0 && q < n - kk + 1) { k = kk; m = kk + q; }
        else if (k == 0) q -= n - kk + 1;
      }
      double lk = 0.0;
      if (k > 0) {
        lk = M[pi * 4 + pi + k] * r;
        M[(pi + k) * 4 + pi + m] = __fma_rn(-lk, M[pi * 4 + pi + m], M[(pi + k) * 4 + pi + m]);
      }
      __syncwarp(0xffffu);
      if (k > 0 && m == k) M[pi * 4 + pi + k] = lk;
      if (tid == 0) S.br[0][pi] = r;
      __syncwarp(0xffffu);
    }
    if (tid == 0) {
      if (bad) *flag = 1;
      double v[4];
      for (int q = 0; q < 4; q++) v[q] = S.bb[0][q];
      solve4(M, S.br[0], v);
      for (int q = 0; q < 4; q++) S.bx[0][q] = v[q];
    }
  }
  __syncthreads();
  if (*flag) return false;
  for (s = s / 2; s >= 1; s /= 2) {
    const int nelim = (nb - 1 - s) / (2 * s) + 1;
    for (int it = tid; it < nelim * 4; it += nt) {
      const int i = s + 2 * s * (it / 4), r = it % 4;
      double v = S.by[i][r];
#pragma unroll
      for (int q = 0; q < 4; q++) v = __fma_rn(-S.BZ[i][r * 4 + q], S.bx[i - s][q], v);
      if (i + s < nb)
#pragma unroll
        for (int q = 0; q < 4; q++) v = __fma_rn(-S.BY[i][r * 4 + q], S.bx[i + s][q], v);
      S.bx[i][r] = v;
    }
    __syncthreads();
  }
  return true;
}

__global__ void __launch_bounds__(512) k_step(Params P, StepArgs A) {
  extern __shared__ double smem[];
  Smem S = carve(smem, P.n_el);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nd = P.nd, ne = P.n_el;
  const bool clamped = P.clamped != 0;
  const int nf = clamped ? nd - 3 : nd;
  const double dt = A.dt;
  const double c_load = 0.5 * dt * dt, c_stiff = 0.25 * dt * dt;
  const double tc = clamped ? A.ep[2] : 0.0, ts = clamped ? A.ep[3] : 0.0;
  const double dS = P.L / (double)P.nm;

  // tables
  if (tid < 5) {
    double xi = 0.5 + 0.5 * c_gx[tid];
    double wl = 0.5 * c_gw[tid] * P.l;
    double D[4];
    shape_ds(xi, P.l, D);
    for (int i = 0; i < 4; i++) S.D[tid * 4 + i] = D[i];
    for (int i = 0; i < 4; i++)
      for (int j = 0; j < 4; j++) S.PD[(tid * 4 + i) * 4 + j] = wl * D[i] * D[j];
  } else if (tid >= 32 && tid < 48) {
    int q = tid - 32;
    S.Ms[q] = mass_ij(P, q / 4, q % 4);
    S.Kb[q] = bend_ij(P, q / 4, q % 4);
  }
  // state, generalised load (thread per coordinate, markers in order), initial increment
  for (int I = tid; I < nd; I += nt) {
    S.en[I] = A.e[I];
    S.vn[I] = A.v[I];
  }
  for (int I = tid; I < nd; I += nt) {
    int node = I / 4, slot = I % 4, a = slot % 2, slope = slot / 2;
    double q = 0.0;
    for (int side = 0; side < 2; side++) {
      int el = node - 1 + side;
      if (el < 0 || el >= ne) continue;
      int i = side == 0 ? 2 + slope : slope;
      for (int k = A.el_first[el]; k < A.el_first[el + 1]; k++)
        q = q + A.mk_S[4 * k + i] * A.F[a * P.nm + k] * dS;
    }
    S.Qf[I] = q;
    S.d[I] = dt * S.vn[I];
  }
  __syncthreads();
  if (clamped && tid == 0) {
    double sigma = S.en[2] * tc + S.en[3] * ts;
    S.d[0] = A.ep[0] - S.en[0];
    S.d[1] = A.ep[1] - S.en[1];
    S.d[2] = sigma * tc - S.en[2];
    S.d[3] = sigma * ts - S.en[3];
  }
  if (tid == 0) {
    S.flags[0] = 0;  // converged
    S.flags[1] = 0;  // failed
  }
  __syncthreads();

  int it;
  for (it = 1; it <= P.newton_max; it++) {
    for (int I = tid; I < nd; I += nt) {
      S.em[I] = S.en[I] + 0.5 * S.d[I];
      S.g[I] = (clamped && I < 2) ? (0.5 * dt) * (A.vp[I] - S.vn[I]) : S.d[I] - dt * S.vn[I];
    }
    __syncthreads();
    // Gauss-point quantities, one thread per (element, point)
    for (int q = tid; q < 5 * ne; q += nt) {
      int el = q / 5, gp = q % 5;
      const double *ee = S.em + 4 * el;
      const double *D = S.D + gp * 4;
      double rs[2];
      for (int b = 0; b < 2; b++) {
        double t = 0.0;
        for (int j = 0; j < 4; j++) t = __fma_rn(D[j], ee[lc(j, b)], t);
        rs[b] = t;
      }
      double n = sqrt(rs[0] * rs[0] + rs[1] * rs[1]);
      double c1 = P.K_S * (1.0 - 1.0 / n);
      double c2 = P.K_S / (n * n * n);
      double wl = 0.5 * c_gw[gp] * P.l;
      S.gt[el][gp][0] = wl * c1 * rs[0];
      S.gt[el][gp][1] = wl * c1 * rs[1];
      for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
          double sab = c2 * rs[a] * rs[b];
          if (a == b) sab = c1 + sab;
          S.gs[el][gp][a * 2 + b] = sab;
        }
    }
    __syncthreads();
    // element rows: residual entry and the upper part of the Jacobian row
    for (int q = tid; q < 8 * ne; q += nt) {
      int el = q / 8, r = q % 8;
      int i = 2 * (r / 4) + (r % 4) / 2, a = r % 2;
      const double *ee = S.em + 4 * el;
      double bend = 0.0;
      for (int j = 0; j < 4; j++) bend = __fma_rn(S.Kb[i * 4 + j], ee[lc(j, a)], bend);
      double axial = 0.0;
      for (int gp = 0; gp < 5; gp++) axial = __fma_rn(S.gt[el][gp][a], S.D[gp * 4 + i], axial);
      double Qi = bend + axial;
      double inert = 0.0;
      for (int j = 0; j < 4; j++) inert = __fma_rn(S.Ms[i * 4 + j], S.g[4 * el + lc(j, a)], inert);
      S.Rel[el][r] = inert + c_load * Qi;
      for (int c = r; c < 8; c++) {
        int j = 2 * (c / 4) + (c % 4) / 2, b = c % 2;
        double k = 0.0;
        for (int gp = 0; gp < 5; gp++) k = __fma_rn(S.PD[(gp * 4 + i) * 4 + j], S.gs[el][gp][a * 2 + b], k);
        double J;
        if (a == b)
          J = S.Ms[i * 4 + j] + c_stiff * (S.Kb[i * 4 + j] + k);
        else
          J = c_stiff * k;
        S.Jel[el][r * 8 + c] = J;
      }
    }
    __syncthreads();
    // assembly in element order: residual and upper band
    for (int I = tid; I < nd; I += nt) {
      int node = I / 4;
      double r = 0.0;
      double band[BW + 1];
      for (int k = 0; k <= BW; k++) band[k] = 0.0;
      if (node >= 1) {  // element node-1, local row I%4 + 4
        int el = node - 1, rr = I % 4 + 4;
        r = r + S.Rel[el][rr];
        for (int k = 0; rr + k < 8; k++) band[k] = band[k] + S.Jel[el][rr * 8 + rr + k];
      }
      if (node < ne) {  // element node, local row I%4
        int el = node, rr = I % 4;
        r = r + S.Rel[el][rr];
        for (int k = 0; rr + k < 8; k++) band[k] = band[k] + S.Jel[el][rr * 8 + rr + k];
      }
      S.R[I] = r - c_load * S.Qf[I];
      for (int k = 0; k <= BW; k++) S.Ag[I][k] = band[k];
    }
    __syncthreads();
    // the free system in node blocks: -R and D_j, Br_j from the band; a clamped plate's
    // block 0 is sigma with three idle unknowns
    const int nb = ne + 1;
    for (int it = tid; it < nb * 36; it += nt) {
      const int j = it / 36, e = it % 36;
      if (e < 32) {
        const int r = (e % 16) / 4, c = e % 4;
        double v;
        if (e < 16) {  // D_j
          int lo = r < c ? r : c, off = r < c ? c - r : r - c;
          v = S.Ag[4 * j + lo][off];
          if (clamped && j == 0) v = r == c ? 1.0 : 0.0;
          if (clamped && j == 0 && r == 0 && c == 0)
            v = tc * (tc * S.Ag[2][0] + ts * S.Ag[2][1]) + ts * (tc * S.Ag[2][1] + ts * S.Ag[3][0]);
          S.BD[j][r * 4 + c] = v;
        } else {       // Br_j
          v = j + 1 < nb ? S.Ag[4 * j + r][4 + c - r] : 0.0;
          if (clamped && j == 0) v = r == 0 ? tc * S.Ag[2][2 + c] + ts * S.Ag[3][1 + c] : 0.0;
          S.BB[j][r * 4 + c] = v;
        }
      } else {
        const int r = e - 32;
        double v;
        if (clamped)
          v = j == 0 ? (r == 0 ? -(tc * S.R[2] + ts * S.R[3]) : 0.0) : -S.R[4 * j + r];
        else
          v = -S.R[4 * j + r];
        S.bb[j][r] = v;
      }
    }
    __syncthreads();
    {
      bool okb = bcr_solve(S, nb, &S.flags[2]);
      for (int i = tid; i < nf; i += nt) {
        int I = clamped ? (i == 0 ? 0 : i + 3) : i;
        S.x[i] = S.bx[I / 4][I % 4];
      }
      if (tid == 0) S.flags[1] = okb ? 0 : 1;
    }
    __syncthreads();
    if (S.flags[1]) break;
    // update; max |increment| over the warp (exact), a NaN fails
    if (tid < 32) {
      double inc = 0.0;
      int nan = 0;
      for (int i = tid; i < nf; i += 32) {
        double a = fabs(S.x[i]);
        if (isnan(a)) nan = 1;
        else if (a > inc) inc = a;
      }
      for (int o = 16; o > 0; o >>= 1) {
        double t = __shfl_xor_sync(0xffffffffu, inc, o);
        inc = t > inc ? t : inc;
        nan |= __shfl_xor_sync(0xffffffffu, nan, o);
      }
      if (tid == 0) {
        S.flags[1] = nan;
        S.flags[0] = !nan && inc <= P.tol * P.L;
      }
    }
    for (int i = tid; i < nf; i += nt) {
      if (clamped && i == 0) {
        S.d[2] = S.d[2] + tc * S.x[0];
        S.d[3] = S.d[3] + ts * S.x[0];
      } else {
        int I = clamped ? i + 3 : i;
        S.d[I] = S.d[I] + S.x[i];
      }
    }
    __syncthreads();
    if (S.flags[1] || S.flags[0]) break;
  }
  const bool ok = S.flags[0] && !S.flags[1];
  for (int I = tid; I < nd; I += nt) {
    if (clamped && I < 2) {
      A.e[I] = A.ep[I];
      A.v[I] = A.vp[I];
    } else {
      A.e[I] = S.en[I] + S.d[I];
      A.v[I] = (2.0 * S.d[I]) / dt - S.vn[I];
    }
  }
  if (tid == 0) {
    if (!ok) atomicOr(A.status, IBFSA_STATUS_NOCONV);
    atomicMax(A.max_iters, it > P.newton_max ? P.newton_max : it);
  }
}

}  // namespace plate

// ---- host object ---------------------------------------------------------------------------
struct Plate {
  ibfsa_plate_desc d;
  plate::Params P;
  cudaStream_t stream;
  int device;
  double t;
  double *e, *v, *Fbar, *X, *U, *dS;  // workspace
  double *mk_S;                       // marker shape values [nm][4]
  double *res;                        // force [2] and power of the last step
  double *Ustep;                      // marker velocities held during the last step [2][nm]
  int *mk_el, *el_first;              // marker elements [nm], first marker per element
  int *status;                        // [0] flags, [1] max Newton iterations
  int threads;
  size_t smem;
};

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

struct PlateLayout {
  size_t e, v, Fbar, X, U, dS, mk_S, mk_el, el_first, res, Ustep, status, total;
};

static PlateLayout plate_layout(const ibfsa_plate_desc &d) {
  PlateLayout L;
  size_t nd = 4 * (size_t)(d.n_el + 1), nm = (size_t)d.n_markers;
  size_t o = 0;
  L.e = o; o = al256(o + nd * 8);
  L.v = o; o = al256(o + nd * 8);
  L.Fbar = o; o = al256(o + 2 * nm * 8);
  L.X = o; o = al256(o + 2 * nm * 8);
  L.U = o; o = al256(o + 2 * nm * 8);
  L.dS = o; o = al256(o + nm * 8);
  L.mk_S = o; o = al256(o + 4 * nm * 8);
  L.mk_el = o; o = al256(o + nm * sizeof(int));
  L.el_first = o; o = al256(o + (size_t)(d.n_el + 1) * sizeof(int));
  L.res = o; o = al256(o + 3 * sizeof(double));
  L.Ustep = o; o = al256(o + 2 * nm * 8);
  L.status = o; o = al256(o + 2 * sizeof(int));
  L.total = o;
  return L;
}

static int check_plate(const ibfsa_plate_desc *d) {
  if (!d) return api_fail(IBFSA_ERR_ARG, "plate descriptor is NULL");
  if (d->n_el < 1 || d->n_el > IBFSA_PLATE_MAX_EL)
    return api_fail(IBFSA_ERR_ARG, "plate n_el outside [1, IBFSA_PLATE_MAX_EL]");
  if (d->n_markers < 1) return api_fail(IBFSA_ERR_ARG, "plate needs n_markers >= 1");
  if (!(d->length > 0.0) || !(d->rho_s > 0.0) || !(d->K_S >= 0.0) || !(d->K_B >= 0.0))
    return api_fail(IBFSA_ERR_ARG, "plate needs length > 0, rho_s > 0, K_S >= 0, K_B >= 0");
  if (d->clamp != IBFSA_PLATE_FREE && d->clamp != IBFSA_PLATE_CLAMPED)
    return api_fail(IBFSA_ERR_ARG, "plate clamp must be IBFSA_PLATE_FREE or IBFSA_PLATE_CLAMPED");
  if (d->newton_max < 1 || !(d->newton_tol > 0.0))
    return api_fail(IBFSA_ERR_ARG, "plate needs newton_max >= 1 and newton_tol > 0");
  return IBFSA_OK;
}

// Clamp motion of Eq. 17 at time t (host, plain libm): node-0 coordinates and rates.
static void clamp_motion(const ibfsa_plate_desc &p, double t, double e4[4], double v4[4]) {
  const double PI = 3.14159265358979323846;
  double w = 2.0 * PI * p.freq;
  double c = cos(w * t), s = sin(w * t);
  double half = 0.5 * p.A0;
  double cb = cos(p.beta), sb = sin(p.beta);
  double am = 0.5 * p.alpha_m;
  double th = p.theta0 + am * sin(w * t + p.phi);
  double thdot = am * w * cos(w * t + p.phi);
  e4[0] = p.x0[0] + half * c * cb;
  e4[1] = p.x0[1] + half * c * sb;
  e4[2] = cos(th);
  e4[3] = sin(th);
  v4[0] = -(half * w * s) * cb;
  v4[1] = -(half * w * s) * sb;
  v4[2] = -sin(th) * thdot;
  v4[3] = cos(th) * thdot;
}

static int cuda_err(cudaError_t e, const char *where) {
  char msg[256];
  snprintf(msg, sizeof(msg), "%s: %s", where, cudaGetErrorString(e));
  return api_fail(IBFSA_ERR_CUDA, msg);
}

static cudaError_t launch_step(Plate &Pl, double dt, const double *F, Prof *prof) {
  plate::StepArgs a;
  a.dt = dt;
  double t_new = Pl.t + dt;
  clamp_motion(Pl.d, t_new, a.ep, a.vp);
  a.e = Pl.e;
  a.v = Pl.v;
  a.F = F;
  a.mk_S = Pl.mk_S;
  a.el_first = Pl.el_first;
  a.status = Pl.status;
  a.max_iters = Pl.status + 1;
  if (prof) prof_begin(prof, Pl.stream);
  plate::k_step<<<1, Pl.threads, Pl.smem, Pl.stream>>>(Pl.P, a);
  if (prof) prof_end(prof, K_PLATE, Pl.stream);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) Pl.t = t_new;
  return e;
}

}  // namespace ibfsa

using namespace ibfsa;

struct ibfsa_plate {
  Plate p;
};

static bool host_ptr(const void *ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

extern "C" {

int ibfsa_plate_workspace_bytes(const ibfsa_plate_desc *desc, size_t *bytes) {
  int rc = check_plate(desc);
  if (rc) return rc;
  if (!bytes) return api_fail(IBFSA_ERR_ARG, "bytes is NULL");
  *bytes = plate_layout(*desc).total;
  return IBFSA_OK;
}

int ibfsa_plate_create(const ibfsa_plate_desc *desc, void *d_workspace, size_t workspace_bytes,
                       void *cuda_stream, ibfsa_plate **out) {
  int rc = check_plate(desc);
  if (rc) return rc;
  if (!out || !d_workspace) return api_fail(IBFSA_ERR_ARG, "NULL workspace or output");
  PlateLayout L = plate_layout(*desc);
  if (workspace_bytes < L.total || ((uintptr_t)d_workspace & 255))
    return api_fail(IBFSA_ERR_WORKSPACE, "plate workspace too small or not 256-byte aligned");
  ibfsa_plate *h = new (std::nothrow) ibfsa_plate;
  if (!h) return api_fail(IBFSA_ERR_ARG, "out of host memory");
  Plate &P = h->p;
  P.d = *desc;
  P.stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&P.device);
  P.t = 0.0;
  char *ws = (char *)d_workspace;
  P.e = (double *)(ws + L.e);
  P.v = (double *)(ws + L.v);
  P.Fbar = (double *)(ws + L.Fbar);
  P.X = (double *)(ws + L.X);
  P.U = (double *)(ws + L.U);
  P.dS = (double *)(ws + L.dS);
  P.mk_S = (double *)(ws + L.mk_S);
  P.mk_el = (int *)(ws + L.mk_el);
  P.el_first = (int *)(ws + L.el_first);
  P.res = (double *)(ws + L.res);
  P.Ustep = (double *)(ws + L.Ustep);
  P.status = (int *)(ws + L.status);
  P.P.n_el = desc->n_el;
  P.P.nd = 4 * (desc->n_el + 1);
  P.P.nm = desc->n_markers;
  P.P.clamped = desc->clamp == IBFSA_PLATE_CLAMPED;
  P.P.newton_max = desc->newton_max;
  P.P.L = desc->length;
  P.P.l = desc->length / desc->n_el;
  P.P.rho_s = desc->rho_s;
  P.P.K_S = desc->K_S;
  P.P.K_B = desc->K_B;
  P.P.tol = desc->newton_tol;
  int need = 8 * desc->n_el > P.P.nd ? 8 * desc->n_el : P.P.nd;
  P.threads = ((need + 31) / 32) * 32;
  if (P.threads < 64) P.threads = 64;
  if (P.threads > 512) P.threads = 512;
  P.smem = plate::smem_doubles(desc->n_el) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(plate::k_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)P.smem);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.status, 0, 2 * sizeof(int), P.stream);
  if (e == cudaSuccess) {
    int n = (desc->n_markers > desc->n_el + 1 ? desc->n_markers : desc->n_el + 1);
    plate::k_tables<<<(n + 127) / 128, 128, 0, P.stream>>>(P.P, P.mk_el, P.mk_S, P.el_first);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    delete h;
    return cuda_err(e, "ibfsa_plate_create");
  }
  *out = h;
  return IBFSA_OK;
}

int ibfsa_plate_destroy(ibfsa_plate *p) {
  delete p;
  return IBFSA_OK;
}

int ibfsa_plate_set_state(ibfsa_plate *p, const double *e, const double *v, double t) {
  if (!p || !e || !v) return api_fail(IBFSA_ERR_ARG, "NULL argument");
  Plate &P = p->p;
  size_t n = sizeof(double) * P.P.nd;
  cudaError_t err = cudaMemcpyAsync(P.e, e, n, cudaMemcpyDefault, P.stream);
  if (err == cudaSuccess) err = cudaMemcpyAsync(P.v, v, n, cudaMemcpyDefault, P.stream);
  if (err != cudaSuccess) return cuda_err(err, "ibfsa_plate_set_state");
  P.t = t;
  return IBFSA_OK;
}

int ibfsa_plate_get_state(ibfsa_plate *p, double *e, double *v, double *host_t) {
  if (!p) return api_fail(IBFSA_ERR_ARG, "NULL plate");
  Plate &P = p->p;
  size_t n = sizeof(double) * P.P.nd;
  cudaError_t err = cudaSuccess;
  bool sync = false;
  if (e) {
    err = cudaMemcpyAsync(e, P.e, n, cudaMemcpyDefault, P.stream);
    sync = sync || host_ptr(e);
  }
  if (v && err == cudaSuccess) {
    err = cudaMemcpyAsync(v, P.v, n, cudaMemcpyDefault, P.stream);
    sync = sync || host_ptr(v);
  }
  if (err == cudaSuccess && sync) err = cudaStreamSynchronize(P.stream);
  if (err != cudaSuccess) return cuda_err(err, "ibfsa_plate_get_state");
  if (host_t) *host_t = P.t;
  return IBFSA_OK;
}

int ibfsa_plate_step(ibfsa_plate *p, double dt, const double *F) {
  if (!p) return api_fail(IBFSA_ERR_ARG, "NULL plate");
  if (!(dt > 0.0)) return api_fail(IBFSA_ERR_ARG, "plate step needs dt > 0");
  Plate &P = p->p;
  size_t n = sizeof(double) * 2 * P.P.nm;
  cudaError_t err = F ? cudaMemcpyAsync(P.Fbar, F, n, cudaMemcpyDefault, P.stream)
                      : cudaMemsetAsync(P.Fbar, 0, n, P.stream);
  if (err == cudaSuccess) {  // the markers' velocities during the step (for ibfsa_plate_force)
    plate::k_markers<<<(P.P.nm + 127) / 128, 128, 0, P.stream>>>(P.P, P.e, P.v, P.mk_el, P.mk_S,
                                                                 P.X, P.U, P.dS, P.P.nm, P.Ustep);
    err = cudaGetLastError();
  }
  if (err == cudaSuccess) err = launch_step(P, dt, P.Fbar, nullptr);
  return err == cudaSuccess ? IBFSA_OK : cuda_err(err, "ibfsa_plate_step");
}

int ibfsa_plate_markers(ibfsa_plate *p, double *X, double *U, double *dS) {
  if (!p || !X || !U || !dS) return api_fail(IBFSA_ERR_ARG, "NULL argument");
  Plate &P = p->p;
  int nm = P.P.nm;
  plate::k_markers<<<(nm + 127) / 128, 128, 0, P.stream>>>(P.P, P.e, P.v, P.mk_el, P.mk_S, P.X,
                                                           P.U, P.dS, nm, nullptr);
  cudaError_t err = cudaGetLastError();
  size_t n2 = sizeof(double) * 2 * nm;
  if (err == cudaSuccess) err = cudaMemcpyAsync(X, P.X, n2, cudaMemcpyDefault, P.stream);
  if (err == cudaSuccess) err = cudaMemcpyAsync(U, P.U, n2, cudaMemcpyDefault, P.stream);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(dS, P.dS, sizeof(double) * nm, cudaMemcpyDefault, P.stream);
  if (err == cudaSuccess && (host_ptr(X) || host_ptr(U) || host_ptr(dS)))
    err = cudaStreamSynchronize(P.stream);
  return err == cudaSuccess ? IBFSA_OK : cuda_err(err, "ibfsa_plate_markers");
}

int ibfsa_plate_get_status(ibfsa_plate *p, int *host_flags, int *host_max_iters) {
  if (!p) return api_fail(IBFSA_ERR_ARG, "NULL plate");
  Plate &P = p->p;
  int h[2] = {0, 0};
  cudaError_t err = cudaMemcpyAsync(h, P.status, sizeof(h), cudaMemcpyDeviceToHost, P.stream);
  if (err == cudaSuccess) err = cudaMemsetAsync(P.status, 0, sizeof(h), P.stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(P.stream);
  if (err != cudaSuccess) return cuda_err(err, "ibfsa_plate_get_status");
  if (host_flags) *host_flags = h[0];
  if (host_max_iters) *host_max_iters = h[1];
  return IBFSA_OK;
}

int ibfsa_plate_force(ibfsa_plate *p, double *host_force, double *host_power) {
  if (!p || !host_force) return api_fail(IBFSA_ERR_ARG, "NULL argument");
  Plate &P = p->p;
  plate::k_force<<<1, 32, 0, P.stream>>>(P.P, P.Fbar, P.Ustep, P.res);
  double h[3] = {0.0, 0.0, 0.0};
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaMemcpyAsync(h, P.res, sizeof(h), cudaMemcpyDeviceToHost, P.stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(P.stream);
  if (err != cudaSuccess) return cuda_err(err, "ibfsa_plate_force");
  host_force[0] = h[0];
  host_force[1] = h[1];
  if (host_power) *host_power = h[2];
  return IBFSA_OK;
}

int ibfsa_fsi_step(ibfsa_grid *g, ibfsa_plate *p, double dt, int nsteps) {
  if (!g || !p) return api_fail(IBFSA_ERR_ARG, "NULL grid or plate");
  if (nsteps < 0 || !(dt > 0.0)) return api_fail(IBFSA_ERR_ARG, "need dt > 0 and nsteps >= 0");
  Grid &G = g->g;
  Plate &P = p->p;
  if (G.p.dim != 2) return api_fail(IBFSA_ERR_ARG, "the plate couples to a 2D grid");
  if (G.d.max_markers < P.P.nm)
    return api_fail(IBFSA_ERR_ARG, "grid max_markers is smaller than the plate's n_markers");
  if (G.stream != P.stream)
    return api_fail(IBFSA_ERR_ARG, "grid and plate must share one stream");
  if (G.d.scheme == IBFSA_MLP_TENO5 && !G.mlp_set)
    return api_fail(IBFSA_ERR_ARG, "IBFSA_MLP_TENO5 grid without weights: call ibfsa_set_mlp");
  const int M = G.d.max_markers, nm = P.P.nm;
  const double A[3] = {0.0, 3.0 / 4.0, 1.0 / 3.0}, B[3] = {1.0, 1.0 / 4.0, 2.0 / 3.0};
  const double Wt[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
  const double C[3] = {0.0, 1.0, 0.5};  // stage times of the fluid's clock
  for (int step = 0; step < nsteps; step++) {
    prof_begin(&G.prof, G.stream);
    plate::k_markers<<<(nm + 127) / 128, 128, 0, G.stream>>>(P.P, P.e, P.v, P.mk_el, P.mk_S,
                                                             G.X, G.U, G.dS, M, P.Ustep);
    prof_end(&G.prof, K_PLATE, G.stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "ibfsa_fsi_step markers");
    G.p.nm = nm;
    const double *in[3] = {G.Q, G.Q1, G.Q2};
    double *outs[3] = {G.Q1, G.Q2, G.Q};
    const double *xin[3] = {G.xi, G.xi1, G.xi2};
    double *xout[3] = {G.xi1, G.xi2, G.xi};
    for (int s = 0; s < 3; s++) {
      StageArgs a{};
      a.Qs = in[s];
      a.Qn = G.Q;
      a.Qo = outs[s];
      a.xis = xin[s];
      a.xin = G.xi;
      a.xio = xout[s];
      a.a = A[s];
      a.b = B[s];
      a.dt = dt;
      a.stage = s;
      a.src_scale = source_scale(G, G.t + C[s] * dt);
      a.prof = &G.prof;
      e = grid_stage(&G, a);
      if (e != cudaSuccess) return cuda_err(e, "ibfsa_fsi_step stage");
      prof_begin(&G.prof, G.stream);
      plate::k_force_average<<<(2 * nm + 127) / 128, 128, 0, G.stream>>>(nm, G.p.F, M, P.Fbar,
                                                                          Wt[s], s == 0);
      prof_end(&G.prof, K_PLATE, G.stream);
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_err(e, "ibfsa_fsi_step force average");
    }
    e = launch_step(P, dt, P.Fbar, &G.prof);
    if (e != cudaSuccess) return cuda_err(e, "ibfsa_fsi_step plate");
    G.t = G.t + dt;
  }
  return IBFSA_OK;
}

}  // extern "C"
