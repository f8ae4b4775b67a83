/*
 * ibfsa_oracle.c -- plain, slow FP64 CPU oracle of the IB-WENO/TENO stage right-hand side
 * (Wang, Tian & Lai, "An immersed boundary method for fluid-structure-acoustics interactions
 * involving large deformations and complex geometries", arXiv:1905.00182, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this file:
 * only the test suite, the smoke check and the bench's CPU-baseline leg use it.  It shares no
 * source, header, table or helper with the CUDA path.
 *
 * Every step is written as a direct loop over a ghost-padded FP64 array, in the order the
 * method states it (compile with -O2 -ffp-contract=off so that no multiply-add is fused).
 * On a stretched grid (the non-uniform mesh of Sec. 2, given as node coordinates and dx/dxi per
 * direction) every difference is taken in the computational coordinate and divided by dx/dxi:
 *
 *   1. ghost fill (4 layers) per boundary rule                 (readings: zero-gradient,
 *                                                                free stream, periodic; a
 *      characteristic face copies its boundary cell, whose normal convective term is then the
 *      characteristic form of Thompson's non-reflecting condition, Sec. 2)
 *   2. alpha_d = max over interior of |u_d| + c                 (global Lax-Friedrichs split)
 *   3. convective term: f+- = (F_d(Q) +- alpha_d Q)/2, fifth-order WENO5-JS or TENO5
 *      reconstruction of every component at every face (or, as an option, of every
 *      characteristic field at the face's Roe average), then -(Fhat_{i+1/2}-Fhat_{i-1/2})/h
 *                                                                (Sec. 2, Eq. 2 and the text
 *                                                                after Eq. 5); or the learned
 *      weights: TENO5's cut-off decides, and where it keeps all three candidates (and the
 *      stencil is not flat) a network gives their weights, the face value taken in delta form
 *   4. viscous term: 4th-order central gradients of u, tau_ij, b = u.tau (no heat flux),
 *      then (1/Re) * 4th-order central divergence of [0, tau_.j, b_j] (Eq. 2-5)
 *   5. optional sponge: L -= sigma(n) (Q - Q_inf); optional periodic Gaussian pressure source
 *      of Sec. 3.6 (Eq. 16) in the energy equation
 *   6. immersed boundary: U_ib(X_k) = sum_j u_j delta_h (X_k - x_j) h^d        (Eq. 8)
 *      F_k = alpha_pen xi_k + beta_pen (U_ib - U_k)                           (Eq. 7)
 *      f_j = - sum_k F_k delta_h(X_k - x_j) dS_k   (in marker order)          (Eq. 9)
 *      delta_h = prod_d lambda(x_d/h_d)/h_d with Peskin's 4-point lambda       (Eq. 10, 11)
 *      S = [0, f, f.u] added to L
 *   7. third-order TVD Runge-Kutta (Shu-Osher) on Q and on xi = int (U_ib - U) dt
 *
 * Parity pins (tests): Peskin-kernel moment identities, interpolation/spreading adjointness and
 * exact force conservation, linear reproduction of WENO/TENO on equal smoothness indicators,
 * TENO's ENO cut-off on a step, fifth-order convergence of the reconstruction, fourth-order
 * convergence of the viscous operator against the continuous PDE, free-stream preservation,
 * entropy-wave exact solution, third-order RK3, convergence of the Sec. 3.1 pulse to the exact
 * linear-acoustics solution, and penalty enforcement of no slip; for the characteristic-wise
 * option, the eigen-system against the flux Jacobian, Roe's property of the face average and
 * Sod's shock tube against the exact Riemann solution.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NG 4 /* ghost layers: viscous D4 of D4 reaches +-4 */

#include "ibfsa_oracle.h"

/* ----------------------------------------------------------------------------------------- */
/* Peskin 4-point kernel, Eq. 11                                                              */
/* ----------------------------------------------------------------------------------------- */
double orc_lambda(double r) {
  double a = fabs(r);
  if (a < 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
  if (a < 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
  return 0.0;
}

/* ----------------------------------------------------------------------------------------- */
/* Fifth-order reconstructions at face i+1/2 from v = (f_{i-2}, f_{i-1}, f_i, f_{i+1}, f_{i+2}) */
/* (upwind-biased to the left; the right-going split flux uses the mirrored stencil).         */
/* Three third-order candidates on the sub-stencils {i-2..i}, {i-1..i+1}, {i..i+2}, their     */
/* Jiang-Shu smoothness indicators and the optimal (linear) weights 1/10, 6/10, 3/10.          */
/* ----------------------------------------------------------------------------------------- */
static void candidates(const double *v, double q[3], double beta[3]) {
  double a = v[0], b = v[1], c = v[2], d = v[3], e = v[4];
  q[0] = (2.0 * a - 7.0 * b + 11.0 * c) / 6.0;
  q[1] = (-b + 5.0 * c + 2.0 * d) / 6.0;
  q[2] = (2.0 * c + 5.0 * d - e) / 6.0;
  double t;
  t = a - 2.0 * b + c;       beta[0] = 13.0 / 12.0 * t * t;
  t = a - 4.0 * b + 3.0 * c; beta[0] += 0.25 * t * t;
  t = b - 2.0 * c + d;       beta[1] = 13.0 / 12.0 * t * t;
  t = b - d;                 beta[1] += 0.25 * t * t;
  t = c - 2.0 * d + e;       beta[2] = 13.0 / 12.0 * t * t;
  t = 3.0 * c - 4.0 * d + e; beta[2] += 0.25 * t * t;
}

static const double DLIN[3] = {0.1, 0.6, 0.3};

/* WENO5-JS: alpha_k = d_k/(eps + beta_k)^2, eps = 1e-6, omega = alpha / sum(alpha). */
double orc_weno5js(const double *v) {
  double q[3], beta[3], al[3];
  candidates(v, q, beta);
  const double eps = 1e-6;
  for (int k = 0; k < 3; k++) al[k] = DLIN[k] / ((eps + beta[k]) * (eps + beta[k]));
  double s = al[0] + al[1] + al[2];
  return (al[0] / s) * q[0] + (al[1] / s) * q[1] + (al[2] / s) * q[2];
}

/* TENO5 (Fu, Hu & Adams 2016 defaults): tau5 = |beta_0 - beta_2|,
 * gamma_k = (C + tau5/(beta_k + eps))^q with C = 1, q = 6, eps = 1e-40,
 * chi_k = gamma_k / sum(gamma), delta_k = [chi_k >= C_T] with C_T = 1e-5,
 * omega_k = d_k delta_k / sum(d_j delta_j). */
double orc_teno5(const double *v) {
  double q[3], beta[3], g[3];
  candidates(v, q, beta);
  const double eps = 1e-40, CT = 1e-5;
  double tau5 = fabs(beta[0] - beta[2]);
  for (int k = 0; k < 3; k++) {
    double x = 1.0 + tau5 / (beta[k] + eps);
    double x2 = x * x;
    g[k] = x2 * x2 * x2;
  }
  double s = g[0] + g[1] + g[2];
  double w[3], sw = 0.0;
  for (int k = 0; k < 3; k++) {
    double chi = g[k] / s;
    w[k] = (chi >= CT) ? DLIN[k] : 0.0;
    sw += w[k];
  }
  return (w[0] / sw) * q[0] + (w[1] / sw) * q[1] + (w[2] / sw) * q[2];
}

/* ----------------------------------------------------------------------------------------- */
/* Learned reconstruction weights (the learned-weight variant of the fifth-order              */
/* reconstruction): TENO5 decides where the data is smooth; there a small network maps the     */
/* normalised stencil to the three weights of the same third-order candidates.                */
/* ----------------------------------------------------------------------------------------- */
/* nearest bfloat16 (ties to even) of x, through its nearest float */
static double bf16_round(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, sizeof(u));
  if ((u & 0x7f800000u) != 0x7f800000u) {
    uint32_t lsb = (u >> 16) & 1u;
    u = (u + 0x7fffu + lsb) & 0xffff0000u;
    memcpy(&f, &u, sizeof(f));
  }
  return (double)f;
}

/* gelu, tanh form: z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) */
static double gelu(double z) {
  const double k = 0.79788456080286535588; /* sqrt(2/pi) */
  return 0.5 * z * (1.0 + tanh(k * (z + 0.044715 * z * z * z)));
}

/* one dense layer: out[i] = b[i] + sum_j W[i][j] in[j], W row-major (nout x nin) */
static void dense(const double *W, const double *b, int nout, int nin, const double *in,
                  double *out) {
  for (int i = 0; i < nout; i++) {
    double s = b[i];
    for (int j = 0; j < nin; j++) s = s + W[i * nin + j] * in[j];
    out[i] = s;
  }
}

/* the network's three softmax weights for the normalised stencil x[5] */
void orc_mlp_weights(const double *theta, int round_act, const double *x, double w[3]) {
  const double *W1 = theta, *b1 = W1 + 160, *W2 = b1 + 32, *b2 = W2 + 1024, *W3 = b2 + 32,
               *b3 = W3 + 1024, *W4 = b3 + 32, *b4 = W4 + 96;
  double a0[5], z[32], h1[32], h2[32], h3[32], l[3];
  for (int j = 0; j < 5; j++) a0[j] = round_act ? bf16_round(x[j]) : x[j];
  dense(W1, b1, 32, 5, a0, z);
  for (int i = 0; i < 32; i++) h1[i] = round_act ? bf16_round(gelu(z[i])) : gelu(z[i]);
  dense(W2, b2, 32, 32, h1, z);
  for (int i = 0; i < 32; i++) h2[i] = round_act ? bf16_round(gelu(z[i])) : gelu(z[i]);
  dense(W3, b3, 32, 32, h2, z);
  for (int i = 0; i < 32; i++) h3[i] = round_act ? bf16_round(gelu(z[i])) : gelu(z[i]);
  dense(W4, b4, 3, 32, h3, l);
  double m = l[0] > l[1] ? l[0] : l[1];
  if (l[2] > m) m = l[2];
  double e0 = exp(l[0] - m), e1 = exp(l[1] - m), e2 = exp(l[2] - m);
  double s = e0 + e1 + e2;
  w[0] = e0 / s;
  w[1] = e1 / s;
  w[2] = e2 / s;
}

/* TENO5's cut-off decision alone: 1 when every stencil is kept (the constants of orc_teno5) */
static int teno5_all_kept(const double *v) {
  double q[3], beta[3], g[3];
  candidates(v, q, beta);
  const double eps = 1e-40, CT = 1e-5;
  double tau5 = fabs(beta[0] - beta[2]);
  for (int k = 0; k < 3; k++) {
    double x = 1.0 + tau5 / (beta[k] + eps);
    double x2 = x * x;
    g[k] = x2 * x2 * x2;
  }
  double s = g[0] + g[1] + g[2];
  for (int k = 0; k < 3; k++)
    if (!(g[k] / s >= CT)) return 0;
  return 1;
}

/* Learned reconstruction at the face from v[5] (upwind-ordered); *used (may be NULL) = 1 when
 * the network supplied the weights, 0 when TENO5 did. */
double orc_learned_recon(const double *theta, int round_act, double floor_amp, const double *v,
                         int *used) {
  if (used) *used = 0;
  if (!teno5_all_kept(v)) return orc_teno5(v);
  double amp = 0.0;
  for (int j = 0; j < 5; j++) {
    double dj = fabs(v[j] - v[2]);
    if (dj > amp) amp = dj;
  }
  if (!(amp > floor_amp)) return orc_teno5(v);
  double x[5], q[3], beta[3], w[3];
  for (int j = 0; j < 5; j++) x[j] = (v[j] - v[2]) / amp;
  candidates(x, q, beta); /* candidates of the normalised stencil (x_2 = 0) */
  orc_mlp_weights(theta, round_act, x, w);
  if (used) *used = 1;
  return v[2] + amp * (w[0] * q[0] + w[1] * q[1] + w[2] * q[2]);
}

/* reconstructions that used the network / all learned reconstructions of the last orc_rhs */
static long long g_mlp_used, g_mlp_seen;

void orc_mlp_counts(long long *used, long long *seen) {
  *used = g_mlp_used;
  *seen = g_mlp_seen;
}

static double recon_d(const orc_desc *d, const double *v) {
  if (d->scheme == 2) {
    int used = 0;
    double r = orc_learned_recon(d->mlp_params, d->mlp_round, d->mlp_floor, v, &used);
    g_mlp_used += used;
    g_mlp_seen += 1;
    return r;
  }
  return d->scheme == 1 ? orc_teno5(v) : orc_weno5js(v);
}

/* ----------------------------------------------------------------------------------------- */
/* Padded grid helpers                                                                       */
/* ----------------------------------------------------------------------------------------- */
typedef struct {
  int dim, nv;
  int n[3];
  int P[3];   /* padded extents */
  int g[3];   /* ghost layers per direction (0 for an inactive z) */
  size_t N;   /* padded cell count */
  double h[3];
  double lo[3];
  const double *xn[3], *xm[3]; /* stretched grid (NULL: uniform) */
} pgrid;

static void pgrid_init(pgrid *G, const orc_desc *d) {
  G->dim = d->dim;
  G->nv = d->dim + 2;
  G->N = 1;
  for (int a = 0; a < 3; a++) {
    int act = a < d->dim;
    G->n[a] = act ? d->n[a] : 1;
    G->g[a] = act ? NG : 0;
    G->P[a] = G->n[a] + 2 * G->g[a];
    G->N *= (size_t)G->P[a];
    G->h[a] = act ? (d->hi[a] - d->lo[a]) / d->n[a] : 1.0;
    G->lo[a] = d->lo[a];
    G->xn[a] = act ? d->xnode[a] : NULL;
    G->xm[a] = act ? d->xmetric[a] : NULL;
  }
}

/* dx/dxi at node i of direction a (the spacing h on a uniform grid) */
static double met(const pgrid *G, int a, int i) {
  return G->xm[a] ? G->xm[a][i + NG] : G->h[a];
}

/* coordinate of node i of direction a */
static double node(const pgrid *G, int a, int i) {
  return G->xn[a] ? G->xn[a][i + NG] : G->lo[a] + ((double)i + 0.5) * G->h[a];
}

/* linear offset of cell (i,j,k), interior-based indices (may be negative down to -g) */
static size_t pidx(const pgrid *G, int i, int j, int k) {
  return ((size_t)(k + G->g[2]) * G->P[1] + (size_t)(j + G->g[1])) * G->P[0] + (size_t)(i + G->g[0]);
}

/* interior (unpadded) offset, layout [nz][ny][nx] */
static size_t uidx(const pgrid *G, int i, int j, int k) {
  return ((size_t)k * G->n[1] + (size_t)j) * G->n[0] + (size_t)i;
}

/* Copy the interior state in and fill ghosts direction by direction (x, then y over the
 * x-padded range, then z over the xy-padded range), so corner ghosts compose the rules. */
static void fill_padded(const pgrid *G, const orc_desc *d, const double *Q, double *W) {
  size_t Nu = (size_t)G->n[0] * G->n[1] * G->n[2];
  for (int c = 0; c < G->nv; c++)
    for (int k = 0; k < G->n[2]; k++)
      for (int j = 0; j < G->n[1]; j++)
        for (int i = 0; i < G->n[0]; i++)
          W[c * G->N + pidx(G, i, j, k)] = Q[c * Nu + uidx(G, i, j, k)];
  for (int a = 0; a < G->dim; a++) {
    /* ranges of the other two directions: padded if already filled (lower a), else interior */
    int lo_[3], hi_[3];
    for (int b = 0; b < 3; b++) {
      if (b < a) { lo_[b] = -G->g[b]; hi_[b] = G->n[b] + G->g[b]; }
      else { lo_[b] = 0; hi_[b] = G->n[b]; }
    }
    for (int side = 0; side < 2; side++) {
      int rule = d->bc[a][side];
      for (int l = 1; l <= NG; l++) {
        int gi = side == 0 ? -l : G->n[a] - 1 + l; /* ghost index along a */
        int src;
        if (rule == 0 || rule == 3) src = side == 0 ? 0 : G->n[a] - 1;
        else if (rule == 2) src = side == 0 ? G->n[a] - l : l - 1;
        else src = -1;
        int I[3];
        for (I[2] = (a == 2 ? 0 : lo_[2]); I[2] < (a == 2 ? 1 : hi_[2]); I[2]++)
          for (I[1] = (a == 1 ? 0 : lo_[1]); I[1] < (a == 1 ? 1 : hi_[1]); I[1]++)
            for (I[0] = (a == 0 ? 0 : lo_[0]); I[0] < (a == 0 ? 1 : hi_[0]); I[0]++) {
              int T[3] = {I[0], I[1], I[2]}, S[3] = {I[0], I[1], I[2]};
              T[a] = gi;
              S[a] = src;
              for (int c = 0; c < G->nv; c++) {
                double val = rule == 1 ? d->qinf[c] : W[c * G->N + pidx(G, S[0], S[1], S[2])];
                W[c * G->N + pidx(G, T[0], T[1], T[2])] = val;
              }
            }
      }
    }
  }
}

/* primitives on the padded grid: rho, u_a = m_a / rho, p = (gamma-1)(E - m.u/2) */
static void primitives(const pgrid *G, const orc_desc *d, const double *W, double *rho,
                       double *u /* [3][N] */, double *p) {
  int nv = G->nv, dim = G->dim;
  for (size_t s = 0; s < G->N; s++) {
    double r = W[0 * G->N + s];
    double ke = 0.0;
    for (int a = 0; a < 3; a++) {
      double ua = a < dim ? W[(1 + a) * G->N + s] / r : 0.0;
      u[a * G->N + s] = ua;
      if (a < dim) ke += W[(1 + a) * G->N + s] * ua;
    }
    rho[s] = r;
    p[s] = (d->gamma - 1.0) * (W[(nv - 1) * G->N + s] - 0.5 * ke);
  }
}

/* ----------------------------------------------------------------------------------------- */
/* Global Lax-Friedrichs speeds alpha_d = max_interior(|u_d| + c), c = sqrt(gamma p / rho)    */
/* ----------------------------------------------------------------------------------------- */
static void wavespeeds(const pgrid *G, const orc_desc *d, const double *rho, const double *u,
                       const double *p, double alpha[3]) {
  for (int a = 0; a < 3; a++) alpha[a] = 0.0;
  for (int k = 0; k < G->n[2]; k++)
    for (int j = 0; j < G->n[1]; j++)
      for (int i = 0; i < G->n[0]; i++) {
        size_t s = pidx(G, i, j, k);
        double c = sqrt(d->gamma * p[s] / rho[s]);
        for (int a = 0; a < G->dim; a++) {
          double w = fabs(u[a * G->N + s]) + c;
          if (w > alpha[a]) alpha[a] = w;
        }
      }
}

/* physical flux component c of direction a at padded cell s (Eq. 3-4):
 * [m_a, m_1 u_a + p delta_1a, ..., (E + p) u_a] */
static double flux(const pgrid *G, const double *W, const double *u, const double *p, int a, int c,
                   size_t s) {
  int nv = G->nv;
  double ua = u[a * G->N + s];
  if (c == 0) return W[(1 + a) * G->N + s];
  if (c == nv - 1) return (W[(nv - 1) * G->N + s] + p[s]) * ua;
  double v = W[c * G->N + s] * ua;
  if (c - 1 == a) v += p[s];
  return v;
}

/* ----------------------------------------------------------------------------------------- */
/* Characteristic non-reflecting boundaries (Sec. 2, after Thompson): on a face whose rule is  */
/* 3, the ghosts copy the boundary cell (for the stencils that reach them), and at the         */
/* boundary cell the convective term normal to the face is taken from the characteristic form  */
/* of the Euler equations along the normal: wave amplitudes from one-sided derivatives of the  */
/* primitives, those of the waves entering the domain set to zero.                             */
/* ----------------------------------------------------------------------------------------- */
/* 1 when cell m of direction a (of na cells) is the boundary cell of a characteristic face */
static int char_cell(const orc_desc *d, int a, int m, int na) {
  return (m == 0 && d->bc[a][0] == 3) || (m == na - 1 && d->bc[a][1] == 3);
}

/* d/dx_a of a padded field phi at interior cell I by the fourth-order one-sided difference
 * into the domain (s = +1 from the low face, -1 from the high face), divided by dx/dxi:
 *   (-25 f0 + 48 f1 - 36 f2 + 16 f3 - 3 f4)/12, written on the differences f_k - f0 (the
 *   weights sum to zero) so that a constant field gives exactly zero */
static double one_sided(const pgrid *G, const double *phi, const int I[3], int a, int s) {
  const double c[5] = {0.0, 48.0, -36.0, 16.0, -3.0};
  double f0 = phi[pidx(G, I[0], I[1], I[2])];
  double acc = 0.0;
  for (int k = 1; k < 5; k++) {
    int J[3] = {I[0], I[1], I[2]};
    J[a] += s * k;
    acc = acc + c[k] * (phi[pidx(G, J[0], J[1], J[2])] - f0);
  }
  return (double)s * acc / (12.0 * met(G, a, I[a]));
}

/* (d F_a / d x_a) at the boundary cell I of the face (a, side) in characteristic form:
 *   L1 = (u - c)(p_x - rho c u_x), L2 = u (c^2 rho_x - p_x), L_t = u (u_t)_x,
 *   L5 = (u + c)(p_x + rho c u_x), u = u_a, x = x_a, u_t the transverse velocities;
 * an amplitude whose speed (u - c, u, u + c) points into the domain is set to zero; then
 *   d1 = (L2 + (L5 + L1)/2)/c^2, d2 = (L5 + L1)/2, d3 = (L5 - L1)/(2 rho c), d_t = L_t
 * are the rates of rho, p, u_a, u_t, and the conservative form is
 *   [d1, u_b d1 + rho d_b (d_a = d3), |u|^2/2 d1 + d2/(gamma - 1) + rho sum_b u_b d_b]. */
static void char_flux_derivative(const pgrid *G, const orc_desc *d, const double *rho,
                                 const double *u, const double *p, const int I[3], int a,
                                 int side, double *out) {
  int dim = G->dim, nv = G->nv;
  int s = side == 0 ? 1 : -1;
  size_t o = pidx(G, I[0], I[1], I[2]);
  double r = rho[o], pr = p[o];
  double c = sqrt(d->gamma * pr / r);
  double ua = u[a * G->N + o];
  double rx = one_sided(G, rho, I, a, s);
  double px = one_sided(G, p, I, a, s);
  double uxa = one_sided(G, u + a * G->N, I, a, s);
  double lam1 = ua - c, lam2 = ua, lam5 = ua + c;
  /* a speed points into the domain when it has the sign of s (low face: > 0) */
  double L1 = (lam1 * (double)s > 0.0) ? 0.0 : lam1 * (px - r * c * uxa);
  double L2 = (lam2 * (double)s > 0.0) ? 0.0 : lam2 * (c * c * rx - px);
  double L5 = (lam5 * (double)s > 0.0) ? 0.0 : lam5 * (px + r * c * uxa);
  double dv[3] = {0.0, 0.0, 0.0}; /* rates of the velocities: d3 along a, d_t across */
  for (int b = 0; b < dim; b++) {
    if (b == a) continue;
    double utx = one_sided(G, u + b * G->N, I, a, s);
    dv[b] = (lam2 * (double)s > 0.0) ? 0.0 : lam2 * utx;
  }
  double d1 = (L2 + 0.5 * (L5 + L1)) / (c * c);
  double d2 = 0.5 * (L5 + L1);
  dv[a] = (L5 - L1) / (2.0 * r * c);
  double ke = 0.0, work = 0.0;
  out[0] = d1;
  for (int b = 0; b < dim; b++) {
    double ub = u[b * G->N + o];
    out[1 + b] = ub * d1 + r * dv[b];
    ke = ke + ub * ub;
    work = work + ub * dv[b];
  }
  out[nv - 1] = 0.5 * ke * d1 + d2 / (d->gamma - 1.0) + r * work;
}

/* L -= (dF_a/dx_a)_char at the boundary cells of every characteristic face */
static void characteristic_faces(const pgrid *G, const orc_desc *d, const double *rho,
                                 const double *u, const double *p, double *L) {
  int nv = G->nv;
  size_t Nu = (size_t)G->n[0] * G->n[1] * G->n[2];
  for (int a = 0; a < G->dim; a++)
    for (int side = 0; side < 2; side++) {
      if (d->bc[a][side] != 3) continue;
      int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
      for (int t2 = 0; t2 < G->n[b2]; t2++)
        for (int t1 = 0; t1 < G->n[b1]; t1++) {
          int I[3];
          I[a] = side == 0 ? 0 : G->n[a] - 1;
          I[b1] = t1;
          I[b2] = t2;
          double D[5];
          char_flux_derivative(G, d, rho, u, p, I, a, side, D);
          for (int c = 0; c < nv; c++) {
            size_t o = c * Nu + uidx(G, I[0], I[1], I[2]);
            L[o] = L[o] - D[c];
          }
        }
    }
}

/* ----------------------------------------------------------------------------------------- */
/* Convective term, component-wise reconstruction of the globally split fluxes               */
/* ----------------------------------------------------------------------------------------- */
static void convective(const pgrid *G, const orc_desc *d, const double *W, const double *u,
                       const double *p, const double alpha[3], double *L) {
  int nv = G->nv;
  size_t Nu = (size_t)G->n[0] * G->n[1] * G->n[2];
  for (int a = 0; a < G->dim; a++) {
    int na = G->n[a];
    double *fp = malloc(sizeof(double) * (na + 2 * NG));
    double *fm = malloc(sizeof(double) * (na + 2 * NG));
    double *Fh = malloc(sizeof(double) * (na + 1));
    int b1 = (a + 1) % 3, b2 = (a + 2) % 3; /* transverse directions */
    for (int t2 = 0; t2 < G->n[b2]; t2++)
      for (int t1 = 0; t1 < G->n[b1]; t1++)
        for (int c = 0; c < nv; c++) {
          for (int l = -NG; l < na + NG; l++) {
            int I[3];
            I[a] = l; I[b1] = t1; I[b2] = t2;
            size_t s = pidx(G, I[0], I[1], I[2]);
            double F = flux(G, W, u, p, a, c, s);
            double q = W[c * G->N + s];
            fp[l + NG] = 0.5 * (F + alpha[a] * q);
            fm[l + NG] = 0.5 * (F - alpha[a] * q);
          }
          /* face m+1/2 for m = -1 .. na-1, stored at Fh[m+1] */
          for (int m = -1; m < na; m++) {
            double vp[5], vm[5];
            for (int r = 0; r < 5; r++) {
              vp[r] = fp[m - 2 + r + NG];   /* f+_{m-2..m+2} */
              vm[r] = fm[m + 3 - r + NG];   /* f-_{m+3..m-1} (mirrored) */
            }
            Fh[m + 1] = recon_d(d, vp) + recon_d(d, vm);
          }
          for (int m = 0; m < na; m++) {
            if (char_cell(d, a, m, na)) continue; /* its normal term: characteristic_faces */
            int I[3];
            I[a] = m; I[b1] = t1; I[b2] = t2;
            size_t o = c * Nu + uidx(G, I[0], I[1], I[2]);
            L[o] = L[o] - (Fh[m + 1] - Fh[m]) / met(G, a, m);
          }
        }
    free(fp); free(fm); free(Fh);
  }
}

/* ----------------------------------------------------------------------------------------- */
/* Characteristic-wise variant: the split fluxes of the stencil are projected on the left      */
/* eigenvectors of the Euler flux Jacobian along the face normal (Roe average of the face's    */
/* two cells), each characteristic field is reconstructed as above, and the face flux is       */
/* projected back with the right eigenvectors.  The splitting stays the global one.            */
/* ----------------------------------------------------------------------------------------- */
int orc_char_eigen(int dim, double gamma, int a, const double *Ql, const double *Qr, double *R,
                   double *Lv, double *lam) {
  if ((dim != 2 && dim != 3) || a < 0 || a >= dim || !(gamma > 1.0)) return ORC_ERR_ARG;
  int nv = dim + 2;
  if (!(Ql[0] > 0.0) || !(Qr[0] > 0.0)) return ORC_ERR_ARG;
  /* Roe average: sqrt(rho)-weighted velocity and total enthalpy */
  double sl = sqrt(Ql[0]), sr = sqrt(Qr[0]);
  double u[3] = {0.0, 0.0, 0.0}, kel = 0.0, ker = 0.0;
  for (int b = 0; b < dim; b++) {
    double ul = Ql[1 + b] / Ql[0], ur = Qr[1 + b] / Qr[0];
    u[b] = (sl * ul + sr * ur) / (sl + sr);
    kel = kel + Ql[1 + b] * ul;
    ker = ker + Qr[1 + b] * ur;
  }
  double pl = (gamma - 1.0) * (Ql[nv - 1] - 0.5 * kel);
  double pr = (gamma - 1.0) * (Qr[nv - 1] - 0.5 * ker);
  double Hl = (Ql[nv - 1] + pl) / Ql[0], Hr = (Qr[nv - 1] + pr) / Qr[0];
  double H = (sl * Hl + sr * Hr) / (sl + sr);
  double q2 = 0.0;
  for (int b = 0; b < dim; b++) q2 = q2 + u[b] * u[b];
  double c2 = (gamma - 1.0) * (H - 0.5 * q2);
  if (!(c2 > 0.0)) return ORC_ERR_ARG;
  double c = sqrt(c2);
  double b1 = (gamma - 1.0) / c2, b2 = 0.5 * q2 * b1;
  double ua = u[a];
  /* transverse directions in increasing order */
  int tr[2], nt = 0;
  for (int b = 0; b < dim; b++)
    if (b != a) tr[nt++] = b;
  for (int i = 0; i < nv * nv; i++) {
    R[i] = 0.0;
    Lv[i] = 0.0;
  }
  /* columns of R (entry [row * nv + col]) */
  int km = 0, ke = 1, kp = nv - 1;
  R[0 * nv + km] = 1.0;
  R[0 * nv + ke] = 1.0;
  R[0 * nv + kp] = 1.0;
  for (int b = 0; b < dim; b++) {
    R[(1 + b) * nv + km] = u[b] - (b == a ? c : 0.0);
    R[(1 + b) * nv + ke] = u[b];
    R[(1 + b) * nv + kp] = u[b] + (b == a ? c : 0.0);
  }
  R[(nv - 1) * nv + km] = H - ua * c;
  R[(nv - 1) * nv + ke] = 0.5 * q2;
  R[(nv - 1) * nv + kp] = H + ua * c;
  for (int t = 0; t < nt; t++) {
    R[(1 + tr[t]) * nv + 2 + t] = 1.0;
    R[(nv - 1) * nv + 2 + t] = u[tr[t]];
  }
  /* rows of L */
  Lv[km * nv + 0] = 0.5 * (b2 + ua / c);
  Lv[kp * nv + 0] = 0.5 * (b2 - ua / c);
  Lv[ke * nv + 0] = 1.0 - b2;
  for (int b = 0; b < dim; b++) {
    Lv[km * nv + 1 + b] = 0.5 * (-b1 * u[b] - (b == a ? 1.0 / c : 0.0));
    Lv[kp * nv + 1 + b] = 0.5 * (-b1 * u[b] + (b == a ? 1.0 / c : 0.0));
    Lv[ke * nv + 1 + b] = b1 * u[b];
  }
  Lv[km * nv + nv - 1] = 0.5 * b1;
  Lv[kp * nv + nv - 1] = 0.5 * b1;
  Lv[ke * nv + nv - 1] = -b1;
  for (int t = 0; t < nt; t++) {
    Lv[(2 + t) * nv + 0] = -u[tr[t]];
    Lv[(2 + t) * nv + 1 + tr[t]] = 1.0;
  }
  if (lam) {
    lam[km] = ua - c;
    lam[kp] = ua + c;
    for (int k = 1; k < nv - 1; k++) lam[k] = ua;
  }
  return ORC_OK;
}

static int convective_charwise(const pgrid *G, const orc_desc *d, const double *W,
                               const double *u, const double *p, const double alpha[3],
                               double *L) {
  int nv = G->nv;
  size_t Nu = (size_t)G->n[0] * G->n[1] * G->n[2];
  for (int a = 0; a < G->dim; a++) {
    int na = G->n[a], len = na + 2 * NG;
    double *fp = malloc(sizeof(double) * nv * len);
    double *fm = malloc(sizeof(double) * nv * len);
    double *Fh = malloc(sizeof(double) * nv * (na + 1));
    int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
    for (int t2 = 0; t2 < G->n[b2]; t2++)
      for (int t1 = 0; t1 < G->n[b1]; t1++) {
        for (int l = -NG; l < na + NG; l++) {
          int I[3];
          I[a] = l; I[b1] = t1; I[b2] = t2;
          size_t s = pidx(G, I[0], I[1], I[2]);
          for (int c = 0; c < nv; c++) {
            double F = flux(G, W, u, p, a, c, s);
            double q = W[c * G->N + s];
            fp[c * len + l + NG] = 0.5 * (F + alpha[a] * q);
            fm[c * len + l + NG] = 0.5 * (F - alpha[a] * q);
          }
        }
        for (int m = -1; m < na; m++) {
          /* the face between cells m and m+1 */
          double Ql[5], Qr[5], R[25], Lv[25];
          int I[3];
          I[a] = m; I[b1] = t1; I[b2] = t2;
          size_t sl = pidx(G, I[0], I[1], I[2]);
          I[a] = m + 1;
          size_t sr = pidx(G, I[0], I[1], I[2]);
          for (int c = 0; c < nv; c++) {
            Ql[c] = W[c * G->N + sl];
            Qr[c] = W[c * G->N + sr];
          }
          if (orc_char_eigen(G->dim, d->gamma, a, Ql, Qr, R, Lv, NULL) != ORC_OK) {
            free(fp); free(fm); free(Fh);
            return ORC_ERR_ARG;
          }
          double h[5];
          for (int k = 0; k < nv; k++) {
            double vp[5], vm[5];
            for (int r = 0; r < 5; r++) {
              double sp = 0.0, sm = 0.0;
              for (int c = 0; c < nv; c++) {
                sp = sp + Lv[k * nv + c] * fp[c * len + m - 2 + r + NG];
                sm = sm + Lv[k * nv + c] * fm[c * len + m + 3 - r + NG];
              }
              vp[r] = sp;
              vm[r] = sm;
            }
            h[k] = recon_d(d, vp) + recon_d(d, vm);
          }
          for (int c = 0; c < nv; c++) {
            double s = 0.0;
            for (int k = 0; k < nv; k++) s = s + R[c * nv + k] * h[k];
            Fh[c * (na + 1) + m + 1] = s;
          }
        }
        for (int c = 0; c < nv; c++)
          for (int m = 0; m < na; m++) {
            if (char_cell(d, a, m, na)) continue;
            int I[3];
            I[a] = m; I[b1] = t1; I[b2] = t2;
            size_t o = c * Nu + uidx(G, I[0], I[1], I[2]);
            L[o] = L[o] - (Fh[c * (na + 1) + m + 1] - Fh[c * (na + 1) + m]) / met(G, a, m);
          }
      }
    free(fp); free(fm); free(Fh);
  }
  return ORC_OK;
}

/* 4th-order central first derivative from f_{-2..+2}: (8(f1 - f_-1) - (f2 - f_-2)) / (12 h) */
static double d4(double fm2, double fm1, double fp1, double fp2, double h) {
  return (8.0 * (fp1 - fm1) - (fp2 - fm2)) / (12.0 * h);
}

/* ----------------------------------------------------------------------------------------- */
/* Viscous term (Eq. 2, 5): (1/Re) sum_a d/dx_a [0, tau_{1a}, tau_{2a}, tau_{3a}, b_a]         */
/* ----------------------------------------------------------------------------------------- */
static void viscous(const pgrid *G, const orc_desc *d, const double *u, double *L) {
  int dim = G->dim, nv = G->nv;
  size_t Nu = (size_t)G->n[0] * G->n[1] * G->n[2];
  /* velocity gradients g[i][j] = du_i/dx_j on the box [-2, n+1] of every active direction */
  double *gr = calloc((size_t)9 * G->N, sizeof(double));
  int lo[3], hi[3];
  for (int a = 0; a < 3; a++) {
    lo[a] = a < dim ? -2 : 0;
    hi[a] = a < dim ? G->n[a] + 2 : 1;
  }
  for (int k = lo[2]; k < hi[2]; k++)
    for (int j = lo[1]; j < hi[1]; j++)
      for (int i = lo[0]; i < hi[0]; i++) {
        size_t s = pidx(G, i, j, k);
        for (int ci = 0; ci < dim; ci++)
          for (int dj = 0; dj < dim; dj++) {
            int o[3] = {0, 0, 0};
            o[dj] = 1;
            const double *ui = u + ci * G->N;
            double f_m2 = ui[pidx(G, i - 2 * o[0], j - 2 * o[1], k - 2 * o[2])];
            double f_m1 = ui[pidx(G, i - o[0], j - o[1], k - o[2])];
            double f_p1 = ui[pidx(G, i + o[0], j + o[1], k + o[2])];
            double f_p2 = ui[pidx(G, i + 2 * o[0], j + 2 * o[1], k + 2 * o[2])];
            int at = dj == 0 ? i : (dj == 1 ? j : k);
            gr[(ci * 3 + dj) * G->N + s] = d4(f_m2, f_m1, f_p1, f_p2, met(G, dj, at));
          }
      }
  /* viscous fluxes Fv[a][c] at the same box: tau_ij = g_ij + g_ji - 2/3 delta_ij div u */
  int nfc = dim + 1; /* components 1..dim (momentum) and energy */
  double *Fv = calloc((size_t)dim * nfc * G->N, sizeof(double));
  for (int k = lo[2]; k < hi[2]; k++)
    for (int j = lo[1]; j < hi[1]; j++)
      for (int i = lo[0]; i < hi[0]; i++) {
        size_t s = pidx(G, i, j, k);
        double div = 0.0;
        for (int a = 0; a < dim; a++) div += gr[(a * 3 + a) * G->N + s];
        for (int a = 0; a < dim; a++) { /* flux direction a */
          double b = 0.0;
          for (int ci = 0; ci < dim; ci++) {
            double tau = gr[(ci * 3 + a) * G->N + s] + gr[(a * 3 + ci) * G->N + s];
            if (ci == a) tau -= 2.0 / 3.0 * div;
            Fv[((size_t)a * nfc + ci) * G->N + s] = tau;
            b += u[ci * G->N + s] * tau;
          }
          Fv[((size_t)a * nfc + dim) * G->N + s] = b;
        }
      }
  for (int k = 0; k < G->n[2]; k++)
    for (int j = 0; j < G->n[1]; j++)
      for (int i = 0; i < G->n[0]; i++)
        for (int fc = 0; fc < nfc; fc++) {
          double sum = 0.0;
          for (int a = 0; a < dim; a++) {
            int o[3] = {0, 0, 0};
            o[a] = 1;
            const double *F = Fv + ((size_t)a * nfc + fc) * G->N;
            sum += d4(F[pidx(G, i - 2 * o[0], j - 2 * o[1], k - 2 * o[2])],
                      F[pidx(G, i - o[0], j - o[1], k - o[2])],
                      F[pidx(G, i + o[0], j + o[1], k + o[2])],
                      F[pidx(G, i + 2 * o[0], j + 2 * o[1], k + 2 * o[2])],
                      met(G, a, a == 0 ? i : (a == 1 ? j : k)));
          }
          int c = fc + 1; /* momentum components 1..dim, energy nv-1 */
          (void)nv;
          size_t o = c * Nu + uidx(G, i, j, k);
          L[o] = L[o] + sum / d->Re;
        }
  free(gr);
  free(Fv);
}

/* ----------------------------------------------------------------------------------------- */
/* Sponge: L -= sigma(n) (Q - Q_inf), n = distance in cells to the nearest outer boundary,   */
/* sigma = sigma_max ((S - n)/S)^3 for n < S                                                  */
/* ----------------------------------------------------------------------------------------- */
static void sponge(const pgrid *G, const orc_desc *d, const double *Q, double *L) {
  int S = d->sponge_cells;
  if (S <= 0) return;
  size_t Nu = (size_t)G->n[0] * G->n[1] * G->n[2];
  for (int k = 0; k < G->n[2]; k++)
    for (int j = 0; j < G->n[1]; j++)
      for (int i = 0; i < G->n[0]; i++) {
        int I[3] = {i, j, k};
        int nmin = 1 << 30;
        for (int a = 0; a < G->dim; a++) {
          int e = I[a] < G->n[a] - 1 - I[a] ? I[a] : G->n[a] - 1 - I[a];
          if (e < nmin) nmin = e;
        }
        if (nmin >= S) continue;
        double r = (double)(S - nmin) / (double)S;
        double sig = d->sponge_sigma * r * r * r;
        for (int c = 0; c < G->nv; c++) {
          size_t o = c * Nu + uidx(G, i, j, k);
          L[o] = L[o] - sig * (Q[o] - d->qinf[c]);
        }
      }
}

/* Periodic Gaussian pressure source of Sec. 3.6 (Eq. 16), A_p = amp exp(-b ln2 r^2) cos(w t):
 * read as a source in the pressure equation, i.e. A_p / (gamma - 1) in the energy equation
 * (no mass or momentum source). */
static void pressure_source(const pgrid *G, const orc_desc *d, double t, double *L) {
  if (d->src_amp == 0.0) return;
  const double LN2 = 0.693147180559945309417;
  size_t Nu = (size_t)G->n[0] * G->n[1] * G->n[2];
  double scale = (d->src_amp * cos(d->src_omega * t)) / (d->gamma - 1.0);
  for (int k = 0; k < G->n[2]; k++)
    for (int j = 0; j < G->n[1]; j++)
      for (int i = 0; i < G->n[0]; i++) {
        int I[3] = {i, j, k};
        double r2 = 0.0;
        for (int a = 0; a < G->dim; a++) {
          double x = node(G, a, I[a]);
          r2 = r2 + (x - d->src_xc[a]) * (x - d->src_xc[a]);
        }
        size_t o = (G->nv - 1) * Nu + uidx(G, i, j, k);
        L[o] = L[o] + exp(-(d->src_b * LN2) * r2) * scale;
      }
}

/* ----------------------------------------------------------------------------------------- */
/* Immersed boundary (Eq. 7-11)                                                               */
/* ----------------------------------------------------------------------------------------- */
/* the 4 support nodes along direction a of position x: first index and the 4 weights; *hl
 * (may be NULL) receives the spacing there.  On a stretched grid the position is inverted
 * through the node coordinates and the support must lie where the metric is constant (else
 * the returned index is -NG - 4, outside every interior). */
static int support(const pgrid *G, const orc_desc *d, int a, double x, double w[4],
                   double *hl) {
  if (!G->xn[a]) {
    double s = (x - d->lo[a]) / G->h[a] - 0.5; /* position in node-index units */
    int j0 = (int)floor(s) - 1;
    for (int r = 0; r < 4; r++) w[r] = orc_lambda(s - (double)(j0 + r));
    if (hl) *hl = G->h[a];
    return j0;
  }
  int n = G->n[a];
  if (!(x >= node(G, a, -NG)) || !(x < node(G, a, n + NG - 1))) return -NG - 4;
  int i = -NG;
  while (node(G, a, i + 1) <= x) i++;
  double m = met(G, a, i);
  double s = (double)i + (x - node(G, a, i)) / m;
  int j0 = (int)floor(s) - 1;
  for (int r = -1; r < 5; r++) {
    int jj = j0 + r;
    if (jj < -NG || jj > n + NG - 1) return -NG - 4;
    if (fabs(met(G, a, jj) - m) > 1e-12 * m) return -NG - 4;
  }
  for (int r = 0; r < 4; r++) w[r] = orc_lambda(s - (double)(j0 + r));
  if (hl) *hl = m;
  return j0;
}

static int marker_inside(const pgrid *G, const orc_desc *d, const double *X, int nm, int k) {
  for (int a = 0; a < G->dim; a++) {
    double w[4];
    int j0 = support(G, d, a, X[a * nm + k], w, NULL);
    if (j0 < 0 || j0 + 3 > G->n[a] - 1) return 0;
  }
  return 1;
}

/* interpolation of a padded cell field at marker k: sum_j phi_j prod_a lambda (Eq. 8) */
static double interp_field(const pgrid *G, const orc_desc *d, const double *phi, const double *X,
                           int nm, int k) {
  double w[3][4] = {{1, 0, 0, 0}, {1, 0, 0, 0}, {1, 0, 0, 0}};
  int j0[3] = {0, 0, 0};
  int cnt[3] = {1, 1, 1};
  for (int a = 0; a < G->dim; a++) {
    j0[a] = support(G, d, a, X[a * nm + k], w[a], NULL);
    cnt[a] = 4;
  }
  double acc = 0.0;
  for (int r2 = 0; r2 < cnt[2]; r2++)
    for (int r1 = 0; r1 < cnt[1]; r1++)
      for (int r0 = 0; r0 < cnt[0]; r0++)
        acc += phi[pidx(G, j0[0] + r0, j0[1] + r1, j0[2] + r2)] * (w[0][r0] * w[1][r1] * w[2][r2]);
  return acc;
}

/* IB source: Uib, F (Eq. 7), rate = Uib - U, and S = [0, f, f.u] added into L. */
static int ib_source(const pgrid *G, const orc_desc *d, const double *u, int nm, const double *X,
                     const double *U, const double *dS, const double *xi, double *L, double *Fout,
                     double *rate) {
  int dim = G->dim, nv = G->nv;
  size_t Nu = (size_t)G->n[0] * G->n[1] * G->n[2];
  for (int k = 0; k < nm; k++)
    if (!marker_inside(G, d, X, nm, k)) return ORC_ERR_BOUNDS;
  double *f = calloc((size_t)3 * Nu, sizeof(double));
  double *F = malloc(sizeof(double) * 3 * (nm > 0 ? nm : 1));
  for (int k = 0; k < nm; k++)
    for (int a = 0; a < dim; a++) {
      double uib = interp_field(G, d, u + a * G->N, X, nm, k);
      double slip = uib - U[a * nm + k];
      F[a * nm + k] = d->alpha_pen * xi[a * nm + k] + d->beta_pen * slip;
      if (rate) rate[a * nm + k] = slip;
      if (Fout) Fout[a * nm + k] = F[a * nm + k];
    }
  /* spreading, in marker order: f_j -= F_k prod lambda dS_k / prod h (Eq. 9) */
  for (int k = 0; k < nm; k++) {
    double w[3][4] = {{1, 0, 0, 0}, {1, 0, 0, 0}, {1, 0, 0, 0}};
    int j0[3] = {0, 0, 0}, cnt[3] = {1, 1, 1};
    double hprod = 1.0; /* the delta's h^d at the marker (Eq. 10) */
    for (int a = 0; a < dim; a++) {
      double hl;
      j0[a] = support(G, d, a, X[a * nm + k], w[a], &hl);
      cnt[a] = 4;
      hprod *= hl;
    }
    for (int r2 = 0; r2 < cnt[2]; r2++)
      for (int r1 = 0; r1 < cnt[1]; r1++)
        for (int r0 = 0; r0 < cnt[0]; r0++) {
          double wt = w[0][r0] * w[1][r1] * w[2][r2];
          size_t o = uidx(G, j0[0] + r0, j0[1] + r1, j0[2] + r2);
          for (int a = 0; a < dim; a++) f[a * Nu + o] -= F[a * nm + k] * wt * dS[k] / hprod;
        }
  }
  for (int kk = 0; kk < G->n[2]; kk++)
    for (int j = 0; j < G->n[1]; j++)
      for (int i = 0; i < G->n[0]; i++) {
        size_t o = uidx(G, i, j, kk), s = pidx(G, i, j, kk);
        double pw = 0.0;
        for (int a = 0; a < dim; a++) {
          L[(1 + a) * Nu + o] = L[(1 + a) * Nu + o] + f[a * Nu + o];
          pw += f[a * Nu + o] * u[a * G->N + s];
        }
        L[(nv - 1) * Nu + o] = L[(nv - 1) * Nu + o] + pw;
      }
  free(f);
  free(F);
  return ORC_OK;
}

/* ----------------------------------------------------------------------------------------- */
/* Public oracle entry points                                                                 */
/* ----------------------------------------------------------------------------------------- */
static int check_desc(const orc_desc *d) {
  if (!d || (d->dim != 2 && d->dim != 3)) return ORC_ERR_ARG;
  if (d->scheme < 0 || d->scheme > 2) return ORC_ERR_ARG;
  if (d->scheme == 2 && !d->mlp_params) return ORC_ERR_ARG;
  for (int a = 0; a < d->dim; a++)
    if (d->n[a] < 1 || !(d->hi[a] > d->lo[a])) return ORC_ERR_ARG;
  if (d->dim == 2 && d->n[2] != 1) return ORC_ERR_ARG;
  for (int a = 0; a < d->dim; a++) {
    int p0 = d->bc[a][0] == 2, p1 = d->bc[a][1] == 2;
    if (p0 != p1) return ORC_ERR_ARG;          /* periodic on both faces or on neither */
    if (p0 && d->n[a] < NG) return ORC_ERR_ARG; /* wrap-around ghosts need n >= 4 */
    for (int s = 0; s < 2; s++) {
      if (d->bc[a][s] < 0 || d->bc[a][s] > 3) return ORC_ERR_ARG;
      if (d->bc[a][s] == 3 && d->n[a] < 5) return ORC_ERR_ARG; /* one-sided 5-point stencil */
    }
  }
  return ORC_OK;
}

/* L = L_conv + L_visc - sponge + S at state Q (interior [nv][nz][ny][nx]).  F and rate
 * (each [dim][nm], may be NULL) receive the marker force of Eq. 7 and U_ib - U.
 * alpha_out (may be NULL) receives the three split speeds. */
static int rhs_impl(const orc_desc *d, const double *Q, int nm, const double *X,
                    const double *U, const double *dS, const double *xi, double *L, double *F,
                    double *rate, double *alpha_out, const double *alpha_in);

int orc_rhs(const orc_desc *d, const double *Q, int nm, const double *X, const double *U,
            const double *dS, const double *xi, double *L, double *F, double *rate,
            double *alpha_out) {
  return rhs_impl(d, Q, nm, X, U, dS, xi, L, F, rate, alpha_out, NULL);
}

/* The same right-hand side with the split speeds given (alpha_in[3]) instead of taken from Q:
 * the speeds are a maximum over the whole domain, so a crop of a large state reproduces the
 * right-hand side at its centre only when it is handed the full state's speeds. */
int orc_rhs_given_alpha(const orc_desc *d, const double *Q, int nm, const double *X,
                        const double *U, const double *dS, const double *xi, double *L,
                        const double *alpha_in) {
  return rhs_impl(d, Q, nm, X, U, dS, xi, L, NULL, NULL, NULL, alpha_in);
}

static int rhs_impl(const orc_desc *d, const double *Q, int nm, const double *X,
                    const double *U, const double *dS, const double *xi, double *L, double *F,
                    double *rate, double *alpha_out, const double *alpha_in) {
  int rc = check_desc(d);
  if (rc) return rc;
  pgrid G;
  pgrid_init(&G, d);
  size_t Nu = (size_t)G.n[0] * G.n[1] * G.n[2];
  double *W = malloc(sizeof(double) * G.nv * G.N);
  double *rho = malloc(sizeof(double) * G.N);
  double *u = calloc((size_t)3 * G.N, sizeof(double));
  double *p = malloc(sizeof(double) * G.N);
  if (!W || !rho || !u || !p) { free(W); free(rho); free(u); free(p); return ORC_ERR_NOMEM; }
  fill_padded(&G, d, Q, W);
  primitives(&G, d, W, rho, u, p);
  double alpha[3];
  wavespeeds(&G, d, rho, u, p, alpha);
  if (alpha_in)
    for (int a = 0; a < 3; a++) alpha[a] = alpha_in[a];
  if (alpha_out) for (int a = 0; a < 3; a++) alpha_out[a] = alpha[a];
  for (size_t o = 0; o < (size_t)G.nv * Nu; o++) L[o] = 0.0;
  g_mlp_used = 0;
  g_mlp_seen = 0;
  if (d->charwise) {
    rc = convective_charwise(&G, d, W, u, p, alpha, L);
    if (rc) { free(W); free(rho); free(u); free(p); return rc; }
  } else {
    convective(&G, d, W, u, p, alpha, L);
  }
  characteristic_faces(&G, d, rho, u, p, L);
  if (d->Re > 0.0) viscous(&G, d, u, L);
  sponge(&G, d, Q, L);
  pressure_source(&G, d, d->time, L);
  if (nm > 0) rc = ib_source(&G, d, u, nm, X, U, dS, xi, L, F, rate);
  free(W); free(rho); free(u); free(p);
  return rc;
}

/* nsteps of third-order TVD Runge-Kutta (Shu-Osher):
 *   Q1 = Qn + dt L(Qn);  Q2 = 3/4 Qn + 1/4 (Q1 + dt L(Q1));  Qn+1 = 1/3 Qn + 2/3 (Q2 + dt L(Q2))
 * written uniformly as Q^(s+1) = a_s Qn + b_s (Q^(s) + dt L(Q^(s))), (a,b) = (0,1),(3/4,1/4),
 * (1/3,2/3), applied to Q and to xi (xi' = U_ib - U).  Markers are fixed during the step.  The
 * stages are evaluated at the times t, t + dt, t + dt/2 from t = d->time (source of Eq. 16). */
int orc_rk3(const orc_desc *d, double *Q, int nm, const double *X, const double *U,
            const double *dS, double *xi, double dt, int nsteps) {
  int rc = check_desc(d);
  if (rc) return rc;
  pgrid G;
  pgrid_init(&G, d);
  size_t M = (size_t)G.nv * G.n[0] * G.n[1] * G.n[2];
  size_t mx = (size_t)d->dim * (nm > 0 ? nm : 1);
  double *Qs = malloc(sizeof(double) * M), *Lb = malloc(sizeof(double) * M);
  double *Q0 = malloc(sizeof(double) * M);
  double *xs = calloc(mx, sizeof(double)), *x0 = calloc(mx, sizeof(double));
  double *rate = calloc(mx, sizeof(double));
  const double A[3] = {0.0, 3.0 / 4.0, 1.0 / 3.0}, B[3] = {1.0, 1.0 / 4.0, 2.0 / 3.0};
  const double C[3] = {0.0, 1.0, 0.5}; /* stage times t + C dt */
  orc_desc ds = *d;
  double t = d->time;
  for (int step = 0; step < nsteps && rc == 0; step++) {
    memcpy(Q0, Q, sizeof(double) * M);
    memcpy(Qs, Q, sizeof(double) * M);
    if (nm > 0) { memcpy(x0, xi, sizeof(double) * mx); memcpy(xs, xi, sizeof(double) * mx); }
    for (int s = 0; s < 3 && rc == 0; s++) {
      ds.time = t + C[s] * dt;
      rc = orc_rhs(&ds, Qs, nm, X, U, dS, xs, Lb, NULL, rate, NULL);
      for (size_t o = 0; o < M; o++) Qs[o] = A[s] * Q0[o] + B[s] * (Qs[o] + dt * Lb[o]);
      for (size_t o = 0; o < (size_t)d->dim * nm; o++)
        xs[o] = A[s] * x0[o] + B[s] * (xs[o] + dt * rate[o]);
    }
    memcpy(Q, Qs, sizeof(double) * M);
    if (nm > 0) memcpy(xi, xs, sizeof(double) * (size_t)d->dim * nm);
    t = t + dt;
  }
  free(Qs); free(Lb); free(Q0); free(xs); free(x0); free(rate);
  return rc;
}

/* Delta-weighted pressure fluctuation at probe points: dp = sum_j p_j prod lambda - p_inf. */
int orc_probe(const orc_desc *d, const double *Q, int np, const double *xp, double *out) {
  int rc = check_desc(d);
  if (rc) return rc;
  pgrid G;
  pgrid_init(&G, d);
  double *W = malloc(sizeof(double) * G.nv * G.N);
  double *rho = malloc(sizeof(double) * G.N);
  double *u = calloc((size_t)3 * G.N, sizeof(double));
  double *p = malloc(sizeof(double) * G.N);
  fill_padded(&G, d, Q, W);
  primitives(&G, d, W, rho, u, p);
  double ke = 0.0;
  for (int a = 0; a < d->dim; a++) ke += d->qinf[1 + a] * (d->qinf[1 + a] / d->qinf[0]);
  double pinf = (d->gamma - 1.0) * (d->qinf[G.nv - 1] - 0.5 * ke);
  for (int k = 0; k < np && rc == 0; k++) {
    if (!marker_inside(&G, d, xp, np, k)) { rc = ORC_ERR_BOUNDS; break; }
    out[k] = interp_field(&G, d, p, xp, np, k) - pinf;
  }
  free(W); free(rho); free(u); free(p);
  return rc;
}

/* Split speeds alpha_d of state Q (for dt = CFL / sum_d alpha_d / h_d). */
int orc_wavespeeds(const orc_desc *d, const double *Q, double *alpha3) {
  int rc = check_desc(d);
  if (rc) return rc;
  pgrid G;
  pgrid_init(&G, d);
  double *W = malloc(sizeof(double) * G.nv * G.N);
  double *rho = malloc(sizeof(double) * G.N);
  double *u = calloc((size_t)3 * G.N, sizeof(double));
  double *p = malloc(sizeof(double) * G.N);
  fill_padded(&G, d, Q, W);
  primitives(&G, d, W, rho, u, p);
  wavespeeds(&G, d, rho, u, p, alpha3);
  free(W); free(rho); free(u); free(p);
  return ORC_OK;
}

/* Stand-alone interpolation of an interior scalar field phi at points X ([dim][nm]) and
 * spreading of point values Fk with weights dS onto an interior field f (f is overwritten):
 *   interp: out_k = sum_j phi_j prod lambda                              (Eq. 8, h^d cancels)
 *   spread: f_j = - sum_k Fk_k prod lambda dS_k / prod h                  (Eq. 9)
 * Used by the adjointness and conservation pins. */
int orc_interp_scalar(const orc_desc *d, const double *phi, int nm, const double *X, double *out) {
  int rc = check_desc(d);
  if (rc) return rc;
  pgrid G;
  pgrid_init(&G, d);
  double *P = calloc(G.N, sizeof(double));
  for (int k = 0; k < G.n[2]; k++)
    for (int j = 0; j < G.n[1]; j++)
      for (int i = 0; i < G.n[0]; i++) P[pidx(&G, i, j, k)] = phi[uidx(&G, i, j, k)];
  for (int k = 0; k < nm; k++) {
    if (!marker_inside(&G, d, X, nm, k)) { rc = ORC_ERR_BOUNDS; break; }
    out[k] = interp_field(&G, d, P, X, nm, k);
  }
  free(P);
  return rc;
}

int orc_spread_scalar(const orc_desc *d, int nm, const double *X, const double *Fk,
                      const double *dS, double *f) {
  int rc = check_desc(d);
  if (rc) return rc;
  pgrid G;
  pgrid_init(&G, d);
  size_t Nu = (size_t)G.n[0] * G.n[1] * G.n[2];
  for (size_t o = 0; o < Nu; o++) f[o] = 0.0;
  for (int k = 0; k < nm; k++) {
    if (!marker_inside(&G, d, X, nm, k)) return ORC_ERR_BOUNDS;
    double w[3][4] = {{1, 0, 0, 0}, {1, 0, 0, 0}, {1, 0, 0, 0}};
    int j0[3] = {0, 0, 0}, cnt[3] = {1, 1, 1};
    double hprod = 1.0;
    for (int a = 0; a < d->dim; a++) {
      double hl;
      j0[a] = support(&G, d, a, X[a * nm + k], w[a], &hl);
      cnt[a] = 4;
      hprod *= hl;
    }
    for (int r2 = 0; r2 < cnt[2]; r2++)
      for (int r1 = 0; r1 < cnt[1]; r1++)
        for (int r0 = 0; r0 < cnt[0]; r0++) {
          double wt = w[0][r0] * w[1][r1] * w[2][r2];
          f[uidx(&G, j0[0] + r0, j0[1] + r1, j0[2] + r2)] -= Fk[k] * wt * dS[k] / hprod;
        }
  }
  return rc;
}
