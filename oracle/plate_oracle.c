/*
 * plate_oracle.c -- plain, slow FP64 CPU oracle of the flexible plate of Sec. 2 (Eq. 1), solved
 * in the absolute nodal coordinate formulation, of its clamp motion (Sec. 4.1, Eq. 17), and of
 * the two-way coupling with the fluid through the penalty forces (Eq. 7-9).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this file:
 * only the test suite, the smoke check and the bench's CPU-baseline leg use it.  It shares no
 * source, header, table or helper with the CUDA path.  Compile with -O2 -ffp-contract=off
 * (no multiply and add is fused).
 *
 * The paper names the formulation (Shabana's ANCF) but prints neither the element nor the time
 * integrator; the readings taken here:
 *
 *  - The plate is a plane curve r(s, t), s in [0, L] its material arc coordinate, cut into n_el
 *    equal elements of length l = L / n_el.  Node j carries e_j = [x, y, x_s, y_s] (position and
 *    slope: the gradient-deficient ANCF beam element).  Inside element k, xi = (s - k l) / l and
 *      r = S0 r_k + S1 r_s,k + S2 r_k+1 + S3 r_s,k+1,
 *      S0 = 1 - 3 xi^2 + 2 xi^3, S1 = l (xi - 2 xi^2 + xi^3), S2 = 3 xi^2 - 2 xi^3,
 *      S3 = l (xi^3 - xi^2)                                  (cubic Hermite interpolation).
 *  - Eq. 1 is taken as the Euler-Lagrange equation of the kinetic energy 1/2 int rho_s |r_t|^2 ds
 *    and the elastic energy 1/2 int [K_S (|r_s| - 1)^2 + K_B |r_ss|^2] ds: tension
 *    K_S (|r_s| - 1) along the unit tangent, bending K_B r_ssss (the curvature taken as |r_ss|,
 *    exact for an inextensible plate).  Discretised: M e'' + Q_int(e) = Q_f with the
 *    consistent mass matrix M, Q_int = K_b e + Q_s(e), the constant bending matrix K_b, and the
 *    stretching force Q_s by five-point Gauss-Legendre quadrature per element.
 *  - Load: the penalty force F_k of Eq. 7 is the force of the fluid on the structure at marker
 *    k; markers sit at s_k = (k + 1/2) L / n_m with weights dS_k = L / n_m, and
 *    Q_f = sum_k S(s_k)^T F_k dS_k, summed in marker order.
 *  - Time: the implicit midpoint rule
 *      e_{n+1} = e_n + dt (v_n + v_{n+1}) / 2,
 *      M (v_{n+1} - v_n) = dt [Q_f - Q_int((e_n + e_{n+1}) / 2)],
 *    solved by Newton's method for d = e_{n+1} - e_n; each Newton system is assembled as a
 *    dense matrix and solved by Gaussian elimination with partial pivoting in natural order,
 *    every operation rounded on its own (no fused multiply-add anywhere).  The rule conserves the linear and angular
 *    momentum of an unloaded free plate and hands the plate exactly the impulse dt Q_f of the
 *    step's load, so what the fluid loses the plate gains.
 *  - Clamp (Sec. 4.1, Eq. 17): r(0, t) = x0 + (A0/2) cos(2 pi f t) [cos b, sin b], and the
 *    slope r_s(0, t) parallel to [cos(theta0 + a), sin(theta0 + a)] with
 *    a(t) = (alpha_m / 2) sin(2 pi f t + phi): the clamp fixes the plate's angle, while the
 *    length of the slope (the stretch at the root) stays free.
 *  - Coupling within a fluid step: markers take the plate's positions and velocities at the
 *    step start and keep them for the three Runge-Kutta stages; the plate is then advanced by
 *    the load of the stage forces weighted as the SSP-RK3 update weights them (1/6, 1/6, 2/3).
 *
 * Pins (tests/test_plate_oracle.py): cantilever under a uniform load (tip deflection
 * q L^4 / (8 K_B)), uniform stretching under an end load, the large-deflection elastica by
 * shooting, the first bending frequency of a cantilever (k_1 = 1.8751, Sec. 4.1) and the first
 * axial frequency of a clamped-free rod, consistent mass matrix against quadrature of S^T S,
 * tangent stiffness against finite differences, exact momentum and angular momentum of a free
 * plate, clamp derivatives against finite differences, and the momentum balance of the
 * coupled plate and fluid in a periodic box.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ibfsa_oracle.h"

typedef struct {
  int n_el;            /* elements */
  int n_markers;       /* Lagrangian markers along the plate */
  double length;       /* L */
  double rho_s;        /* mass per unit length */
  double K_S, K_B;     /* stretching and bending rigidity of Eq. 1 */
  int clamped;         /* 1: node 0 follows the clamp motion; 0: free plate */
  double x0[2];        /* clamp mean position */
  double theta0;       /* chord direction of the clamp at a = 0 */
  double A0, freq, beta, alpha_m, phi;  /* Eq. 17 */
  int newton_max;      /* Newton iteration limit */
  double newton_tol;   /* converged when max |increment of d| <= newton_tol * L */
} orc_plate;

enum { ORC_PLATE_NOCONV = -8 };


static const double PI = 3.14159265358979323846;

/* Gauss-Legendre nodes and weights on [-1, 1], five points */
static const double GX[5] = {-0.90617984593866399280, -0.53846931010568309104, 0.0,
                             0.53846931010568309104, 0.90617984593866399280};
static const double GW[5] = {0.23692688505618908751, 0.47862867049936646804,
                             0.56888888888888888889, 0.47862867049936646804,
                             0.23692688505618908751};

static int check_plate(const orc_plate *p) {
  if (!p || p->n_el < 1 || p->n_markers < 0 || !(p->length > 0.0) || !(p->rho_s > 0.0) ||
      p->K_S < 0.0 || p->K_B < 0.0 || p->newton_max < 1 || !(p->newton_tol > 0.0))
    return ORC_ERR_ARG;
  return ORC_OK;
}

/* local coordinate of shape function i (0..3) and component a (0 = x, 1 = y) in the 8 element
 * coordinates [x_k, y_k, x_s,k, y_s,k, x_k+1, y_k+1, x_s,k+1, y_s,k+1] */
static int loc(int i, int a) { return 4 * (i / 2) + 2 * (i % 2) + a; }

/* Hermite shape functions at xi and their derivatives with respect to s */
static void shape(double xi, double l, double S[4]) {
  double x2 = xi * xi, x3 = x2 * xi;
  S[0] = 1.0 - 3.0 * x2 + 2.0 * x3;
  S[1] = l * (xi - 2.0 * x2 + x3);
  S[2] = 3.0 * x2 - 2.0 * x3;
  S[3] = l * (x3 - x2);
}

static void dshape(double xi, double l, double D[4]) {
  double x2 = xi * xi;
  D[0] = (6.0 * x2 - 6.0 * xi) / l;
  D[1] = 1.0 - 4.0 * xi + 3.0 * x2;
  D[2] = (6.0 * xi - 6.0 * x2) / l;
  D[3] = 3.0 * x2 - 2.0 * xi;
}

/* consistent mass matrix rho_s int S_i S_j ds and bending matrix K_B int S_i'' S_j'' ds of one
 * element (per component) */
static void element_mass(const orc_plate *p, double Ms[4][4]) {
  double l = p->length / p->n_el;
  double c = p->rho_s * l / 420.0;
  double m[4][4] = {{156.0, 22.0 * l, 54.0, -13.0 * l},
                    {22.0 * l, 4.0 * l * l, 13.0 * l, -3.0 * l * l},
                    {54.0, 13.0 * l, 156.0, -22.0 * l},
                    {-13.0 * l, -3.0 * l * l, -22.0 * l, 4.0 * l * l}};
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) Ms[i][j] = c * m[i][j];
}

static void element_bending(const orc_plate *p, double Kb[4][4]) {
  double l = p->length / p->n_el;
  double c = p->K_B / (l * l * l);
  double k[4][4] = {{12.0, 6.0 * l, -12.0, 6.0 * l},
                    {6.0 * l, 4.0 * l * l, -6.0 * l, 2.0 * l * l},
                    {-12.0, -6.0 * l, 12.0, -6.0 * l},
                    {6.0 * l, 2.0 * l * l, -6.0 * l, 4.0 * l * l}};
  for (int i = 0; i < 4; i++)
    for (int j = 0; j < 4; j++) Kb[i][j] = c * k[i][j];
}

/* Internal force Q_int (8) and tangent dQ_int/de (8x8) of one element at coordinates ee (8):
 * bending K_b ee plus the stretching force int K_S (1 - 1/|r_s|) S'^T r_s ds, whose derivative
 * is int S'^T [K_S (1 - 1/|r_s|) I + K_S r_s r_s^T / |r_s|^3] S' ds. */
static void element_internal(const orc_plate *p, const double *ee, double Qi[8], double Kt[8][8]) {
  double l = p->length / p->n_el;
  double Kb[4][4];
  element_bending(p, Kb);
  double D[5][4], wl[5], c1[5], c2[5], rs[5][2];
  for (int g = 0; g < 5; g++) {
    double xi = 0.5 + 0.5 * GX[g];
    wl[g] = 0.5 * GW[g] * l;
    dshape(xi, l, D[g]);
    for (int a = 0; a < 2; a++) {
      double r = 0.0;
      for (int j = 0; j < 4; j++) r = r + D[g][j] * ee[loc(j, a)];
      rs[g][a] = r;
    }
    double n = sqrt(rs[g][0] * rs[g][0] + rs[g][1] * rs[g][1]);
    c1[g] = p->K_S * (1.0 - 1.0 / n);
    c2[g] = p->K_S / (n * n * n);
  }
  for (int i = 0; i < 4; i++)
    for (int a = 0; a < 2; a++) {
      double bend = 0.0;
      for (int j = 0; j < 4; j++) bend = bend + Kb[i][j] * ee[loc(j, a)];
      double axial = 0.0;
      for (int g = 0; g < 5; g++) axial = axial + wl[g] * c1[g] * rs[g][a] * D[g][i];
      Qi[loc(i, a)] = bend + axial;
    }
  if (!Kt) return;
  for (int i = 0; i < 4; i++)
    for (int a = 0; a < 2; a++)
      for (int j = 0; j < 4; j++)
        for (int b = 0; b < 2; b++) {
          double k = 0.0;
          for (int g = 0; g < 5; g++) {
            double s = c2[g] * rs[g][a] * rs[g][b];
            if (a == b) s = c1[g] + s;
            k = k + wl[g] * D[g][i] * D[g][j] * s;
          }
          Kt[loc(i, a)][loc(j, b)] = a == b ? Kb[i][j] + k : k;
        }
}

/* Clamp motion of Eq. 17 at time t: the prescribed coordinates of node 0 and their rates. */
void orc_plate_motion(const orc_plate *p, double t, double e4[4], double v4[4]) {
  double w = 2.0 * PI * p->freq;
  double c = cos(w * t), s = sin(w * t);
  double half = 0.5 * p->A0;
  double cb = cos(p->beta), sb = sin(p->beta);
  double am = 0.5 * p->alpha_m;
  double th = p->theta0 + am * sin(w * t + p->phi);
  double thdot = am * w * cos(w * t + p->phi);
  e4[0] = p->x0[0] + half * c * cb;
  e4[1] = p->x0[1] + half * c * sb;
  e4[2] = cos(th);
  e4[3] = sin(th);
  v4[0] = -(half * w * s) * cb;
  v4[1] = -(half * w * s) * sb;
  v4[2] = -sin(th) * thdot;
  v4[3] = cos(th) * thdot;
}

/* element index and local coordinate of marker k */
static int marker_site(const orc_plate *p, int k, double *xi) {
  double l = p->length / p->n_el;
  double s = ((double)k + 0.5) * p->length / (double)p->n_markers;
  int el = (int)(s / l);
  if (el > p->n_el - 1) el = p->n_el - 1;
  *xi = (s - (double)el * l) / l;
  return el;
}

/* Marker positions X and velocities U ([2][n_markers]) and weights dS of the plate state. */
int orc_plate_markers(const orc_plate *p, const double *e, const double *v, double *X,
                      double *U, double *dS) {
  int rc = check_plate(p);
  if (rc) return rc;
  int nm = p->n_markers;
  double l = p->length / p->n_el;
  for (int k = 0; k < nm; k++) {
    double xi, S[4];
    int el = marker_site(p, k, &xi);
    shape(xi, l, S);
    for (int a = 0; a < 2; a++) {
      double x = 0.0, u = 0.0;
      for (int i = 0; i < 4; i++) {
        x = x + S[i] * e[4 * el + loc(i, a)];
        u = u + S[i] * v[4 * el + loc(i, a)];
      }
      X[a * nm + k] = x;
      U[a * nm + k] = u;
    }
    dS[k] = p->length / (double)nm;
  }
  return ORC_OK;
}

/* Generalised load Q_f = sum_k S(s_k)^T F_k dS_k of marker forces F [2][n_markers]. */
int orc_plate_load(const orc_plate *p, const double *F, double *Qf) {
  int rc = check_plate(p);
  if (rc) return rc;
  int nm = p->n_markers, nd = 4 * (p->n_el + 1);
  double l = p->length / p->n_el;
  double dS = p->length / (double)nm;
  for (int I = 0; I < nd; I++) Qf[I] = 0.0;
  for (int k = 0; k < nm; k++) {
    double xi, S[4];
    int el = marker_site(p, k, &xi);
    shape(xi, l, S);
    for (int i = 0; i < 4; i++)
      for (int a = 0; a < 2; a++) {
        int I = 4 * el + loc(i, a);
        Qf[I] = Qf[I] + S[i] * F[a * nm + k] * dS;
      }
  }
  return ORC_OK;
}

/* Global internal force, tangent (dense nd x nd, may be NULL) and mass matrix (dense, may be
 * NULL), assembled element by element.  For the pins. */
int orc_plate_internal(const orc_plate *p, const double *e, double *Qint, double *K, double *M) {
  int rc = check_plate(p);
  if (rc) return rc;
  int nd = 4 * (p->n_el + 1);
  double Ms[4][4];
  element_mass(p, Ms);
  for (int I = 0; I < nd; I++) Qint[I] = 0.0;
  if (K) memset(K, 0, sizeof(double) * nd * nd);
  if (M) memset(M, 0, sizeof(double) * nd * nd);
  for (int el = 0; el < p->n_el; el++) {
    double Qi[8], Kt[8][8];
    element_internal(p, e + 4 * el, Qi, K ? Kt : NULL);
    for (int r = 0; r < 8; r++) {
      Qint[4 * el + r] = Qint[4 * el + r] + Qi[r];
      for (int c = 0; c < 8; c++) {
        if (K) K[(4 * el + r) * nd + 4 * el + c] += Kt[r][c];
        if (M && (r % 2) == (c % 2))
          M[(4 * el + r) * nd + 4 * el + c] += Ms[(r / 4) * 2 + (r % 4) / 2][(c / 4) * 2 + (c % 4) / 2];
      }
    }
  }
  return ORC_OK;
}

/* Solve A x = b (n x n, row-major; A and b are overwritten, x returned in b) by Gaussian
 * elimination with partial pivoting in natural order, then back substitution.  Returns 0, or -1
 * on a zero or non-finite pivot. */
static int gauss_solve(int n, double *A, double *b) {
  for (int k = 0; k < n; k++) {
    int piv = k;
    double best = fabs(A[(size_t)k * n + k]);
    for (int r = k + 1; r < n; r++)
      if (fabs(A[(size_t)r * n + k]) > best) {
        best = fabs(A[(size_t)r * n + k]);
        piv = r;
      }
    if (!(best > 0.0) || !isfinite(best)) return -1;
    if (piv != k) {
      for (int c = 0; c < n; c++) {
        double t = A[(size_t)k * n + c];
        A[(size_t)k * n + c] = A[(size_t)piv * n + c];
        A[(size_t)piv * n + c] = t;
      }
      double t = b[k];
      b[k] = b[piv];
      b[piv] = t;
    }
    for (int r = k + 1; r < n; r++) {
      double f = A[(size_t)r * n + k] / A[(size_t)k * n + k];
      if (f == 0.0) continue; /* rows outside the band stay untouched */
      for (int c = k; c < n; c++) A[(size_t)r * n + c] = A[(size_t)r * n + c] - f * A[(size_t)k * n + c];
      b[r] = b[r] - f * b[k];
    }
  }
  for (int k = n - 1; k >= 0; k--) {
    double t = b[k];
    for (int c = k + 1; c < n; c++) t = t - A[(size_t)k * n + c] * b[c];
    b[k] = t / A[(size_t)k * n + k];
  }
  return 0;
}

/* Newton solve shared by the dynamic step (dt > 0) and the static solve (dt = 0).
 *   dynamic: unknown d = e_{n+1} - e_n, midpoint em = e_n + d/2,
 *            R = M g + (dt^2/2) (Q_int(em) - Q_f) with g = (dt/2)(v_{n+1} - v_n), which is
 *            d - dt v_n wherever v_{n+1} = 2 d/dt - v_n; Jacobian M + (dt^2/4) dQ_int/de;
 *   static:  unknown e, R = Q_int(e) - Q_f, Jacobian dQ_int/de.
 * A clamped plate prescribes the position of node 0 (e_p[0..1], rates v_p[0..1]) and the
 * direction of its slope, t = (e_p[2], e_p[3]): the slope is sigma t with sigma free, so the
 * clamp holds the plate's angle without holding its stretch.  The unknowns are then sigma and
 * the coordinates of nodes 1..n_el (free index 0 and 1.., global 4.. = free + 3); the sigma
 * row and column are the slope rows and columns projected on t. */
static int newton(const orc_plate *p, double *e, double *v, const double *Qf, double dt,
                  const double *e_p, const double *v_p, int *iters) {
  int ne = p->n_el, nd = 4 * (ne + 1);
  int clamped = p->clamped != 0;
  int nf = clamped ? nd - 3 : nd;
  double tc = clamped ? e_p[2] : 0.0, ts = clamped ? e_p[3] : 0.0;
  double Ms[4][4];
  element_mass(p, Ms);
  double *d = calloc(nd, sizeof(double)), *em = calloc(nd, sizeof(double));
  double *g = calloc(nd, sizeof(double)), *R = calloc(nd, sizeof(double));
  double *x = calloc(nf, sizeof(double));
  double *J = calloc((size_t)nd * nd, sizeof(double));  /* Jacobian of every coordinate */
  double *A = calloc((size_t)nf * nf, sizeof(double));  /* Jacobian of the free unknowns */
  double (*Rel)[8] = calloc((size_t)ne, sizeof(*Rel));
  double (*Jel)[8][8] = calloc((size_t)ne, sizeof(*Jel));
  int dynamic = dt > 0.0;
  double c_load = 0.5 * dt * dt, c_stiff = 0.25 * dt * dt;
  if (dynamic) {
    for (int I = 0; I < nd; I++) d[I] = dt * v[I];
    if (clamped) {
      double sigma = e[2] * tc + e[3] * ts; /* old slope projected on the new direction */
      d[0] = e_p[0] - e[0];
      d[1] = e_p[1] - e[1];
      d[2] = sigma * tc - e[2];
      d[3] = sigma * ts - e[3];
    }
  } else if (clamped) {
    double sigma = e[2] * tc + e[3] * ts;
    e[0] = e_p[0];
    e[1] = e_p[1];
    e[2] = sigma * tc;
    e[3] = sigma * ts;
  }
  int rc = ORC_PLATE_NOCONV, it;
  for (it = 1; it <= p->newton_max; it++) {
    /* state at which the forces are evaluated */
    for (int I = 0; I < nd; I++) em[I] = dynamic ? e[I] + 0.5 * d[I] : e[I];
    if (dynamic)
      for (int I = 0; I < nd; I++)
        g[I] = (clamped && I < 2) ? (0.5 * dt) * (v_p[I] - v[I]) : d[I] - dt * v[I];
    /* element residuals and Jacobians */
    for (int el = 0; el < ne; el++) {
      double Qi[8], Kt[8][8];
      element_internal(p, em + 4 * el, Qi, Kt);
      for (int i = 0; i < 4; i++)
        for (int a = 0; a < 2; a++) {
          int r = loc(i, a);
          if (dynamic) {
            double inert = 0.0;
            for (int j = 0; j < 4; j++) inert = inert + Ms[i][j] * g[4 * el + loc(j, a)];
            Rel[el][r] = inert + c_load * Qi[r];
          } else {
            Rel[el][r] = Qi[r];
          }
          for (int j = 0; j < 4; j++)
            for (int b = 0; b < 2; b++) {
              int c = loc(j, b);
              if (!dynamic)
                Jel[el][r][c] = Kt[r][c];
              else if (a == b)
                Jel[el][r][c] = Ms[i][j] + c_stiff * Kt[r][c];
              else
                Jel[el][r][c] = c_stiff * Kt[r][c];
            }
        }
    }
    /* assembly in element order: residual and Jacobian */
    for (int I = 0; I < nd; I++) R[I] = 0.0;
    memset(J, 0, sizeof(double) * (size_t)nd * nd);
    for (int el = 0; el < ne; el++)
      for (int r = 0; r < 8; r++) {
        int I = 4 * el + r;
        R[I] = R[I] + Rel[el][r];
        for (int c = 0; c < 8; c++) J[(size_t)I * nd + 4 * el + c] += Jel[el][r][c];
      }
    for (int I = 0; I < nd; I++) R[I] = R[I] - (dynamic ? c_load * Qf[I] : Qf[I]);
    /* the free system A x = -R: a clamped plate's first unknown is sigma, the slope of node 0
     * along t, whose row and column are the slope rows and columns projected on t; the others
     * are the coordinates of nodes 1.. (global index = free index + 3) */
    if (clamped) {
      x[0] = -(tc * R[2] + ts * R[3]);
      for (int i = 1; i < nf; i++) x[i] = -R[i + 3];
      A[0] = tc * (tc * J[2 * nd + 2] + ts * J[2 * nd + 3]) +
             ts * (tc * J[3 * nd + 2] + ts * J[3 * nd + 3]);
      for (int j = 1; j < nf; j++) {
        A[j] = tc * J[2 * nd + j + 3] + ts * J[3 * nd + j + 3];
        A[(size_t)j * nf] = tc * J[(size_t)(j + 3) * nd + 2] + ts * J[(size_t)(j + 3) * nd + 3];
      }
      for (int i = 1; i < nf; i++)
        for (int j = 1; j < nf; j++) A[(size_t)i * nf + j] = J[(size_t)(i + 3) * nd + j + 3];
    } else {
      for (int i = 0; i < nf; i++) x[i] = -R[i];
      memcpy(A, J, sizeof(double) * (size_t)nd * nd);
    }
    if (gauss_solve(nf, A, x) != 0) { rc = ORC_PLATE_NOCONV; break; }
    /* update: sigma moves the clamped slope along t */
    double *u = dynamic ? d : e;
    double inc = 0.0;
    int bad = 0;
    for (int i = 0; i < nf; i++) {
      if (clamped && i == 0) {
        u[2] = u[2] + tc * x[0];
        u[3] = u[3] + ts * x[0];
      } else {
        int I = clamped ? i + 3 : i;
        u[I] = u[I] + x[i];
      }
      double a = fabs(x[i]);
      if (isnan(a)) bad = 1;
      else if (a > inc) inc = a;
    }
    if (bad) { rc = ORC_PLATE_NOCONV; break; } /* a non-finite increment never converges */
    if (inc <= p->newton_tol * p->length) { rc = ORC_OK; break; }
  }
  if (iters) *iters = it > p->newton_max ? p->newton_max : it;
  if (dynamic) {
    for (int I = 0; I < nd; I++) {
      if (clamped && I < 2) {
        e[I] = e_p[I];
        v[I] = v_p[I];
      } else {
        double vn = v[I];
        e[I] = e[I] + d[I];
        v[I] = (2.0 * d[I]) / dt - vn;
      }
    }
  }
  free(d); free(em); free(g); free(R); free(x); free(J); free(A); free(Rel); free(Jel);
  return rc;
}

/* One implicit-midpoint step of size dt > 0 under the generalised load Qf (held over the step;
 * NULL = no load), the clamp (if any) taken to time t_new.  e, v ([4 (n_el + 1)]) advance in
 * place; *iters receives the Newton iterations.  Returns ORC_OK or ORC_PLATE_NOCONV. */
int orc_plate_step(const orc_plate *p, double *e, double *v, double t_new, double dt,
                   const double *Qf, int *iters) {
  int rc = check_plate(p);
  if (rc) return rc;
  if (!(dt > 0.0)) return ORC_ERR_ARG;
  int nd = 4 * (p->n_el + 1);
  double *zero = NULL;
  if (!Qf) Qf = zero = calloc(nd, sizeof(double));
  double ep[4], vp[4];
  orc_plate_motion(p, t_new, ep, vp);
  rc = newton(p, e, v, Qf, dt, ep, vp, iters);
  free(zero);
  return rc;
}

/* Static equilibrium Q_int(e) = Qf by Newton's method from the initial guess e (clamp at t = 0).
 * For the pins. */
int orc_plate_static(const orc_plate *p, double *e, const double *Qf, int *iters) {
  int rc = check_plate(p);
  if (rc) return rc;
  double ep[4], vp[4];
  orc_plate_motion(p, 0.0, ep, vp);
  return newton(p, e, NULL, Qf, 0.0, ep, vp, iters);
}

/* Force of the fluid on the plate and the power it delivers over a step (Sec. 4.1, Eq. 19):
 * force[a] = sum_k F_k,a dS_k and *power = sum_k (F_k . U_k) dS_k, in marker order, from the
 * step's load F [2][n_markers] and the marker velocities U [2][n_markers] held during the step.
 * The thrust, lift and power coefficients of Eq. 19 are -force[0], force[1] and -power scaled
 * by 2 / (rho U^2 L) (power: 2 / (rho U^3 L)). */
int orc_plate_force(const orc_plate *p, const double *F, const double *U, double force[2],
                    double *power) {
  int rc = check_plate(p);
  if (rc) return rc;
  int nm = p->n_markers;
  double dS = p->length / (double)nm;
  double fx = 0.0, fy = 0.0, pw = 0.0;
  for (int k = 0; k < nm; k++) {
    fx = fx + F[k] * dS;
    fy = fy + F[nm + k] * dS;
    pw = pw + (F[k] * U[k] + F[nm + k] * U[nm + k]) * dS;
  }
  force[0] = fx;
  force[1] = fy;
  *power = pw;
  return ORC_OK;
}

/* The load Fbar the coupled step hands the plate (last step), for the force pin. */
static double *g_last_fbar = NULL;
static int g_last_fbar_n = 0;

int orc_fsi_last_load(double *F, int n) {
  if (!g_last_fbar || n != g_last_fbar_n) return ORC_ERR_ARG;
  memcpy(F, g_last_fbar, sizeof(double) * n);
  return ORC_OK;
}

/* nsteps coupled steps of plate and fluid (2D):
 *   markers <- plate (positions, velocities, weights) at the step start;
 *   three SSP-RK3 stages of the fluid and of xi with those markers (as orc_rk3), collecting
 *   Fbar = F1/6 + F2/6 + 2 F3/3 from the penalty forces of the stages;
 *   plate step of dt under Q_f(Fbar), clamp at t + dt.
 * Q [4][ny][nx], xi [2][n_markers], e and v advance in place; *t advances by nsteps dt.
 * iters (may be NULL) receives the Newton iterations of each step. */
int orc_fsi_step(const orc_desc *d, const orc_plate *p, double *Q, double *xi, double *e,
                 double *v, double *t, double dt, int nsteps, int *iters) {
  int rc = check_plate(p);
  if (rc) return rc;
  if (!d || d->dim != 2 || !(dt > 0.0)) return ORC_ERR_ARG;
  int nm = p->n_markers, nd = 4 * (p->n_el + 1);
  size_t M = (size_t)4 * d->n[0] * d->n[1];
  size_t mx = (size_t)2 * (nm > 0 ? nm : 1);
  double *Qs = malloc(sizeof(double) * M), *Lb = malloc(sizeof(double) * M);
  double *Q0 = malloc(sizeof(double) * M);
  double *xs = calloc(mx, sizeof(double)), *x0 = calloc(mx, sizeof(double));
  double *rate = calloc(mx, sizeof(double)), *F = calloc(mx, sizeof(double));
  double *Fbar = calloc(mx, sizeof(double));
  double *X = calloc(mx, sizeof(double)), *U = calloc(mx, sizeof(double));
  double *dS = calloc(nm > 0 ? nm : 1, sizeof(double));
  double *Qf = calloc(nd, sizeof(double));
  const double A[3] = {0.0, 3.0 / 4.0, 1.0 / 3.0}, B[3] = {1.0, 1.0 / 4.0, 2.0 / 3.0};
  const double W[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
  const double C[3] = {0.0, 1.0, 0.5};
  orc_desc ds = *d;
  double tf = d->time;  /* the fluid's clock (pressure source of Eq. 16) */
  for (int step = 0; step < nsteps && rc == ORC_OK; step++) {
    orc_plate_markers(p, e, v, X, U, dS);
    memcpy(Q0, Q, sizeof(double) * M);
    memcpy(Qs, Q, sizeof(double) * M);
    memcpy(x0, xi, sizeof(double) * 2 * nm);
    memcpy(xs, xi, sizeof(double) * 2 * nm);
    for (int s = 0; s < 3 && rc == ORC_OK; s++) {
      ds.time = tf + C[s] * dt;
      rc = orc_rhs(&ds, Qs, nm, X, U, dS, xs, Lb, F, rate, NULL);
      for (size_t o = 0; o < (size_t)2 * nm; o++)
        Fbar[o] = s == 0 ? W[0] * F[o] : Fbar[o] + W[s] * F[o];
      for (size_t o = 0; o < M; o++) Qs[o] = A[s] * Q0[o] + B[s] * (Qs[o] + dt * Lb[o]);
      for (size_t o = 0; o < (size_t)2 * nm; o++)
        xs[o] = A[s] * x0[o] + B[s] * (xs[o] + dt * rate[o]);
    }
    if (rc != ORC_OK) break;
    memcpy(Q, Qs, sizeof(double) * M);
    memcpy(xi, xs, sizeof(double) * 2 * nm);
    orc_plate_load(p, Fbar, Qf);
    free(g_last_fbar);
    g_last_fbar = malloc(sizeof(double) * 2 * nm);
    g_last_fbar_n = 2 * nm;
    if (g_last_fbar) memcpy(g_last_fbar, Fbar, sizeof(double) * 2 * nm);
    double t_new = *t + dt;
    int it = 0;
    rc = orc_plate_step(p, e, v, t_new, dt, Qf, &it);
    if (iters) iters[step] = it;
    *t = t_new;
    tf = tf + dt;
  }
  free(Qs); free(Lb); free(Q0); free(xs); free(x0); free(rate); free(F); free(Fbar);
  free(X); free(U); free(dS); free(Qf);
  return rc;
}
