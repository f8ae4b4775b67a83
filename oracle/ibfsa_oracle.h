/*
 * ibfsa_oracle.h -- descriptor and entry points of the FP64 CPU oracle of the fluid stage
 * (ibfsa_oracle.c), shared with the plate oracle (plate_oracle.c) for the coupled step.
 *
 * TEST INFRASTRUCTURE ONLY: no product code includes this header.
 */
#ifndef IBFSA_ORACLE_H
#define IBFSA_ORACLE_H

typedef struct {
  int dim;              /* 2 or 3 */
  int n[3];             /* interior cells per direction (n[2] = 1 in 2D) */
  double lo[3], hi[3];  /* domain box; h_d = (hi_d - lo_d)/n_d, nodes at lo + (i+1/2) h */
  double gamma, Re;     /* Re <= 0: inviscid */
  double qinf[5];       /* free-stream conservative state [rho, m_x, m_y, (m_z), E] */
  int scheme;           /* 0 = WENO5-JS, 1 = TENO5 */
  int bc[3][2];         /* 0 = zero gradient, 1 = free stream, 2 = periodic, 3 = characteristic
                           (Thompson's non-reflecting condition; needs n >= 5) */
  int sponge_cells;     /* 0: no sponge */
  double sponge_sigma;  /* sigma_max */
  double alpha_pen, beta_pen; /* Eq. 7 constants */
  /* periodic Gaussian pressure source (Sec. 3.6, Eq. 16), added to the energy equation:
   * S_E = src_amp exp(-src_b ln2 |x - src_xc|^2) cos(src_omega t) / (gamma - 1); src_amp = 0: none */
  double src_amp, src_b, src_omega, src_xc[3];
  double time;          /* time at which orc_rhs evaluates the source; start time of orc_rk3 */
  /* 0: component-wise reconstruction of the split fluxes; 1: characteristic-wise, projected on
   * the eigenvectors of the Euler flux Jacobian at the Roe average of the two cells of each face */
  int charwise;
  /* stretched (non-uniform) grid, per direction; NULL: uniform.  Node coordinates x_i and the
   * metric dx/dxi at the nodes for i = -4 .. n+3, stored at i + 4 (n + 8 entries), of a mapping
   * x(xi) of a computational coordinate with unit spacing per cell.  Immersed-boundary markers
   * and probes must have their four-point support where the metric is constant. */
  const double *xnode[3], *xmetric[3];
  /* learned reconstruction weights (scheme 2): where TENO5 keeps all three stencils and the
   * stencil amplitude amp = max_j |v_j - v_2| exceeds mlp_floor, the weights of the candidates
   * come from the network 5 -> 32 -> 32 -> 32 (gelu) -> 3 (softmax) on x = (v - v_2)/amp, and
   * the face value is v_2 + amp sum_k w_k qhat_k(x); elsewhere TENO5.  mlp_params: 2403
   * parameters [W1 (32x5), b1, W2 (32x32), b2, W3 (32x32), b3, W4 (3x32), b4], rows = output
   * units, used as given; mlp_round = 1 rounds the network's input and hidden activations to
   * bfloat16 (the operand precision of the tensor-core products), accumulating in FP64. */
  const double *mlp_params;
  int mlp_round;
  double mlp_floor;
} orc_desc;

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_BOUNDS = -4, ORC_ERR_NOMEM = -7 };

/* Roe average of the conservative states Ql, Qr (nv = dim + 2) and the right (columns) and
 * left (rows) eigenvectors of the flux Jacobian along direction a there, row-major nv x nv;
 * lam (may be NULL) receives the eigenvalues u_a - c, u_a (entropy, then shear), u_a + c. */
int orc_char_eigen(int dim, double gamma, int a, const double *Ql, const double *Qr, double *R,
                   double *Lv, double *lam);

int orc_rhs(const orc_desc *d, const double *Q, int nm, const double *X, const double *U,
            const double *dS, const double *xi, double *L, double *F, double *rate,
            double *alpha_out);

#endif
