// ibfsa_internal.h -- grid object, device plan and launch interface shared by the CUDA
// translation units of libibfsa (never by anything outside this library).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ibfsa.h"

namespace ibfsa {

constexpr int NG = 4;  // ghost layers: a fourth-order derivative of a fourth-order derivative

// Everything a kernel needs, passed by value.  Padded arrays cover [-4, n+4) in every active
// direction (one layer of extent 1 in an inactive z), x fastest.
struct Plan {
  int dim, nv;
  int charwise;   // characteristic-wise reconstruction (FP64 forms)
  int n[3];       // interior extents (n[2] = 1 in 2D)
  int P[3];       // padded extents
  int g[3];       // ghost layers per direction (4 or 0)
  long long N;    // interior cells
  long long NP;   // padded cells
  double lo[3], h[3], inv_h[3], h12[3], inv_h12[3];  // h12 = 12 h
  double gamma, gm1, Re, inv_Re;
  double qinf[5];
  double prim_inf[4];  // u, v, w, p of the free stream
  double p_inf;
  int scheme;
  int bc[3][2];
  int sponge_cells;
  double sponge_sigma;
  double alpha_pen, beta_pen;
  // periodic Gaussian pressure source (Sec. 3.6, Eq. 16) in the energy equation:
  // src_scale exp(-src_b ln2 |x - src_xc|^2), src_scale = amp cos(omega t_stage) / (gamma - 1)
  int src_on;
  double src_b, src_xc[3], src_scale;
  double hprod;        // product of h over active directions
  // non-uniform mesh (Sec. 2): per direction, node coordinates x_i, the metric dx/dxi, 1/(dx/dxi)
  // and 1/(12 dx/dxi) at the nodes i = -NG .. n+NG-1 (stored at i + NG), FP64, and the two
  // reciprocals in FP32.  NULL: the direction is uniform with spacing h (the formulas then use
  // h itself, so a uniform grid computes exactly what it computes without these arrays).
  const double *mx[3], *mm[3], *minv[3], *minv12[3];
  const float *minv32[3], *minv12_32[3];
  // TENO: 1/sum of kept linear weights per cut-off mask (bit k = stencil k kept)
  double teno_w[8][3];
  // single-precision copies for the FP32 perturbation form
  float teno_w32[8][3];
  float inv_h32[3], inv_h12_32[3], inv_Re32;
  float rho_inf32, p_inf32, H_inf32, gamma32, gm1_32, u_inf32[3], m_inf32[3];

  // device buffers
  double *Qp;          // padded conservative state [nv][NP]
  double *Wp;          // padded primitives [u, v, (w), p] -> [dim+1][NP]
  double *L;           // right-hand side accumulator [nv][N]
  double *V;           // viscous fluxes on the box [-2, n+2): [dim][dim+1][NB]
  int B[3];            // box extents (n + 4 per active direction)
  long long NB;
  double *f;           // strict mode: spread force [dim][N]
  // FP32 perturbation form: the same buffers viewed as float (q - q_inf, primitive
  // perturbations [u', v', w', p'], viscous fluxes, right-hand side)
  float *Qp32, *Wp32, *V32, *L32;
  // the FP32 form carries the stage values of a step as FP32 increments over the FP64 state:
  // qn32 = (float)(Qn - q_inf), d1 = Q1 - Qn, d2 = Q2 - Qn
  float *qn32, *d1, *d2;
  // learned weights (scheme IBFSA_MLP_TENO5): packed bf16 image, counters of the
  // reconstructions that used the network / all reconstructions evaluated, guard floor
  const unsigned char *mlp_img;
  unsigned long long *mlp_counts;
  float mlp_floor;
  double *probe_scratch;   // small reduction results (body force, power)
  unsigned long long *alpha_bits;  // [3] ordered bits of the split speeds
  int *status;
  // markers
  int nm;
  int max_markers;
  const double *X, *U, *dS;   // [dim][max_markers]
  double *F;                  // marker force of Eq. 7 [dim][max_markers]
};

// Kernel classes for launch counting and CUDA-event timing (instrumentation only).
enum KClass {
  K_PAD = 0, K_INTERP, K_CONV_X, K_CONV_Y, K_CONV_Z, K_VISC_FLUX, K_VISC_DIV, K_SPREAD, K_FINISH,
  K_PROBE, K_PLATE, K_NCLASS
};

// Launch counters (always on) and, when enabled, event pairs around every launch on the grid's
// stream; harvested (one synchronisation) when the pool fills or when read.
struct Prof {
  static constexpr int POOL = 1024;
  bool on = false;
  bool created = false;
  long long launches[K_NCLASS] = {};
  long long timed[K_NCLASS] = {};
  double ms[K_NCLASS] = {};
  cudaEvent_t ev[2 * POOL];
  int cls[POOL];
  int used = 0;
};
void prof_begin(Prof *pr, cudaStream_t st);
void prof_end(Prof *pr, int cls, cudaStream_t st);
cudaError_t prof_harvest(Prof *pr);

struct Grid {
  ibfsa_grid_desc d;
  Plan p;
  cudaStream_t stream;
  int device;
  // carved workspace
  double *Q, *Q1, *Q2;         // interior states [nv][N]
  double *X, *U, *dS;          // markers
  double *xi, *xi1, *xi2;      // penalty integrals [dim][max_markers]
  double *probe_xp, *probe_out;
  int max_probes;
  bool qn32_valid;  // FP32 form: qn32 matches Qn
  bool mlp_set;     // learned weights attached (ibfsa_set_mlp)
  double t;         // the grid's clock (stage times t, t + dt, t + dt/2 of a step)
  double src_amp, src_omega;  // pressure source amplitude and angular frequency
  void *mesh_ws[3];           // workspace of each direction's mesh arrays
  Prof prof;
};

// Workspace layout: byte offsets of every buffer for a descriptor.
struct Layout {
  size_t Q, Q1, Q2, Qp, Wp, L, V, f, X, U, dS, F, xi, xi1, xi2, alpha, status, probe_xp,
      probe_out, mlp_img, mlp_counts, reduce, mesh[3], total;
};
// the mesh arrays of one direction with n cells: 4 FP64 and 2 FP32 arrays of n + 2 NG entries
inline size_t mesh_bytes(int n) { return (size_t)(n + 2 * NG) * (4 * sizeof(double) + 2 * sizeof(float)); }
// fills 1/(dx/dxi) and 1/(12 dx/dxi) (FP64, FP32) from the metric of one direction (api.cu)
cudaError_t mesh_derive(int count, const double *metric, double *inv, double *inv12, float *inv32,
                        float *inv12_32, cudaStream_t st);
Layout layout_for(const ibfsa_grid_desc &d);
void record_error(const char *msg);  // sets the thread-local message of ibfsa_last_error
void plan_geometry(const ibfsa_grid_desc &d, Plan &p);


// Launchers, one set per arithmetic mode (strict_fp = 1 / 0), defined in the two stage TUs.
// `stage` < 0 evaluates the right-hand side only (into Lout); otherwise it applies
// Qo = a Qn + b (Qs + dt L(Qs)) and the same to xi.
struct StageArgs {
  const double *Qs;   // stage input, interior
  const double *Qn;   // step start (stage >= 0)
  double *Qo;         // stage output (stage >= 0)
  double *Lout;       // right-hand side output (stage < 0)
  const double *xis, *xin;
  double *xio;
  double a, b, dt;
  int stage;
  double src_scale;   // amp cos(omega t_stage) / (gamma - 1) of the pressure source (0: none)
  Prof *prof;
};
cudaError_t strict_stage(const Plan &p, const StageArgs &s, cudaStream_t st);
cudaError_t fast_stage(const Plan &p, const StageArgs &s, cudaStream_t st);
cudaError_t strict_wavespeed(const Plan &p, const double *Q, cudaStream_t st);
cudaError_t fast_wavespeed(const Plan &p, const double *Q, cudaStream_t st);
cudaError_t fp32_stage(const Plan &p, const StageArgs &s, cudaStream_t st);
cudaError_t fp32_wavespeed(const Plan &p, const double *Q, cudaStream_t st);
cudaError_t fp32_refresh(const Plan &p, const double *Q, cudaStream_t st);
cudaError_t fp32_mlp_sample(const Plan &p, const double *Q, int n_max, unsigned long long seed,
                            int attempts, float *stencils, float *targets, int *count,
                            cudaStream_t st);
cudaError_t body_force(const Plan &p, const double *U, double *out, cudaStream_t st);
cudaError_t wait_selftest(const Plan &p, cudaStream_t st);  // bounded-wait self-test (stage_fp32.cu)
size_t mlp_image_offset();   // byte offset of the packed image inside a training state
size_t mlp_image_bytes();
cudaError_t fp32_probe(const Plan &p, const double *Q, int np, const double *xp, double *out,
                       cudaStream_t st, Prof *pr);
cudaError_t strict_probe(const Plan &p, const double *Q, int np, const double *xp, double *out,
                         cudaStream_t st, Prof *pr);
cudaError_t fast_probe(const Plan &p, const double *Q, int np, const double *xp, double *out,
                       cudaStream_t st, Prof *pr);
// Time statistics of probe signals (stats.cu): acc is [count | mean | M2] per probe.
cudaError_t probe_fold(int np, const double *dp, double *acc, cudaStream_t st);
cudaError_t probe_moments(int np, const double *acc, double *mean, double *rms, cudaStream_t st);

// One stage (or right-hand side) of a grid in its arithmetic form (api.cu).
cudaError_t grid_stage(Grid *G, const StageArgs &s);
// The pressure source's stage factor amp cos(omega t) / (gamma - 1) at time t (api.cu).
double source_scale(const Grid &G, double t);
int api_fail(int code, const char *msg);  // records the message, returns code

}  // namespace ibfsa

struct ibfsa_grid {
  ibfsa::Grid g;
};
