// api.cu -- the C ABI of libibfsa (include/ibfsa.h): descriptor checks, workspace layout, grid
// object, and the host sequence of stages of the third-order SSP Runge-Kutta step
// (arXiv:1905.00182, Sec. 2, text after Eq. 5).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "ibfsa_internal.h"

namespace ibfsa {

static thread_local char g_err[512] = "";

static int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

void record_error(const char *msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

static int cuda_fail(cudaError_t e, const char *where) {
  return fail(IBFSA_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static int check_desc(const ibfsa_grid_desc *d) {
  if (!d) return fail(IBFSA_ERR_ARG, "descriptor is NULL");
  if (d->dim != 2 && d->dim != 3) return fail(IBFSA_ERR_ARG, "dim must be 2 or 3 (got %d)", d->dim);
  for (int a = 0; a < d->dim; a++) {
    if (d->n[a] < 1) return fail(IBFSA_ERR_ARG, "n[%d] = %d must be >= 1", a, d->n[a]);
    if (!(d->hi[a] > d->lo[a])) return fail(IBFSA_ERR_ARG, "hi[%d] must exceed lo[%d]", a, a);
    for (int s = 0; s < 2; s++) {
      if (d->bc[a][s] < 0 || d->bc[a][s] > 3)
        return fail(IBFSA_ERR_ARG, "bc[%d][%d] = %d is not a boundary rule", a, s, d->bc[a][s]);
      if (d->bc[a][s] == IBFSA_BC_CHARACTERISTIC && d->n[a] < 5)
        return fail(IBFSA_ERR_ARG, "a characteristic face needs n[%d] >= 5 (got %d)", a, d->n[a]);
    }
    bool p0 = d->bc[a][0] == IBFSA_BC_PERIODIC, p1 = d->bc[a][1] == IBFSA_BC_PERIODIC;
    if (p0 != p1) return fail(IBFSA_ERR_ARG, "periodic direction %d needs both faces periodic", a);
    if (p0 && d->n[a] < NG) return fail(IBFSA_ERR_ARG, "periodic direction %d needs n >= %d", a, NG);
  }
  if (d->dim == 2 && d->n[2] != 1) return fail(IBFSA_ERR_ARG, "n[2] must be 1 in 2D");
  long long cells = 1, padded = 1;
  for (int a = 0; a < d->dim; a++) {
    cells *= d->n[a];
    padded *= d->n[a] + 2 * NG;
  }
  // offsets inside one component array are 32-bit in the kernels
  if (padded >= (1LL << 31)) return fail(IBFSA_ERR_ARG, "grid too large (padded cells >= 2^31)");
  if (!(d->gamma > 1.0)) return fail(IBFSA_ERR_ARG, "gamma must exceed 1");
  if (!(d->qinf[0] > 0.0)) return fail(IBFSA_ERR_ARG, "free-stream density must be positive");
  if (d->scheme != IBFSA_WENO5JS && d->scheme != IBFSA_TENO5 && d->scheme != IBFSA_MLP_TENO5)
    return fail(IBFSA_ERR_UNSUPPORTED, "scheme %d is not provided by the library", d->scheme);
  if (d->scheme == IBFSA_MLP_TENO5 && d->precision != IBFSA_FP32_PERTURB)
    return fail(IBFSA_ERR_UNSUPPORTED, "the learned weights run in the FP32 perturbation form");
  if (d->precision != IBFSA_FP64 && d->precision != IBFSA_FP32_PERTURB)
    return fail(IBFSA_ERR_UNSUPPORTED, "precision %d is not provided by the library", d->precision);
  if (d->precision == IBFSA_FP32_PERTURB && d->strict_fp)
    return fail(IBFSA_ERR_UNSUPPORTED, "strict_fp applies to the FP64 arithmetic only");
  if (d->sponge_cells < 0 || d->max_markers < 0 || d->max_probes < 0)
    return fail(IBFSA_ERR_ARG, "negative sponge width or capacity");
  if (d->charwise != 0 && d->charwise != 1) return fail(IBFSA_ERR_ARG, "charwise must be 0 or 1");
  if (d->charwise && d->scheme == IBFSA_MLP_TENO5)
    return fail(IBFSA_ERR_UNSUPPORTED, "the learned weights reconstruct component-wise");
  (void)cells;
  return IBFSA_OK;
}

void plan_geometry(const ibfsa_grid_desc &d, Plan &p) {
  memset(&p, 0, sizeof(p));
  p.dim = d.dim;
  p.nv = d.dim + 2;
  p.charwise = d.charwise;
  p.N = 1;
  p.NP = 1;
  p.NB = 1;
  for (int a = 0; a < 3; a++) {
    bool act = a < d.dim;
    p.n[a] = act ? d.n[a] : 1;
    p.g[a] = act ? NG : 0;
    p.P[a] = p.n[a] + 2 * p.g[a];
    p.B[a] = act ? p.n[a] + 4 : 1;
    p.N *= p.n[a];
    p.NP *= p.P[a];
    p.NB *= p.B[a];
    p.lo[a] = d.lo[a];
    p.h[a] = act ? (d.hi[a] - d.lo[a]) / d.n[a] : 1.0;
    p.inv_h[a] = 1.0 / p.h[a];
    p.h12[a] = 12.0 * p.h[a];
    p.inv_h12[a] = 1.0 / p.h12[a];
  }
  p.gamma = d.gamma;
  p.gm1 = d.gamma - 1.0;
  p.Re = d.Re;
  p.inv_Re = d.Re > 0.0 ? 1.0 / d.Re : 0.0;
  for (int c = 0; c < 5; c++) p.qinf[c] = d.qinf[c];
  double ke = 0.0;
  for (int a = 0; a < d.dim; a++) {
    p.prim_inf[a] = d.qinf[1 + a] / d.qinf[0];
    ke += d.qinf[1 + a] * (d.qinf[1 + a] / d.qinf[0]);
  }
  p.p_inf = (d.gamma - 1.0) * (d.qinf[d.dim + 1] - 0.5 * ke);
  p.prim_inf[3] = p.p_inf;
  p.scheme = d.scheme;
  for (int a = 0; a < 3; a++)
    for (int s = 0; s < 2; s++) p.bc[a][s] = d.bc[a][s];
  p.sponge_cells = d.sponge_cells;
  p.sponge_sigma = d.sponge_sigma;
  p.alpha_pen = d.alpha_pen;
  p.beta_pen = d.beta_pen;
  p.hprod = 1.0;
  for (int a = 0; a < d.dim; a++) p.hprod *= p.h[a];
  // TENO5 weights of the kept stencils: d_k delta_k / sum_j d_j delta_j, d = (0.1, 0.6, 0.3)
  const double dlin[3] = {0.1, 0.6, 0.3};
  for (int m = 0; m < 8; m++) {
    double w[3], sw = 0.0;
    for (int k = 0; k < 3; k++) {
      w[k] = (m >> k) & 1 ? dlin[k] : 0.0;
      sw += w[k];
    }
    for (int k = 0; k < 3; k++) p.teno_w[m][k] = sw > 0.0 ? w[k] / sw : 0.0;
  }
  p.max_markers = d.max_markers;
  for (int m = 0; m < 8; m++)
    for (int k = 0; k < 3; k++) p.teno_w32[m][k] = (float)p.teno_w[m][k];
  for (int a = 0; a < 3; a++) {
    p.inv_h32[a] = (float)p.inv_h[a];
    p.inv_h12_32[a] = (float)p.inv_h12[a];
    p.u_inf32[a] = a < d.dim ? (float)p.prim_inf[a] : 0.f;
    p.m_inf32[a] = a < d.dim ? (float)d.qinf[1 + a] : 0.f;
  }
  p.inv_Re32 = (float)p.inv_Re;
  p.rho_inf32 = (float)d.qinf[0];
  p.p_inf32 = (float)p.p_inf;
  p.H_inf32 = (float)(d.qinf[d.dim + 1] + p.p_inf);
  p.gamma32 = (float)d.gamma;
  p.gm1_32 = (float)(d.gamma - 1.0);
}

Layout layout_for(const ibfsa_grid_desc &d) {
  Plan p;
  plan_geometry(d, p);
  Layout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(bytes);
    return o;
  };
  size_t state = sizeof(double) * p.nv * (size_t)p.N;
  size_t M = (size_t)(d.max_markers > 0 ? d.max_markers : 1);
  size_t Pn = (size_t)(d.max_probes > 0 ? d.max_probes : 1);
  L.Q = take(state);
  if (d.precision == IBFSA_FP32_PERTURB) {
    // FP32 form: [qn32 | d1] and d2, FP32 each (the FP64 stage states are not needed)
    L.Q1 = take(2 * sizeof(float) * p.nv * (size_t)p.N);
    L.Q2 = take(sizeof(float) * p.nv * (size_t)p.N);
  } else {
    L.Q1 = take(state);
    L.Q2 = take(state);
  }
  // the FP32 perturbation form keeps the right-hand side and the padded stencil inputs in FP32
  size_t el = d.precision == IBFSA_FP32_PERTURB ? sizeof(float) : sizeof(double);
  L.L = take(el * p.nv * (size_t)p.N);
  L.Qp = take(el * p.nv * (size_t)p.NP);
  L.Wp = take(el * (p.dim + 1) * (size_t)p.NP);
  L.V = d.Re > 0.0 ? take(el * p.dim * (p.dim + 1) * (size_t)p.NB) : take(0);
  L.f = (d.strict_fp && d.max_markers > 0) ? take(sizeof(double) * p.dim * (size_t)p.N) : take(0);
  L.X = take(sizeof(double) * p.dim * M);
  L.U = take(sizeof(double) * p.dim * M);
  L.dS = take(sizeof(double) * M);
  L.F = take(sizeof(double) * p.dim * M);
  L.xi = take(sizeof(double) * p.dim * M);
  L.xi1 = take(sizeof(double) * p.dim * M);
  L.xi2 = take(sizeof(double) * p.dim * M);
  L.alpha = take(sizeof(unsigned long long) * 4);
  L.status = take(sizeof(int) * 4);
  L.probe_xp = take(sizeof(double) * p.dim * Pn);
  L.probe_out = take(sizeof(double) * Pn);
  L.mlp_img = take(d.scheme == IBFSA_MLP_TENO5 ? mlp_image_bytes() : 0);
  L.mlp_counts = take(sizeof(unsigned long long) * 4);
  L.reduce = take(sizeof(double) * 4);
  for (int a = 0; a < 3; a++) L.mesh[a] = a < d.dim ? take(mesh_bytes(p.n[a])) : take(0);
  L.total = off;
  return L;
}

// 1/(dx/dxi) and 1/(12 dx/dxi) of one direction's nodes, in FP64 (correctly rounded divisions)
// and rounded to FP32
__global__ void k_mesh_derive(int count, const double *__restrict__ m, double *inv, double *inv12,
                              float *inv32, float *inv12_32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double a = 1.0 / m[i], b = 1.0 / (12.0 * m[i]);
  inv[i] = a;
  inv12[i] = b;
  inv32[i] = (float)a;
  inv12_32[i] = (float)b;
}

cudaError_t mesh_derive(int count, const double *metric, double *inv, double *inv12, float *inv32,
                        float *inv12_32, cudaStream_t st) {
  k_mesh_derive<<<(count + 127) / 128, 128, 0, st>>>(count, metric, inv, inv12, inv32, inv12_32);
  return cudaGetLastError();
}

void prof_begin(Prof *pr, cudaStream_t st) {
  if (!pr || !pr->on) return;
  if (pr->used == Prof::POOL) prof_harvest(pr);
  cudaEventRecord(pr->ev[2 * pr->used], st);
}

void prof_end(Prof *pr, int cls, cudaStream_t st) {
  if (!pr) return;
  pr->launches[cls]++;
  if (!pr->on) return;
  cudaEventRecord(pr->ev[2 * pr->used + 1], st);
  pr->cls[pr->used++] = cls;
}

cudaError_t prof_harvest(Prof *pr) {
  if (!pr || pr->used == 0) return cudaSuccess;
  cudaError_t e = cudaEventSynchronize(pr->ev[2 * pr->used - 1]);
  for (int i = 0; i < pr->used && e == cudaSuccess; i++) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, pr->ev[2 * i], pr->ev[2 * i + 1]);
    pr->ms[pr->cls[i]] += ms;
    pr->timed[pr->cls[i]]++;
  }
  pr->used = 0;
  return e;
}

static cudaError_t run_stage(Grid *G, const StageArgs &s) {
  if (G->d.scheme == IBFSA_MLP_TENO5 && !G->mlp_set) return cudaErrorInvalidValue;
  if (G->d.precision == IBFSA_FP32_PERTURB) {
    if (!G->qn32_valid) {
      cudaError_t e = fp32_refresh(G->p, G->Q, G->stream);
      if (e != cudaSuccess) return e;
      G->qn32_valid = true;
    }
    return fp32_stage(G->p, s, G->stream);
  }
  return G->d.strict_fp ? strict_stage(G->p, s, G->stream) : fast_stage(G->p, s, G->stream);
}

cudaError_t grid_stage(Grid *G, const StageArgs &s) { return run_stage(G, s); }

double source_scale(const Grid &G, double t) {
  return G.p.src_on ? (G.src_amp * cos(G.src_omega * t)) / (G.d.gamma - 1.0) : 0.0;
}

int api_fail(int code, const char *msg) { return fail(code, "%s", msg); }

}  // namespace ibfsa

using namespace ibfsa;

extern "C" {

const char *ibfsa_last_error(void) { return g_err; }

int ibfsa_workspace_bytes(const ibfsa_grid_desc *desc, size_t *bytes) {
  int rc = check_desc(desc);
  if (rc) return rc;
  if (!bytes) return fail(IBFSA_ERR_ARG, "bytes is NULL");
  *bytes = layout_for(*desc).total;
  return IBFSA_OK;
}

int ibfsa_create_grid(const ibfsa_grid_desc *desc, void *d_workspace, size_t workspace_bytes,
                      void *cuda_stream, ibfsa_grid **out) {
  int rc = check_desc(desc);
  if (rc) return rc;
  if (!out) return fail(IBFSA_ERR_ARG, "out is NULL");
  *out = nullptr;
  Layout L = layout_for(*desc);
  if (!d_workspace || workspace_bytes < L.total)
    return fail(IBFSA_ERR_WORKSPACE, "workspace of %zu bytes given, %zu needed", workspace_bytes,
                L.total);
  if (((uintptr_t)d_workspace & 255) != 0)
    return fail(IBFSA_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  ibfsa_grid *h = new (std::nothrow) ibfsa_grid;
  if (!h) return fail(IBFSA_ERR_ARG, "host allocation of the grid object failed");
  Grid &G = h->g;
  G.d = *desc;
  plan_geometry(*desc, G.p);
  G.stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&G.device);
  char *w = (char *)d_workspace;
  G.Q = (double *)(w + L.Q);
  G.Q1 = (double *)(w + L.Q1);
  G.Q2 = (double *)(w + L.Q2);
  G.p.qn32 = (float *)(w + L.Q1);
  G.p.d1 = G.p.qn32 + (size_t)G.p.nv * G.p.N;
  G.p.d2 = (float *)(w + L.Q2);
  G.qn32_valid = false;
  G.p.L = (double *)(w + L.L);
  G.p.Qp = (double *)(w + L.Qp);
  G.p.Wp = (double *)(w + L.Wp);
  G.p.V = (double *)(w + L.V);
  G.p.Qp32 = (float *)(w + L.Qp);
  G.p.Wp32 = (float *)(w + L.Wp);
  G.p.V32 = (float *)(w + L.V);
  G.p.L32 = (float *)(w + L.L);
  G.p.f = (double *)(w + L.f);
  G.X = (double *)(w + L.X);
  G.U = (double *)(w + L.U);
  G.dS = (double *)(w + L.dS);
  G.p.X = G.X;
  G.p.U = G.U;
  G.p.dS = G.dS;
  G.p.F = (double *)(w + L.F);
  G.xi = (double *)(w + L.xi);
  G.xi1 = (double *)(w + L.xi1);
  G.xi2 = (double *)(w + L.xi2);
  G.p.alpha_bits = (unsigned long long *)(w + L.alpha);
  G.p.status = (int *)(w + L.status);
  G.probe_xp = (double *)(w + L.probe_xp);
  G.probe_out = (double *)(w + L.probe_out);
  G.max_probes = desc->max_probes;
  G.p.mlp_img = (const unsigned char *)(w + L.mlp_img);
  G.p.mlp_counts = (unsigned long long *)(w + L.mlp_counts);
  G.p.probe_scratch = (double *)(w + L.reduce);
  G.p.mlp_floor = 1e-9f;
  for (int a = 0; a < 3; a++) G.mesh_ws[a] = w + L.mesh[a];  // directions start uniform
  G.mlp_set = false;
  G.t = 0.0;
  G.src_amp = 0.0;
  G.src_omega = 0.0;
  G.p.nm = 0;
  cudaError_t e = cudaMemsetAsync(G.p.status, 0, sizeof(int) * 4, G.stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(G.p.mlp_counts, 0, sizeof(unsigned long long) * 4, G.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(G.p.F, 0, L.xi - L.F, G.stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(G.xi, 0, sizeof(double) * G.p.dim * (desc->max_markers > 0 ? desc->max_markers : 1), G.stream);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "ibfsa_create_grid");
  }
  *out = h;
  return IBFSA_OK;
}

int ibfsa_destroy_grid(ibfsa_grid *g) {
  if (g && g->g.prof.created)
    for (int i = 0; i < 2 * Prof::POOL; i++) cudaEventDestroy(g->g.prof.ev[i]);
  delete g;
  return IBFSA_OK;
}

int ibfsa_profile_enable(ibfsa_grid *g, int enable) {
  if (!g) return fail(IBFSA_ERR_ARG, "NULL grid");
  Prof &pr = g->g.prof;
  if (enable && !pr.created) {
    for (int i = 0; i < 2 * Prof::POOL; i++) {
      cudaError_t e = cudaEventCreate(&pr.ev[i]);
      if (e != cudaSuccess) return cuda_fail(e, "ibfsa_profile_enable");
    }
    pr.created = true;
  }
  if (!enable) {
    cudaError_t e = prof_harvest(&pr);
    if (e != cudaSuccess) return cuda_fail(e, "ibfsa_profile_enable");
  }
  pr.on = enable != 0;
  return IBFSA_OK;
}

int ibfsa_profile_read(ibfsa_grid *g, int nclass, double *host_ms, long long *host_launches,
                       long long *host_timed) {
  if (!g || nclass < 0) return fail(IBFSA_ERR_ARG, "bad argument");
  Prof &pr = g->g.prof;
  cudaError_t e = prof_harvest(&pr);
  if (e != cudaSuccess) return cuda_fail(e, "ibfsa_profile_read");
  for (int c = 0; c < nclass && c < K_NCLASS; c++) {
    if (host_ms) host_ms[c] = pr.ms[c];
    if (host_launches) host_launches[c] = pr.launches[c];
    if (host_timed) host_timed[c] = pr.timed[c];
    pr.ms[c] = 0.0;
    pr.launches[c] = 0;
    pr.timed[c] = 0;
  }
  return IBFSA_OK;
}

static bool is_host_pointer(const void *ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeUnregistered;
}

int ibfsa_set_state(ibfsa_grid *g, const double *Q) {
  if (!g || !Q) return fail(IBFSA_ERR_ARG, "NULL argument");
  Grid &G = g->g;
  cudaError_t e = cudaMemcpyAsync(G.Q, Q, sizeof(double) * G.p.nv * G.p.N, cudaMemcpyDefault,
                                  G.stream);
  G.qn32_valid = false;
  return e == cudaSuccess ? IBFSA_OK : cuda_fail(e, "ibfsa_set_state");
}

int ibfsa_get_state(ibfsa_grid *g, double *Q) {
  if (!g || !Q) return fail(IBFSA_ERR_ARG, "NULL argument");
  Grid &G = g->g;
  cudaError_t e = cudaMemcpyAsync(Q, G.Q, sizeof(double) * G.p.nv * G.p.N, cudaMemcpyDefault,
                                  G.stream);
  if (e == cudaSuccess && is_host_pointer(Q)) e = cudaStreamSynchronize(G.stream);
  return e == cudaSuccess ? IBFSA_OK : cuda_fail(e, "ibfsa_get_state");
}

int ibfsa_set_markers(ibfsa_grid *g, int n, const double *X, const double *U, const double *dS,
                      int reset_integral) {
  if (!g) return fail(IBFSA_ERR_ARG, "NULL grid");
  Grid &G = g->g;
  if (n < 0 || n > G.d.max_markers)
    return fail(IBFSA_ERR_ARG, "marker count %d outside [0, %d]", n, G.d.max_markers);
  if (n > 0 && (!X || !U || !dS)) return fail(IBFSA_ERR_ARG, "NULL marker array");
  int M = G.d.max_markers, dim = G.p.dim;
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < dim && e == cudaSuccess && n > 0; a++) {
    e = cudaMemcpyAsync(G.X + (size_t)a * M, X + (size_t)a * n, sizeof(double) * n,
                        cudaMemcpyDefault, G.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(G.U + (size_t)a * M, U + (size_t)a * n, sizeof(double) * n,
                          cudaMemcpyDefault, G.stream);
  }
  if (e == cudaSuccess && n > 0)
    e = cudaMemcpyAsync(G.dS, dS, sizeof(double) * n, cudaMemcpyDefault, G.stream);
  if (e == cudaSuccess && reset_integral)
    e = cudaMemsetAsync(G.xi, 0, sizeof(double) * dim * (M > 0 ? M : 1), G.stream);
  if (e != cudaSuccess) return cuda_fail(e, "ibfsa_set_markers");
  G.p.nm = n;
  return IBFSA_OK;
}

static int copy_marker_array(Grid &G, double *dst_user, const double *src_ws, bool to_user) {
  int M = G.d.max_markers, n = G.p.nm;
  cudaError_t e = cudaSuccess;
  for (int a = 0; a < G.p.dim && e == cudaSuccess && n > 0; a++) {
    if (to_user)
      e = cudaMemcpyAsync(dst_user + (size_t)a * n, src_ws + (size_t)a * M, sizeof(double) * n,
                          cudaMemcpyDefault, G.stream);
    else
      e = cudaMemcpyAsync((double *)src_ws + (size_t)a * M, dst_user + (size_t)a * n,
                          sizeof(double) * n, cudaMemcpyDefault, G.stream);
  }
  if (e == cudaSuccess && to_user && n > 0 && is_host_pointer(dst_user))
    e = cudaStreamSynchronize(G.stream);
  return e == cudaSuccess ? IBFSA_OK : cuda_fail(e, "marker copy");
}

int ibfsa_get_marker_forces(ibfsa_grid *g, double *F) {
  if (!g || !F) return fail(IBFSA_ERR_ARG, "NULL argument");
  return copy_marker_array(g->g, F, g->g.p.F, true);
}

int ibfsa_get_penalty_integral(ibfsa_grid *g, double *xi) {
  if (!g || !xi) return fail(IBFSA_ERR_ARG, "NULL argument");
  return copy_marker_array(g->g, xi, g->g.xi, true);
}

int ibfsa_set_penalty_integral(ibfsa_grid *g, const double *xi) {
  if (!g || !xi) return fail(IBFSA_ERR_ARG, "NULL argument");
  return copy_marker_array(g->g, (double *)xi, g->g.xi, false);
}

int ibfsa_rhs(ibfsa_grid *g, double *L) {
  if (!g || !L) return fail(IBFSA_ERR_ARG, "NULL argument");
  Grid &G = g->g;
  StageArgs s{};
  s.Qs = G.Q;
  s.Qn = G.Q;
  s.Lout = L;
  s.xis = G.xi;
  s.stage = -1;
  s.src_scale = source_scale(G, G.t);
  s.prof = &G.prof;
  if (G.d.scheme == IBFSA_MLP_TENO5 && !G.mlp_set)
    return fail(IBFSA_ERR_ARG, "IBFSA_MLP_TENO5 grid without weights: call ibfsa_set_mlp");
  cudaError_t e = run_stage(&G, s);
  return e == cudaSuccess ? IBFSA_OK : cuda_fail(e, "ibfsa_rhs");
}

int ibfsa_rk3_step(ibfsa_grid *g, double dt, int nsteps) {
  if (!g) return fail(IBFSA_ERR_ARG, "NULL grid");
  if (nsteps < 0 || !(dt > 0.0) || !isfinite(dt))
    return fail(IBFSA_ERR_ARG, "need a finite dt > 0 and nsteps >= 0");
  Grid &G = g->g;
  if (G.d.scheme == IBFSA_MLP_TENO5 && !G.mlp_set)
    return fail(IBFSA_ERR_ARG, "IBFSA_MLP_TENO5 grid without weights: call ibfsa_set_mlp");
  // Shu-Osher coefficients: Q^(s+1) = a_s Qn + b_s (Q^(s) + dt L(Q^(s)))
  const double A[3] = {0.0, 3.0 / 4.0, 1.0 / 3.0}, B[3] = {1.0, 1.0 / 4.0, 2.0 / 3.0};
  const double C[3] = {0.0, 1.0, 0.5};  // stage times t + C dt
  for (int step = 0; step < nsteps; step++) {
    const double *in[3] = {G.Q, G.Q1, G.Q2};
    double *outs[3] = {G.Q1, G.Q2, G.Q};  // stage 3 overwrites Qn cell by cell (pointwise read)
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
      cudaError_t e = run_stage(&G, a);
      if (e != cudaSuccess) return cuda_fail(e, "ibfsa_rk3_step");
    }
    G.t = G.t + dt;
  }
  return IBFSA_OK;
}

int ibfsa_set_source(ibfsa_grid *g, double amp, double b, double omega, const double *xc) {
  if (!g) return fail(IBFSA_ERR_ARG, "NULL grid");
  Grid &G = g->g;
  if (amp != 0.0 && (!xc || !(b > 0.0) || !isfinite(amp) || !isfinite(omega)))
    return fail(IBFSA_ERR_ARG, "pressure source needs b > 0, finite amp and omega, and a centre");
  G.src_amp = amp;
  G.src_omega = omega;
  G.p.src_on = amp != 0.0;
  G.p.src_b = b;
  for (int a = 0; a < 3; a++) G.p.src_xc[a] = (amp != 0.0 && a < G.p.dim) ? xc[a] : 0.0;
  return IBFSA_OK;
}

int ibfsa_set_mesh(ibfsa_grid *g, int a, const double *x_nodes, const double *dxdxi) {
  if (!g) return fail(IBFSA_ERR_ARG, "NULL grid");
  Grid &G = g->g;
  if (a < 0 || a >= G.p.dim) return fail(IBFSA_ERR_ARG, "direction %d outside [0, %d)", a, G.p.dim);
  if (!x_nodes != !dxdxi) return fail(IBFSA_ERR_ARG, "give both node coordinates and metric, or neither");
  if (!x_nodes) {  // back to the uniform spacing of the descriptor's box
    G.p.mx[a] = G.p.mm[a] = G.p.minv[a] = G.p.minv12[a] = nullptr;
    G.p.minv32[a] = G.p.minv12_32[a] = nullptr;
    return IBFSA_OK;
  }
  if (G.d.bc[a][0] == IBFSA_BC_PERIODIC)
    return fail(IBFSA_ERR_UNSUPPORTED, "a stretched direction cannot be periodic");
  const int cnt = G.p.n[a] + 2 * NG;
  // checked on the host: finite, strictly increasing nodes, positive finite metric
  double *hx = new (std::nothrow) double[2 * (size_t)cnt];
  if (!hx) return fail(IBFSA_ERR_ARG, "host allocation failed");
  double *hm = hx + cnt;
  cudaError_t e = cudaMemcpy(hx, x_nodes, sizeof(double) * cnt, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(hm, dxdxi, sizeof(double) * cnt, cudaMemcpyDefault);
  if (e != cudaSuccess) {
    delete[] hx;
    return cuda_fail(e, "ibfsa_set_mesh");
  }
  for (int i = 0; i < cnt; i++) {
    bool ok = isfinite(hx[i]) && isfinite(hm[i]) && hm[i] > 0.0 && (i == 0 || hx[i] > hx[i - 1]);
    if (!ok) {
      delete[] hx;
      return fail(IBFSA_ERR_ARG, "direction %d: node %d is not finite and increasing with a "
                  "positive metric", a, i - NG);
    }
  }
  char *base = (char *)G.mesh_ws[a];
  double *dx = (double *)base, *dm = dx + cnt, *di = dm + cnt, *di12 = di + cnt;
  float *f32 = (float *)(di12 + cnt), *f12 = f32 + cnt;
  e = cudaMemcpyAsync(dx, hx, sizeof(double) * 2 * cnt, cudaMemcpyHostToDevice, G.stream);
  if (e == cudaSuccess) e = mesh_derive(cnt, dm, di, di12, f32, f12, G.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(G.stream);  // hx is freed below
  delete[] hx;
  if (e != cudaSuccess) return cuda_fail(e, "ibfsa_set_mesh");
  G.p.mx[a] = dx;
  G.p.mm[a] = dm;
  G.p.minv[a] = di;
  G.p.minv12[a] = di12;
  G.p.minv32[a] = f32;
  G.p.minv12_32[a] = f12;
  return IBFSA_OK;
}

int ibfsa_set_time(ibfsa_grid *g, double t) {
  if (!g || !isfinite(t)) return fail(IBFSA_ERR_ARG, "NULL grid or non-finite time");
  g->g.t = t;
  return IBFSA_OK;
}

int ibfsa_get_time(ibfsa_grid *g, double *host_t) {
  if (!g || !host_t) return fail(IBFSA_ERR_ARG, "NULL argument");
  *host_t = g->g.t;
  return IBFSA_OK;
}

int ibfsa_max_wavespeed(ibfsa_grid *g, double *host_alpha) {
  if (!g || !host_alpha) return fail(IBFSA_ERR_ARG, "NULL argument");
  Grid &G = g->g;
  cudaError_t e = G.d.precision == IBFSA_FP32_PERTURB ? fp32_wavespeed(G.p, G.Q, G.stream)
                  : G.d.strict_fp                       ? strict_wavespeed(G.p, G.Q, G.stream)
                                                        : fast_wavespeed(G.p, G.Q, G.stream);
  unsigned long long bits[3] = {0, 0, 0};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bits, G.p.alpha_bits, sizeof(bits), cudaMemcpyDeviceToHost, G.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(G.stream);
  if (e != cudaSuccess) return cuda_fail(e, "ibfsa_max_wavespeed");
  for (int a = 0; a < G.p.dim; a++) memcpy(&host_alpha[a], &bits[a], sizeof(double));
  return IBFSA_OK;
}

// Stages the np probe points and samples dp at them into G.probe_out (stream-ordered).
static cudaError_t sample_probes(Grid &G, int np, const double *xp) {
  cudaError_t e = cudaMemcpyAsync(G.probe_xp, xp, sizeof(double) * G.p.dim * np,
                                  cudaMemcpyDefault, G.stream);
  if (e != cudaSuccess) return e;
  return G.d.precision == IBFSA_FP32_PERTURB
             ? fp32_probe(G.p, G.Q, np, G.probe_xp, G.probe_out, G.stream, &G.prof)
         : G.d.strict_fp ? strict_probe(G.p, G.Q, np, G.probe_xp, G.probe_out, G.stream, &G.prof)
                         : fast_probe(G.p, G.Q, np, G.probe_xp, G.probe_out, G.stream, &G.prof);
}

int ibfsa_probe(ibfsa_grid *g, int np, const double *xp, double *out) {
  if (!g || (np > 0 && (!xp || !out))) return fail(IBFSA_ERR_ARG, "NULL argument");
  Grid &G = g->g;
  if (np < 0 || np > G.max_probes)
    return fail(IBFSA_ERR_ARG, "probe count %d outside [0, %d]", np, G.max_probes);
  if (np == 0) return IBFSA_OK;
  cudaError_t e = sample_probes(G, np, xp);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, G.probe_out, sizeof(double) * np, cudaMemcpyDefault, G.stream);
  if (e == cudaSuccess && is_host_pointer(out)) e = cudaStreamSynchronize(G.stream);
  return e == cudaSuccess ? IBFSA_OK : cuda_fail(e, "ibfsa_probe");
}

int ibfsa_probe_accumulate(ibfsa_grid *g, int np, const double *xp, double *out, double *acc) {
  if (!g || (np > 0 && (!xp || !acc))) return fail(IBFSA_ERR_ARG, "NULL argument");
  Grid &G = g->g;
  if (np < 0 || np > G.max_probes)
    return fail(IBFSA_ERR_ARG, "probe count %d outside [0, %d]", np, G.max_probes);
  if (np == 0) return IBFSA_OK;
  if (is_host_pointer(acc)) return fail(IBFSA_ERR_ARG, "acc must be device memory");
  cudaError_t e = sample_probes(G, np, xp);
  if (e == cudaSuccess) e = probe_fold(np, G.probe_out, acc, G.stream);
  if (e == cudaSuccess && out)
    e = cudaMemcpyAsync(out, G.probe_out, sizeof(double) * np, cudaMemcpyDefault, G.stream);
  if (e == cudaSuccess && out && is_host_pointer(out)) e = cudaStreamSynchronize(G.stream);
  return e == cudaSuccess ? IBFSA_OK : cuda_fail(e, "ibfsa_probe_accumulate");
}

int ibfsa_probe_stats(ibfsa_grid *g, int np, const double *acc, double *mean, double *rms) {
  if (!g || (np > 0 && (!acc || !mean || !rms))) return fail(IBFSA_ERR_ARG, "NULL argument");
  Grid &G = g->g;
  if (np < 0) return fail(IBFSA_ERR_ARG, "negative probe count %d", np);
  if (np == 0) return IBFSA_OK;
  if (is_host_pointer(acc) || is_host_pointer(mean) || is_host_pointer(rms))
    return fail(IBFSA_ERR_ARG, "acc, mean and rms must be device memory");
  cudaError_t e = probe_moments(np, acc, mean, rms, G.stream);
  return e == cudaSuccess ? IBFSA_OK : cuda_fail(e, "ibfsa_probe_stats");
}

int ibfsa_set_mlp(ibfsa_grid *g, const void *d_state) {
  if (!g || !d_state) return fail(IBFSA_ERR_ARG, "NULL argument");
  Grid &G = g->g;
  if (G.d.scheme != IBFSA_MLP_TENO5)
    return fail(IBFSA_ERR_ARG, "the grid's scheme is not IBFSA_MLP_TENO5");
  cudaError_t e = cudaMemcpyAsync((void *)G.p.mlp_img, (const char *)d_state + mlp_image_offset(),
                                  mlp_image_bytes(), cudaMemcpyDeviceToDevice, G.stream);
  if (e != cudaSuccess) return cuda_fail(e, "ibfsa_set_mlp");
  G.mlp_set = true;
  return IBFSA_OK;
}

int ibfsa_mlp_stats(ibfsa_grid *g, unsigned long long *host_counts) {
  if (!g || !host_counts) return fail(IBFSA_ERR_ARG, "NULL argument");
  Grid &G = g->g;
  cudaError_t e = cudaMemcpyAsync(host_counts, G.p.mlp_counts, 2 * sizeof(unsigned long long),
                                  cudaMemcpyDeviceToHost, G.stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(G.p.mlp_counts, 0, 2 * sizeof(unsigned long long), G.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(G.stream);
  return e == cudaSuccess ? IBFSA_OK : cuda_fail(e, "ibfsa_mlp_stats");
}

int ibfsa_mlp_sample(ibfsa_grid *g, int n_max, unsigned long long seed, int attempts,
                     float *d_stencils, float *d_targets, int *d_count) {
  if (!g || n_max < 0 || attempts < 1 || !d_stencils || !d_targets || !d_count)
    return fail(IBFSA_ERR_ARG, "bad argument");
  Grid &G = g->g;
  if (G.d.precision != IBFSA_FP32_PERTURB)
    return fail(IBFSA_ERR_UNSUPPORTED, "sampling reads the FP32 perturbation form");
  cudaError_t e = fp32_mlp_sample(G.p, G.Q, n_max, seed, attempts, d_stencils, d_targets,
                                  d_count, G.stream);
  G.qn32_valid = true;
  return e == cudaSuccess ? IBFSA_OK : cuda_fail(e, "ibfsa_mlp_sample");
}

int ibfsa_body_force(ibfsa_grid *g, double *host_force, double *host_power) {
  if (!g || !host_force) return fail(IBFSA_ERR_ARG, "NULL argument");
  Grid &G = g->g;
  double out[4] = {0.0, 0.0, 0.0, 0.0};
  cudaError_t e = body_force(G.p, G.U, G.p.probe_scratch, G.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, G.p.probe_scratch, sizeof(out), cudaMemcpyDeviceToHost, G.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(G.stream);
  if (e != cudaSuccess) return cuda_fail(e, "ibfsa_body_force");
  for (int a = 0; a < G.p.dim; a++) host_force[a] = out[a];
  if (host_power) *host_power = out[3];
  return IBFSA_OK;
}

int ibfsa_selftest_wait(ibfsa_grid *g) {
  if (!g) return fail(IBFSA_ERR_ARG, "NULL grid");
  cudaError_t e = wait_selftest(g->g.p, g->g.stream);
  return e == cudaSuccess ? IBFSA_OK : cuda_fail(e, "ibfsa_selftest_wait");
}

int ibfsa_get_status(ibfsa_grid *g, int *host_flags) {
  if (!g || !host_flags) return fail(IBFSA_ERR_ARG, "NULL argument");
  Grid &G = g->g;
  int v = 0;
  cudaError_t e = cudaMemcpyAsync(&v, G.p.status, sizeof(int), cudaMemcpyDeviceToHost, G.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(G.p.status, 0, sizeof(int), G.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(G.stream);
  if (e != cudaSuccess) return cuda_fail(e, "ibfsa_get_status");
  *host_flags = v;
  return IBFSA_OK;
}

}  // extern "C"
