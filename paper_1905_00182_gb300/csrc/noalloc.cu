// noalloc.cu -- right-hand side evaluation for callers that cannot allocate device memory.
//
// Some callers of this library have no way to call cudaMalloc: plug-ins whose host application
// owns the whole device-memory budget, latency-critical loops where the implicit device-wide
// synchronisation of cudaMalloc/cudaFree is not acceptable, and foreign-language front ends that
// can only hand over pointers they were given.  ibfsa_rhs_noalloc serves them: it evaluates the
// same right-hand side as ibfsa_rhs, but instead of a caller-allocated workspace it uses one
// file-scope device array of fixed size (IBFSA_NOALLOC_SCRATCH_BYTES) that is part of the
// library image, so every GPU that loads the library holds it until the process exits.
//
// The array's name is only a host-side stand-in in host code, not a device address: handing it
// to a kernel would fault or, on a GPU that can reach host memory, silently touch the wrong
// memory.  So the first call on each device looks up the real device address with
// cudaGetSymbolAddress (with that device current) and caches it, keyed by the device and by the
// unique id of its current context; later calls in the same context reuse it.  A context that
// is destroyed and re-created (cudaDeviceReset) has a new id, so the first call after it looks
// the address up again instead of handing the kernels a stale one.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "ibfsa_internal.h"

namespace ibfsa {
namespace {

constexpr size_t SCRATCH = IBFSA_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_ptr[MAX_DEVICES] = {};
unsigned long long g_ctx[MAX_DEVICES] = {};  // context id the cached address belongs to

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// unique id of the calling thread's current context (driver entry points fetched through the
// runtime, so the library needs no link against the driver library)
cudaError_t current_context_id(unsigned long long *id) {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_cur || !get_id) {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess || q2 != cudaDriverEntryPointSuccess)
      return cudaErrorNotSupported;
    get_cur = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  return get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

int fail(int code, const char *fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  record_error(msg);  // read back with ibfsa_last_error()
  return code;
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// device address of the static scratch on the current device (looked up once per device and
// context)
int scratch_address(void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(IBFSA_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= MAX_DEVICES) return fail(IBFSA_ERR_ARG, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long ctx = 0;
  // no current context yet (a fresh thread before any runtime call made one): the symbol lookup
  // below creates the primary context; its id is then read again
  bool have_ctx = current_context_id(&ctx) == cudaSuccess;
  if (!g_ptr[dev] || !have_ctx || g_ctx[dev] != ctx) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(IBFSA_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s",
                  cudaGetErrorString(e));
    e = current_context_id(&ctx);
    if (e != cudaSuccess)
      return fail(IBFSA_ERR_CUDA, "current context id: %s", cudaGetErrorString(e));
    g_ptr[dev] = p;
    g_ctx[dev] = ctx;
  }
  *out = g_ptr[dev];
  return IBFSA_OK;
}

}  // namespace
}  // namespace ibfsa

using namespace ibfsa;

extern "C" int ibfsa_rhs_noalloc(const ibfsa_grid_desc *desc, const double *Q, int n_markers,
                                 const double *X, const double *U, const double *dS,
                                 const double *xi, double *L, double *F, int *status,
                                 void *cuda_stream) {
  if (!desc || !Q || !L) return fail(IBFSA_ERR_ARG, "NULL descriptor, state or output");
  // the descriptor rules are those of the grid API; ibfsa_workspace_bytes checks them
  size_t ws = 0;
  int rc = ibfsa_workspace_bytes(desc, &ws);
  if (rc) return rc;  // ibfsa_last_error() already names the offending field
  if (desc->precision != IBFSA_FP64)
    return fail(IBFSA_ERR_UNSUPPORTED, "ibfsa_rhs_noalloc evaluates the FP64 arithmetic only");
  if (n_markers < 0) return fail(IBFSA_ERR_ARG, "negative marker count");
  if (n_markers > 0 && (!X || !U || !dS || !xi))
    return fail(IBFSA_ERR_ARG, "NULL marker array with %d markers", n_markers);

  Plan p;
  plan_geometry(*desc, p);
  p.max_markers = n_markers;
  p.nm = n_markers;
  // scratch carve-up: padded state, primitives, viscous fluxes, strict-mode force field,
  // marker forces (when the caller passes none), split speeds, status word
  size_t need = 0;
  size_t o_Qp = need; need += a256(sizeof(double) * p.nv * (size_t)p.NP);
  size_t o_Wp = need; need += a256(sizeof(double) * (p.dim + 1) * (size_t)p.NP);
  size_t o_V = need;
  if (desc->Re > 0.0) need += a256(sizeof(double) * p.dim * (p.dim + 1) * (size_t)p.NB);
  size_t o_f = need;
  if (desc->strict_fp && n_markers > 0) need += a256(sizeof(double) * p.dim * (size_t)p.N);
  size_t o_F = need;
  if (!F && n_markers > 0) need += a256(sizeof(double) * p.dim * (size_t)n_markers);
  size_t o_al = need; need += 256;
  size_t o_st = need; need += 256;
  if (need > SCRATCH)
    return fail(IBFSA_ERR_WORKSPACE,
                "this grid needs %zu bytes of scratch; the static scratch of ibfsa_rhs_noalloc "
                "holds %zu bytes (use ibfsa_rhs with a caller-allocated workspace)",
                need, (size_t)SCRATCH);

  void *base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  char *s = (char *)base;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  p.Qp = (double *)(s + o_Qp);
  p.Wp = (double *)(s + o_Wp);
  p.V = (double *)(s + o_V);
  p.f = (double *)(s + o_f);
  p.F = F ? F : (double *)(s + o_F);
  p.alpha_bits = (unsigned long long *)(s + o_al);
  p.status = (int *)(s + o_st);
  p.L = L;  // the output doubles as the accumulator; the finish pass rewrites it in place
  p.X = X;
  p.U = U;
  p.dS = dS;

  // the scratch keeps the previous call's contents: zero the status word (the split speeds and
  // the strict-mode force field are zeroed by the stage sequence itself)
  cudaError_t e = cudaMemsetAsync(p.status, 0, sizeof(int), st);
  if (e != cudaSuccess) return fail(IBFSA_ERR_CUDA, "status reset: %s", cudaGetErrorString(e));

  StageArgs a{};
  a.Qs = Q;
  a.Lout = L;
  a.xis = xi;
  a.stage = -1;
  a.prof = nullptr;
  e = desc->strict_fp ? strict_stage(p, a, st) : fast_stage(p, a, st);
  if (e != cudaSuccess) return fail(IBFSA_ERR_CUDA, "stage kernels: %s", cudaGetErrorString(e));
  if (status) {
    e = cudaMemcpyAsync(status, p.status, sizeof(int), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(IBFSA_ERR_CUDA, "status copy: %s", cudaGetErrorString(e));
  }
  return IBFSA_OK;
}
