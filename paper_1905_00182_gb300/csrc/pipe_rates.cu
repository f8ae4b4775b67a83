// pipe_rates.cu -- throughput of the arithmetic pipes the stage kernels lean on: the FP64
// fused multiply-add (the FP64 forms' bound), the FP32 fused multiply-add scalar and packed
// (FP32x2), the multi-function unit's tanh, exp2 and reciprocal approximations (the learned
// weights' gelu and softmax), and the FP64 <-> FP32 conversions.  Standalone executable, no
// library calls on a hot path; prints one line per operation: elements per second over the
// whole GPU and elements per clock per SM at the device's maximum SM clock.
//
// Each thread runs eight independent dependency chains of the operation (enough to fill the
// pipes at 8 warps per SM quarter); the grid is 8 blocks of 256 threads per SM; each kernel is
// launched 3 times untimed, then 10 times between CUDA events.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

namespace {

constexpr int ITERS = 2048, CHAINS = 8;

__global__ void k_dfma(double *out, double s) {
  double x[CHAINS];
  for (int c = 0; c < CHAINS; c++) x[c] = s * (threadIdx.x + c + 1);
  for (int i = 0; i < ITERS; i++)
#pragma unroll
    for (int c = 0; c < CHAINS; c++) x[c] = fma(x[c], 0.999, 1e-3);
  double r = 0;
  for (int c = 0; c < CHAINS; c++) r += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void k_ffma(double *out, double s) {
  float x[CHAINS];
  for (int c = 0; c < CHAINS; c++) x[c] = (float)s * (threadIdx.x + c + 1);
  for (int i = 0; i < ITERS; i++)
#pragma unroll
    for (int c = 0; c < CHAINS; c++) x[c] = fmaf(x[c], 0.999f, 1e-3f);
  float r = 0;
  for (int c = 0; c < CHAINS; c++) r += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void k_ffma2(double *out, double s) {
  float2 x[CHAINS];
  for (int c = 0; c < CHAINS; c++) x[c] = make_float2((float)s * (threadIdx.x + c + 1), (float)s * c);
  const float2 a = make_float2(0.999f, 0.999f), b = make_float2(1e-3f, 1e-3f);
  for (int i = 0; i < ITERS; i++)
#pragma unroll
    for (int c = 0; c < CHAINS; c++) x[c] = __ffma2_rn(x[c], a, b);
  float r = 0;
  for (int c = 0; c < CHAINS; c++) r += x[c].x + x[c].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void k_tanh(double *out, double s) {
  float x[CHAINS];
  for (int c = 0; c < CHAINS; c++) x[c] = (float)s * (threadIdx.x + c + 1);
  for (int i = 0; i < ITERS; i++)
#pragma unroll
    for (int c = 0; c < CHAINS; c++) asm volatile("tanh.approx.f32 %0, %0;" : "+f"(x[c]));
  float r = 0;
  for (int c = 0; c < CHAINS; c++) r += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void k_tanh_h2(double *out, double s) {
  uint32_t x[CHAINS];
  for (int c = 0; c < CHAINS; c++) {
    __half2 h = __floats2half2_rn((float)s * (threadIdx.x + c + 1), (float)s * (c + 2));
    x[c] = *reinterpret_cast<uint32_t *>(&h);
  }
  for (int i = 0; i < ITERS; i++)
#pragma unroll
    for (int c = 0; c < CHAINS; c++) asm volatile("tanh.approx.f16x2 %0, %0;" : "+r"(x[c]));
  float r = 0;
  for (int c = 0; c < CHAINS; c++) {
    __half2 h = *reinterpret_cast<__half2 *>(&x[c]);
    r += __low2float(h) + __high2float(h);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void k_ex2(double *out, double s) {
  float x[CHAINS];
  for (int c = 0; c < CHAINS; c++) x[c] = -(float)s * (threadIdx.x + c + 1);
  for (int i = 0; i < ITERS; i++)
#pragma unroll
    for (int c = 0; c < CHAINS; c++) asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(x[c]));
  float r = 0;
  for (int c = 0; c < CHAINS; c++) r += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void k_rcp(double *out, double s) {
  float x[CHAINS];
  for (int c = 0; c < CHAINS; c++) x[c] = 1.f + (float)s * (threadIdx.x + c + 1);
  // x <- 1/x + 1 (a reciprocal of a reciprocal could be folded away; the added 1 keeps every
  // reciprocal, and one addition per element on the fused multiply-add pipe is far below it)
  for (int i = 0; i < ITERS; i++)
#pragma unroll
    for (int c = 0; c < CHAINS; c++)
      asm volatile("rcp.approx.ftz.f32 %0, %0;\n\tadd.ftz.f32 %0, %0, 0f3F800000;" : "+f"(x[c]));
  float r = 0;
  for (int c = 0; c < CHAINS; c++) r += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// double -> float -> double: two conversions per element (the pipe they issue to bounds it)
__global__ void k_cvt(double *out, double s) {
  double x[CHAINS];
  for (int c = 0; c < CHAINS; c++) x[c] = 1.0 + s * (threadIdx.x + c + 1);
  for (int i = 0; i < ITERS; i++)
#pragma unroll
    for (int c = 0; c < CHAINS; c++) {
      float f;
      asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(f) : "d"(x[c]));
      asm volatile("cvt.f64.f32 %0, %1;" : "=d"(x[c]) : "f"(f));
    }
  double r = 0;
  for (int c = 0; c < CHAINS; c++) r += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

struct Op {
  const char *name;
  void (*k)(double *, double);
  int per_instr;  // elements per thread instruction
};

}  // namespace

int main() {
  int sms = 0, khz = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess ||
      cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, 0) != cudaSuccess) {
    fprintf(stderr, "no CUDA device\n");
    return 1;
  }
  const int grid = sms * 8, block = 256;
  double *out = nullptr;
  if (cudaMalloc(&out, sizeof(double) * grid * block) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const Op ops[] = {{"fma.rn.f64", k_dfma, 1},         {"fma.rn.f32", k_ffma, 1},
                    {"fma.rn.f32x2 (packed)", k_ffma2, 2}, {"tanh.approx.f32", k_tanh, 1},
                    {"tanh.approx.f16x2", k_tanh_h2, 2}, {"ex2.approx.ftz.f32", k_ex2, 1},
                    {"rcp.approx.ftz.f32 (+1)", k_rcp, 1},
                    {"cvt f64->f32->f64 (pairs)", k_cvt, 2}};
  printf("SMs %d, maximum SM clock %.0f MHz\n", sms, khz / 1e3);
  for (const Op &op : ops) {
    for (int r = 0; r < 3; r++) op.k<<<grid, block>>>(out, 1e-3);
    cudaEventRecord(e0);
    for (int r = 0; r < 10; r++) op.k<<<grid, block>>>(out, 1e-3);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double elems = 10.0 * grid * block * (double)ITERS * CHAINS * op.per_instr;
    const double rate = elems / (ms * 1e-3);
    printf("%-24s %9.3f ms  %.3e elements/s  %6.1f elements/clk/SM\n", op.name, ms, rate,
           rate / sms / (khz * 1e3));
  }
  cudaError_t err = cudaDeviceSynchronize();
  printf("status: %s\n", cudaGetErrorString(err));
  cudaFree(out);
  return err == cudaSuccess ? 0 : 1;
}
