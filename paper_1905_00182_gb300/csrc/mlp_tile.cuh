// mlp_tile.cuh -- warp-level BF16 tensor-core evaluation of the learned reconstruction weights
// (the learned-weight variant of the fifth-order reconstruction, arXiv:1905.00182 Sec. 2):
//   x = (v - v_2)/amp (5 inputs) -> 32 -> 32 -> 32 (gelu, tanh form) -> 3 logits -> softmax.
// One warp evaluates a tile of 16 stencils with mma.sync m16n8k16 (BF16 operands, FP32
// accumulation); each layer's FP32 accumulator fragment is re-packed in registers as the next
// layer's BF16 operand fragment, so activations never leave the registers.
//
// Fragment layout of m16n8k16 (g = lane/4, t = lane%4):
//   A (16x16, row-major): a0 = (g, 2t..2t+1), a1 = (g+8, 2t..), a2 = (g, 2t+8..), a3 = (g+8, 2t+8..)
//   B (16x8,  k x n):     b0 = (k = 2t..2t+1, n = g), b1 = (k = 2t+8.., n = g)
//   C (16x8, f32):        c0 = (g, 2t), c1 = (g, 2t+1), c2 = (g+8, 2t), c3 = (g+8, 2t+1)
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace ibfsa {
namespace mlp {

constexpr int NPARAM = 2403;
// packed device image (bytes): forward weights, transposed copies for the backward pass, biases
constexpr int OFF_W1 = 0;        // [32][16] bf16 (inputs 5..15 zero)
constexpr int OFF_W2 = 1024;     // [32][32] bf16
constexpr int OFF_W3 = 3072;     // [32][32] bf16
constexpr int OFF_W4 = 5120;     // [8][32]  bf16 (rows 3..7 zero)
constexpr int OFF_W2T = 5632;    // [32][32] bf16, W2 transposed
constexpr int OFF_W3T = 7680;    // [32][32] bf16
constexpr int OFF_W4T = 9728;    // [32][16] bf16, W4 transposed (logits 3..15 zero)
constexpr int OFF_B1 = 10752;    // [32] f32 (bf16-rounded values)
constexpr int OFF_B2 = 10880;
constexpr int OFF_B3 = 11008;
constexpr int OFF_B4 = 11136;    // [8] f32
constexpr int PACKED_BYTES = 11264;
// offsets of the flat parameter vector [W1 (32x5), b1, W2, b2, W3, b3, W4 (3x32), b4]
constexpr int P_W1 = 0, P_B1 = 160, P_W2 = 192, P_B2 = 1216, P_W3 = 1248, P_B3 = 2272,
              P_W4 = 2304, P_B4 = 2400;

constexpr float GELU_K = 0.7978845608028654f;  // sqrt(2/pi)
constexpr float GELU_C = 0.044715f;

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
  return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma16816(float d[4], const uint32_t a[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float gelu(float z) {
  return 0.5f * z * (1.f + tanhf(GELU_K * (z + GELU_C * z * z * z)));
}

__device__ __forceinline__ float gelu_grad(float z) {
  float t = tanhf(GELU_K * (z + GELU_C * z * z * z));
  return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * GELU_K * (1.f + 3.f * GELU_C * z * z);
}

// 32-bit load of two consecutive bf16 of a packed matrix with `ld` columns
__device__ __forceinline__ uint32_t ldw(const unsigned char *img, int off, int ld, int row,
                                        int col) {
  return *reinterpret_cast<const uint32_t *>(img + off + 2 * (row * ld + col));
}

__device__ __forceinline__ float ldb(const unsigned char *img, int off, int i) {
  return reinterpret_cast<const float *>(img + off)[i];
}

// 16x32 hidden layer: acc[j][.] (n-tile j = units 8j..8j+7) = bias + A(16 x K) W^T
template <int KSTEPS>
__device__ __forceinline__ void dense32(float acc[4][4], const uint32_t A[KSTEPS][4],
                                        const unsigned char *img, int offW, int ldW, int offB,
                                        int g, int t) {
#pragma unroll
  for (int j = 0; j < 4; j++) {
    float b0 = ldb(img, offB, 8 * j + 2 * t), b1 = ldb(img, offB, 8 * j + 2 * t + 1);
    acc[j][0] = b0; acc[j][1] = b1; acc[j][2] = b0; acc[j][3] = b1;
#pragma unroll
    for (int s = 0; s < KSTEPS; s++) {
      uint32_t w0 = ldw(img, offW, ldW, 8 * j + g, 16 * s + 2 * t);
      uint32_t w1 = ldw(img, offW, ldW, 8 * j + g, 16 * s + 2 * t + 8);
      mma16816(acc[j], A[s], w0, w1);
    }
  }
}

// gelu of a 16x32 accumulator, packed as the next layer's two BF16 k-step fragments
__device__ __forceinline__ void gelu_pack(const float z[4][4], uint32_t A[2][4]) {
#pragma unroll
  for (int s = 0; s < 2; s++) {
    A[s][0] = pack2(gelu(z[2 * s][0]), gelu(z[2 * s][1]));
    A[s][1] = pack2(gelu(z[2 * s][2]), gelu(z[2 * s][3]));
    A[s][2] = pack2(gelu(z[2 * s + 1][0]), gelu(z[2 * s + 1][1]));
    A[s][3] = pack2(gelu(z[2 * s + 1][2]), gelu(z[2 * s + 1][3]));
  }
}

// input fragment of layer 1 from the normalised stencils of rows g (xa) and g+8 (xb)
__device__ __forceinline__ void input_fragment(const float xa[5], const float xb[5], int t,
                                               uint32_t A[1][4]) {
  float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
  if (t == 0) { a0 = xa[0]; a1 = xa[1]; b0 = xb[0]; b1 = xb[1]; }
  if (t == 1) { a0 = xa[2]; a1 = xa[3]; b0 = xb[2]; b1 = xb[3]; }
  if (t == 2) { a0 = xa[4]; b0 = xb[4]; }
  A[0][0] = pack2(a0, a1);
  A[0][1] = pack2(b0, b1);
  A[0][2] = 0u;
  A[0][3] = 0u;
}

// logits of layer 4 (16 x 8 accumulator, logits 0..2 used)
__device__ __forceinline__ void logits(float z4[4], const uint32_t A3[2][4],
                                       const unsigned char *img, int g, int t) {
  z4[0] = ldb(img, OFF_B4, 2 * t);
  z4[1] = ldb(img, OFF_B4, 2 * t + 1);
  z4[2] = z4[0];
  z4[3] = z4[1];
#pragma unroll
  for (int s = 0; s < 2; s++) {
    uint32_t w0 = ldw(img, OFF_W4, 32, g, 16 * s + 2 * t);
    uint32_t w1 = ldw(img, OFF_W4, 32, g, 16 * s + 2 * t + 8);
    mma16816(z4, A3[s], w0, w1);
  }
}

// Full forward of one 16-row tile.  On return, lanes with t == 0 hold the three softmax
// weights of rows g (wa) and g+8 (wb).  z1..z3 keep the pre-activations for a backward pass.
__device__ __forceinline__ void forward_tile(const unsigned char *img, const float xa[5],
                                             const float xb[5], int g, int t, float z1[4][4],
                                             float z2[4][4], float z3[4][4], uint32_t A1[2][4],
                                             uint32_t A2[2][4], uint32_t A3[2][4], float wa[3],
                                             float wb[3], float z4[4]) {
  uint32_t A0[1][4];
  input_fragment(xa, xb, t, A0);
  dense32<1>(z1, A0, img, OFF_W1, 16, OFF_B1, g, t);
  gelu_pack(z1, A1);
  dense32<2>(z2, A1, img, OFF_W2, 32, OFF_B2, g, t);
  gelu_pack(z2, A2);
  dense32<2>(z3, A2, img, OFF_W3, 32, OFF_B3, g, t);
  gelu_pack(z3, A3);
  logits(z4, A3, img, g, t);
  // logits 0,1 live in lane t = 0, logit 2 in lane t = 1 (c0 / c2 for rows g / g+8)
  float l2a = __shfl_down_sync(0xffffffffu, z4[0], 1);
  float l2b = __shfl_down_sync(0xffffffffu, z4[2], 1);
  float ma = fmaxf(z4[0], fmaxf(z4[1], l2a)), mb = fmaxf(z4[2], fmaxf(z4[3], l2b));
  float ea0 = __expf(z4[0] - ma), ea1 = __expf(z4[1] - ma), ea2 = __expf(l2a - ma);
  float eb0 = __expf(z4[2] - mb), eb1 = __expf(z4[3] - mb), eb2 = __expf(l2b - mb);
  float ia = 1.f / (ea0 + ea1 + ea2), ib = 1.f / (eb0 + eb1 + eb2);
  wa[0] = ea0 * ia; wa[1] = ea1 * ia; wa[2] = ea2 * ia;
  wb[0] = eb0 * ib; wb[1] = eb1 * ib; wb[2] = eb2 * ib;
}

// normalised stencil, its amplitude and the three candidates (q of the normalised data)
__device__ __forceinline__ float normalise(const float v[5], float x[5]) {
  float amp = 0.f;
#pragma unroll
  for (int j = 0; j < 5; j++) amp = fmaxf(amp, fabsf(v[j] - v[2]));
  float inv = amp > 1e-30f ? 1.f / amp : 0.f;  // no overflow from denormal amplitudes
#pragma unroll
  for (int j = 0; j < 5; j++) x[j] = (v[j] - v[2]) * inv;
  return amp;
}

__device__ __forceinline__ void candidates(const float x[5], float q[3]) {
  const float s6 = 1.f / 6.f;
  q[0] = (2.f * x[0] - 7.f * x[1] + 11.f * x[2]) * s6;
  q[1] = (-x[1] + 5.f * x[2] + 2.f * x[3]) * s6;
  q[2] = (2.f * x[2] + 5.f * x[3] - x[4]) * s6;
}

}  // namespace mlp
}  // namespace ibfsa

namespace ibfsa {
namespace mlp {

// gelu with the hardware tanh approximation (one MUFU operation, ~2^-11 relative error, below
// the bfloat16 rounding that follows): used for inference inside the stencil kernels
__device__ __forceinline__ float gelu_fast(float z) {
  float u = z * (GELU_K + GELU_K * GELU_C * z * z), th;
  asm("tanh.approx.f32 %0, %1;" : "=f"(th) : "f"(u));
  float hz = 0.5f * z;
  return fmaf(hz, th, hz);
}

__device__ __forceinline__ void gelu_pack_fast(const float z[4][4], uint32_t A[2][4]) {
#pragma unroll
  for (int s = 0; s < 2; s++) {
    A[s][0] = pack2(gelu_fast(z[2 * s][0]), gelu_fast(z[2 * s][1]));
    A[s][1] = pack2(gelu_fast(z[2 * s][2]), gelu_fast(z[2 * s][3]));
    A[s][2] = pack2(gelu_fast(z[2 * s + 1][0]), gelu_fast(z[2 * s + 1][1]));
    A[s][3] = pack2(gelu_fast(z[2 * s + 1][2]), gelu_fast(z[2 * s + 1][3]));
  }
}

// inference only: softmax weights of rows g (wa) and g+8 (wb) in lanes t == 0
__device__ __forceinline__ void infer_tile(const unsigned char *img, const float xa[5],
                                           const float xb[5], int g, int t, float wa[3],
                                           float wb[3]) {
  float z[4][4], z4[4];
  uint32_t A0[1][4], A[2][4];
  input_fragment(xa, xb, t, A0);
  dense32<1>(z, A0, img, OFF_W1, 16, OFF_B1, g, t);
  gelu_pack_fast(z, A);
  dense32<2>(z, A, img, OFF_W2, 32, OFF_B2, g, t);
  gelu_pack_fast(z, A);
  dense32<2>(z, A, img, OFF_W3, 32, OFF_B3, g, t);
  gelu_pack_fast(z, A);
  logits(z4, A, img, g, t);
  float l2a = __shfl_down_sync(0xffffffffu, z4[0], 1);
  float l2b = __shfl_down_sync(0xffffffffu, z4[2], 1);
  float ma = fmaxf(z4[0], fmaxf(z4[1], l2a)), mb = fmaxf(z4[2], fmaxf(z4[3], l2b));
  float ea0 = __expf(z4[0] - ma), ea1 = __expf(z4[1] - ma), ea2 = __expf(l2a - ma);
  float eb0 = __expf(z4[2] - mb), eb1 = __expf(z4[3] - mb), eb2 = __expf(l2b - mb);
  float ia = 1.f / (ea0 + ea1 + ea2), ib = 1.f / (eb0 + eb1 + eb2);
  wa[0] = ea0 * ia; wa[1] = ea1 * ia; wa[2] = ea2 * ia;
  wb[0] = eb0 * ib; wb[1] = eb1 * ib; wb[2] = eb2 * ib;
}

// Weights for one stencil per lane, evaluated by the whole warp on the tensor cores (two
// 16-row tiles: lanes 0..15 and 16..31).  x: this lane's normalised stencil; active: whether
// this lane wants the network (tiles with no active lane are skipped).  Must be called by all
// 32 lanes.  Active lanes get the network's three weights in w; the others keep w.
__device__ __forceinline__ void warp_weights(const unsigned char *img, const float x[5],
                                             bool active, float w[3]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  unsigned any = __ballot_sync(0xffffffffu, active);
#pragma unroll
  for (int T = 0; T < 2; T++) {
    if (((any >> (16 * T)) & 0xffffu) == 0u) continue;  // warp-uniform
    float xa[5], xb[5];
#pragma unroll
    for (int j = 0; j < 5; j++) {
      xa[j] = __shfl_sync(0xffffffffu, x[j], 16 * T + g);
      xb[j] = __shfl_sync(0xffffffffu, x[j], 16 * T + g + 8);
    }
    float wa[3], wb[3];
    infer_tile(img, xa, xb, g, t, wa, wb);
    // row r of tile T belongs to lane 16 T + r; lane 4 (r mod 8) holds it (wa for r < 8)
    int r = lane - 16 * T;
    int src = 4 * (r & 7);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      float va = __shfl_sync(0xffffffffu, wa[k], src);
      float vb = __shfl_sync(0xffffffffu, wb[k], src);
      if (active && r >= 0 && r < 16) w[k] = r < 8 ? va : vb;
    }
  }
}

}  // namespace mlp
}  // namespace ibfsa
