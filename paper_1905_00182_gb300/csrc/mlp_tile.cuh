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

// Two activations with the hardware tanh approximation (one MUFU operation each, ~2^-11
// relative error, below the bfloat16 rounding that follows), the rest on packed FP32x2
// arithmetic: u = z (K + (K C z) z) with the inner sum as one fused multiply-add, then
// z + z tanh(u) = 2 gelu(z), packed to bf16x2 as the next layer's operand.  The factor 2 is
// taken back exactly by the halved weights of the next layer in the inference image
// (stage_inference_image): a power of two commutes with every rounding on the way.  Used for
// inference inside the stencil kernels.
__device__ __forceinline__ uint32_t gelu2_fast(float z0, float z1) {
  const float2 z = make_float2(z0, z1);
  const float2 a = __fmul2_rn(make_float2(GELU_K * GELU_C, GELU_K * GELU_C), z);
  const float2 u = __fmul2_rn(z, __ffma2_rn(a, z, make_float2(GELU_K, GELU_K)));
  float t0, t1;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t0) : "f"(u.x));
  asm("tanh.approx.f32 %0, %1;" : "=f"(t1) : "f"(u.y));
  const float2 g = __ffma2_rn(z, make_float2(t0, t1), z);
  return pack2(g.x, g.y);
}

// Copy of the packed parameter image into shared memory for inference, with the weights of
// layers 2, 3 and 4 halved (bfloat16 times 0.5 is exact above 2^-126), to take the activations
// of gelu2_fast (twice gelu) back to gelu.  Called by all threads of the block.
__device__ __forceinline__ void stage_inference_image(uint4 *dst, const uint4 *src, int tid,
                                                      int nthreads) {
  for (int i = tid; i < PACKED_BYTES / 16; i += nthreads) {
    uint4 v = src[i];
    if (i >= OFF_W2 / 16 && i < OFF_W2T / 16) {
      uint32_t *w = reinterpret_cast<uint32_t *>(&v);
      const __nv_bfloat162 h = __floats2bfloat162_rn(0.5f, 0.5f);
#pragma unroll
      for (int k = 0; k < 4; k++) {
        __nv_bfloat162 x = *reinterpret_cast<__nv_bfloat162 *>(&w[k]);
        x = __hmul2(x, h);
        w[k] = *reinterpret_cast<uint32_t *>(&x);
      }
    }
    dst[i] = v;
  }
}

// D = A B + C with the accumulator input in separate registers (the bias, without copies)
__device__ __forceinline__ void mma16816_c(float d[4], const uint32_t a[4], uint32_t b0,
                                           uint32_t b1, float c0, float c1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%10,%11,%10,%11};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c0), "f"(c1));
}

// One hidden layer (32 units, gelu) for the warp's two 16-row tiles at once: each weight
// fragment is read from shared memory once and used by both tiles' products, and each n-tile of
// 8 units is activated and packed into the next layer's operand as soon as it is accumulated
// (n-tile j fills k-step j/2, fragment registers 2 (j mod 2) and 2 (j mod 2) + 1).
template <int KSTEPS>
__device__ __forceinline__ void hidden2(const unsigned char *img, int offW, int ldW, int offB,
                                        const uint32_t (&Ain)[2][KSTEPS][4],
                                        uint32_t (&Aout)[2][2][4], int g, int t) {
#pragma unroll
  for (int j = 0; j < 4; j++) {
    const float b0 = ldb(img, offB, 8 * j + 2 * t), b1 = ldb(img, offB, 8 * j + 2 * t + 1);
    float acc[2][4];
#pragma unroll
    for (int s = 0; s < KSTEPS; s++) {
      const uint32_t w0 = ldw(img, offW, ldW, 8 * j + g, 16 * s + 2 * t);
      const uint32_t w1 = ldw(img, offW, ldW, 8 * j + g, 16 * s + 2 * t + 8);
#pragma unroll
      for (int T = 0; T < 2; T++) {
        if (s == 0) mma16816_c(acc[T], Ain[T][0], w0, w1, b0, b1);
        else mma16816(acc[T], Ain[T][s], w0, w1);
      }
    }
#pragma unroll
    for (int T = 0; T < 2; T++) {
      Aout[T][j >> 1][2 * (j & 1)] = gelu2_fast(acc[T][0], acc[T][1]);
      Aout[T][j >> 1][2 * (j & 1) + 1] = gelu2_fast(acc[T][2], acc[T][3]);
    }
  }
}

// The network's three weights for one stencil per lane, the whole warp evaluating its two
// 16-row tiles together on the tensor cores (lane 16 T + r is row r of tile T).  x: this lane's
// normalised stencil.  Must be called by all 32 lanes; every lane gets the weights of its own
// stencil (the caller keeps them where it wants the network).
__device__ __forceinline__ void warp_weights2(const unsigned char *img, const float x[5],
                                              float w[3]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // layer 1's operand: row g (+8) of tile T takes the bf16 pair k = 2t, 2t+1 of its stencil,
  // (x0 x1), (x2 x3), (x4 0) for t = 0, 1, 2 and zeros for t = 3 and k >= 8
  const uint32_t p0 = pack2(x[0], x[1]), p1 = pack2(x[2], x[3]), p2 = pack2(x[4], 0.f);
  uint32_t A0[2][1][4];
#pragma unroll
  for (int T = 0; T < 2; T++) {
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int src = 16 * T + g + 8 * h;
      const uint32_t q0 = __shfl_sync(0xffffffffu, p0, src);
      const uint32_t q1 = __shfl_sync(0xffffffffu, p1, src);
      const uint32_t q2 = __shfl_sync(0xffffffffu, p2, src);
      A0[T][0][h] = t == 0 ? q0 : (t == 1 ? q1 : (t == 2 ? q2 : 0u));
    }
    A0[T][0][2] = 0u;
    A0[T][0][3] = 0u;
  }
  uint32_t Ab[2][2][4], Ac[2][2][4];
  hidden2<1>(img, OFF_W1, 16, OFF_B1, A0, Ab, g, t);
  hidden2<2>(img, OFF_W2, 32, OFF_B2, Ab, Ac, g, t);
  hidden2<2>(img, OFF_W3, 32, OFF_B3, Ac, Ab, g, t);
  // logits (n-tile 0: logits 0..7, 0..2 used): rows g / g+8 in c0, c1 / c2, c3 of lane 4g
  // (logits 0, 1) and lane 4g + 1 (logit 2)
  float z4[2][4];
  {
    const float b0 = ldb(img, OFF_B4, 2 * t), b1 = ldb(img, OFF_B4, 2 * t + 1);
#pragma unroll
    for (int s = 0; s < 2; s++) {
      const uint32_t w0 = ldw(img, OFF_W4, 32, g, 16 * s + 2 * t);
      const uint32_t w1 = ldw(img, OFF_W4, 32, g, 16 * s + 2 * t + 8);
#pragma unroll
      for (int T = 0; T < 2; T++) {
        if (s == 0) mma16816_c(z4[T], Ab[T][0], w0, w1, b0, b1);
        else mma16816(z4[T], Ab[T][1], w0, w1);
      }
    }
  }
  // each lane gathers the three logits of its own stencil and takes their softmax
  const int T = lane >> 4, r = lane & 15, s0 = 4 * (r & 7), hi = r >> 3;
  float l[2][2][3];  // [tile][row half][logit]
#pragma unroll
  for (int u = 0; u < 2; u++) {
#pragma unroll
    for (int h = 0; h < 2; h++) {
      l[u][h][0] = __shfl_sync(0xffffffffu, z4[u][2 * h], s0);
      l[u][h][1] = __shfl_sync(0xffffffffu, z4[u][2 * h + 1], s0);
      l[u][h][2] = __shfl_sync(0xffffffffu, z4[u][2 * h], s0 + 1);
    }
  }
  float v[3];
#pragma unroll
  for (int k = 0; k < 3; k++)
    v[k] = T ? (hi ? l[1][1][k] : l[1][0][k]) : (hi ? l[0][1][k] : l[0][0][k]);
  const float m = fmaxf(v[0], fmaxf(v[1], v[2]));
  const float e0 = __expf(v[0] - m), e1 = __expf(v[1] - m), e2 = __expf(v[2] - m);
  const float inv = __fdividef(1.f, e0 + e1 + e2);  // the sum lies in [1, 3]
  w[0] = e0 * inv;
  w[1] = e1 * inv;
  w[2] = e2 * inv;
}

}  // namespace mlp
}  // namespace ibfsa
