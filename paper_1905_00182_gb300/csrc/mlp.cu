// mlp.cu -- training and stand-alone inference of the learned reconstruction weights on the
// tensor cores (BF16 operands, FP32 accumulation), and Adam on FP32 master parameters.
//
// Loss of a batch of n stencils: mean_b (sum_k omega_k qhat_k - that_b)^2, with x, qhat and the
// target that in the normalised units of each stencil (x = (v - v_2)/amp).  The backward pass
// propagates through softmax, the four dense layers and gelu; weight gradients
// dW_l = dZ_l^T H_{l-1} are tensor-core products over the 16 samples of a tile, accumulated per
// warp, reduced per block and added to the global FP32 gradient with one atomic per parameter
// and block.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include "ibfsa_internal.h"
#include "mlp_tile.cuh"

namespace ibfsa {
namespace mlp {

// training state (device): floats [master | m | v | grad] (NPAD each), loss, then the packed image
constexpr int NPAD = 2432;
constexpr size_t OFF_MASTER = 0, OFF_M = NPAD, OFF_V = 2 * NPAD, OFF_GRAD = 3 * NPAD,
                 OFF_LOSS = 4 * NPAD;
constexpr size_t STATE_FLOATS = 4 * NPAD + 64;
constexpr size_t OFF_IMAGE_BYTES = STATE_FLOATS * sizeof(float);
constexpr size_t STATE_BYTES = OFF_IMAGE_BYTES + PACKED_BYTES;

constexpr int TRAIN_WARPS = 4;

__device__ __forceinline__ float bf16r(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

// packed image from the FP32 master parameters (all parameters rounded to bf16)
__global__ void k_pack(const float *__restrict__ th, unsigned char *__restrict__ img) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  __nv_bfloat16 *W1 = (__nv_bfloat16 *)(img + OFF_W1), *W2 = (__nv_bfloat16 *)(img + OFF_W2);
  __nv_bfloat16 *W3 = (__nv_bfloat16 *)(img + OFF_W3), *W4 = (__nv_bfloat16 *)(img + OFF_W4);
  __nv_bfloat16 *W2T = (__nv_bfloat16 *)(img + OFF_W2T), *W3T = (__nv_bfloat16 *)(img + OFF_W3T);
  __nv_bfloat16 *W4T = (__nv_bfloat16 *)(img + OFF_W4T);
  float *B1 = (float *)(img + OFF_B1), *B2 = (float *)(img + OFF_B2);
  float *B3 = (float *)(img + OFF_B3), *B4 = (float *)(img + OFF_B4);
  if (i < 32 * 16) {  // W1 [32][16]
    int r = i / 16, c = i % 16;
    W1[i] = __float2bfloat16_rn(c < 5 ? th[P_W1 + r * 5 + c] : 0.f);
  }
  if (i < 32 * 32) {
    int r = i / 32, c = i % 32;
    W2[i] = __float2bfloat16_rn(th[P_W2 + i]);
    W3[i] = __float2bfloat16_rn(th[P_W3 + i]);
    W2T[i] = __float2bfloat16_rn(th[P_W2 + c * 32 + r]);
    W3T[i] = __float2bfloat16_rn(th[P_W3 + c * 32 + r]);
  }
  if (i < 8 * 32) {  // W4 [8][32]
    int r = i / 32;
    W4[i] = __float2bfloat16_rn(r < 3 ? th[P_W4 + i] : 0.f);
  }
  if (i < 32 * 16) {  // W4T [32][16]: row = hidden unit, col = logit
    int r = i / 16, c = i % 16;
    W4T[i] = __float2bfloat16_rn(c < 3 ? th[P_W4 + c * 32 + r] : 0.f);
  }
  if (i < 32) {
    B1[i] = bf16r(th[P_B1 + i]);
    B2[i] = bf16r(th[P_B2 + i]);
    B3[i] = bf16r(th[P_B3 + i]);
  }
  if (i < 8) B4[i] = i < 3 ? bf16r(th[P_B4 + i]) : 0.f;
}

// --- per-warp helpers of the backward pass -------------------------------------------------
// store a 16x32 C-layout tile transposed into smem: dst[unit][sample], float
__device__ __forceinline__ void store_T_f32(float (*dst)[17], const float c[4][4], int g, int t) {
#pragma unroll
  for (int j = 0; j < 4; j++) {
    dst[8 * j + 2 * t][g] = c[j][0];
    dst[8 * j + 2 * t + 1][g] = c[j][1];
    dst[8 * j + 2 * t][g + 8] = c[j][2];
    dst[8 * j + 2 * t + 1][g + 8] = c[j][3];
  }
}

// store a 16x32 BF16 operand tile (two k-step A fragments) transposed: dst[unit][sample]
__device__ __forceinline__ void store_T_bf16(__nv_bfloat16 (*dst)[24], const uint32_t A[2][4],
                                             int g, int t) {
#pragma unroll
  for (int s = 0; s < 2; s++) {
#pragma unroll
    for (int r = 0; r < 4; r++) {
      __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(&A[s][r]);
      int row = (r & 1) ? g + 8 : g;
      int col = 16 * s + ((r & 2) ? 8 : 0) + 2 * t;
      dst[col][row] = v.x;
      dst[col + 1][row] = v.y;
    }
  }
}

// dW (M = 16*MT units x N = 8*NT inputs) += dZ^T (units x 16 samples) H (16 samples x inputs)
template <int MT, int NT>
__device__ __forceinline__ void accumulate_dW(float acc[MT][NT][4], float (*dzT)[17],
                                              __nv_bfloat16 (*hT)[24], int g, int t) {
#pragma unroll
  for (int mt = 0; mt < MT; mt++) {
    uint32_t a[4];
    int r0 = 16 * mt + g;
    a[0] = pack2(dzT[r0][2 * t], dzT[r0][2 * t + 1]);
    a[1] = pack2(dzT[r0 + 8][2 * t], dzT[r0 + 8][2 * t + 1]);
    a[2] = pack2(dzT[r0][2 * t + 8], dzT[r0][2 * t + 9]);
    a[3] = pack2(dzT[r0 + 8][2 * t + 8], dzT[r0 + 8][2 * t + 9]);
#pragma unroll
    for (int nt = 0; nt < NT; nt++) {
      uint32_t b0 = *reinterpret_cast<const uint32_t *>(&hT[8 * nt + g][2 * t]);
      uint32_t b1 = *reinterpret_cast<const uint32_t *>(&hT[8 * nt + g][2 * t + 8]);
      mma16816(acc[mt][nt], a, b0, b1);
    }
  }
}

// dH (16 x 32) = dZ (16 x K) W (K x 32), W given transposed ([32][ldT], row = input unit)
template <int KSTEPS>
__device__ __forceinline__ void backprop32(float dh[4][4], const uint32_t A[KSTEPS][4],
                                           const unsigned char *img, int offWT, int ldT, int g,
                                           int t) {
#pragma unroll
  for (int j = 0; j < 4; j++) {
    dh[j][0] = dh[j][1] = dh[j][2] = dh[j][3] = 0.f;
#pragma unroll
    for (int s = 0; s < KSTEPS; s++) {
      uint32_t w0 = ldw(img, offWT, ldT, 8 * j + g, 16 * s + 2 * t);
      uint32_t w1 = ldw(img, offWT, ldT, 8 * j + g, 16 * s + 2 * t + 8);
      mma16816(dh[j], A[s], w0, w1);
    }
  }
}

__device__ __forceinline__ void pack_C_as_A(const float c[4][4], uint32_t A[2][4]) {
#pragma unroll
  for (int s = 0; s < 2; s++) {
    A[s][0] = pack2(c[2 * s][0], c[2 * s][1]);
    A[s][1] = pack2(c[2 * s][2], c[2 * s][3]);
    A[s][2] = pack2(c[2 * s + 1][0], c[2 * s + 1][1]);
    A[s][3] = pack2(c[2 * s + 1][2], c[2 * s + 1][3]);
  }
}

// loads one stencil row (raw values), its normalised form, candidates and normalised target
__device__ __forceinline__ bool load_row(const float *S, const float *T, int n, int m, float x[5],
                                         float q[3], float &tn) {
  float v[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  bool ok = m < n;
  if (ok)
#pragma unroll
    for (int j = 0; j < 5; j++) v[j] = S[(size_t)m * 5 + j];
  float amp = normalise(v, x);
  candidates(x, q);
  tn = 0.f;
  bool live = amp > 1e-30f;  // the same cut as normalise: no overflow from denormal amplitudes
  if (ok && T && live) tn = (T[m] - v[2]) / amp;
  return ok && live;
}

__global__ void __launch_bounds__(32 * TRAIN_WARPS, 1)
    k_train(const unsigned char *__restrict__ gimg, int n, const float *__restrict__ S,
            const float *__restrict__ T, float inv_n, float *__restrict__ grad,
            float *__restrict__ loss) {
  __shared__ __align__(16) unsigned char img[PACKED_BYTES];
  __shared__ float dzT[TRAIN_WARPS][32][17];
  __shared__ __align__(16) __nv_bfloat16 hT[TRAIN_WARPS][32][24];
  for (int i = threadIdx.x; i < PACKED_BYTES / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(img)[i] = reinterpret_cast<const uint4 *>(gimg)[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  float aW1[2][2][4] = {}, aW2[2][4][4] = {}, aW3[2][4][4] = {}, aW4[1][4][4] = {};
  float db1 = 0.f, db2 = 0.f, db3 = 0.f, db4 = 0.f, lsum = 0.f;
  const int tiles = (n + 15) / 16;
  for (int tile = blockIdx.x * TRAIN_WARPS + w; tile < tiles; tile += gridDim.x * TRAIN_WARPS) {
    int ma = tile * 16 + g, mb = ma + 8;
    float xa[5], xb[5], qa[3], qb[3], ta, tb;
    bool va = load_row(S, T, n, ma, xa, qa, ta), vb = load_row(S, T, n, mb, xb, qb, tb);
    float z1[4][4], z2[4][4], z3[4][4], z4[4], wa[3], wb[3];
    uint32_t A1[2][4], A2[2][4], A3[2][4];
    forward_tile(img, xa, xb, g, t, z1, z2, z3, A1, A2, A3, wa, wb, z4);
    // loss and d(logits) for rows g and g+8 (lane t == 0 holds the weights)
    float d4a[3] = {0.f, 0.f, 0.f}, d4b[3] = {0.f, 0.f, 0.f};
    if (t == 0) {
      float fa = wa[0] * qa[0] + wa[1] * qa[1] + wa[2] * qa[2];
      float fb = wb[0] * qb[0] + wb[1] * qb[1] + wb[2] * qb[2];
      float ra = va ? fa - ta : 0.f, rb = vb ? fb - tb : 0.f;
      lsum += ra * ra + rb * rb;
      float dfa = 2.f * ra * inv_n, dfb = 2.f * rb * inv_n;
      float sa = 0.f, sb = 0.f;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        sa += wa[k] * dfa * qa[k];
        sb += wb[k] * dfb * qb[k];
      }
#pragma unroll
      for (int k = 0; k < 3; k++) {
        d4a[k] = wa[k] * (dfa * qa[k] - sa);
        d4b[k] = wb[k] * (dfb * qb[k] - sb);
      }
    }
    // dz4 in C layout of the 16x8 logit tile: lane t holds logits 2t, 2t+1
    float c4[4];
    {
      float x0 = __shfl_sync(0xffffffffu, d4a[0], lane & ~3), x1 = __shfl_sync(0xffffffffu, d4a[1], lane & ~3);
      float x2 = __shfl_sync(0xffffffffu, d4a[2], lane & ~3);
      float y0 = __shfl_sync(0xffffffffu, d4b[0], lane & ~3), y1 = __shfl_sync(0xffffffffu, d4b[1], lane & ~3);
      float y2 = __shfl_sync(0xffffffffu, d4b[2], lane & ~3);
      c4[0] = t == 0 ? x0 : (t == 1 ? x2 : 0.f);
      c4[1] = t == 0 ? x1 : 0.f;
      c4[2] = t == 0 ? y0 : (t == 1 ? y2 : 0.f);
      c4[3] = t == 0 ? y1 : 0.f;
    }
    // ---- layer 4: dW4 = dz4^T h3, db4, dh3 = dz4 W4
    {
      float (*dT)[17] = dzT[w];
      __syncwarp();
      for (int i = lane; i < 32 * 17; i += 32) (&dT[0][0])[i] = 0.f;
      __syncwarp();
      dT[2 * t][g] = c4[0];
      dT[2 * t + 1][g] = c4[1];
      dT[2 * t][g + 8] = c4[2];
      dT[2 * t + 1][g + 8] = c4[3];
      store_T_bf16(hT[w], A3, g, t);
      __syncwarp();
      accumulate_dW<1, 4>(aW4, dT, hT[w], g, t);
      if (lane < 3) {
        float s = 0.f;
        for (int m = 0; m < 16; m++) s += dT[lane][m];
        db4 += s;
      }
      __syncwarp();
    }
    uint32_t Ad4[1][4];
    Ad4[0][0] = pack2(c4[0], c4[1]);
    Ad4[0][1] = pack2(c4[2], c4[3]);
    Ad4[0][2] = 0u;
    Ad4[0][3] = 0u;
    float dz[4][4];
    backprop32<1>(dz, Ad4, img, OFF_W4T, 16, g, t);
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int r = 0; r < 4; r++) dz[j][r] *= gelu_grad(z3[j][r]);
    // ---- layer 3: dW3 = dz3^T h2, db3, dh2 = dz3 W3
    store_T_f32(dzT[w], dz, g, t);
    store_T_bf16(hT[w], A2, g, t);
    __syncwarp();
    accumulate_dW<2, 4>(aW3, dzT[w], hT[w], g, t);
    {
      float s = 0.f;
      for (int m = 0; m < 16; m++) s += dzT[w][lane][m];
      db3 += s;
    }
    __syncwarp();
    uint32_t Ad[2][4];
    pack_C_as_A(dz, Ad);
    backprop32<2>(dz, Ad, img, OFF_W3T, 32, g, t);
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int r = 0; r < 4; r++) dz[j][r] *= gelu_grad(z2[j][r]);
    // ---- layer 2
    store_T_f32(dzT[w], dz, g, t);
    store_T_bf16(hT[w], A1, g, t);
    __syncwarp();
    accumulate_dW<2, 4>(aW2, dzT[w], hT[w], g, t);
    {
      float s = 0.f;
      for (int m = 0; m < 16; m++) s += dzT[w][lane][m];
      db2 += s;
    }
    __syncwarp();
    pack_C_as_A(dz, Ad);
    backprop32<2>(dz, Ad, img, OFF_W2T, 32, g, t);
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int r = 0; r < 4; r++) dz[j][r] *= gelu_grad(z1[j][r]);
    // ---- layer 1: dW1 = dz1^T x (inputs padded to 16)
    store_T_f32(dzT[w], dz, g, t);
    {
      __nv_bfloat16 (*xT)[24] = hT[w];
      __syncwarp();
      for (int i = lane; i < 32 * 24; i += 32) (&xT[0][0])[i] = __float2bfloat16_rn(0.f);
      __syncwarp();
      if (t == 0)
#pragma unroll
        for (int j = 0; j < 5; j++) {
          xT[j][g] = __float2bfloat16_rn(xa[j]);
          xT[j][g + 8] = __float2bfloat16_rn(xb[j]);
        }
    }
    __syncwarp();
    accumulate_dW<2, 2>(aW1, dzT[w], hT[w], g, t);
    {
      float s = 0.f;
      for (int m = 0; m < 16; m++) s += dzT[w][lane][m];
      db1 += s;
    }
    __syncwarp();
  }
  // ---- per-block reduction into the global gradient (one atomic per parameter and block)
  __shared__ float acc[NPAD];
  for (int i = threadIdx.x; i < NPAD; i += blockDim.x) acc[i] = 0.f;
  __syncthreads();
  // weight fragments: C element (mt, nt, r) -> unit 16 mt + g (+8), input 8 nt + 2t (+1)
#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
      for (int r = 0; r < 4; r++) {
        int u = 16 * mt + g + ((r & 2) ? 8 : 0), in = 8 * nt + 2 * t + (r & 1);
        atomicAdd(&acc[P_W2 + u * 32 + in], aW2[mt][nt][r]);
        atomicAdd(&acc[P_W3 + u * 32 + in], aW3[mt][nt][r]);
        if (nt < 2 && in < 5) atomicAdd(&acc[P_W1 + u * 5 + in], aW1[mt][nt][r]);
        if (mt == 0 && u < 3) atomicAdd(&acc[P_W4 + u * 32 + in], aW4[0][nt][r]);
      }
  atomicAdd(&acc[P_B1 + lane], db1);
  atomicAdd(&acc[P_B2 + lane], db2);
  atomicAdd(&acc[P_B3 + lane], db3);
  if (lane < 3) atomicAdd(&acc[P_B4 + lane], db4);
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) atomicAdd(&acc[NPAD - 1], lsum);
  __syncthreads();
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) atomicAdd(&grad[i], acc[i]);
  if (threadIdx.x == 0) atomicAdd(loss, acc[NPAD - 1] * inv_n);
}

__global__ void k_adam(float *__restrict__ th, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ grad, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  float gi = grad[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// stand-alone inference: face values, weights and (with targets) the mean squared loss
__global__ void __launch_bounds__(256) k_eval(const unsigned char *__restrict__ gimg, int n,
                                              const float *__restrict__ S,
                                              const float *__restrict__ T, float *__restrict__ face,
                                              float *__restrict__ omega, float inv_n,
                                              float *__restrict__ loss) {
  __shared__ __align__(16) unsigned char img[PACKED_BYTES];
  for (int i = threadIdx.x; i < PACKED_BYTES / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(img)[i] = reinterpret_cast<const uint4 *>(gimg)[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
  const int warps = blockDim.x >> 5;
  float lsum = 0.f;
  for (int tile = blockIdx.x * warps + w; tile < (n + 15) / 16; tile += gridDim.x * warps) {
    int ma = tile * 16 + g, mb = ma + 8;
    float xa[5], xb[5], qa[3], qb[3], ta, tb;
    bool va = load_row(S, T, n, ma, xa, qa, ta), vb = load_row(S, T, n, mb, xb, qb, tb);
    float z1[4][4], z2[4][4], z3[4][4], z4[4], wa[3], wb[3];
    uint32_t A1[2][4], A2[2][4], A3[2][4];
    forward_tile(img, xa, xb, g, t, z1, z2, z3, A1, A2, A3, wa, wb, z4);
    if (t == 0) {
      float fa = wa[0] * qa[0] + wa[1] * qa[1] + wa[2] * qa[2];
      float fb = wb[0] * qb[0] + wb[1] * qb[1] + wb[2] * qb[2];
      if (ma < n) {
        float v2 = S[(size_t)ma * 5 + 2], amp = 0.f;
        for (int j = 0; j < 5; j++) amp = fmaxf(amp, fabsf(S[(size_t)ma * 5 + j] - v2));
        if (face) face[ma] = v2 + amp * fa;
        if (omega)
          for (int k = 0; k < 3; k++) omega[(size_t)ma * 3 + k] = wa[k];
        if (va && T) lsum += (fa - ta) * (fa - ta);
      }
      if (mb < n) {
        float v2 = S[(size_t)mb * 5 + 2], amp = 0.f;
        for (int j = 0; j < 5; j++) amp = fmaxf(amp, fabsf(S[(size_t)mb * 5 + j] - v2));
        if (face) face[mb] = v2 + amp * fb;
        if (omega)
          for (int k = 0; k < 3; k++) omega[(size_t)mb * 3 + k] = wb[k];
        if (vb && T) lsum += (fb - tb) * (fb - tb);
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (loss && lane == 0) atomicAdd(loss, lsum * inv_n);
}

}  // namespace mlp

size_t mlp_image_offset() { return mlp::OFF_IMAGE_BYTES; }
size_t mlp_image_bytes() { return mlp::PACKED_BYTES; }

}  // namespace ibfsa

using namespace ibfsa;
using namespace ibfsa::mlp;

extern "C" {

size_t ibfsa_mlp_state_bytes(void) { return STATE_BYTES; }

static int cerr(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return IBFSA_OK;
  char msg[256];
  snprintf(msg, sizeof(msg), "%s: %s", what, cudaGetErrorString(e));
  record_error(msg);
  return IBFSA_ERR_CUDA;
}

int ibfsa_mlp_init(void *d_state, const float *params, void *stream) {
  if (!d_state || !params) {
    record_error("ibfsa_mlp_init: NULL argument");
    return IBFSA_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  float *s = (float *)d_state;
  cudaError_t e = cudaMemsetAsync(s, 0, STATE_FLOATS * sizeof(float), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s + OFF_MASTER, params, NPARAM * sizeof(float), cudaMemcpyDefault, st);
  if (e == cudaSuccess) {
    k_pack<<<4, 256, 0, st>>>(s + OFF_MASTER, (unsigned char *)d_state + OFF_IMAGE_BYTES);
    e = cudaGetLastError();
  }
  return cerr(e, "ibfsa_mlp_init");
}

int ibfsa_mlp_train_step(void *d_state, int n, const float *stencils, const float *targets,
                         float lr, int step, void *stream) {
  if (!d_state || n <= 0 || !stencils || !targets || step < 1) {
    record_error("ibfsa_mlp_train_step: bad argument");
    return IBFSA_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  float *s = (float *)d_state;
  unsigned char *img = (unsigned char *)d_state + OFF_IMAGE_BYTES;
  cudaError_t e = cudaMemsetAsync(s + OFF_GRAD, 0, (NPAD + 64) * sizeof(float), st);
  if (e != cudaSuccess) return cerr(e, "ibfsa_mlp_train_step");
  int tiles = (n + 15) / 16;
  int blocks = (tiles + TRAIN_WARPS - 1) / TRAIN_WARPS;
  if (blocks > 152 * 4) blocks = 152 * 4;
  k_train<<<blocks, 32 * TRAIN_WARPS, 0, st>>>(img, n, stencils, targets, 1.f / (float)n,
                                                s + OFF_GRAD, s + OFF_LOSS);
  if ((e = cudaGetLastError()) != cudaSuccess) return cerr(e, "ibfsa_mlp_train_step");
  if (lr > 0.f) {
    const float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f / (1.f - powf(b1, (float)step)), c2 = 1.f / (1.f - powf(b2, (float)step));
    k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(s + OFF_MASTER, s + OFF_M, s + OFF_V,
                                                 s + OFF_GRAD, lr, b1, b2, 1e-8f, c1, c2);
    if ((e = cudaGetLastError()) != cudaSuccess) return cerr(e, "ibfsa_mlp_train_step");
    k_pack<<<4, 256, 0, st>>>(s + OFF_MASTER, img);
    e = cudaGetLastError();
  }
  return cerr(e, "ibfsa_mlp_train_step");
}

int ibfsa_mlp_read(const void *d_state, float *params, float *grad, float *loss, void *stream) {
  if (!d_state) {
    record_error("ibfsa_mlp_read: NULL state");
    return IBFSA_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const float *s = (const float *)d_state;
  cudaError_t e = cudaSuccess;
  if (params) e = cudaMemcpyAsync(params, s + OFF_MASTER, NPARAM * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, s + OFF_GRAD, NPARAM * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, s + OFF_LOSS, 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cerr(e, "ibfsa_mlp_read");
}

int ibfsa_mlp_eval(const void *d_state, int n, const float *stencils, const float *targets,
                   float *face, float *omega, float *loss, void *stream) {
  if (!d_state || n < 0 || (n > 0 && !stencils)) {
    record_error("ibfsa_mlp_eval: bad argument");
    return IBFSA_ERR_ARG;
  }
  if (n == 0) return IBFSA_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (loss) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (e != cudaSuccess) return cerr(e, "ibfsa_mlp_eval");
  int tiles = (n + 15) / 16;
  int blocks = (tiles + 7) / 8;
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_eval<<<blocks, 256, 0, st>>>((const unsigned char *)d_state + OFF_IMAGE_BYTES, n, stencils,
                                 targets, face, omega, 1.f / (float)n, loss);
  return cerr(cudaGetLastError(), "ibfsa_mlp_eval");
}

}  // extern "C"
