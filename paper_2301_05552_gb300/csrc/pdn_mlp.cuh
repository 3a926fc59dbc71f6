// Warp-level building blocks of the learned surrogate of the intralaminar
// law (a multilayer perceptron 10 -> 64 -> 64 -> 64 -> 10 with ReLU): BF16
// operands on the tensor cores through mma.sync m16n8k16 with FP32
// accumulation, operands staged in shared memory and loaded with ldmatrix.
//
// Conventions.  Activations of 16 points form one row-major tile [16][width]
// in shared memory (one point per row).  A layer with weights W [out][in]
// (row-major) computes z = x W^T + b.  Row strides are padded (kS16, kS64
// elements) so that the eight 16-byte rows read by one ldmatrix phase fall in
// distinct shared-memory banks.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace pdn {
namespace mlp {

constexpr int kIn = 10, kOut = 10, kHid = 64;
constexpr int kInPad = 16, kOutPad = 16;
constexpr int kS16 = 24;  // row stride (elements) of 16-wide bf16 tiles
constexpr int kS64 = 72;  // row stride (elements) of 64-wide bf16 tiles
// parameters in the exchange order W1[64][10], b1, W2[64][64], b2, W3, b3, W4[10][64], b4
constexpr int kNumParams = kHid * kIn + kHid + 2 * (kHid * kHid + kHid) + kOut * kHid + kOut;
static_assert(kNumParams == 9674, "10-64-64-64-10 perceptron");

// The network in shared memory, in the layouts the MMA loads expect.
struct SmemNet {
  __nv_bfloat16 W1[kHid * kS16];
  __nv_bfloat16 W2[kHid * kS64];
  __nv_bfloat16 W3[kHid * kS64];
  __nv_bfloat16 W4[kOutPad * kS64];
  float b1[kHid], b2[kHid], b3[kHid], b4[kOutPad];
};

// Input / output scaling and the training box (raw units).
struct Scaling {
  float in_shift[kIn], in_mul[kIn];    // x_n = (x - in_shift) * in_mul
  float out_shift[kOut], out_mul[kOut];  // y = y_n * out_mul + out_shift
  float lo[kIn], hi[kIn];              // inputs seen in training
};

// Fill the shared copy from the FP32 master parameters (exchange order).
__device__ inline void load_net(SmemNet &N, const float *p) {
  const float *W1 = p, *b1 = W1 + kHid * kIn, *W2 = b1 + kHid, *b2 = W2 + kHid * kHid, *W3 = b2 + kHid,
              *b3 = W3 + kHid * kHid, *W4 = b3 + kHid, *b4 = W4 + kOut * kHid;
  for (int i = threadIdx.x; i < kHid * kS16; i += blockDim.x) {
    const int r = i / kS16, c = i % kS16;
    N.W1[i] = __float2bfloat16_rn(c < kIn ? W1[r * kIn + c] : 0.0f);
  }
  for (int i = threadIdx.x; i < kHid * kS64; i += blockDim.x) {
    const int r = i / kS64, c = i % kS64;
    N.W2[i] = __float2bfloat16_rn(c < kHid ? W2[r * kHid + c] : 0.0f);
    N.W3[i] = __float2bfloat16_rn(c < kHid ? W3[r * kHid + c] : 0.0f);
  }
  for (int i = threadIdx.x; i < kOutPad * kS64; i += blockDim.x) {
    const int r = i / kS64, c = i % kS64;
    N.W4[i] = __float2bfloat16_rn(r < kOut && c < kHid ? W4[r * kHid + c] : 0.0f);
  }
  for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
    N.b1[i] = b1[i];
    N.b2[i] = b2[i];
    N.b3[i] = b3[i];
  }
  for (int i = threadIdx.x; i < kOutPad; i += blockDim.x) N.b4[i] = i < kOut ? b4[i] : 0.0f;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x2(uint32_t (&r)[2], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_addr(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t (&r)[2], const void *p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_addr(p)));
}
// D = A B + D: A 16x16 (row), B 16x8 (col), BF16 in, FP32 accumulate.
__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Fragment addresses (lane l).  A tile [16 rows][16 cols] at column k0 of a
// row-major array with stride s: rows l & 15, column half l >> 4.
__device__ __forceinline__ const __nv_bfloat16 *a_ptr(const __nv_bfloat16 *X, int s, int k0) {
  const int l = threadIdx.x & 31;
  return X + (l & 15) * s + k0 + (l >> 4) * 8;
}
// B = W^T slice (k0..k0+15, n0..n0+7) with W [n][k] row-major: rows n0 + (l & 7),
// column half (l >> 3) & 1 (lanes 16..31 repeat lanes 0..15).
__device__ __forceinline__ const __nv_bfloat16 *bt_ptr(const __nv_bfloat16 *W, int s, int n0, int k0) {
  const int l = threadIdx.x & 31;
  return W + (n0 + (l & 7)) * s + k0 + ((l >> 3) & 1) * 8;
}

// acc[NT][4] = b + X[16][16*KT] W^T, W [8*NT][16*KT] (row-major, strides xs, ws).
template <int KT, int NT>
__device__ __forceinline__ void layer_fwd(const __nv_bfloat16 *X, int xs, const __nv_bfloat16 *W, int ws,
                                          const float *b, float (&acc)[NT][4]) {
  const int l = threadIdx.x & 31, t = l & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const float b0 = b[nt * 8 + 2 * t], b1 = b[nt * 8 + 2 * t + 1];
    acc[nt][0] = b0;
    acc[nt][1] = b1;
    acc[nt][2] = b0;
    acc[nt][3] = b1;
  }
#pragma unroll
  for (int kt = 0; kt < KT; ++kt) {
    uint32_t a[4];
    ldsm_x4(a, a_ptr(X, xs, kt * 16));
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      uint32_t bb[2];
      ldsm_x2(bb, bt_ptr(W, ws, nt * 8, kt * 16));
      mma16816(acc[nt], a, bb);
    }
  }
}

// Store relu(acc) as bf16 into Y [16][8*NT] (stride ys); optionally the
// pre-activations into Z (fp32, stride zs).
template <int NT>
__device__ __forceinline__ void store_relu(const float (&acc)[NT][4], __nv_bfloat16 *Y, int ys, float *Z, int zs) {
  const int l = threadIdx.x & 31, g = l >> 2, t = l & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const int r = g + 8 * hf, c = nt * 8 + 2 * t;
      const float v0 = acc[nt][2 * hf], v1 = acc[nt][2 * hf + 1];
      if (Z) {
        Z[r * zs + c] = v0;
        Z[r * zs + c + 1] = v1;
      }
      *reinterpret_cast<__nv_bfloat162 *>(Y + r * ys + c) =
          __floats2bfloat162_rn(v0 > 0.0f ? v0 : 0.0f, v1 > 0.0f ? v1 : 0.0f);
    }
}

template <int NT>
__device__ __forceinline__ void store_f32(const float (&acc)[NT][4], float *Y, int ys) {
  const int l = threadIdx.x & 31, g = l >> 2, t = l & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int hf = 0; hf < 2; ++hf) {
      const int r = g + 8 * hf, c = nt * 8 + 2 * t;
      Y[r * ys + c] = acc[nt][2 * hf];
      Y[r * ys + c + 1] = acc[nt][2 * hf + 1];
    }
}

// Forward pass of one 16-point tile: x [16][kS16] (normalised inputs, bf16,
// columns >= kIn zero) -> y [16][ys] fp32 (normalised outputs, columns
// kOut..15 zero).  h0, h1: scratch tiles [16][kS64].  With z non-null the
// hidden pre-activations are kept as z[layer][16][64] (training).
__device__ __forceinline__ void warp_forward16(const SmemNet &N, const __nv_bfloat16 *x, __nv_bfloat16 *h0,
                                               __nv_bfloat16 *h1, float *y, int ys, float *z) {
  {
    float acc[8][4];
    layer_fwd<1, 8>(x, kS16, N.W1, kS16, N.b1, acc);
    store_relu<8>(acc, h0, kS64, z, kHid);
  }
  __syncwarp();
  {
    float acc[8][4];
    layer_fwd<4, 8>(h0, kS64, N.W2, kS64, N.b2, acc);
    store_relu<8>(acc, h1, kS64, z ? z + 16 * kHid : nullptr, kHid);
  }
  __syncwarp();
  {
    float acc[8][4];
    layer_fwd<4, 8>(h1, kS64, N.W3, kS64, N.b3, acc);
    store_relu<8>(acc, h0, kS64, z ? z + 32 * kHid : nullptr, kHid);
  }
  __syncwarp();
  {
    float acc[2][4];
    layer_fwd<4, 2>(h0, kS64, N.W4, kS64, N.b4, acc);
    store_f32<2>(acc, y, ys);
  }
  __syncwarp();
}

}  // namespace mlp
}  // namespace pdn

#include "pdn_umma.cuh"

namespace pdn {
namespace mlp {

// ---------------------------------------------------------------------------
// The same network on the Blackwell tensor cores (tcgen05, TMEM accumulators),
// 128 points per CTA of 128 threads, one point per thread (pdn_umma.cuh).

constexpr int kTcRows = 128;            // points per evaluation (MMA M)
constexpr uint32_t kTmemCols = 128;     // two 64-column accumulators
constexpr uint32_t kMaxPolls = 1u << 22;

// Weights in the core-matrix K-major layout (B operands), biases in FP32.
struct UmmaNet {
  __nv_bfloat16 W1[kHid * kInPad];   // [64 out][16 in]
  __nv_bfloat16 W2[kHid * kHid];     // [64][64]
  __nv_bfloat16 W3[kHid * kHid];
  __nv_bfloat16 W4[kOutPad * kHid];  // [16 out][64 in]
  float b1[kHid], b2[kHid], b3[kHid], b4[kOutPad];
};
// Activations of the 128 points (A operands), the MMA completion barrier
// and the TMEM base address written by the allocation.
struct UmmaTile {
  __nv_bfloat16 x[kTcRows * kInPad];
  __nv_bfloat16 h[kTcRows * kHid];
  uint64_t bar;
  uint32_t tmem;
  uint32_t pad;
};
static_assert(sizeof(UmmaNet) % 16 == 0 && sizeof(UmmaTile) % 16 == 0, "16-byte aligned operand tiles");

// Fill the shared copy from the FP32 master parameters (exchange order).
__device__ inline void load_net_umma(UmmaNet &N, const float *p) {
  const float *W1 = p, *b1 = W1 + kHid * kIn, *W2 = b1 + kHid, *b2 = W2 + kHid * kHid, *W3 = b2 + kHid,
              *b3 = W3 + kHid * kHid, *W4 = b3 + kHid, *b4 = W4 + kOut * kHid;
  for (int i = threadIdx.x; i < kHid * kInPad; i += blockDim.x) {
    const int r = i / kInPad, c = i % kInPad;
    N.W1[umma::core_offset(r, c, kInPad) / 2] = __float2bfloat16_rn(c < kIn ? W1[r * kIn + c] : 0.0f);
  }
  for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x) {
    const int r = i / kHid, c = i % kHid;
    N.W2[umma::core_offset(r, c, kHid) / 2] = __float2bfloat16_rn(W2[i]);
    N.W3[umma::core_offset(r, c, kHid) / 2] = __float2bfloat16_rn(W3[i]);
  }
  for (int i = threadIdx.x; i < kOutPad * kHid; i += blockDim.x) {
    const int r = i / kHid, c = i % kHid;
    N.W4[umma::core_offset(r, c, kHid) / 2] = __float2bfloat16_rn(r < kOut ? W4[r * kHid + c] : 0.0f);
  }
  for (int i = threadIdx.x; i < kHid; i += blockDim.x) {
    N.b1[i] = b1[i];
    N.b2[i] = b2[i];
    N.b3[i] = b3[i];
  }
  for (int i = threadIdx.x; i < kOutPad; i += blockDim.x) N.b4[i] = i < kOut ? b4[i] : 0.0f;
}

// Eight bf16 values as one 16-byte core-matrix row.
__device__ __forceinline__ uint4 pack8(const float *v) {
  uint4 q;
  uint32_t *w = reinterpret_cast<uint32_t *>(&q);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    w[k] = *reinterpret_cast<const uint32_t *>(&b);
  }
  return q;
}

// Row r of the input tile: the normalised inputs (kInPad values, columns
// kIn.. zero), rounded to bf16.
__device__ __forceinline__ void tc_store_input(UmmaTile &T, int r, const float (&xn)[kInPad]) {
  unsigned char *base = reinterpret_cast<unsigned char *>(T.x);
  *reinterpret_cast<uint4 *>(base + umma::core_offset(r, 0, kInPad)) = pack8(xn);
  *reinterpret_cast<uint4 *>(base + umma::core_offset(r, 8, kInPad)) = pack8(xn + 8);
}

// Forward pass of the 128 points whose normalised inputs are in T.x (row t
// written by thread t): y = the thread's normalised outputs (columns kOut..
// zero).  Called by all 128 threads; thread 0 issues the MMAs.  T.tmem holds
// kTmemCols allocated columns; phase is the completion barrier's current
// parity (the same in every thread).  Returns false in every thread when a
// wait on the tensor core gave up (after a second bounded wait for the MMA in
// flight); y is then not valid and no further MMA may be issued.
__device__ __forceinline__ bool tc_forward128(const UmmaNet &N, UmmaTile &T, uint32_t &phase, float (&y)[kOutPad]) {
  const int t = threadIdx.x;
  const uint32_t lane = ((uint32_t)(t & ~31)) << 16;  // warp w reads TMEM lanes 32 w ..
  umma::fence_smem_to_async();
  __syncthreads();
#pragma unroll 1
  for (int L = 0; L < 4; ++L) {
    const int K = L == 0 ? kInPad : kHid, Nn = L == 3 ? kOutPad : kHid;
    const __nv_bfloat16 *A = L == 0 ? T.x : T.h;
    const __nv_bfloat16 *B = L == 0 ? N.W1 : (L == 1 ? N.W2 : (L == 2 ? N.W3 : N.W4));
    const float *bias = L == 0 ? N.b1 : (L == 1 ? N.b2 : (L == 2 ? N.b3 : N.b4));
    const uint32_t col = (uint32_t)(L & 1) * 64u;
    if (t == 0) {
      umma::fence_after_sync();
      const uint32_t idesc = umma::idesc_bf16_f32(kTcRows, Nn);
      const uint32_t a0 = umma::saddr(A), b0 = umma::saddr(B);
      for (int kk = 0; kk < K / 16; ++kk)
        umma::mma_bf16(T.tmem + col, umma::smem_desc(a0 + 256u * kk, 128u, 16u * K),
                       umma::smem_desc(b0 + 256u * kk, 128u, 16u * K), idesc, kk > 0);
      umma::mma_commit(&T.bar);
    }
    const bool done = umma::mbar_wait(&T.bar, phase, kMaxPolls);
    if (__syncthreads_or(!done)) {
      umma::mbar_wait(&T.bar, phase, kMaxPolls);  // let an MMA in flight finish
      __syncthreads();
      return false;
    }
    phase ^= 1u;
    umma::fence_after_sync();
    if (L < 3) {
      unsigned char *hb = reinterpret_cast<unsigned char *>(T.h);
#pragma unroll 1
      for (int c = 0; c < kHid; c += 16) {
        float v[16];
        umma::tmem_ld16(T.tmem + lane + col + (uint32_t)c, v);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float z = v[k] + bias[c + k];
          v[k] = z > 0.0f ? z : 0.0f;
        }
        *reinterpret_cast<uint4 *>(hb + umma::core_offset(t, c, kHid)) = pack8(v);
        *reinterpret_cast<uint4 *>(hb + umma::core_offset(t, c + 8, kHid)) = pack8(v + 8);
      }
    } else {
      float v[16];
      umma::tmem_ld16(T.tmem + lane + col, v);
#pragma unroll
      for (int k = 0; k < kOutPad; ++k) y[k] = v[k] + bias[k];
    }
    umma::fence_before_sync();
    umma::fence_smem_to_async();
    __syncthreads();
  }
  return true;
}

// CTA set-up and tear-down of the tensor-core path: the barrier and the TMEM
// columns (allocated by warp 0, released by warp 0 after everyone is done).
__device__ __forceinline__ void tc_setup(UmmaTile &T) {
  if (threadIdx.x == 0) umma::mbar_init(&T.bar, 1);
  if (threadIdx.x < 32) umma::tmem_alloc(&T.tmem, kTmemCols);
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
}
__device__ __forceinline__ void tc_teardown(UmmaTile &T) {
  umma::fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    umma::fence_after_sync();
    umma::tmem_dealloc(T.tmem, kTmemCols);
  }
}

}  // namespace mlp
}  // namespace pdn
