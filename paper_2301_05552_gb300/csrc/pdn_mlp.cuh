// The learned surrogate of the intralaminar law, a multilayer perceptron
// 10 -> 64 -> 64 -> 64 -> 10 with ReLU, on the Blackwell tensor cores: BF16
// operands, FP32 accumulation in TMEM (tcgen05.mma, pdn_umma.cuh), 128 points
// per CTA of 128 threads, one point per thread.
//
// Conventions.  A layer with weights W [out][in] (row-major in the parameter
// exchange order) computes z = x W^T + b.  Activations of the 128 points are
// the A operand (row t: point t), the weights the B operand (K-major: row n
// holds output n's input weights), both in the no-swizzle core-matrix layout.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

namespace pdn {
namespace mlp {

constexpr int kIn = 10, kOut = 10, kHid = 64;
constexpr int kInPad = 16, kOutPad = 16;
// parameters in the exchange order W1[64][10], b1, W2[64][64], b2, W3, b3, W4[10][64], b4
constexpr int kNumParams = kHid * kIn + kHid + 2 * (kHid * kHid + kHid) + kOut * kHid + kOut;
static_assert(kNumParams == 9674, "10-64-64-64-10 perceptron");

// Input / output scaling and the training box (raw units).
struct Scaling {
  float in_shift[kIn], in_mul[kIn];    // x_n = (x - in_shift) * in_mul
  float out_shift[kOut], out_mul[kOut];  // y = y_n * out_mul + out_shift
  float lo[kIn], hi[kIn];              // inputs seen in training
};

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

// D (TMEM columns from dtmem) = A B for the 128 rows of A (128 x K, bf16,
// K-major core matrices) and B (N x K, K-major: row n holds the K inputs of
// output n).  Called by all 128 threads after they wrote their operand rows;
// thread 0 issues the MMAs.  Returns false in every thread when the wait
// gave up (after a second bounded wait for the MMA in flight); the result is
// then not valid and no further MMA may be issued.
__device__ __forceinline__ bool tc_mma128(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int K, int N,
                                          uint32_t dtmem, UmmaTile &T, uint32_t &phase) {
  umma::fence_before_sync();
  umma::fence_smem_to_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    umma::fence_after_sync();
    const uint32_t idesc = umma::idesc_bf16_f32(kTcRows, N);
    const uint32_t a0 = umma::saddr(A), b0 = umma::saddr(B);
    for (int kk = 0; kk < K / 16; ++kk)
      umma::mma_bf16(dtmem, umma::smem_desc(a0 + 256u * kk, 128u, 16u * K),
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
  return true;
}

// TMEM address of this thread's lane (warp w reads lanes 32 w ..) at column col.
__device__ __forceinline__ uint32_t tc_lane(const UmmaTile &T, uint32_t col) {
  return T.tmem + (((uint32_t)(threadIdx.x & ~31)) << 16) + col;
}

// Store 16 values as bf16 into row r, columns c..c+15, of a K-major tile with
// K columns; returns the two 16-byte rows written.
__device__ __forceinline__ void tc_store16(__nv_bfloat16 *tile, int K, int r, int c, const float (&v)[16], uint4 &lo,
                                           uint4 &hi) {
  unsigned char *b = reinterpret_cast<unsigned char *>(tile);
  lo = pack8(v);
  hi = pack8(v + 8);
  *reinterpret_cast<uint4 *>(b + umma::core_offset(r, c, K)) = lo;
  *reinterpret_cast<uint4 *>(b + umma::core_offset(r, c + 8, K)) = hi;
}

struct NoHidden {
  __device__ void operator()(int, int, const uint4 &, const uint4 &) const {}
};

// Forward pass of the 128 points whose normalised inputs are in T.x (row t
// written by thread t): y = the thread's normalised outputs (columns kOut..
// zero).  Called by all 128 threads; thread 0 issues the MMAs.  T.tmem holds
// kTmemCols allocated columns; phase is the completion barrier's current
// parity (the same in every thread).  on_hidden(layer, column, lo, hi)
// receives each 16-column piece of the thread's bf16 hidden activations.
// Returns false in every thread when a wait on the tensor core gave up; y is
// then not valid and no further MMA may be issued.
template <typename OnHidden = NoHidden>
__device__ __forceinline__ bool tc_forward128(const UmmaNet &N, UmmaTile &T, uint32_t &phase, float (&y)[kOutPad],
                                              OnHidden &&on_hidden = OnHidden{}) {
  const int t = threadIdx.x;
#pragma unroll 1
  for (int L = 0; L < 4; ++L) {
    const int K = L == 0 ? kInPad : kHid, Nn = L == 3 ? kOutPad : kHid;
    const __nv_bfloat16 *A = L == 0 ? T.x : T.h;
    const __nv_bfloat16 *B = L == 0 ? N.W1 : (L == 1 ? N.W2 : (L == 2 ? N.W3 : N.W4));
    const float *bias = L == 0 ? N.b1 : (L == 1 ? N.b2 : (L == 2 ? N.b3 : N.b4));
    const uint32_t col = (uint32_t)(L & 1) * 64u;
    if (!tc_mma128(A, B, K, Nn, T.tmem + col, T, phase)) return false;
    if (L < 3) {
#pragma unroll 1
      for (int c = 0; c < kHid; c += 16) {
        float v[16];
        umma::tmem_ld16(tc_lane(T, col + (uint32_t)c), v);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const float z = v[k] + bias[c + k];
          v[k] = z > 0.0f ? z : 0.0f;
        }
        uint4 lo, hi;
        tc_store16(T.h, kHid, t, c, v, lo, hi);
        on_hidden(L, c, lo, hi);
      }
    } else {
      float v[16];
      umma::tmem_ld16(tc_lane(T, col), v);
#pragma unroll
      for (int k = 0; k < kOutPad; ++k) y[k] = v[k] + bias[k];
    }
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
