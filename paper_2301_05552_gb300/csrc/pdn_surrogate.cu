// Learned surrogate of the intralaminar damage law (include/pdn_surrogate.h):
// training data from the exact law on the GPU, training (forward, backward,
// weight gradients, Adam) and inference on the Blackwell tensor cores
// (tcgen05.mma with TMEM accumulators, 128 points per CTA), BF16 operands and
// FP32 accumulation, and the hook that lets the hex kernel use it.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pdn.h"
#include "pdn_context.h"
#include "pdn_device.cuh"
#include "pdn_internal.h"
#include "pdn_mlp.cuh"
#include "pdn_surrogate.h"

namespace pdn {
template <typename T>
int fill_mat_public(Mat<T> &M, const pdn_material &m, const double *ply_angle, int n_plies, int damage_on,
                    int plasticity_on, std::string &why);

namespace {

using namespace detail;
using namespace mlp;

constexpr int kChunk = 128;               // points per weight-gradient partial
constexpr int kLayers = 4;
// padded output and input widths of layer l (0..3)
__host__ __device__ constexpr int layer_out(int l) { return l == 3 ? kOutPad : kHid; }
__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? kInPad : kHid; }

// ---------------------------------------------------------------------------
// Exact damage law on elastic strains (the plastic part of Algorithm 4 is
// not an input of the surrogate).

struct LawArgs {
  Mat<double> M;
  ElemLaw<double> L;
  double lc;
};

__device__ __forceinline__ void law_point(const LawArgs &A, const double (&ee)[6], double (&h)[7], double (&s)[6]) {
  double lc = A.lc;
  cdm_damage(A.M, A.L, (const double(*)[3]) nullptr, 0.0, lc, ee, h, s);
}

__device__ __forceinline__ double u01(uint64_t seed, int64_t p, int k) {
  const uint64_t z = splitmix64(seed ^ ((uint64_t)p * 0x100000001B3ULL) ^ ((uint64_t)k << 40));
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

// One elastic-strain path per thread from the undamaged state.  Pass 1
// (X == nullptr) counts the kept points of each path; pass 2 writes them at
// the path's offset, in path order.
__global__ void k_law_paths(LawArgs A, int64_t n_paths, int steps, double emax, double cyc, double ratio2,
                            uint64_t seed, int32_t *count, const int64_t *offset, float *X, float *Y) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_paths) return;
  const bool cyclic = u01(seed, p, 0) < cyc;
  const double amp = 1.0 - u01(seed, p, 1);
  double d[6];
  for (int i = 0; i < 6; ++i) d[i] = (2.0 * u01(seed, p, 2 + i) - 1.0) * (i < 3 ? emax : 2.0 * emax);
  const double waves = 1.0 + floor(3.0 * u01(seed, p, 8));
  double h[7] = {1.0, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0};
  int kept = 0;
  const int64_t o = offset ? offset[p] : 0;
  for (int k = 0; k < steps; ++k) {
    const double t = (double)(k + 1) / steps;
    const double f = cyclic ? sinpi(waves * t) : t;
    double ee[6];
    for (int i = 0; i < 6; ++i) ee[i] = amp * f * d[i];
    const double r2 = cdm_onset_ratio2(A.M, A.L, ee, h);
    double h2[7], s[6];
    for (int i = 0; i < 7; ++i) h2[i] = h[i];
    law_point(A, ee, h2, s);
    if (r2 <= ratio2) {
      if (X) {
        float *x = X + (o + kept) * kIn, *y = Y + (o + kept) * kOut;
        for (int i = 0; i < 6; ++i) {
          x[i] = (float)ee[i];
          y[i] = (float)s[i];
        }
        for (int i = 0; i < 4; ++i) {
          x[6 + i] = (float)h[i];
          y[6 + i] = (float)h2[i];
        }
      }
      ++kept;
    }
    for (int i = 0; i < 7; ++i) h[i] = h2[i];
  }
  if (count) count[p] = kept;
}

__global__ void k_law_points(LawArgs A, const float *in, float *out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double ee[6], h[7], s[6];
  for (int k = 0; k < 6; ++k) ee[k] = in[i * kIn + k];
  for (int k = 0; k < 4; ++k) h[k] = in[i * kIn + 6 + k];
  h[4] = h[5] = h[6] = 0.0;
  law_point(A, ee, h, s);
  for (int k = 0; k < 6; ++k) out[i * kOut + k] = (float)s[k];
  for (int k = 0; k < 4; ++k) out[i * kOut + 6 + k] = (float)h[k];
}

// ---------------------------------------------------------------------------
struct TrainBufs {
  __nv_bfloat16 *A0;      // [B][16]
  __nv_bfloat16 *A[3];    // [B][64]
  float *DZ[3];           // [B][64] gradients of the hidden pre-activations
  float *DY;              // [B][16] gradient of the outputs
  float *loss_part;       // [B / 16] per tile
};

// Forward and backward through the activations for B points on the Blackwell
// tensor cores: 128 points per CTA, one per thread (tcgen05.mma, FP32
// accumulators in TMEM); rows of X (raw inputs) and T (raw targets), drawn by
// a seeded hash when random, scaled by sc.  Loss = mean over points and the
// kOut outputs of (y_n - t_n)^2; its partial is per CTA (loss_part).  The
// backward products take the transposed weights as K-major operands (row n:
// the weights from input n to every output), so that every operand is
// K-major.  Stored for the weight gradients: the bf16 inputs and hidden
// activations, the FP32 output gradient and hidden pre-activation gradients.  A wait on the tensor core that gives up
// sets *status to PDN_E_TIMEOUT.
struct TrainTcSmem {
  UmmaNet N;                               // forward weights (K-major) and biases
  __nv_bfloat16 W4T[kHid * kOutPad];       // [64 inputs][16 outputs]
  __nv_bfloat16 W3T[kHid * kHid];          // [64 inputs][64 outputs]
  __nv_bfloat16 W2T[kHid * kHid];
  UmmaTile T;                              // inputs, hidden activations, barrier, TMEM address
  __nv_bfloat16 g16[kTcRows * kOutPad];    // output gradient
  __nv_bfloat16 g64[kTcRows * kHid];       // hidden gradient
  float red[kTcRows / 32];
};
static_assert(sizeof(UmmaNet) % 16 == 0 && sizeof(UmmaTile) % 16 == 0, "16-byte aligned operand tiles");

__device__ inline void load_net_transposed(TrainTcSmem &S, const float *p) {
  const float *W2 = p + kHid * kIn + kHid, *W3 = W2 + kHid * kHid + kHid, *W4 = W3 + kHid * kHid + kHid;
  for (int i = threadIdx.x; i < kHid * kOutPad; i += blockDim.x) {
    const int n = i / kOutPad, k = i % kOutPad;  // n: input of layer 4, k: its output
    S.W4T[umma::core_offset(n, k, kOutPad) / 2] = __float2bfloat16_rn(k < kOut ? W4[k * kHid + n] : 0.0f);
  }
  for (int i = threadIdx.x; i < kHid * kHid; i += blockDim.x) {
    const int n = i / kHid, k = i % kHid;
    S.W3T[umma::core_offset(n, k, kHid) / 2] = __float2bfloat16_rn(W3[k * kHid + n]);
    S.W2T[umma::core_offset(n, k, kHid) / 2] = __float2bfloat16_rn(W2[k * kHid + n]);
  }
}

__global__ void __launch_bounds__(kTcRows) k_train_tiles_tc(const float *params, Scaling sc, const float *X,
                                                            const float *Tgt, int64_t n_rows, int64_t B,
                                                            int32_t random, uint64_t seed, TrainBufs tb,
                                                            int32_t *status) {
  extern __shared__ __align__(16) unsigned char smem[];
  TrainTcSmem &S = *reinterpret_cast<TrainTcSmem *>(smem);
  const int t = threadIdx.x;
  load_net_umma(S.N, params);
  load_net_transposed(S, params);
  const int64_t row = (int64_t)blockIdx.x * kTcRows + t;  // B is a multiple of 128
  const int64_t src = random ? (int64_t)(splitmix64(seed ^ (uint64_t)row) % (uint64_t)n_rows) : row;
  {
    float xn[kInPad];
#pragma unroll
    for (int c = 0; c < kInPad; ++c) xn[c] = c < kIn ? (X[src * kIn + c] - sc.in_shift[c]) * sc.in_mul[c] : 0.0f;
    uint4 lo, hi;
    tc_store16(S.T.x, kInPad, t, 0, xn, lo, hi);
    uint4 *dst = reinterpret_cast<uint4 *>(tb.A0 + row * kInPad);
    dst[0] = lo;
    dst[1] = hi;
  }
  tc_setup(S.T);
  uint32_t phase = 0;
  float y[kOutPad];
  bool ok = tc_forward128(S.N, S.T, phase, y, [&](int L, int c, const uint4 &lo, const uint4 &hi) {
    uint4 *dst = reinterpret_cast<uint4 *>(tb.A[L] + row * kHid + c);
    dst[0] = lo;
    dst[1] = hi;
  });
  float lsum = 0.0f;
  if (ok) {
    // output gradient dL/dy_n = 2 (y_n - t_n) / (B kOut), padded columns 0
    const float gscale = 2.0f / ((float)B * (float)kOut);
    float g[16];
#pragma unroll
    for (int c = 0; c < kOutPad; ++c) {
      float gv = 0.0f;
      if (c < kOut) {
        const float tn = (Tgt[src * kOut + c] - sc.out_shift[c]) / sc.out_mul[c];
        const float dlt = y[c] - tn;
        lsum += dlt * dlt;
        gv = gscale * dlt;
      }
      g[c] = gv;
      tb.DY[row * kOutPad + c] = gv;
    }
    uint4 lo, hi;
    tc_store16(S.g16, kOutPad, t, 0, g, lo, hi);
    // backward through the hidden layers: dZ_L = (G W_{L+1}) * relu'(a_L)
#pragma unroll 1
    for (int L = 2; L >= 0 && ok; --L) {
      const __nv_bfloat16 *A = L == 2 ? S.g16 : S.g64;
      const __nv_bfloat16 *Bt = L == 2 ? S.W4T : (L == 1 ? S.W3T : S.W2T);
      const uint32_t col = (uint32_t)(L & 1) * 64u;
      ok = tc_mma128(A, Bt, L == 2 ? kOutPad : kHid, kHid, S.T.tmem + col, S.T, phase);
      if (!ok) break;
#pragma unroll 1
      for (int c = 0; c < kHid; c += 16) {
        float v[16];
        umma::tmem_ld16(tc_lane(S.T, col + (uint32_t)c), v);
        const __nv_bfloat16 *act = tb.A[L] + row * kHid + c;
        float *dz = tb.DZ[L] + row * kHid + c;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          v[k] = __bfloat162float(act[k]) > 0.0f ? v[k] : 0.0f;
          dz[k] = v[k];
        }
        tc_store16(S.g64, kHid, t, c, v, lo, hi);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((t & 31) == 0) S.red[t >> 5] = lsum;
  __syncthreads();
  if (t == 0) {
    float tot = 0.0f;
    for (int w = 0; w < kTcRows / 32; ++w) tot += S.red[w];
    tb.loss_part[blockIdx.x] = tot / ((float)B * (float)kOut);
    if (!ok) atomicExch(status, PDN_E_TIMEOUT);
  }
  tc_teardown(S.T);
}

// Weight and bias gradients of one layer over one chunk of kChunk points, on
// the Blackwell tensor cores: one CTA per (chunk of 128 points, layer).  dW[n][k] = sum_m dZ[m][n] A[m][k] is the MMA
// D[n][k] = sum over K = the 128 points of dZ^T[n][m] A^T[k][m]: both
// operands are staged transposed (rows n and k, the points along K), rows of
// the 128-row A operand past the layer's outputs are zero.  Lane n of TMEM
// then holds dW[n][:] for thread n.  The bias gradient is the fixed-order
// FP32 sum of dZ over the chunk as before.
struct WgradTcSmem {
  __nv_bfloat16 gT[kTcRows * kChunk];    // dZ^T [128 (outputs, padded)][128 points]
  __nv_bfloat16 aT[kHid * kChunk];       // A^T [64 (inputs)][128 points]
  UmmaTile T;                            // barrier and TMEM address (its tiles unused)
};

__global__ void __launch_bounds__(kTcRows) k_train_wgrad_tc(TrainBufs tb, int64_t B, float *partW, float *partB,
                                                            int64_t n_chunks, int32_t *status) {
  extern __shared__ __align__(16) unsigned char smem[];
  WgradTcSmem &S = *reinterpret_cast<WgradTcSmem *>(smem);
  const int layer = blockIdx.y;
  const int64_t chunk = blockIdx.x;
  const int M = layer_out(layer), K = layer_in(layer);
  const float *dz = layer == 3 ? tb.DY : tb.DZ[layer];
  const __nv_bfloat16 *act = layer == 0 ? tb.A0 : tb.A[layer - 1];
  const int t = threadIdx.x;
  const int64_t r0 = chunk * kChunk;
  unsigned char *gb = reinterpret_cast<unsigned char *>(S.gT), *ab = reinterpret_cast<unsigned char *>(S.aT);
  // thread t stages point t: its M gradients into column t of dZ^T, its K
  // activations into column t of A^T; rows of dZ^T past M are zero
  for (int n = 0; n < kTcRows; ++n) {
    const float v = n < M ? dz[(r0 + t) * M + n] : 0.0f;
    *reinterpret_cast<__nv_bfloat16 *>(gb + umma::core_offset(n, t, kChunk)) = __float2bfloat16_rn(v);
  }
  for (int k = 0; k < K; ++k)
    *reinterpret_cast<__nv_bfloat16 *>(ab + umma::core_offset(k, t, kChunk)) = act[(r0 + t) * K + k];
  tc_setup(S.T);
  uint32_t phase = 0;
  const bool ok = tc_mma128(S.gT, S.aT, kChunk, K, S.T.tmem, S.T, phase);
  float *pW = partW + ((size_t)layer * n_chunks + chunk) * (kHid * kHid);
  float *pB = partB + ((size_t)layer * n_chunks + chunk) * kHid;
  if (ok) {
#pragma unroll 1
    for (int c = 0; c < K; c += 16) {
      float v[16];
      umma::tmem_ld16(tc_lane(S.T, (uint32_t)c), v);
      if (t < M) {
#pragma unroll
        for (int k = 0; k < 16; ++k) pW[t * K + c + k] = v[k];
      }
    }
  }
  if (t < M) {
    float sb = 0.0f;
    for (int r = 0; r < kChunk; ++r) sb += dz[(r0 + r) * M + t];
    pB[t] = sb;
  }
  if (!ok && t == 0) atomicExch(status, PDN_E_TIMEOUT);
  tc_teardown(S.T);
}

// Parameter p of the exchange order -> (layer, row, column or -1 for a bias).
__device__ __forceinline__ void param_site(int p, int &layer, int &row, int &col) {
  const int sizes[8] = {kHid * kIn, kHid, kHid * kHid, kHid, kHid * kHid, kHid, kOut * kHid, kOut};
  const int cols[4] = {kIn, kHid, kHid, kHid};
  int q = p;
  for (int s = 0; s < 8; ++s) {
    if (q < sizes[s]) {
      layer = s >> 1;
      if (s & 1) {
        row = q;
        col = -1;
      } else {
        row = q / cols[layer];
        col = q % cols[layer];
      }
      return;
    }
    q -= sizes[s];
  }
  layer = row = col = -1;
}

// Sum of the chunk partials (in chunk order) for every parameter; then an
// Adam step (lr > 0) and/or the gradient copy.  Thread 0 also sums the loss.
__global__ void k_train_update(float *params, float *m1, float *m2, float *grad_out, const float *partW,
                               const float *partB, int64_t n_chunks, float lr, float bc1, float bc2,
                               const float *loss_part, int64_t n_tiles, double *loss_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p == 0 && loss_out) {
    double s = 0.0;
    for (int64_t i = 0; i < n_tiles; ++i) s += loss_part[i];
    *loss_out = s;
  }
  if (p >= kNumParams) return;
  int layer, row, col;
  param_site(p, layer, row, col);
  const int K = layer_in(layer);
  float g = 0.0f;
  for (int64_t c = 0; c < n_chunks; ++c) {
    const size_t base = (size_t)layer * n_chunks + c;
    g += col < 0 ? partB[base * kHid + row] : partW[base * (kHid * kHid) + row * K + col];
  }
  if (grad_out) grad_out[p] = g;
  if (lr > 0.0f) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float mm = b1 * m1[p] + (1.0f - b1) * g;
    const float vv = b2 * m2[p] + (1.0f - b2) * g * g;
    m1[p] = mm;
    m2[p] = vv;
    params[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + 1e-8f);
  }
}

// Inference on raw points on the Blackwell tensor cores: 128 points per CTA,
// one per thread (tc_forward128).  A wait on the tensor core that gives up
// sets *status to PDN_E_TIMEOUT and leaves the CTA's outputs unwritten.
struct SurTcSmem {
  UmmaNet N;
  UmmaTile T;
};
constexpr int kTcBlock = kTcRows;
// dynamic shared memory of the inference kernel, more than it uses: at most
// three CTAs per SM, so that their TMEM columns (3 x 128) always fit the
// SM's 512 and no allocation has to wait for another CTA
constexpr size_t kSurTcSmem = 64 * 1024;
static_assert(sizeof(SurTcSmem) <= kSurTcSmem, "inference tiles fit the reserved shared memory");

__global__ void __launch_bounds__(kTcBlock) k_sur_forward_tc(const float *params, Scaling sc, const float *in,
                                                             float *out, int64_t n, int32_t *status) {
  extern __shared__ __align__(16) unsigned char smem[];
  SurTcSmem &S = *reinterpret_cast<SurTcSmem *>(smem);
  const int t = threadIdx.x;
  load_net_umma(S.N, params);
  const int64_t i = (int64_t)blockIdx.x * kTcBlock + t;
  float xn[kInPad];
#pragma unroll
  for (int c = 0; c < kInPad; ++c) {
    const float raw = (c < kIn && i < n) ? in[i * kIn + c] : 0.0f;
    xn[c] = c < kIn ? (raw - sc.in_shift[c]) * sc.in_mul[c] : 0.0f;
  }
  tc_store_input(S.T, t, xn);
  tc_setup(S.T);
  uint32_t phase = 0;
  float y[kOutPad];
  const bool ok = tc_forward128(S.N, S.T, phase, y);
  if (ok && i < n) {
#pragma unroll
    for (int c = 0; c < kOut; ++c) out[i * kOut + c] = y[c] * sc.out_mul[c] + sc.out_shift[c];
  }
  if (!ok && t == 0) atomicExch(status, PDN_E_TIMEOUT);
  tc_teardown(S.T);
}

// He-uniform initial weights (bound sqrt(6 / fan_in)), zero biases.
__global__ void k_init_params(float *p, uint64_t seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNumParams) return;
  int layer, row, col;
  param_site(i, layer, row, col);
  if (col < 0) {
    p[i] = 0.0f;
    return;
  }
  const float fan_in = (float)(layer == 0 ? kIn : kHid);
  const double u = (double)(splitmix64(seed ^ (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
  p[i] = (float)((2.0 * u - 1.0) * sqrt(6.0 / fan_in));
}

// ---------------------------------------------------------------------------
// Hex8 of an axis-aligned box (FP32) with the learned law where it applies.
// Same formulation and arithmetic as the scalar element of pdn_items.cuh
// (Eq. fcont, Algorithm 4); at each Gauss point the exact plasticity runs
// first, then either the network (all loading-function ratios at most the
// context's onset ratio and every input inside the training box: the
// thresholds do not change there) or the exact damage part.  The network
// runs on the tensor cores (tcgen05, TMEM accumulators) for the 128 points of
// the CTA (one element per thread, the same Gauss point) whenever any thread
// of the CTA needs it; threads past the last element follow the same control
// flow on a valid element and store nothing.  A bounded wait on the tensor
// core that gives up raises the control block's timeout word (the tail then
// halts the run with PDN_E_TIMEOUT) and the CTA finishes with the exact law.

constexpr int kHexSurBlock = kTcRows;  // at most three CTAs per SM (registers): 3 x 128 TMEM columns
struct HexSurSmem {
  UmmaNet N;
  UmmaTile T;
  Scaling sc;
};
constexpr size_t kHexSurSmem = sizeof(HexSurSmem);
static_assert(sizeof(Scaling) == PDN_SUR_SCALING * sizeof(float), "scaling record of 60 floats");
static_assert(sizeof(Scaling) % 16 == 0, "16-byte aligned shared tiles");

__global__ void __launch_bounds__(kHexSurBlock, 3) k_hex_sur(Dev<float> D, Mat<float> M) {
  extern __shared__ __align__(16) unsigned char smem[];
  HexSurSmem &S = *reinterpret_cast<HexSurSmem *>(smem);
  const Ctl *ctl = D.ctl;
  const int mode = ctl->mode;
  if (mode >= MODE_DONE) return;
  load_net_umma(S.N, D.sur_params);
  for (int k = threadIdx.x; k < PDN_SUR_SCALING; k += blockDim.x)
    reinterpret_cast<float *>(&S.sc)[k] = D.sur_params[kNumParams + k];
  const Scaling &sc = S.sc;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nh = D.nh;
  // a repeated pass evaluates only the marked elements (local repetition);
  // the others follow the CTA on their own element and store nothing
  bool act = e < nh;
  if (mode == MODE_REPEAT && act) act = repeat_take(D.rmark_e, e);
  if (!__syncthreads_or(act)) return;  // nothing to do in this CTA (no TMEM held yet)
  tc_setup(S.T);
  uint32_t phase = 0;
  bool tc_ok = true;
  const int64_t el = e < nh ? e : nh - 1;
  const int ub = (mode == MODE_FORCES) ? (ctl->dpar ^ 1) : ctl->dpar;
  const int hb = ctl->hpar;
  const float4 *__restrict__ U = D.u4[ub];
  const int4 c0 = __ldg(reinterpret_cast<const int4 *>(D.hex) + 2 * el);
  const int4 c1 = __ldg(reinterpret_cast<const int4 *>(D.hex) + 2 * el + 1);
  int nd[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  if (!nodes_in_range(D, nd)) {
    // PDN_CHECK build: the element is skipped (its CTA still takes part in
    // every network evaluation)
#pragma unroll
    for (int a = 0; a < 8; ++a) nd[a] = 0;
    act = false;
  }
  const float *__restrict__ hin = D.hist[hb] + el;
  float *__restrict__ hout = D.hist[hb ^ 1] + el;
  const bool pristine_in = D.pflag[0] != nullptr && D.pflag[hb][el] != 0;
  bool dirty = false;
  float bm[8][3], jd[3], wd[3], vol;
  {
    float ua[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const float4 u = U[nd[a]];
      ua[a][0] = u.x;
      ua[a][1] = u.y;
      ua[a][2] = u.z;
    }
    to_modes(ua, bm);
    const float4 x0 = D.X4[nd[0]], x6 = D.X4[nd[6]];
    const float J0 = 0.5f * (x6.x - x0.x), J1 = 0.5f * (x6.y - x0.y), J2 = 0.5f * (x6.z - x0.z);
    const float det = J0 * (J1 * J2);
    jd[0] = 1.0f / J0;
    jd[1] = 1.0f / J1;
    jd[2] = 1.0f / J2;
    wd[0] = det * jd[0];
    wd[1] = det * jd[1];
    wd[2] = det * jd[2];
    vol = 8.0f * det;
  }
  const int ply = D.ply[el];
  const float cs = M.ply_c[ply], sn = M.ply_s[ply];
  const float c2 = cs * cs, s2 = sn * sn, csn = cs * sn;
  const ElemLaw<float> L = elem_law(M, el);
  float lc = -1.0f;
  float C[8][3];
#pragma unroll
  for (int m = 0; m < 8; ++m) C[m][0] = C[m][1] = C[m][2] = 0.0f;
  const float gp = 0.57735026918962576451f;
#pragma unroll 1
  for (int g = 0; g < 8; ++g) {
    float h[7];
#pragma unroll
    for (int f = 0; f < 7; ++f) h[f] = pristine_in ? (f < 4 ? 1.0f : 0.0f) : hin[(int64_t)(f * 8 + g) * nh];
    const float xi = float(sgn_x(g)) * gp, et = float(sgn_y(g)) * gp, ze = float(sgn_z(g)) * gp;
    float Du[3][3], H[3][3];
    jac_cols(bm, xi, et, ze, Du);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) H[i][k] = Du[i][k] * jd[k];
    float E[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = i; k < 3; ++k) {
        E[i][k] = 0.5f * (H[i][k] + H[k][i] + H[0][i] * H[0][k] + H[1][i] * H[1][k] + H[2][i] * H[2][k]);
        E[k][i] = E[i][k];
      }
    float ep[6];
    ep[0] = c2 * E[0][0] + 2.0f * csn * E[0][1] + s2 * E[1][1];
    ep[1] = s2 * E[0][0] - 2.0f * csn * E[0][1] + c2 * E[1][1];
    ep[2] = E[2][2];
    ep[3] = 2.0f * (-csn * E[0][0] + (c2 - s2) * E[0][1] + csn * E[1][1]);
    ep[4] = 2.0f * (cs * E[0][2] + sn * E[1][2]);
    ep[5] = 2.0f * (-sn * E[0][2] + cs * E[1][2]);
    cdm_plastic(M, ep, h);
    const float eel[6] = {ep[0], ep[1], ep[2], ep[3] - h[4], ep[4] - h[5], ep[5]};
    bool inbox = true;
#pragma unroll
    for (int k = 0; k < 6; ++k) inbox = inbox && eel[k] >= sc.lo[k] && eel[k] <= sc.hi[k];
#pragma unroll
    for (int k = 0; k < 4; ++k) inbox = inbox && h[k] >= sc.lo[6 + k] && h[k] <= sc.hi[6 + k];
    const bool use = act && inbox && cdm_onset_ratio2(M, L, eel, h) <= D.sur_ratio2;
    float sm[6];
    bool net = false;
    if (__syncthreads_or(use) && tc_ok) {
      float xn[kInPad];
#pragma unroll
      for (int c = 0; c < kInPad; ++c) {
        const float raw = c < 6 ? eel[c] : (c < kIn ? h[c - 6] : 0.0f);
        xn[c] = c < kIn ? (raw - sc.in_shift[c]) * sc.in_mul[c] : 0.0f;
      }
      tc_store_input(S.T, threadIdx.x, xn);
      float y[kOutPad];
      tc_ok = tc_forward128(S.N, S.T, phase, y);
      net = use && tc_ok;
      if (net) {
#pragma unroll
        for (int k = 0; k < 6; ++k) sm[k] = y[k] * sc.out_mul[k] + sc.out_shift[k];
      }
    }
    if (!net) cdm_damage(M, L, (const float(*)[3]) nullptr, vol, lc, ep, h, sm);
    if (act) {
      if (!pristine_in) {
#pragma unroll
        for (int f = 0; f < 7; ++f) hout[(int64_t)(f * 8 + g) * nh] = h[f];
      } else {
        const bool changed = h[0] > 1.0f || h[1] > 1.0f || h[2] > 1.0f || h[3] > 1.0f || h[4] != 0.0f ||
                             h[5] != 0.0f || h[6] != 0.0f;
        if (changed && !dirty) {
          for (int gg = 0; gg < g; ++gg)
#pragma unroll
            for (int f = 0; f < 7; ++f) hout[(int64_t)(f * 8 + gg) * nh] = f < 4 ? 1.0f : 0.0f;
          dirty = true;
        }
        if (dirty) {
#pragma unroll
          for (int f = 0; f < 7; ++f) hout[(int64_t)(f * 8 + g) * nh] = h[f];
        }
      }
    }
    float Sg[3][3];
    Sg[0][0] = c2 * sm[0] - 2.0f * csn * sm[3] + s2 * sm[1];
    Sg[1][1] = s2 * sm[0] + 2.0f * csn * sm[3] + c2 * sm[1];
    Sg[2][2] = sm[2];
    Sg[0][1] = Sg[1][0] = csn * sm[0] + (c2 - s2) * sm[3] - csn * sm[1];
    Sg[0][2] = Sg[2][0] = cs * sm[4] - sn * sm[5];
    Sg[1][2] = Sg[2][1] = sn * sm[4] + cs * sm[5];
    float Q[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int I = 0; I < 3; ++I)
        Q[k][I] = wd[k] * (Sg[k][I] + Sg[k][0] * H[I][0] + Sg[k][1] * H[I][1] + Sg[k][2] * H[I][2]);
#pragma unroll
    for (int I = 0; I < 3; ++I) {
      C[1][I] += Q[0][I];
      C[2][I] += Q[1][I];
      C[3][I] += Q[2][I];
      C[4][I] += et * Q[0][I] + xi * Q[1][I];
      C[5][I] += ze * Q[1][I] + et * Q[2][I];
      C[6][I] += ze * Q[0][I] + xi * Q[2][I];
      C[7][I] += et * ze * Q[0][I] + xi * ze * Q[1][I] + xi * et * Q[2][I];
    }
  }
  tc_teardown(S.T);
  if (!tc_ok && threadIdx.x == 0) atomicOr(&D.ctl->timeout, 1);
  if (!act) return;
  if (mode == MODE_REPEAT) repeat_mark_nodes(D.rmark_n, nd);
  if (D.pflag[0] != nullptr) D.pflag[hb ^ 1][el] = (pristine_in && !dirty) ? 1 : 0;
  float f[8][3];
  from_modes(C, f);
  int ps[8];
  element_slots(D, D.hex, el, reinterpret_cast<const int4 *>(D.pos) + 2 * el,
                D.rank != nullptr ? __ldg(D.rank + el) : 0u, ps);
#pragma unroll
  for (int a = 0; a < 8; ++a) D.fe[ps[a]] = make_float4(f[a][0], f[a][1], f[a][2], 0.0f);
}

thread_local std::string g_sur_error;

}  // namespace
}  // namespace pdn

namespace pdn {
cudaError_t launch_hex_sur(const Dev<float> &D, const Mat<float> &M, cudaStream_t s) {
  const int64_t g = (D.nh + kHexSurBlock - 1) / kHexSurBlock;
  k_hex_sur<<<(unsigned)(g < 1 ? 1 : g), kHexSurBlock, kHexSurSmem, s>>>(D, M);
  return cudaGetLastError();
}
}  // namespace pdn

using namespace pdn;
using namespace pdn::mlp;

struct pdn_surrogate {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  LawArgs law{};
  Scaling sc{};
  float *params = nullptr, *m1 = nullptr, *m2 = nullptr;  // device, kNumParams each
  int64_t adam_t = 0;
  // training set
  float *X = nullptr, *Y = nullptr;
  int64_t n = 0;
  // work buffers for a minibatch of cap points
  int64_t cap = 0;
  TrainBufs tb{};
  float *partW = nullptr, *partB = nullptr, *grad = nullptr;
  double *loss_dev = nullptr;
  int32_t *status_dev = nullptr;  // error word of the tensor-core inference kernel
  std::string err;
};

namespace {

int sfail(pdn_surrogate *s, int code, const std::string &m) {
  if (s) s->err = m;
  return code;
}
int scuda(pdn_surrogate *s, cudaError_t e, const char *where) {
  return sfail(s, PDN_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define PS_CU(call, where)                             \
  do {                                                 \
    cudaError_t _e = (call);                           \
    if (_e != cudaSuccess) return scuda(s, _e, where); \
  } while (0)


void free_bufs(pdn_surrogate *s) {
  cudaFree(s->tb.A0);
  for (int k = 0; k < 3; ++k) {
    cudaFree(s->tb.A[k]);
    cudaFree(s->tb.DZ[k]);
  }
  cudaFree(s->tb.DY);
  cudaFree(s->tb.loss_part);
  cudaFree(s->partW);
  cudaFree(s->partB);
  s->tb = TrainBufs{};
  s->partW = s->partB = nullptr;
  s->cap = 0;
}

int ensure_bufs(pdn_surrogate *s, int64_t B) {
  if (B <= s->cap) return PDN_OK;
  free_bufs(s);
  const int64_t nch = B / kChunk;
  PS_CU(cudaMalloc(&s->tb.A0, sizeof(__nv_bfloat16) * B * kInPad), "surrogate buffers");
  for (int k = 0; k < 3; ++k) {
    PS_CU(cudaMalloc(&s->tb.A[k], sizeof(__nv_bfloat16) * B * kHid), "surrogate buffers");
    PS_CU(cudaMalloc(&s->tb.DZ[k], sizeof(float) * B * kHid), "surrogate buffers");
  }
  PS_CU(cudaMalloc(&s->tb.DY, sizeof(float) * B * kOutPad), "surrogate buffers");
  PS_CU(cudaMalloc(&s->tb.loss_part, sizeof(float) * (B / 16)), "surrogate buffers");
  PS_CU(cudaMalloc(&s->partW, sizeof(float) * kLayers * nch * kHid * kHid), "surrogate buffers");
  PS_CU(cudaMalloc(&s->partB, sizeof(float) * kLayers * nch * kHid), "surrogate buffers");
  s->cap = B;
  return PDN_OK;
}

// One forward/backward over B points (rows of X/T; random: seeded draws),
// weight gradients, then the update (lr > 0: Adam) and/or gradient copy.
int train_step(pdn_surrogate *s, const Scaling &sc, const float *X, const float *T, int64_t n_rows, int64_t B,
               int random, uint64_t seed, float lr, float *grad_out, double *loss_out) {
  int rc = ensure_bufs(s, B);
  if (rc) return rc;
  const int64_t tiles = B / kTcRows, nch = B / kChunk;
  k_train_tiles_tc<<<(unsigned)tiles, kTcRows, sizeof(TrainTcSmem), s->stream>>>(s->params, sc, X, T, n_rows, B,
                                                                                random, seed, s->tb, s->status_dev);
  PS_CU(cudaGetLastError(), "train tiles");
  k_train_wgrad_tc<<<dim3((unsigned)nch, kLayers), kTcRows, sizeof(WgradTcSmem), s->stream>>>(
      s->tb, B, s->partW, s->partB, nch, s->status_dev);
  PS_CU(cudaGetLastError(), "weight gradients");
  float bc1 = 1.0f, bc2 = 1.0f;
  if (lr > 0.0f) {
    ++s->adam_t;
    bc1 = 1.0f - std::pow(0.9f, (float)s->adam_t);
    bc2 = 1.0f - std::pow(0.999f, (float)s->adam_t);
  }
  k_train_update<<<(kNumParams + 255) / 256, 256, 0, s->stream>>>(s->params, s->m1, s->m2, grad_out, s->partW,
                                                                    s->partB, nch, lr, bc1, bc2, s->tb.loss_part,
                                                                    tiles, loss_out);
  PS_CU(cudaGetLastError(), "update");
  return PDN_OK;
}

Scaling identity_scaling() {
  Scaling sc{};
  for (int i = 0; i < kIn; ++i) {
    sc.in_shift[i] = 0.0f;
    sc.in_mul[i] = 1.0f;
    sc.lo[i] = -1e30f;
    sc.hi[i] = 1e30f;
  }
  for (int i = 0; i < kOut; ++i) {
    sc.out_shift[i] = 0.0f;
    sc.out_mul[i] = 1.0f;
  }
  return sc;
}

}  // namespace

extern "C" {

const char *pdn_sur_last_error(const pdn_surrogate *s) { return s ? s->err.c_str() : g_sur_error.c_str(); }

void pdn_sur_destroy(pdn_surrogate *s) {
  if (!s) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  free_bufs(s);
  cudaFree(s->params);
  cudaFree(s->m1);
  cudaFree(s->m2);
  cudaFree(s->X);
  cudaFree(s->Y);
  cudaFree(s->grad);
  cudaFree(s->loss_dev);
  cudaFree(s->status_dev);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  cudaSetDevice(prev);
  delete s;
}

static int pdn_sur_create_body(pdn_surrogate **out, const pdn_material *mat, double lc, uint64_t seed, void *stream) {
  g_sur_error.clear();
  if (!out) {
    g_sur_error = "out is NULL";
    return PDN_E_ARG;
  }
  *out = nullptr;
  if (!mat || !(lc > 0.0)) {
    g_sur_error = "a material and lc > 0 are required";
    return PDN_E_ARG;
  }
  pdn_surrogate *s = new (std::nothrow) pdn_surrogate();
  if (!s) {
    g_sur_error = "host allocation failed";
    return PDN_E_OOM;
  }
  auto bad = [&](int code, const std::string &m) {
    g_sur_error = m;
    pdn_sur_destroy(s);
    return code;
  };
  cudaGetDevice(&s->device);
  std::string why;
  const double zero_angle = 0.0;
  int rc = fill_mat_public(s->law.M, *mat, &zero_angle, 1, 1, 0, why);
  if (rc) return bad(rc, why);
  Mat<double> &M = s->law.M;
  s->law.L.XT = M.XT;
  s->law.L.YT = M.YT;
  s->law.L.SL = M.SL;
  s->law.L.iXT = 1.0 / M.XT;
  s->law.L.iYT = 1.0 / M.YT;
  s->law.L.iSL2 = 1.0 / (M.SL * M.SL);
  s->law.L.etaL = M.SL * M.etaLc;
  s->law.lc = lc;
  // below the snap-back length only: past it the law drops to zero stress at
  // onset (d jumps at r = 1), which a smooth network cannot represent
  const double X[5] = {M.XT, M.XC, M.YT, M.YC, M.SL}, E[5] = {M.E1, M.E1, M.E2, M.E2, M.G12},
               G[5] = {M.GXT, M.GXC, M.GYT, M.GYC, M.GSL};
  for (int k = 0; k < 5; ++k)
    if (!(2.0 * E[k] * G[k] - lc * X[k] * X[k] > 0.0))
      return bad(PDN_E_UNSTABLE, "crack-band length too large for this material (snap-back)");
  s->sc = identity_scaling();
  if (stream) {
    s->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bad(PDN_E_CUDA, "stream create failed");
    s->own_stream = true;
  }
  if (cudaMalloc(&s->params, sizeof(float) * kNumParams) != cudaSuccess ||
      cudaMalloc(&s->m1, sizeof(float) * kNumParams) != cudaSuccess ||
      cudaMalloc(&s->m2, sizeof(float) * kNumParams) != cudaSuccess ||
      cudaMalloc(&s->grad, sizeof(float) * kNumParams) != cudaSuccess ||
      cudaMalloc(&s->loss_dev, sizeof(double) * 1) != cudaSuccess ||
      cudaMalloc(&s->status_dev, sizeof(int32_t)) != cudaSuccess)
    return bad(PDN_E_OOM, "surrogate parameters");
  cudaMemsetAsync(s->m1, 0, sizeof(float) * kNumParams, s->stream);
  cudaMemsetAsync(s->m2, 0, sizeof(float) * kNumParams, s->stream);
  k_init_params<<<(kNumParams + 255) / 256, 256, 0, s->stream>>>(s->params, seed);
  if (cudaFuncSetAttribute(k_sur_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSurTcSmem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_train_tiles_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(TrainTcSmem)) != cudaSuccess ||
      cudaFuncSetAttribute(k_train_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(WgradTcSmem)) != cudaSuccess)
    return bad(PDN_E_CUDA, "shared-memory attribute");
  if (cudaStreamSynchronize(s->stream) != cudaSuccess) return bad(PDN_E_CUDA, "surrogate init");
  *out = s;
  return PDN_OK;
}

// No exception leaves the library: a failed host allocation is PDN_E_OOM.
int pdn_sur_create(pdn_surrogate **out, const pdn_material *mat, double lc, uint64_t seed, void *stream) {
  try {
    return pdn_sur_create_body(out, mat, lc, seed, stream);
  } catch (const std::bad_alloc &) {
    return PDN_E_OOM;
  } catch (...) {
    return PDN_E_ARG;
  }
}

static int pdn_sur_generate_body(pdn_surrogate *s, int64_t n_paths, int32_t steps, double strain_max, double cyclic_fraction,
                     double onset_ratio, uint64_t seed, int64_t *n_kept) {
  if (!s) return PDN_E_ARG;
  if (n_paths < 1 || steps < 1 || steps > 1024 || !(strain_max > 0.0) || !(onset_ratio > 0.0) ||
      !(cyclic_fraction >= 0.0 && cyclic_fraction <= 1.0))
    return sfail(s, PDN_E_ARG, "bad path parameters");
  int32_t *cnt = nullptr;
  int64_t *off = nullptr;
  PS_CU(cudaMalloc(&cnt, sizeof(int32_t) * n_paths), "path counts");
  const double r2 = onset_ratio * onset_ratio;
  const unsigned grid = (unsigned)((n_paths + 127) / 128);
  k_law_paths<<<grid, 128, 0, s->stream>>>(s->law, n_paths, steps, strain_max, cyclic_fraction, r2, seed, cnt,
                                           nullptr, nullptr, nullptr);
  std::vector<int32_t> hc(n_paths);
  cudaError_t e = cudaMemcpyAsync(hc.data(), cnt, sizeof(int32_t) * n_paths, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    cudaFree(cnt);
    return scuda(s, e, "count pass");
  }
  std::vector<int64_t> ho(n_paths);
  int64_t tot = 0;
  for (int64_t p = 0; p < n_paths; ++p) {
    ho[p] = tot;
    tot += hc[p];
  }
  if (tot < 128) {
    cudaFree(cnt);
    return sfail(s, PDN_E_ARG, "fewer than 128 points in the surrogate regime");
  }
  cudaFree(s->X);
  cudaFree(s->Y);
  s->X = s->Y = nullptr;
  s->n = 0;
  e = cudaMalloc(&off, sizeof(int64_t) * n_paths);
  if (e == cudaSuccess) e = cudaMalloc(&s->X, sizeof(float) * kIn * tot);
  if (e == cudaSuccess) e = cudaMalloc(&s->Y, sizeof(float) * kOut * tot);
  if (e == cudaSuccess) e = cudaMemcpyAsync(off, ho.data(), sizeof(int64_t) * n_paths, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) {
    k_law_paths<<<grid, 128, 0, s->stream>>>(s->law, n_paths, steps, strain_max, cyclic_fraction, r2, seed, nullptr,
                                             off, s->X, s->Y);
    e = cudaGetLastError();
  }
  std::vector<float> hx, hy;
  if (e == cudaSuccess) {
    hx.resize((size_t)kIn * tot);
    hy.resize((size_t)kOut * tot);
    e = cudaMemcpyAsync(hx.data(), s->X, sizeof(float) * kIn * tot, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hy.data(), s->Y, sizeof(float) * kOut * tot, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  }
  cudaFree(cnt);
  cudaFree(off);
  if (e != cudaSuccess) return scuda(s, e, "training set");
  s->n = tot;
  // scaling: mean and spread of the kept points; box: their range
  Scaling sc{};
  for (int c = 0; c < kIn; ++c) {
    double m = 0.0, q = 0.0, lo = 1e300, hi = -1e300;
    for (int64_t i = 0; i < tot; ++i) {
      const double v = hx[i * kIn + c];
      m += v;
      q += v * v;
      lo = std::min(lo, v);
      hi = std::max(hi, v);
    }
    m /= tot;
    const double sd = std::sqrt(std::max(q / tot - m * m, 0.0));
    const double floor = c < 6 ? 1e-7 : 1e-3;
    sc.in_shift[c] = (float)m;
    sc.in_mul[c] = (float)(1.0 / std::max(sd, floor));
    sc.lo[c] = (float)lo;
    sc.hi[c] = (float)hi;
  }
  for (int c = 0; c < kOut; ++c) {
    double m = 0.0, q = 0.0;
    for (int64_t i = 0; i < tot; ++i) {
      const double v = hy[i * kOut + c];
      m += v;
      q += v * v;
    }
    m /= tot;
    const double sd = std::sqrt(std::max(q / tot - m * m, 0.0));
    sc.out_shift[c] = (float)m;
    sc.out_mul[c] = (float)std::max(sd, c < 6 ? 1e-3 : 1e-3);
  }
  s->sc = sc;
  if (n_kept) *n_kept = tot;
  return PDN_OK;
}

// No exception leaves the library: a failed host allocation is PDN_E_OOM.
int pdn_sur_generate(pdn_surrogate *s, int64_t n_paths, int32_t steps, double strain_max, double cyclic_fraction,
                     double onset_ratio, uint64_t seed, int64_t *n_kept) {
  try {
    return pdn_sur_generate_body(s, n_paths, steps, strain_max, cyclic_fraction, onset_ratio, seed, n_kept);
  } catch (const std::bad_alloc &) {
    return PDN_E_OOM;
  } catch (...) {
    return PDN_E_ARG;
  }
}

int pdn_sur_get_data(pdn_surrogate *s, int64_t offset, int64_t n, float *x, float *y) {
  if (!s) return PDN_E_ARG;
  if (offset < 0 || n < 0 || offset + n > s->n) return sfail(s, PDN_E_ARG, "range outside the training set");
  if (n == 0) return PDN_OK;
  if (x) PS_CU(cudaMemcpyAsync(x, s->X + offset * kIn, sizeof(float) * kIn * n, cudaMemcpyDeviceToHost, s->stream), "read set");
  if (y) PS_CU(cudaMemcpyAsync(y, s->Y + offset * kOut, sizeof(float) * kOut * n, cudaMemcpyDeviceToHost, s->stream), "read set");
  PS_CU(cudaStreamSynchronize(s->stream), "read set");
  return PDN_OK;
}

int pdn_sur_train(pdn_surrogate *s, int64_t iters, int32_t batch, double lr, uint64_t seed, double *loss) {
  if (!s) return PDN_E_ARG;
  if (iters < 0 || batch < kChunk || batch % kChunk || !(lr > 0.0)) return sfail(s, PDN_E_ARG, "bad training parameters");
  if (s->n < kChunk) return sfail(s, PDN_E_STATE, "no training set (pdn_sur_generate)");
  std::vector<double> lh;
  double *ld = nullptr;
  if (loss) PS_CU(cudaMalloc(&ld, sizeof(double) * std::max<int64_t>(iters, 1)), "loss buffer");
  PS_CU(cudaMemsetAsync(s->status_dev, 0, sizeof(int32_t), s->stream), "status");
  for (int64_t it = 0; it < iters; ++it) {
    const double frac = iters > 1 ? (double)it / (double)(iters - 1) : 0.0;
    const double lr_it = lr * (0.01 + 0.99 * 0.5 * (1.0 + std::cos(M_PI * frac)));
    const uint64_t sd = splitmix64(seed + 0x51ED270B2A3F1C07ULL * (uint64_t)(it + 1));
    int rc = train_step(s, s->sc, s->X, s->Y, s->n, batch, 1, sd, (float)lr_it, nullptr, ld ? ld + it : nullptr);
    if (rc) {
      cudaFree(ld);
      return rc;
    }
  }
  cudaError_t e = cudaSuccess;
  int32_t st = 0;
  if (ld && iters > 0) e = cudaMemcpyAsync(loss, ld, sizeof(double) * iters, cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, s->status_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(ld);
  if (e != cudaSuccess) return scuda(s, e, "training");
  if (st) return sfail(s, st, "training: a bounded wait on the tensor core gave up");
  return PDN_OK;
}

int pdn_sur_gradient(pdn_surrogate *s, const float *xn, const float *tn, int64_t n, float *grad, double *loss) {
  if (!s) return PDN_E_ARG;
  if (!xn || !tn || !grad || n < kChunk || n % kChunk) return sfail(s, PDN_E_ARG, "need n a multiple of 128 and host arrays");
  float *dx = nullptr, *dt = nullptr;
  PS_CU(cudaMalloc(&dx, sizeof(float) * kIn * n), "gradient inputs");
  cudaError_t e = cudaMalloc(&dt, sizeof(float) * kOut * n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dx, xn, sizeof(float) * kIn * n, cudaMemcpyHostToDevice, s->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dt, tn, sizeof(float) * kOut * n, cudaMemcpyHostToDevice, s->stream);
  int rc = PDN_OK;
  if (e == cudaSuccess) e = cudaMemsetAsync(s->status_dev, 0, sizeof(int32_t), s->stream);
  if (e == cudaSuccess) rc = train_step(s, identity_scaling(), dx, dt, n, n, 0, 0, 0.0f, s->grad, s->loss_dev);
  if (e == cudaSuccess && rc == PDN_OK)
    e = cudaMemcpyAsync(grad, s->grad, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, s->stream);
  double lh = 0.0;
  int32_t st = 0;
  if (e == cudaSuccess && rc == PDN_OK) e = cudaMemcpyAsync(&lh, s->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess && rc == PDN_OK)
    e = cudaMemcpyAsync(&st, s->status_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(dx);
  cudaFree(dt);
  if (rc) return rc;
  if (e != cudaSuccess) return scuda(s, e, "gradient");
  if (st) return sfail(s, st, "gradient: a bounded wait on the tensor core gave up");
  if (loss) *loss = lh;
  return PDN_OK;
}

static int sur_points(pdn_surrogate *s, const float *in, float *out, int64_t n, int32_t on_device, bool exact) {
  if (!s) return PDN_E_ARG;
  if (!in || !out || n < 0) return sfail(s, PDN_E_ARG, "bad point arrays");
  if (n == 0) return PDN_OK;
  const float *din = in;
  float *dout = out;
  float *tmp_in = nullptr, *tmp_out = nullptr;
  if (!on_device) {
    PS_CU(cudaMalloc(&tmp_in, sizeof(float) * kIn * n), "point buffers");
    PS_CU(cudaMalloc(&tmp_out, sizeof(float) * kOut * n), "point buffers");
    PS_CU(cudaMemcpyAsync(tmp_in, in, sizeof(float) * kIn * n, cudaMemcpyHostToDevice, s->stream), "copy points");
    din = tmp_in;
    dout = tmp_out;
  }
  if (exact) {
    k_law_points<<<(unsigned)((n + 127) / 128), 128, 0, s->stream>>>(s->law, din, dout, n);
  } else {
    cudaMemsetAsync(s->status_dev, 0, sizeof(int32_t), s->stream);
    k_sur_forward_tc<<<(unsigned)((n + kTcBlock - 1) / kTcBlock), kTcBlock, kSurTcSmem, s->stream>>>(
        s->params, s->sc, din, dout, n, s->status_dev);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && !on_device)
    e = cudaMemcpyAsync(out, dout, sizeof(float) * kOut * n, cudaMemcpyDeviceToHost, s->stream);
  int32_t st = 0;
  if (e == cudaSuccess && !exact)
    e = cudaMemcpyAsync(&st, s->status_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  cudaFree(tmp_in);
  cudaFree(tmp_out);
  if (e != cudaSuccess) return scuda(s, e, exact ? "exact law" : "surrogate forward");
  if (st) return sfail(s, st, "surrogate forward: a bounded wait on the tensor core gave up");
  return PDN_OK;
}

int pdn_sur_forward(pdn_surrogate *s, const float *in, float *out, int64_t n, int32_t on_device) {
  return sur_points(s, in, out, n, on_device, false);
}

int pdn_sur_exact(pdn_surrogate *s, const float *in, float *out, int64_t n, int32_t on_device) {
  return sur_points(s, in, out, n, on_device, true);
}

int pdn_sur_get_params(pdn_surrogate *s, float *params, float *scaling) {
  if (!s) return PDN_E_ARG;
  if (params) {
    PS_CU(cudaMemcpyAsync(params, s->params, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, s->stream), "read params");
    PS_CU(cudaStreamSynchronize(s->stream), "read params");
  }
  if (scaling) std::memcpy(scaling, &s->sc, sizeof(float) * PDN_SUR_SCALING);
  return PDN_OK;
}

int pdn_set_surrogate(pdn_ctx *ctx, pdn_surrogate *s, double onset_ratio) {
  if (!ctx) return PDN_E_ARG;
  if (!s) {
    ctx->Df.sur_params = nullptr;
    return PDN_OK;
  }
  if (ctx->precision != PDN_FP32_FORCE || !ctx->Df.all_boxes) {
    ctx->err = "the learned law needs FP32 element mode and axis-aligned box elements";
    return PDN_E_ARG;
  }
  if (!(onset_ratio > 0.0 && onset_ratio <= 1.0)) {
    ctx->err = "onset_ratio must be in (0, 1]";
    return PDN_E_ARG;
  }
  if (cudaFuncSetAttribute(k_hex_sur, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHexSurSmem) != cudaSuccess) {
    ctx->err = "shared-memory attribute of the learned-law hex kernel";
    return PDN_E_CUDA;
  }
  if (!ctx->sur_buf) {
    if (cudaMalloc(&ctx->sur_buf, sizeof(float) * (kNumParams + PDN_SUR_SCALING)) != cudaSuccess) {
      ctx->err = "learned-law parameters";
      return PDN_E_OOM;
    }
  }
  // the context's copy: parameters, then the scaling, on the context's stream
  cudaError_t e = cudaStreamSynchronize(s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->sur_buf, s->params, sizeof(float) * kNumParams, cudaMemcpyDeviceToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->sur_buf + kNumParams, &s->sc, sizeof(float) * PDN_SUR_SCALING, cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    ctx->err = std::string("learned-law parameters: ") + cudaGetErrorString(e);
    return PDN_E_CUDA;
  }
  ctx->Df.sur_params = ctx->sur_buf;
  ctx->Df.sur_ratio2 = (float)(onset_ratio * onset_ratio);
  // the captured graph holds the old kernel choice
  if (ctx->graph) {
    cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
  }
  return PDN_OK;
}

int pdn_sur_set_params(pdn_surrogate *s, const float *params, const float *scaling) {
  if (!s) return PDN_E_ARG;
  if (params) {
    PS_CU(cudaMemcpyAsync(s->params, params, sizeof(float) * kNumParams, cudaMemcpyHostToDevice, s->stream), "write params");
    PS_CU(cudaStreamSynchronize(s->stream), "write params");
  }
  if (scaling) std::memcpy(&s->sc, scaling, sizeof(float) * PDN_SUR_SCALING);
  return PDN_OK;
}

}  // extern "C"
