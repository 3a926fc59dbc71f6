// CUDA kernels of the explicit PDN impact step for GB300 (sm_103a).
//
// One pass = contact -> (hex8 || interface) -> gather -> tail.  The tail owns
// the device-side state machine (pdn_internal.h): it
// commits the step, or marks a repetition after releasing adhesive contact
// nodes (Algorithm 2), or halts on a non-finite state.  Every kernel first
// reads the mode and returns at once when there is nothing to do, so a fixed
// sequence of passes (a CUDA graph) can be replayed without host decisions.
//
// Precision: the element kernels run in T (float for PDN_FP32_FORCE, double
// for PDN_FP64); nodal displacement/velocity accumulation, the striker, the
// contact gap test and the reaction sum are double in both modes.
#include "pdn_internal.h"

#include <cstdint>
#include <cstdlib>
#include <algorithm>
#include <type_traits>

#include "pdn.h"
#include "pdn_device.cuh"
#include "pdn_items.cuh"

namespace pdn {
namespace {

using namespace detail;

// Programmatic dependent launch: the next kernel of the pass may be
// scheduled once every block of this one has started (its blocks then take
// SM slots as this kernel's last wave drains), and every kernel waits for the
// previous grid's completion before it reads anything.  Without the launch
// attribute both instructions have no effect.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Kernels of a pass (one launch per step part); the per-item bodies are in
// pdn_items.cuh, shared with the batched persistent kernel.
template <typename T>
__global__ void __launch_bounds__(kActRun) k_contact(Dev<T> D) {
  pdl_enter();
  const int mode = D.ctl->mode;
  if (mode != MODE_ADVANCE && mode != MODE_REPEAT) return;
  const bool on = contact_item(D, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, mode);
  // the run's count of active nodes, for the tail's ordered list
  const int c = __syncthreads_count(on);
  if (D.act_cnt != nullptr && threadIdx.x == 0) D.act_cnt[blockIdx.x] = c;
}

template <typename T, bool BOX, int MINB>
__global__ void __launch_bounds__(128, MINB) k_hex(Dev<T> D, Mat<T> M) {
  pdl_enter();
  const int mode = D.ctl->mode;
  if (mode >= MODE_DONE) return;
  hex_item<T, BOX>(D, M, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, mode);
}

template <typename T, bool FLAT, int MINB>
__global__ void __launch_bounds__(128, MINB) k_coh(Dev<T> D, Mat<T> M) {
  pdl_enter();
  const int mode = D.ctl->mode;
  if (mode >= MODE_DONE) return;
  coh_item<T, FLAT>(D, M, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, mode);
}

// Hex and interface elements in one launch: blocks alternate between a tile
// of hexes and a tile of interface elements (then the remainder of the
// larger kind), so that every SM runs both the compute-bound hex warps and
// the latency-bound interface warps at the same time.
template <typename T, bool BOX, int MINB>
__global__ void __launch_bounds__(128, MINB) k_elem(Dev<T> D, Mat<T> M, int nbh, int nbc) {
  pdl_enter();
  const int mode = D.ctl->mode;
  if (mode >= MODE_DONE) return;
  const int b = blockIdx.x, m = nbh < nbc ? nbh : nbc;
  int kind, idx;
  if (b < 2 * m) {
    kind = b & 1;
    idx = b >> 1;
  } else {
    kind = nbh > nbc ? 0 : 1;
    idx = m + (b - 2 * m);
  }
  const int64_t i = (int64_t)idx * blockDim.x + threadIdx.x;
  if (kind == 0)
    hex_item<T, BOX>(D, M, i, mode);
  else if (D.all_flat_coh)
    coh_item<T, true>(D, M, i, mode);
  else
    coh_item<T, false>(D, M, i, mode);
}

template <typename T>
__global__ void __launch_bounds__(256) k_gather(Dev<T> D) {
  pdl_enter();
  const int mode = D.ctl->mode;
  if (mode >= MODE_DONE) return;
  gather_item(D, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, mode);
}

// Kernel 4 with interfaces as node pairs: the gather also evaluates the
// cohesive law of each interface node pair (no interface kernel runs).
// (FP32: at most 64 registers, four blocks of 256 per SM for this
// memory-bound kernel)
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) k_gather_pairs(Dev<T> D, Mat<T> M) {
  pdl_enter();
  const int mode = D.ctl->mode;
  if (mode >= MODE_DONE) return;
  gather_pair_item(D, M, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, mode);
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) k_gather_pairs_layered(Dev<T> D, Mat<T> M) {
  pdl_enter();
  const int mode = D.ctl->mode;
  if (mode >= MODE_DONE) return;
  gather_pair_layered_item(D, M, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, mode);
}

// The element layout of the interface thresholds (rD, cflag at the
// committed history parity) from the node pairs' thresholds, for the readers
// of that layout (history read-back, energy ledger, damage field).
template <typename T>
__global__ void k_pairs_to_elements(Dev<T> D) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D.nc) return;
  const int hb = D.ctl->hpar;
  bool zero = true;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const T r = D.rDn[hb][D.coh[8 * c + p]];
    D.rD[hb][(int64_t)p * D.nc + c] = r;
    zero = zero && r == T(0);
  }
  D.cflag[hb][c] = zero ? 1 : 0;
}

// Kernel 5: the tail of a pass as its own small launch (kept out of the
// gather, whose occupancy depends on a low register count).
template <typename T>
__global__ void __launch_bounds__(256) k_tail(Dev<T> D) {
  pdl_enter();
  const int mode = D.ctl->mode;
  if (mode >= MODE_DONE) return;
  tail_block<T, true>(D, mode);
}

// Column sweep (Sweep, pdn_internal.h): one block per tile of TX x TY
// element columns and z-chunk, one thread per column.  Stage by stage (hex or
// interface layer, bottom to top) each thread evaluates its column's element;
// the force of every corner whose node column has all its elements in this
// tile goes to a shared-memory slot (the node's rank, as in the gather), the
// others to the global slots.  After a stage its bottom node layer is
// complete: the nodes of the tile's complete columns sum their eight slots in
// rank order, exactly as the gather does, take the same update (node_update)
// and clear their slots for the layer two above.  Nodes on tile and chunk
// boundaries are left to the gather over the list (k_gather_list).
template <int TX, int TY>
struct SweepSmem {
  static constexpr int NC = (TX + 1) * (TY + 1);  // node columns of a tile
  float s[2][8][3][NC];                            // [layer parity][rank][component][column]
  double dv[6][NC];                                // d and v of the layer to update, copied ahead
  uint32_t flw[NC];                                // the 4-byte word holding each node's flag byte
  float im[NC];                                    // inverse lumped mass
};

// 4-byte asynchronous copy global -> shared.
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src)
               : "memory");
}

// 8-byte asynchronous copy global -> shared (cp.async; completed by
// cp_async_wait_all in the issuing thread).
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}

template <int TX, int TY>
__global__ void __launch_bounds__(TX * TY, 512 / (TX * TY)) k_sweep(Dev<float> D, Mat<float> M, Sweep S) {
  constexpr int NT = TX * TY, NC = (TX + 1) * (TY + 1);
  __shared__ SweepSmem<TX, TY> sm;
  pdl_enter();
  const int mode = D.ctl->mode;
  if (mode >= MODE_DONE) return;
  const int t = threadIdx.x;
  const int tile = blockIdx.x % (S.tiles_x * S.tiles_y), chunk = blockIdx.x / (S.tiles_x * S.tiles_y);
  const int i0 = (tile % S.tiles_x) * TX, j0 = (tile / S.tiles_x) * TY;
  const int txe = min(TX, S.nx - i0), tye = min(TY, S.ny - j0);  // the tile's columns
  const int k0 = chunk * S.chunk_len, k1 = min(S.n_stages, k0 + S.chunk_len);
  // node column (ni, nj) of the tile: all its elements in the tile
  auto complete = [&](int ni, int nj) {
    return ni <= txe && nj <= tye && (ni > 0 || i0 == 0) && (ni < txe || i0 + txe == S.nx) &&
           (nj > 0 || j0 == 0) && (nj < tye || j0 + tye == S.ny);
  };
  // a node layer is summed here unless it is shared with the chunk below/above
  auto layer_here = [&](int L) { return (L > S.bot[k0] || k0 == 0) && (L < S.bot[k1 - 1] + 1 || k1 == S.n_stages); };
  for (int q = t; q < 2 * 8 * 3 * NC; q += NT) (&sm.s[0][0][0][0])[q] = 0.0f;
  const int ti = t % TX, tj = t / TX;
  const bool col = ti < txe && tj < tye;
  const int gi = i0 + ti, gj = j0 + tj;
  // corners 0..3: (0,0), (1,0), (1,1), (0,1) of the column's quad; 4..7 above
  const int cdx[4] = {0, 1, 1, 0}, cdy[4] = {0, 0, 1, 1};
  bool cmask[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) cmask[a] = complete(ti + cdx[a], tj + cdy[a]);
  __syncthreads();

  // the displacement and velocity of the nodes a gather of layer L updates,
  // copied into shared memory while the stage's elements are computed
  const int cur = D.ctl->dpar;
  auto prefetch_layer = [&](int L) {
    if (mode == MODE_FORCES) return;
    for (int q = t; q < NC; q += NT) {
      const int ni = q % (TX + 1), nj = q / (TX + 1);
      if (!complete(ni, nj)) continue;
      const int64_t j = (int64_t)L * S.per_layer + (int64_t)(j0 + nj) * S.nxn + (i0 + ni);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        cp_async8(&sm.dv[i][q], D.d[cur] + i * D.nn + j);
        cp_async8(&sm.dv[3 + i][q], D.v[cur] + i * D.nn + j);
      }
      // the flag array is padded to whole 4-byte words
      cp_async4(&sm.flw[q], D.nflag + (j & ~int64_t(3)));
      cp_async4(&sm.im[q], D.inv_mass + j);
    }
  };
  auto gather_layer = [&](int L) {
    const int p = L & 1;
    for (int q = t; q < NC; q += NT) {
      const int ni = q % (TX + 1), nj = q / (TX + 1);
      if (!complete(ni, nj)) continue;
      const int64_t j = (int64_t)L * S.per_layer + (int64_t)(j0 + nj) * S.nxn + (i0 + ni);
      NodeState<float> st;
      st.fl = 0;
      st.im = 0.0f;
#pragma unroll
      for (int i = 0; i < 3; ++i) st.dc[i] = st.vc[i] = 0.0;
      if (mode != MODE_FORCES) {
        st.fl = (uint8_t)(sm.flw[q] >> (8 * (int)(j & 3)));
        st.im = sm.im[q];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          st.dc[i] = sm.dv[i][q];
          st.vc[i] = sm.dv[3 + i][q];
        }
      }
      float fx = 0.0f, fy = 0.0f, fz = 0.0f;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        fx += sm.s[p][r][0][q];
        fy += sm.s[p][r][1][q];
        fz += sm.s[p][r][2][q];
        sm.s[p][r][0][q] = 0.0f;
        sm.s[p][r][1][q] = 0.0f;
        sm.s[p][r][2][q] = 0.0f;
      }
      node_update(D, j, mode, st, fx, fy, fz);
    }
  };

  for (int k = k0; k < k1; ++k) {
    const int L = S.bot[k];
    const bool lo_here = layer_here(L), hi_here = layer_here(L + 1);
    if (lo_here) prefetch_layer(L);
    if (col) {
      const int64_t el = (int64_t)S.base[k] + (int64_t)gj * S.nx + gi;
      auto store = [&](const float (&f)[8][3], const int (&nd)[8]) {
        const uint32_t rk = __ldg(D.rank + (S.kind[k] ? D.nh + el : el));
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const int r = (int)((rk >> (3 * a)) & 7u);
          const int c = a & 3;
          const bool here = cmask[c] && (a < 4 ? lo_here : hi_here);
          if (here) {
            const int q = (tj + cdy[c]) * (TX + 1) + ti + cdx[c];
            const int p = (a < 4 ? L : L + 1) & 1;
            sm.s[p][r][0][q] = f[a][0];
            sm.s[p][r][1][q] = f[a][1];
            sm.s[p][r][2][q] = f[a][2];
          } else {
            D.fe[8 * (int64_t)nd[a] + r] = make_float4(f[a][0], f[a][1], f[a][2], 0.0f);
          }
        }
      };
      if (S.kind[k] == 0)
        hex_box_forces(D, M, el, mode, store);
      else
        coh_forces<float, true>(D, M, el, mode, store);
    }
    cp_async_wait_all();
    __syncthreads();
    if (lo_here) gather_layer(L);
    __syncthreads();
  }
  const int Ltop = S.bot[k1 - 1] + 1;
  if (layer_here(Ltop)) {
    prefetch_layer(Ltop);
    cp_async_wait_all();
    __syncthreads();
    gather_layer(Ltop);
  }
}

// The gather over a list of nodes (the sweep's boundary nodes).
template <typename T>
__global__ void __launch_bounds__(256) k_gather_list(Dev<T> D, const int32_t *list, int64_t n) {
  pdl_enter();
  const int mode = D.ctl->mode;
  if (mode >= MODE_DONE) return;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) gather_item(D, (int64_t)list[q], mode);
}

// After pdn_set_impactor: the striker of the first step to be computed.
__global__ void k_striker_init(Striker *S, StrikerStep *ss, double dt) {
  double c1[3], w1[3], aI[3];
  striker_rk4(*S, dt, c1, w1, aI);
  for (int i = 0; i < 3; ++i) {
    ss->c[i] = c1[i];
    ss->w[i] = w1[i];
    ss->aI[i] = aI[i];
  }
}

// ---------------------------------------------------------------------------
// Field output: per element maximum over its points of the committed history.
template <typename T>
__global__ void k_damage_field(Dev<T> D, Mat<T> M, int which, float *out) {
  using V4 = typename Vec4T<T>::type;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int hb = D.ctl->hpar;
  if (which == PDN_FIELD_DCOH) {
    if (e >= D.nc) return;
    T m = T(0);
    if (D.cflag[0] != nullptr && D.cflag[hb][e]) {
      out[e] = 0.0f;  // undamaged: the threshold buffer is not maintained
      return;
    }
    for (int p = 0; p < 4; ++p) {
      const T r = D.rD[hb][(int64_t)p * D.nc + e];
      m = r > m ? r : m;
    }
    out[e] = (float)m;
    return;
  }
  if (e >= D.nh) return;
  const int64_t nh = D.nh;
  const T *h = D.hist[hb];
  if (D.pflag[0] != nullptr && D.pflag[hb][e]) {
    out[e] = 0.0f;  // initial history: no damage, no plastic strain
    return;
  }
  if (which == PDN_FIELD_PLASTIC) {
    T m = T(0);
    for (int g = 0; g < 8; ++g) {
      const T p = h[((int64_t)6 * 8 + g) * nh + e];
      m = p > m ? p : m;
    }
    out[e] = (float)m;
    return;
  }
  const int4 c0 = reinterpret_cast<const int4 *>(D.hex)[2 * e];
  const int4 c1 = reinterpret_cast<const int4 *>(D.hex)[2 * e + 1];
  const int nd[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  T xa[8][3], am[8][3];
  for (int a = 0; a < 8; ++a) {
    const V4 x = D.X4[nd[a]];
    xa[a][0] = x.x;
    xa[a][1] = x.y;
    xa[a][2] = x.z;
  }
  to_modes(xa, am);
  const T lc = xcbrt(hex_volume(am));
  const T XT = M.XT * strength_factor(M, e, 0), YT = M.YT * strength_factor(M, e, 1),
          SL = M.SL * strength_factor(M, e, 2);
  T m = T(0);
  for (int g = 0; g < 8; ++g) {
    const T rFT = h[((int64_t)0 * 8 + g) * nh + e], rFC = h[((int64_t)1 * 8 + g) * nh + e];
    const T rMT = h[((int64_t)2 * 8 + g) * nh + e], rMC = h[((int64_t)3 * 8 + g) * nh + e];
    T v;
    if (which == PDN_FIELD_D1) {
      const T a = dmg(rFT, soft_A(lc, XT, M.E1, M.GXT)), b = dmg(rFC, soft_A(lc, M.XC, M.E1, M.GXC));
      v = a > b ? a : b;
    } else if (which == PDN_FIELD_D2) {
      const T a = dmg(rMT, soft_A(lc, YT, M.E2, M.GYT)), b = dmg(rMC, soft_A(lc, M.YC, M.E2, M.GYC));
      v = a > b ? a : b;
    } else {
      v = dmg(rMT, soft_A(lc, SL, M.G12, M.GSL));
    }
    m = v > m ? v : m;
  }
  out[e] = (float)m;
}

// Launch on the pass's main stream, with the programmatic-dependency
// attribute unless PDN_PDL=0.
bool pdl_on() {
  static const bool on = [] {
    const char *e = std::getenv("PDN_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

template <typename... KArgs, typename... Args>
void launch_k(void (*k)(KArgs...), int grid, int block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_on() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, args...);
}

inline int grid_of(int64_t n, int b) {
  int64_t g = (n + b - 1) / b;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

// Element kernel variants chosen per context by the autotuner: 0..3 hex
// kernel (interface kernel on the side stream) with an occupancy target of 4,
// 5, 6 or 3 blocks of 128 per SM (which caps the registers per thread);
// 4..7 the same targets for the mixed hex + interface kernel.
constexpr int kMixedVariant = 4;

template <typename T, bool BOX>
void launch_elem_box(const Dev<T> &D, const Mat<T> &M, cudaStream_t s) {
  const int nbh = grid_of(D.nh, 128), nbc = D.nc > 0 ? (int)((D.nc + 127) / 128) : 0;
  const int g = nbh + nbc;
  switch (D.hex_variant) {
    case 5: launch_k(k_elem<T, BOX, 5>, g, 128, s, D, M, nbh, nbc); break;
    case 6: launch_k(k_elem<T, BOX, 6>, g, 128, s, D, M, nbh, nbc); break;
    case 7: launch_k(k_elem<T, BOX, 3>, g, 128, s, D, M, nbh, nbc); break;
    default: launch_k(k_elem<T, BOX, 4>, g, 128, s, D, M, nbh, nbc); break;
  }
}

template <typename T>
void launch_elem(const Dev<T> &D, const Mat<T> &M, cudaStream_t s) {
  if (D.all_boxes)
    launch_elem_box<T, true>(D, M, s);
  else
    launch_elem_box<T, false>(D, M, s);
}

template <typename T>
void launch_hex(const Dev<T> &D, const Mat<T> &M, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (D.sur_params != nullptr && D.all_boxes) {
      launch_hex_sur(D, M, s);
      return;
    }
  }
  const int g = grid_of(D.nh, 128);
  if (D.all_boxes) {
    switch (D.hex_variant) {
      case 1: launch_k(k_hex<T, true, 5>, g, 128, s, D, M); break;
      case 2: launch_k(k_hex<T, true, 6>, g, 128, s, D, M); break;
      case 3: launch_k(k_hex<T, true, 3>, g, 128, s, D, M); break;
      default: launch_k(k_hex<T, true, 4>, g, 128, s, D, M); break;
    }
  } else {
    switch (D.hex_variant) {
      case 1: launch_k(k_hex<T, false, 5>, g, 128, s, D, M); break;
      case 2: launch_k(k_hex<T, false, 6>, g, 128, s, D, M); break;
      case 3: launch_k(k_hex<T, false, 3>, g, 128, s, D, M); break;
      default: launch_k(k_hex<T, false, 4>, g, 128, s, D, M); break;
    }
  }
}

// Interface kernel: the flat-rectangle specialisation when every interface
// allows it; pdl = launched with programmatic dependent launch (not on the
// forked side stream).
template <typename T>
void launch_coh(const Dev<T> &D, const Mat<T> &M, cudaStream_t s, bool pdl) {
  // FP32 flat interfaces fit 64 registers without spilling (8 blocks per
  // SM); the others keep the compiler's budget
  constexpr int kFlatMinBlocks = std::is_same<T, float>::value ? 8 : 1;
  const int g = grid_of(D.nc, 128);
  if (D.all_flat_coh) {
    if (pdl)
      launch_k(k_coh<T, true, kFlatMinBlocks>, g, 128, s, D, M);
    else
      k_coh<T, true, kFlatMinBlocks><<<g, 128, 0, s>>>(D, M);
  } else {
    if (pdl)
      launch_k(k_coh<T, false, 1>, g, 128, s, D, M);
    else
      k_coh<T, false, 1><<<g, 128, 0, s>>>(D, M);
  }
}

// One pass: contact, then the hex and interface kernels (concurrently when a
// side stream with fork/join events is given: the interface kernel runs on the
// side stream), then the gather and the tail.  With ev
// (profiling) the kernels run one after another with an event between each.
// The sweep's element-and-node launch for its tile shape.
inline void launch_sweep(const Dev<float> &D, const Mat<float> &M, cudaStream_t s) {
  const Sweep &S = *D.sweep;
  const int g = S.tiles_x * S.tiles_y * S.chunks;
  switch (S.tile) {
    case 0: launch_k(k_sweep<16, 8>, g, 128, s, D, M, S); break;
    case 1: launch_k(k_sweep<8, 8>, g, 64, s, D, M, S); break;
    default: launch_k(k_sweep<8, 4>, g, 32, s, D, M, S); break;
  }
}

template <typename T>
cudaError_t launch_pass(const Dev<T> &D, const Mat<T> &M, cudaStream_t s, int32_t gather_block,
                        cudaEvent_t *ev, cudaStream_t side, cudaEvent_t fork, cudaEvent_t join) {
  if constexpr (std::is_same<T, float>::value) {
    if (D.sweep != nullptr && D.sur_params == nullptr) {
      // contact, the sweep (elements and most nodes), the gather over the
      // boundary nodes, the tail; the interface event pair is empty
      if (ev) cudaEventRecord(ev[0], s);
      launch_k(k_contact<T>, grid_of(D.ns, kActRun), kActRun, s, D);
      if (ev) cudaEventRecord(ev[1], s);
      launch_sweep(D, M, s);
      if (ev) cudaEventRecord(ev[2], s);
      if (ev) cudaEventRecord(ev[3], s);
      if (D.sweep->n_bnodes > 0)
        launch_k(k_gather_list<T>, grid_of(D.sweep->n_bnodes, 256), 256, s, D, D.sweep->bnodes, D.sweep->n_bnodes);
      if (ev) cudaEventRecord(ev[4], s);
      launch_k(k_tail<T>, 1, 256, s, D);
      if (ev) cudaEventRecord(ev[5], s);
      return cudaGetLastError();
    }
  }
  bool mixed = D.hex_variant >= kMixedVariant && D.ipair == nullptr;
  if constexpr (std::is_same<T, float>::value) mixed = mixed && D.sur_params == nullptr;
  if (D.ipair != nullptr) {
    // interfaces as node pairs: no interface kernel; the interface event
    // pair is empty
    if (ev) cudaEventRecord(ev[0], s);
    launch_k(k_contact<T>, grid_of(D.ns, kActRun), kActRun, s, D);
    if (ev) cudaEventRecord(ev[1], s);
    launch_hex(D, M, s);
    if (ev) cudaEventRecord(ev[2], s);
    if (ev) cudaEventRecord(ev[3], s);
    if (D.pair_layer > 0)
      launch_k(k_gather_pairs_layered<T>, grid_of(D.nn, gather_block), gather_block, s, D, M);
    else
      launch_k(k_gather_pairs<T>, grid_of(D.nn, gather_block), gather_block, s, D, M);
    if (ev) cudaEventRecord(ev[4], s);
    launch_k(k_tail<T>, 1, 256, s, D);
    if (ev) cudaEventRecord(ev[5], s);
    return cudaGetLastError();
  }
  if (mixed) {
    // one launch for both element kinds; the interface event pair is empty
    if (ev) cudaEventRecord(ev[0], s);
    launch_k(k_contact<T>, grid_of(D.ns, kActRun), kActRun, s, D);
    if (ev) cudaEventRecord(ev[1], s);
    launch_elem(D, M, s);
    if (ev) cudaEventRecord(ev[2], s);
    if (ev) cudaEventRecord(ev[3], s);
    launch_k(k_gather<T>, grid_of(D.nn, gather_block), gather_block, s, D);
    if (ev) cudaEventRecord(ev[4], s);
    launch_k(k_tail<T>, 1, 256, s, D);
    if (ev) cudaEventRecord(ev[5], s);
    return cudaGetLastError();
  }
  const bool concurrent = side != nullptr && ev == nullptr && D.nc > 0;
  if (ev) cudaEventRecord(ev[0], s);
  launch_k(k_contact<T>, grid_of(D.ns, kActRun), kActRun, s, D);
  if (ev) cudaEventRecord(ev[1], s);
  if (concurrent) {
    cudaEventRecord(fork, s);
    cudaStreamWaitEvent(side, fork, 0);
    launch_coh(D, M, side, false);
    cudaEventRecord(join, side);
  }
  launch_hex(D, M, s);
  if (ev) cudaEventRecord(ev[2], s);
  if (!concurrent && D.nc > 0) launch_coh(D, M, s, true);
  if (concurrent) cudaStreamWaitEvent(s, join, 0);
  if (ev) cudaEventRecord(ev[3], s);
  launch_k(k_gather<T>, grid_of(D.nn, gather_block), gather_block, s, D);
  if (ev) cudaEventRecord(ev[4], s);
  launch_k(k_tail<T>, 1, 256, s, D);
  if (ev) cudaEventRecord(ev[5], s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pairs_to_elements(const Dev<T> &D, cudaStream_t s) {
  if (D.ipair == nullptr || D.nc == 0) return cudaSuccess;
  k_pairs_to_elements<T><<<grid_of(D.nc, 256), 256, 0, s>>>(D);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_damage_field(const Dev<T> &D, const Mat<T> &M, int which, float *out,
                                cudaStream_t s) {
  if (which == PDN_FIELD_DCOH) {
    const cudaError_t e = launch_pairs_to_elements(D, s);
    if (e != cudaSuccess) return e;
  }
  const int64_t n = (which == PDN_FIELD_DCOH) ? D.nc : D.nh;
  k_damage_field<T><<<grid_of(n, 128), 128, 0, s>>>(D, M, which, out);
  return cudaGetLastError();
}

cudaError_t launch_striker_init(Striker *S, StrikerStep *ss, double dt, cudaStream_t s) {
  k_striker_init<<<1, 1, 0, s>>>(S, ss, dt);
  return cudaGetLastError();
}

template cudaError_t launch_pass<float>(const Dev<float> &, const Mat<float> &, cudaStream_t, int32_t,
                                        cudaEvent_t *, cudaStream_t, cudaEvent_t, cudaEvent_t);
template cudaError_t launch_pass<double>(const Dev<double> &, const Mat<double> &, cudaStream_t, int32_t,
                                         cudaEvent_t *, cudaStream_t, cudaEvent_t, cudaEvent_t);
template cudaError_t launch_pairs_to_elements<float>(const Dev<float> &, cudaStream_t);
template cudaError_t launch_pairs_to_elements<double>(const Dev<double> &, cudaStream_t);
template cudaError_t launch_damage_field<float>(const Dev<float> &, const Mat<float> &, int, float *,
                                                cudaStream_t);
template cudaError_t launch_damage_field<double>(const Dev<double> &, const Mat<double> &, int, float *,
                                                 cudaStream_t);

}  // namespace pdn
