// Batched persistent launch (include/pdn_batch.h): many independent plates
// advanced by one cooperative kernel that loops over passes; each pass walks
// four phases (contact, elements, gather, tails) over a work queue of tiles
// that spans all plates, with a bounded grid barrier between phases, or in the
// dataflow schedule with bounded per-plate dependency waits instead.
//
// Every tile applies the same per-item bodies as the per-pass kernels
// (pdn_items.cuh) to one plate, with that plate's state machine (Ctl), so a
// plate stepped in a batch follows the same arithmetic as pdn_step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pdn.h"
#include "pdn_batch.h"
#include "pdn_context.h"
#include "pdn_device.cuh"
#include "pdn_internal.h"
// the items run inside one persistent launch whose earlier phases write the
// state they read: no read-only data path for that state
#define PDN_ITEMS_IN_PERSISTENT_KERNEL 1
#include "pdn_items.cuh"

namespace pdn {
namespace {

using namespace detail;

enum TileKind : int32_t { TK_CONTACT = 0, TK_HEX = 1, TK_COH = 2, TK_GATHER = 3, TK_TAIL = 4 };

// The gather of one node of a plate: with the plate's interfaces as node
// pairs (Dev::ipair) the gather evaluates them too, and the plate has no
// interface tiles.
template <typename T>
__device__ __forceinline__ void batch_gather(const Dev<T> &D, const Mat<T> &M, int64_t i, int mode) {
  if (D.ipair == nullptr)
    gather_item(D, i, mode);
  else if (D.pair_layer > 0)
    gather_pair_layered_item(D, M, i, mode);
  else
    gather_pair_item(D, M, i, mode);
}
constexpr int kPhases = 4;          // contact, elements (hex + interface), gather, tails
constexpr int kBatchBlock = 128;    // threads per block (the hex register budget is set for 128)
constexpr int kBatchPasses = 32;    // passes per persistent launch (it stops early when all plates are done)
constexpr int kMaxCand = 16;

// Control words of one launch, zeroed before it starts.
struct BatchSync {
  uint32_t bar_count;   // blocks arrived at the current barrier
  uint32_t bar_gen;     // barrier generation
  uint32_t queue[kPhases];
  uint32_t live[2];     // plates still running after a pass (by pass parity)
  int32_t error;        // 1: a barrier or dependency wait gave up
  int32_t passes_done;
  uint32_t next;        // dataflow schedule: next queue position
  uint32_t pad[5];
};

template <typename T>
struct BatchArgs {
  const Dev<T> *D;       // [n_plates]
  const Mat<T> *M;       // [n_plates]
  const int4 *tiles;     // (plate, kind, begin, end) per tile, phase after phase
  int32_t tile_off[kPhases + 1];
  int32_t passes;
  int32_t stall_block;   // testing only: this block leaves at once (-1: none)
  BatchSync *sync;
  int64_t timeout_ns;
};

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of a cooperative launch (every block resident).  A block
// waits at most timeout_ns (or until another block has given up); it then
// raises sync->error and the barrier returns false, after which the caller
// returns from the kernel.
__device__ bool grid_barrier(BatchSync *sy, int64_t timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t *gen = &sy->bar_gen;
    volatile int32_t *err = &sy->error;
    const uint32_t g = *gen;
    __threadfence();
    const uint32_t arrived = atomicAdd(&sy->bar_count, 1u) + 1u;
    int ok = 1;
    if (arrived == gridDim.x) {
      atomicExch(&sy->bar_count, 0u);
      __threadfence();
      atomicAdd(&sy->bar_gen, 1u);
    } else {
      const uint64_t t0 = global_ns();
      while (*gen == g) {
        if (*err) {
          ok = 0;
          break;
        }
        if ((int64_t)(global_ns() - t0) > timeout_ns) {
          atomicExch(&sy->error, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ void copy_words(T *dst, const T *src) {
  static_assert(sizeof(T) % 4 == 0, "record of whole words");
  const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
  uint32_t *d = reinterpret_cast<uint32_t *>(dst);
  for (int k = threadIdx.x; k < (int)(sizeof(T) / 4); k += blockDim.x) d[k] = s[k];
}

template <typename T, int MINB>
__global__ void __launch_bounds__(kBatchBlock, MINB) k_batch(BatchArgs<T> A) {
  // the current tile's plate: its state pointers and constants
  __shared__ Dev<T> sD;
  __shared__ Mat<T> sM;
  __shared__ int s_tile;
  BatchSync *sy = A.sync;
  if ((int)blockIdx.x == A.stall_block) return;
  int cur = -1;
  int pass = 0;
  for (; pass < A.passes; ++pass) {
    for (int ph = 0; ph < kPhases; ++ph) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        // counters of later phases, untouched until the next barrier
        sy->queue[(ph + 1) % kPhases] = 0u;
        if (ph == 1) sy->live[(pass + 1) & 1] = 0u;
      }
      const int n = A.tile_off[ph + 1] - A.tile_off[ph];
      for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&sy->queue[ph], 1u);
        __syncthreads();
        const int t = s_tile;
        if (t >= n) break;  // uniform over the block
        const int4 tl = A.tiles[A.tile_off[ph] + t];
        if (tl.x != cur) {
          copy_words(&sD, &A.D[tl.x]);
          copy_words(&sM, &A.M[tl.x]);
          cur = tl.x;
        }
        __syncthreads();
        const int mode = *(volatile const int32_t *)&sD.ctl->mode;
        switch (tl.y) {
          case TK_CONTACT:
            if (mode == MODE_ADVANCE || mode == MODE_REPEAT)
              for (int64_t i = tl.z + threadIdx.x; i < tl.w; i += blockDim.x) contact_item(sD, i, mode);
            break;
          case TK_HEX:
            if (mode < MODE_DONE) {
              if (sD.all_boxes)
                for (int64_t i = tl.z + threadIdx.x; i < tl.w; i += blockDim.x) hex_item<T, true>(sD, sM, i, mode);
              else
                for (int64_t i = tl.z + threadIdx.x; i < tl.w; i += blockDim.x) hex_item<T, false>(sD, sM, i, mode);
            }
            break;
          case TK_COH:
            if (mode < MODE_DONE)
              for (int64_t i = tl.z + threadIdx.x; i < tl.w; i += blockDim.x)
                if (sD.all_flat_coh)
                  coh_item<T, true>(sD, sM, i, mode);
                else
                  coh_item<T, false>(sD, sM, i, mode);
            break;
          case TK_GATHER:
            if (mode < MODE_DONE)
              for (int64_t i = tl.z + threadIdx.x; i < tl.w; i += blockDim.x) batch_gather(sD, sM, i, mode);
            break;
          default:  // TK_TAIL
            if (mode < MODE_DONE) {
              tail_block(sD, mode);
              if (threadIdx.x == 0 && *(volatile const int32_t *)&sD.ctl->mode < MODE_DONE)
                atomicAdd(&sy->live[pass & 1], 1u);
            }
            break;
        }
        __syncthreads();  // s_tile and sD/sM are rewritten next
      }
      if (!grid_barrier(sy, A.timeout_ns)) return;
    }
    // every plate done or halted: the remaining passes would do nothing
    if (*(volatile uint32_t *)&sy->live[pass & 1] == 0u) {
      ++pass;
      break;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) sy->passes_done = pass;
}

// Dataflow schedule: one queue of (pass, phase, tile) positions, pass after
// pass in the phase order of the tile list.  A block takes the next position
// and waits (bounded in time) only until the previous phase of the same plate
// is complete: every tile of it for this pass, or the plate's tail of the
// previous pass for its contact tiles.  Completed tiles are counted per plate
// and phase.  Dependencies always sit earlier in the queue and every block is
// resident (cooperative launch), so the earliest unfinished tile can always
// run.  Phases of different plates overlap (one plate's gather with another
// plate's elements) instead of draining the GPU at a barrier.
template <typename T>
struct FlowArgs {
  const Dev<T> *D;
  const Mat<T> *M;
  const int4 *tiles;     // one pass: (plate, kind, begin, end), phase after phase
  const int4 *ntiles;    // [n_plates]: tiles of the contact, element and gather phases, 1 tail
  uint32_t *done;        // [n_plates][4] completed tiles in this launch
  int32_t *live;         // plates not yet done or halted
  BatchSync *sync;
  int32_t tiles_per_pass;
  int32_t passes;
  int64_t timeout_ns;
};

__device__ __forceinline__ int phase_of(int kind) {
  return kind == TK_CONTACT ? 0 : (kind == TK_GATHER ? 2 : (kind == TK_TAIL ? 3 : 1));
}

template <typename T, int MINB>
__global__ void __launch_bounds__(kBatchBlock, MINB) k_batch_flow(FlowArgs<T> A) {
  __shared__ Dev<T> sD;
  __shared__ Mat<T> sM;
  __shared__ int64_t s_g;
  __shared__ int s_go;
  BatchSync *sy = A.sync;
  const int64_t total = (int64_t)A.passes * A.tiles_per_pass;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0)
      s_g = (*(volatile int32_t *)A.live <= 0 || *(volatile int32_t *)&sy->error) ? total
                                                                                 : (int64_t)atomicAdd(&sy->next, 1u);
    __syncthreads();
    const int64_t g = s_g;
    if (g >= total) break;  // uniform over the block
    const int pass = (int)(g / A.tiles_per_pass);
    const int4 tl = A.tiles[g % A.tiles_per_pass];
    const int P = tl.x, ph = phase_of(tl.y);
    if (threadIdx.x == 0) {
      int go = 1;
      const Ctl *ctl = A.D[P].ctl;
      if (*(volatile const int32_t *)&ctl->mode < MODE_DONE) {
        const int4 nt = A.ntiles[P];
        int dep;
        uint32_t need;
        if (ph == 0 || (ph == 1 && nt.x == 0)) {
          dep = 3;  // the plate's tail of the previous pass
          need = (uint32_t)pass;
        } else {
          dep = ph - 1;
          need = (uint32_t)(pass + 1) * (uint32_t)(dep == 0 ? nt.x : (dep == 1 ? nt.y : nt.z));
        }
        volatile uint32_t *cnt = &A.done[P * 4 + dep];
        if (*cnt < need) {
          const uint64_t t0 = global_ns();
          while (*cnt < need) {
            if (*(volatile int32_t *)&sy->error) {
              go = 0;
              break;
            }
            if ((int64_t)(global_ns() - t0) > A.timeout_ns) {
              atomicExch(&sy->error, 1);
              go = 0;
              break;
            }
            __nanosleep(64);
          }
        }
        __threadfence();
      }
      s_go = go;
    }
    __syncthreads();
    if (!s_go) return;
    if (P != cur) {
      copy_words(&sD, &A.D[P]);
      copy_words(&sM, &A.M[P]);
      cur = P;
    }
    __syncthreads();
    const int mode = *(volatile const int32_t *)&sD.ctl->mode;
    switch (tl.y) {
      case TK_CONTACT:
        if (mode == MODE_ADVANCE || mode == MODE_REPEAT)
          for (int64_t i = tl.z + threadIdx.x; i < tl.w; i += blockDim.x) contact_item(sD, i, mode);
        break;
      case TK_HEX:
        if (mode < MODE_DONE) {
          if (sD.all_boxes)
            for (int64_t i = tl.z + threadIdx.x; i < tl.w; i += blockDim.x) hex_item<T, true>(sD, sM, i, mode);
          else
            for (int64_t i = tl.z + threadIdx.x; i < tl.w; i += blockDim.x) hex_item<T, false>(sD, sM, i, mode);
        }
        break;
      case TK_COH:
        if (mode < MODE_DONE)
          for (int64_t i = tl.z + threadIdx.x; i < tl.w; i += blockDim.x)
            if (sD.all_flat_coh)
              coh_item<T, true>(sD, sM, i, mode);
            else
              coh_item<T, false>(sD, sM, i, mode);
        break;
      case TK_GATHER:
        if (mode < MODE_DONE)
          for (int64_t i = tl.z + threadIdx.x; i < tl.w; i += blockDim.x) batch_gather(sD, sM, i, mode);
        break;
      default:  // TK_TAIL
        if (mode < MODE_DONE) {
          tail_block(sD, mode);
          if (threadIdx.x == 0) {
            atomicMax(&sy->passes_done, pass + 1);
            if (*(volatile const int32_t *)&sD.ctl->mode >= MODE_DONE) atomicSub(A.live, 1);
          }
        }
        break;
    }
    __syncthreads();  // every item of the tile is issued before it counts as done
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&A.done[P * 4 + ph], 1u);
    }
  }
}

// Mode and target of every plate (plates that halted keep their state).
template <typename T>
__global__ void k_batch_set_mode(const Dev<T> *D, int n, int32_t mode, int64_t nsteps, int32_t *live) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  Ctl *c = D[p].ctl;
  if (c->mode == MODE_HALT) return;
  c->mode = mode;
  c->target = c->step + nsteps;
  if (mode < MODE_DONE) atomicAdd(live, 1);
}

// Every plate's control block and the launch's sync words, for one copy.
template <typename T>
__global__ void k_batch_collect(const Dev<T> *D, int n, const BatchSync *sy, Ctl *out, BatchSync *sy_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) out[p] = *D[p].ctl;
  if (p == 0) *sy_out = *sy;
}

thread_local std::string g_batch_init_error;

}  // namespace
}  // namespace pdn

using namespace pdn;

struct pdn_batch {
  int n = 0;
  int precision = PDN_FP32_FORCE;
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<pdn_ctx *> plates;
  void *d_dev = nullptr;       // Dev<T>[n]
  void *d_mat = nullptr;       // Mat<T>[n]
  int4 *d_tiles = nullptr;
  size_t tiles_cap = 0;
  BatchSync *d_sync = nullptr;
  uint32_t *d_done = nullptr;  // dataflow: completed tiles per plate and phase [n][4]
  int32_t *d_live = nullptr;   // plates not yet done or halted
  int4 *d_ntiles = nullptr;    // tiles per plate of the contact, element, gather phases, 1 tail
  Ctl *d_ctl_all = nullptr;    // [n] followed by a BatchSync copy
  unsigned char *h_buf = nullptr;  // pinned copy of the same
  int32_t tile_off[kPhases + 1] = {0, 0, 0, 0, 0};
  // schedule
  int var = 0, bps = 0, tile_items = 256, grid = 0;
  int flow = 0;  // 0: grid barriers between phases, 1: dataflow dependencies
  bool tuned = false;
  cudaGraphExec_t graph = nullptr;
  bool graph_ok = false;
  int n_cand = 0;
  double tune_ms[kMaxCand] = {};
  int32_t tune_bps[kMaxCand] = {}, tune_tile[kMaxCand] = {}, tune_var[kMaxCand] = {}, tune_flow[kMaxCand] = {};
  int64_t launches = 0, passes = 0;
  int status = PDN_OK;
  std::string err;

  Ctl *h_ctl() { return reinterpret_cast<Ctl *>(h_buf); }
  BatchSync *h_sync() { return reinterpret_cast<BatchSync *>(h_buf + sizeof(Ctl) * (size_t)n); }
};

namespace {

int bfail(pdn_batch *b, int code, const std::string &msg) {
  if (b) b->err = msg;
  return code;
}

int bcuda(pdn_batch *b, cudaError_t e, const char *where) {
  return bfail(b, PDN_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PB_CU(call, where)                              \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return bcuda(b, _e, where);  \
  } while (0)

template <typename T, int MINB>
const void *kernel_of() {
  return reinterpret_cast<const void *>(&k_batch<T, MINB>);
}

template <typename T>
const void *kernel_for(int flow, int var) {
  if (flow)
    return var == 0 ? reinterpret_cast<const void *>(&k_batch_flow<T, 4>)
                    : reinterpret_cast<const void *>(&k_batch_flow<T, 1>);
  return var == 0 ? kernel_of<T, 4>() : kernel_of<T, 1>();
}

const void *kernel_ptr(const pdn_batch *b, int flow, int var) {
  return b->precision == PDN_FP64 ? kernel_for<double>(flow, var) : kernel_for<float>(flow, var);
}

// Interface elements a plate's element phase evaluates: none when its
// interfaces are node pairs (the gather evaluates them).
int64_t coh_items(const pdn_batch *b, int p) {
  const pdn_ctx *c = b->plates[p];
  const bool pairs = (b->precision == PDN_FP64 ? c->Dd.ipair : c->Df.ipair) != nullptr;
  return pairs ? 0 : c->nc;
}

// Tiles of every phase for a tile size; heavier element tiles (hexes) are
// queued before the interface tiles.
int build_tiles(pdn_batch *b, int tile_items) {
  std::vector<int4> t;
  auto add = [&](int p, int kind, int64_t n) {
    for (int64_t i = 0; i < n; i += tile_items)
      t.push_back(make_int4(p, kind, (int)i, (int)std::min<int64_t>(n, i + tile_items)));
  };
  b->tile_off[0] = 0;
  for (int p = 0; p < b->n; ++p) add(p, TK_CONTACT, b->plates[p]->ns);
  b->tile_off[1] = (int32_t)t.size();
  for (int p = 0; p < b->n; ++p) add(p, TK_HEX, b->plates[p]->nh);
  for (int p = 0; p < b->n; ++p) add(p, TK_COH, coh_items(b, p));
  b->tile_off[2] = (int32_t)t.size();
  for (int p = 0; p < b->n; ++p) add(p, TK_GATHER, b->plates[p]->nn);
  b->tile_off[3] = (int32_t)t.size();
  for (int p = 0; p < b->n; ++p) t.push_back(make_int4(p, TK_TAIL, 0, 0));
  b->tile_off[4] = (int32_t)t.size();
  std::vector<int4> nt(b->n);
  for (int p = 0; p < b->n; ++p) {
    auto tiles = [&](int64_t n) { return (int)((n + tile_items - 1) / tile_items); };
    const pdn_ctx *c = b->plates[p];
    nt[p] = make_int4(tiles(c->ns), tiles(c->nh) + tiles(coh_items(b, p)), tiles(c->nn), 1);
  }
  PB_CU(cudaMemcpy(b->d_ntiles, nt.data(), sizeof(int4) * b->n, cudaMemcpyHostToDevice), "upload tile counts");
  if (t.size() > b->tiles_cap) {
    if (b->d_tiles) cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    b->tiles_cap = 0;
    PB_CU(cudaMalloc(&b->d_tiles, sizeof(int4) * t.size()), "tile list");
    b->tiles_cap = t.size();
  }
  PB_CU(cudaMemcpy(b->d_tiles, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice), "upload tiles");
  b->tile_items = tile_items;
  return PDN_OK;
}

template <typename T>
BatchArgs<T> args_of(pdn_batch *b, int passes, int stall_block, int64_t timeout_ns) {
  BatchArgs<T> A{};
  A.D = reinterpret_cast<const Dev<T> *>(b->d_dev);
  A.M = reinterpret_cast<const Mat<T> *>(b->d_mat);
  A.tiles = b->d_tiles;
  for (int k = 0; k <= kPhases; ++k) A.tile_off[k] = b->tile_off[k];
  A.passes = passes;
  A.stall_block = stall_block;
  A.sync = b->d_sync;
  A.timeout_ns = timeout_ns;
  return A;
}

constexpr int64_t kBarrierTimeoutNs = 2000000000LL;  // 2 s: far beyond any phase of a pass

// One persistent launch (cooperative) of the chosen schedule.
template <typename T>
FlowArgs<T> flow_args_of(pdn_batch *b, int passes, int64_t timeout_ns) {
  FlowArgs<T> A{};
  A.D = reinterpret_cast<const Dev<T> *>(b->d_dev);
  A.M = reinterpret_cast<const Mat<T> *>(b->d_mat);
  A.tiles = b->d_tiles;
  A.ntiles = b->d_ntiles;
  A.done = b->d_done;
  A.live = b->d_live;
  A.sync = b->d_sync;
  A.tiles_per_pass = b->tile_off[kPhases];
  A.passes = passes;
  A.timeout_ns = timeout_ns;
  return A;
}

cudaError_t launch_batch(pdn_batch *b, int flow, int var, int grid, int passes, int stall_block,
                         int64_t timeout_ns) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBatchBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = b->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaError_t e = cudaMemsetAsync(b->d_sync, 0, sizeof(BatchSync), b->stream);
  if (e != cudaSuccess) return e;
  if (flow) {
    e = cudaMemsetAsync(b->d_done, 0, sizeof(uint32_t) * 4 * (size_t)b->n, b->stream);
    if (e != cudaSuccess) return e;
    if (b->precision == PDN_FP64) {
      FlowArgs<double> A = flow_args_of<double>(b, passes, timeout_ns);
      return var == 0 ? cudaLaunchKernelEx(&cfg, k_batch_flow<double, 4>, A)
                      : cudaLaunchKernelEx(&cfg, k_batch_flow<double, 1>, A);
    }
    FlowArgs<float> A = flow_args_of<float>(b, passes, timeout_ns);
    return var == 0 ? cudaLaunchKernelEx(&cfg, k_batch_flow<float, 4>, A)
                    : cudaLaunchKernelEx(&cfg, k_batch_flow<float, 1>, A);
  }
  if (b->precision == PDN_FP64) {
    BatchArgs<double> A = args_of<double>(b, passes, stall_block, timeout_ns);
    return var == 0 ? cudaLaunchKernelEx(&cfg, k_batch<double, 4>, A) : cudaLaunchKernelEx(&cfg, k_batch<double, 1>, A);
  }
  BatchArgs<float> A = args_of<float>(b, passes, stall_block, timeout_ns);
  return var == 0 ? cudaLaunchKernelEx(&cfg, k_batch<float, 4>, A) : cudaLaunchKernelEx(&cfg, k_batch<float, 1>, A);
}

int set_modes(pdn_batch *b, int32_t mode, int64_t nsteps) {
  const int g = (b->n + 127) / 128;
  PB_CU(cudaMemsetAsync(b->d_live, 0, sizeof(int32_t), b->stream), "live plates");
  if (b->precision == PDN_FP64)
    k_batch_set_mode<double><<<g, 128, 0, b->stream>>>(reinterpret_cast<const Dev<double> *>(b->d_dev), b->n, mode,
                                                       nsteps, b->d_live);
  else
    k_batch_set_mode<float><<<g, 128, 0, b->stream>>>(reinterpret_cast<const Dev<float> *>(b->d_dev), b->n, mode,
                                                      nsteps, b->d_live);
  PB_CU(cudaGetLastError(), "set modes");
  return PDN_OK;
}

// Copy every plate's control block and the sync words to the host.
int collect(pdn_batch *b) {
  const int g = (b->n + 127) / 128;
  BatchSync *sy_out = reinterpret_cast<BatchSync *>(b->d_ctl_all + b->n);
  if (b->precision == PDN_FP64)
    k_batch_collect<double><<<g, 128, 0, b->stream>>>(reinterpret_cast<const Dev<double> *>(b->d_dev), b->n, b->d_sync,
                                                      b->d_ctl_all, sy_out);
  else
    k_batch_collect<float><<<g, 128, 0, b->stream>>>(reinterpret_cast<const Dev<float> *>(b->d_dev), b->n, b->d_sync,
                                                     b->d_ctl_all, sy_out);
  PB_CU(cudaGetLastError(), "collect control blocks");
  PB_CU(cudaMemcpyAsync(b->h_buf, b->d_ctl_all, sizeof(Ctl) * (size_t)b->n + sizeof(BatchSync), cudaMemcpyDeviceToHost,
                        b->stream),
        "read control blocks");
  PB_CU(cudaStreamSynchronize(b->stream), "batch synchronize");
  return PDN_OK;
}

// Resident blocks per SM of a kernel variant (the cooperative limit).
int max_bps(pdn_batch *b, int flow, int var) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel_ptr(b, flow, var), kBatchBlock, 0) != cudaSuccess)
    return 0;
  return nb;
}

// Autotuner: time one internal-force pass (elements and gather of every
// plate; the committed state does not change) for each candidate schedule.
int autotune(pdn_batch *b) {
  if (b->tuned) return PDN_OK;
  struct Cand {
    int flow, var, bps, tile;
  };
  std::vector<Cand> cands;
  const int tiles[3] = {1024, 2048, 4096};
  // PDN_BATCH_SCHEDULE="s" or "s,r" restricts the candidates to schedule s
  // (0 barrier, 1 dataflow) and selects register variant r (default 0)
  int flow0 = 0, flow1 = 1, var0 = 0, var1 = 0;  // the 240-register variant only on request
  if (const char *fs = std::getenv("PDN_BATCH_SCHEDULE")) {
    if (fs[0] == '0' || fs[0] == '1') {
      flow0 = flow1 = fs[0] - '0';
      if (fs[1] == ',' && (fs[2] == '0' || fs[2] == '1')) var0 = var1 = fs[2] - '0';
    }
  }
  for (int flow = flow0; flow <= flow1; ++flow)
    for (int var = var0; var <= var1; ++var) {
      const int lim = max_bps(b, flow, var);
      for (int bps = std::min(lim, 4); bps >= 1; --bps) {
        if (var == 0 && bps < 3) continue;  // the 128-register kernel: 4 or 3 blocks per SM
        if (var == 1 && bps != 2) continue;  // the 240-register kernel: 2 blocks per SM
        for (int ti : tiles) cands.push_back({flow, var, bps, ti});
      }
    }
  if (cands.empty()) return bfail(b, PDN_E_CUDA, "no resident block fits the batch kernel");
  if ((int)cands.size() > kMaxCand) cands.resize(kMaxCand);
  cudaEvent_t e0, e1;
  PB_CU(cudaEventCreate(&e0), "tune event");
  PB_CU(cudaEventCreate(&e1), "tune event");
  double best = 1e30;
  Cand pick = cands[0];
  b->n_cand = 0;
  for (const Cand &c : cands) {
    int rc = build_tiles(b, c.tile);
    if (rc) return rc;
    const int grid = c.bps * b->sms;
    double sum = 0.0;
    const int reps = 3;
    for (int r = 0; r <= reps; ++r) {
      rc = set_modes(b, MODE_FORCES, 0);
      if (rc) return rc;
      PB_CU(cudaEventRecord(e0, b->stream), "tune record");
      PB_CU(launch_batch(b, c.flow, c.var, grid, 1, -1, kBarrierTimeoutNs), "tune launch");
      PB_CU(cudaEventRecord(e1, b->stream), "tune record");
      rc = collect(b);
      if (rc) return rc;
      if (b->h_sync()->error) {
        b->status = PDN_E_TIMEOUT;
        return bfail(b, PDN_E_TIMEOUT, "a grid barrier wait gave up while tuning");
      }
      float ms = 0.f;
      PB_CU(cudaEventElapsedTime(&ms, e0, e1), "tune time");
      if (r > 0) sum += ms;
    }
    const double ms = sum / reps;
    const int k = b->n_cand++;
    b->tune_ms[k] = ms;
    b->tune_bps[k] = c.bps;
    b->tune_tile[k] = c.tile;
    b->tune_var[k] = c.var;
    b->tune_flow[k] = c.flow;
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int rc = build_tiles(b, pick.tile);
  if (rc) return rc;
  b->var = pick.var;
  b->flow = pick.flow;
  b->bps = pick.bps;
  b->grid = pick.bps * b->sms;
  b->tuned = true;
  // the schedule as one graph: zero the sync words, then the persistent kernel
  cudaGraph_t g = nullptr;
  b->graph_ok = false;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    cudaError_t e = launch_batch(b, b->flow, b->var, b->grid, kBatchPasses, -1, kBarrierTimeoutNs);
    cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
    if (e == cudaSuccess && e2 == cudaSuccess && g && cudaGraphInstantiate(&b->graph, g, 0) == cudaSuccess)
      b->graph_ok = true;
    if (g) cudaGraphDestroy(g);
  }
  cudaGetLastError();  // a refused capture leaves no error behind: direct launches are used instead
  return PDN_OK;
}

template <typename T>
Dev<T> &dev_of(pdn_ctx *c);
template <>
Dev<float> &dev_of<float>(pdn_ctx *c) {
  return c->Df;
}
template <>
Dev<double> &dev_of<double>(pdn_ctx *c) {
  return c->Dd;
}
template <typename T>
Mat<T> &mat_of(pdn_ctx *c);
template <>
Mat<float> &mat_of<float>(pdn_ctx *c) {
  return c->Mf;
}
template <>
Mat<double> &mat_of<double>(pdn_ctx *c) {
  return c->Md;
}

template <typename T>
int upload_records(pdn_batch *b) {
  std::vector<Dev<T>> D(b->n);
  std::vector<Mat<T>> M(b->n);
  for (int p = 0; p < b->n; ++p) {
    D[p] = dev_of<T>(b->plates[p]);
    D[p].act_cnt = nullptr;  // the batch's contact tiles do not count: its tails scan the flags
    M[p] = mat_of<T>(b->plates[p]);
  }
  PB_CU(cudaMalloc(&b->d_dev, sizeof(Dev<T>) * b->n), "plate records");
  PB_CU(cudaMalloc(&b->d_mat, sizeof(Mat<T>) * b->n), "plate materials");
  PB_CU(cudaMemcpy(b->d_dev, D.data(), sizeof(Dev<T>) * b->n, cudaMemcpyHostToDevice), "upload plate records");
  PB_CU(cudaMemcpy(b->d_mat, M.data(), sizeof(Mat<T>) * b->n, cudaMemcpyHostToDevice), "upload plate materials");
  return PDN_OK;
}

const char *kind_of_status(int s) {
  switch (s) {
    case PDN_E_NONFINITE: return "non-finite acceleration or displacement";
    case PDN_E_RELEASE_LIMIT: return "contact release limit reached (Algorithm 2)";
    default: return "device error";
  }
}

}  // namespace

extern "C" {

const char *pdn_batch_last_error(const pdn_batch *b) {
  if (!b) return g_batch_init_error.c_str();
  return b->err.c_str();
}

void pdn_batch_destroy(pdn_batch *b) {
  if (!b) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (pdn_ctx *c : b->plates) pdn_destroy(c);
  if (b->d_dev) cudaFree(b->d_dev);
  if (b->d_mat) cudaFree(b->d_mat);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_sync) cudaFree(b->d_sync);
  if (b->d_done) cudaFree(b->d_done);
  if (b->d_live) cudaFree(b->d_live);
  if (b->d_ntiles) cudaFree(b->d_ntiles);
  if (b->d_ctl_all) cudaFree(b->d_ctl_all);
  if (b->h_buf) cudaFreeHost(b->h_buf);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  cudaSetDevice(prev);
  delete b;
}

static int pdn_batch_init_body(pdn_batch **out, int32_t n_plates, const pdn_mesh_desc *meshes, const pdn_material *mats,
                   const pdn_options *opt) {
  g_batch_init_error.clear();
  if (!out) {
    g_batch_init_error = "out is NULL";
    return PDN_E_ARG;
  }
  *out = nullptr;
  auto bad = [](int code, const std::string &m) {
    g_batch_init_error = m;
    return code;
  };
  if (n_plates < 1 || n_plates > 4096) return bad(PDN_E_ARG, "n_plates must be in 1..4096");
  if (!meshes || !mats || !opt) return bad(PDN_E_ARG, "meshes, mats and opt are required");
  if (opt->precision != PDN_FP64 && opt->precision != PDN_FP32_FORCE) return bad(PDN_E_ARG, "unknown precision");
  pdn_batch *b = new (std::nothrow) pdn_batch();
  if (!b) return bad(PDN_E_OOM, "host allocation failed");
  b->n = n_plates;
  b->precision = opt->precision;
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device);
  auto fail_init = [&](int code, const std::string &m) {
    pdn_batch_destroy(b);
    return bad(code, m);
  };
  if (!coop) return fail_init(PDN_E_CUDA, "the device does not support cooperative launches");
  if (opt->stream) {
    b->stream = (cudaStream_t)opt->stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
      return fail_init(PDN_E_CUDA, "stream create failed");
    b->own_stream = true;
  }
  pdn_options o = *opt;
  o.stream = b->stream;
  b->plates.assign(n_plates, nullptr);
  for (int p = 0; p < n_plates; ++p) {
    int rc = pdn_init_mesh(&b->plates[p], &meshes[p], &mats[p], &o);
    if (rc) return fail_init(rc, "plate " + std::to_string(p) + ": " + pdn_last_error(nullptr));
  }
  int rc = b->precision == PDN_FP64 ? upload_records<double>(b) : upload_records<float>(b);
  if (rc) return fail_init(rc, b->err);
  if (cudaMalloc(&b->d_sync, sizeof(BatchSync)) != cudaSuccess ||
      cudaMalloc(&b->d_done, sizeof(uint32_t) * 4 * (size_t)n_plates) != cudaSuccess ||
      cudaMalloc(&b->d_live, sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&b->d_ntiles, sizeof(int4) * (size_t)n_plates) != cudaSuccess ||
      cudaMalloc(&b->d_ctl_all, sizeof(Ctl) * (size_t)n_plates + sizeof(BatchSync)) != cudaSuccess ||
      cudaMallocHost(&b->h_buf, sizeof(Ctl) * (size_t)n_plates + sizeof(BatchSync)) != cudaSuccess)
    return fail_init(PDN_E_OOM, "batch control buffers");
  cudaMemset(b->d_sync, 0, sizeof(BatchSync));
  *out = b;
  return PDN_OK;
}

// No exception leaves the library: a failed host allocation is PDN_E_OOM.
int pdn_batch_init(pdn_batch **out, int32_t n_plates, const pdn_mesh_desc *meshes, const pdn_material *mats,
                   const pdn_options *opt) {
  try {
    return pdn_batch_init_body(out, n_plates, meshes, mats, opt);
  } catch (const std::bad_alloc &) {
    return PDN_E_OOM;
  } catch (...) {
    return PDN_E_ARG;
  }
}

pdn_ctx *pdn_batch_plate(pdn_batch *b, int32_t p) {
  if (!b || p < 0 || p >= b->n) return nullptr;
  return b->plates[p];
}

int pdn_batch_step(pdn_batch *b, int64_t nsteps) {
  if (!b) return PDN_E_ARG;
  if (b->status == PDN_E_TIMEOUT) return bfail(b, b->status, "batch unusable after a barrier timeout");
  if (nsteps < 0) return bfail(b, PDN_E_ARG, "nsteps < 0");
  for (int p = 0; p < b->n; ++p)
    if (!b->plates[p]->has_imp)
      return bfail(b, PDN_E_STATE, "plate " + std::to_string(p) + " has no striker (pdn_set_impactor)");
  int rc = collect(b);
  if (rc) return rc;
  for (int p = 0; p < b->n; ++p)
    if (b->h_ctl()[p].status)
      return bfail(b, b->h_ctl()[p].status, "plate " + std::to_string(p) + " halted earlier (sticky status)");
  if (nsteps == 0) return PDN_OK;
  rc = autotune(b);
  if (rc) return rc;
  std::vector<int64_t> target(b->n);
  for (int p = 0; p < b->n; ++p) target[p] = b->h_ctl()[p].step + nsteps;
  rc = set_modes(b, MODE_ADVANCE, nsteps);
  if (rc) return rc;
  int max_rep = 0;
  for (pdn_ctx *c : b->plates) max_rep = std::max(max_rep, c->max_repeats);
  const int64_t guard_max = (nsteps * (int64_t)(max_rep + 1)) / kBatchPasses + 4;
  for (int64_t guard = 0;; ++guard) {
    cudaError_t e = b->graph_ok ? cudaGraphLaunch(b->graph, b->stream)
                                : launch_batch(b, b->flow, b->var, b->grid, kBatchPasses, -1, kBarrierTimeoutNs);
    if (e != cudaSuccess) return bcuda(b, e, "batch launch");
    ++b->launches;
    rc = collect(b);
    if (rc) return rc;
    const BatchSync &sy = *b->h_sync();
    b->passes += sy.passes_done;
    if (sy.error) {
      b->status = PDN_E_TIMEOUT;
      return bfail(b, PDN_E_TIMEOUT, "a grid barrier or dependency wait gave up (bounded wait)");
    }
    bool done = true;
    for (int p = 0; p < b->n; ++p) {
      const Ctl &c = b->h_ctl()[p];
      if (c.status) return bfail(b, c.status, "plate " + std::to_string(p) + ": " + kind_of_status(c.status));
      if (c.step < target[p]) done = false;
    }
    if (done) break;
    if (guard > guard_max) return bfail(b, PDN_E_STATE, "batch step loop made no progress");
  }
  return PDN_OK;
}

int pdn_batch_get_info(pdn_batch *b, pdn_batch_info *info) {
  if (!b || !info) return PDN_E_ARG;
  std::memset(info, 0, sizeof(*info));
  info->n_plates = b->n;
  info->precision = b->precision;
  info->status = b->status;
  info->tuned = b->tuned ? 1 : 0;
  info->blocks_per_sm = b->bps;
  info->tile_items = b->tile_items;
  info->reg_variant = b->var;
  info->grid = b->grid;
  info->graph = b->graph_ok ? 1 : 0;
  info->n_candidates = b->n_cand;
  for (int k = 0; k < kPhases; ++k) info->n_tiles[k] = b->tile_off[k + 1] - b->tile_off[k];
  info->launches = b->launches;
  info->passes = b->passes;
  info->dataflow = b->flow;
  for (int k = 0; k < b->n_cand && k < 16; ++k) {
    info->tune_flow[k] = b->tune_flow[k];
    info->tune_ms[k] = b->tune_ms[k];
    info->tune_bps[k] = b->tune_bps[k];
    info->tune_tile[k] = b->tune_tile[k];
    info->tune_var[k] = b->tune_var[k];
  }
  return PDN_OK;
}

int pdn_batch_test_barrier_timeout(pdn_batch *b, double timeout_ms) {
  if (!b) return PDN_E_ARG;
  if (!(timeout_ms > 0.0) || timeout_ms > 10000.0) return bfail(b, PDN_E_ARG, "timeout_ms must be in (0, 10000]");
  if (b->status == PDN_E_TIMEOUT) return bfail(b, b->status, "batch unusable after a barrier timeout");
  int rc = collect(b);
  if (rc) return rc;
  for (int p = 0; p < b->n; ++p) {
    const int m = b->h_ctl()[p].mode;
    if (m != MODE_DONE && m != MODE_HALT) return bfail(b, PDN_E_STATE, "plates must be idle (after a completed step)");
  }
  if (b->tile_off[kPhases] == 0) {
    rc = build_tiles(b, b->tile_items);
    if (rc) return rc;
  }
  const int var = b->tuned ? b->var : 0;
  const int bps = std::max(1, std::min(2, max_bps(b, 0, var)));
  const int grid = b->tuned ? b->grid : bps * b->sms;
  if (grid < 2) return bfail(b, PDN_E_STATE, "the test needs at least two blocks");
  cudaError_t e = launch_batch(b, 0, var, grid, 1, 0, (int64_t)(timeout_ms * 1e6));
  if (e != cudaSuccess) return bcuda(b, e, "test launch");
  rc = collect(b);
  if (rc) return rc;
  return b->h_sync()->error ? bfail(b, PDN_E_TIMEOUT, "barrier wait gave up as designed") : PDN_OK;
}

}  // extern "C"
