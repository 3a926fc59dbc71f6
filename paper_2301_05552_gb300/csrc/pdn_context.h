// Host-side context record of the GB300 explicit PDN impact step, shared by
// the translation units of the library (single plate: pdn_api.cu; batch of
// plates: pdn_batch.cu).  Not part of the public C ABI (pdn.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "pdn.h"
#include "pdn_internal.h"

namespace pdn {

// Arena of device memory: one cudaMalloc, 256-byte aligned sub-allocations.
struct Arena {
  char *base = nullptr;
  size_t size = 0, used = 0;
  template <typename P>
  P *take(size_t bytes) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + bytes;
    return base ? reinterpret_cast<P *>(base + off) : nullptr;
  }
};

}  // namespace pdn

struct pdn_ctx {
  int precision = PDN_FP32_FORCE;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t nn = 0, nh = 0, nc = 0, ns = 0;
  pdn::Arena arena;
  pdn::Dev<float> Df{};
  pdn::Dev<double> Dd{};
  pdn::Mat<float> Mf{};
  pdn::Mat<double> Md{};
  pdn::Ctl *ctl_dev = nullptr;
  pdn::Ctl *ctl_host = nullptr;  // pinned
  pdn::Striker *imp_dev = nullptr;
  float *field = nullptr;
  double dt = 0, dt_bulk = 0, dt_coh = 0, phi = 1;
  double grav[3] = {0, 0, 0};
  int max_repeats = 8;
  int64_t hist_cap = 0;
  bool has_imp = false;
  double imp_e0 = 0.0;                 // striker kinetic energy when set (energy ledger)
  double imp_c0[3] = {0.0, 0.0, 0.0};  // striker centre when set
  bool tuned = false;
  float tune_ms[12] = {};  // mean internal-force pass time per variant (autotuner)
  cudaGraphExec_t graph = nullptr;
  // side stream for the interface kernel, forked from and joined back into
  // the main stream inside every pass
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  std::vector<cudaEvent_t> prof_ev;
  float *sur_buf = nullptr;  // learned-law parameters and scaling (pdn_set_surrogate)
  pdn::Sweep sweep{};        // column sweep plan (Df.sweep points here when it is used)
  uint8_t *rmark_e_buf = nullptr, *rmark_n_buf = nullptr;  // repetition marks (separate kernels)
  bool full_repeat = false;  // PDN_FULL_REPEAT=1 at creation
  std::string err;

  // Pointers common to both precisions.
  template <typename F>
  void both(F &&f) {
    f(Df);
    f(Dd);
  }
};
