// pdn_internal_force_noalloc: the internal-force evaluation of
// pdn_internal_force for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a memory manager
// which owns all device memory (a framework's caching allocator, a fixed
// memory budget) and forbids allocations outside its control, or code that
// must not trigger the device-wide synchronisation of cudaMalloc/cudaFree in
// its steady state.  They cannot create a pdn context (pdn_init_mesh
// allocates).  This entry point takes every input and the output as caller
// buffers and keeps its working memory (mirrors, element forces, trial
// history, control block) in one file-scope __device__
// array of fixed size, so it allocates nothing.
//
// The scratch array lives on every device that loads this library until the
// process exits.  All calls share it and it keeps the last call's contents.
// Given inputs that meet the preconditions stated in pdn.h (in particular a
// csr_col that is a permutation of the element slots, as every node -> slot
// map is), each call rewrites every scratch byte it reads before reading it
// (control block, mirrors, slot positions, element forces, history when none
// is given), so nothing depends on what an earlier call left.  Calls whose
// work overlaps on the GPU (different streams or host threads on the same
// device) race on the array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "pdn.h"
#include "pdn_internal.h"

using namespace pdn;

namespace {

constexpr int kBlock = 256;

// Byte sizes of the scratch regions at the maxima, FP64 element precision
// (the larger of the two).
constexpr size_t kCtlBytes = 256;
constexpr size_t kNodeV4Bytes = (size_t)PDN_NOALLOC_MAX_NODES * 32;
constexpr size_t kHistBytes = (size_t)PDN_NOALLOC_MAX_HEX * 8 * 7 * 8;
constexpr size_t kFeBytes = (size_t)PDN_NOALLOC_MAX_HEX * 8 * 32;
constexpr size_t round256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffX4 = round256(kCtlBytes);
constexpr size_t kOffU4 = kOffX4 + round256(kNodeV4Bytes);
constexpr size_t kOffHin = kOffU4 + round256(kNodeV4Bytes);
constexpr size_t kOffHout = kOffHin + round256(kHistBytes);
constexpr size_t kOffFe = kOffHout + round256(kHistBytes);
constexpr size_t kPosBytes = (size_t)PDN_NOALLOC_MAX_HEX * 8 * sizeof(int32_t);
constexpr size_t kOffPos = kOffFe + round256(kFeBytes);
constexpr size_t kScratchBytes = kOffPos + round256(kPosBytes);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

template <typename T>
__global__ void k_noalloc_prepare(Ctl *ctl, const double *X, const double *d, typename Vec4T<T>::type *X4,
                                  typename Vec4T<T>::type *u4, int64_t nn, T *hist_pristine, int64_t per_field) {
  using V4 = typename Vec4T<T>::type;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    Ctl c{};
    c.mode = MODE_FORCES;
    c.dpar = 1;  // element kernels read node buffer dpar ^ 1 = 0
    c.hpar = 0;
    *ctl = c;
  }
  if (i < nn) {
    V4 x, u;
    x.x = (T)X[i];
    x.y = (T)X[nn + i];
    x.z = (T)X[2 * nn + i];
    x.w = T(0);
    u.x = (T)d[i];
    u.y = (T)d[nn + i];
    u.z = (T)d[2 * nn + i];
    u.w = T(0);
    X4[i] = x;
    u4[i] = u;
  }
  if (hist_pristine) {
    for (int64_t k = i; k < per_field * 7; k += (int64_t)gridDim.x * blockDim.x)
      hist_pristine[k] = (k < per_field * 4) ? T(1) : T(0);  // r_N = 1, plastic strain 0
  }
}

// CSR position of every element slot: the inverse of the caller's csr_col
// (the element kernel writes each nodal force at its node's CSR position).
__global__ void k_noalloc_pos(const int32_t *col, int32_t *pos, int64_t nnz) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nnz) return;
  const int32_t c = col[r];
  if (c >= 0 && c < nnz) pos[c] = (int32_t)r;
}

template <typename T>
cudaError_t run_noalloc(unsigned char *base, int64_t nn, int64_t nh, const int32_t *hex, const int8_t *ply,
                        const double *X, const double *d, const void *history, const int32_t *row,
                        const int32_t *col, const Mat<T> &M, double *f_int, cudaStream_t s) {
  using V4 = typename Vec4T<T>::type;
  Dev<T> D{};
  D.nn = nn;
  D.nh = nh;
  D.nc = 0;
  D.ns = 0;
  D.surf_base = -1;
  D.act_cnt = nullptr;
  D.hex = hex;
  D.coh = nullptr;
  D.ply = ply;
  D.X4 = reinterpret_cast<const V4 *>(base + kOffX4);
  D.row = row;
  D.col = col;
  V4 *u4 = reinterpret_cast<V4 *>(base + kOffU4);
  D.u4[0] = u4;
  D.u4[1] = u4;
  T *hin = history ? const_cast<T *>(reinterpret_cast<const T *>(history)) : reinterpret_cast<T *>(base + kOffHin);
  D.hist[0] = hin;
  D.hist[1] = reinterpret_cast<T *>(base + kOffHout);
  D.fe = reinterpret_cast<V4 *>(base + kOffFe);
  D.ctl = reinterpret_cast<Ctl *>(base);
  D.fout = f_int;
  const int64_t work = std::max<int64_t>(nn, 1);
  const int grid = (int)((work + kBlock - 1) / kBlock);
  k_noalloc_prepare<T><<<grid, kBlock, 0, s>>>(D.ctl, X, d, const_cast<V4 *>(D.X4), u4, nn,
                                                history ? nullptr : reinterpret_cast<T *>(base + kOffHin), nh * 8);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int32_t *pos = reinterpret_cast<int32_t *>(base + kOffPos);
  const int64_t nnz = nh * 8;
  k_noalloc_pos<<<(int)((nnz + kBlock - 1) / kBlock), kBlock, 0, s>>>(col, pos, nnz);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  D.pos = pos;
  return launch_pass<T>(D, M, s, kBlock, nullptr);
}

}  // namespace

namespace pdn {
void set_thread_error(const std::string &msg);
template <typename T>
int fill_mat_public(Mat<T> &M, const pdn_material &m, const double *ply_angle, int n_plies, int damage_on,
                    int plasticity_on, std::string &why);
}  // namespace pdn

extern "C" int pdn_internal_force_noalloc(int64_t n_nodes, int64_t n_hex, const int32_t *hex, const int8_t *ply_of_hex,
                                          const double *X, const double *d, const void *history,
                                          const int32_t *csr_row, const int32_t *csr_col, const pdn_material *mat,
                                          const double *ply_angle_deg, int32_t n_plies, int32_t precision,
                                          int32_t damage_on, int32_t plasticity_on, double *f_int, void *stream) {
  auto bad = [](int code, const std::string &m) {
    set_thread_error(m);
    return code;
  };
  if (n_nodes <= 0 || n_hex <= 0) return bad(PDN_E_ARG, "need n_nodes > 0 and n_hex > 0");
  if (n_hex > PDN_NOALLOC_MAX_HEX || n_nodes > PDN_NOALLOC_MAX_NODES)
    return bad(PDN_E_ARG, "pdn_internal_force_noalloc: mesh exceeds the static scratch (at most " +
                              std::to_string(PDN_NOALLOC_MAX_HEX) + " hexes and " +
                              std::to_string(PDN_NOALLOC_MAX_NODES) + " nodes)");
  if (!hex || !ply_of_hex || !X || !d || !csr_row || !csr_col || !mat || !ply_angle_deg || !f_int)
    return bad(PDN_E_ARG, "pdn_internal_force_noalloc: a required pointer is NULL");
  if (n_plies < 1 || n_plies > kMaxPlies) return bad(PDN_E_ARG, "n_plies must be in 1..64");
  if (precision != PDN_FP64 && precision != PDN_FP32_FORCE) return bad(PDN_E_ARG, "unknown precision");
  // Device address of the scratch array in the context current on this
  // thread.  Host code may not use the symbol itself as a device address.  It
  // is looked up on every call (a host-side query that allocates nothing):
  // after cudaDeviceReset, or under another context on the same device, the
  // module is loaded again and the array can sit at another address, so a
  // cached address could be stale.  The first call in a context loads the
  // module there; make it before any stream capture.
  void *addr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
  if (e != cudaSuccess || addr == nullptr)
    return bad(PDN_E_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
  std::string why;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == PDN_FP64) {
    Mat<double> M{};
    int rc = fill_mat_public(M, *mat, ply_angle_deg, n_plies, damage_on, plasticity_on, why);
    if (rc) return bad(rc, why);
    e = run_noalloc<double>((unsigned char *)addr, n_nodes, n_hex, hex, ply_of_hex, X, d, history, csr_row, csr_col,
                            M, f_int, s);
  } else {
    Mat<float> M{};
    int rc = fill_mat_public(M, *mat, ply_angle_deg, n_plies, damage_on, plasticity_on, why);
    if (rc) return bad(rc, why);
    e = run_noalloc<float>((unsigned char *)addr, n_nodes, n_hex, hex, ply_of_hex, X, d, history, csr_row, csr_col,
                           M, f_int, s);
  }
  if (e != cudaSuccess) return bad(PDN_E_CUDA, std::string("pdn_internal_force_noalloc launch: ") + cudaGetErrorString(e));
  return PDN_OK;
}
