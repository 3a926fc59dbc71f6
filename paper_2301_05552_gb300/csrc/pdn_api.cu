// Host runtime and C ABI (include/pdn.h) of the GB300 explicit PDN impact step.
//
// Set-up (lumped mass, stable steps, node-to-element CSR, constants) runs once
// on the host in pdn_init_mesh; every per-step operation runs in the kernels of
// pdn_kernels.cu.  pdn_step replays a captured CUDA graph of passes; the
// device-side state machine decides advance / repeat / halt, so the host only
// checks the committed step count once per call.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "pdn.h"
#include "pdn_context.h"
#include "pdn_internal.h"

using namespace pdn;

namespace {

thread_local std::string g_init_error;

constexpr int kGatherBlock = 256;
constexpr int kGraphPasses = 32;
constexpr int kProfilePasses = 64;


__global__ void k_fill_hist_float(float *h, int64_t per_field, int64_t n_init_fields) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < per_field * 7) h[i] = (i < per_field * n_init_fields) ? 1.0f : 0.0f;
}
__global__ void k_fill_hist_double(double *h, int64_t per_field, int64_t n_init_fields) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < per_field * 7) h[i] = (i < per_field * n_init_fields) ? 1.0 : 0.0;
}
template <typename V4>
__global__ void k_mirror(const double *d, V4 *u, int64_t nn) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nn) return;
  V4 o;
  o.x = d[j];
  o.y = d[nn + j];
  o.z = d[2 * nn + j];
  o.w = 0;
  u[j] = o;
}
__global__ void k_set_mode(Ctl *ctl, int32_t mode, int64_t target) {
  if (ctl->mode == MODE_HALT) return;
  ctl->mode = mode;
  ctl->target = target;
}

inline int grid_of(int64_t n, int b) {
  int64_t g = (n + b - 1) / b;
  return (int)(g < 1 ? 1 : g);
}

// NVTX range over a public call (named as the call), so that a profiler can
// select the kernels one call launched (ncu --nvtx --nvtx-include "name/").
// Header-only NVTX: without a profiler attached the push and pop are no-ops.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace


namespace {

int fail(pdn_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(pdn_ctx *c, cudaError_t e, const char *where) {
  return fail(c, PDN_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define PDN_CU(call, where)                      \
  do {                                           \
    cudaError_t _e = (call);                     \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, where); \
  } while (0)

cudaError_t run_pass(pdn_ctx *ctx, cudaEvent_t *ev) {
  if (ctx->precision == PDN_FP64)
    return launch_pass<double>(ctx->Dd, ctx->Md, ctx->stream, kGatherBlock, ev, ctx->side, ctx->fork, ctx->join);
  return launch_pass<float>(ctx->Df, ctx->Mf, ctx->stream, kGatherBlock, ev, ctx->side, ctx->fork, ctx->join);
}

cudaError_t build_graph(pdn_ctx *ctx) {
  if (ctx->graph) return cudaSuccess;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < kGraphPasses; ++k) {
    e = run_pass(ctx, nullptr);
    if (e != cudaSuccess) break;
  }
  cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return e;
  }
  e = cudaGraphInstantiate(&ctx->graph, g, 0);
  cudaGraphDestroy(g);
  return e;
}

// Launch n passes: whole graphs, then single passes for the remainder.
cudaError_t launch_passes(pdn_ctx *ctx, int64_t n) {
  cudaError_t e = build_graph(ctx);
  if (e != cudaSuccess) return e;
  for (int64_t k = 0; k + kGraphPasses <= n; k += kGraphPasses) {
    e = cudaGraphLaunch(ctx->graph, ctx->stream);
    if (e != cudaSuccess) return e;
  }
  for (int64_t k = 0; k < n % kGraphPasses; ++k) {
    e = run_pass(ctx, nullptr);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int read_ctl(pdn_ctx *ctx) {
  PDN_CU(cudaMemcpyAsync(ctx->ctl_host, ctx->ctl_dev, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream),
         "read control block");
  PDN_CU(cudaStreamSynchronize(ctx->stream), "stream synchronize");
  return PDN_OK;
}

int set_mode(pdn_ctx *ctx, int32_t mode, int64_t target) {
  k_set_mode<<<1, 1, 0, ctx->stream>>>(ctx->ctl_dev, mode, target);
  PDN_CU(cudaGetLastError(), "set mode");
  return PDN_OK;
}

// Acceleration of the installed state, without contact (momentum equation of
// Sec. 2.2.1): one pass in MODE_PRIME computes a = m^-1 (m g - f^i(d)) and
// the predictor of Eq. (TW) from it, then makes the installed state the
// committed one; history, step and time stay as they are.
static int prime_state(pdn_ctx *ctx) {
  int rc = set_mode(ctx, MODE_PRIME, ctx->ctl_host->step);
  if (rc) return rc;
  cudaError_t e = run_pass(ctx, nullptr);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "prime pass");
  rc = read_ctl(ctx);
  if (rc) return rc;
  if (ctx->ctl_host->status) return fail(ctx, ctx->ctl_host->status, "non-finite state installed");
  return PDN_OK;
}

// Material constants in precision T from the double-precision record.
template <typename T>
int fill_mat(Mat<T> &M, const pdn_material &m, const double *ply_angle, int n_plies, int damage_on,
             int plasticity_on, std::string &why) {
  double H[3][3] = {{1 / m.E1, -m.nu12 / m.E1, -m.nu13 / m.E1},
                    {-m.nu12 / m.E1, 1 / m.E2, -m.nu23 / m.E2},
                    {-m.nu13 / m.E1, -m.nu23 / m.E2, 1 / m.E3}};
  double det = H[0][0] * (H[1][1] * H[2][2] - H[1][2] * H[2][1]) - H[0][1] * (H[1][0] * H[2][2] - H[1][2] * H[2][0]) +
               H[0][2] * (H[1][0] * H[2][1] - H[1][1] * H[2][0]);
  if (!(det > 0)) {
    why = "elastic constants give a non positive-definite compliance";
    return PDN_E_ARG;
  }
  double C[3][3];
  C[0][0] = (H[1][1] * H[2][2] - H[1][2] * H[2][1]) / det;
  C[0][1] = (H[0][2] * H[2][1] - H[0][1] * H[2][2]) / det;
  C[0][2] = (H[0][1] * H[1][2] - H[0][2] * H[1][1]) / det;
  C[1][1] = (H[0][0] * H[2][2] - H[0][2] * H[2][0]) / det;
  C[1][2] = (H[0][2] * H[1][0] - H[0][0] * H[1][2]) / det;
  C[2][2] = (H[0][0] * H[1][1] - H[0][1] * H[1][0]) / det;
  M.C11 = (T)C[0][0];
  M.C12 = (T)C[0][1];
  M.C13 = (T)C[0][2];
  M.C22 = (T)C[1][1];
  M.C23 = (T)C[1][2];
  M.C33 = (T)C[2][2];
  M.G12 = (T)m.G12;
  M.G13 = (T)m.G13;
  M.G23 = (T)m.G23;
  M.h11 = (T)H[0][0];
  M.h22 = (T)H[1][1];
  M.h33 = (T)H[2][2];
  M.h12 = (T)H[0][1];
  M.h13 = (T)H[0][2];
  M.h23 = (T)H[1][2];
  M.E1 = (T)m.E1;
  M.E2 = (T)m.E2;
  M.XT = (T)m.XT;
  M.XC = (T)m.XC;
  M.YT = (T)m.YT;
  M.YC = (T)m.YC;
  M.SL = (T)m.SL;
  M.GXT = (T)m.GXT;
  M.GXC = (T)m.GXC;
  M.GYT = (T)m.GYT;
  M.GYC = (T)m.GYC;
  M.GSL = (T)m.GSL;
  const double a0 = m.alpha0_deg * M_PI / 180.0;
  const double ca = std::cos(a0), sa = std::sin(a0), t2 = std::tan(2.0 * a0);
  M.ca = (T)ca;
  M.sa = (T)sa;
  M.etaT = (T)(-1.0 / t2);
  M.ST = (T)(m.YC * ca * (sa + ca / t2));
  M.etaLc = (T)(-std::cos(2.0 * a0) / (m.YC * ca * ca));
  M.g = (T)(m.GYT / m.GSL);
  M.Sp = (T)m.Sp;
  M.Kp = (T)m.Kp;
  M.g1 = (T)(1.0 - m.GYT / m.GSL);
  M.iXC = (T)(1.0 / m.XC);
  {
    const double ST = m.YC * ca * (sa + ca / t2);
    M.iST2 = (T)(1.0 / (ST * ST));
  }
  M.kT = (T)(ca * (sa + ca / t2));  // ca (sa - etaT ca) with etaT = -1/tan(2 a0)
  M.KpG12 = (T)(m.Kp * m.G12);
  M.iG1Kp = (T)(1.0 / (m.G12 * (1.0 + m.Kp)));
  const double KI = m.KI;
  const double Ksh = KI * (m.GIc / m.GIIc) * (m.tauII / m.tauI) * (m.tauII / m.tauI);
  const double D3o = m.tauI / KI, D3c = 2.0 * m.GIc / m.tauI;
  const double Dsho = m.tauII / Ksh, Dshc = 2.0 * m.GIIc / m.tauII;
  M.KI = (T)KI;
  M.Ksh = (T)Ksh;
  M.KI_D3o2 = (T)(KI * D3o * D3o);
  M.Ksh_Dsho2 = (T)(Ksh * Dsho * Dsho);
  M.KI_D3oD3c = (T)(KI * D3o * D3c);
  M.Ksh_DshoDshc = (T)(Ksh * Dsho * Dshc);
  M.eta = (T)m.eta;
  M.onset_floor = (T)(0.999 * std::min(KI * D3o * D3o, Ksh * Dsho * Dsho));
  M.spread = (T)m.spread;
  M.seed = m.seed;
  M.damage_on = damage_on;
  M.plasticity_on = plasticity_on;
  for (int p = 0; p < kMaxPlies; ++p) {
    const double th = p < n_plies ? ply_angle[p] * M_PI / 180.0 : 0.0;
    M.ply_c[p] = (T)std::cos(th);
    M.ply_s[p] = (T)std::sin(th);
  }
  return PDN_OK;
}

// Hex8 geometry on the host (set-up only): det J and N_a at the 2x2x2 points.
// Shape functions and their natural derivatives at the 2x2x2 Gauss points,
// the same for every element: evaluated once.
struct HexGaussTables {
  double N[8][8];      // [point][node]
  double dN[8][8][3];  // [point][node][xi, eta, zeta]
};
const HexGaussTables &hex_gauss_tables() {
  static const HexGaussTables T = [] {
    static const int S[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};
    HexGaussTables t{};
    const double gp = 1.0 / std::sqrt(3.0);
    for (int g = 0; g < 8; ++g) {
      const double xi = S[g][0] * gp, et = S[g][1] * gp, ze = S[g][2] * gp;
      for (int a = 0; a < 8; ++a) {
        const double sx = S[a][0], sy = S[a][1], sz = S[a][2];
        t.dN[g][a][0] = 0.125 * sx * (1 + et * sy) * (1 + ze * sz);
        t.dN[g][a][1] = 0.125 * sy * (1 + xi * sx) * (1 + ze * sz);
        t.dN[g][a][2] = 0.125 * sz * (1 + xi * sx) * (1 + et * sy);
        t.N[g][a] = 0.125 * (1 + xi * sx) * (1 + et * sy) * (1 + ze * sz);
      }
    }
    return t;
  }();
  return T;
}

void hex_gauss(const double X[8][3], double detJ[8], double N[8][8]) {
  const HexGaussTables &T = hex_gauss_tables();
  for (int g = 0; g < 8; ++g) {
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < 8; ++a) {
      const double *dN = T.dN[g][a];
      N[g][a] = T.N[g][a];
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) J[i][k] += X[a][i] * dN[k];
    }
    detJ[g] = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
              J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  }
}

}  // namespace

namespace {

// Column sweep plan (pdn_internal.h, Sweep) of a layered plate: every hex
// layer and interface layer is a full nx x ny grid of columns numbered x
// fastest, nodes are numbered node layer by node layer (x fastest), element
// layer s joins node layers b and b + 1, and the layers chain from the bottom
// node layer to the top one.  Checked element by element; false (no sweep)
// for any other mesh.  The tile shape and the z-chunks give enough blocks to
// fill the GPU; bnodes lists the nodes on tile and chunk boundaries, which the
// gather over the list updates.
bool plan_sweep(int64_t nn, int64_t nh, int64_t nc, const int32_t *hex, const int32_t *coh, int n_sm, Sweep &S,
                std::vector<int32_t> &bnodes) {
  if (nh < 1) return false;
  const int64_t nxn = (int64_t)hex[3] - hex[0];
  const int64_t per_layer = (int64_t)hex[4] - hex[0];
  if (hex[0] != 0 || hex[1] != 1 || nxn < 2 || per_layer <= 0 || per_layer % nxn != 0) return false;
  const int64_t nx = nxn - 1, nyn = per_layer / nxn, ny = nyn - 1;
  const int64_t cols = nx * ny;
  if (ny < 1 || nh % cols != 0 || nc % cols != 0 || nn % per_layer != 0) return false;
  const int64_t n_hl = nh / cols, n_cl = nc / cols, n_nl = nn / per_layer;
  const int64_t n_st = n_hl + n_cl;
  if (n_st > kMaxStages || n_st != n_nl - 1) return false;
  // layer of each element layer; every element checked against the pattern
  std::vector<int32_t> stage_of_bottom(n_nl, -1);
  std::vector<int32_t> kind(n_st), base(n_st), bot(n_st);
  auto check_layer = [&](const int32_t *conn, int64_t first, int k, int kd) {
    const int64_t b = conn[8 * first] / per_layer;
    if (conn[8 * first] != b * per_layer || conn[8 * first + 4] != (b + 1) * per_layer) return false;
    for (int64_t r = 0; r < cols; ++r) {
      const int64_t i = r % nx, j = r / nx, n00 = j * nxn + i;
      const int32_t *q = conn + 8 * (first + r);
      const int64_t want[4] = {n00, n00 + 1, n00 + 1 + nxn, n00 + nxn};
      for (int a = 0; a < 4; ++a)
        if (q[a] != b * per_layer + want[a] || q[a + 4] != (b + 1) * per_layer + want[a]) return false;
    }
    if (b < 0 || b >= n_nl - 1 || stage_of_bottom[b] >= 0) return false;
    stage_of_bottom[b] = k;
    kind[k] = kd;
    base[k] = (int32_t)first;
    bot[k] = (int32_t)b;
    return true;
  };
  for (int64_t s = 0; s < n_hl; ++s)
    if (!check_layer(hex, s * cols, (int)s, 0)) return false;
  for (int64_t s = 0; s < n_cl; ++s)
    if (!check_layer(coh, s * cols, (int)(n_hl + s), 1)) return false;
  // stages bottom to top
  S = Sweep{};
  S.nx = (int32_t)nx;
  S.ny = (int32_t)ny;
  S.nxn = (int32_t)nxn;
  S.n_stages = (int32_t)n_st;
  S.per_layer = per_layer;
  for (int64_t L = 0; L < n_nl - 1; ++L) {
    const int k = stage_of_bottom[L];
    if (k < 0) return false;
    S.kind[L] = kind[k];
    S.base[L] = base[k];
    S.bot[L] = bot[k];
  }
  // tile shape: the largest whose tiles alone give every SM at least eight
  // blocks; z-chunks: enough blocks for about eight rounds of the resident
  // blocks (4, 8 or 16 per SM for the three shapes at 128 registers), so that
  // the last, partial round is a small part of the launch
  static const int TXS[3] = {16, 8, 8}, TYS[3] = {8, 8, 4};
  int t = 2;
  for (int c = 0; c < 3; ++c) {
    const int64_t tiles = ((nx + TXS[c] - 1) / TXS[c]) * ((ny + TYS[c] - 1) / TYS[c]);
    if (tiles >= (int64_t)8 * n_sm) {
      t = c;
      break;
    }
  }
  S.tile = t;
  S.tiles_x = (int32_t)((nx + TXS[t] - 1) / TXS[t]);
  S.tiles_y = (int32_t)((ny + TYS[t] - 1) / TYS[t]);
  const int64_t tiles = (int64_t)S.tiles_x * S.tiles_y;
  const int64_t resident = (int64_t)n_sm * (512 / (TXS[t] * TYS[t]));
  const int64_t want = 8 * resident;
  int64_t chunks = std::max<int64_t>(1, (want + tiles - 1) / tiles);
  chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, n_st / 8));  // at least eight stages per chunk
  S.chunk_len = (int32_t)((n_st + chunks - 1) / chunks);
  S.chunks = (int32_t)((n_st + S.chunk_len - 1) / S.chunk_len);
  // boundary nodes: tile-boundary columns of every node layer, and every
  // column of the node layers shared by two z-chunks
  std::vector<uint8_t> bcol((size_t)per_layer, 0);
  for (int64_t j = 0; j <= ny; ++j)
    for (int64_t i = 0; i <= nx; ++i)
      bcol[j * nxn + i] = ((i > 0 && i < nx && i % TXS[t] == 0) || (j > 0 && j < ny && j % TYS[t] == 0)) ? 1 : 0;
  bnodes.clear();
  for (int64_t L = 0; L < n_nl; ++L) {
    const bool shared = L % S.chunk_len == 0 && L > 0 && L < n_st;
    for (int64_t q = 0; q < per_layer; ++q)
      if (shared || bcol[q]) bnodes.push_back((int32_t)(L * per_layer + q));
  }
  return true;
}

}  // namespace

namespace {

// The history of an element (interface element) flagged pristine is not
// maintained in the buffers; it is the initial history (r = 1, plastic
// strain 0; interface r_D = 0), which is what is returned for it.
template <typename T>
static int get_history_t(pdn_ctx *ctx, const Dev<T> &D, T *hist, T *rD) {
  const int hb = ctx->ctl_host->hpar;
  const int64_t nh = ctx->nh, nc = ctx->nc;
  if (hist && nh > 0) {
    std::vector<uint8_t> pf(nh);
    PDN_CU(cudaMemcpy(hist, D.hist[hb], sizeof(T) * 7 * 8 * nh, cudaMemcpyDeviceToHost), "read history");
    PDN_CU(cudaMemcpy(pf.data(), D.pflag[hb], nh, cudaMemcpyDeviceToHost), "read history flags");
    for (int64_t e = 0; e < nh; ++e)
      if (pf[e])
        for (int f = 0; f < 7; ++f)
          for (int g = 0; g < 8; ++g) hist[((int64_t)f * 8 + g) * nh + e] = f < 4 ? T(1) : T(0);
  }
  if (rD && nc > 0) {
    std::vector<uint8_t> cf(nc);
    PDN_CU(launch_pairs_to_elements(D, ctx->stream), "interface thresholds from node pairs");
    PDN_CU(cudaStreamSynchronize(ctx->stream), "interface thresholds from node pairs");
    PDN_CU(cudaMemcpy(rD, D.rD[hb], sizeof(T) * 4 * nc, cudaMemcpyDeviceToHost), "read interface history");
    PDN_CU(cudaMemcpy(cf.data(), D.cflag[hb], nc, cudaMemcpyDeviceToHost), "read interface flags");
    for (int64_t e = 0; e < nc; ++e)
      if (cf[e])
        for (int p = 0; p < 4; ++p) rD[(int64_t)p * nc + e] = T(0);
  }
  return PDN_OK;
}

// A vector element type's allocator that leaves new elements uninitialised:
// the set-up's large arrays are written in full by the threads' chunks, so
// a serial zero fill (and its first-touch page faults on one core) is saved.
template <typename T>
struct NoInitAlloc : std::allocator<T> {
  using std::allocator<T>::allocator;
  template <typename U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  template <typename U>
  void construct(U *p) noexcept {
    ::new (static_cast<void *>(p)) U;
  }
  template <typename U, typename... A>
  void construct(U *p, A &&...a) {
    ::new (static_cast<void *>(p)) U(std::forward<A>(a)...);
  }
};
template <typename T>
using RawVec = std::vector<T, NoInitAlloc<T>>;

}  // namespace

extern "C" {

const char *pdn_last_error(const pdn_ctx *ctx) {
  if (!ctx) return g_init_error.c_str();
  return ctx->err.c_str();
}

void pdn_destroy(pdn_ctx *ctx) {
  if (!ctx) return;
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->arena.base) cudaFree(ctx->arena.base);
  if (ctx->sur_buf) cudaFree(ctx->sur_buf);
  if (ctx->ctl_host) cudaFreeHost(ctx->ctl_host);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->fork) cudaEventDestroy(ctx->fork);
  if (ctx->join) cudaEventDestroy(ctx->join);
  delete ctx;
}

static int pdn_init_mesh_body(pdn_ctx **out, const pdn_mesh_desc *mesh, const pdn_material *mat,
                              const pdn_options *opt) {
  g_init_error.clear();
  if (!out) {
    g_init_error = "out is NULL";
    return PDN_E_ARG;
  }
  *out = nullptr;
  auto bad = [](const std::string &m) {
    g_init_error = m;
    return PDN_E_ARG;
  };
  if (!mesh || !mat || !opt) return bad("mesh, material and options are required");
  const int64_t nn = mesh->n_nodes, nh = mesh->n_hex, nc = mesh->n_coh, ns = mesh->n_surf;
  if (nn <= 0 || nh <= 0 || nc < 0 || ns < 0) return bad("need n_nodes > 0, n_hex > 0, n_coh >= 0, n_surf >= 0");
  if (nn >= (int64_t)INT32_MAX || (nh + nc) * 8 >= (int64_t)INT32_MAX)
    return bad("mesh too large for 32-bit node/slot ids");
  if (!mesh->X || !mesh->hex || !mesh->ply_of_hex || !mesh->ply_angle_deg) return bad("X, hex, ply_of_hex, ply_angle_deg are required");
  if (nc > 0 && !mesh->coh) return bad("coh is NULL with n_coh > 0");
  if (ns > 0 && !mesh->surf) return bad("surf is NULL with n_surf > 0");
  if (mesh->n_plies < 1 || mesh->n_plies > kMaxPlies) return bad("n_plies must be in 1..64");
  if (opt->precision != PDN_FP64 && opt->precision != PDN_FP32_FORCE) return bad("unknown precision");
  // The loops over elements and nodes of the set-up run on the host's cores
  // in contiguous chunks; every result is the same for any number of threads
  // (per-thread partial results are combined in a fixed order).
  const int n_threads = std::max(1, std::min(16, (int)std::thread::hardware_concurrency()));
  auto parallel_chunks = [&](int64_t n, auto &&body) {
    const int nt = n < 4096 ? 1 : n_threads;
    const int64_t chunk = (n + nt - 1) / nt;
    if (nt == 1) {
      body(int64_t(0), n, 0);
      return;
    }
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) {
      const int64_t b = t * chunk, e = std::min<int64_t>(n, b + chunk);
      if (b >= e) continue;
      // a chunk whose thread cannot be started runs here (no exception may
      // leave the library)
      try {
        th.emplace_back([&, b, e, t]() { body(b, e, t); });
      } catch (...) {
        body(b, e, t);
      }
    }
    for (auto &x : th) x.join();
  };
  // index of the first item in [0, n) for which fails(i) holds, or -1
  auto first_failing = [&](int64_t n, auto &&fails) {
    std::vector<int64_t> first(n_threads, -1);
    parallel_chunks(n, [&](int64_t b, int64_t e, int t) {
      for (int64_t i = b; i < e; ++i)
        if (fails(i)) {
          first[t] = i;
          return;
        }
    });
    for (int t = 0; t < n_threads; ++t)
      if (first[t] >= 0) return first[t];
    return int64_t(-1);
  };
  if (first_failing(nh * 8, [&](int64_t k) { return mesh->hex[k] < 0 || mesh->hex[k] >= nn; }) >= 0)
    return bad("hex node id out of range");
  if (first_failing(nc * 8, [&](int64_t k) { return mesh->coh[k] < 0 || mesh->coh[k] >= nn; }) >= 0)
    return bad("interface node id out of range");
  if (first_failing(nh, [&](int64_t e) { return mesh->ply_of_hex[e] < 0 || mesh->ply_of_hex[e] >= mesh->n_plies; }) >= 0)
    return bad("ply id out of range");
  std::vector<int32_t> surf_of(nn, -1);
  for (int64_t s = 0; s < ns; ++s) {
    const int32_t j = mesh->surf[s];
    if (j < 0 || j >= nn) return bad("surface node id out of range");
    if (surf_of[j] >= 0) return bad("duplicate surface node id");
    surf_of[j] = (int32_t)s;
  }
  // a contact surface numbered as one ascending run of node ids
  int32_t surf_base = ns > 0 ? mesh->surf[0] : -1;
  for (int64_t s = 1; s < ns && surf_base >= 0; ++s)
    if (mesh->surf[s] != mesh->surf[0] + s) surf_base = -1;
  if (first_failing(nc, [&](int64_t c) {
        for (int a = 0; a < 4; ++a)
          for (int i = 0; i < 3; ++i)
            if (mesh->X[i * nn + mesh->coh[c * 8 + a]] != mesh->X[i * nn + mesh->coh[c * 8 + a + 4]]) return true;
        return false;
      }) >= 0)
    return bad("interface element faces must coincide in the reference configuration (zero thickness)");
  if (mesh->fixed)
    for (int64_t j = 0; j < nn; ++j)
      if (mesh->fixed[j] > 7) return bad("fixed entries must be constraint bits 0..7");
  const pdn_material &m = *mat;
  if (!(m.rho > 0 && m.E1 > 0 && m.E2 > 0 && m.E3 > 0 && m.G12 > 0 && m.G13 > 0 && m.G23 > 0))
    return bad("density and moduli must be positive");
  if (!(m.KI > 0 && m.tauI > 0 && m.tauII > 0 && m.GIc > 0 && m.GIIc > 0)) return bad("interface constants must be positive");

  pdn_ctx *ctx = new (std::nothrow) pdn_ctx();
  if (!ctx) return bad("host allocation failed");
  ctx->precision = opt->precision;
  ctx->nn = nn;
  ctx->nh = nh;
  ctx->nc = nc;
  ctx->ns = ns;
  ctx->phi = opt->phi == 0.0 ? 1.0 : opt->phi;
  for (int i = 0; i < 3; ++i) ctx->grav[i] = opt->gravity[i];
  ctx->max_repeats = opt->max_release_iters > 0 ? opt->max_release_iters : (opt->max_release_iters < 0 ? 0 : 8);
  ctx->hist_cap = opt->history_cap > 0 ? opt->history_cap : (int64_t)1 << 20;
  cudaGetDevice(&ctx->device);
  auto die = [&](int code, const std::string &msg) {
    g_init_error = msg;
    pdn_destroy(ctx);
    return code;
  };

  // --- set-up on the host: lumped mass, lengths, stable steps -------------
  // The element loop runs on the host's cores in contiguous chunks: each
  // element's nodal mass contributions (summed over its Gauss points) go to
  // its own slots, and the nodes sum them afterwards in element order, so the
  // result does not depend on the number of threads.
  RawVec<double> mass(nn);  // every entry written by the per-node sums below
  RawVec<double> vol(nh);
  RawVec<double> cm;  // [nh][8] each element's nodal mass contributions
  double cmax = 0.0;
  {
    Mat<double> tmp{};
    std::string why;
    int rc = fill_mat(tmp, m, mesh->ply_angle_deg, mesh->n_plies, opt->damage_on, opt->plasticity_on, why);
    if (rc) return die(rc, why);
    const double Cv[] = {tmp.C11, tmp.C12, tmp.C13, tmp.C22, tmp.C23, tmp.C33, tmp.G12, tmp.G13, tmp.G23};
    for (double c : Cv) cmax = std::max(cmax, std::fabs(c));
  }
  double dtb = INFINITY;
  const double sqrho = std::sqrt(m.rho / cmax);
  {
    cm.resize((size_t)nh * 8);
    std::vector<double> dtb_t(n_threads, INFINITY);
    std::vector<int64_t> bad_t(n_threads, -1);
    parallel_chunks(nh, [&](int64_t b, int64_t e1, int t) {
      for (int64_t e = b; e < e1; ++e) {
        double Xe[8][3], detJ[8], N[8][8];
        for (int a = 0; a < 8; ++a)
          for (int i = 0; i < 3; ++i) Xe[a][i] = mesh->X[i * nn + mesh->hex[e * 8 + a]];
        hex_gauss(Xe, detJ, N);
        double V = 0.0, s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int g = 0; g < 8; ++g) {
          if (!(detJ[g] > 0)) {
            bad_t[t] = e;
            return;
          }
          V += detJ[g];
          for (int a = 0; a < 8; ++a) s[a] += m.rho * N[g][a] * detJ[g];
        }
        for (int a = 0; a < 8; ++a) cm[e * 8 + a] = s[a];
        vol[e] = V;
        dtb_t[t] = std::min(dtb_t[t], std::cbrt(V) * sqrho);
      }
    });
    for (int t = 0; t < n_threads; ++t)
      if (bad_t[t] >= 0)
        return die(PDN_E_ARG, "hex with non-positive Jacobian (element " + std::to_string(bad_t[t]) + ")");
    for (int t = 0; t < n_threads; ++t) dtb = std::min(dtb, dtb_t[t]);
  }
  // Axis-aligned boxes whose corner coordinates coincide exactly in pairs in
  // the element precision: then the higher trilinear modes of X vanish
  // exactly in the kernel's butterfly and J is constant over the element.
  bool all_boxes = true;
  {
    auto is_box = [&](int64_t e, auto tag) {
      using T = decltype(tag);
      const int32_t *c = mesh->hex + e * 8;
      auto P = [&](int a, int i) { return (T)mesh->X[i * nn + c[a]]; };
      return P(0, 0) == P(3, 0) && P(0, 0) == P(4, 0) && P(0, 0) == P(7, 0) && P(1, 0) == P(2, 0) &&
             P(1, 0) == P(5, 0) && P(1, 0) == P(6, 0) && P(0, 1) == P(1, 1) && P(0, 1) == P(4, 1) &&
             P(0, 1) == P(5, 1) && P(2, 1) == P(3, 1) && P(2, 1) == P(6, 1) && P(2, 1) == P(7, 1) &&
             P(0, 2) == P(1, 2) && P(0, 2) == P(2, 2) && P(0, 2) == P(3, 2) && P(4, 2) == P(5, 2) &&
             P(4, 2) == P(6, 2) && P(4, 2) == P(7, 2);
    };
    all_boxes = first_failing(nh, [&](int64_t e) {
                  return !(opt->precision == PDN_FP64 ? is_box(e, double{}) : is_box(e, float{}));
                }) < 0;
  }
  bool all_flat_coh = true;
  {
    auto is_flat = [&](int64_t c, auto tag) {
      using T = decltype(tag);
      const int32_t *q = mesh->coh + c * 8;
      auto P = [&](int a, int i) { return (T)mesh->X[i * nn + q[a]]; };
      return P(0, 0) == P(3, 0) && P(1, 0) == P(2, 0) && P(0, 1) == P(1, 1) && P(2, 1) == P(3, 1) &&
             P(0, 2) == P(1, 2) && P(0, 2) == P(2, 2) && P(0, 2) == P(3, 2) && P(1, 0) > P(0, 0) &&
             P(3, 1) > P(0, 1);
    };
    all_flat_coh = first_failing(nc, [&](int64_t c) {
                     return !(opt->precision == PDN_FP64 ? is_flat(c, double{}) : is_flat(c, float{}));
                   }) < 0;
  }
  // node -> element-force slot CSR (hexes ascending, then interfaces
  // ascending).  Slot k of the entry list is 8 e + a for hexes and
  // 8 (n_hex + c) + a for interfaces, so each row is its slots in ascending
  // order: counted and filled at atomic cursors from the threads' chunks,
  // then every row sorted, which makes it independent of their interleaving.
  const int64_t n_ent = (nh + nc) * 8;
  std::vector<int32_t> row(nn + 1, 0);
  RawVec<int32_t> col((size_t)n_ent);
  auto node_of = [&](int64_t k) { return k < nh * 8 ? mesh->hex[k] : mesh->coh[k - nh * 8]; };
  parallel_chunks(n_ent, [&](int64_t b, int64_t e, int) {
    for (int64_t k = b; k < e; ++k) __atomic_fetch_add(&row[node_of(k) + 1], 1, __ATOMIC_RELAXED);
  });
  for (int64_t j = 0; j < nn; ++j) row[j + 1] += row[j];
  {
    std::vector<int32_t> fill(row.begin(), row.end() - 1);
    parallel_chunks(n_ent, [&](int64_t b, int64_t e, int) {
      for (int64_t k = b; k < e; ++k) col[__atomic_fetch_add(&fill[node_of(k)], 1, __ATOMIC_RELAXED)] = (int32_t)k;
    });
  }
  parallel_chunks(nn, [&](int64_t b, int64_t e, int) {
    for (int64_t j = b; j < e; ++j) std::sort(col.begin() + row[j], col.begin() + row[j + 1]);
  });
  // lumped mass: each node sums its hexes' contributions in element order
  // (its CSR row), the same sum for any number of threads
  parallel_chunks(nn, [&](int64_t b, int64_t e, int) {
    for (int64_t j = b; j < e; ++j) {
      double mj = 0.0;
      for (int32_t r = row[j]; r < row[j + 1]; ++r)
        if (col[r] < nh * 8) mj += cm[col[r]];
      mass[j] = mj;
    }
  });
  RawVec<double>().swap(cm);
  // Slots of the element forces.  When no node has more than eight
  // incident elements (every structured laminate: 8 hexes inside a layer,
  // 4 hexes and 4 interfaces on an interface layer), node j owns slots
  // 8 j .. 8 j + 7, filled in CSR order and zero-padded: the gather then
  // reads a node's slots in the same load round as its state, without the
  // CSR row first, and sums them in the same order.  Otherwise the slots are
  // the CSR positions.
  const bool ell = first_failing(nn, [&](int64_t j) { return row[j + 1] - row[j] > 8; }) < 0 && 8 * nn <= INT32_MAX;
  const int64_t n_slots = ell ? 8 * nn : 8 * (nh + nc);
  RawVec<int32_t> pos(col.size());
  parallel_chunks(nn, [&](int64_t b, int64_t e, int) {
    for (int64_t j = b; j < e; ++j)
      for (int32_t r = row[j]; r < row[j + 1]; ++r) pos[col[r]] = ell ? (int32_t)(8 * j + (r - row[j])) : r;
  });
  std::vector<uint32_t> rank(ell ? nh + nc : 0);
  if (ell) {
    parallel_chunks(nh + nc, [&](int64_t b, int64_t e1, int) {
      for (int64_t e = b; e < e1; ++e) {
        const int32_t *cn = e < nh ? mesh->hex + e * 8 : mesh->coh + (e - nh) * 8;
        uint32_t w = 0;
        for (int a = 0; a < 8; ++a) w |= (uint32_t)(pos[e * 8 + a] - 8 * cn[a]) << (3 * a);
        rank[e] = w;
      }
    });
  }
  // column sweep (FP32 box hexes, flat interfaces, eight slots per node),
  // planned only on request (PDN_SWEEP=1, read here): it measured slower
  // than the separate kernels (400x600x32 plate: 1.59 against 1.29 ms per
  // step), and a planned sweep keeps the interface elements
  Sweep sweep{};
  std::vector<int32_t> bnodes;
  bool sweep_on = false;
  {
    const char *sv = std::getenv("PDN_SWEEP");
    const bool allowed = sv && sv[0] == '1' && sv[1] == '\0';
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n_sm < 1) {
      cudaGetLastError();
      n_sm = 1;
    }
    if (allowed && opt->precision == PDN_FP32_FORCE && all_boxes && all_flat_coh && ell)
      sweep_on = plan_sweep(nn, nh, nc, mesh->hex, mesh->coh, n_sm, sweep, bnodes);
  }
  // Interfaces as node pairs (flat interfaces, eight slots per node, no
  // column sweep): per node its partner across the interface, the counts of
  // its incident hexes and interface elements, and the area weights of the
  // latter in CSR order, in the element precision and with the interface
  // kernel's arithmetic.  The pairing must be mutual and the same for every
  // incident interface element of a node.  PDN_COH_PAIRS=0, read here, keeps
  // the interface elements.
  bool pairs_on = false, pairs_uniform = true;
  int32_t pair_layer = 0;
  uint64_t pair_mask[2][2] = {{0, 0}, {0, 0}};
  bool slot_compact = false;
  int32_t layer_off[kMaxPairLayers] = {};  // compact slots: first slot of layer l minus l L width(l)
  std::vector<int2> ipair;
  std::vector<char> iw;  // [nn] 4 weights of the element precision
  double coh_w = 0.0;
  {
    const char *pv = std::getenv("PDN_COH_PAIRS");
    const bool allowed = !(pv && pv[0] == '0' && pv[1] == '\0');
    auto build_pairs = [&](auto tag) -> bool {
      using T = decltype(tag);
      ipair.assign(nn, int2{-1, 0});
      iw.assign(sizeof(T) * 4 * nn, 0);
      T *wn = reinterpret_cast<T *>(iw.data());
      // per thread: the first weight it met, whether all its weights equal
      // it, whether all its nodes qualify
      std::vector<T> w_first(n_threads, T(0));
      std::vector<char> has_w(n_threads, 0), same_w(n_threads, 1), ok_t(n_threads, 1);
      parallel_chunks(nn, [&](int64_t b, int64_t e, int t) {
        for (int64_t j = b; j < e; ++j) {
          int nhx = 0, kc = 0, top = 0;
          int32_t partner = -1;
          for (int32_t r = row[j]; r < row[j + 1]; ++r) {
            const int32_t slot = col[r];
            if (slot < nh * 8) {
              if (kc) {  // hexes first (CSR order)
                ok_t[t] = 0;
                return;
              }
              ++nhx;
              continue;
            }
            const int64_t c = slot / 8 - nh;
            const int a = slot % 8;
            const int32_t *q = mesh->coh + c * 8;
            const int32_t pj = q[a ^ 4];
            const int tp = a >= 4 ? 1 : 0;
            if (kc == 0) {
              partner = pj;
              top = tp;
            } else if (pj != partner || tp != top || kc == 4) {
              ok_t[t] = 0;
              return;
            }
            const T x0 = (T)mesh->X[q[0]], x2 = (T)mesh->X[q[2]];
            const T y0 = (T)mesh->X[nn + q[0]], y2 = (T)mesh->X[nn + q[2]];
            const T w = T(0.25) * (x2 - x0) * (y2 - y0);
            wn[4 * j + kc] = w;
            if (!has_w[t]) {
              w_first[t] = w;
              has_w[t] = 1;
            } else if (w != w_first[t]) {
              same_w[t] = 0;
            }
            ++kc;
          }
          if (nhx > 8 || partner == (int32_t)j) {
            ok_t[t] = 0;
            return;
          }
          ipair[j] = int2{partner, kc | (top << 3) | (nhx << 4)};
        }
      });
      T w0 = T(0);
      bool first = true;
      for (int t = 0; t < n_threads; ++t) {
        if (!ok_t[t]) return false;
        if (!has_w[t]) continue;
        if (!same_w[t]) pairs_uniform = false;
        if (first) {
          w0 = w_first[t];
          first = false;
        } else if (w_first[t] != w0) {
          pairs_uniform = false;
        }
      }
      if (first_failing(nn, [&](int64_t j) {
            const int32_t pj = ipair[j].x;
            return pj >= 0 && (ipair[pj].x != (int32_t)j || ((ipair[pj].y ^ ipair[j].y) & 8) == 0);
          }) >= 0)
        return false;
      coh_w = (double)w0;
      return true;
    };
    if (allowed && nc > 0 && all_flat_coh && ell && !sweep_on)
      pairs_on = opt->precision == PDN_FP64 ? build_pairs(double{}) : build_pairs(float{});
    // a layered numbering: blocks of L consecutive ids are node layers, and
    // every interface node's partner is the same position one layer up (lower
    // side) or down (upper side), with at most four hexes per interface node
    if (pairs_on) {
      int64_t L = 0;
      for (int64_t j = 0; j < nn && L == 0; ++j)
        if (ipair[j].x >= 0) L = std::llabs((int64_t)ipair[j].x - j);
      bool ok = L > 0 && nn % L == 0 && nn / L <= kMaxPairLayers;
      if (ok) {
        // each node against its layer's kind (that of the layer's first node)
        auto kind_of = [&](int64_t j) { return ipair[j].x < 0 ? 0 : (((ipair[j].y >> 3) & 1) ? 2 : 1); };
        ok = first_failing(nn, [&](int64_t j) {
               const int kind = kind_of((j / L) * L);
               const int2 ip = ipair[j];
               if (kind == 0) return ip.x >= 0;
               return !(ip.x == (kind == 1 ? j + L : j - L) && ((ip.y >> 3) & 1) == (kind == 2 ? 1 : 0) &&
                        ((ip.y >> 4) & 15) <= 4);
             }) < 0;
        for (int64_t l = 0; ok && l < nn / L; ++l) {
          const int kind = kind_of(l * L);
          if (kind) pair_mask[kind - 1][l >> 6] |= uint64_t(1) << (l & 63);
        }
      }
      if (ok) pair_layer = (int32_t)L;
    }
    // compact force slots (4 per interface-layer node): every hex's lower
    // face in one node layer and its upper face in one; PDN_SLOTS_COMPACT=0,
    // read here, keeps 8 slots per node
    if (pair_layer > 0) {
      const char *cv = std::getenv("PDN_SLOTS_COMPACT");
      const bool want = !(cv && cv[0] == '0' && cv[1] == '\0');
      const int64_t L = pair_layer;
      auto faces_in_layers = [&](int64_t e) {
        const int32_t *q = mesh->hex + e * 8;
        return q[0] / L == q[1] / L && q[0] / L == q[2] / L && q[0] / L == q[3] / L && q[4] / L == q[5] / L &&
               q[4] / L == q[6] / L && q[4] / L == q[7] / L;
      };
      // (node ids below 2^24, exact in FP32, for the device's layer lookup)
      slot_compact = want && nn <= (int64_t(1) << 24) &&
                     first_failing(nh, [&](int64_t e) { return !faces_in_layers(e); }) < 0;
      if (slot_compact) {
        // slot positions of the generic element path in the compact layout
        const uint64_t m0 = pair_mask[0][0] | pair_mask[1][0], m1 = pair_mask[0][1] | pair_mask[1][1];
        auto base_of = [&](int64_t j) {
          const int64_t lay = j / L;
          const int below = lay < 64 ? __builtin_popcountll(m0 & ((1ull << lay) - 1ull))
                                     : __builtin_popcountll(m0) + __builtin_popcountll(m1 & ((1ull << (lay - 64)) - 1ull));
          const bool pair = (((lay < 64 ? m0 : m1) >> (lay & 63)) & 1) != 0;
          return L * (8 * lay - 4 * (int64_t)below) + (j - lay * L) * (pair ? 4 : 8);
        };
        parallel_chunks(nn, [&](int64_t b, int64_t e, int) {
          for (int64_t j = b; j < e; ++j)
            for (int32_t r = row[j]; r < row[j + 1]; ++r) pos[col[r]] = (int32_t)(base_of(j) + (r - row[j]));
        });
        for (int64_t l = 0; l < nn / L; ++l) {
          const bool pair = (((l < 64 ? m0 : m1) >> (l & 63)) & 1) != 0;
          layer_off[l] = (int32_t)(base_of(l * L) - l * L * (pair ? 4 : 8));
        }
      }
    }
    if (!pairs_on) {
      std::vector<int2>().swap(ipair);
      std::vector<char>().swap(iw);
      pairs_uniform = true;
    } else if (pairs_uniform) {
      std::vector<char>().swap(iw);
    }
  }
  // interface stable step: rho_bar = rho * h, h = volume / face area of the
  // thinner hex sharing a face with the interface element
  double dtc = INFINITY;
  std::vector<double> dtc_t(n_threads, INFINITY);
  parallel_chunks(nc, [&](int64_t c0, int64_t c1, int t) {
  for (int64_t c = c0; c < c1; ++c) {
    double hmin = INFINITY;
    for (int side = 0; side < 2; ++side) {
      const int32_t *fn = mesh->coh + c * 8 + side * 4;
      for (int32_t r = row[fn[0]]; r < row[fn[0] + 1]; ++r) {
        const int32_t slot = col[r];
        if (slot >= nh * 8) break;
        const int64_t e = slot / 8;
        int hit = 0;
        for (int k = 0; k < 4; ++k)
          for (int a = 0; a < 8; ++a)
            if (mesh->hex[e * 8 + a] == fn[k]) {
              ++hit;
              break;
            }
        if (hit != 4) continue;
        double p[4][3];
        for (int k = 0; k < 4; ++k)
          for (int i = 0; i < 3; ++i) p[k][i] = mesh->X[i * nn + fn[k]];
        double u1[3], u2[3];
        for (int i = 0; i < 3; ++i) {
          u1[i] = p[2][i] - p[0][i];
          u2[i] = p[3][i] - p[1][i];
        }
        const double cr0 = u1[1] * u2[2] - u1[2] * u2[1], cr1 = u1[2] * u2[0] - u1[0] * u2[2],
                     cr2 = u1[0] * u2[1] - u1[1] * u2[0];
        const double A = 0.5 * std::sqrt(cr0 * cr0 + cr1 * cr1 + cr2 * cr2);
        hmin = std::min(hmin, vol[e] / A);
      }
    }
    if (std::isfinite(hmin)) dtc_t[t] = std::min(dtc_t[t], std::sqrt(m.rho * hmin / m.KI));
  }
  });
  for (int t = 0; t < n_threads; ++t) dtc = std::min(dtc, dtc_t[t]);
  ctx->dt_bulk = dtb;
  ctx->dt_coh = dtc;
  const double safety = opt->dt_safety > 0 ? opt->dt_safety : 0.5;
  ctx->dt = opt->dt > 0 ? opt->dt : safety * std::min(dtb, dtc);
  if (!(ctx->dt > 0) || !std::isfinite(ctx->dt)) return die(PDN_E_UNSTABLE, "no finite stable time step");
  {
    const int64_t j = first_failing(nn, [&](int64_t k) { return !(mass[k] > 0); });
    if (j >= 0) return die(PDN_E_ARG, "node " + std::to_string(j) + " has no mass (not in any hex)");
  }

  // --- device arena ---------------------------------------------------------
  const bool fp64 = ctx->precision == PDN_FP64;
  const size_t ts = fp64 ? 8 : 4;
  struct Ptrs {
    int32_t *hex, *coh, *surf, *surf_of, *row, *col, *pos, *act_cnt, *bnodes;
    int2 *ipair;
    char *iw, *rDn[2];
    uint32_t *rank;
    int8_t *ply;
    char *X4, *imass, *u4[2], *hist[2], *rD[2], *fe;
    uint8_t *nflag, *act[2], *rel, *rmark_e, *rmark_n, *pflag[2], *cflag[2];
    double *Xs, *mass, *d[2], *v[2], *nrm, *lam, *trial, *fhist, *fout;
    Ctl *ctl;
    Striker *imp;
    StrikerStep *imp_step;
    float *field;
  } P{};
  const int64_t ns1 = std::max<int64_t>(ns, 1), nc1 = std::max<int64_t>(nc, 1);
  // One layout function for both the sizing pass (base == nullptr) and the
  // real pass, so the two cannot diverge.
  auto layout = [&](Arena &A) {
    P.hex = A.take<int32_t>(sizeof(int32_t) * nh * 8);
    P.coh = A.take<int32_t>(sizeof(int32_t) * nc1 * 8);
    P.ply = A.take<int8_t>((nh + 15) & ~int64_t(15));  // whole 16-byte words (read as words)
    P.X4 = A.take<char>(ts * 4 * nn);
    P.nflag = A.take<uint8_t>((nn + 3) & ~int64_t(3));  // whole 4-byte words (the sweep copies words)
    P.surf = A.take<int32_t>(sizeof(int32_t) * ns1);
    P.surf_of = A.take<int32_t>(sizeof(int32_t) * nn);
    P.Xs = A.take<double>(sizeof(double) * 3 * ns1);
    P.row = A.take<int32_t>(sizeof(int32_t) * (nn + 1));
    P.col = A.take<int32_t>(sizeof(int32_t) * (nh + nc) * 8);
    P.pos = A.take<int32_t>(sizeof(int32_t) * (nh + nc) * 8);
    P.rank = A.take<uint32_t>(sizeof(uint32_t) * std::max<int64_t>(rank.size(), 1));
    P.mass = A.take<double>(sizeof(double) * nn);
    P.imass = A.take<char>(ts * nn);
    for (int b = 0; b < 2; ++b) {
      P.d[b] = A.take<double>(sizeof(double) * 3 * nn);
      P.v[b] = A.take<double>(sizeof(double) * 3 * nn);
      P.u4[b] = A.take<char>(ts * 4 * nn);
      P.hist[b] = A.take<char>(ts * 7 * 8 * nh);
      P.rD[b] = A.take<char>(ts * 4 * nc1);
      P.act[b] = A.take<uint8_t>((ns1 + 15) & ~int64_t(15));  // read in 16-byte words by the tail
      P.pflag[b] = A.take<uint8_t>((nh + 15) & ~int64_t(15));
      P.cflag[b] = A.take<uint8_t>(nc1);
    }
    P.fe = A.take<char>(ts * 4 * n_slots);
    P.rel = A.take<uint8_t>(ns1);
    P.act_cnt = A.take<int32_t>(sizeof(int32_t) * ((ns1 + kActRun - 1) / kActRun));
    P.rmark_e = A.take<uint8_t>(nh + nc);
    P.rmark_n = A.take<uint8_t>(nn);
    P.nrm = A.take<double>(sizeof(double) * 3 * ns1);
    P.lam = A.take<double>(sizeof(double) * ns1);
    P.trial = A.take<double>(sizeof(double) * 6 * ns1);
    P.ctl = A.take<Ctl>(sizeof(Ctl));
    P.imp = A.take<Striker>(sizeof(Striker));
    P.imp_step = A.take<StrikerStep>(sizeof(StrikerStep));
    P.fhist = A.take<double>(sizeof(double) * ctx->hist_cap);
    P.fout = A.take<double>(sizeof(double) * 3 * nn);
    P.field = A.take<float>(sizeof(float) * std::max(nh, nc1));
    P.bnodes = A.take<int32_t>(sizeof(int32_t) * std::max<size_t>(bnodes.size(), 1));
    P.ipair = A.take<int2>(sizeof(int2) * std::max<size_t>(ipair.size(), 1));
    P.iw = A.take<char>(std::max<size_t>(iw.size(), 16));
    for (int b = 0; b < 2; ++b) P.rDn[b] = A.take<char>(pairs_on ? ts * nn : 16);
  };
  Arena probe;
  layout(probe);
  cudaError_t ce = cudaMalloc(&ctx->arena.base, probe.used);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    return die(PDN_E_OOM, std::string("device allocation of ") + std::to_string(probe.used) + " bytes failed: " +
                              cudaGetErrorString(ce));
  }
  ctx->arena.size = probe.used;
  ctx->arena.used = 0;
  layout(ctx->arena);
  int32_t *d_hex = P.hex, *d_coh = P.coh, *d_surf = P.surf, *d_surf_of = P.surf_of, *d_row = P.row, *d_col = P.col;
  int8_t *d_ply = P.ply;
  char *d_X4 = P.X4, *d_imass = P.imass, *d_fe = P.fe;
  uint8_t *d_nflag = P.nflag, *d_rel = P.rel, *d_rmark_e = P.rmark_e, *d_rmark_n = P.rmark_n;
  double *d_Xs = P.Xs, *d_mass = P.mass, *d_nrm = P.nrm, *d_lam = P.lam, *d_trial = P.trial, *d_fhist = P.fhist,
         *d_fout = P.fout;
  double *d_d[2] = {P.d[0], P.d[1]}, *d_v[2] = {P.v[0], P.v[1]};
  char *d_u4[2] = {P.u4[0], P.u4[1]}, *d_hist[2] = {P.hist[0], P.hist[1]}, *d_rD[2] = {P.rD[0], P.rD[1]};
  uint8_t *d_act[2] = {P.act[0], P.act[1]};
  ctx->ctl_dev = P.ctl;
  ctx->imp_dev = P.imp;
  StrikerStep *d_imp_step = P.imp_step;
  ctx->field = P.field;

  if (opt->stream) {
    ctx->stream = (cudaStream_t)opt->stream;
  } else {
    ce = cudaStreamCreate(&ctx->stream);  // blocking: ordered with the legacy default stream
    if (ce != cudaSuccess) return die(PDN_E_CUDA, std::string("stream create: ") + cudaGetErrorString(ce));
    ctx->own_stream = true;
  }
  ce = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming);
  if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming);
  if (ce != cudaSuccess) return die(PDN_E_CUDA, std::string("side stream/events: ") + cudaGetErrorString(ce));
  ce = cudaMallocHost(&ctx->ctl_host, sizeof(Ctl));
  if (ce != cudaSuccess) return die(PDN_E_CUDA, std::string("pinned allocation: ") + cudaGetErrorString(ce));

  // host-side staging of the uploads
  RawVec<uint8_t> nflag(nn);
  parallel_chunks(nn, [&](int64_t b, int64_t e, int) {
    for (int64_t j = b; j < e; ++j) {
      nflag[j] = mesh->fixed ? mesh->fixed[j] : 0;
      if (surf_of[j] >= 0) nflag[j] |= 8;
      if (pairs_on && ipair[j].x >= 0) nflag[j] |= (uint8_t)((ipair[j].y & 7) << kFlagPairShift);
    }
  });
  std::vector<double> Xs(3 * std::max<int64_t>(ns, 1), 0.0);
  for (int64_t s = 0; s < ns; ++s)
    for (int i = 0; i < 3; ++i) Xs[i * ns + s] = mesh->X[i * nn + mesh->surf[s]];
  RawVec<char> X4(ts * 4 * nn), imass(ts * nn);
  parallel_chunks(nn, [&](int64_t b, int64_t e, int) {
  for (int64_t j = b; j < e; ++j) {
    if (fp64) {
      double *q = reinterpret_cast<double *>(X4.data()) + 4 * j;
      q[0] = mesh->X[j];
      q[1] = mesh->X[nn + j];
      q[2] = mesh->X[2 * nn + j];
      q[3] = 0.0;
      reinterpret_cast<double *>(imass.data())[j] = 1.0 / mass[j];
    } else {
      float *q = reinterpret_cast<float *>(X4.data()) + 4 * j;
      q[0] = (float)mesh->X[j];
      q[1] = (float)mesh->X[nn + j];
      q[2] = (float)mesh->X[2 * nn + j];
      q[3] = 0.0f;
      reinterpret_cast<float *>(imass.data())[j] = (float)(1.0 / mass[j]);
    }
  }
  });
  auto up = [&](void *dst, const void *src, size_t bytes) {
    return bytes ? cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  chk(up(d_hex, mesh->hex, sizeof(int32_t) * nh * 8));
  if (nc) chk(up(d_coh, mesh->coh, sizeof(int32_t) * nc * 8));
  chk(up(d_ply, mesh->ply_of_hex, nh));
  chk(up(d_X4, X4.data(), X4.size()));
  chk(cudaMemset(d_nflag, 0, (nn + 3) & ~int64_t(3)));
  chk(up(d_nflag, nflag.data(), nn));
  if (ns) chk(up(d_surf, mesh->surf, sizeof(int32_t) * ns));
  chk(up(d_surf_of, surf_of.data(), sizeof(int32_t) * nn));
  chk(up(d_Xs, Xs.data(), sizeof(double) * Xs.size()));
  chk(up(d_row, row.data(), sizeof(int32_t) * (nn + 1)));
  chk(up(d_col, col.data(), sizeof(int32_t) * col.size()));
  chk(up(P.pos, pos.data(), sizeof(int32_t) * pos.size()));
  chk(up(P.rank, rank.data(), sizeof(uint32_t) * rank.size()));
  if (sweep_on) chk(up(P.bnodes, bnodes.data(), sizeof(int32_t) * bnodes.size()));
  if (pairs_on) {
    chk(up(P.ipair, ipair.data(), sizeof(int2) * ipair.size()));
    chk(up(P.iw, iw.data(), iw.size()));
    for (int b = 0; b < 2; ++b) chk(cudaMemset(P.rDn[b], 0, ts * nn));
  }
  chk(up(d_mass, mass.data(), sizeof(double) * nn));
  chk(up(d_imass, imass.data(), imass.size()));
  for (int b = 0; b < 2; ++b) {
    chk(cudaMemset(d_d[b], 0, sizeof(double) * 3 * nn));
    chk(cudaMemset(d_v[b], 0, sizeof(double) * 3 * nn));
    chk(cudaMemset(d_u4[b], 0, ts * 4 * nn));
    chk(cudaMemset(d_rD[b], 0, ts * 4 * std::max<int64_t>(nc, 1)));
    chk(cudaMemset(d_act[b], 0, (std::max<int64_t>(ns, 1) + 15) & ~int64_t(15)));  // padding included
    chk(cudaMemset(P.pflag[b], 1, nh));  // every element starts with the initial history
    chk(cudaMemset(P.cflag[b], 1, std::max<int64_t>(nc, 1)));
    if (fp64)
      k_fill_hist_double<<<grid_of(nh * 8 * 7, 256), 256>>>(reinterpret_cast<double *>(d_hist[b]), nh * 8, 4);
    else
      k_fill_hist_float<<<grid_of(nh * 8 * 7, 256), 256>>>(reinterpret_cast<float *>(d_hist[b]), nh * 8, 4);
    chk(cudaGetLastError());
  }
  chk(cudaMemset(d_fe, 0, ts * 4 * n_slots));  // the padding slots stay zero
  chk(cudaMemset(d_rel, 0, std::max<int64_t>(ns, 1)));
  chk(cudaMemset(d_rmark_e, 0, nh + nc));
  chk(cudaMemset(d_rmark_n, 0, nn));
  chk(cudaMemset(d_nrm, 0, sizeof(double) * 3 * std::max<int64_t>(ns, 1)));
  chk(cudaMemset(d_lam, 0, sizeof(double) * std::max<int64_t>(ns, 1)));
  Ctl c0{};
  c0.mode = MODE_DONE;
  c0.max_repeats = ctx->max_repeats;
  chk(up(ctx->ctl_dev, &c0, sizeof(Ctl)));
  Striker s0{};
  s0.axis[2] = -1.0;
  s0.M = 1.0;
  s0.iM = 1.0;
  for (int i = 0; i < 3; ++i) s0.g[i] = ctx->grav[i];
  chk(up(ctx->imp_dev, &s0, sizeof(Striker)));
  chk(cudaMemset(d_imp_step, 0, sizeof(StrikerStep)));
  chk(cudaDeviceSynchronize());
  if (e != cudaSuccess) return die(PDN_E_CUDA, std::string("upload: ") + cudaGetErrorString(e));

  std::string why;
  int rc = fill_mat(ctx->Mf, m, mesh->ply_angle_deg, mesh->n_plies, opt->damage_on, opt->plasticity_on, why);
  if (!rc) rc = fill_mat(ctx->Md, m, mesh->ply_angle_deg, mesh->n_plies, opt->damage_on, opt->plasticity_on, why);
  if (rc) return die(rc, why);

  auto wire = [&](auto &D, auto tag) {
    using T = decltype(tag);
    using V4 = typename Vec4T<T>::type;
    D.nn = nn;
    D.nh = nh;
    D.nc = nc;
    D.ns = ns;
    D.hex = d_hex;
    D.coh = d_coh;
    D.ply = d_ply;
    D.X4 = reinterpret_cast<const V4 *>(d_X4);
    D.nflag = d_nflag;
    D.surf = d_surf;
    D.surf_of = d_surf_of;
    D.Xs = d_Xs;
    D.row = d_row;
    D.col = d_col;
    D.pos = P.pos;
    D.rank = ell ? P.rank : nullptr;
    D.mass = d_mass;
    D.inv_mass = reinterpret_cast<const T *>(d_imass);
    for (int b = 0; b < 2; ++b) {
      D.d[b] = d_d[b];
      D.v[b] = d_v[b];
      D.u4[b] = reinterpret_cast<V4 *>(d_u4[b]);
      D.hist[b] = reinterpret_cast<T *>(d_hist[b]);
      D.rD[b] = reinterpret_cast<T *>(d_rD[b]);
      D.act[b] = d_act[b];
      D.pflag[b] = P.pflag[b];
      D.cflag[b] = P.cflag[b];
    }
    D.fe = reinterpret_cast<V4 *>(d_fe);
    D.rel = d_rel;
    D.act_cnt = P.act_cnt;
    // PDN_FULL_REPEAT=1: repeated passes evaluate every element and node
    // again (the reference for the local repetition, same results)
    const char *fr = std::getenv("PDN_FULL_REPEAT");
    const bool full = fr != nullptr && fr[0] == '1' && fr[1] == '\0';
    // the column sweep evaluates every element and node again in a repeated
    // pass (the same results as the local repetition)
    D.rmark_e = (full || sweep_on) ? nullptr : d_rmark_e;
    D.rmark_n = (full || sweep_on) ? nullptr : d_rmark_n;
    D.sweep = nullptr;
    D.ipair = pairs_on ? P.ipair : nullptr;
    D.iw = (pairs_on && !pairs_uniform) ? reinterpret_cast<const V4 *>(P.iw) : nullptr;
    D.coh_w = (T)coh_w;
    for (int b = 0; b < 2; ++b) D.rDn[b] = pairs_on ? reinterpret_cast<T *>(P.rDn[b]) : nullptr;
    D.pair_layer = pair_layer;
    D.slot_compact = slot_compact ? 1 : 0;
    D.pair_inv_L = pair_layer > 0 ? 1.0f / (float)pair_layer : 0.0f;
    for (int l = 0; l < kMaxPairLayers; ++l) D.layer_off[l] = layer_off[l];
    for (int k = 0; k < 2; ++k)
      for (int w = 0; w < 2; ++w) D.pair_mask[k][w] = pair_mask[k][w];
    D.nrm = d_nrm;
    D.lam = d_lam;
    D.trial = d_trial;
    D.ctl = ctx->ctl_dev;
    D.imp = ctx->imp_dev;
    D.imp_step = d_imp_step;
    D.fhist = d_fhist;
    D.hist_cap = ctx->hist_cap;
    D.fout = d_fout;
    D.dt = ctx->dt;
    D.phi = ctx->phi;
    for (int i = 0; i < 3; ++i) {
      D.grav[i] = ctx->grav[i];
      D.grav_t[i] = (T)ctx->grav[i];
    }
    D.all_boxes = all_boxes ? 1 : 0;
    D.all_flat_coh = all_flat_coh ? 1 : 0;
    D.ell = ell ? 1 : 0;
    D.surf_base = surf_base;
  };
  if (fp64)
    wire(ctx->Dd, double{});
  else
    wire(ctx->Df, float{});
  ctx->rmark_e_buf = d_rmark_e;
  ctx->rmark_n_buf = d_rmark_n;
  {
    const char *fr = std::getenv("PDN_FULL_REPEAT");
    ctx->full_repeat = fr != nullptr && fr[0] == '1' && fr[1] == '\0';
  }
  if (sweep_on) {
    sweep.bnodes = P.bnodes;
    sweep.n_bnodes = (int64_t)bnodes.size();
    ctx->sweep = sweep;
    ctx->Df.sweep = &ctx->sweep;
  }
  // a^0 from the momentum equation at step 0 (Sec. 2.2.1): d^0 = 0 and no
  // contact at t^0, so the gravity acceleration on every free degree of
  // freedom; the first step then predicts d^1 and v^1 from it
  rc = read_ctl(ctx);
  if (!rc) rc = prime_state(ctx);
  if (rc) return die(rc, std::string("initial acceleration: ") + ctx->err);
  *out = ctx;
  return PDN_OK;
}

// No exception leaves the library: a failed host allocation is PDN_E_OOM.
int pdn_init_mesh(pdn_ctx **out, const pdn_mesh_desc *mesh, const pdn_material *mat, const pdn_options *opt) {
  try {
    return pdn_init_mesh_body(out, mesh, mat, opt);
  } catch (const std::bad_alloc &) {
    g_init_error = "host allocation failed";
    return PDN_E_OOM;
  } catch (...) {
    g_init_error = "unexpected host error";
    return PDN_E_ARG;
  }
}

int pdn_set_impactor(pdn_ctx *ctx, double radius, double mass, const double centre[3], const double velocity[3]) {
  if (!ctx) return PDN_E_ARG;
  if (!centre || !velocity || !(radius > 0) || !(mass > 0)) return fail(ctx, PDN_E_ARG, "radius and mass must be positive");
  Striker s{};
  const double n = std::sqrt(velocity[0] * velocity[0] + velocity[1] * velocity[1] + velocity[2] * velocity[2]);
  for (int i = 0; i < 3; ++i) {
    s.c[i] = centre[i];
    s.w[i] = velocity[i];
    s.F[i] = 0.0;
    s.axis[i] = n > 0 ? velocity[i] / n : (i == 2 ? -1.0 : 0.0);
    s.g[i] = ctx->grav[i];
  }
  s.R = radius;
  s.M = mass;
  s.iM = 1.0 / mass;
  s.has = 1;
  // reference of the energy ledger: the striker's kinetic energy and centre
  // when it is set (the plate's kinetic and stored energy enter as they are)
  ctx->imp_e0 = 0.5 * mass * (velocity[0] * velocity[0] + velocity[1] * velocity[1] + velocity[2] * velocity[2]);
  for (int i = 0; i < 3; ++i) ctx->imp_c0[i] = centre[i];
  PDN_CU(cudaMemcpyAsync(ctx->imp_dev, &s, sizeof(Striker), cudaMemcpyHostToDevice, ctx->stream), "set impactor");
  StrikerStep *ss = ctx->precision == PDN_FP64 ? ctx->Dd.imp_step : ctx->Df.imp_step;
  PDN_CU(launch_striker_init(ctx->imp_dev, ss, ctx->dt, ctx->stream), "striker init");
  PDN_CU(cudaStreamSynchronize(ctx->stream), "set impactor");
  ctx->has_imp = true;
  return PDN_OK;
}

// Autotuner: times every hex-kernel variant on force-evaluation passes of the
// committed state (no side effect on the simulation) and keeps the fastest.
// The variants differ only in their register budget.  The assembler may
// contract multiply-adds differently under another budget, so results can
// differ at FP32 rounding between variants (measured: the 3-block variant on
// the cut-down AS4 coupon, 2e-7 relative after 2,000 steps; the 5- and
// 6-block variants equal the 4-block one bit for bit).  Runs once per context, before the step
// graph is captured.
int autotune(pdn_ctx *ctx) {
  if (ctx->tuned) return PDN_OK;
  ctx->tuned = true;
  // variants timed by default: the hex kernel's four occupancy targets with
  // separate element and gather kernels, and the column sweep where it was
  // planned (the mixed hex + interface kernel, 4..7, is selected only by
  // PDN_HEX_VARIANT: it times well in the first passes but loses once damage
  // spreads)
  const int nvar = ctx->precision == PDN_FP64 ? 1 : 4;
  const int nsel = ctx->precision == PDN_FP64 ? 1 : 8;
  if (nvar == 1) return PDN_OK;
  const Sweep *sw = ctx->Df.sweep;
  // the sweep is kept only on request (PDN_SWEEP=1): the internal-force pass
  // the autotuner times does not show the cost of the node update in a
  // stepping pass, which the sweep carries inside its element launch; there
  // it measured slower (400x600x32 plate: 1.59 against 1.29 ms per step)
  const char *sv = std::getenv("PDN_SWEEP");
  const bool keep_sweep = sw && sv && sv[0] == '1' && sv[1] == '\0';
  auto drop_sweep = [&] {
    ctx->Df.sweep = nullptr;
    if (!ctx->full_repeat) {
      // separate kernels: the local repetition of released steps again
      ctx->Df.rmark_e = ctx->rmark_e_buf;
      ctx->Df.rmark_n = ctx->rmark_n_buf;
    }
  };
  // a fixed variant instead of timing (reproducible profiling runs)
  if (const char *fv = std::getenv("PDN_HEX_VARIANT")) {
    if (fv[0] >= '0' && fv[0] < '0' + nsel && fv[1] == '\0') {
      ctx->Df.hex_variant = fv[0] - '0';
      if (sw && !keep_sweep) drop_sweep();
      return PDN_OK;
    }
  }
  cudaEvent_t ev[2];
  for (int k = 0; k < 2; ++k) PDN_CU(cudaEventCreate(&ev[k]), "tune event");
  const int reps = 8;
  // mean time of a whole internal-force pass as the graph runs it (the
  // interface kernel on the forked stream where the variant uses one)
  auto time_pass = [&](float &mean) -> int {
    float sum = 0.f;
    for (int r = 0; r <= reps; ++r) {
      int rc = set_mode(ctx, MODE_FORCES, ctx->ctl_host->step);
      if (rc) return rc;
      PDN_CU(cudaEventRecord(ev[0], ctx->stream), "autotune record");
      cudaError_t e = run_pass(ctx, nullptr);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune pass");
      PDN_CU(cudaEventRecord(ev[1], ctx->stream), "autotune record");
      PDN_CU(cudaStreamSynchronize(ctx->stream), "autotune");
      float ms = 0.f;
      PDN_CU(cudaEventElapsedTime(&ms, ev[0], ev[1]), "autotune time");
      if (r > 0) sum += ms;  // the first pass warms up
    }
    mean = sum / reps;
    return PDN_OK;
  };
  int best = 0;
  float best_ms = 1e30f;
  ctx->Df.sweep = nullptr;
  for (int v = 0; v < nvar; ++v) {
    ctx->Df.hex_variant = v;
    int rc = time_pass(ctx->tune_ms[v]);
    if (rc) return rc;
    if (ctx->tune_ms[v] < best_ms) {
      best_ms = ctx->tune_ms[v];
      best = v;
    }
  }
  ctx->Df.hex_variant = best;
  if (sw) {
    ctx->Df.sweep = sw;
    int rc = time_pass(ctx->tune_ms[8]);
    if (rc) return rc;
    if (!keep_sweep) drop_sweep();
  }
  for (int k = 0; k < 2; ++k) cudaEventDestroy(ev[k]);
  return PDN_OK;
}

int pdn_step(pdn_ctx *ctx, int64_t nsteps) {
  if (!ctx) return PDN_E_ARG;
  NvtxRange range("pdn_step");
  if (nsteps < 0) return fail(ctx, PDN_E_ARG, "nsteps < 0");
  if (!ctx->has_imp) return fail(ctx, PDN_E_STATE, "pdn_set_impactor must be called before pdn_step");
  int rc = read_ctl(ctx);
  if (rc) return rc;
  if (ctx->ctl_host->status) return fail(ctx, ctx->ctl_host->status, "device halted earlier (sticky status)");
  if (nsteps == 0) return PDN_OK;
  rc = autotune(ctx);
  if (rc) return rc;
  const int64_t target = ctx->ctl_host->step + nsteps;
  rc = set_mode(ctx, MODE_ADVANCE, target);
  if (rc) return rc;
  int64_t remaining = nsteps;
  for (int guard = 0; remaining > 0; ++guard) {
    cudaError_t e = launch_passes(ctx, remaining);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launch step passes");
    rc = read_ctl(ctx);
    if (rc) return rc;
    const Ctl &c = *ctx->ctl_host;
    if (c.status) {
      return fail(ctx, c.status,
                  c.check == CHECK_ELEMENT_NODE   ? "device bounds check: an element names a node out of range"
                  : c.check == CHECK_SURFACE_NODE ? "device bounds check: a surface entry names a node out of range"
                  : c.status == PDN_E_NONFINITE   ? "non-finite acceleration or displacement"
                  : c.status == PDN_E_TIMEOUT ? "a bounded wait on the tensor core gave up (learned law)"
                                              : "contact release limit reached (Algorithm 2)");
    }
    remaining = target - c.step;
    if (guard > 64 * (ctx->max_repeats + 1)) return fail(ctx, PDN_E_STATE, "step loop made no progress");
  }
  return PDN_OK;
}

int pdn_profile_kernels(pdn_ctx *ctx, int64_t nsteps, float *ms_per_launch, int64_t *launches) {
  if (!ctx) return PDN_E_ARG;
  NvtxRange range("pdn_profile_kernels");
  if (nsteps < 0) return fail(ctx, PDN_E_ARG, "nsteps < 0");
  if (!ctx->has_imp) return fail(ctx, PDN_E_STATE, "pdn_set_impactor must be called first");
  if (ctx->prof_ev.empty()) {
    ctx->prof_ev.resize(6 * kProfilePasses);
    for (auto &e : ctx->prof_ev) PDN_CU(cudaEventCreate(&e), "event create");
  }
  int rc = read_ctl(ctx);
  if (rc) return rc;
  if (ctx->ctl_host->status) return fail(ctx, ctx->ctl_host->status, "device halted earlier (sticky status)");
  const int64_t target = ctx->ctl_host->step + nsteps;
  rc = set_mode(ctx, MODE_ADVANCE, target);
  if (rc) return rc;
  double tot[PDN_K_COUNT] = {0};
  int64_t cnt[PDN_K_COUNT] = {0};
  int64_t remaining = nsteps;
  while (remaining > 0) {
    const int64_t chunk = std::min<int64_t>(remaining, kProfilePasses);
    for (int64_t p = 0; p < chunk; ++p) {
      cudaError_t e = run_pass(ctx, ctx->prof_ev.data() + 6 * p);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "profile pass");
    }
    rc = read_ctl(ctx);
    if (rc) return rc;
    for (int64_t p = 0; p < chunk; ++p)
      for (int k = 0; k < PDN_K_COUNT; ++k) {
        if (k == PDN_K_COH && ctx->nc == 0) continue;
        float ms = 0.f;
        PDN_CU(cudaEventElapsedTime(&ms, ctx->prof_ev[6 * p + k], ctx->prof_ev[6 * p + k + 1]), "event time");
        tot[k] += ms;
        cnt[k] += 1;
      }
    const Ctl &c = *ctx->ctl_host;
    if (c.status) return fail(ctx, c.status, "device halted during profiling");
    remaining = target - c.step;
  }
  for (int k = 0; k < PDN_K_COUNT; ++k) {
    if (ms_per_launch) ms_per_launch[k] = cnt[k] ? (float)(tot[k] / cnt[k]) : 0.f;
    if (launches) launches[k] = cnt[k];
  }
  return PDN_OK;
}

int64_t pdn_contact_force(pdn_ctx *ctx, double f_now[3], double *f_peak, double *history, int64_t cap) {
  if (!ctx) return PDN_E_ARG;
  int rc = read_ctl(ctx);
  if (rc) return rc;
  if (f_now) {
    Striker s;
    PDN_CU(cudaMemcpy(&s, ctx->imp_dev, sizeof(Striker), cudaMemcpyDeviceToHost), "read striker");
    for (int i = 0; i < 3; ++i) f_now[i] = s.F[i];
  }
  if (f_peak) *f_peak = ctx->ctl_host->f_peak;
  int64_t n = std::min<int64_t>(ctx->ctl_host->hist_count, cap > 0 ? cap : 0);
  if (history && n > 0) {
    const double *src = ctx->precision == PDN_FP64 ? ctx->Dd.fhist : ctx->Df.fhist;
    PDN_CU(cudaMemcpy(history, src, sizeof(double) * n, cudaMemcpyDeviceToHost), "read force history");
  }
  return history ? n : ctx->ctl_host->hist_count;
}

int pdn_damage_field(pdn_ctx *ctx, int32_t which, float *out, int64_t n, int32_t out_on_device) {
  if (!ctx) return PDN_E_ARG;
  if (which < PDN_FIELD_D1 || which > PDN_FIELD_PLASTIC) return fail(ctx, PDN_E_ARG, "unknown field");
  const int64_t need = which == PDN_FIELD_DCOH ? ctx->nc : ctx->nh;
  if (!out || n != need) return fail(ctx, PDN_E_ARG, "output size must equal the element count of the field");
  if (need == 0) return PDN_OK;
  cudaError_t e = ctx->precision == PDN_FP64 ? launch_damage_field<double>(ctx->Dd, ctx->Md, which, ctx->field, ctx->stream)
                                             : launch_damage_field<float>(ctx->Df, ctx->Mf, which, ctx->field, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "damage field kernel");
  PDN_CU(cudaMemcpyAsync(out, ctx->field, sizeof(float) * n,
                         out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream),
         "copy damage field");
  PDN_CU(cudaStreamSynchronize(ctx->stream), "damage field");
  return PDN_OK;
}

int pdn_get_state(pdn_ctx *ctx, double *d, double *v, double *imp) {
  if (!ctx) return PDN_E_ARG;
  int rc = read_ctl(ctx);
  if (rc) return rc;
  const int b = ctx->ctl_host->dpar ^ 1;
  double *const *dd = ctx->precision == PDN_FP64 ? ctx->Dd.d : ctx->Df.d;
  double *const *vv = ctx->precision == PDN_FP64 ? ctx->Dd.v : ctx->Df.v;
  if (d) PDN_CU(cudaMemcpy(d, dd[b], sizeof(double) * 3 * ctx->nn, cudaMemcpyDeviceToHost), "read d");
  if (v) PDN_CU(cudaMemcpy(v, vv[b], sizeof(double) * 3 * ctx->nn, cudaMemcpyDeviceToHost), "read v");
  if (imp) {
    Striker s;
    PDN_CU(cudaMemcpy(&s, ctx->imp_dev, sizeof(Striker), cudaMemcpyDeviceToHost), "read striker");
    for (int i = 0; i < 3; ++i) {
      imp[i] = s.c[i];
      imp[3 + i] = s.w[i];
      imp[6 + i] = s.F[i];
    }
    imp[9] = ctx->ctl_host->time;
  }
  return PDN_OK;
}

static int pdn_set_state_body(pdn_ctx *ctx, const double *d, const double *v) {
  if (!ctx) return PDN_E_ARG;
  if (!d || !v) return fail(ctx, PDN_E_ARG, "d and v are required");
  int rc = read_ctl(ctx);
  if (rc) return rc;
  if (ctx->ctl_host->status) return fail(ctx, ctx->ctl_host->status, "device halted earlier (sticky status)");
  const int b = ctx->ctl_host->dpar;
  const int64_t nn = ctx->nn;
  std::vector<uint8_t> nflag(nn);
  const uint8_t *fl = ctx->precision == PDN_FP64 ? ctx->Dd.nflag : ctx->Df.nflag;
  PDN_CU(cudaMemcpy(nflag.data(), fl, nn, cudaMemcpyDeviceToHost), "read flags");
  std::vector<double> dh(d, d + 3 * nn), vh(v, v + 3 * nn);
  for (int64_t j = 0; j < nn; ++j)
    for (int i = 0; i < 3; ++i)
      if ((nflag[j] >> i) & 1) {
        dh[i * nn + j] = 0.0;
        vh[i * nn + j] = 0.0;
      }
  double *const *dd = ctx->precision == PDN_FP64 ? ctx->Dd.d : ctx->Df.d;
  double *const *vv = ctx->precision == PDN_FP64 ? ctx->Dd.v : ctx->Df.v;
  PDN_CU(cudaMemcpy(dd[b], dh.data(), sizeof(double) * 3 * nn, cudaMemcpyHostToDevice), "write d");
  PDN_CU(cudaMemcpy(vv[b], vh.data(), sizeof(double) * 3 * nn, cudaMemcpyHostToDevice), "write v");
  if (ctx->precision == PDN_FP64)
    k_mirror<double4_32a><<<grid_of(nn, 256), 256, 0, ctx->stream>>>(dd[b], ctx->Dd.u4[b], nn);
  else
    k_mirror<float4><<<grid_of(nn, 256), 256, 0, ctx->stream>>>(dd[b], ctx->Df.u4[b], nn);
  PDN_CU(cudaGetLastError(), "mirror kernel");
  return prime_state(ctx);
}

// No exception leaves the library: a failed host allocation is PDN_E_OOM.
int pdn_set_state(pdn_ctx *ctx, const double *d, const double *v) {
  try {
    return pdn_set_state_body(ctx, d, v);
  } catch (const std::bad_alloc &) {
    return PDN_E_OOM;
  } catch (...) {
    return PDN_E_ARG;
  }
}

static int pdn_get_contact_body(pdn_ctx *ctx, uint8_t *active, double *lambda) {
  if (!ctx) return PDN_E_ARG;
  int rc = read_ctl(ctx);
  if (rc) return rc;
  const int64_t ns = ctx->ns;
  if (ns == 0) return PDN_OK;
  const int par = (int)(ctx->ctl_host->step & 1);
  uint8_t *const *act = ctx->precision == PDN_FP64 ? ctx->Dd.act : ctx->Df.act;
  const double *lam = ctx->precision == PDN_FP64 ? ctx->Dd.lam : ctx->Df.lam;
  std::vector<uint8_t> a(ns);
  PDN_CU(cudaMemcpy(a.data(), act[par], ns, cudaMemcpyDeviceToHost), "read contact set");
  if (active) std::memcpy(active, a.data(), ns);
  if (lambda) {
    PDN_CU(cudaMemcpy(lambda, lam, sizeof(double) * ns, cudaMemcpyDeviceToHost), "read reactions");
    for (int64_t s = 0; s < ns; ++s)
      if (!a[s]) lambda[s] = 0.0;
  }
  return PDN_OK;
}

// No exception leaves the library: a failed host allocation is PDN_E_OOM.
int pdn_get_contact(pdn_ctx *ctx, uint8_t *active, double *lambda) {
  try {
    return pdn_get_contact_body(ctx, active, lambda);
  } catch (const std::bad_alloc &) {
    return PDN_E_OOM;
  } catch (...) {
    return PDN_E_ARG;
  }
}

static int pdn_get_history_body(pdn_ctx *ctx, void *hist, void *rD) {
  if (!ctx) return PDN_E_ARG;
  int rc = read_ctl(ctx);
  if (rc) return rc;
  if (ctx->precision == PDN_FP64)
    return get_history_t<double>(ctx, ctx->Dd, static_cast<double *>(hist), static_cast<double *>(rD));
  return get_history_t<float>(ctx, ctx->Df, static_cast<float *>(hist), static_cast<float *>(rD));
}

int pdn_get_history(pdn_ctx *ctx, void *hist, void *rD) {
  try {
    return pdn_get_history_body(ctx, hist, rD);
  } catch (const std::bad_alloc &) {
    return PDN_E_OOM;
  } catch (...) {
    return PDN_E_ARG;
  }
}

// The committed state sits in the node buffer dpar ^ 1 and the prediction of
// the next step (v' = v + dt a, before contact) in buffer dpar; no pass has
// touched the prediction since the commit.
static int pdn_get_acceleration_body(pdn_ctx *ctx, double *a) {
  if (!ctx) return PDN_E_ARG;
  if (!a) return fail(ctx, PDN_E_ARG, "a is NULL");
  int rc = read_ctl(ctx);
  if (rc) return rc;
  const int b = ctx->ctl_host->dpar;
  const int64_t n3 = 3 * ctx->nn;
  double *const *vv = ctx->precision == PDN_FP64 ? ctx->Dd.v : ctx->Df.v;
  std::vector<double> vp(n3);
  PDN_CU(cudaMemcpy(vp.data(), vv[b], sizeof(double) * n3, cudaMemcpyDeviceToHost), "read predicted v");
  PDN_CU(cudaMemcpy(a, vv[b ^ 1], sizeof(double) * n3, cudaMemcpyDeviceToHost), "read v");
  const double idt = 1.0 / ctx->dt;
  for (int64_t k = 0; k < n3; ++k) a[k] = (vp[k] - a[k]) * idt;
  return PDN_OK;
}

int pdn_get_acceleration(pdn_ctx *ctx, double *a) {
  try {
    return pdn_get_acceleration_body(ctx, a);
  } catch (const std::bad_alloc &) {
    return PDN_E_OOM;
  } catch (...) {
    return PDN_E_ARG;
  }
}

int pdn_internal_force(pdn_ctx *ctx, double *f_int) {
  if (!ctx) return PDN_E_ARG;
  NvtxRange range("pdn_internal_force");
  if (!f_int) return fail(ctx, PDN_E_ARG, "f_int is NULL");
  int rc = read_ctl(ctx);
  if (rc) return rc;
  if (ctx->ctl_host->status) return fail(ctx, ctx->ctl_host->status, "device halted earlier (sticky status)");
  rc = set_mode(ctx, MODE_FORCES, ctx->ctl_host->step);
  if (rc) return rc;
  cudaError_t e = run_pass(ctx, nullptr);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "force pass");
  const double *fo = ctx->precision == PDN_FP64 ? ctx->Dd.fout : ctx->Df.fout;
  PDN_CU(cudaMemcpyAsync(f_int, fo, sizeof(double) * 3 * ctx->nn, cudaMemcpyDeviceToHost, ctx->stream), "read forces");
  PDN_CU(cudaStreamSynchronize(ctx->stream), "force pass");
  return PDN_OK;
}

int pdn_get_info(pdn_ctx *ctx, pdn_info *info) {
  if (!ctx || !info) return PDN_E_ARG;
  int rc = read_ctl(ctx);
  if (rc) return rc;
  const Ctl &c = *ctx->ctl_host;
  info->dt = ctx->dt;
  info->dt_bulk = ctx->dt_bulk;
  info->dt_coh = ctx->dt_coh;
  info->time = c.time;
  info->f_peak = c.f_peak;
  info->step = c.step;
  info->n_active = c.n_active;
  info->n_repeats = c.n_repeats_total;
  info->n_nodes = ctx->nn;
  info->n_hex = ctx->nh;
  info->n_coh = ctx->nc;
  info->n_surf = ctx->ns;
  info->device_bytes = (int64_t)ctx->arena.size;
  info->status = c.status;
  info->precision = ctx->precision;
  info->hex_variant = ctx->precision == PDN_FP64 ? ctx->Dd.hex_variant : ctx->Df.hex_variant;
  info->sweep = (ctx->precision == PDN_FP32_FORCE && ctx->Df.sweep != nullptr) ? 1 + ctx->sweep.tile : 0;
  {
    const bool f64 = ctx->precision == PDN_FP64;
    const bool pairs = (f64 ? ctx->Dd.ipair : ctx->Df.ipair) != nullptr;
    const bool layered = (f64 ? ctx->Dd.pair_layer : ctx->Df.pair_layer) > 0;
    info->coh_pairs = pairs ? (layered ? 2 : 1) : 0;
  }
  info->reserved = 0;
  for (int v = 0; v < 12; ++v) info->tune_ms[v] = ctx->tune_ms[v];
  return PDN_OK;
}

}  // extern "C"

// Helpers for other translation units of the library (pdn_noalloc.cu).
namespace pdn {
void set_thread_error(const std::string &msg) { g_init_error = msg; }
int ctx_fail(pdn_ctx *c, int code, const std::string &msg) { return fail(c, code, msg); }
int ctx_cuda_fail(pdn_ctx *c, cudaError_t e, const char *where) { return cuda_fail(c, e, where); }
int ctx_read_ctl(pdn_ctx *ctx) { return read_ctl(ctx); }
template <typename T>
int fill_mat_public(Mat<T> &M, const pdn_material &m, const double *ply_angle, int n_plies, int damage_on,
                    int plasticity_on, std::string &why) {
  return fill_mat(M, m, ply_angle, n_plies, damage_on, plasticity_on, why);
}
template int fill_mat_public<float>(Mat<float> &, const pdn_material &, const double *, int, int, int, std::string &);
template int fill_mat_public<double>(Mat<double> &, const pdn_material &, const double *, int, int, int,
                                     std::string &);
}  // namespace pdn
