// Energy ledger of a context (pdn_energies, include/pdn.h): kinetic energy of
// plate and striker, elastic energy stored in the hexes and the interface
// elements, and the work of gravity, at the committed state, evaluated on the
// device in FP64 (Sec. 3.2 reports the energy-time curves of the impact).
//
// The stored energies are those of the secant (damaged) material: per Gauss
// point 1/2 sigma : eps_e (ply axes, elastic strain = strain minus the plastic
// shear strains, the law's nominal stress at the committed history), per
// interface point 1/2 w tau . Delta.  With the exact law the sum
//   kinetic (plate + striker) + stored - work of gravity
// is conserved by the elastic impact up to the time integrator's error, and
// decreases by the dissipated energy once damage or plasticity develop.
//
// Reductions are deterministic: a fixed tree per block, then the blocks'
// partial sums in block order on the host.  The partials go to the context's
// internal-force output buffer (3 n_nodes doubles, larger than any grid here).
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "pdn.h"
#include "pdn_context.h"
#include "pdn_device.cuh"
#include "pdn_internal.h"

namespace pdn {
// context helpers of pdn_api.cu: error message and code, control-block read
int ctx_fail(pdn_ctx *c, int code, const std::string &msg);
int ctx_cuda_fail(pdn_ctx *c, cudaError_t e, const char *where);
int ctx_read_ctl(pdn_ctx *ctx);
}  // namespace pdn

using namespace pdn;
using namespace pdn::detail;

namespace {

constexpr int kBlock = 256;

// Sum of v over the block (fixed tree), written by thread 0 to out.
__device__ __forceinline__ void block_sum(double v, double *out) {
  __shared__ double s[kBlock];
  s[threadIdx.x] = v;
  __syncthreads();
#pragma unroll
  for (int h = kBlock / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = s[0];
}

// Nodes: 1/2 m v.v and m g.d (the plate's share of the work of gravity).
// The velocity is the one at the committed time level: the stored velocity
// of the Tchamwa-Wielgosz scheme is the central-difference velocity half a
// step back (phi = 1), so the level value is v + dt/2 a = the mean of the
// stored velocity and the predicted one of the next step (v' = v + dt a).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_energy_nodes(Dev<T> D, double *part_ke, double *part_wg) {
  const int64_t j = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  const int b = D.ctl->dpar ^ 1;  // committed state; buffer b ^ 1 holds the prediction
  double ke = 0.0, wg = 0.0;
  if (j < D.nn) {
    const double m = D.mass[j];
    for (int i = 0; i < 3; ++i) {
      const double v = 0.5 * (D.v[b][i * D.nn + j] + D.v[b ^ 1][i * D.nn + j]), d = D.d[b][i * D.nn + j];
      ke += 0.5 * m * v * v;
      wg += m * D.grav[i] * d;
    }
  }
  block_sum(ke, part_ke + blockIdx.x);
  block_sum(wg, part_wg + blockIdx.x);
}

// Hexes: sum over the 2x2x2 Gauss points of det J * 1/2 sigma : eps_e, with
// the law of Algorithm 4 evaluated at the committed displacement and history
// (FP64; the history of a pristine-flagged element is the initial one).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_energy_hex(Dev<T> D, Mat<double> M, double *part) {
  const int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  double u = 0.0;
  if (e < D.nh) {
    const int b = D.ctl->dpar ^ 1, hb = D.ctl->hpar;
    const int64_t nn = D.nn, nh = D.nh;
    double xa[8][3], ua[8][3], am[8][3], bm[8][3];
    for (int a = 0; a < 8; ++a) {
      const int j = D.hex[8 * e + a];
      const auto x = D.X4[j];
      xa[a][0] = (double)x.x;
      xa[a][1] = (double)x.y;
      xa[a][2] = (double)x.z;
      for (int i = 0; i < 3; ++i) ua[a][i] = D.d[b][i * nn + j];
    }
    to_modes(xa, am);
    to_modes(ua, bm);
    const int ply = D.ply[e];
    const double cs = M.ply_c[ply], sn = M.ply_s[ply];
    const double c2 = cs * cs, s2 = sn * sn, csn = cs * sn;
    const ElemLaw<double> L = elem_law(M, e);
    const bool pristine = D.pflag[0] != nullptr && D.pflag[hb][e] != 0;
    double lc = -1.0;
    const double gp = 0.57735026918962576451;
    for (int g = 0; g < 8; ++g) {
      const double xi = sgn_x(g) * gp, et = sgn_y(g) * gp, ze = sgn_z(g) * gp;
      double J[3][3], Du[3][3], Ji[3][3], H[3][3];
      jac_cols(am, xi, et, ze, J);
      jac_cols(bm, xi, et, ze, Du);
      const double det = det3(J), id = 1.0 / det;
      Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
      Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
      Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
      Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
      Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
      Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
      Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
      Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
      Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
      // H = du/dX = (du/dxi) (dxi/dX)
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) H[i][k] = Du[i][0] * Ji[0][k] + Du[i][1] * Ji[1][k] + Du[i][2] * Ji[2][k];
      double E[3][3];
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
          E[i][k] = 0.5 * (H[i][k] + H[k][i] + H[0][i] * H[0][k] + H[1][i] * H[1][k] + H[2][i] * H[2][k]);
      double ep[6];
      ep[0] = c2 * E[0][0] + 2.0 * csn * E[0][1] + s2 * E[1][1];
      ep[1] = s2 * E[0][0] - 2.0 * csn * E[0][1] + c2 * E[1][1];
      ep[2] = E[2][2];
      ep[3] = 2.0 * (-csn * E[0][0] + (c2 - s2) * E[0][1] + csn * E[1][1]);
      ep[4] = 2.0 * (cs * E[0][2] + sn * E[1][2]);
      ep[5] = 2.0 * (-sn * E[0][2] + cs * E[1][2]);
      double h[7];
      for (int f = 0; f < 7; ++f)
        h[f] = pristine ? (f < 4 ? 1.0 : 0.0) : (double)D.hist[hb][((int64_t)f * 8 + g) * nh + e];
      double s[6];
      cdm(M, L, am, 0.0, lc, ep, h, s);
      const double ee[6] = {ep[0], ep[1], ep[2], ep[3] - h[4], ep[4] - h[5], ep[5]};
      double w = 0.0;
      for (int k = 0; k < 6; ++k) w += s[k] * ee[k];
      u += 0.5 * w * det;
    }
  }
  block_sum(u, part + blockIdx.x);
}

// Interface elements: per Newton-Cotes point (the corners) 1/2 w tau . Delta,
// the jump Delta = u_top - u_bottom in the frame of the reference mid-surface
// at the element centre (e1 along the xi tangent, e3 the normal), w the
// mid-surface area Jacobian at the corner, tau from the cohesive law at the
// committed threshold (Algorithm 5).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_energy_coh(Dev<T> D, Mat<double> M, double *part) {
  const int64_t c = (int64_t)blockIdx.x * kBlock + threadIdx.x;
  double u = 0.0;
  if (c < D.nc) {
    const int b = D.ctl->dpar ^ 1, hb = D.ctl->hpar;
    const int64_t nn = D.nn, nc = D.nc;
    const bool pristine = D.cflag[0] != nullptr && D.cflag[hb][c] != 0;
    int nd[8];
    double xm[4][3];
    for (int a = 0; a < 8; ++a) nd[a] = D.coh[8 * c + a];
    for (int a = 0; a < 4; ++a) {
      const auto x0 = D.X4[nd[a]], x1 = D.X4[nd[a + 4]];
      xm[a][0] = 0.5 * ((double)x0.x + (double)x1.x);
      xm[a][1] = 0.5 * ((double)x0.y + (double)x1.y);
      xm[a][2] = 0.5 * ((double)x0.z + (double)x1.z);
    }
    // corner signs of the bilinear face, counter-clockwise
    const double sx[4] = {-1, 1, 1, -1}, sy[4] = {-1, -1, 1, 1};
    double t1[3] = {0, 0, 0}, t2[3] = {0, 0, 0};
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) {
        t1[i] += 0.25 * sx[a] * xm[a][i];
        t2[i] += 0.25 * sy[a] * xm[a][i];
      }
    double n[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2], t1[0] * t2[1] - t1[1] * t2[0]};
    const double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    const double tl = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
    double e1[3], e2[3], e3[3];
    for (int i = 0; i < 3; ++i) {
      e3[i] = n[i] / nl;
      e1[i] = t1[i] / tl;
    }
    e2[0] = e3[1] * e1[2] - e3[2] * e1[1];
    e2[1] = e3[2] * e1[0] - e3[0] * e1[2];
    e2[2] = e3[0] * e1[1] - e3[1] * e1[0];
    for (int p = 0; p < 4; ++p) {
      double ta[3] = {0, 0, 0}, tb[3] = {0, 0, 0};
      for (int a = 0; a < 4; ++a) {
        const double dxi = 0.25 * sx[a] * (1.0 + sy[p] * sy[a]);
        const double deta = 0.25 * sy[a] * (1.0 + sx[p] * sx[a]);
        for (int i = 0; i < 3; ++i) {
          ta[i] += dxi * xm[a][i];
          tb[i] += deta * xm[a][i];
        }
      }
      const double nx = ta[1] * tb[2] - ta[2] * tb[1], ny = ta[2] * tb[0] - ta[0] * tb[2],
                   nz = ta[0] * tb[1] - ta[1] * tb[0];
      const double w = sqrt(nx * nx + ny * ny + nz * nz);
      double dg[3];
      for (int i = 0; i < 3; ++i) dg[i] = D.d[b][i * nn + nd[p + 4]] - D.d[b][i * nn + nd[p]];
      const double dl[3] = {e1[0] * dg[0] + e1[1] * dg[1] + e1[2] * dg[2],
                            e2[0] * dg[0] + e2[1] * dg[1] + e2[2] * dg[2],
                            e3[0] * dg[0] + e3[1] * dg[1] + e3[2] * dg[2]};
      const double r = pristine ? 0.0 : (double)D.rD[hb][(int64_t)p * nc + c];
      double rout, tau[3];
      czm(M, dl, M.damage_on ? r : 0.0, rout, tau);
      u += 0.5 * w * (tau[0] * dl[0] + tau[1] * dl[1] + tau[2] * dl[2]);
    }
  }
  block_sum(u, part + blockIdx.x);
}

inline int blocks_of(int64_t n) { return (int)((n + kBlock - 1) / kBlock); }

template <typename T>
int energies_t(pdn_ctx *ctx, const Dev<T> &D, double out[6]) {
  const int nbn = blocks_of(D.nn), nbh = blocks_of(D.nh), nbc = D.nc > 0 ? blocks_of(D.nc) : 0;
  double *part = D.fout;  // 3 nn doubles: room for 2 nbn + nbh + nbc partials
  if (nbc > 0) {
    const cudaError_t ep = launch_pairs_to_elements(D, ctx->stream);
    if (ep != cudaSuccess) return ctx_cuda_fail(ctx, ep, "interface thresholds from node pairs");
  }
  k_energy_nodes<T><<<nbn, kBlock, 0, ctx->stream>>>(D, part, part + nbn);
  if (D.nh > 0) k_energy_hex<T><<<nbh, kBlock, 0, ctx->stream>>>(D, ctx->Md, part + 2 * nbn);
  if (nbc > 0) k_energy_coh<T><<<nbc, kBlock, 0, ctx->stream>>>(D, ctx->Md, part + 2 * nbn + nbh);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "energy kernels");
  std::vector<double> h((size_t)(2 * nbn + nbh + nbc));
  e = cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "energy read-back");
  double ke = 0.0, wg = 0.0, uh = 0.0, uc = 0.0;
  for (int k = 0; k < nbn; ++k) ke += h[k];
  for (int k = 0; k < nbn; ++k) wg += h[nbn + k];
  for (int k = 0; k < nbh; ++k) uh += h[2 * nbn + k];
  for (int k = 0; k < nbc; ++k) uc += h[2 * nbn + nbh + k];
  Striker s;
  e = cudaMemcpy(&s, ctx->imp_dev, sizeof(Striker), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e, "read striker");
  double kes = 0.0, wgs = 0.0;
  if (s.has) {
    for (int i = 0; i < 3; ++i) {
      kes += 0.5 * s.M * s.w[i] * s.w[i];
      wgs += s.M * s.g[i] * (s.c[i] - ctx->imp_c0[i]);
    }
  }
  out[0] = ke;
  out[1] = kes;
  out[2] = uh;
  out[3] = uc;
  out[4] = wg + wgs;
  out[5] = ctx->imp_e0;
  return PDN_OK;
}

}  // namespace

extern "C" int pdn_energies(pdn_ctx *ctx, double out[6]) {
  if (!ctx) return PDN_E_ARG;
  if (!out) return ctx_fail(ctx, PDN_E_ARG, "out is NULL");
  int rc = ctx_read_ctl(ctx);
  if (rc) return rc;
  if (ctx->precision == PDN_FP64) return energies_t<double>(ctx, ctx->Dd, out);
  return energies_t<float>(ctx, ctx->Df, out);
}
