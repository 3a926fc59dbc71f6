// Per-item bodies of the step kernels (one contact-surface node, one hex8,
// one interface element, one node for the gather, the tail of a pass),
// shared by the per-pass kernels (pdn_kernels.cu) and the batched persistent
// kernel (pdn_batch.cu).
#pragma once

#include <cstdint>
#include <type_traits>

#include "pdn.h"
#include "pdn_device.cuh"
#include "pdn_internal.h"

// Pointers to state that other blocks write in the course of a pass (the
// element-precision mirror of the displacement, the Gauss-point history, the
// interface thresholds).  The per-pass kernels never write these buffers in
// the launch that reads them through such a pointer, so their loads may take
// the read-only data path (restrict-qualified pointers).  The batched
// persistent kernel writes them in earlier phases of the same launch, where a
// read-only cached line could be stale; it compiles these items with plain
// pointers by defining PDN_ITEMS_IN_PERSISTENT_KERNEL before including this
// file.
#ifdef PDN_ITEMS_IN_PERSISTENT_KERNEL
#define PDN_STATE_RESTRICT
#else
#define PDN_STATE_RESTRICT __restrict__
#endif

namespace pdn {
namespace detail {

// ---------------------------------------------------------------------------
// Kernel 1: contact detection and projection (Sec. 2.1, Fig. 1, Algorithm 1).
// One thread per contact-surface node.  The striker state of the step being
// computed (its RK4 update with the committed contact force held over the
// step, Eq. rk4) was produced by the tail of the previous pass, or by
// k_striker_init after pdn_set_impactor; this kernel only reads it.
// Returns whether node s is in the contact set when the item is done.
template <typename T>
__device__ __forceinline__ bool contact_item(const Dev<T> &D, int64_t s, int mode) {
  using V4 = typename Vec4T<T>::type;
  const Ctl *ctl = D.ctl;
  if (s >= D.ns) return false;
  const Striker *S = D.imp;
  const StrikerStep *ss = D.imp_step;
  const int64_t nn = D.nn, ns = D.ns;
  const int64_t j = D.surf_base >= 0 ? D.surf_base + s : D.surf[s];
#ifdef PDN_CHECK
  if (j < 0 || j >= D.nn) {
    atomicCAS(&D.ctl->check, 0, (int32_t)CHECK_SURFACE_NODE);
    return false;
  }
#endif
  const int cur = ctl->dpar;
  const int spar = (int)((ctl->step + 1) & 1), ppar = (int)(ctl->step & 1);
  double *d = D.d[cur];
  double *v = D.v[cur];
  if (mode == MODE_ADVANCE) {
    D.rel[s] = 0;
    uint8_t a = 0;
    const uint8_t fl = D.nflag[j];
    const bool was_active = D.act[ppar][s] != 0;
    bool near = was_active;
    if (!near && S->has && (fl & 7) != 7) {
      // FP32 prefilter: nodes farther than R + 0.05 mm from the centre cannot
      // be in contact (the FP32 distance error here is below 1e-4 mm); only
      // the others take the FP64 gap test below.
      const V4 xr = D.X4[j];
      const V4 ur = D.u4[cur][j];
      const float dx = (float)xr.x + (float)ur.x - (float)ss->c[0];
      const float dy = (float)xr.y + (float)ur.y - (float)ss->c[1];
      const float dz = (float)xr.z + (float)ur.z - (float)ss->c[2];
      const float mag = fabsf((float)xr.x) + fabsf((float)xr.y) + fabsf((float)xr.z);
      const float rr = (float)S->R + 0.05f + 4e-6f * mag;
      near = dx * dx + dy * dy + dz * dz < rr * rr;
    }
    if (near && S->has && (fl & 7) != 7) {
      // every load of the node and the striker is issued before the first
      // store (a store to the trial copy could alias them otherwise)
      double x[3], r2 = 0.0, dj[3], vj[3], w[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        dj[i] = d[i * nn + j];
        vj[i] = v[i * nn + j];
        w[i] = ss->w[i];
        x[i] = D.Xs[i * ns + s] + dj[i] - ss->c[i];
        r2 += x[i] * x[i];
      }
      const double r = sqrt(r2);
      const double gap = r - S->R;
      if (gap < 0.0 || was_active) {
        a = 1;
        const double ir = 1.0 / r;
        double n[3] = {x[0] * ir, x[1] * ir, x[2] * ir};
        double vn = 0.0, wn = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          D.trial[i * ns + s] = dj[i];
          D.trial[(3 + i) * ns + s] = vj[i];
          vn += vj[i] * n[i];
          wn += w[i] * n[i];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          if (!((fl >> i) & 1)) {
            dj[i] -= gap * n[i];
            vj[i] += (wn - vn) * n[i];
          }
          d[i * nn + j] = dj[i];
          v[i * nn + j] = vj[i];
          D.nrm[i * ns + s] = n[i];
        }
        V4 u;
        u.x = (T)dj[0];
        u.y = (T)dj[1];
        u.z = (T)dj[2];
        u.w = T(0);
        D.u4[cur][j] = u;
      }
    }
    D.act[spar][s] = a;
    return a != 0;
  } else {  // MODE_REPEAT: restore the released nodes to their trial state
    const bool on = D.act[spar][s] != 0;
    if (D.rel[s] && on) {
      double dj[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        dj[i] = D.trial[i * ns + s];
        d[i * nn + j] = dj[i];
        v[i * nn + j] = D.trial[(3 + i) * ns + s];
      }
      V4 u;
      u.x = (T)dj[0];
      u.y = (T)dj[1];
      u.z = (T)dj[2];
      u.w = T(0);
      D.u4[cur][j] = u;
      D.act[spar][s] = 0;
      // the elements of the released node are evaluated again; with
      // interfaces as node pairs its hexes, and the node on the other side of
      // its interface pair (whose jump changed) in the gather
      if (D.rmark_e != nullptr) {
        if (D.ipair == nullptr) {
          for (int k = D.row[j], k1 = D.row[j + 1]; k < k1; ++k) D.rmark_e[D.col[k] >> 3] = 1;
        } else {
          for (int k = D.row[j], k1 = D.row[j + 1]; k < k1; ++k) {
            const int32_t e = D.col[k] >> 3;
            if (e < D.nh) D.rmark_e[e] = 1;
          }
          const int32_t partner = D.ipair[j].x;
          if (partner >= 0) D.rmark_n[partner] = 1;
        }
      }
      return false;
    }
    return on;
  }
}

// ---------------------------------------------------------------------------
// Packed FP32 pairs: one sm_100-family instruction computes both lanes, each
// lane rounded exactly as the scalar operation.
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }

// Gauss point of lane l (0: xi < 0, 1: xi > 0) in xi-pair p (bit 0: eta > 0,
// bit 1: zeta > 0), in the point numbering of the node signs (sgn_x/y/z).
__host__ __device__ constexpr int pair_point(int p, int l) {
  return ((p >> 1) << 2) + ((p & 1) ? (l ? 2 : 3) : (l ? 1 : 0));
}

// The FP32 hex8 of an axis-aligned box, two Gauss points per step.  The two
// points of a pair differ only in the sign of xi, so the displacement
// gradient, the Green strain, both rotations, P = S F^T and the mode-space
// force sums run as packed pairs; the intralaminar law runs per point.
// Same formulation as the scalar element below (Eq. fcont, Algorithm 4).
// The compute of hex_item_box_pairs from the element's node displacements
// ua (by node) and the x-y-z extents of the box (corner 6 minus corner 0);
// the element's nodal forces f[8][3] are handed to store(f).
template <typename Store>
__device__ __forceinline__ void hex_box_pairs_core(const Dev<float> &D, const Mat<float> &M, int64_t e, int mode,
                                                   const float (&ua)[8][3], float ex, float ey, float ez,
                                                   bool pristine_in, int ply, Store &&store);

// Nodal forces of hex e (box, FP32) at the displacement mirror of the pass,
// handed to store(f, nd) with the element's node ids; false when a repeated
// pass does not evaluate it.
template <typename Store>
__device__ __forceinline__ bool hex_box_forces(const Dev<float> &D, const Mat<float> &M, int64_t e, int mode,
                                               Store &&store) {
  using V4 = float4;
  const Ctl *ctl = D.ctl;
  if (mode == MODE_REPEAT && !repeat_take(D.rmark_e, e)) return false;
  const int ub = (mode == MODE_FORCES) ? (ctl->dpar ^ 1) : ctl->dpar;
  const V4 *PDN_STATE_RESTRICT U = D.u4[ub];
  const int4 c0 = __ldg(reinterpret_cast<const int4 *>(D.hex) + 2 * e);
  const int4 c1 = __ldg(reinterpret_cast<const int4 *>(D.hex) + 2 * e + 1);
  const int nd[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  if (!nodes_in_range(D, nd)) return false;
  if (mode == MODE_REPEAT) repeat_mark_nodes(D.rmark_n, nd);
  float ua[8][3];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const V4 u = U[nd[a]];
    ua[a][0] = u.x;
    ua[a][1] = u.y;
    ua[a][2] = u.z;
  }
  const V4 x0 = D.X4[nd[0]], x6 = D.X4[nd[6]];
  const bool pristine_in = D.pflag[0] != nullptr && D.pflag[ctl->hpar][e] != 0;
  hex_box_pairs_core(D, M, e, mode, ua, x6.x - x0.x, x6.y - x0.y, x6.z - x0.z, pristine_in, D.ply[e],
                     [&](const float (&f)[8][3]) { store(f, nd); });
  return true;
}

__device__ __forceinline__ void hex_item_box_pairs(const Dev<float> &D, const Mat<float> &M, int64_t e, int mode) {
  if (e >= D.nh) return;
  const uint32_t rk = D.rank != nullptr ? __ldg(D.rank + e) : 0u;
  const int4 *pos2 = reinterpret_cast<const int4 *>(D.pos) + 2 * e;
  hex_box_forces(D, M, e, mode, [&](const float (&f)[8][3], const int (&nd)[8]) {
    int ps[8];
    element_slots(D, D.hex, e, pos2, rk, ps);
#pragma unroll
    for (int a = 0; a < 8; ++a) D.fe[ps[a]] = make_float4(f[a][0], f[a][1], f[a][2], 0.0f);
  });
}

template <typename Store>
__device__ __forceinline__ void hex_box_pairs_core(const Dev<float> &D, const Mat<float> &M, int64_t e, int mode,
                                                   const float (&ua)[8][3], float ex, float ey, float ez,
                                                   bool pristine_in, int ply, Store &&store) {
  const Ctl *ctl = D.ctl;
  const int64_t nh = D.nh;
  const int hb = ctl->hpar;
  const float *PDN_STATE_RESTRICT hin = D.hist[hb] + e;
  float *PDN_STATE_RESTRICT hout = D.hist[hb ^ 1] + e;
  bool dirty = false;
  float bm[8][3];
  float jd[3], wd[3], vol;
  {
    to_modes(ua, bm);
    const float J0 = 0.5f * ex, J1 = 0.5f * ey, J2 = 0.5f * ez;
    const float det = J0 * (J1 * J2);
    jd[0] = xrcp(J0);
    jd[1] = xrcp(J1);
    jd[2] = xrcp(J2);
    wd[0] = det * jd[0];
    wd[1] = det * jd[1];
    wd[2] = det * jd[2];
    vol = 8.0f * det;
  }
  const float cs = M.ply_c[ply], sn = M.ply_s[ply];
  const float c2 = cs * cs, s2 = sn * sn, csn = cs * sn;
  const ElemLaw<float> L = elem_law(M, e);
  float lc = -1.0f;
  // mode-space force sums
  float C[8][3];
#pragma unroll
  for (int m = 0; m < 8; ++m) C[m][0] = C[m][1] = C[m][2] = 0.0f;
  const float gp = 0.57735026918962576451f;
  const float2 xi = make_float2(-gp, gp);
#pragma unroll 1
  for (int p = 0; p < 4; ++p) {
    const int gx = pair_point(p, 0), gy = pair_point(p, 1);
    // the pair's history, in flight while the strains are computed; an
    // element with the initial history takes it without a load (a branch,
    // uniform over the warp wherever its elements are all pristine)
    float2 h[7];
    if (pristine_in) {
#pragma unroll
      for (int f = 0; f < 7; ++f) h[f] = p2(f < 4 ? 1.0f : 0.0f);
    } else {
#pragma unroll
      for (int f = 0; f < 7; ++f) h[f] = make_float2(hin[(int64_t)(f * 8 + gx) * nh], hin[(int64_t)(f * 8 + gy) * nh]);
    }
    const float et = (p & 1) ? gp : -gp, ze = (p & 2) ? gp : -gp;
    const float etze = et * ze;
    // H = du/dX: the xi column is the same in both lanes; the eta and zeta
    // columns are a + xi b
    float2 H[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      H[i][0] = p2((bm[1][i] + et * bm[4][i] + ze * bm[6][i] + etze * bm[7][i]) * jd[0]);
      const float a1 = (bm[2][i] + ze * bm[5][i]) * jd[1], b1 = (bm[4][i] + ze * bm[7][i]) * jd[1];
      const float a2 = (bm[3][i] + et * bm[5][i]) * jd[2], b2 = (bm[6][i] + et * bm[7][i]) * jd[2];
      H[i][1] = pfma(xi, p2(b1), p2(a1));
      H[i][2] = pfma(xi, p2(b2), p2(a2));
    }
    // Green strain E = 1/2 (H + H^T + H^T H), then to ply axes (rotation about z)
    float2 E[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = i; k < 3; ++k) {
        float2 t = padd(H[i][k], H[k][i]);
        t = pfma(H[0][i], H[0][k], t);
        t = pfma(H[1][i], H[1][k], t);
        t = pfma(H[2][i], H[2][k], t);
        E[i][k] = pmul(p2(0.5f), t);
      }
    float2 ep[6];
    ep[0] = pfma(p2(s2), E[1][1], pfma(p2(2.0f * csn), E[0][1], pmul(p2(c2), E[0][0])));
    ep[1] = pfma(p2(c2), E[1][1], pfma(p2(-2.0f * csn), E[0][1], pmul(p2(s2), E[0][0])));
    ep[2] = E[2][2];
    ep[3] = pfma(p2(2.0f * csn), E[1][1], pfma(p2(2.0f * (c2 - s2)), E[0][1], pmul(p2(-2.0f * csn), E[0][0])));
    ep[4] = pfma(p2(2.0f * sn), E[1][2], pmul(p2(2.0f * cs), E[0][2]));
    ep[5] = pfma(p2(2.0f * cs), E[1][2], pmul(p2(-2.0f * sn), E[0][2]));
    // the law.  Pristine points (initial history) that stay below yield and
    // below every onset, in both lanes, keep their history and take the
    // effective stress as nominal stress: the same tests as cdm_plastic and
    // cdm_damage with r = 1 and no plastic strain, in packed arithmetic.
    // Every other pair takes the full law, one point at a time.
    float2 sm[6];
    bool elastic = false;
    if (pristine_in) {
      const float2 s11 = pfma(p2(M.C13), ep[2], pfma(p2(M.C12), ep[1], pmul(p2(M.C11), ep[0])));
      const float2 s22 = pfma(p2(M.C23), ep[2], pfma(p2(M.C22), ep[1], pmul(p2(M.C12), ep[0])));
      const float2 s33 = pfma(p2(M.C33), ep[2], pfma(p2(M.C23), ep[1], pmul(p2(M.C13), ep[0])));
      const float2 s12 = pmul(p2(M.G12), ep[3]), s13 = pmul(p2(M.G13), ep[4]), s23 = pmul(p2(M.G23), ep[5]);
      bool ok = true;
      if (M.plasticity_on) {
        const float2 t12 = pmul(p2(M.G12), ep[3]), t13 = pmul(p2(M.G12), ep[4]);
        const float2 tn2 = pfma(t13, t13, pmul(t12, t12));
        const float ty2 = M.Sp * M.Sp;
        ok = tn2.x <= ty2 && tn2.y <= ty2;
      }
      if (ok && M.damage_on) {
        const float2 phiFT = pmul(pmul(p2(M.E1), ep[0]), p2(L.iXT));
        const float2 tl2 = pfma(s13, s13, pmul(s12, s12));
        const float2 a = pmul(s22, p2(L.iYT));
        const float2 s23q = pmul(pmul(s23, s23), p2(M.iST2));
        // matrix tension: (1-g) a + g a^2 + tauL^2/SL^2 + s23^2/ST^2
        const float2 qmt = padd(pfma(tl2, p2(L.iSL2), pfma(pmul(p2(M.g), a), a, pmul(p2(M.g1), a))), s23q);
        // matrix compression: the bound (tT^2 + s23^2)/ST^2 + tauL^2/SL^2
        const float tTx = fmaxf(-s22.x * M.kT, 0.0f), tTy = fmaxf(-s22.y * M.kT, 0.0f);
        const float2 tT = make_float2(tTx, tTy);
        const float2 qmc = pfma(tl2, p2(L.iSL2), pmul(pfma(tT, tT, pmul(s23, s23)), p2(M.iST2)));
        const float qx = s22.x >= 0.0f ? qmt.x : qmc.x, qy = s22.y >= 0.0f ? qmt.y : qmc.y;
        const float fcx = fmaxf(-s11.x, 0.0f) * M.iXC, fcy = fmaxf(-s11.y, 0.0f) * M.iXC;
        ok = phiFT.x <= 1.0f && phiFT.y <= 1.0f && fcx <= 1.0f && fcy <= 1.0f && qx <= 1.0f && qy <= 1.0f;
      }
      if (ok) {
        sm[0] = s11;
        sm[1] = s22;
        sm[2] = s33;
        sm[3] = s12;
        sm[4] = s13;
        sm[5] = s23;
        elastic = true;
      }
    }
    if (!elastic) {
      float el[6], hl[7], sl[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) el[k] = ep[k].x;
#pragma unroll
      for (int f = 0; f < 7; ++f) hl[f] = h[f].x;
      cdm(M, L, (const float(*)[3]) nullptr, vol, lc, el, hl, sl);
#pragma unroll
      for (int k = 0; k < 6; ++k) sm[k].x = sl[k];
#pragma unroll
      for (int f = 0; f < 7; ++f) h[f].x = hl[f];
#pragma unroll
      for (int k = 0; k < 6; ++k) el[k] = ep[k].y;
#pragma unroll
      for (int f = 0; f < 7; ++f) hl[f] = h[f].y;
      cdm(M, L, (const float(*)[3]) nullptr, vol, lc, el, hl, sl);
#pragma unroll
      for (int k = 0; k < 6; ++k) sm[k].y = sl[k];
#pragma unroll
      for (int f = 0; f < 7; ++f) h[f].y = hl[f];
    }
    if (!pristine_in) {
#pragma unroll
      for (int f = 0; f < 7; ++f) {
        hout[(int64_t)(f * 8 + gx) * nh] = h[f].x;
        hout[(int64_t)(f * 8 + gy) * nh] = h[f].y;
      }
    } else {
      // a pair that passed the elastic test kept the initial history
      const bool changed = !elastic &&
                           (h[0].x > 1.0f || h[1].x > 1.0f || h[2].x > 1.0f || h[3].x > 1.0f || h[4].x != 0.0f ||
                            h[5].x != 0.0f || h[6].x != 0.0f || h[0].y > 1.0f || h[1].y > 1.0f ||
                            h[2].y > 1.0f || h[3].y > 1.0f || h[4].y != 0.0f || h[5].y != 0.0f || h[6].y != 0.0f);
      if (changed && !dirty) {
        // first change in a pristine element: the points of the earlier
        // pairs keep the initial history, not yet in the output buffer
        for (int q = 0; q < p; ++q)
#pragma unroll
          for (int f = 0; f < 7; ++f) {
            hout[(int64_t)(f * 8 + pair_point(q, 0)) * nh] = f < 4 ? 1.0f : 0.0f;
            hout[(int64_t)(f * 8 + pair_point(q, 1)) * nh] = f < 4 ? 1.0f : 0.0f;
          }
        dirty = true;
      }
      if (dirty) {
#pragma unroll
        for (int f = 0; f < 7; ++f) {
          hout[(int64_t)(f * 8 + gx) * nh] = h[f].x;
          hout[(int64_t)(f * 8 + gy) * nh] = h[f].y;
        }
      }
    }
    // back to global axes: S = R Sm R^T
    float2 S[3][3];
    S[0][0] = pfma(p2(s2), sm[1], pfma(p2(-2.0f * csn), sm[3], pmul(p2(c2), sm[0])));
    S[1][1] = pfma(p2(c2), sm[1], pfma(p2(2.0f * csn), sm[3], pmul(p2(s2), sm[0])));
    S[2][2] = sm[2];
    S[0][1] = S[1][0] = pfma(p2(-csn), sm[1], pfma(p2(c2 - s2), sm[3], pmul(p2(csn), sm[0])));
    S[0][2] = S[2][0] = pfma(p2(-sn), sm[5], pmul(p2(cs), sm[4]));
    S[1][2] = S[2][1] = pfma(p2(cs), sm[5], pmul(p2(sn), sm[4]));
    // P = S F^T with F = I + H
    float2 P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        P[i][k] = pfma(S[i][2], H[k][2], pfma(S[i][1], H[k][1], pfma(S[i][0], H[k][0], S[i][k])));
    // mode sums of Q_k = w_k P_k (w_k = det J / J_kk) times the Gauss-point
    // values of the mode derivatives; the lanes enter through their sum
    // (xi-even modes) and difference (xi-odd modes)
    const float e0 = et * wd[0], z1 = ze * wd[1], e2 = et * wd[2], z0 = ze * wd[0], ez0 = etze * wd[0];
    const float g1 = gp * wd[1], g2 = gp * wd[2], gz1 = g1 * ze, ge2 = g2 * et;
    // components 0 and 1 as a packed pair, component 2 alone
    {
      const float2 s0 = make_float2(P[0][0].x + P[0][0].y, P[0][1].x + P[0][1].y);
      const float2 s1 = make_float2(P[1][0].x + P[1][0].y, P[1][1].x + P[1][1].y);
      const float2 s2s = make_float2(P[2][0].x + P[2][0].y, P[2][1].x + P[2][1].y);
      const float2 d1 = make_float2(P[1][0].y - P[1][0].x, P[1][1].y - P[1][1].x);
      const float2 d2 = make_float2(P[2][0].y - P[2][0].x, P[2][1].y - P[2][1].x);
      float2 c;
      c = pfma(p2(wd[0]), s0, make_float2(C[1][0], C[1][1]));
      C[1][0] = c.x, C[1][1] = c.y;
      c = pfma(p2(wd[1]), s1, make_float2(C[2][0], C[2][1]));
      C[2][0] = c.x, C[2][1] = c.y;
      c = pfma(p2(wd[2]), s2s, make_float2(C[3][0], C[3][1]));
      C[3][0] = c.x, C[3][1] = c.y;
      c = padd(make_float2(C[4][0], C[4][1]), pfma(p2(g1), d1, pmul(p2(e0), s0)));
      C[4][0] = c.x, C[4][1] = c.y;
      c = padd(make_float2(C[5][0], C[5][1]), pfma(p2(e2), s2s, pmul(p2(z1), s1)));
      C[5][0] = c.x, C[5][1] = c.y;
      c = padd(make_float2(C[6][0], C[6][1]), pfma(p2(g2), d2, pmul(p2(z0), s0)));
      C[6][0] = c.x, C[6][1] = c.y;
      c = padd(make_float2(C[7][0], C[7][1]), pfma(p2(ge2), d2, pfma(p2(gz1), d1, pmul(p2(ez0), s0))));
      C[7][0] = c.x, C[7][1] = c.y;
    }
    {
      const float s0 = P[0][2].x + P[0][2].y, s1 = P[1][2].x + P[1][2].y, s2s = P[2][2].x + P[2][2].y;
      const float d1 = P[1][2].y - P[1][2].x, d2 = P[2][2].y - P[2][2].x;
      C[1][2] = fmaf(wd[0], s0, C[1][2]);
      C[2][2] = fmaf(wd[1], s1, C[2][2]);
      C[3][2] = fmaf(wd[2], s2s, C[3][2]);
      C[4][2] = C[4][2] + fmaf(g1, d1, e0 * s0);
      C[5][2] = C[5][2] + fmaf(e2, s2s, z1 * s1);
      C[6][2] = C[6][2] + fmaf(g2, d2, z0 * s0);
      C[7][2] = C[7][2] + fmaf(ge2, d2, fmaf(gz1, d1, ez0 * s0));
    }
  }
  if (D.pflag[0] != nullptr) D.pflag[hb ^ 1][e] = (pristine_in && !dirty) ? 1 : 0;
  float f[8][3];
  from_modes(C, f);
  store(f);
}

// ---------------------------------------------------------------------------
// Kernel 2: hex8 internal forces, total Lagrangian, 2x2x2 Gauss (Sec. 2,
// Eq. fcont), with the intralaminar law per Gauss point.  One thread per
// element; geometry and displacement enter through their trilinear modes, so
// that J = [dx/dxi], du/dxi and the returned force are cheap mode sums.
// f_a = sum_g sum_k dN_a/dxi_k Q_g[k][:],  Q_g = det J_g  J_g^-1 P_g,
// P = S F^T (nominal stress), S rotated from ply axes (angle about z).
// BOX: every element is an axis-aligned box (checked on the host), so J is
// the constant diagonal diag((x6-x0)/2, (y6-y0)/2, (z6-z0)/2).
// The next Gauss point's history is loaded while the current one computes.
template <typename T, bool BOX>
__device__ __forceinline__ void hex_item(const Dev<T> &D, const Mat<T> &M, int64_t e, int mode) {
  if constexpr (BOX && std::is_same<T, float>::value) {
    hex_item_box_pairs(D, M, e, mode);
    return;
  }
  using V4 = typename Vec4T<T>::type;
  const Ctl *ctl = D.ctl;
  if (e >= D.nh) return;
  if (mode == MODE_REPEAT && !repeat_take(D.rmark_e, e)) return;
  const int64_t nh = D.nh;
  const int ub = (mode == MODE_FORCES) ? (ctl->dpar ^ 1) : ctl->dpar;
  const int hb = ctl->hpar;
  const V4 *PDN_STATE_RESTRICT U = D.u4[ub];
  const int4 c0 = __ldg(reinterpret_cast<const int4 *>(D.hex) + 2 * e);
  const int4 c1 = __ldg(reinterpret_cast<const int4 *>(D.hex) + 2 * e + 1);
  const int nd[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  if (!nodes_in_range(D, nd)) return;
  if (mode == MODE_REPEAT) repeat_mark_nodes(D.rmark_n, nd);
  const T *PDN_STATE_RESTRICT hin = D.hist[hb] + e;
  T *PDN_STATE_RESTRICT hout = D.hist[hb ^ 1] + e;
  // An element whose points all still hold the initial history skips the
  // history traffic: it is not read, and written only once a point changes.
  const bool pristine_in = D.pflag[0] != nullptr && D.pflag[hb][e] != 0;
  bool dirty = false;
  // history of Gauss point 0 in flight first
  T hn[7];
#pragma unroll
  for (int f = 0; f < 7; ++f) hn[f] = pristine_in ? (f < 4 ? T(1) : T(0)) : hin[(int64_t)(f * 8) * nh];
  T am[8][3], bm[8][3];
  T jd[3] = {T(0), T(0), T(0)}, wd[3] = {T(0), T(0), T(0)}, vol = T(0);
  {
    T ua[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const V4 u = U[nd[a]];
      ua[a][0] = u.x;
      ua[a][1] = u.y;
      ua[a][2] = u.z;
    }
    to_modes(ua, bm);
    if constexpr (BOX) {
      const V4 x0 = D.X4[nd[0]], x6 = D.X4[nd[6]];
      const T J0 = T(0.5) * (x6.x - x0.x), J1 = T(0.5) * (x6.y - x0.y), J2 = T(0.5) * (x6.z - x0.z);
      const T det = J0 * (J1 * J2);
      jd[0] = T(1) / J0;
      jd[1] = T(1) / J1;
      jd[2] = T(1) / J2;
      wd[0] = det * jd[0];
      wd[1] = det * jd[1];
      wd[2] = det * jd[2];
      vol = T(8) * det;
    } else {
      T xa[8][3];
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const V4 x = D.X4[nd[a]];
        xa[a][0] = x.x;
        xa[a][1] = x.y;
        xa[a][2] = x.z;
      }
      to_modes(xa, am);
    }
  }
  const int ply = D.ply[e];
  const T cs = M.ply_c[ply], sn = M.ply_s[ply];
  const T c2 = cs * cs, s2 = sn * sn, csn = cs * sn;
  const ElemLaw<T> L = elem_law(M, e);
  T lc = T(-1);
  T C[8][3];
#pragma unroll
  for (int m = 0; m < 8; ++m) C[m][0] = C[m][1] = C[m][2] = T(0);
  const T gp = T(0.57735026918962576451);
#pragma unroll 1
  for (int g = 0; g < 8; ++g) {
    T h[7];
#pragma unroll
    for (int f = 0; f < 7; ++f) h[f] = hn[f];
    if (g < 7 && !pristine_in) {
#pragma unroll
      for (int f = 0; f < 7; ++f) hn[f] = hin[(int64_t)(f * 8 + g + 1) * nh];
    }
    const T xi = T(sgn_x(g)) * gp, et = T(sgn_y(g)) * gp, ze = T(sgn_z(g)) * gp;
    T Du[3][3], H[3][3], Ji[3][3], det = T(0);
    jac_cols(bm, xi, et, ze, Du);
    if constexpr (BOX) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) H[i][k] = Du[i][k] * jd[k];
    } else {
      T J[3][3];
      jac_cols(am, xi, et, ze, J);
      det = det3(J);
      const T id = T(1) / det;
      Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
      Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
      Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
      Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
      Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
      Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
      Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
      Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
      Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) H[i][k] = Du[i][0] * Ji[0][k] + Du[i][1] * Ji[1][k] + Du[i][2] * Ji[2][k];
    }
    // Green strain E = 1/2 (H + H^T + H^T H)
    T E[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = i; k < 3; ++k) {
        E[i][k] = T(0.5) * (H[i][k] + H[k][i] + H[0][i] * H[0][k] + H[1][i] * H[1][k] + H[2][i] * H[2][k]);
        E[k][i] = E[i][k];
      }
    // to ply axes (rotation about z): Em = R^T E R
    T ep[6];
    ep[0] = c2 * E[0][0] + T(2) * csn * E[0][1] + s2 * E[1][1];
    ep[1] = s2 * E[0][0] - T(2) * csn * E[0][1] + c2 * E[1][1];
    ep[2] = E[2][2];
    ep[3] = T(2) * (-csn * E[0][0] + (c2 - s2) * E[0][1] + csn * E[1][1]);
    ep[4] = T(2) * (cs * E[0][2] + sn * E[1][2]);
    ep[5] = T(2) * (-sn * E[0][2] + cs * E[1][2]);
    T sm[6];
    if constexpr (BOX)
      cdm(M, L, (const T(*)[3]) nullptr, vol, lc, ep, h, sm);
    else
      cdm(M, L, (const T(*)[3])am, T(0), lc, ep, h, sm);
    if (!pristine_in) {
#pragma unroll
      for (int f = 0; f < 7; ++f) hout[(int64_t)(f * 8 + g) * nh] = h[f];
    } else {
      const bool changed = h[0] > T(1) || h[1] > T(1) || h[2] > T(1) || h[3] > T(1) || h[4] != T(0) ||
                           h[5] != T(0) || h[6] != T(0);
      if (changed && !dirty) {
        // first change in a pristine element: the earlier points keep the
        // initial history, which the output buffer does not hold yet
        for (int gg = 0; gg < g; ++gg)
#pragma unroll
          for (int f = 0; f < 7; ++f) hout[(int64_t)(f * 8 + gg) * nh] = f < 4 ? T(1) : T(0);
        dirty = true;
      }
      if (dirty) {
#pragma unroll
        for (int f = 0; f < 7; ++f) hout[(int64_t)(f * 8 + g) * nh] = h[f];
      }
    }
    // back to global axes: S = R Sm R^T
    T S[3][3];
    S[0][0] = c2 * sm[0] - T(2) * csn * sm[3] + s2 * sm[1];
    S[1][1] = s2 * sm[0] + T(2) * csn * sm[3] + c2 * sm[1];
    S[2][2] = sm[2];
    S[0][1] = S[1][0] = csn * sm[0] + (c2 - s2) * sm[3] - csn * sm[1];
    S[0][2] = S[2][0] = cs * sm[4] - sn * sm[5];
    S[1][2] = S[2][1] = sn * sm[4] + cs * sm[5];
    // P = S F^T with F = I + H; Q = det J^-1 P
    T P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        P[i][k] = S[i][k] + S[i][0] * H[k][0] + S[i][1] * H[k][1] + S[i][2] * H[k][2];
    T Q[3][3];
    if constexpr (BOX) {
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int I = 0; I < 3; ++I) Q[k][I] = wd[k] * P[k][I];
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int I = 0; I < 3; ++I) Q[k][I] = det * (Ji[k][0] * P[0][I] + Ji[k][1] * P[1][I] + Ji[k][2] * P[2][I]);
    }
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
  if (D.pflag[0] != nullptr) D.pflag[hb ^ 1][e] = (pristine_in && !dirty) ? 1 : 0;
  T f[8][3];
  from_modes(C, f);
  // element forces go straight to their CSR positions, so that the gather
  // reads each node's contributions as one contiguous run
  const int4 p0 = __ldg(reinterpret_cast<const int4 *>(D.pos) + 2 * e);
  const int4 p1 = __ldg(reinterpret_cast<const int4 *>(D.pos) + 2 * e + 1);
  const int ps[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    V4 o;
    o.x = f[a][0];
    o.y = f[a][1];
    o.z = f[a][2];
    o.w = T(0);
    D.fe[ps[a]] = o;
  }
}

// ---------------------------------------------------------------------------
// Kernel 3: zero-thickness interface elements with Newton-Cotes integration
// (Sec. 2.3.2) and the cohesive law (Algorithm 5).  One thread per element.
// FLAT: every interface is a flat axis-aligned rectangle (Dev::all_flat_coh):
// the frame is the global axes and all four area weights are Lx Ly / 4, so
// only two corners of the geometry are read and no root is taken.
// Nodal forces of interface element c at the displacement mirror of the
// pass, handed to store(f, nd) with the element's node ids; false when a
// repeated pass does not evaluate it.
template <typename T, bool FLAT, typename Store>
__device__ __forceinline__ bool coh_forces(const Dev<T> &D, const Mat<T> &M, int64_t c, int mode, Store &&store) {
  using V4 = typename Vec4T<T>::type;
  const Ctl *ctl = D.ctl;
  if (mode == MODE_REPEAT && !repeat_take(D.rmark_e, D.nh + c)) return false;
  const int64_t nc = D.nc;
  const int ub = (mode == MODE_FORCES) ? (ctl->dpar ^ 1) : ctl->dpar;
  const int hb = ctl->hpar;
  const V4 *PDN_STATE_RESTRICT U = D.u4[ub];
  const int4 c0 = __ldg(reinterpret_cast<const int4 *>(D.coh) + 2 * c);
  const int4 c1 = __ldg(reinterpret_cast<const int4 *>(D.coh) + 2 * c + 1);
  const int nd[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  if (!nodes_in_range(D, nd)) return false;
  if (mode == MODE_REPEAT) repeat_mark_nodes(D.rmark_n, nd);
  constexpr int QX[4] = {-1, 1, 1, -1}, QY[4] = {-1, -1, 1, 1};
  // the upper face coincides with the lower one in the reference
  // configuration (zero thickness), so the lower face gives the mid-surface
  T xm[4][3], uu[8][3];
  if constexpr (FLAT) {
    const V4 x0 = D.X4[nd[0]], x2 = D.X4[nd[2]];
    xm[0][0] = x0.x;
    xm[0][1] = x0.y;
    xm[2][0] = x2.x;
    xm[2][1] = x2.y;
  } else {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const V4 xb = D.X4[nd[a]];
      xm[a][0] = xb.x;
      xm[a][1] = xb.y;
      xm[a][2] = xb.z;
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const V4 u = U[nd[a]];
    uu[a][0] = u.x;
    uu[a][1] = u.y;
    uu[a][2] = u.z;
  }
  // frame at the element centre
  T e1[3], e2[3], e3[3];
  if constexpr (!FLAT) {
    T tx[3] = {T(0), T(0), T(0)}, ty[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        tx[i] += T(0.25) * T(QX[a]) * xm[a][i];
        ty[i] += T(0.25) * T(QY[a]) * xm[a][i];
      }
    const T n0 = tx[1] * ty[2] - tx[2] * ty[1], n1 = tx[2] * ty[0] - tx[0] * ty[2],
            n2 = tx[0] * ty[1] - tx[1] * ty[0];
    const T inn = T(1) / xsqrt(n0 * n0 + n1 * n1 + n2 * n2);
    const T itn = T(1) / xsqrt(tx[0] * tx[0] + tx[1] * tx[1] + tx[2] * tx[2]);
    e3[0] = n0 * inn;
    e3[1] = n1 * inn;
    e3[2] = n2 * inn;
#pragma unroll
    for (int i = 0; i < 3; ++i) e1[i] = tx[i] * itn;
    e2[0] = e3[1] * e1[2] - e3[2] * e1[1];
    e2[1] = e3[2] * e1[0] - e3[0] * e1[2];
    e2[2] = e3[0] * e1[1] - e3[1] * e1[0];
  }
  const T *PDN_STATE_RESTRICT rin = D.rD[hb];
  T *PDN_STATE_RESTRICT rout = D.rD[hb ^ 1];
  // undamaged interface elements (all r_D = 0) skip the threshold traffic
  const bool pristine_in = D.cflag[0] != nullptr && D.cflag[hb][c] != 0;
  T rv[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) rv[p] = pristine_in ? T(0) : rin[(int64_t)p * nc + c];
  T f[8][3];
  if constexpr (FLAT) {
    const T w = T(0.25) * (xm[2][0] - xm[0][0]) * (xm[2][1] - xm[0][1]);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const T dl[3] = {uu[p + 4][0] - uu[p][0], uu[p + 4][1] - uu[p][1], uu[p + 4][2] - uu[p][2]};
      T tau[3], r1;
      czm(M, dl, rv[p], r1, tau);
      rv[p] = r1;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const T tg = rmul(w, tau[i]);  // rounded alone, as in the node-pair gather
        f[p + 4][i] = tg;
        f[p][i] = -tg;
      }
    }
  } else {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const T xi = T(QX[p]), et = T(QY[p]);
    T tx[3] = {T(0), T(0), T(0)}, ty[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const T dxi = T(0.25) * T(QX[a]) * (T(1) + et * T(QY[a]));
      const T deta = T(0.25) * T(QY[a]) * (T(1) + xi * T(QX[a]));
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        tx[i] += dxi * xm[a][i];
        ty[i] += deta * xm[a][i];
      }
    }
    const T n0 = tx[1] * ty[2] - tx[2] * ty[1], n1 = tx[2] * ty[0] - tx[0] * ty[2],
            n2 = tx[0] * ty[1] - tx[1] * ty[0];
    const T w = xsqrt(n0 * n0 + n1 * n1 + n2 * n2);
    const T dg0 = uu[p + 4][0] - uu[p][0], dg1 = uu[p + 4][1] - uu[p][1], dg2 = uu[p + 4][2] - uu[p][2];
    const T dl[3] = {e1[0] * dg0 + e1[1] * dg1 + e1[2] * dg2, e2[0] * dg0 + e2[1] * dg1 + e2[2] * dg2,
                     e3[0] * dg0 + e3[1] * dg1 + e3[2] * dg2};
    T tau[3], r1;
    czm(M, dl, rv[p], r1, tau);
    rv[p] = r1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T tg = w * (tau[0] * e1[i] + tau[1] * e2[i] + tau[2] * e3[i]);
      f[p + 4][i] = tg;
      f[p][i] = -tg;
    }
  }
  }
  const bool still = pristine_in && rv[0] == T(0) && rv[1] == T(0) && rv[2] == T(0) && rv[3] == T(0);
  if (!still) {
#pragma unroll
    for (int p = 0; p < 4; ++p) rout[(int64_t)p * nc + c] = rv[p];
  }
  if (D.cflag[0] != nullptr) D.cflag[hb ^ 1][c] = still ? 1 : 0;
  store(f, nd);
  return true;
}

template <typename T, bool FLAT>
__device__ __forceinline__ void coh_item(const Dev<T> &D, const Mat<T> &M, int64_t c, int mode) {
  using V4 = typename Vec4T<T>::type;
  if (c >= D.nc) return;
  const uint32_t rk = D.rank != nullptr ? __ldg(D.rank + D.nh + c) : 0u;
  coh_forces<T, FLAT>(D, M, c, mode, [&](const T (&f)[8][3], const int (&nd)[8]) {
    int ps[8];
    element_slots(D, D.coh, c, reinterpret_cast<const int4 *>(D.pos) + 2 * (D.nh + c), rk, ps);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      V4 o;
      o.x = f[a][0];
      o.y = f[a][1];
      o.z = f[a][2];
      o.w = T(0);
      D.fe[ps[a]] = o;
    }
  });
}

// ---------------------------------------------------------------------------
// Tail of a pass (one block, after the gather).  Sums the reactions of the
// active contact nodes in surface order (each thread a contiguous range, then
// a fixed tree), counts the adhesive ones, then commits the step (contact
// force F = sum lambda_j n_j to the striker, Sec. 2.2.2; step counter,
// history and node-buffer parities, force history), or marks the step for
// repetition when adhesive nodes were released (Algorithm 2: the MPI_MAX of
// kfl_reset becomes this single-block decision), or halts.  On commit it also
// advances the striker for the next pass (RK4 with the committed force).
// The 0/1 flag bytes of 16 consecutive surface nodes as a 16-bit mask, bit b
// for node b: per 32-bit part, the multiply moves the low bits of its four
// bytes (0, 8, 16, 24) to bits 21..24 with no two partial products on the
// same bit, so there is no carry.
__device__ __forceinline__ uint32_t flag_mask16(uint4 q) {
  const auto four = [](uint32_t x) { return (((x & 0x01010101u) * 0x00204081u) >> 21) & 0xFu; };
  return four(q.x) | (four(q.y) << 4) | (four(q.z) << 8) | (four(q.w) << 12);
}

// RUNS: build the list from the contact kernel's per-run counts when the
// context has them (the per-pass kernel); the batched kernel, whose contact
// tiles do not count, instantiates the flag-word scan alone and so does not
// carry the runs' shared arrays.
template <typename T, bool RUNS = false>
__device__ void tail_block(const Dev<T> &D, int mode) {
  Ctl *ctl = D.ctl;
  // the control block and the striker are read once, early, into registers;
  // the striker only by passes that can commit a step (an internal-force
  // evaluation may have no striker at all: D.imp is then null)
  const bool stepping = (mode == MODE_ADVANCE || mode == MODE_REPEAT);
  Ctl c;
  Striker S;
  StrikerStep ss;
  int nf = 0;
  if (threadIdx.x == 0) {
    // the pass's non-finite flag (raised by the gather, which has completed)
    // is read here, early, so that its latency overlaps the reduction
    nf = *(volatile int *)&ctl->nonfinite;
    c = *ctl;
    if (stepping) {
      S = *D.imp;
      ss = *D.imp_step;
    }
  }
  // Reaction sum over the active contact nodes in a fixed order that does
  // not depend on the launch shape: the active nodes are listed in surface
  // order (flags counted per range of 16-flag words, ranges prefix-summed,
  // indices written in order); list entry i goes to virtual lane i mod
  // kTailLanes, each lane sums its entries in list order, lanes are reduced
  // by xor-shuffles within groups of 32 and the groups in order.  A block of
  // any size that divides kTailLanes (>= 32) plays the lanes in turn.  The
  // list lets every thread issue its loads of lambda and n together; when
  // more than kTailCap nodes are active, each lane instead sums the active
  // nodes of its own word range in order.
  constexpr int kTailLanes = 256;
  constexpr int kTailCap = 4096;
  __shared__ double tf[3][kTailLanes / 32];
  __shared__ int ti[2][kTailLanes / 32];
  __shared__ int s_off[kTailLanes];
  __shared__ int s_list[kTailCap];
  const int64_t ns = D.ns;
  const int64_t words = (ns + 15) / 16;
  const int64_t per = (words + kTailLanes - 1) / kTailLanes;
  // the flag arrays are 256-byte aligned, sized to a multiple of 16 bytes,
  // and hold 0 or 1 per node
  const uint4 *aw = stepping ? reinterpret_cast<const uint4 *>(D.act[(int)((ctl->step + 1) & 1)]) : nullptr;
  int total = 0;
  // With the contact kernel's counts per run of kActRun surface nodes, the
  // list is built from them: an exclusive prefix over the runs, then the
  // warps take the non-empty runs and read a run's 16 flag words with one
  // load per lane of a half-warp, writing the run's nodes in surface order
  // from the run's offset.  The list is the same as the one the flag
  // words alone give (below); only fewer words are read, and in fewer rounds.
  bool listed = false;
  if constexpr (RUNS) {
    constexpr int kRunWords = kActRun / 16;
    constexpr int kRunCap = 2048;
    static_assert(kRunWords == 16, "a run is one flag word per lane of a half-warp");
    __shared__ int s_pre[kRunCap + 1];
    __shared__ int s_wsum[32];
    const int64_t nrun = (ns + kActRun - 1) / kActRun;
    if (stepping && D.act_cnt != nullptr && nrun <= kRunCap) {
      listed = true;
      const int nt = (int)blockDim.x, lane = (int)threadIdx.x & 31, wid = (int)threadIdx.x >> 5;
      const int nw = (nt + 31) >> 5;
      const int64_t pr = (nrun + nt - 1) / nt;
      const int64_t r0 = (int64_t)threadIdx.x * pr;
      const int64_t r1 = r0 + pr < nrun ? r0 + pr : nrun;
      int tsum = 0;
#pragma unroll 4
      for (int64_t r = r0; r < r1; ++r) tsum += D.act_cnt[r];
      int inc = tsum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      if (lane == 31) s_wsum[wid] = inc;
      __syncthreads();
      if (wid == 0) {
        const int x = lane < nw ? s_wsum[lane] : 0;
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, xi, o);
          if (lane >= o) xi += t;
        }
        if (lane < nw) s_wsum[lane] = xi - x;
        if (lane == nw - 1) s_pre[nrun] = xi;
      }
      __syncthreads();
      int run_base = s_wsum[wid] + inc - tsum;
      for (int64_t r = r0; r < r1; ++r) {
        s_pre[r] = run_base;
        run_base += D.act_cnt[r];
      }
      __syncthreads();
      total = s_pre[nrun];
      if (total <= kTailCap) {
        // warp wid looks at runs wid, wid + nw, wid + 2 nw, ... (32 per ballot),
        // so that the runs of one contact patch spread over the warps; each
        // half-warp reads one non-empty run (one flag word per lane)
        const int half = lane >> 4, hl = lane & 15;
        for (int64_t g = 0; wid + (int64_t)nw * 32 * g < nrun; ++g) {
          const int64_t r = wid + (int64_t)nw * (32 * g + lane);
          uint32_t todo = __ballot_sync(0xffffffffu, r < nrun && s_pre[r + 1] > s_pre[r]);
          while (todo != 0u) {
            const int ka = __ffs(todo) - 1;
            todo &= todo - 1u;
            int kb = -1;
            if (todo != 0u) {
              kb = __ffs(todo) - 1;
              todo &= todo - 1u;
            }
            const int k = half ? kb : ka;
            const int64_t rr = wid + (int64_t)nw * (32 * g + (k < 0 ? 0 : k));
            const int64_t w = rr * kRunWords + hl;
            const uint32_t m = (k >= 0 && w < words) ? flag_mask16(aw[w]) : 0u;
            const int c = __popc(m);
            int ci = c;
#pragma unroll
            for (int o = 1; o < 16; o <<= 1) {
              const int t = __shfl_up_sync(0xffffffffu, ci, o, 16);
              if (hl >= o) ci += t;
            }
            int o = (k >= 0 ? s_pre[rr] : 0) + ci - c;
            for (uint32_t mm = m; mm != 0u; mm &= mm - 1u, ++o)
              if (o < kTailCap) s_list[o] = (int)(w * 16 + __ffs(mm) - 1);
          }
        }
        __syncthreads();
      }
    }
  }
  if (stepping && !listed) {
    for (int v0 = 0; v0 < kTailLanes; v0 += blockDim.x) {
      const int v = v0 + (int)threadIdx.x;
      const int64_t w0 = (int64_t)v * per;
      const int64_t w1 = w0 + per < words ? w0 + per : words;
      int cnt = 0;
#pragma unroll 4
      for (int64_t wi = w0; wi < w1; ++wi) {
        const uint4 q = aw[wi];
        cnt += __popc(q.x & 0x01010101u) + __popc(q.y & 0x01010101u) + __popc(q.z & 0x01010101u) +
               __popc(q.w & 0x01010101u);
      }
      s_off[v] = cnt;
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive prefix over the lanes, 8 per thread
      const int l = threadIdx.x;
      int loc[kTailLanes / 32], acc = 0;
#pragma unroll
      for (int k = 0; k < kTailLanes / 32; ++k) {
        loc[k] = acc;
        acc += s_off[l * (kTailLanes / 32) + k];
      }
      int inc = acc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (l >= o) inc += t;
      }
      const int base = inc - acc;
#pragma unroll
      for (int k = 0; k < kTailLanes / 32; ++k) s_off[l * (kTailLanes / 32) + k] = base + loc[k];
      if (l == 31) s_list[0] = inc;  // total, read below before the list is written
    }
    __syncthreads();
    total = s_list[0];
    __syncthreads();
    if (total <= kTailCap) {
      for (int v0 = 0; v0 < kTailLanes; v0 += blockDim.x) {
        const int v = v0 + (int)threadIdx.x;
        const int64_t w0 = (int64_t)v * per;
        const int64_t w1 = w0 + per < words ? w0 + per : words;
        int o = s_off[v];
#pragma unroll 4
        for (int64_t wi = w0; wi < w1; ++wi) {
          for (uint32_t m = flag_mask16(aw[wi]); m != 0u; m &= m - 1u) s_list[o++] = (int)(wi * 16 + __ffs(m) - 1);
        }
      }
      __syncthreads();
    }
  }
  for (int v0 = 0; v0 < kTailLanes; v0 += blockDim.x) {
    const int v = v0 + (int)threadIdx.x;  // virtual lane
    double f0 = 0.0, f1 = 0.0, f2 = 0.0;
    int nact = 0, nadh = 0;
    if (stepping && total <= kTailCap) {
      // the lane's entries in list order, kTailBatch at a time: every load of
      // a batch (lambda and the normal of each entry) is issued before any
      // is used, so a batch costs one round of memory latency
      constexpr int kTailBatch = 4;
      for (int i0 = v; i0 < total; i0 += kTailBatch * kTailLanes) {
        double lam[kTailBatch], n0[kTailBatch], n1[kTailBatch], n2[kTailBatch];
#pragma unroll
        for (int u = 0; u < kTailBatch; ++u) {
          const int i = i0 + u * kTailLanes;
          int64_t s = i < total ? s_list[i] : 0;
          s = (s >= 0 && s < ns) ? s : 0;  // a list entry is always a surface index
          lam[u] = i < total ? D.lam[s] : 0.0;
          n0[u] = i < total ? D.nrm[s] : 0.0;
          n1[u] = i < total ? D.nrm[ns + s] : 0.0;
          n2[u] = i < total ? D.nrm[2 * ns + s] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kTailBatch; ++u) {
          if (i0 + u * kTailLanes >= total) break;
          if (lam[u] < 0.0) {
            ++nadh;
          } else {
            ++nact;
            f0 += lam[u] * n0[u];
            f1 += lam[u] * n1[u];
            f2 += lam[u] * n2[u];
          }
        }
      }
    } else if (stepping) {
      const int64_t w0 = (int64_t)v * per;
      const int64_t w1 = w0 + per < words ? w0 + per : words;
      for (int64_t wi = w0; wi < w1; ++wi) {
        for (uint32_t m = flag_mask16(aw[wi]); m != 0u; m &= m - 1u) {
          const int64_t s = wi * 16 + __ffs(m) - 1;
          const double lam = D.lam[s];
          if (lam < 0.0) {
            ++nadh;
          } else {
            ++nact;
            f0 += lam * D.nrm[s];
            f1 += lam * D.nrm[ns + s];
            f2 += lam * D.nrm[2 * ns + s];
          }
        }
      }
    }
    if (__any_sync(0xffffffffu, nact > 0)) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        f0 += __shfl_xor_sync(0xffffffffu, f0, o);
        f1 += __shfl_xor_sync(0xffffffffu, f1, o);
        f2 += __shfl_xor_sync(0xffffffffu, f2, o);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nact += __shfl_xor_sync(0xffffffffu, nact, o);
      nadh += __shfl_xor_sync(0xffffffffu, nadh, o);
    }
    if ((threadIdx.x & 31) == 0) {
      const int g = v >> 5;
      tf[0][g] = f0;
      tf[1][g] = f1;
      tf[2][g] = f2;
      ti[0][g] = nact;
      ti[1][g] = nadh;
    }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double F[3] = {0.0, 0.0, 0.0};
  int na = 0, nd = 0;
  for (int k = 0; k < kTailLanes / 32; ++k) {
    if (ti[0][k] > 0) {
      F[0] += tf[0][k];
      F[1] += tf[1][k];
      F[2] += tf[2][k];
    }
    na += ti[0][k];
    nd += ti[1][k];
  }
  c.nonfinite = 0;  // for the next pass
  if (c.check) {
    c.status = PDN_E_ARG;
    c.mode = MODE_HALT;
  } else if (c.timeout) {
    c.status = PDN_E_TIMEOUT;
    c.mode = MODE_HALT;
  } else if (mode == MODE_FORCES) {
    c.mode = MODE_DONE;
  } else if (nf) {
    c.status = PDN_E_NONFINITE;
    c.mode = MODE_HALT;
  } else if (mode == MODE_PRIME) {
    c.dpar ^= 1;
    c.mode = (c.step >= c.target) ? MODE_DONE : MODE_ADVANCE;
  } else if (nd > 0) {
    if (c.repeats >= c.max_repeats) {
      c.status = PDN_E_RELEASE_LIMIT;
      c.mode = MODE_HALT;
    } else {
      c.repeats += 1;
      c.n_repeats_total += 1;
      c.mode = MODE_REPEAT;
    }
  } else {
    // commit step n+1
    for (int i = 0; i < 3; ++i) {
      S.c[i] = ss.c[i];
      S.w[i] = ss.w[i];
      S.F[i] = F[i];
    }
    const double fc = F[0] * S.axis[0] + F[1] * S.axis[1] + F[2] * S.axis[2];
    if (c.hist_count < D.hist_cap) D.fhist[c.hist_count++] = fc;
    if (fc > c.f_peak) c.f_peak = fc;
    c.n_active = na;
    c.step += 1;
    c.time += D.dt;
    c.dpar ^= 1;
    c.hpar ^= 1;
    c.repeats = 0;
    c.mode = (c.step >= c.target) ? MODE_DONE : MODE_ADVANCE;
    // striker of the next step (Algorithm 1: the rigid instance moves first,
    // with the contact force just committed)
    StrikerStep nx;
    striker_rk4(S, D.dt, nx.c, nx.w, nx.aI);
    *D.imp = S;
    *D.imp_step = nx;
  }
  *ctl = c;
}

// ---------------------------------------------------------------------------
// Kernel 4: deterministic CSR gather of element forces per node (fixed
// ascending order: hexes, then interface elements), lumped-mass acceleration
// a = m^-1 (f^e - f^i) (Sec. 2.2.1), contact reaction of active nodes
// lambda = m (a_I . n) - f . n with release of adhesive nodes (Eq. anodes,
// Algorithm 2), and the Tchamwa-Wielgosz predictor of the next step:
// v' = v + dt a, d' = d + dt v + phi dt^2 a.  One thread per node.  The
// contact reaction of an active node is stored per surface node (its sum is
// the tail's job); a non-finite acceleration raises the pass's flag in the
// control block.
//
// One node.  Loads are grouped so that each thread waits on two rounds of
// memory latency: first the node's CSR range together with its state (flags,
// inverse mass, d and v of the current buffer), then its element forces, up
// to eight at once.  The forces are contiguous (written at their CSR
// positions) and summed in CSR order: hexes, then interfaces, ascending.
// State of node j that its update reads (flags, inverse mass, d and v of the
// current buffer); issued before the element forces so that both rounds of
// loads are in flight together.
template <typename T>
struct NodeState {
  uint8_t fl;
  T im;
  double dc[3], vc[3];
};
template <typename T>
__device__ __forceinline__ void node_state_load(const Dev<T> &D, int64_t j, int mode, NodeState<T> &q) {
  q.fl = 0;
  q.im = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) q.dc[i] = q.vc[i] = 0.0;
  if (mode == MODE_FORCES) return;
  const int cur = D.ctl->dpar;
  q.fl = D.nflag[j];
  q.im = D.inv_mass[j];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    q.dc[i] = D.d[cur][i * D.nn + j];
    q.vc[i] = D.v[cur][i * D.nn + j];
  }
}

// The update of node j from the sum (fx, fy, fz) of its element forces: the
// internal-force output (MODE_FORCES), or the acceleration, the contact
// reaction of an active node, and the predictor of the next step.
template <typename T>
__device__ __forceinline__ void node_update(const Dev<T> &D, int64_t j, int mode, const NodeState<T> &q, T fx,
                                            T fy, T fz) {
  using V4 = typename Vec4T<T>::type;
  Ctl *ctl = D.ctl;
  const int64_t nn = D.nn;
  if (mode == MODE_FORCES) {
    D.fout[j] = (double)fx;
    D.fout[nn + j] = (double)fy;
    D.fout[2 * nn + j] = (double)fz;
    return;
  }
  const uint8_t fl = q.fl;
  const T im = q.im;
  const int cur = ctl->dpar;
  int nonfin = 0;
  const int nxt = cur ^ 1;
  double a[3];
  bool done = false;
  if ((fl & 8) && mode != MODE_PRIME) {
    const int64_t s = D.surf_base >= 0 ? j - D.surf_base : D.surf_of[j];
    const int spar = (int)((ctl->step + 1) & 1);
    // the contact flag, the normal, the mass and the striker's acceleration
    // in one round of loads (the normal of an inactive node is not used)
    const int64_t ns = D.ns;
    const bool on = D.act[spar][s] != 0;
    const double m = D.mass[j];
    const double n[3] = {D.nrm[s], D.nrm[ns + s], D.nrm[2 * ns + s]};
    const StrikerStep *ss = D.imp_step;
    const double aI[3] = {ss->aI[0], ss->aI[1], ss->aI[2]};
    if (on) {
      const double fr[3] = {m * D.grav[0] - (double)fx, m * D.grav[1] - (double)fy, m * D.grav[2] - (double)fz};
      const double fdot = fr[0] * n[0] + fr[1] * n[1] + fr[2] * n[2];
      const double adot = aI[0] * n[0] + aI[1] * n[1] + aI[2] * n[2];
      const double lam = m * adot - fdot;
      D.lam[s] = lam;
      if (lam < 0.0) {
        D.rel[s] = 1;
        a[0] = fr[0] / m;
        a[1] = fr[1] / m;
        a[2] = fr[2] / m;
      } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) a[i] = (fr[i] + lam * n[i]) / m;
      }
      done = true;
    }
  }
  if (!done) {
    // free node: acceleration in the element precision, checked before
    // widening (the element force is already rounded to T)
    const T ax = D.grav_t[0] - fx * im, ay = D.grav_t[1] - fy * im, az = D.grav_t[2] - fz * im;
    if (!xfinite(ax) || !xfinite(ay) || !xfinite(az)) nonfin = 1;
    a[0] = to_f64(ax);
    a[1] = to_f64(ay);
    a[2] = to_f64(az);
  } else if (!xfinite(a[0]) || !xfinite(a[1]) || !xfinite(a[2])) {
    nonfin = 1;
  }
  const double dt = D.dt;
  double *dn = D.d[nxt];
  double *vn = D.v[nxt];
  double dd[3];
  const bool phi1 = (D.phi == 1.0);
  const double pdt2 = D.phi * dt * dt;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double ai = ((fl >> i) & 1) ? 0.0 : a[i];
    const double v1 = q.vc[i] + dt * ai;
    const double d1 = phi1 ? q.dc[i] + dt * v1 : q.dc[i] + dt * q.vc[i] + pdt2 * ai;
    vn[i * nn + j] = v1;
    dn[i * nn + j] = d1;
    dd[i] = d1;
  }
  V4 u;
  u.x = to_elem(dd[0], T(0));
  u.y = to_elem(dd[1], T(0));
  u.z = to_elem(dd[2], T(0));
  u.w = T(0);
  D.u4[nxt][j] = u;
  if (nonfin) atomicOr(&ctl->nonfinite, 1);
}

template <typename T>
__device__ __forceinline__ void gather_item(const Dev<T> &D, int64_t j, int mode) {
  using V4 = typename Vec4T<T>::type;
  if (j >= D.nn) return;
  if (mode == MODE_REPEAT && !repeat_take(D.rmark_n, j)) return;
  const bool ell = D.ell != 0;
  const int r0 = ell ? 0 : D.row[j], r1 = ell ? 0 : D.row[j + 1];
  NodeState<T> q;
  node_state_load(D, j, mode, q);
  T fx = T(0), fy = T(0), fz = T(0);
  if (ell) {
    // the node's eight slots (CSR order, zero padding): one load round with
    // the node state above
    const V4 *fs = D.fe + 8 * j;
    V4 f[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = fs[k];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      fx += f[k].x;
      fy += f[k].y;
      fz += f[k].z;
    }
  }
  for (int rb = r0; rb < r1; rb += 8) {
    V4 f[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (rb + k < r1) f[k] = D.fe[rb + k];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (rb + k < r1) {
        fx += f[k].x;
        fy += f[k].y;
        fz += f[k].z;
      }
  }
  node_update(D, j, mode, q, fx, fy, fz);
}

// The interface part of a node's force when interfaces are node pairs: the
// cohesive law (Algorithm 5) evaluated once for the Newton-Cotes point that
// the pair forms in each incident interface element (Sec. 2.3.2), from the
// jump upper minus lower and the pair's committed threshold rin, and each
// element's share w tau (upper node) or -w tau (lower node) added in CSR
// order: the sums of the interface kernel's slots, in the same order and
// rounding.  The lower node writes the pair's new threshold; an undamaged
// pair (r_D = 0 before and after) in a new step writes nothing, since the
// other buffer then holds 0 as well (r_D never decreases, and only the
// passes of the step write it).
template <typename T>
__device__ __forceinline__ void pair_forces(const Dev<T> &D, const Mat<T> &M, int64_t j, int mode, bool top,
                                            const T (&us)[3], const T (&up)[3], T rin, int kc, const T (&w)[4],
                                            T &fx, T &fy, T &fz) {
  const T dl[3] = {top ? us[0] - up[0] : up[0] - us[0], top ? us[1] - up[1] : up[1] - us[1],
                   top ? us[2] - up[2] : up[2] - us[2]};
  T tau[3], r1;
  czm(M, dl, rin, r1, tau);
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (k < kc) {
      const T tx = rmul(w[k], tau[0]), ty = rmul(w[k], tau[1]), tz = rmul(w[k], tau[2]);
      if (top) {
        fx += tx;
        fy += ty;
        fz += tz;
      } else {
        fx -= tx;
        fy -= ty;
        fz -= tz;
      }
    }
  if (!top && (mode == MODE_REPEAT || (mode == MODE_ADVANCE && (rin != T(0) || r1 != T(0)))))
    D.rDn[D.ctl->hpar ^ 1][j] = r1;
}

template <typename T>
__device__ __forceinline__ void pair_weights(const Dev<T> &D, int64_t j, T (&w)[4]) {
  using V4 = typename Vec4T<T>::type;
  if (D.iw != nullptr) {
    const V4 wv = D.iw[j];
    w[0] = wv.x;
    w[1] = wv.y;
    w[2] = wv.z;
    w[3] = wv.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = D.coh_w;
  }
}

// The node's own displacement mirror: in the stepping passes it is the
// element-precision rounding of the committed FP64 displacement already
// loaded (the mirror is always written as that rounding), so it is not read
// again; an internal-force pass reads it.
template <typename T>
__device__ __forceinline__ void own_mirror(const Dev<T> &D, int64_t j, int mode, int ub, const NodeState<T> &q,
                                           T (&us)[3]) {
  if (mode == MODE_FORCES) {
    const auto u = D.u4[ub][j];
    us[0] = u.x;
    us[1] = u.y;
    us[2] = u.z;
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) us[i] = to_elem(q.dc[i], T(0));
  }
}

// The gather of one node when interfaces are node pairs with partners from
// Dev::ipair: the node's hex slots come in the first load round with its
// state (the first four always, the rest when it has more hexes); an
// interface node then reads its partner's displacement mirror and the pair's
// threshold (a second round) and adds the interface part (pair_forces).
template <typename T>
__device__ __forceinline__ void gather_pair_item(const Dev<T> &D, const Mat<T> &M, int64_t j, int mode) {
  using V4 = typename Vec4T<T>::type;
  if (j >= D.nn) return;
  if (mode == MODE_REPEAT && !repeat_take(D.rmark_n, j)) return;
  NodeState<T> q;
  node_state_load(D, j, mode, q);
  const int2 ip = D.ipair[j];
  const V4 *fs = D.fe + 8 * j;
  V4 f[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) f[k] = fs[k];
  const int nhx = (ip.y >> 4) & 15;
#pragma unroll
  for (int k = 4; k < 8; ++k)
    if (k < nhx) f[k] = fs[k];
  T fx = T(0), fy = T(0), fz = T(0);
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (k < nhx) {
      fx += f[k].x;
      fy += f[k].y;
      fz += f[k].z;
    }
  if (ip.x >= 0) {
    const Ctl *ctl = D.ctl;
    const int ub = (mode == MODE_FORCES) ? (ctl->dpar ^ 1) : ctl->dpar;
    const bool top = (ip.y >> 3) & 1;
    const V4 u = D.u4[ub][ip.x];
    const T up[3] = {u.x, u.y, u.z};
    const T rin = D.rDn[ctl->hpar][top ? (int64_t)ip.x : j];
    T w[4], us[3];
    pair_weights(D, j, w);
    own_mirror(D, j, mode, ub, q, us);
    pair_forces(D, M, j, mode, top, us, up, rin, ip.y & 7, w, fx, fy, fz);
  }
  node_update(D, j, mode, q, fx, fy, fz);
}

// The same for a layered numbering (Dev::pair_layer): the node's layer, and
// with it whether it has a partner and which, follows from its id, so its
// partner's mirror and the pair's threshold load in the same round as its
// state and slots.  An interface node has at most four hexes, all on one
// side; its other four slots belong to interface elements, which write no
// slots here, so the first four slots hold its hex forces followed by zeros.
template <typename T>
__device__ __forceinline__ void gather_pair_layered_item(const Dev<T> &D, const Mat<T> &M, int64_t j, int mode) {
  using V4 = typename Vec4T<T>::type;
  if (j >= D.nn) return;
  if (mode == MODE_REPEAT && !repeat_take(D.rmark_n, j)) return;
  const Ctl *ctl = D.ctl;
  const int ub = (mode == MODE_FORCES) ? (ctl->dpar ^ 1) : ctl->dpar;
  const uint32_t L = (uint32_t)D.pair_layer;
  const uint32_t lay = (uint32_t)j / L;
  const int wd = lay >> 6, bit = lay & 63;
  const bool lower = (((wd ? D.pair_mask[0][1] : D.pair_mask[0][0]) >> bit) & 1) != 0;
  const bool upper = (((wd ? D.pair_mask[1][1] : D.pair_mask[1][0]) >> bit) & 1) != 0;
  const bool pair = lower || upper;
  NodeState<T> q;
  node_state_load(D, j, mode, q);
  const uint8_t fl = D.nflag[j];
  const int64_t pj = upper ? j - (int64_t)L : j + (int64_t)L;
  const V4 *fs = D.fe + (D.slot_compact ? compact_slot_base(D, lay, j) : 8 * j);
  V4 f[8];
#pragma unroll
  for (int k = 0; k < 4; ++k) f[k] = fs[k];
  if (!pair) {
#pragma unroll
    for (int k = 4; k < 8; ++k) f[k] = fs[k];
  }
  V4 u;
  T rin = T(0);
  if (pair) {
    u = D.u4[ub][pj];
    rin = D.rDn[ctl->hpar][upper ? pj : j];
  }
  T w[4];
  if (pair) pair_weights(D, j, w);
  T fx = T(0), fy = T(0), fz = T(0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    fx += f[k].x;
    fy += f[k].y;
    fz += f[k].z;
  }
  if (!pair) {
#pragma unroll
    for (int k = 4; k < 8; ++k) {
      fx += f[k].x;
      fy += f[k].y;
      fz += f[k].z;
    }
  } else {
    const T up[3] = {u.x, u.y, u.z};
    T us[3];
    own_mirror(D, j, mode, ub, q, us);
    pair_forces(D, M, j, mode, upper, us, up, rin, (fl >> kFlagPairShift) & 7, w, fx, fy, fz);
  }
  node_update(D, j, mode, q, fx, fy, fz);
}

}  // namespace detail
}  // namespace pdn
