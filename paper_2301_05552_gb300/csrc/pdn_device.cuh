// Device building blocks of the explicit PDN step shared by the kernel
// translation units: scalar helpers, exact float<->double conversions, hex8
// trilinear modes, the intralaminar law (Algorithm 4), the cohesive law
// (Algorithm 5) and the striker's RK4 update (Eq. rk4).
#pragma once

#include <cstdint>

#include "pdn_internal.h"

namespace pdn {
namespace detail {

// ---------------------------------------------------------------------------
// Scalar helpers with float/double overloads.
__device__ __forceinline__ float xsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double xsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float xexp(float x) { return expf(x); }
__device__ __forceinline__ double xexp(double x) { return exp(x); }
__device__ __forceinline__ float xcbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double xcbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float xpow(float x, float y) { return powf(x, y); }
// Correctly rounded reciprocals (the same value as 1 / x under IEEE
// division, without the division's general path).
__device__ __forceinline__ float xrcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double xrcp(double x) { return __drcp_rn(x); }
__device__ __forceinline__ double xpow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ bool xfinite(double x) { return isfinite(x); }
__device__ __forceinline__ bool xfinite(float x) { return isfinite(x); }
// Operations rounded one at a time, which no multiply-add contraction may
// merge: code evaluated in several kernels (the cohesive law: the interface
// kernel, the node-pair gather, the sweep, the batched kernel) then rounds
// identically in all of them.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rsqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double rsqrt_rn(double a) { return __dsqrt_rn(a); }

// Exact float <-> double conversions with integer instructions.  On this part
// the hardware conversions issue at the FP64 rate (about 0.6 T/s, measured),
// 30x slower than the integer pipe, and the node update needs six per node.
// Zeros and normal numbers take the integer path; subnormals, infinities,
// NaNs and out-of-range values fall back to the hardware conversion.
__device__ __forceinline__ double to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t ex = (u >> 23) & 0xffu;
  const uint32_t sign = u & 0x80000000u;
  if ((u & 0x7fffffffu) == 0u) return __hiloint2double((int)sign, 0);
  if (ex == 0u || ex == 0xffu) return (double)f;
  const uint32_t man = u & 0x7fffffu;
  const uint32_t hi = sign | ((ex + (1023u - 127u)) << 20) | (man >> 3);
  return __hiloint2double((int)hi, (int)(man << 29));
}
__device__ __forceinline__ double to_f64(double d) { return d; }

// Round to nearest, ties to even.
__device__ __forceinline__ float to_elem(double d, float) {
  const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
  const uint32_t ex = (hi >> 20) & 0x7ffu;
  const uint32_t sign = hi & 0x80000000u;
  if ((hi & 0x7fffffffu) == 0u && lo == 0u) return __uint_as_float(sign);
  if (ex < 897u || ex > 1150u) return (float)d;  // float subnormal / overflow range or inf/nan
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rest = lo & 0x1fffffffu;
  uint32_t bits = sign | ((ex - 896u) << 23) | m;
  if (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) bits += 1u;
  return __uint_as_float(bits);
}
__device__ __forceinline__ double to_elem(double d, double) { return d; }

// Natural-coordinate signs of hex8 node a (bottom face CCW, then top face).
__host__ __device__ constexpr int sgn_x(int a) { return ((a ^ (a >> 1)) & 1) ? 1 : -1; }
__host__ __device__ constexpr int sgn_y(int a) { return ((a >> 1) & 1) ? 1 : -1; }
__host__ __device__ constexpr int sgn_z(int a) { return ((a >> 2) & 1) ? 1 : -1; }
// Position of node a in the binary order (bit0 = +xi, bit1 = +eta, bit2 = +zeta).
__host__ __device__ constexpr int bin_of(int a) {
  return (sgn_x(a) > 0 ? 1 : 0) | (sgn_y(a) > 0 ? 2 : 0) | (sgn_z(a) > 0 ? 4 : 0);
}

// Hex8 trilinear map written in the monomial basis {1, xi, eta, zeta, xi eta,
// eta zeta, xi zeta, xi eta zeta}: x(xi) = sum_m phi_m(xi) c_m with
// c_m = 1/8 sum_a phi_m(node a) x_a.  to_modes computes c_1..c_7 by a
// three-stage butterfly; from_modes is the transpose (f_a = 1/8 sum_m
// phi_m(node a) C_m), used to return the mode-space force to the nodes.
// Mode index m: 1 xi, 2 eta, 3 zeta, 4 xi eta, 5 eta zeta, 6 xi zeta, 7 xi eta zeta.
__host__ __device__ constexpr int mode_bin(int m) {
  return m == 0 ? 0 : m == 1 ? 1 : m == 2 ? 2 : m == 3 ? 4 : m == 4 ? 3 : m == 5 ? 6 : m == 6 ? 5 : 7;
}

template <typename T>
__device__ __forceinline__ void to_modes(const T (&x)[8][3], T (&c)[8][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T r[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) r[bin_of(a)] = x[a][i];
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (!(k & bit)) {
          T lo = r[k], hi = r[k | bit];
          r[k] = hi + lo;
          r[k | bit] = hi - lo;
        }
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) c[m][i] = T(0.125) * r[mode_bin(m)];
  }
}

template <typename T>
__device__ __forceinline__ void from_modes(const T (&C)[8][3], T (&f)[8][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    T r[8];
    r[0] = T(0);
#pragma unroll
    for (int m = 1; m < 8; ++m) r[mode_bin(m)] = C[m][i];
#pragma unroll
    for (int bit = 1; bit < 8; bit <<= 1) {
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (!(k & bit)) {
          T c1 = r[k], cx = r[k | bit];
          r[k] = c1 - cx;
          r[k | bit] = c1 + cx;
        }
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) f[a][i] = T(0.125) * r[bin_of(a)];
  }
}

// Jacobian columns d x / d(xi, eta, zeta) at a point from the modes.
template <typename T>
__device__ __forceinline__ void jac_cols(const T (&c)[8][3], T xi, T et, T ze, T (&J)[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    J[i][0] = c[1][i] + et * c[4][i] + ze * c[6][i] + et * ze * c[7][i];
    J[i][1] = c[2][i] + xi * c[4][i] + ze * c[5][i] + xi * ze * c[7][i];
    J[i][2] = c[3][i] + et * c[5][i] + xi * c[6][i] + xi * et * c[7][i];
  }
}

template <typename T>
__device__ __forceinline__ T det3(const T (&A)[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// Element volume: sum of det J over the 2x2x2 Gauss points.
template <typename T>
__device__ T hex_volume(const T (&am)[8][3]) {
  const T gp = T(0.57735026918962576451);
  T V = T(0);
#pragma unroll 1
  for (int g = 0; g < 8; ++g) {
    T J[3][3];
    jac_cols(am, T(sgn_x(g)) * gp, T(sgn_y(g)) * gp, T(sgn_z(g)) * gp, J);
    V += det3(J);
  }
  return V;
}

// SplitMix64 finaliser of (seed ^ (4 e + k)) mapped to [1 - spread, 1 + spread].
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__device__ __forceinline__ float strength_factor(const Mat<float> &M, int64_t e, int k) {
  uint64_t z = splitmix64(M.seed ^ (uint64_t)(e * 4 + k));
  float u = (float)(uint32_t)(z >> 40) * (1.0f / 16777216.0f);
  return 1.0f + M.spread * (2.0f * u - 1.0f);
}
__device__ __forceinline__ double strength_factor(const Mat<double> &M, int64_t e, int k) {
  uint64_t z = splitmix64(M.seed ^ (uint64_t)(e * 4 + k));
  double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  return 1.0 + M.spread * (2.0 * u - 1.0);
}

// ---------------------------------------------------------------------------
// Local repetition of a step (Algorithm 2).  A repeated pass differs from the
// pass before it only at the released nodes, which the contact item puts back
// to their state before projection.  Only the elements around those nodes
// (marked by the contact item) and the nodes of those elements (marked by the
// element items) are evaluated again; every other element force and nodal
// update of the previous pass came from identical inputs and stands.  An item
// consumes its mark (clears it), so no mark outlives its pass; a mark left
// behind would only cost one more evaluation with the same result.  Without
// mark buffers (null) a repeated pass evaluates everything again.
__device__ __forceinline__ bool repeat_take(uint8_t *mark, int64_t i) {
  if (mark == nullptr) return true;
  if (mark[i] == 0) return false;
  mark[i] = 0;
  return true;
}
__device__ __forceinline__ void repeat_mark_nodes(uint8_t *mark, const int nd[8]) {
  if (mark == nullptr) return;
#pragma unroll
  for (int a = 0; a < 8; ++a) mark[nd[a]] = 1;
}

// ---------------------------------------------------------------------------
// Compact force slots (Dev::slot_compact): the node layer of node j, whether
// layer lay is an interface layer, and the first slot of node j in layer
// lay.
template <typename T>
__device__ __forceinline__ uint32_t node_layer(const Dev<T> &D, int64_t j) {
  const uint32_t L = (uint32_t)D.pair_layer, jj = (uint32_t)j;
  uint32_t lay = (uint32_t)((float)jj * D.pair_inv_L);
  if (lay * L > jj) --lay;
  else if ((lay + 1) * L <= jj) ++lay;
  return lay;
}
template <typename T>
__device__ __forceinline__ bool layer_is_pair(const Dev<T> &D, uint32_t lay) {
  const uint64_t m = lay < 64 ? (D.pair_mask[0][0] | D.pair_mask[1][0]) : (D.pair_mask[0][1] | D.pair_mask[1][1]);
  return ((m >> (lay & 63)) & 1) != 0;
}
template <typename T>
__device__ __forceinline__ int64_t compact_slot_base(const Dev<T> &D, uint32_t lay, int64_t j) {
  return j * (layer_is_pair(D, lay) ? 4 : 8) + D.layer_off[lay];
}

// ---------------------------------------------------------------------------
// Slots of an element's eight nodal forces.  With eight slots per node
// (D.rank set) slot = 8 node + rank, the node ids re-read from the
// connectivity (still in L1 from the element's start) and the ranks packed
// 3 bits per corner; otherwise the precomputed positions.
template <typename T>
__device__ __forceinline__ void element_slots(const Dev<T> &D, const int32_t *conn, int64_t e, const int4 *pos2,
                                              uint32_t rk, int (&ps)[8]) {
  if (D.rank != nullptr) {
    const int4 c0 = __ldg(reinterpret_cast<const int4 *>(conn) + 2 * e);
    const int4 c1 = __ldg(reinterpret_cast<const int4 *>(conn) + 2 * e + 1);
    const int nd[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    if (D.slot_compact) {
      // a hex's lower face lies in one node layer, its upper face in one
      // (checked by the host before it turns compact slots on)
      const uint32_t lb = node_layer(D, nd[0]), lt = node_layer(D, nd[4]);
      const int wb = layer_is_pair(D, lb) ? 4 : 8, wt = layer_is_pair(D, lt) ? 4 : 8;
      const int ob = D.layer_off[lb], ot = D.layer_off[lt];
#pragma unroll
      for (int a = 0; a < 8; ++a)
        ps[a] = nd[a] * (a < 4 ? wb : wt) + (a < 4 ? ob : ot) + (int)((rk >> (3 * a)) & 7u);
    } else {
#pragma unroll
      for (int a = 0; a < 8; ++a) ps[a] = 8 * nd[a] + (int)((rk >> (3 * a)) & 7u);
    }
  } else {
    const int4 p0 = __ldg(pos2), p1 = __ldg(pos2 + 1);
    ps[0] = p0.x, ps[1] = p0.y, ps[2] = p0.z, ps[3] = p0.w;
    ps[4] = p1.x, ps[5] = p1.y, ps[6] = p1.z, ps[7] = p1.w;
  }
}

// PDN_CHECK builds: the eight node ids of an element lie in [0, n_nodes);
// otherwise the first failure is recorded (CheckCode) and the caller skips
// the element.  Always true in other builds.
template <typename T>
__device__ __forceinline__ bool nodes_in_range(const Dev<T> &D, const int (&nd)[8]) {
#ifdef PDN_CHECK
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 8; ++a) ok = ok && nd[a] >= 0 && (int64_t)nd[a] < D.nn;
  if (!ok) atomicCAS(&D.ctl->check, 0, (int32_t)CHECK_ELEMENT_NODE);
  return ok;
#else
  (void)D;
  (void)nd;
  return true;
#endif
}

// ---------------------------------------------------------------------------
// Intralaminar law (Algorithm 4) at one Gauss point, ply axes.
// eps: engineering strain [11 22 33 12 13 23]; h: history in/out
// {rFT, rFC, rMT, rMC, gp12, gp13, pbar}; sig: nominal stress.
// Loading functions, thresholds, exponential softening regularised by the
// element length and the damaged compliance are those of the oracle (see the
// header of oracle/pdn_oracle.c); the element length is computed lazily (only
// once some threshold exceeds 1).
// At or past the snap-back length (lc X^2 >= 2 E G) the law takes its limit
// from below, A = +inf: the stress drops to zero right after onset.
template <typename T>
__device__ __forceinline__ T soft_A(T lc, T X, T E, T G) {
  const T lx2 = lc * X * X, den = T(2) * E * G - lx2;
  return den > T(0) ? T(2) * lx2 / den : static_cast<T>(INFINITY);
}
template <typename T>
__device__ __forceinline__ T dmg(T r, T A) {
  return r <= T(1) ? T(0) : T(1) - xexp(A * (T(1) - r)) / r;
}

// Per-element constants of the law: the seeded strengths and reciprocals.
template <typename T>
struct ElemLaw {
  T XT, YT, SL, iXT, iYT, iSL2, etaL;
};

template <typename T>
__device__ __forceinline__ ElemLaw<T> elem_law(const Mat<T> &M, int64_t e) {
  ElemLaw<T> L;
  const T f0 = M.damage_on ? strength_factor(M, e, 0) : T(1);
  const T f1 = M.damage_on ? strength_factor(M, e, 1) : T(1);
  const T f2 = M.damage_on ? strength_factor(M, e, 2) : T(1);
  L.XT = M.XT * f0;
  L.YT = M.YT * f1;
  L.SL = M.SL * f2;
  L.iXT = xrcp(L.XT);
  L.iYT = xrcp(L.YT);
  const T iSL = xrcp(L.SL);
  L.iSL2 = iSL * iSL;
  L.etaL = L.SL * M.etaLc;
  return L;
}

// The loading functions are evaluated squared and compared with the squared
// thresholds (phi > r <=> phi^2 > r^2 for r >= 1), so square roots are taken
// only when a threshold grows; likewise the yield test of the plasticity.
// vol is the element volume when known up front (boxes), else am is used to
// compute it lazily.
// Shear plasticity of Algorithm 4 (radial return on the 12/13 pair), in
// place on the history h[4..6].
template <typename T>
__device__ __forceinline__ void cdm_plastic(const Mat<T> &M, const T (&ep)[6], T (&h)[7]) {
  if (!M.plasticity_on) return;
  T gp12 = h[4], gp13 = h[5], pb = h[6];
  const T t12 = M.G12 * (ep[3] - gp12);
  const T t13 = M.G12 * (ep[4] - gp13);
  const T tn2 = t12 * t12 + t13 * t13;
  const T ty = M.Sp + M.KpG12 * pb;
  if (tn2 > ty * ty) {
    const T tn = xsqrt(tn2);
    const T dp = (tn - ty) * M.iG1Kp;
    const T f = dp / tn;
    gp12 += f * t12;
    gp13 += f * t13;
    pb += dp;
  }
  h[4] = gp12;
  h[5] = gp13;
  h[6] = pb;
}

// Largest squared ratio phi_N^2 / r_N^2 over the four mechanisms of the
// intralaminar law at elastic strain ee (the loading functions of cdm_damage,
// evaluated without updating anything): > 1 means a threshold would grow.
template <typename T>
__device__ __forceinline__ T cdm_onset_ratio2(const Mat<T> &M, const ElemLaw<T> &L, const T (&ee)[6],
                                              const T (&h)[7]) {
  const T e0 = ee[0], e1 = ee[1], e2 = ee[2];
  const T s11 = M.C11 * e0 + M.C12 * e1 + M.C13 * e2;
  const T s22 = M.C12 * e0 + M.C22 * e1 + M.C23 * e2;
  const T s12 = M.G12 * ee[3], s13 = M.G13 * ee[4], s23 = M.G23 * ee[5];
  const T phiFT = M.E1 * e0 * L.iXT;
  const T phiFC = (s11 < T(0) ? -s11 : T(0)) * M.iXC;
  const T tl2 = s12 * s12 + s13 * s13;
  T rat = phiFT * phiFT / (h[0] * h[0]);
  const T rc = phiFC * phiFC / (h[1] * h[1]);
  rat = rc > rat ? rc : rat;
  if (s22 >= T(0)) {
    const T a = s22 * L.iYT;
    const T q = M.g1 * a + M.g * a * a + tl2 * L.iSL2 + s23 * s23 * M.iST2;
    const T rm = q / (h[2] * h[2]);
    rat = rm > rat ? rm : rat;
  } else {
    T tT = -s22 * M.kT;
    tT = tT > T(0) ? tT : T(0);
    T tL = xsqrt(tl2) + L.etaL * s22;
    tL = tL > T(0) ? tL : T(0);
    const T q = (tT * tT + s23 * s23) * M.iST2 + tL * tL * L.iSL2;
    const T rm = q / (h[3] * h[3]);
    rat = rm > rat ? rm : rat;
  }
  return rat;
}

// Intralaminar law (Algorithm 4) at one point: the plasticity of
// cdm_plastic, then the damage part (cdm_damage) on the elastic strain.
template <typename T>
__device__ __forceinline__ void cdm_damage(const Mat<T> &M, const ElemLaw<T> &L, const T (*am)[3], T vol, T &lc,
                                           const T (&ep)[6], T (&h)[7], T (&s)[6]);

template <typename T>
__device__ __forceinline__ void cdm(const Mat<T> &M, const ElemLaw<T> &L, const T (*am)[3], T vol, T &lc,
                                    const T (&ep)[6], T (&h)[7], T (&s)[6]) {
  cdm_plastic(M, ep, h);
  cdm_damage(M, L, am, vol, lc, ep, h, s);
}

// Damage part of Algorithm 4: loading functions on the effective stress of
// the elastic strain (ep minus the plastic shear strains h[4], h[5]),
// thresholds, damage variables and the nominal stress.
template <typename T>
__device__ __forceinline__ void cdm_damage(const Mat<T> &M, const ElemLaw<T> &L, const T (*am)[3], T vol, T &lc,
                                           const T (&ep)[6], T (&h)[7], T (&s)[6]) {
  T rFT = h[0], rFC = h[1], rMT = h[2], rMC = h[3];
  const T gp12 = h[4], gp13 = h[5];
  const T e0 = ep[0], e1 = ep[1], e2 = ep[2], e3 = ep[3] - gp12, e4 = ep[4] - gp13, e5 = ep[5];
  const T s11 = M.C11 * e0 + M.C12 * e1 + M.C13 * e2;
  const T s22 = M.C12 * e0 + M.C22 * e1 + M.C23 * e2;
  const T s33 = M.C13 * e0 + M.C23 * e1 + M.C33 * e2;
  const T s12 = M.G12 * e3, s13 = M.G13 * e4, s23 = M.G23 * e5;
  T D1 = T(0), D2 = T(0), D6 = T(0);
  if (M.damage_on) {
    const T phiFT = M.E1 * e0 * L.iXT;
    const T phiFC = (s11 < T(0) ? -s11 : T(0)) * M.iXC;
    const T tl2 = s12 * s12 + s13 * s13;
    if (s22 >= T(0)) {
      const T a = s22 * L.iYT;
      const T q = M.g1 * a + M.g * a * a + tl2 * L.iSL2 + s23 * s23 * M.iST2;
      if (q > rMT * rMT) rMT = xsqrt(q);
    } else {
      T tT = -s22 * M.kT;
      tT = tT > T(0) ? tT : T(0);
      const T base = (tT * tT + s23 * s23) * M.iST2;
      // <tauL + etaL s22> <= tauL for s22 < 0: test the bound before the root
      if (base + tl2 * L.iSL2 > rMC * rMC) {
        T tL = xsqrt(tl2) + L.etaL * s22;
        tL = tL > T(0) ? tL : T(0);
        const T q = base + tL * tL * L.iSL2;
        if (q > rMC * rMC) rMC = xsqrt(q);
      }
    }
    rFC = phiFC > rFC ? phiFC : rFC;
    rFT = phiFT > rFT ? phiFT : rFT;
    rFT = rFC > rFT ? rFC : rFT;
    rMT = rMC > rMT ? rMC : rMT;
    if (rFT > T(1) || rMT > T(1)) {
      if (lc < T(0)) lc = xcbrt(am ? hex_volume(*reinterpret_cast<const T(*)[8][3]>(am)) : vol);
      D1 = (s11 >= T(0)) ? dmg(rFT, soft_A(lc, L.XT, M.E1, M.GXT)) : dmg(rFC, soft_A(lc, M.XC, M.E1, M.GXC));
      D2 = (s22 >= T(0)) ? dmg(rMT, soft_A(lc, L.YT, M.E2, M.GYT)) : dmg(rMC, soft_A(lc, M.YC, M.E2, M.GYC));
      D6 = dmg(rMT, soft_A(lc, L.SL, M.G12, M.GSL));
    }
  }
  if (D1 > T(0) || D2 > T(0) || D6 > T(0)) {
    // M sigma = q o eps_e with M = diag(q) H(D), q = (1-D1, 1-D2, 1)
    const T q1 = T(1) - D1, q2 = T(1) - D2;
    const T A[3][3] = {{M.h11, q1 * M.h12, q1 * M.h13}, {q2 * M.h12, M.h22, q2 * M.h23},
                       {M.h13, M.h23, M.h33}};
    const T b0 = q1 * e0, b1 = q2 * e1, b2 = e2;
    const T det = det3(A);
    const T id = T(1) / det;
    s[0] = id * (b0 * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (b1 * A[2][2] - A[1][2] * b2) +
                 A[0][2] * (b1 * A[2][1] - A[1][1] * b2));
    s[1] = id * (A[0][0] * (b1 * A[2][2] - A[1][2] * b2) - b0 * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                 A[0][2] * (A[1][0] * b2 - b1 * A[2][0]));
    s[2] = id * (A[0][0] * (A[1][1] * b2 - b1 * A[2][1]) - A[0][1] * (A[1][0] * b2 - b1 * A[2][0]) +
                 b0 * (A[1][0] * A[2][1] - A[1][1] * A[2][0]));
    s[3] = (T(1) - D6) * s12;
    s[4] = (T(1) - D6) * s13;
    s[5] = (T(1) - D2) * s23;
  } else {
    s[0] = s11;
    s[1] = s22;
    s[2] = s33;
    s[3] = s12;
    s[4] = s13;
    s[5] = s23;
  }
  h[0] = rFT;
  h[1] = rFC;
  h[2] = rMT;
  h[3] = rMC;
}

// ---------------------------------------------------------------------------
// Cohesive law (Algorithm 5) at one interface point, local frame
// (1, 2 tangential, 3 normal).  Same reading as the oracle.
template <typename T>
__device__ __forceinline__ void czm(const Mat<T> &M, const T (&dl)[3], T rin, T &rout, T (&tau)[3]) {
  // every product, sum and quotient rounded on its own (rmul, radd, ...),
  // in the order written
  const T dsh2 = radd(rmul(dl[0], dl[0]), rmul(dl[1], dl[1]));
  const T d3p = dl[2] > T(0) ? dl[2] : T(0);
  const T kd3 = rmul(rmul(M.KI, d3p), d3p), ksh = rmul(M.Ksh, dsh2);
  const T en = radd(kd3, ksh);  // K_B lambda^2
  T D = T(0);
  T r = rin;
  if (rin > T(0) || en >= M.onset_floor) {
    const T B = en > T(0) ? rdiv(ksh, en) : T(0);
    const T KB = radd(rmul(rsub(T(1), B), M.KI), rmul(B, M.Ksh));
    const T lam = rsqrt_rn(rdiv(en, KB));
    const T Beta = xpow(B, M.eta);
    const T lo = rsqrt_rn(rdiv(radd(M.KI_D3o2, rmul(rsub(M.Ksh_Dsho2, M.KI_D3o2), Beta)), KB));
    const T lcr = rdiv(radd(M.KI_D3oD3c, rmul(rsub(M.Ksh_DshoDshc, M.KI_D3oD3c), Beta)), rmul(KB, lo));
    T H = rdiv(rsub(lam, lo), rsub(lcr, lo));
    H = H < T(0) ? T(0) : (H > T(1) ? T(1) : H);
    r = rin > H ? rin : H;
    const T rl = rmul(r, lcr);
    D = rdiv(rl, radd(rl, rmul(rsub(T(1), r), lo)));
  }
  const T s = rsub(T(1), D);
  tau[0] = rmul(rmul(s, M.Ksh), dl[0]);
  tau[1] = rmul(rmul(s, M.Ksh), dl[1]);
  tau[2] = (dl[2] >= T(0)) ? rmul(rmul(s, M.KI), dl[2]) : rmul(M.KI, dl[2]);
  rout = r;
}


__device__ __forceinline__ void striker_rk4(const Striker &S, double dt, double (&c1)[3],
                                            double (&w1)[3], double (&aI)[3]) {
  double ga[3];
  const double iM = S.iM;
#pragma unroll
  for (int i = 0; i < 3; ++i) ga[i] = S.g[i] - S.F[i] * iM;
  const double an = ga[0] * S.axis[0] + ga[1] * S.axis[1] + ga[2] * S.axis[2];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    aI[i] = an * S.axis[i];
    const double k1c = dt * S.w[i], k1w = dt * aI[i];
    const double k2c = dt * (S.w[i] + 0.5 * k1w), k2w = dt * aI[i];
    const double k3c = dt * (S.w[i] + 0.5 * k2w), k3w = dt * aI[i];
    const double k4c = dt * (S.w[i] + k3w), k4w = dt * aI[i];
    // weights 1/6, 1/3, 1/3, 1/6 as products (FP64 division is a long
    // dependent sequence on this part and this runs on the critical path)
    constexpr double s6 = 1.0 / 6.0, s3 = 1.0 / 3.0;
    c1[i] = S.c[i] + k1c * s6 + k2c * s3 + k3c * s3 + k4c * s6;
    w1[i] = S.w[i] + k1w * s6 + k2w * s3 + k3w * s3 + k4w * s6;
  }
}

}  // namespace detail
}  // namespace pdn
