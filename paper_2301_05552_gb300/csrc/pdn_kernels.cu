// CUDA kernels of the explicit PDN impact step for GB300 (sm_103a).
//
// One pass = contact -> hex8 -> interface -> gather -> tail, all on one stream.
// The tail kernel owns the device-side state machine (pdn_internal.h): it
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

#include "pdn.h"

namespace pdn {
namespace {

// ---------------------------------------------------------------------------
// Scalar helpers with float/double overloads.
__device__ __forceinline__ float xsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double xsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float xexp(float x) { return expf(x); }
__device__ __forceinline__ double xexp(double x) { return exp(x); }
__device__ __forceinline__ float xcbrt(float x) { return cbrtf(x); }
__device__ __forceinline__ double xcbrt(double x) { return cbrt(x); }
__device__ __forceinline__ float xpow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double xpow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ bool xfinite(double x) { return isfinite(x); }

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
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
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
// Intralaminar law (Algorithm 4) at one Gauss point, ply axes.
// eps: engineering strain [11 22 33 12 13 23]; h: history in/out
// {rFT, rFC, rMT, rMC, gp12, gp13, pbar}; sig: nominal stress.
// Loading functions, thresholds, exponential softening regularised by the
// element length and the damaged compliance are those of the oracle (see the
// header of oracle/pdn_oracle.c); the element length is computed lazily (only
// once some threshold exceeds 1).
template <typename T>
__device__ __forceinline__ T soft_A(T lc, T X, T E, T G) {
  T lx2 = lc * X * X;
  return T(2) * lx2 / (T(2) * E * G - lx2);
}
template <typename T>
__device__ __forceinline__ T dmg(T r, T A) {
  return r <= T(1) ? T(0) : T(1) - xexp(A * (T(1) - r)) / r;
}

template <typename T>
__device__ __forceinline__ void cdm(const Mat<T> &M, const T (&am)[8][3], T &lc, const T (&sf)[3],
                                    const T (&ep)[6], T (&h)[7], T (&s)[6]) {
  T rFT = h[0], rFC = h[1], rMT = h[2], rMC = h[3], gp12 = h[4], gp13 = h[5], pb = h[6];
  if (M.plasticity_on) {
    T t12 = M.G12 * (ep[3] - gp12);
    T t13 = M.G12 * (ep[4] - gp13);
    T tn = xsqrt(t12 * t12 + t13 * t13);
    T ty = M.Sp + M.Kp * M.G12 * pb;
    if (tn > ty) {
      T dp = (tn - ty) / (M.G12 * (T(1) + M.Kp));
      gp12 += dp * t12 / tn;
      gp13 += dp * t13 / tn;
      pb += dp;
    }
  }
  const T e0 = ep[0], e1 = ep[1], e2 = ep[2], e3 = ep[3] - gp12, e4 = ep[4] - gp13, e5 = ep[5];
  const T s11 = M.C11 * e0 + M.C12 * e1 + M.C13 * e2;
  const T s22 = M.C12 * e0 + M.C22 * e1 + M.C23 * e2;
  const T s33 = M.C13 * e0 + M.C23 * e1 + M.C33 * e2;
  const T s12 = M.G12 * e3, s13 = M.G13 * e4, s23 = M.G23 * e5;
  T D1 = T(0), D2 = T(0), D6 = T(0);
  if (M.damage_on) {
    const T XT = M.XT * sf[0], YT = M.YT * sf[1], SL = M.SL * sf[2];
    const T tauL = xsqrt(s12 * s12 + s13 * s13);
    const T phiFT = M.E1 * e0 / XT;
    const T phiFC = (s11 < T(0) ? -s11 : T(0)) / M.XC;
    T phiMT = T(0), phiMC = T(0);
    if (s22 >= T(0)) {
      const T a = s22 / YT, b = tauL / SL, c = s23 / M.ST;
      phiMT = xsqrt((T(1) - M.g) * a + M.g * a * a + b * b + c * c);
    } else {
      T tT = -s22 * M.ca * (M.sa - M.etaT * M.ca);
      tT = tT > T(0) ? tT : T(0);
      T tL = tauL + SL * M.etaLc * s22;
      tL = tL > T(0) ? tL : T(0);
      const T b = tL / SL;
      phiMC = xsqrt((tT * tT + s23 * s23) / (M.ST * M.ST) + b * b);
    }
    rFC = phiFC > rFC ? phiFC : rFC;
    rFT = phiFT > rFT ? phiFT : rFT;
    rFT = rFC > rFT ? rFC : rFT;
    rMC = phiMC > rMC ? phiMC : rMC;
    rMT = phiMT > rMT ? phiMT : rMT;
    rMT = rMC > rMT ? rMC : rMT;
    if (rFT > T(1) || rMT > T(1)) {
      if (lc < T(0)) lc = xcbrt(hex_volume(am));
      D1 = (s11 >= T(0)) ? dmg(rFT, soft_A(lc, XT, M.E1, M.GXT)) : dmg(rFC, soft_A(lc, M.XC, M.E1, M.GXC));
      D2 = (s22 >= T(0)) ? dmg(rMT, soft_A(lc, YT, M.E2, M.GYT)) : dmg(rMC, soft_A(lc, M.YC, M.E2, M.GYC));
      D6 = dmg(rMT, soft_A(lc, SL, M.G12, M.GSL));
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
  h[4] = gp12;
  h[5] = gp13;
  h[6] = pb;
}

// ---------------------------------------------------------------------------
// Cohesive law (Algorithm 5) at one interface point, local frame
// (1, 2 tangential, 3 normal).  Same reading as the oracle.
template <typename T>
__device__ __forceinline__ void czm(const Mat<T> &M, const T (&dl)[3], T rin, T &rout, T (&tau)[3]) {
  const T dsh2 = dl[0] * dl[0] + dl[1] * dl[1];
  const T d3p = dl[2] > T(0) ? dl[2] : T(0);
  const T en = M.KI * d3p * d3p + M.Ksh * dsh2;  // K_B lambda^2
  T D = T(0);
  T r = rin;
  if (rin > T(0) || en >= M.onset_floor) {
    const T den = M.Ksh * dsh2 + M.KI * d3p * d3p;
    const T B = den > T(0) ? M.Ksh * dsh2 / den : T(0);
    const T KB = (T(1) - B) * M.KI + B * M.Ksh;
    const T lam = xsqrt(en / KB);
    const T Beta = xpow(B, M.eta);
    const T lo = xsqrt((M.KI_D3o2 + (M.Ksh_Dsho2 - M.KI_D3o2) * Beta) / KB);
    const T lcr = (M.KI_D3oD3c + (M.Ksh_DshoDshc - M.KI_D3oD3c) * Beta) / (KB * lo);
    T H = (lam - lo) / (lcr - lo);
    H = H < T(0) ? T(0) : (H > T(1) ? T(1) : H);
    r = rin > H ? rin : H;
    D = r * lcr / (r * lcr + (T(1) - r) * lo);
  }
  tau[0] = (T(1) - D) * M.Ksh * dl[0];
  tau[1] = (T(1) - D) * M.Ksh * dl[1];
  tau[2] = (dl[2] >= T(0)) ? (T(1) - D) * M.KI * dl[2] : M.KI * dl[2];
  rout = r;
}

// ---------------------------------------------------------------------------
// Kernel 1: contact detection and projection (Sec. 2.1, Fig. 1, Algorithm 1).
// One thread per contact-surface node.  Thread 0 of every block also
// advances the rigid striker by one RK4 step with the contact force of the
// committed step (Eq. rk4; the force is held over the step), block 0 storing
// the result for the gather and tail kernels.
__device__ __forceinline__ void striker_rk4(const Striker &S, double dt, double (&c1)[3],
                                            double (&w1)[3], double (&aI)[3]) {
  double ga[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) ga[i] = S.g[i] - S.F[i] / S.M;
  const double an = ga[0] * S.axis[0] + ga[1] * S.axis[1] + ga[2] * S.axis[2];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    aI[i] = an * S.axis[i];
    const double k1c = dt * S.w[i], k1w = dt * aI[i];
    const double k2c = dt * (S.w[i] + 0.5 * k1w), k2w = dt * aI[i];
    const double k3c = dt * (S.w[i] + 0.5 * k2w), k3w = dt * aI[i];
    const double k4c = dt * (S.w[i] + k3w), k4w = dt * aI[i];
    c1[i] = S.c[i] + k1c / 6.0 + k2c / 3.0 + k3c / 3.0 + k4c / 6.0;
    w1[i] = S.w[i] + k1w / 6.0 + k2w / 3.0 + k3w / 3.0 + k4w / 6.0;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_contact(Dev<T> D) {
  using V4 = typename Vec4T<T>::type;
  const Ctl *ctl = D.ctl;
  const int mode = ctl->mode;
  if (mode != MODE_ADVANCE && mode != MODE_REPEAT) return;
  __shared__ double sh[9];
  const Striker *S = D.imp;
  if (threadIdx.x == 0) {
    double c1[3], w1[3], aI[3];
    striker_rk4(*S, D.dt, c1, w1, aI);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      sh[i] = c1[i];
      sh[3 + i] = w1[i];
      sh[6 + i] = aI[i];
    }
    if (blockIdx.x == 0) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        D.imp_step->c[i] = c1[i];
        D.imp_step->w[i] = w1[i];
        D.imp_step->aI[i] = aI[i];
      }
    }
  }
  __syncthreads();
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= D.ns) return;
  const int64_t nn = D.nn, ns = D.ns;
  const int64_t j = D.surf[s];
  const int cur = ctl->dpar;
  const int spar = (int)((ctl->step + 1) & 1), ppar = (int)(ctl->step & 1);
  double *d = D.d[cur];
  double *v = D.v[cur];
  if (mode == MODE_ADVANCE) {
    D.rel[s] = 0;
    uint8_t a = 0;
    const uint8_t fl = D.nflag[j];
    if (S->has && (fl & 7) != 7) {
      double x[3], r2 = 0.0;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        x[i] = D.Xs[i * ns + s] + d[i * nn + j] - sh[i];
        r2 += x[i] * x[i];
      }
      const double r = sqrt(r2);
      const double gap = r - S->R;
      if (gap < 0.0 || D.act[ppar][s]) {
        a = 1;
        double n[3] = {x[0] / r, x[1] / r, x[2] / r};
        double dj[3], vj[3], vn = 0.0, wn = 0.0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          dj[i] = d[i * nn + j];
          vj[i] = v[i * nn + j];
          D.trial[i * ns + s] = dj[i];
          D.trial[(3 + i) * ns + s] = vj[i];
          vn += vj[i] * n[i];
          wn += sh[3 + i] * n[i];
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
  } else {  // MODE_REPEAT: restore the released nodes to their trial state
    if (D.rel[s] && D.act[spar][s]) {
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
    }
  }
}

// ---------------------------------------------------------------------------
// Kernel 2: hex8 internal forces, total Lagrangian, 2x2x2 Gauss (Sec. 2,
// Eq. fcont), with the intralaminar law per Gauss point.  One thread per
// element; geometry and displacement enter through their trilinear modes, so
// that J = [dx/dxi], du/dxi and the returned force are cheap mode sums.
// f_a = sum_g sum_k dN_a/dxi_k Q_g[k][:],  Q_g = det J_g  J_g^-1 P_g,
// P = S F^T (nominal stress), S rotated from ply axes (angle about z).
template <typename T>
__global__ void __launch_bounds__(128) k_hex(Dev<T> D, Mat<T> M) {
  using V4 = typename Vec4T<T>::type;
  const Ctl *ctl = D.ctl;
  const int mode = ctl->mode;
  if (mode >= MODE_DONE) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D.nh) return;
  const int64_t nh = D.nh;
  const int ub = (mode == MODE_FORCES) ? (ctl->dpar ^ 1) : ctl->dpar;
  const int hb = ctl->hpar;
  const V4 *__restrict__ U = D.u4[ub];
  const int4 c0 = __ldg(reinterpret_cast<const int4 *>(D.hex) + 2 * e);
  const int4 c1 = __ldg(reinterpret_cast<const int4 *>(D.hex) + 2 * e + 1);
  const int nd[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  T am[8][3], bm[8][3];
  {
    T xa[8][3], ua[8][3];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const V4 x = D.X4[nd[a]];
      const V4 u = U[nd[a]];
      xa[a][0] = x.x;
      xa[a][1] = x.y;
      xa[a][2] = x.z;
      ua[a][0] = u.x;
      ua[a][1] = u.y;
      ua[a][2] = u.z;
    }
    to_modes(xa, am);
    to_modes(ua, bm);
  }
  const int ply = D.ply[e];
  const T cs = M.ply_c[ply], sn = M.ply_s[ply];
  T sf[3] = {T(1), T(1), T(1)};
  if (M.damage_on) {
    sf[0] = strength_factor(M, e, 0);
    sf[1] = strength_factor(M, e, 1);
    sf[2] = strength_factor(M, e, 2);
  }
  T lc = T(-1);
  const T *__restrict__ hin = D.hist[hb];
  T *__restrict__ hout = D.hist[hb ^ 1];
  T C[8][3];
#pragma unroll
  for (int m = 0; m < 8; ++m) C[m][0] = C[m][1] = C[m][2] = T(0);
  const T gp = T(0.57735026918962576451);
#pragma unroll 1
  for (int g = 0; g < 8; ++g) {
    const T xi = T(sgn_x(g)) * gp, et = T(sgn_y(g)) * gp, ze = T(sgn_z(g)) * gp;
    T J[3][3], Du[3][3];
    jac_cols(am, xi, et, ze, J);
    jac_cols(bm, xi, et, ze, Du);
    const T det = det3(J);
    const T id = T(1) / det;
    T Ji[3][3];
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    T H[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) H[i][k] = Du[i][0] * Ji[0][k] + Du[i][1] * Ji[1][k] + Du[i][2] * Ji[2][k];
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
    const T c2 = cs * cs, s2 = sn * sn, csn = cs * sn;
    T ep[6];
    ep[0] = c2 * E[0][0] + T(2) * csn * E[0][1] + s2 * E[1][1];
    ep[1] = s2 * E[0][0] - T(2) * csn * E[0][1] + c2 * E[1][1];
    ep[2] = E[2][2];
    ep[3] = T(2) * (-csn * E[0][0] + (c2 - s2) * E[0][1] + csn * E[1][1]);
    ep[4] = T(2) * (cs * E[0][2] + sn * E[1][2]);
    ep[5] = T(2) * (-sn * E[0][2] + cs * E[1][2]);
    T h[7];
#pragma unroll
    for (int f = 0; f < 7; ++f) h[f] = hin[((int64_t)f * 8 + g) * nh + e];
    T sm[6];
    cdm(M, am, lc, sf, ep, h, sm);
#pragma unroll
    for (int f = 0; f < 7; ++f) hout[((int64_t)f * 8 + g) * nh + e] = h[f];
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
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int I = 0; I < 3; ++I) Q[k][I] = det * (Ji[k][0] * P[0][I] + Ji[k][1] * P[1][I] + Ji[k][2] * P[2][I]);
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
  T f[8][3];
  from_modes(C, f);
  V4 *fe = D.fe + e * 8;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    V4 o;
    o.x = f[a][0];
    o.y = f[a][1];
    o.z = f[a][2];
    o.w = T(0);
    fe[a] = o;
  }
}

// ---------------------------------------------------------------------------
// Kernel 3: zero-thickness interface elements with Newton-Cotes integration
// (Sec. 2.3.2) and the cohesive law (Algorithm 5).  One thread per element.
template <typename T>
__global__ void __launch_bounds__(128) k_coh(Dev<T> D, Mat<T> M) {
  using V4 = typename Vec4T<T>::type;
  const Ctl *ctl = D.ctl;
  const int mode = ctl->mode;
  if (mode >= MODE_DONE) return;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D.nc) return;
  const int64_t nc = D.nc;
  const int ub = (mode == MODE_FORCES) ? (ctl->dpar ^ 1) : ctl->dpar;
  const int hb = ctl->hpar;
  const V4 *__restrict__ U = D.u4[ub];
  const int4 c0 = __ldg(reinterpret_cast<const int4 *>(D.coh) + 2 * c);
  const int4 c1 = __ldg(reinterpret_cast<const int4 *>(D.coh) + 2 * c + 1);
  const int nd[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  constexpr int QX[4] = {-1, 1, 1, -1}, QY[4] = {-1, -1, 1, 1};
  T xm[4][3], uu[8][3];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const V4 xb = D.X4[nd[a]];
    const V4 xt = D.X4[nd[a + 4]];
    xm[a][0] = T(0.5) * (xb.x + xt.x);
    xm[a][1] = T(0.5) * (xb.y + xt.y);
    xm[a][2] = T(0.5) * (xb.z + xt.z);
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
  {
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
  const T *__restrict__ rin = D.rD[hb];
  T *__restrict__ rout = D.rD[hb ^ 1];
  T f[8][3];
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
    czm(M, dl, rin[(int64_t)p * nc + c], r1, tau);
    rout[(int64_t)p * nc + c] = r1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const T tg = w * (tau[0] * e1[i] + tau[1] * e2[i] + tau[2] * e3[i]);
      f[p + 4][i] = tg;
      f[p][i] = -tg;
    }
  }
  V4 *fe = D.fe + (D.nh + c) * 8;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    V4 o;
    o.x = f[a][0];
    o.y = f[a][1];
    o.z = f[a][2];
    o.w = T(0);
    fe[a] = o;
  }
}

// ---------------------------------------------------------------------------
// Kernel 4: deterministic CSR gather of element forces per node (fixed
// ascending order: hexes, then interface elements), lumped-mass acceleration
// a = m^-1 (f^e - f^i) (Sec. 2.2.1), contact reaction of active nodes
// lambda = m (a_I . n) - f . n with release of adhesive nodes (Eq. anodes,
// Algorithm 2), and the Tchamwa-Wielgosz predictor of the next step:
// v' = v + dt a, d' = d + dt v + phi dt^2 a.  One thread per node; per-block
// reaction partial sums in a fixed tree order.
template <typename T>
__global__ void __launch_bounds__(256) k_gather(Dev<T> D) {
  using V4 = typename Vec4T<T>::type;
  const Ctl *ctl = D.ctl;
  const int mode = ctl->mode;
  if (mode >= MODE_DONE) return;
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nn = D.nn;
  double pf0 = 0.0, pf1 = 0.0, pf2 = 0.0;
  int nact = 0, nadh = 0, nonfin = 0;
  if (j < nn) {
    T fx = T(0), fy = T(0), fz = T(0);
    const int r0 = D.row[j], r1 = D.row[j + 1];
    for (int r = r0; r < r1; ++r) {
      const V4 f = D.fe[D.col[r]];
      fx += f.x;
      fy += f.y;
      fz += f.z;
    }
    if (mode == MODE_FORCES) {
      D.fout[j] = (double)fx;
      D.fout[nn + j] = (double)fy;
      D.fout[2 * nn + j] = (double)fz;
    } else {
      const int cur = ctl->dpar, nxt = cur ^ 1;
      const uint8_t fl = D.nflag[j];
      double a[3];
      bool done = false;
      if ((fl & 8) && mode != MODE_PRIME) {
        const int64_t s = D.surf_of[j];
        const int spar = (int)((ctl->step + 1) & 1);
        if (D.act[spar][s]) {
          const int64_t ns = D.ns;
          const double m = D.mass[j];
          const double n[3] = {D.nrm[s], D.nrm[ns + s], D.nrm[2 * ns + s]};
          const double fr[3] = {m * D.grav[0] - (double)fx, m * D.grav[1] - (double)fy,
                                m * D.grav[2] - (double)fz};
          const StrikerStep *ss = D.imp_step;
          const double fdot = fr[0] * n[0] + fr[1] * n[1] + fr[2] * n[2];
          const double adot = ss->aI[0] * n[0] + ss->aI[1] * n[1] + ss->aI[2] * n[2];
          const double lam = m * adot - fdot;
          D.lam[s] = lam;
          if (lam < 0.0) {
            D.rel[s] = 1;
            nadh = 1;
            a[0] = fr[0] / m;
            a[1] = fr[1] / m;
            a[2] = fr[2] / m;
          } else {
            nact = 1;
            pf0 = lam * n[0];
            pf1 = lam * n[1];
            pf2 = lam * n[2];
#pragma unroll
            for (int i = 0; i < 3; ++i) a[i] = (fr[i] + lam * n[i]) / m;
          }
          done = true;
        }
      }
      if (!done) {
        const T im = D.inv_mass[j];
        a[0] = (double)((T)D.grav[0] - fx * im);
        a[1] = (double)((T)D.grav[1] - fy * im);
        a[2] = (double)((T)D.grav[2] - fz * im);
      }
      const double dt = D.dt;
      const double *dc = D.d[cur];
      const double *vc = D.v[cur];
      double *dn = D.d[nxt];
      double *vn = D.v[nxt];
      double dd[3];
      const bool phi1 = (D.phi == 1.0);
      const double pdt2 = D.phi * dt * dt;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        double ai = ((fl >> i) & 1) ? 0.0 : a[i];
        if (!xfinite(ai)) nonfin = 1;
        const double vi = vc[i * nn + j];
        const double di = dc[i * nn + j];
        const double v1 = vi + dt * ai;
        const double d1 = phi1 ? di + dt * v1 : di + dt * vi + pdt2 * ai;
        vn[i * nn + j] = v1;
        dn[i * nn + j] = d1;
        dd[i] = d1;
      }
      V4 u;
      u.x = (T)dd[0];
      u.y = (T)dd[1];
      u.z = (T)dd[2];
      u.w = T(0);
      D.u4[nxt][j] = u;
    }
  }
  // block partials (fixed order: warp butterfly, then warps in index order)
  const int any = __syncthreads_or(nact | nadh | nonfin);
  if (!any) {
    if (threadIdx.x == 0) {
      Partial p;
      p.f[0] = p.f[1] = p.f[2] = 0.0;
      p.n_act = p.n_adh = p.nonfinite = p.pad = 0;
      D.part[blockIdx.x] = p;
    }
    return;
  }
  __shared__ double sf[3][8];
  __shared__ int si[3][8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pf0 += __shfl_xor_sync(0xffffffffu, pf0, o);
    pf1 += __shfl_xor_sync(0xffffffffu, pf1, o);
    pf2 += __shfl_xor_sync(0xffffffffu, pf2, o);
    nact += __shfl_xor_sync(0xffffffffu, nact, o);
    nadh += __shfl_xor_sync(0xffffffffu, nadh, o);
    nonfin |= __shfl_xor_sync(0xffffffffu, nonfin, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sf[0][w] = pf0;
    sf[1][w] = pf1;
    sf[2][w] = pf2;
    si[0][w] = nact;
    si[1][w] = nadh;
    si[2][w] = nonfin;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Partial p;
    p.f[0] = p.f[1] = p.f[2] = 0.0;
    p.n_act = p.n_adh = p.nonfinite = p.pad = 0;
    const int nw = blockDim.x >> 5;
    for (int k = 0; k < nw; ++k) {
      p.f[0] += sf[0][k];
      p.f[1] += sf[1][k];
      p.f[2] += sf[2][k];
      p.n_act += si[0][k];
      p.n_adh += si[1][k];
      p.nonfinite |= si[2][k];
    }
    D.part[blockIdx.x] = p;
  }
}

// ---------------------------------------------------------------------------
// Kernel 5: tail.  Sums the gather partials in a fixed order, then commits
// the step (contact force F = sum lambda_j n_j to the striker, Sec. 2.2.2;
// step counter, history and node-buffer parities, force history), or marks
// the step for repetition when adhesive nodes were released (Algorithm 2,
// the MPI_MAX of kfl_reset becomes this single-block decision), or halts.
template <typename T>
__global__ void __launch_bounds__(256) k_tail(Dev<T> D) {
  Ctl *ctl = D.ctl;
  const int mode = ctl->mode;
  if (mode >= MODE_DONE) return;
  double f0 = 0.0, f1 = 0.0, f2 = 0.0;
  int nact = 0, nadh = 0, nonfin = 0;
  for (int k = threadIdx.x; k < D.n_part; k += blockDim.x) {
    const Partial p = D.part[k];
    f0 += p.f[0];
    f1 += p.f[1];
    f2 += p.f[2];
    nact += p.n_act;
    nadh += p.n_adh;
    nonfin |= p.nonfinite;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f0 += __shfl_xor_sync(0xffffffffu, f0, o);
    f1 += __shfl_xor_sync(0xffffffffu, f1, o);
    f2 += __shfl_xor_sync(0xffffffffu, f2, o);
    nact += __shfl_xor_sync(0xffffffffu, nact, o);
    nadh += __shfl_xor_sync(0xffffffffu, nadh, o);
    nonfin |= __shfl_xor_sync(0xffffffffu, nonfin, o);
  }
  __shared__ double sf[3][8];
  __shared__ int si[3][8];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sf[0][w] = f0;
    sf[1][w] = f1;
    sf[2][w] = f2;
    si[0][w] = nact;
    si[1][w] = nadh;
    si[2][w] = nonfin;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double F[3] = {0.0, 0.0, 0.0};
  int na = 0, nd = 0, nf = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
    F[0] += sf[0][k];
    F[1] += sf[1][k];
    F[2] += sf[2][k];
    na += si[0][k];
    nd += si[1][k];
    nf |= si[2][k];
  }
  if (mode == MODE_FORCES) {
    ctl->mode = MODE_DONE;
    return;
  }
  if (nf) {
    ctl->status = PDN_E_NONFINITE;
    ctl->mode = MODE_HALT;
    return;
  }
  if (mode == MODE_PRIME) {
    ctl->dpar ^= 1;
    ctl->mode = (ctl->step >= ctl->target) ? MODE_DONE : MODE_ADVANCE;
    return;
  }
  if (nd > 0) {
    if (ctl->repeats >= ctl->max_repeats) {
      ctl->status = PDN_E_RELEASE_LIMIT;
      ctl->mode = MODE_HALT;
      return;
    }
    ctl->repeats += 1;
    ctl->n_repeats_total += 1;
    ctl->mode = MODE_REPEAT;
    return;
  }
  // commit step n+1
  Striker *S = D.imp;
  const StrikerStep *ss = D.imp_step;
  for (int i = 0; i < 3; ++i) {
    S->c[i] = ss->c[i];
    S->w[i] = ss->w[i];
    S->F[i] = F[i];
  }
  const double fc = F[0] * S->axis[0] + F[1] * S->axis[1] + F[2] * S->axis[2];
  if (ctl->hist_count < D.hist_cap) D.fhist[ctl->hist_count++] = fc;
  if (fc > ctl->f_peak) ctl->f_peak = fc;
  ctl->n_active = na;
  ctl->step += 1;
  ctl->time += D.dt;
  ctl->dpar ^= 1;
  ctl->hpar ^= 1;
  ctl->repeats = 0;
  ctl->mode = (ctl->step >= ctl->target) ? MODE_DONE : MODE_ADVANCE;
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

inline int grid_of(int64_t n, int b) {
  int64_t g = (n + b - 1) / b;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

template <typename T>
cudaError_t launch_pass(const Dev<T> &D, const Mat<T> &M, cudaStream_t s, int32_t gather_block,
                        cudaEvent_t *ev) {
  if (ev) cudaEventRecord(ev[0], s);
  k_contact<T><<<grid_of(D.ns, 256), 256, 0, s>>>(D);
  if (ev) cudaEventRecord(ev[1], s);
  k_hex<T><<<grid_of(D.nh, 128), 128, 0, s>>>(D, M);
  if (ev) cudaEventRecord(ev[2], s);
  if (D.nc > 0) k_coh<T><<<grid_of(D.nc, 128), 128, 0, s>>>(D, M);
  if (ev) cudaEventRecord(ev[3], s);
  k_gather<T><<<grid_of(D.nn, gather_block), gather_block, 0, s>>>(D);
  if (ev) cudaEventRecord(ev[4], s);
  k_tail<T><<<1, 256, 0, s>>>(D);
  if (ev) cudaEventRecord(ev[5], s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_damage_field(const Dev<T> &D, const Mat<T> &M, int which, float *out,
                                cudaStream_t s) {
  const int64_t n = (which == PDN_FIELD_DCOH) ? D.nc : D.nh;
  k_damage_field<T><<<grid_of(n, 128), 128, 0, s>>>(D, M, which, out);
  return cudaGetLastError();
}

template cudaError_t launch_pass<float>(const Dev<float> &, const Mat<float> &, cudaStream_t, int32_t,
                                        cudaEvent_t *);
template cudaError_t launch_pass<double>(const Dev<double> &, const Mat<double> &, cudaStream_t, int32_t,
                                         cudaEvent_t *);
template cudaError_t launch_damage_field<float>(const Dev<float> &, const Mat<float> &, int, float *,
                                                cudaStream_t);
template cudaError_t launch_damage_field<double>(const Dev<double> &, const Mat<double> &, int, float *,
                                                 cudaStream_t);

}  // namespace pdn
