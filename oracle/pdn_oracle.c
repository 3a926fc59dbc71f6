/*
 * Plain FP64 CPU oracle of the explicit partial Dirichlet-Neumann (PDN) impact
 * step of Guillamet et al., "Application of the partial Dirichlet-Neumann
 * contact algorithm to simulate low-velocity impact events on composite
 * structures" (Composites Part A, 2022; arXiv 2301.05552).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * Everything is double precision, written as straightforward loops in the
 * order of the paper's algorithms:
 *   - Algorithm 1 (main PDN loop): rigid body first with the contact force of
 *     the previous step (Gauss-Seidel), then the deformable body: predictor,
 *     contact detection, projection (Dirichlet condition), internal forces,
 *     accelerations with the contact reactions, release of adhesion nodes and
 *     repetition of the step (Algorithm 2).
 *   - Sec. 2.2.1: Tchamwa-Wielgosz update with parameter phi (phi = 1 is the
 *     central-difference scheme) and the lumped mass.
 *   - Sec. 2.2.2, Eq. (rk4): RK4 for the rigid striker, m a = m g - f^e.
 *   - Sec. 2 (total Lagrangian hex8, Green strain, 2nd Piola-Kirchhoff S,
 *     nominal stress P, Eq. (fcont)) for the internal forces.
 *   - Algorithm 4 for the intralaminar damage law; Algorithm 5 for the
 *     cohesive law on zero-thickness interface elements (Newton-Cotes).
 *   - Sec. 2.3.1/2.3.2 for the stable time steps.
 *
 * The paper states the order of the constitutive steps but not their closed
 * forms (it cites Maimi 2007, Soto 2018 and Turon 2018).  The closed forms
 * used here are this project's reading of those published models, stated at
 * each function; the same readings are listed in the design notes.
 *
 * Parity status: the hex8 kinematics, the elastic law, the exponential
 * softening laws, the cohesive law, the time integrators and the contact
 * detection are pinned by closed forms and invariants in tests/.  The
 * multiaxial branches of the intralaminar law are pinned against closed-form
 * onset loci solved for the load factor with the ply's Poisson coupling:
 * matrix tension with g = G_YT/G_SL < 1 under combined transverse tension
 * and shear, matrix compression with the fracture-plane friction terms, the
 * damaged compliance with Poisson terms (at D = 1 and in between) and the
 * threshold coupling under mixed loading.  What stays unpinned is the
 * choice of criteria itself (the readings of Algorithm 4 listed below),
 * which the paper does not print.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Records exchanged with the Python test harness (field order matters).    */

typedef struct {
  double rho, E1, E2, E3, nu12, nu13, nu23, G12, G13, G23;
  double XT, XC, YT, YC, SL, alpha0_deg;
  double GXT, GXC, GYT, GYC, GSL;
  double Sp, Kp;
  double GIc, GIIc, tauI, tauII, eta, KI;
  double spread;
  uint64_t seed;
} orc_material;

typedef struct {
  int32_t damage_on, plasticity_on, max_release_iters, n_threads;
  double phi, dt, dt_safety;
  double gravity[3];
} orc_options;

enum { ORC_OK = 0, ORC_E_ARG = -1, ORC_E_NONFINITE = -4, ORC_E_RELEASE_LIMIT = -5 };

#define NH 7 /* history fields per Gauss point: rFT rFC rMT rMC gp12 gp13 pbar */

/* ------------------------------------------------------------------------ */
/* Small dense helpers.                                                     */

static double det3(const double A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

/* Inverse by the adjugate; returns the determinant. */
static double inv3(const double A[3][3], double B[3][3]) {
  double d = det3(A);
  B[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / d;
  B[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / d;
  B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / d;
  B[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / d;
  B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / d;
  B[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / d;
  B[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / d;
  B[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / d;
  B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / d;
  return d;
}

/* Solve A x = b (3x3) by Gaussian elimination with partial pivoting. */
static void solve3(const double Ain[3][3], const double bin[3], double x[3]) {
  double A[3][4];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) A[i][j] = Ain[i][j];
    A[i][3] = bin[i];
  }
  for (int k = 0; k < 3; ++k) {
    int p = k;
    for (int i = k + 1; i < 3; ++i)
      if (fabs(A[i][k]) > fabs(A[p][k])) p = i;
    if (p != k)
      for (int j = 0; j < 4; ++j) {
        double t = A[k][j];
        A[k][j] = A[p][j];
        A[p][j] = t;
      }
    for (int i = k + 1; i < 3; ++i) {
      double f = A[i][k] / A[k][k];
      for (int j = k; j < 4; ++j) A[i][j] -= f * A[k][j];
    }
  }
  for (int i = 2; i >= 0; --i) {
    double s = A[i][3];
    for (int j = i + 1; j < 3; ++j) s -= A[i][j] * x[j];
    x[i] = s / A[i][i];
  }
}

/* ------------------------------------------------------------------------ */
/* Material: undamaged orthotropic compliance H0 and stiffness C0 in ply axes.
 * Voigt order [11, 22, 33, 12, 13, 23] with engineering shear strains.
 * (Algorithm 4: sigma_e = H^-1 eps_e.)                                      */

void orc_compliance(const orc_material *m, double H[6][6]) {
  memset(H, 0, sizeof(double) * 36);
  H[0][0] = 1.0 / m->E1;
  H[1][1] = 1.0 / m->E2;
  H[2][2] = 1.0 / m->E3;
  H[0][1] = H[1][0] = -m->nu12 / m->E1;
  H[0][2] = H[2][0] = -m->nu13 / m->E1;
  H[1][2] = H[2][1] = -m->nu23 / m->E2;
  H[3][3] = 1.0 / m->G12;
  H[4][4] = 1.0 / m->G13;
  H[5][5] = 1.0 / m->G23;
}

void orc_stiffness(const orc_material *m, double C[6][6]) {
  double H[6][6], Hn[3][3], Cn[3][3];
  orc_compliance(m, H);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Hn[i][j] = H[i][j];
  inv3(Hn, Cn);
  memset(C, 0, sizeof(double) * 36);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[i][j] = Cn[i][j];
  C[3][3] = m->G12;
  C[4][4] = m->G13;
  C[5][5] = m->G23;
}

/* ------------------------------------------------------------------------ */
/* Intralaminar damage (Algorithm 4).  Reading of Maimi et al. 2007 with the
 * shear plasticity of Soto et al. 2018, restated:
 *
 *  1. Plasticity on the longitudinal shear pair (12, 13): trial effective
 *     shear tau = G12 (gamma - gamma_p); yield |tau| <= Sp + Kp*G12*pbar
 *     (linear isotropic hardening with modulus Kp*G12); radial return.
 *  2. eps_e = eps - eps_p;  sigma~ = C0 eps_e  (effective stress).
 *  3. Loading functions:
 *       FT: phi = E1 eps_e11 / XT                      (maximum strain)
 *       FC: phi = <-sigma~11> / XC
 *       MT (sigma~22 >= 0): phi^2 = (1-g) s22/YT + g (s22/YT)^2
 *                                  + (tauL/SL)^2 + (s23/ST)^2,
 *           g = GYT/GSL, tauL = sqrt(s12^2 + s13^2)
 *       MC (sigma~22 < 0): phi^2 = (tT^2 + s23^2)/ST^2 + (tL/SL)^2,
 *           tT = <-s22 cos a0 (sin a0 - etaT cos a0)>, tL = <tauL + etaL s22>,
 *           etaT = -1/tan(2 a0), ST = YC cos a0 (sin a0 + cos a0 / tan 2a0),
 *           etaL = -SL cos(2 a0) / (YC cos^2 a0)   (fracture angle a0)
 *  4. Thresholds (irreversible): rFC = max(rFC, phiFC);
 *     rFT = max(rFT, phiFT, rFC); rMC = max(rMC, phiMC);
 *     rMT = max(rMT, phiMT, rMC).
 *  5. Damage: d(r) = 1 - exp(A (1 - r)) / r with
 *     A = 2 lc X^2 / (2 E G - lc X^2)  (crack band: G/lc per unit volume);
 *     A = +inf (d = 1 once r > 1) for elements at or past the snap-back
 *     length lc >= 2 E G / X^2, the limit of the law from below.
 *     D1 = dFT or dFC by the sign of sigma~11 (E1, XT|XC, GXT|GXC);
 *     D2 = dMT or dMC by the sign of sigma~22 (E2, YT|YC, GYT|GYC);
 *     D6 = d6(rMT) with (G12, SL, GSL).
 *  6. Nominal stress sigma = H(D)^-1 eps_e with the damaged compliance
 *     H11 = 1/(E1 (1-D1)), H22 = 1/(E2 (1-D2)), 1/(G12 (1-D6)),
 *     1/(G13 (1-D6)), 1/(G23 (1-D2)); 33 and off-diagonal terms undamaged.
 *     The normal block is solved as M sigma = q o eps_e with M = diag(q) H(D),
 *     q = (1-D1, 1-D2, 1), which stays finite at D = 1.
 * sf = per-element strength factors for (XT, YT, SL).                      */

static double damage_of(double r, double A) {
  if (r <= 1.0) return 0.0;
  return 1.0 - exp(A * (1.0 - r)) / r;
}

/* Past the snap-back length (lc X^2 >= 2 E G) no exponential branch with
 * onset at X dissipates G/lc; the law takes its limit from below, A -> +inf:
 * the stress drops to zero right after onset (dissipation X^2/(2E) per
 * volume, the least possible with that onset). */
static double softening_A(double lc, double X, double E, double G) {
  const double lx2 = lc * X * X, den = 2.0 * E * G - lx2;
  return den > 0.0 ? 2.0 * lx2 / den : INFINITY;
}

static void cdm_point_c(const orc_material *m, const double C0[6][6], const double H[6][6],
                        double lc, const double sf[3], const double eps[6], const double hin[NH],
                        double hout[NH], double sig[6], int damage_on, int plasticity_on);

void orc_cdm_point(const orc_material *m, double lc, const double sf[3], const double eps[6],
                   const double hin[NH], double hout[NH], double sig[6], int damage_on,
                   int plasticity_on) {
  double C0[6][6], H[6][6];
  orc_stiffness(m, C0);
  orc_compliance(m, H);
  cdm_point_c(m, C0, H, lc, sf, eps, hin, hout, sig, damage_on, plasticity_on);
}

/* Same, with the undamaged stiffness C0 and compliance H of the material
 * passed in (computed once per element). */
static void cdm_point_c(const orc_material *m, const double C0[6][6], const double H[6][6],
                        double lc, const double sf[3], const double eps[6], const double hin[NH],
                        double hout[NH], double sig[6], int damage_on, int plasticity_on) {
  double XT = m->XT * sf[0], YT = m->YT * sf[1], SL = m->SL * sf[2];
  double rFT = hin[0], rFC = hin[1], rMT = hin[2], rMC = hin[3];
  double gp12 = hin[4], gp13 = hin[5], pbar = hin[6];

  /* 1. plasticity (longitudinal shear pair) */
  if (plasticity_on) {
    double t12 = m->G12 * (eps[3] - gp12);
    double t13 = m->G12 * (eps[4] - gp13);
    double tn = sqrt(t12 * t12 + t13 * t13);
    double ty = m->Sp + m->Kp * m->G12 * pbar;
    if (tn > ty) {
      double dp = (tn - ty) / (m->G12 * (1.0 + m->Kp));
      gp12 += dp * t12 / tn;
      gp13 += dp * t13 / tn;
      pbar += dp;
    }
  }
  /* 2. elastic strain and effective stress */
  double ee[6] = {eps[0], eps[1], eps[2], eps[3] - gp12, eps[4] - gp13, eps[5]};
  double se[6];
  for (int i = 0; i < 6; ++i) {
    se[i] = 0.0;
    for (int j = 0; j < 6; ++j) se[i] += C0[i][j] * ee[j];
  }
  double D1 = 0.0, D2 = 0.0, D6 = 0.0;
  if (damage_on) {
    /* 3. loading functions */
    double a0 = m->alpha0_deg * M_PI / 180.0;
    double ca = cos(a0), sa = sin(a0);
    double etaT = -1.0 / tan(2.0 * a0);
    double ST = m->YC * ca * (sa + ca / tan(2.0 * a0));
    double etaL = -SL * cos(2.0 * a0) / (m->YC * ca * ca);
    double g = m->GYT / m->GSL;
    double s11 = se[0], s22 = se[1], s12 = se[3], s13 = se[4], s23 = se[5];
    double tauL = sqrt(s12 * s12 + s13 * s13);
    double phiFT = m->E1 * ee[0] / XT;
    double phiFC = (-s11 > 0.0 ? -s11 : 0.0) / m->XC;
    double phiMT = 0.0, phiMC = 0.0;
    if (s22 >= 0.0) {
      double q = (1.0 - g) * s22 / YT + g * (s22 / YT) * (s22 / YT) + (tauL / SL) * (tauL / SL) +
                 (s23 / ST) * (s23 / ST);
      phiMT = sqrt(q);
    } else {
      double tT = -s22 * ca * (sa - etaT * ca);
      if (tT < 0.0) tT = 0.0;
      double tL = tauL + etaL * s22;
      if (tL < 0.0) tL = 0.0;
      phiMC = sqrt((tT * tT + s23 * s23) / (ST * ST) + (tL / SL) * (tL / SL));
    }
    /* 4. thresholds */
    if (phiFC > rFC) rFC = phiFC;
    if (phiFT > rFT) rFT = phiFT;
    if (rFC > rFT) rFT = rFC;
    if (phiMC > rMC) rMC = phiMC;
    if (phiMT > rMT) rMT = phiMT;
    if (rMC > rMT) rMT = rMC;
    /* 5. damage variables */
    double AFT = softening_A(lc, XT, m->E1, m->GXT);
    double AFC = softening_A(lc, m->XC, m->E1, m->GXC);
    double AMT = softening_A(lc, YT, m->E2, m->GYT);
    double AMC = softening_A(lc, m->YC, m->E2, m->GYC);
    double A6 = softening_A(lc, SL, m->G12, m->GSL);
    D1 = (s11 >= 0.0) ? damage_of(rFT, AFT) : damage_of(rFC, AFC);
    D2 = (s22 >= 0.0) ? damage_of(rMT, AMT) : damage_of(rMC, AMC);
    D6 = damage_of(rMT, A6);
  }
  /* 6. nominal stress through the damaged compliance */
  double q[3] = {1.0 - D1, 1.0 - D2, 1.0};
  double M3[3][3], rhs[3], sn[3];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) M3[i][j] = (i == j) ? H[i][i] : q[i] * H[i][j];
    rhs[i] = q[i] * ee[i];
  }
  solve3(M3, rhs, sn);
  sig[0] = sn[0];
  sig[1] = sn[1];
  sig[2] = sn[2];
  sig[3] = (1.0 - D6) * m->G12 * ee[3];
  sig[4] = (1.0 - D6) * m->G13 * ee[4];
  sig[5] = (1.0 - D2) * m->G23 * ee[5];
  hout[0] = rFT;
  hout[1] = rFC;
  hout[2] = rMT;
  hout[3] = rMC;
  hout[4] = gp12;
  hout[5] = gp13;
  hout[6] = pbar;
}

/* Damage variables of a history record (for field output):
 * out = {max(dFT,dFC), max(dMT,dMC), d6}. */
void orc_damage_of_history(const orc_material *m, double lc, const double sf[3],
                           const double h[NH], double out[3]) {
  double XT = m->XT * sf[0], YT = m->YT * sf[1], SL = m->SL * sf[2];
  double dFT = damage_of(h[0], softening_A(lc, XT, m->E1, m->GXT));
  double dFC = damage_of(h[1], softening_A(lc, m->XC, m->E1, m->GXC));
  double dMT = damage_of(h[2], softening_A(lc, YT, m->E2, m->GYT));
  double dMC = damage_of(h[3], softening_A(lc, m->YC, m->E2, m->GYC));
  out[0] = dFT > dFC ? dFT : dFC;
  out[1] = dMT > dMC ? dMT : dMC;
  out[2] = damage_of(h[2], softening_A(lc, SL, m->G12, m->GSL));
}

/* ------------------------------------------------------------------------ */
/* Cohesive law (Algorithm 5), reading of Turon et al. 2018:
 *   Kpen_I = KI, Kpen_sh = KI (GIc/GIIc) (tauII/tauI)^2
 *   D3o = tauI/KI, D3c = 2 GIc/tauI, Dsho = tauII/Ksh, Dshc = 2 GIIc/tauII
 *   Dsh = sqrt(D1^2 + D2^2), <D3> = max(D3, 0)
 *   B   = Ksh Dsh^2 / (Ksh Dsh^2 + KI <D3>^2)             (mixed-mode ratio)
 *   KB  = (1 - B) KI + B Ksh                              (mixed-mode stiffness)
 *   lam = sqrt((KI <D3>^2 + Ksh Dsh^2) / KB)              (equivalent jump)
 *   lo  = sqrt((KI D3o^2 + (Ksh Dsho^2 - KI D3o^2) B^eta) / KB)
 *   lc  = (KI D3o D3c + (Ksh Dsho Dshc - KI D3o D3c) B^eta) / (KB lo)
 *   H   = (lam - lo)/(lc - lo);  rD = max(rD, min(1, max(0, H)))
 *   D   = rD lc / (rD lc + (1 - rD) lo)
 *   tau_coh = (1 - D) K Delta; contact part restores KI D3 for D3 < 0.
 * Delta and tau are in the local interface frame (1, 2 tangential, 3 normal). */
void orc_czm_point(const orc_material *m, const double dl[3], double rD_in, double *rD_out,
                   double tau[3]) {
  double KI = m->KI;
  double Ksh = KI * (m->GIc / m->GIIc) * (m->tauII / m->tauI) * (m->tauII / m->tauI);
  double D3o = m->tauI / KI, D3c = 2.0 * m->GIc / m->tauI;
  double Dsho = m->tauII / Ksh, Dshc = 2.0 * m->GIIc / m->tauII;
  double dsh = sqrt(dl[0] * dl[0] + dl[1] * dl[1]);
  double d3p = dl[2] > 0.0 ? dl[2] : 0.0;
  double num = Ksh * dsh * dsh, den = Ksh * dsh * dsh + KI * d3p * d3p;
  double B = den > 0.0 ? num / den : 0.0;
  double KB = (1.0 - B) * KI + B * Ksh;
  double lam = sqrt((KI * d3p * d3p + Ksh * dsh * dsh) / KB);
  double Beta = pow(B, m->eta);
  double lo = sqrt((KI * D3o * D3o + (Ksh * Dsho * Dsho - KI * D3o * D3o) * Beta) / KB);
  double lcr = (KI * D3o * D3c + (Ksh * Dsho * Dshc - KI * D3o * D3c) * Beta) / (KB * lo);
  double Hl = (lam - lo) / (lcr - lo);
  if (Hl < 0.0) Hl = 0.0;
  if (Hl > 1.0) Hl = 1.0;
  double rD = rD_in > Hl ? rD_in : Hl;
  double D = rD * lcr / (rD * lcr + (1.0 - rD) * lo);
  tau[0] = (1.0 - D) * Ksh * dl[0];
  tau[1] = (1.0 - D) * Ksh * dl[1];
  tau[2] = (dl[2] >= 0.0) ? (1.0 - D) * KI * dl[2] : KI * dl[2];
  *rD_out = rD;
}

/* Interface damage of a stored threshold at a given jump direction's B is
 * direction dependent; the field output reports the threshold rD itself. */

/* ------------------------------------------------------------------------ */
/* Hex8 element, total Lagrangian, 2x2x2 Gauss (Sec. 2; Eq. fcont).         */

static const double SGN[8][3] = {{-1, -1, -1}, {1, -1, -1}, {1, 1, -1}, {-1, 1, -1},
                                 {-1, -1, 1},  {1, -1, 1},  {1, 1, 1},  {-1, 1, 1}};

static void shape_grad_nat(double xi, double eta, double zeta, double dN[8][3]) {
  for (int a = 0; a < 8; ++a) {
    double sx = SGN[a][0], sy = SGN[a][1], sz = SGN[a][2];
    dN[a][0] = 0.125 * sx * (1.0 + eta * sy) * (1.0 + zeta * sz);
    dN[a][1] = 0.125 * sy * (1.0 + xi * sx) * (1.0 + zeta * sz);
    dN[a][2] = 0.125 * sz * (1.0 + xi * sx) * (1.0 + eta * sy);
  }
}

/* Reference-configuration gradients at Gauss point g: dN/dX and det J. */
static double hex8_gauss_grad(const double X[8][3], int g, double dNdX[8][3]) {
  double gpv = 1.0 / sqrt(3.0);
  double dN[8][3], J[3][3], Ji[3][3];
  shape_grad_nat(SGN[g][0] * gpv, SGN[g][1] * gpv, SGN[g][2] * gpv, dN);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      J[i][j] = 0.0;
      for (int a = 0; a < 8; ++a) J[i][j] += X[a][i] * dN[a][j];
    }
  double detJ = inv3(J, Ji);
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i) {
      dNdX[a][i] = 0.0;
      for (int j = 0; j < 3; ++j) dNdX[a][i] += dN[a][j] * Ji[j][i];
    }
  return detJ;
}

double orc_hex8_volume(const double X[8][3]) {
  double dNdX[8][3], V = 0.0;
  for (int g = 0; g < 8; ++g) V += hex8_gauss_grad(X, g, dNdX);
  return V;
}

/* Internal force of one hex8: f[a][i] = sum_g w detJ dN_a/dX_j P_ji with
 * P = S F^T, S from the ply law on the Green strain rotated into ply axes
 * (rotation by the ply angle about z, fixed in the reference configuration).
 * Returns the element's strain energy sum_g 1/2 S:E detJ (meaningful for
 * elastic states). */
double orc_hex8_force(const orc_material *m, double angle_deg, double lc, const double sf[3],
                      const double X[8][3], const double u[8][3], const double *hin,
                      double *hout, double f[8][3], int damage_on, int plasticity_on) {
  double th = angle_deg * M_PI / 180.0;
  double c = cos(th), s = sin(th);
  /* columns of R are the ply axes in global coordinates */
  double R[3][3] = {{c, -s, 0.0}, {s, c, 0.0}, {0.0, 0.0, 1.0}};
  double C0[6][6], Hc[6][6];
  orc_stiffness(m, C0);
  orc_compliance(m, Hc);
  double energy = 0.0;
  for (int a = 0; a < 8; ++a) f[a][0] = f[a][1] = f[a][2] = 0.0;
  for (int g = 0; g < 8; ++g) {
    double dNdX[8][3];
    double detJ = hex8_gauss_grad(X, g, dNdX);
    double Hg[3][3], F[3][3], E[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        Hg[i][j] = 0.0;
        for (int a = 0; a < 8; ++a) Hg[i][j] += u[a][i] * dNdX[a][j];
      }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) F[i][j] = Hg[i][j] + (i == j ? 1.0 : 0.0);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double ftf = 0.0;
        for (int k = 0; k < 3; ++k) ftf += F[k][i] * F[k][j];
        E[i][j] = 0.5 * (ftf - (i == j ? 1.0 : 0.0));
      }
    /* E in ply axes: Em = R^T E R */
    double Em[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double t = 0.0;
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) t += R[k][i] * E[k][l] * R[l][j];
        Em[i][j] = t;
      }
    double eps[6] = {Em[0][0], Em[1][1], Em[2][2], 2.0 * Em[0][1], 2.0 * Em[0][2], 2.0 * Em[1][2]};
    double sig[6];
    cdm_point_c(m, C0, Hc, lc, sf, eps, hin + g * NH, hout + g * NH, sig, damage_on, plasticity_on);
    double Sm[3][3] = {{sig[0], sig[3], sig[4]}, {sig[3], sig[1], sig[5]}, {sig[4], sig[5], sig[2]}};
    /* back to global axes: S = R Sm R^T */
    double S[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double t = 0.0;
        for (int k = 0; k < 3; ++k)
          for (int l = 0; l < 3; ++l) t += R[i][k] * Sm[k][l] * R[j][l];
        S[i][j] = t;
      }
    double se = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) se += S[i][j] * E[i][j];
    energy += 0.5 * se * detJ;
    /* P = S F^T */
    double P[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double t = 0.0;
        for (int k = 0; k < 3; ++k) t += S[i][k] * F[j][k];
        P[i][j] = t;
      }
    for (int a = 0; a < 8; ++a)
      for (int i = 0; i < 3; ++i) {
        double t = 0.0;
        for (int j = 0; j < 3; ++j) t += dNdX[a][j] * P[j][i];
        f[a][i] += t * detJ; /* Gauss weight 1 */
      }
  }
  return energy;
}

/* ------------------------------------------------------------------------ */
/* Zero-thickness 8-node interface element with Newton-Cotes (nodal)
 * integration (Sec. 2.3.2).  Nodes 0-3 bottom face, 4-7 top face, node a+4
 * coincident with node a.  Local frame from the reference mid-surface at the
 * element centre (e1 along the xi tangent, e3 the unit normal, e2 = e3 x e1);
 * point weights are the surface Jacobians at the corners. Internal force on
 * the top node +w tau, on the bottom node -w tau. Returns nothing. */
static const double QS[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};

void orc_coh8_force(const orc_material *m, const double X[8][3], const double u[8][3],
                    const double rD_in[4], double rD_out[4], double f[8][3]) {
  double Xm[4][3];
  for (int a = 0; a < 4; ++a)
    for (int i = 0; i < 3; ++i) Xm[a][i] = 0.5 * (X[a][i] + X[a + 4][i]);
  /* tangents at a point (xi, eta) of the bilinear quad */
  double e1[3], e2[3], e3[3];
  {
    double tx[3] = {0, 0, 0}, ty[3] = {0, 0, 0};
    for (int a = 0; a < 4; ++a)
      for (int i = 0; i < 3; ++i) {
        tx[i] += 0.25 * QS[a][0] * Xm[a][i];
        ty[i] += 0.25 * QS[a][1] * Xm[a][i];
      }
    double n[3] = {tx[1] * ty[2] - tx[2] * ty[1], tx[2] * ty[0] - tx[0] * ty[2],
                   tx[0] * ty[1] - tx[1] * ty[0]};
    double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double tn = sqrt(tx[0] * tx[0] + tx[1] * tx[1] + tx[2] * tx[2]);
    for (int i = 0; i < 3; ++i) {
      e3[i] = n[i] / nn;
      e1[i] = tx[i] / tn;
    }
    e2[0] = e3[1] * e1[2] - e3[2] * e1[1];
    e2[1] = e3[2] * e1[0] - e3[0] * e1[2];
    e2[2] = e3[0] * e1[1] - e3[1] * e1[0];
  }
  for (int a = 0; a < 8; ++a) f[a][0] = f[a][1] = f[a][2] = 0.0;
  for (int p = 0; p < 4; ++p) {
    double xi = QS[p][0], eta = QS[p][1];
    double tx[3] = {0, 0, 0}, ty[3] = {0, 0, 0};
    for (int a = 0; a < 4; ++a) {
      double dxi = 0.25 * QS[a][0] * (1.0 + eta * QS[a][1]);
      double deta = 0.25 * QS[a][1] * (1.0 + xi * QS[a][0]);
      for (int i = 0; i < 3; ++i) {
        tx[i] += dxi * Xm[a][i];
        ty[i] += deta * Xm[a][i];
      }
    }
    double n[3] = {tx[1] * ty[2] - tx[2] * ty[1], tx[2] * ty[0] - tx[0] * ty[2],
                   tx[0] * ty[1] - tx[1] * ty[0]};
    double w = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]); /* Newton-Cotes weight 1 */
    double dg[3], dl[3], tau[3];
    for (int i = 0; i < 3; ++i) dg[i] = u[p + 4][i] - u[p][i];
    dl[0] = e1[0] * dg[0] + e1[1] * dg[1] + e1[2] * dg[2];
    dl[1] = e2[0] * dg[0] + e2[1] * dg[1] + e2[2] * dg[2];
    dl[2] = e3[0] * dg[0] + e3[1] * dg[1] + e3[2] * dg[2];
    orc_czm_point(m, dl, rD_in[p], &rD_out[p], tau);
    for (int i = 0; i < 3; ++i) {
      double tg = tau[0] * e1[i] + tau[1] * e2[i] + tau[2] * e3[i];
      f[p + 4][i] += w * tg;
      f[p][i] -= w * tg;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Seeded strength factors: SplitMix64 (Steele, Lea and Flood 2014) applied
 * to seed XOR (element*4 + k), mapped to U[1 - spread, 1 + spread].        */
static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double orc_strength_factor(uint64_t seed, int64_t elem, int k, double spread) {
  uint64_t z = splitmix64(seed ^ (uint64_t)(elem * 4 + k));
  double u = (double)(z >> 11) * (1.0 / 9007199254740992.0); /* [0,1) */
  return 1.0 + spread * (2.0 * u - 1.0);
}

/* ------------------------------------------------------------------------ */
/* The model.                                                               */

typedef struct {
  int64_t nn, nh, nc, ns;
  double *X;       /* [nn][3] */
  int32_t *hex;    /* [nh][8] */
  int32_t *coh;    /* [nc][8] */
  int8_t *ply_hex; /* [nh] */
  double *ply_angle;
  int32_t n_plies;
  uint8_t *fixed; /* [nn] constraint bits: 1 x, 2 y, 4 z (7 = clamped) */
  int32_t *surf;  /* [ns] */
  orc_material mat;
  orc_options opt;
  double *mass; /* [nn] */
  double *lc;   /* [nh] */
  double *sf;   /* [nh][3] */
  double dt, dt_bulk, dt_coh;
  /* state */
  double *d, *v, *a; /* [nn][3] */
  double *hist;      /* [nh][8][NH] */
  double *rD;        /* [nc][4] */
  double R, Mimp, c[3], w[3], axis[3];
  int has_imp;
  double F[3]; /* contact force on the plate, sum_j lambda_j n_j */
  int64_t step;
  double time;
  double *fhist;
  int64_t fhist_cap, fhist_n;
  double fpeak;
  /* last committed step */
  uint8_t *active;   /* [ns] */
  double *lambda;    /* [ns] */
  int64_t n_active, n_repeats_total, last_repeats;
  /* work */
  double *fe_hex, *fe_coh, *hist_new, *rD_new, *dn, *vn, *an, *fi;
  uint8_t *released, *act_try;
  double *lam_try;
  int status;
} orc_model;

static void *xcalloc(size_t n, size_t s) {
  void *p = calloc(n ? n : 1, s);
  if (!p) {
    fprintf(stderr, "oracle: out of memory\n");
    abort();
  }
  return p;
}

static void gather_X(const orc_model *M, const int32_t *conn, double Xe[8][3]) {
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i) Xe[a][i] = M->X[(int64_t)conn[a] * 3 + i];
}

static void gather_u(const orc_model *M, const double *d, const int32_t *conn, double ue[8][3]) {
  (void)M;
  for (int a = 0; a < 8; ++a)
    for (int i = 0; i < 3; ++i) ue[a][i] = d[(int64_t)conn[a] * 3 + i];
}

/* Create: X is SoA [3][nn] as delivered by the input generator. */
static void acceleration_of_state(orc_model *M);

orc_model *orc_create(int64_t nn, int64_t nh, int64_t nc, int64_t ns, const double *X_soa,
                      const int32_t *hex, const int32_t *coh, const int8_t *ply_hex,
                      const double *ply_angle, int32_t n_plies, const uint8_t *fixed,
                      const int32_t *surf, const orc_material *mat, const orc_options *opt,
                      int64_t fhist_cap) {
  orc_model *M = (orc_model *)xcalloc(1, sizeof(orc_model));
  M->nn = nn;
  M->nh = nh;
  M->nc = nc;
  M->ns = ns;
  M->mat = *mat;
  M->opt = *opt;
  M->X = (double *)xcalloc((size_t)nn * 3, sizeof(double));
  for (int64_t j = 0; j < nn; ++j)
    for (int i = 0; i < 3; ++i) M->X[j * 3 + i] = X_soa[i * nn + j];
  M->hex = (int32_t *)xcalloc((size_t)nh * 8, sizeof(int32_t));
  memcpy(M->hex, hex, sizeof(int32_t) * nh * 8);
  M->coh = (int32_t *)xcalloc((size_t)nc * 8, sizeof(int32_t));
  if (nc) memcpy(M->coh, coh, sizeof(int32_t) * nc * 8);
  M->ply_hex = (int8_t *)xcalloc((size_t)nh, 1);
  memcpy(M->ply_hex, ply_hex, nh);
  M->n_plies = n_plies;
  M->ply_angle = (double *)xcalloc(n_plies, sizeof(double));
  memcpy(M->ply_angle, ply_angle, sizeof(double) * n_plies);
  M->fixed = (uint8_t *)xcalloc((size_t)nn, 1);
  memcpy(M->fixed, fixed, nn);
  M->surf = (int32_t *)xcalloc((size_t)ns, sizeof(int32_t));
  memcpy(M->surf, surf, sizeof(int32_t) * ns);

  /* Lumped (row-sum) mass, Sec. 2.2.1: m_a = sum_e sum_g rho N_a(xi_g) detJ_g. */
  M->mass = (double *)xcalloc((size_t)nn, sizeof(double));
  M->lc = (double *)xcalloc((size_t)nh, sizeof(double));
  M->sf = (double *)xcalloc((size_t)nh * 3, sizeof(double));
  double C0[6][6];
  orc_stiffness(mat, C0);
  double cmax = 0.0;
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j)
      if (fabs(C0[i][j]) > cmax) cmax = fabs(C0[i][j]);
  double gpv = 1.0 / sqrt(3.0);
  double dtb = INFINITY;
  for (int64_t e = 0; e < nh; ++e) {
    double Xe[8][3];
    gather_X(M, M->hex + e * 8, Xe);
    double V = 0.0;
    for (int g = 0; g < 8; ++g) {
      double dNdX[8][3];
      double detJ = hex8_gauss_grad(Xe, g, dNdX);
      V += detJ;
      double xi = SGN[g][0] * gpv, eta = SGN[g][1] * gpv, zeta = SGN[g][2] * gpv;
      for (int a = 0; a < 8; ++a) {
        double Na = 0.125 * (1 + xi * SGN[a][0]) * (1 + eta * SGN[a][1]) * (1 + zeta * SGN[a][2]);
        M->mass[M->hex[e * 8 + a]] += mat->rho * Na * detJ;
      }
    }
    /* Sec. 2.3.1: lc ~ V^(1/3); dt = lc sqrt(rho / max Cij) */
    M->lc[e] = cbrt(V);
    double dte = M->lc[e] * sqrt(mat->rho / cmax);
    if (dte < dtb) dtb = dte;
    for (int k = 0; k < 3; ++k) M->sf[e * 3 + k] = orc_strength_factor(mat->seed, e, k, mat->spread);
  }
  /* Sec. 2.3.2: dt_coh = sqrt(rho_bar / Kcoh), rho_bar = rho * h with h the
   * thickness (volume / interface area) of the thinner adjacent hex. */
  double dtc = INFINITY;
  if (nc) {
    /* node -> adjacent hexes (CSR) to find the hexes on each side of a face */
    int64_t *cnt = (int64_t *)xcalloc((size_t)nn + 1, sizeof(int64_t));
    for (int64_t e = 0; e < nh; ++e)
      for (int a = 0; a < 8; ++a) cnt[M->hex[e * 8 + a] + 1]++;
    for (int64_t j = 0; j < nn; ++j) cnt[j + 1] += cnt[j];
    int64_t *adj = (int64_t *)xcalloc((size_t)cnt[nn], sizeof(int64_t));
    int64_t *fill = (int64_t *)xcalloc((size_t)nn, sizeof(int64_t));
    for (int64_t e = 0; e < nh; ++e)
      for (int a = 0; a < 8; ++a) {
        int64_t j = M->hex[e * 8 + a];
        adj[cnt[j] + fill[j]++] = e;
      }
    for (int64_t ce = 0; ce < nc; ++ce) {
      double hmin = INFINITY;
      for (int side = 0; side < 2; ++side) {
        const int32_t *fn = M->coh + ce * 8 + side * 4;
        for (int64_t q = cnt[fn[0]]; q < cnt[fn[0] + 1]; ++q) {
          int64_t e = adj[q];
          const int32_t *hn = M->hex + e * 8;
          int hit = 0;
          for (int k = 0; k < 4; ++k)
            for (int a = 0; a < 8; ++a)
              if (hn[a] == fn[k]) {
                ++hit;
                break;
              }
          if (hit != 4) continue;
          double Xe[8][3];
          gather_X(M, hn, Xe);
          double V = orc_hex8_volume(Xe);
          /* area of the interface quad from its diagonals */
          double p[4][3];
          for (int k = 0; k < 4; ++k)
            for (int i = 0; i < 3; ++i) p[k][i] = M->X[(int64_t)fn[k] * 3 + i];
          double u1[3], u2[3], cr[3];
          for (int i = 0; i < 3; ++i) {
            u1[i] = p[2][i] - p[0][i];
            u2[i] = p[3][i] - p[1][i];
          }
          cr[0] = u1[1] * u2[2] - u1[2] * u2[1];
          cr[1] = u1[2] * u2[0] - u1[0] * u2[2];
          cr[2] = u1[0] * u2[1] - u1[1] * u2[0];
          double A = 0.5 * sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
          double h = V / A;
          if (h < hmin) hmin = h;
        }
      }
      double dte = sqrt(mat->rho * hmin / mat->KI);
      if (dte < dtc) dtc = dte;
    }
    free(cnt);
    free(adj);
    free(fill);
  }
  M->dt_bulk = dtb;
  M->dt_coh = dtc;
  double dtmin = dtb < dtc ? dtb : dtc;
  M->dt = opt->dt > 0.0 ? opt->dt : opt->dt_safety * dtmin;

  M->d = (double *)xcalloc((size_t)nn * 3, sizeof(double));
  M->v = (double *)xcalloc((size_t)nn * 3, sizeof(double));
  M->a = (double *)xcalloc((size_t)nn * 3, sizeof(double));
  M->dn = (double *)xcalloc((size_t)nn * 3, sizeof(double));
  M->vn = (double *)xcalloc((size_t)nn * 3, sizeof(double));
  M->an = (double *)xcalloc((size_t)nn * 3, sizeof(double));
  M->fi = (double *)xcalloc((size_t)nn * 3, sizeof(double));
  M->hist = (double *)xcalloc((size_t)nh * 8 * NH, sizeof(double));
  M->hist_new = (double *)xcalloc((size_t)nh * 8 * NH, sizeof(double));
  for (int64_t e = 0; e < nh; ++e)
    for (int g = 0; g < 8; ++g)
      for (int k = 0; k < 4; ++k) M->hist[(e * 8 + g) * NH + k] = 1.0; /* r_N = 1 */
  M->rD = (double *)xcalloc((size_t)nc * 4, sizeof(double));
  M->rD_new = (double *)xcalloc((size_t)nc * 4, sizeof(double));
  M->fe_hex = (double *)xcalloc((size_t)nh * 24, sizeof(double));
  M->fe_coh = (double *)xcalloc((size_t)nc * 24, sizeof(double));
  M->active = (uint8_t *)xcalloc((size_t)ns, 1);
  M->act_try = (uint8_t *)xcalloc((size_t)ns, 1);
  M->released = (uint8_t *)xcalloc((size_t)ns, 1);
  M->lambda = (double *)xcalloc((size_t)ns, sizeof(double));
  M->lam_try = (double *)xcalloc((size_t)ns, sizeof(double));
  M->fhist_cap = fhist_cap;
  M->fhist = (double *)xcalloc((size_t)(fhist_cap > 0 ? fhist_cap : 1), sizeof(double));
  M->axis[2] = -1.0;
  /* The discrete momentum equation (Sec. 2.2.1) holds at step 0 as well:
   * a^0 = m^-1 (f^e - f^i(d^0)); with d^0 = 0 and no contact at t^0 this is
   * the gravity acceleration on every free degree of freedom. */
  acceleration_of_state(M);
  return M;
}

void orc_destroy(orc_model *M) {
  if (!M) return;
  void *ps[] = {M->X, M->hex, M->coh, M->ply_hex, M->ply_angle, M->fixed, M->surf, M->mass,
                M->lc, M->sf, M->d, M->v, M->a, M->hist, M->rD, M->fhist, M->active,
                M->lambda, M->fe_hex, M->fe_coh, M->hist_new, M->rD_new, M->dn, M->vn, M->an,
                M->fi, M->released, M->act_try, M->lam_try};
  for (size_t i = 0; i < sizeof(ps) / sizeof(ps[0]); ++i) free(ps[i]);
  free(M);
}

void orc_set_impactor(orc_model *M, double R, double mass, const double c[3], const double w[3]) {
  M->R = R;
  M->Mimp = mass;
  double n = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  for (int i = 0; i < 3; ++i) {
    M->c[i] = c[i];
    M->w[i] = w[i];
    M->axis[i] = n > 0.0 ? w[i] / n : (i == 2 ? -1.0 : 0.0);
    M->F[i] = 0.0;
  }
  M->has_imp = 1;
}

/* Internal forces at displacement d with history hin -> hout; results into
 * M->fi (nodal, [nn][3]) by scattering element forces in ascending element
 * order (hexes first, then interface elements).  Element forces are
 * independent, so they are evaluated in parallel; the scatter is serial. */
static void internal_forces(orc_model *M, const double *d, const double *hin, double *hout,
                            const double *rDin, double *rDout) {
  int64_t nh = M->nh, nc = M->nc;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < nh; ++e) {
    double Xe[8][3], ue[8][3], fe[8][3];
    gather_X(M, M->hex + e * 8, Xe);
    gather_u(M, d, M->hex + e * 8, ue);
    orc_hex8_force(&M->mat, M->ply_angle[M->ply_hex[e]], M->lc[e], M->sf + e * 3, Xe, ue,
                   hin + e * 8 * NH, hout + e * 8 * NH, fe, M->opt.damage_on, M->opt.plasticity_on);
    memcpy(M->fe_hex + e * 24, fe, sizeof(fe));
  }
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < nc; ++e) {
    double Xe[8][3], ue[8][3], fe[8][3];
    gather_X(M, M->coh + e * 8, Xe);
    gather_u(M, d, M->coh + e * 8, ue);
    if (M->opt.damage_on) {
      orc_coh8_force(&M->mat, Xe, ue, rDin + e * 4, rDout + e * 4, fe);
    } else {
      /* interface stays elastic: evaluate with a frozen undamaged threshold */
      double r0[4] = {0, 0, 0, 0}, r1[4];
      orc_coh8_force(&M->mat, Xe, ue, r0, r1, fe);
      for (int p = 0; p < 4; ++p) rDout[e * 4 + p] = rDin[e * 4 + p];
    }
    memcpy(M->fe_coh + e * 24, fe, sizeof(fe));
  }
  memset(M->fi, 0, sizeof(double) * M->nn * 3);
  for (int64_t e = 0; e < nh; ++e)
    for (int a = 0; a < 8; ++a)
      for (int i = 0; i < 3; ++i) M->fi[(int64_t)M->hex[e * 8 + a] * 3 + i] += M->fe_hex[e * 24 + a * 3 + i];
  for (int64_t e = 0; e < nc; ++e)
    for (int a = 0; a < 8; ++a)
      for (int i = 0; i < 3; ++i) M->fi[(int64_t)M->coh[e * 8 + a] * 3 + i] += M->fe_coh[e * 24 + a * 3 + i];
}

/* Nodal internal force at the current state, without advancing (for checks). */
void orc_internal_force(orc_model *M, double *f_out_soa) {
  internal_forces(M, M->d, M->hist, M->hist_new, M->rD, M->rD_new);
  for (int64_t j = 0; j < M->nn; ++j)
    for (int i = 0; i < 3; ++i) f_out_soa[i * M->nn + j] = M->fi[j * 3 + i];
}

/* One time step n -> n+1 (Algorithm 1 with the reset loop of Algorithm 2). */
/* Acceleration of the installed state (d, v) without contact, from the
 * momentum equation of Sec. 2.2.1: a = m^-1 (m g - f^i(d)) on free degrees
 * of freedom, 0 on fixed ones.  The history is left as it is. */
static void acceleration_of_state(orc_model *M) {
  internal_forces(M, M->d, M->hist, M->hist_new, M->rD, M->rD_new);
  const double *g = M->opt.gravity;
  for (int64_t j = 0; j < M->nn; ++j)
    for (int i = 0; i < 3; ++i)
      M->a[j * 3 + i] =
          ((M->fixed[j] >> i) & 1) ? 0.0 : (M->mass[j] * g[i] - M->fi[j * 3 + i]) / M->mass[j];
}

static int one_step(orc_model *M) {
  int64_t nn = M->nn, ns = M->ns;
  double dt = M->dt, phi = M->opt.phi;
  const double *g = M->opt.gravity;

  /* Rigid body (Sec. 2.2.2): m a = m g - f^e, f^e = sum of contact forces,
   * the body constrained to its impact axis; RK4 of Eq. (rk4) with the
   * contact force of the previous step held over the step. */
  double aI[3] = {0, 0, 0}, cn[3], wn[3];
  if (M->has_imp) {
    double ga[3];
    for (int i = 0; i < 3; ++i) ga[i] = g[i] - M->F[i] / M->Mimp;
    double an = ga[0] * M->axis[0] + ga[1] * M->axis[1] + ga[2] * M->axis[2];
    for (int i = 0; i < 3; ++i) aI[i] = an * M->axis[i];
    /* y = (c, w), y' = (w, aI) */
    double k1c[3], k1w[3], k2c[3], k2w[3], k3c[3], k3w[3], k4c[3], k4w[3];
    for (int i = 0; i < 3; ++i) {
      k1c[i] = dt * M->w[i];
      k1w[i] = dt * aI[i];
      k2c[i] = dt * (M->w[i] + 0.5 * k1w[i]);
      k2w[i] = dt * aI[i];
      k3c[i] = dt * (M->w[i] + 0.5 * k2w[i]);
      k3w[i] = dt * aI[i];
      k4c[i] = dt * (M->w[i] + k3w[i]);
      k4w[i] = dt * aI[i];
      cn[i] = M->c[i] + k1c[i] / 6.0 + k2c[i] / 3.0 + k3c[i] / 3.0 + k4c[i] / 6.0;
      wn[i] = M->w[i] + k1w[i] / 6.0 + k2w[i] / 3.0 + k3w[i] / 3.0 + k4w[i] / 6.0;
    }
  } else {
    for (int i = 0; i < 3; ++i) {
      cn[i] = M->c[i];
      wn[i] = M->w[i];
    }
  }

  memset(M->released, 0, ns);
  int iter = 0;
  int64_t n_act = 0;
  for (;;) {
    /* Deformable body: Tchamwa-Wielgosz predictor (Sec. 2.2.1) */
    for (int64_t j = 0; j < nn; ++j)
      for (int i = 0; i < 3; ++i) {
        int64_t k = j * 3 + i;
        if ((M->fixed[j] >> i) & 1) {
          M->dn[k] = 0.0;
          M->vn[k] = 0.0;
        } else {
          M->dn[k] = M->d[k] + dt * M->v[k] + phi * dt * dt * M->a[k];
          M->vn[k] = M->v[k] + dt * M->a[k];
        }
      }
    /* Contact detection and projection onto the rigid sphere (Sec. 2.1):
     * penetrated slave nodes (gap < 0), and nodes that were in contact at the
     * end of the previous step, get a Dirichlet condition on the master
     * surface: position projected along the sphere normal, normal velocity set
     * to the striker's, tangential motion free.  A node leaves the contact set
     * only through the release of Algorithm 2 (adhesive reaction). */
    n_act = 0;
    for (int64_t s = 0; s < ns; ++s) {
      M->act_try[s] = 0;
      M->lam_try[s] = 0.0;
      int64_t j = M->surf[s];
      if (!M->has_imp || M->released[s] || M->fixed[j] == 7) continue;
      double x[3], r2 = 0.0;
      for (int i = 0; i < 3; ++i) {
        x[i] = M->X[j * 3 + i] + M->dn[j * 3 + i] - cn[i];
        r2 += x[i] * x[i];
      }
      double r = sqrt(r2);
      double gap = r - M->R;
      if (gap < 0.0 || M->active[s]) {
        M->act_try[s] = 1;
        ++n_act;
        double nrm[3] = {x[0] / r, x[1] / r, x[2] / r};
        double vn_dot = 0.0, wn_dot = 0.0;
        for (int i = 0; i < 3; ++i) {
          vn_dot += M->vn[j * 3 + i] * nrm[i];
          wn_dot += wn[i] * nrm[i];
        }
        for (int i = 0; i < 3; ++i) {
          if ((M->fixed[j] >> i) & 1) continue;
          M->dn[j * 3 + i] -= gap * nrm[i];
          M->vn[j * 3 + i] += (wn_dot - vn_dot) * nrm[i];
        }
      }
    }
    /* Internal forces at d^{n+1} with trial history */
    internal_forces(M, M->dn, M->hist, M->hist_new, M->rD, M->rD_new);
    /* Accelerations: a = m^-1 (f^e - f^i) for free nodes (Sec. 2.2.1) */
    for (int64_t j = 0; j < nn; ++j)
      for (int i = 0; i < 3; ++i) {
        int64_t k = j * 3 + i;
        M->an[k] = ((M->fixed[j] >> i) & 1) ? 0.0 : (M->mass[j] * g[i] - M->fi[k]) / M->mass[j];
      }
    /* Contact nodes: reaction lambda_j along n_j such that the normal
     * acceleration follows the striker's; adhesion iff lambda_j < 0
     * (Eq. anodes; Algorithm 2). */
    int any_adh = 0;
    for (int64_t s = 0; s < ns; ++s) {
      if (!M->act_try[s]) continue;
      int64_t j = M->surf[s];
      double x[3], r2 = 0.0;
      for (int i = 0; i < 3; ++i) {
        x[i] = M->X[j * 3 + i] + M->dn[j * 3 + i] - cn[i];
        r2 += x[i] * x[i];
      }
      double r = sqrt(r2);
      double nrm[3] = {x[0] / r, x[1] / r, x[2] / r};
      double fdot = 0.0, adot = 0.0;
      for (int i = 0; i < 3; ++i) {
        fdot += (M->mass[j] * g[i] - M->fi[j * 3 + i]) * nrm[i];
        adot += aI[i] * nrm[i];
      }
      double lam = M->mass[j] * adot - fdot;
      M->lam_try[s] = lam;
      if (lam < 0.0) {
        any_adh = 1;
        M->released[s] = 1;
      } else {
        for (int i = 0; i < 3; ++i)
          if (!((M->fixed[j] >> i) & 1)) M->an[j * 3 + i] += lam * nrm[i] / M->mass[j];
      }
    }
    if (!any_adh) break;
    if (iter >= M->opt.max_release_iters) {
      M->status = ORC_E_RELEASE_LIMIT;
      return M->status;
    }
    ++iter;
  }
  /* Commit: the contact force returned to the rigid body, state, history. */
  double F[3] = {0, 0, 0};
  for (int64_t s = 0; s < ns; ++s) {
    M->active[s] = M->act_try[s];
    M->lambda[s] = M->act_try[s] ? M->lam_try[s] : 0.0;
    if (!M->act_try[s]) continue;
    int64_t j = M->surf[s];
    double x[3], r2 = 0.0;
    for (int i = 0; i < 3; ++i) {
      x[i] = M->X[j * 3 + i] + M->dn[j * 3 + i] - cn[i];
      r2 += x[i] * x[i];
    }
    double r = sqrt(r2);
    for (int i = 0; i < 3; ++i) F[i] += M->lam_try[s] * x[i] / r;
  }
  int nonfinite = 0;
  for (int64_t k = 0; k < nn * 3; ++k)
    if (!isfinite(M->an[k]) || !isfinite(M->dn[k])) nonfinite = 1;
  double *t;
  t = M->d; M->d = M->dn; M->dn = t;
  t = M->v; M->v = M->vn; M->vn = t;
  t = M->a; M->a = M->an; M->an = t;
  t = M->hist; M->hist = M->hist_new; M->hist_new = t;
  t = M->rD; M->rD = M->rD_new; M->rD_new = t;
  for (int i = 0; i < 3; ++i) {
    M->F[i] = F[i];
    M->c[i] = cn[i];
    M->w[i] = wn[i];
  }
  M->n_active = n_act;
  M->last_repeats = iter;
  M->n_repeats_total += iter;
  M->step += 1;
  M->time += dt;
  double fc = F[0] * M->axis[0] + F[1] * M->axis[1] + F[2] * M->axis[2];
  if (M->fhist_n < M->fhist_cap) M->fhist[M->fhist_n++] = fc;
  if (fc > M->fpeak) M->fpeak = fc;
  if (nonfinite) {
    M->status = ORC_E_NONFINITE;
    return M->status;
  }
  return ORC_OK;
}

int orc_step(orc_model *M, int64_t nsteps) {
#ifdef _OPENMP
  if (M->opt.n_threads > 0) omp_set_num_threads(M->opt.n_threads);
#endif
  if (M->status) return M->status;
  for (int64_t s = 0; s < nsteps; ++s) {
    int rc = one_step(M);
    if (rc) return rc;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Accessors (SoA [3][nn] for nodal fields).                                */

void orc_get_state(const orc_model *M, double *d, double *v, double *a) {
  for (int64_t j = 0; j < M->nn; ++j)
    for (int i = 0; i < 3; ++i) {
      if (d) d[i * M->nn + j] = M->d[j * 3 + i];
      if (v) v[i * M->nn + j] = M->v[j * 3 + i];
      if (a) a[i * M->nn + j] = M->a[j * 3 + i];
    }
}

/* Install a state: displacement and velocity (SoA); the acceleration is
 * recomputed from the internal forces at d (no contact), as at a restart. */
void orc_set_state(orc_model *M, const double *d, const double *v) {
  for (int64_t j = 0; j < M->nn; ++j)
    for (int i = 0; i < 3; ++i) {
      M->d[j * 3 + i] = ((M->fixed[j] >> i) & 1) ? 0.0 : d[i * M->nn + j];
      M->v[j * 3 + i] = ((M->fixed[j] >> i) & 1) ? 0.0 : v[i * M->nn + j];
    }
  acceleration_of_state(M);
}

/* Install a complete committed state of step `step` taken from another solver
 * of the same model, so that the oracle continues from it: displacement,
 * velocity and acceleration (SoA [3][nn]; the acceleration the next
 * predictor uses), the contact set active[ns], and imp[10] = striker centre
 * c[3], velocity w[3], the contact force F[3] of that step (held over the
 * next step, Algorithm 1) and the time.  Nothing is recomputed.  The force
 * history restarts empty; the history of the integration points is installed
 * separately (orc_set_history). */
void orc_install_state(orc_model *M, const double *d, const double *v, const double *a,
                       const uint8_t *active, const double imp[10], int64_t step) {
  for (int64_t j = 0; j < M->nn; ++j)
    for (int i = 0; i < 3; ++i) {
      int held = (M->fixed[j] >> i) & 1;
      M->d[j * 3 + i] = held ? 0.0 : d[i * M->nn + j];
      M->v[j * 3 + i] = held ? 0.0 : v[i * M->nn + j];
      M->a[j * 3 + i] = held ? 0.0 : a[i * M->nn + j];
    }
  M->n_active = 0;
  for (int64_t s = 0; s < M->ns; ++s) {
    M->active[s] = active[s] ? 1 : 0;
    M->lambda[s] = 0.0;
    M->n_active += M->active[s];
  }
  for (int i = 0; i < 3; ++i) {
    M->c[i] = imp[i];
    M->w[i] = imp[3 + i];
    M->F[i] = imp[6 + i];
  }
  M->time = imp[9];
  M->step = step;
  M->fhist_n = 0;
  M->fpeak = 0.0;
  M->status = ORC_OK;
}

void orc_get_impactor(const orc_model *M, double out[10]) {
  for (int i = 0; i < 3; ++i) {
    out[i] = M->c[i];
    out[3 + i] = M->w[i];
    out[6 + i] = M->F[i];
  }
  out[9] = M->time;
}

void orc_get_info(const orc_model *M, double out[8]) {
  out[0] = M->dt;
  out[1] = M->dt_bulk;
  out[2] = M->dt_coh;
  out[3] = (double)M->step;
  out[4] = (double)M->n_active;
  out[5] = (double)M->n_repeats_total;
  out[6] = M->fpeak;
  out[7] = (double)M->status;
}

void orc_get_mass(const orc_model *M, double *m) { memcpy(m, M->mass, sizeof(double) * M->nn); }

void orc_get_active(const orc_model *M, uint8_t *act, double *lam) {
  memcpy(act, M->active, M->ns);
  if (lam) memcpy(lam, M->lambda, sizeof(double) * M->ns);
}

int64_t orc_get_force_history(const orc_model *M, double *out, int64_t cap) {
  int64_t n = M->fhist_n < cap ? M->fhist_n : cap;
  memcpy(out, M->fhist, sizeof(double) * n);
  return n;
}

void orc_get_history(const orc_model *M, double *hist, double *rD) {
  if (hist) memcpy(hist, M->hist, sizeof(double) * M->nh * 8 * NH);
  if (rD && M->nc) memcpy(rD, M->rD, sizeof(double) * M->nc * 4);
}

void orc_set_history(orc_model *M, const double *hist, const double *rD) {
  if (hist) memcpy(M->hist, hist, sizeof(double) * M->nh * 8 * NH);
  if (rD && M->nc) memcpy(M->rD, rD, sizeof(double) * M->nc * 4);
}

void orc_get_strength_factors(const orc_model *M, double *sf) {
  memcpy(sf, M->sf, sizeof(double) * M->nh * 3);
}

void orc_get_lc(const orc_model *M, double *lc) { memcpy(lc, M->lc, sizeof(double) * M->nh); }

/* Energies: kinetic of the plate (1/2 sum m v.v), kinetic of the striker,
 * strain energy sum over hexes of 1/2 S:E dV at the current state (elastic
 * meaning), interface elastic energy 1/2 tau.Delta w (undamaged meaning). */
void orc_energies(orc_model *M, double out[4]) {
  double ke = 0.0;
  for (int64_t j = 0; j < M->nn; ++j)
    for (int i = 0; i < 3; ++i) ke += 0.5 * M->mass[j] * M->v[j * 3 + i] * M->v[j * 3 + i];
  double kei = 0.5 * M->Mimp * (M->w[0] * M->w[0] + M->w[1] * M->w[1] + M->w[2] * M->w[2]);
  double we = 0.0;
#pragma omp parallel for reduction(+ : we) schedule(static)
  for (int64_t e = 0; e < M->nh; ++e) {
    double Xe[8][3], ue[8][3], fe[8][3];
    double hout[8 * NH];
    gather_X(M, M->hex + e * 8, Xe);
    gather_u(M, M->d, M->hex + e * 8, ue);
    we += orc_hex8_force(&M->mat, M->ply_angle[M->ply_hex[e]], M->lc[e], M->sf + e * 3, Xe, ue,
                         M->hist + e * 8 * NH, hout, fe, M->opt.damage_on, M->opt.plasticity_on);
  }
  double wc = 0.0;
  for (int64_t e = 0; e < M->nc; ++e) {
    double Xe[8][3], ue[8][3], fe[8][3], r1[4];
    gather_X(M, M->coh + e * 8, Xe);
    gather_u(M, M->d, M->coh + e * 8, ue);
    orc_coh8_force(&M->mat, Xe, ue, M->rD + e * 4, r1, fe);
    for (int a = 0; a < 8; ++a)
      for (int i = 0; i < 3; ++i) wc += 0.5 * fe[a][i] * ue[a][i];
  }
  out[0] = ke;
  out[1] = kei;
  out[2] = we;
  out[3] = wc;
}
