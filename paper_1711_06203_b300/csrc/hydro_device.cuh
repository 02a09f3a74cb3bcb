// Device-side arithmetic of the CTU-PPM step (FP64, sm_103a).
//
// Each function is one stage of the unsplit PPM scheme named in the paper
// (Sec. 3.2): gamma-law EOS conversion, Colella-Woodward flattening and PPM
// reconstruction, reference-state characteristic tracing, HLLC Riemann flux,
// and the conservative transverse correction of CTU.  Operation order is
// fixed (the same order every time a quantity is formed) so that a build with
// contraction disabled reproduces the scheme's FP64 arithmetic exactly.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hydro {

constexpr int NG = 4;  // ghost zones per side: the stencil reaches 4 zones
// primitive fields stored per zone on the grown box
enum { QRHO = 0, QU = 1, QV = 2, QW = 3, QP = 4, QC = 5, QRC = 6, QCR = 7, QIC2 = 8, NQ = 9 };

constexpr double FLAT_OMEGA1 = 0.75, FLAT_OMEGA2 = 10.0, FLAT_EPS = 0.33;
constexpr double SIXTH = 1.0 / 6.0, TWOTHIRDS = 2.0 / 3.0, THIRD = 1.0 / 3.0;

struct StepConst {
  double gamma, gm1, gm1inv;  // gamma, gamma - 1, 1/(gamma - 1)
  double small_dens, small_pres;
  double grav[3];
  double dt, hdt;             // dt, dt/2
  double dtdx[3];             // dt/dx per axis
  int dim, flatten, has_grav;
};

// min/max as explicit selects: ties return the first argument
__device__ __forceinline__ double dmin(double a, double b) { return (b < a) ? b : a; }
__device__ __forceinline__ double dmax(double a, double b) { return (a < b) ? b : a; }
__device__ __forceinline__ bool same_sign_strict(double a, double b) {
  return (a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0);
}

// ---------------------------------------------------------------- EOS
// conserved -> primitive with floors; sets *bad for a non-physical state
__device__ __forceinline__ void cons_to_prim_flag(const double U[5], const StepConst& K, double q[5],
                                                  double* inv_out, bool* bad) {
  double rho = U[0];
  if (!(rho > 0.0 && isfinite(rho))) *bad = true;
  rho = dmax(rho, K.small_dens);
  double inv = 1.0 / rho;
  double u = U[1] * inv, v = U[2] * inv, w = U[3] * inv;
  double ke = 0.5 * rho * ((u * u + v * v) + w * w);
  double p = K.gm1 * (U[4] - ke);
  if (!(p > 0.0 && isfinite(p) && isfinite(U[1]) && isfinite(U[2]) && isfinite(U[3]))) *bad = true;
  p = dmax(p, K.small_pres);
  q[0] = rho; q[1] = u; q[2] = v; q[3] = w; q[4] = p;
  *inv_out = inv;
}

// face state for the Riemann solver: rho, u, v, w, p, rho*E, 1/rho
enum { S_RHO = 0, S_P = 4, S_E = 5, S_INV = 6, NS = 7 };

__device__ __forceinline__ double energy_of(const double q[5], const StepConst& K) {
  return q[4] * K.gm1inv + 0.5 * q[0] * ((q[1] * q[1] + q[2] * q[2]) + q[3] * q[3]);
}

__device__ __forceinline__ void state_from_prim(const double q[5], const StepConst& K, double s[NS]) {
#pragma unroll
  for (int c = 0; c < 5; ++c) s[c] = q[c];
  s[S_E] = energy_of(q, K);
  s[S_INV] = 1.0 / q[0];
}

__device__ __forceinline__ void state_from_cons(const double U[5], const StepConst& K, double s[NS]) {
  double rho = dmax(U[0], K.small_dens);
  double inv = 1.0 / rho;
  double u = U[1] * inv, v = U[2] * inv, w = U[3] * inv;
  double ke = 0.5 * rho * ((u * u + v * v) + w * w);
  double p = K.gm1 * (U[4] - ke);
  p = dmax(p, K.small_pres);
  s[0] = rho; s[1] = u; s[2] = v; s[3] = w; s[4] = p;
  s[S_E] = U[4];
  s[S_INV] = inv;
}

// ---------------------------------------------------------------- flattening (CW84 App. A)
// line arrays hold offsets -3..3 about the zone (index 3)
__device__ __forceinline__ double flat_tilde(const double* p, const double* un, int m, double small_pres) {
  double dp1 = p[m + 1] - p[m - 1];
  double dp2 = p[m + 2] - p[m - 2];
  if (un[m - 1] - un[m + 1] > 0.0 && fabs(dp1) > FLAT_EPS * dmin(p[m + 1], p[m - 1])) {
    double z = fabs(dp1) / dmax(fabs(dp2), small_pres);
    double f = dmax(0.0, dmin(1.0, FLAT_OMEGA2 * (z - FLAT_OMEGA1)));
    return 1.0 - f;
  }
  return 1.0;
}

__device__ __forceinline__ double flat_coef(const double* p, const double* un, double small_pres) {
  double dp1 = p[4] - p[2];
  int s = (dp1 < 0.0) ? 1 : -1;
  return dmin(flat_tilde(p, un, 3, small_pres), flat_tilde(p, un, 3 + s, small_pres));
}

// ---------------------------------------------------------------- PPM (CW84 eqs. 1.6-1.10)
__device__ __forceinline__ double mc_slope(const double* a, int m) {
  double dl = a[m] - a[m - 1], dr = a[m + 1] - a[m];
  if (!same_sign_strict(dl, dr)) return 0.0;
  double da = 0.5 * (a[m + 1] - a[m - 1]);
  double lim = dmin(fabs(da), dmin(2.0 * fabs(dl), 2.0 * fabs(dr)));
  return copysign(lim, da);
}

__device__ __forceinline__ void ppm_parabola(const double* a, double chi, double& am, double& ap, double& a6) {
  double ai = a[3];
  double s2 = mc_slope(a, 2), s3 = mc_slope(a, 3), s4 = mc_slope(a, 4);
  double aP = 0.5 * (a[3] + a[4]) - SIXTH * (s4 - s3);
  double aM = 0.5 * (a[2] + a[3]) - SIXTH * (s3 - s2);
  if (!same_sign_strict(aP - ai, ai - aM)) {
    aP = ai; aM = ai;
  } else {
    double D = aP - aM, M = ai - 0.5 * (aM + aP);
    double up = M - SIXTH * D, dn = M + SIXTH * D;
    if (same_sign_strict(D, up)) aM = 3.0 * ai - 2.0 * aP;
    else if ((D > 0.0 && dn < 0.0) || (D < 0.0 && dn > 0.0)) aP = 3.0 * ai - 2.0 * aM;
  }
  aP = chi * aP + (1.0 - chi) * ai;
  aM = chi * aM + (1.0 - chi) * ai;
  am = aM; ap = aP; a6 = 6.0 * (ai - 0.5 * (aM + aP));
}

// averages of the parabola over the part of the zone swept by a wave of
// Courant number s toward the high (I+) / low (I-) face
__device__ __forceinline__ double integ_plus(double am, double ap, double a6, double s) {
  return ap - 0.5 * s * ((ap - am) - (1.0 - TWOTHIRDS * s) * a6);
}
__device__ __forceinline__ double integ_minus(double am, double ap, double a6, double s) {
  return am + 0.5 * s * ((ap - am) + (1.0 - TWOTHIRDS * s) * a6);
}

// ---------------------------------------------------------------- HLLC (Toro-Spruce-Speares)
__device__ __forceinline__ void hllc_flux(const double sL[NS], const double sR[NS], int d, const StepConst& K,
                                          double F[5]) {
  double rl = sL[S_RHO], pl = sL[S_P], ul = sL[1 + d];
  double rr = sR[S_RHO], pr = sR[S_P], ur = sR[1 + d];
  double cl = sqrt(K.gamma * pl * sL[S_INV]);
  double cr = sqrt(K.gamma * pr * sR[S_INV]);
  double sl = dmin(ul - cl, ur - cr);
  double sr = dmax(ul + cl, ur + cr);
  double ml = rl * (sl - ul), mr = rr * (sr - ur);
  double sstar = ((pr - pl) + ml * ul - mr * ur) / (ml - mr);
  int region = (sl >= 0.0) ? 0 : (sstar >= 0.0) ? 1 : (sr > 0.0) ? 2 : 3;
  bool left = region <= 1;
  const double* s = left ? sL : sR;
  double rho = s[S_RHO], un = s[1 + d], p = s[S_P], E = s[S_E];
  double mass = rho * un;
  double Fk[5];
  Fk[0] = mass;
#pragma unroll
  for (int k = 0; k < 3; ++k) Fk[1 + k] = (k == d) ? mass * un + p : mass * s[1 + k];
  Fk[4] = un * (E + p);
  if (region == 0 || region == 3) {
#pragma unroll
    for (int c = 0; c < 5; ++c) F[c] = Fk[c];
    return;
  }
  double sk = left ? sl : sr, mk = left ? ml : mr;
  double Uk[5] = {rho, rho * s[1], rho * s[2], rho * s[3], E};
  double r = 1.0 / (sk - sstar);
  double f = mk * r;
  double Us[5];
  Us[0] = f;
#pragma unroll
  for (int k = 0; k < 3; ++k) Us[1 + k] = (k == d) ? f * sstar : f * s[1 + k];
  Us[4] = f * (E * s[S_INV]) + (sstar - un) * (f * sstar + p * r);
#pragma unroll
  for (int c = 0; c < 5; ++c) F[c] = Fk[c] + sk * (Us[c] - Uk[c]);
}

}  // namespace hydro
