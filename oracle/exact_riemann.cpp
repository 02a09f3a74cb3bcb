/* Exact Riemann solver for the 1-D gamma-law Euler equations — TEST
 * INFRASTRUCTURE ONLY (the reference solution the oracle's Sod run is pinned
 * to).  Written from the wave-curve analysis of the Riemann problem: the star
 * pressure is the root of f(p) = f_L(p) + f_R(p) + (u_R - u_L), where f_K is
 * the Rankine-Hugoniot shock curve for p > p_K and the isentropic rarefaction
 * curve for p <= p_K; u* follows from the same functions, and the solution is
 * sampled on the self-similar variable xi = x/t.
 * States are W = (rho, u, p). */
#include <cmath>
#include "oracle.h"

namespace {

struct Side {
  double rho, u, p, c, A, B;
};

Side make_side(const double* W, double g) {
  Side s;
  s.rho = W[0]; s.u = W[1]; s.p = W[2];
  s.c = std::sqrt(g * s.p / s.rho);
  s.A = 2.0 / ((g + 1.0) * s.rho);
  s.B = (g - 1.0) / (g + 1.0) * s.p;
  return s;
}

/* velocity jump across the wave connecting state K to pressure p, and its derivative */
void wave_curve(const Side& s, double p, double g, double* f, double* df) {
  if (p > s.p) { /* shock: Rankine-Hugoniot */
    double q = std::sqrt(s.A / (p + s.B));
    *f = (p - s.p) * q;
    *df = q * (1.0 - 0.5 * (p - s.p) / (p + s.B));
  } else { /* rarefaction: isentropic, Riemann invariant */
    double e = (g - 1.0) / (2.0 * g);
    *f = 2.0 * s.c / (g - 1.0) * (std::pow(p / s.p, e) - 1.0);
    *df = 1.0 / (s.rho * s.c) * std::pow(p / s.p, -(g + 1.0) / (2.0 * g));
  }
}

int solve_star(const Side& L, const Side& R, double g, double* ps, double* us) {
  double du = R.u - L.u;
  if (2.0 / (g - 1.0) * (L.c + R.c) <= du) return ORACLE_EINVAL; /* vacuum generated */
  /* f is increasing in p: bracket the root, then safeguarded Newton */
  auto F = [&](double p, double* d) {
    double fl, dl, fr, dr;
    wave_curve(L, p, g, &fl, &dl);
    wave_curve(R, p, g, &fr, &dr);
    if (d) *d = dl + dr;
    return fl + fr + du;
  };
  double lo = 0.0, hi = std::fmax(L.p, R.p);
  while (F(hi, nullptr) < 0.0) { lo = hi; hi *= 2.0; }
  double p = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    double d, f = F(p, &d);
    if (f == 0.0) break;
    if (f < 0.0) lo = p; else hi = p;
    double pn = p - f / d;
    if (!(pn > lo && pn < hi)) pn = 0.5 * (lo + hi);
    if (std::fabs(pn - p) <= 1e-15 * p) { p = pn; break; }
    p = pn;
  }
  double fl, fr, dd;
  wave_curve(L, p, g, &fl, &dd);
  wave_curve(R, p, g, &fr, &dd);
  *ps = p;
  *us = 0.5 * (L.u + R.u) + 0.5 * (fr - fl);
  return ORACLE_OK;
}

void sample(const Side& L, const Side& R, double g, double ps, double us, double xi, double* W) {
  double g1 = (g - 1.0) / (g + 1.0), g2 = 2.0 / (g + 1.0);
  if (xi <= us) {
    if (ps > L.p) { /* left shock */
      double sL = L.u - L.c * std::sqrt((g + 1.0) / (2.0 * g) * ps / L.p + (g - 1.0) / (2.0 * g));
      if (xi <= sL) { W[0] = L.rho; W[1] = L.u; W[2] = L.p; }
      else { W[0] = L.rho * (ps / L.p + g1) / (g1 * ps / L.p + 1.0); W[1] = us; W[2] = ps; }
    } else { /* left rarefaction */
      double cs = L.c * std::pow(ps / L.p, (g - 1.0) / (2.0 * g));
      double head = L.u - L.c, tail = us - cs;
      if (xi <= head) { W[0] = L.rho; W[1] = L.u; W[2] = L.p; }
      else if (xi >= tail) { W[0] = L.rho * std::pow(ps / L.p, 1.0 / g); W[1] = us; W[2] = ps; }
      else {
        double b = g2 + g1 / L.c * (L.u - xi);
        W[0] = L.rho * std::pow(b, 2.0 / (g - 1.0));
        W[1] = g2 * (L.c + 0.5 * (g - 1.0) * L.u + xi);
        W[2] = L.p * std::pow(b, 2.0 * g / (g - 1.0));
      }
    }
  } else {
    if (ps > R.p) { /* right shock */
      double sR = R.u + R.c * std::sqrt((g + 1.0) / (2.0 * g) * ps / R.p + (g - 1.0) / (2.0 * g));
      if (xi >= sR) { W[0] = R.rho; W[1] = R.u; W[2] = R.p; }
      else { W[0] = R.rho * (ps / R.p + g1) / (g1 * ps / R.p + 1.0); W[1] = us; W[2] = ps; }
    } else { /* right rarefaction */
      double cs = R.c * std::pow(ps / R.p, (g - 1.0) / (2.0 * g));
      double head = R.u + R.c, tail = us + cs;
      if (xi >= head) { W[0] = R.rho; W[1] = R.u; W[2] = R.p; }
      else if (xi <= tail) { W[0] = R.rho * std::pow(ps / R.p, 1.0 / g); W[1] = us; W[2] = ps; }
      else {
        double b = g2 - g1 / R.c * (R.u - xi);
        W[0] = R.rho * std::pow(b, 2.0 / (g - 1.0));
        W[1] = g2 * (-R.c + 0.5 * (g - 1.0) * R.u + xi);
        W[2] = R.p * std::pow(b, 2.0 * g / (g - 1.0));
      }
    }
  }
}

} /* namespace */

extern "C" {

int oracle_exact_star(const double* WL, const double* WR, double gamma, double* out) {
  Side L = make_side(WL, gamma), R = make_side(WR, gamma);
  return solve_star(L, R, gamma, &out[0], &out[1]);
}

int oracle_exact_sample(const double* WL, const double* WR, double gamma, const double* xi, int n, double* W) {
  Side L = make_side(WL, gamma), R = make_side(WR, gamma);
  double ps, us;
  int rc = solve_star(L, R, gamma, &ps, &us);
  if (rc) return rc;
  for (int i = 0; i < n; ++i) sample(L, R, gamma, ps, us, xi[i], W + 3 * i);
  return ORACLE_OK;
}

} /* extern "C" */
