/* CPU oracle: one unsplit corner-transport-upwind (CTU) PPM Godunov step for
 * the gamma-law Euler equations on a ghost-zoned box.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * FP64 statement of the scheme that the CUDA path is checked against.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * load it; the product library never does, and the two share no code.
 *
 * The paper (Sec. 3.2, "Castro") names the method only: an unsplit piecewise
 * parabolic method for compressible hydrodynamics, with a general equation of
 * state (here gamma-law), conservative source terms (here constant gravity),
 * run box by box on ghost-zoned patches handed to a kernel by an iterator
 * (Sec. 3 intro; Sec. 4, GPU port paragraph).  Every step below is the
 * textbook method it names:
 *   - reconstruction and limiter: Colella & Woodward 1984 (CW84) eqs. 1.6-1.10
 *   - flattening: CW84 appendix A (omega1 = 0.75, omega2 = 10, epsilon = 0.33)
 *   - characteristic tracing: reference-state tracing (Miller & Colella 2002)
 *   - transverse corrections: Colella 1990 (2-D), Saltzman 1994 (3-D, 12 solves)
 *   - Riemann solver: HLLC (Toro, Spruce & Speares 1994), Davis wave speeds
 *   - update: conservative flux difference + time-centred gravity source
 * Where the scheme leaves a choice open, the choice made is stated at the
 * point of use.  Arithmetic is FP64; compiled with -ffp-contract=off so that
 * no multiply-add is fused behind the reader's back.
 *
 * Layout: a box is 5 conserved fields (rho, rho*u, rho*v, rho*w, rho*E),
 * component-major, each a (gz, gy, gx) array with x fastest, over the grown
 * box: interior n[a] zones plus ng = 4 ghost zones on each side of every
 * active axis (z has no ghosts in 2-D, where n[2] = 1).
 *
 * Built twice: the normal build (real = double) and the counting build
 * (-DORACLE_COUNT_FLOPS, real = counted) that tallies the arithmetic.
 */
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#ifdef ORACLE_COUNT_FLOPS
#include "flopcount.h"
typedef counted real;
op_tally g_tally;
/* tallies per stage of the step: prim, trace, flux1, flux2, flux3, update */
static op_tally g_stage_tally[6];
static op_tally g_mark;
static void stage_mark(int stage) {
  if (stage > 0) {
    op_tally& t = g_stage_tally[stage - 1];
    t.add += g_tally.add - g_mark.add; t.mul += g_tally.mul - g_mark.mul; t.div += g_tally.div - g_mark.div;
    t.sqrt += g_tally.sqrt - g_mark.sqrt; t.cmp += g_tally.cmp - g_mark.cmp;
  }
  g_mark = g_tally;
}
#define STAGE_MARK(k) stage_mark(k)
#else
#define STAGE_MARK(k) ((void)0)
typedef double real;
using std::isfinite;
using std::sqrt;
using std::fabs;
using std::copysign;
#endif

#include "oracle.h"

namespace {

const int NG = 4;          /* ghost zones per side: the CTU-PPM stencil reaches 4 zones */
const int NV = 5;          /* conserved / primitive variables */
/* primitive fields on the grown box: rho, u, v, w, p, c and the zone's
 * eigenvector coefficients rho/c, c/rho, 1/c^2 (shared by all directions) */
enum { QRHO = 0, QU = 1, QV = 2, QW = 3, QP = 4, QC = 5, QRC = 6, QCR = 7, QIC2 = 8, NQ = 9 };

/* CW84 appendix A flattening constants */
const double FLAT_OMEGA1 = 0.75, FLAT_OMEGA2 = 10.0, FLAT_EPS = 0.33;
const double SIXTH = 1.0 / 6.0, TWOTHIRDS = 2.0 / 3.0, THIRD = 1.0 / 3.0;

/* min / max written as explicit comparisons (ties return the first argument) */
inline real rmin(real a, real b) { return (b < a) ? b : a; }
inline real rmax(real a, real b) { return (a < b) ? b : a; }

struct Grid {
  int dim, n[3], gx, gy, gz, ngz;
  long sy, sz, sc, str[3];
  Grid(const oracle_params& P) {
    dim = P.dim;
    for (int a = 0; a < 3; ++a) n[a] = P.n[a];
    ngz = (dim == 3) ? NG : 0;
    gx = n[0] + 2 * NG; gy = n[1] + 2 * NG; gz = n[2] + 2 * ngz;
    sy = gx; sz = (long)gx * gy; sc = sz * gz;
    str[0] = 1; str[1] = sy; str[2] = sz;
  }
  long id(int i, int j, int k) const { return (long)(k + ngz) * sz + (long)(j + NG) * sy + (i + NG); }
};

/* ---- Step 1: ghost-zone fill (outflow / reflect / periodic / prefilled) ---- */
void fill_ghosts(real* W, const Grid& g, const oracle_params& P, int nf = NV) {
  for (int a = 0; a < g.dim; ++a) {
    /* fill axis a over the full grown range of earlier axes (already
     * filled) and, on later axes, over the interior plus any prefilled ghost
     * layers (caller data): edges and corners are then the product of the
     * per-axis maps, a prefilled face mapping each zone to itself */
    int lo[3], hi[3];
    for (int b = 0; b < 3; ++b) {
      int gb = (b == 2) ? g.ngz : NG;
      if (b < a) { lo[b] = -gb; hi[b] = g.n[b] + gb; }
      else {
        lo[b] = (b < g.dim && P.bc[b][0] == ORACLE_BC_PREFILLED) ? -gb : 0;
        hi[b] = (b < g.dim && P.bc[b][1] == ORACLE_BC_PREFILLED) ? g.n[b] + gb : g.n[b];
      }
    }
    for (int side = 0; side < 2; ++side) {
      int bc = P.bc[a][side];
      if (bc == ORACLE_BC_PREFILLED) continue;
      for (int m = 1; m <= NG; ++m) {
        int dst = side == 0 ? -m : g.n[a] - 1 + m, src;
        if (bc == ORACLE_BC_OUTFLOW) src = side == 0 ? 0 : g.n[a] - 1;
        else if (bc == ORACLE_BC_REFLECT) src = side == 0 ? m - 1 : g.n[a] - m;
        else src = side == 0 ? g.n[a] - m : m - 1; /* periodic */
        int l0[3] = {lo[0], lo[1], lo[2]}, h0[3] = {hi[0], hi[1], hi[2]};
        l0[a] = dst; h0[a] = dst + 1;
        for (int k = l0[2]; k < h0[2]; ++k)
          for (int j = l0[1]; j < h0[1]; ++j)
            for (int i = l0[0]; i < h0[0]; ++i) {
              int s[3] = {i, j, k};
              s[a] = src;
              long di = g.id(i, j, k), si = g.id(s[0], s[1], s[2]);
              for (int c = 0; c < nf; ++c) {
                real v = W[c * g.sc + si];
                if (bc == ORACLE_BC_REFLECT && c == 1 + a) v = -v; /* mirror the normal momentum */
                W[c * g.sc + di] = v;
              }
            }
      }
    }
  }
}

/* ---- Step 2: conserved -> primitive with density / pressure floors (gamma-law EOS) ----
 * q = (rho, u, v, w, p); flags a non-physical input (rho <= 0, p <= 0, non-finite). */
void cons_to_prim(const real U[5], const oracle_params& P, real q[5], real* inv_out, int* bad) {
  real rho = U[0];
  if (bad && !(rho > 0.0 && isfinite(rho))) *bad = 1;
  rho = rmax(rho, real(P.small_dens));
  real inv = 1.0 / rho;
  real u = U[1] * inv, v = U[2] * inv, w = U[3] * inv;
  real ke = 0.5 * rho * ((u * u + v * v) + w * w);
  real p = (P.gamma - 1.0) * (U[4] - ke);
  if (bad && !(p > 0.0 && isfinite(p) && isfinite(U[1]) && isfinite(U[2]) && isfinite(U[3]))) *bad = 1;
  p = rmax(p, real(P.small_pres));
  q[0] = rho; q[1] = u; q[2] = v; q[3] = w; q[4] = p;
  if (inv_out) *inv_out = inv;
}

/* sound speed c = sqrt(gamma p / rho), given inv = 1/rho */
real sound_speed(real p, real inv, double gamma) { return sqrt(gamma * p * inv); }

/* per-step constants */
struct Consts {
  double gamma;
  real gm1inv; /* 1/(gamma - 1) */
};

/* primitive -> conserved, rho*E = p/(gamma-1) + rho |u|^2 / 2 */
void prim_to_cons(const real q[5], const Consts& K, real U[5]) {
  U[0] = q[0];
  U[1] = q[0] * q[1]; U[2] = q[0] * q[2]; U[3] = q[0] * q[3];
  U[4] = q[4] * K.gm1inv + 0.5 * q[0] * ((q[1] * q[1] + q[2] * q[2]) + q[3] * q[3]);
}

/* A face state as the Riemann solver consumes it: primitive variables, the
 * total energy density rho*E and 1/rho. */
enum { S_RHO = 0, S_P = 4, S_E = 5, S_INV = 6, NS = 7 };

/* from a traced primitive state */
void state_from_prim(const real q[5], const Consts& K, real s[NS]) {
  for (int c = 0; c < 5; ++c) s[c] = q[c];
  s[S_E] = q[4] * K.gm1inv + 0.5 * q[0] * ((q[1] * q[1] + q[2] * q[2]) + q[3] * q[3]);
  s[S_INV] = 1.0 / q[0];
}

/* from a transversely corrected conserved state, with floors */
void state_from_cons(const real U[5], const oracle_params& P, real s[NS]) {
  real rho = rmax(U[0], real(P.small_dens));
  real inv = 1.0 / rho;
  real u = U[1] * inv, v = U[2] * inv, w = U[3] * inv;
  real ke = 0.5 * rho * ((u * u + v * v) + w * w);
  real p = (P.gamma - 1.0) * (U[4] - ke);
  p = rmax(p, real(P.small_pres));
  s[0] = rho; s[1] = u; s[2] = v; s[3] = w; s[4] = p;
  s[S_E] = U[4];
  s[S_INV] = inv;
}

/* ---- Step 4: CW84 flattening along one line ----
 * a line holds 7 values at offsets -3..3 about the zone (index 3): flattening
 * reaches 3 zones, the reconstruction 2.
 * chi is the fraction of the reconstruction that is KEPT (1 = unflattened). */
real flat_tilde(const real* p, const real* un, int m, double small_pres) {
  real dp1 = p[m + 1] - p[m - 1];
  real dp2 = p[m + 2] - p[m - 2];
  /* shock detector: compression and a pressure jump larger than epsilon */
  if (un[m - 1] - un[m + 1] > 0.0 && fabs(dp1) > FLAT_EPS * rmin(p[m + 1], p[m - 1])) {
    real z = fabs(dp1) / rmax(fabs(dp2), real(small_pres));
    real f = rmax(real(0.0), rmin(real(1.0), FLAT_OMEGA2 * (z - FLAT_OMEGA1)));
    return 1.0 - f;
  }
  return 1.0;
}
real flat_coef(const real* p, const real* un, double small_pres) {
  real dp1 = p[4] - p[2];
  int s = (dp1 < 0.0) ? 1 : -1; /* the neighbour on the low-pressure side, into which a shock runs */
  return rmin(flat_tilde(p, un, 3, small_pres), flat_tilde(p, un, 3 + s, small_pres));
}

/* ---- Step 5: PPM reconstruction (CW84 eqs. 1.6-1.10) ---- */
/* monotonised centred slope delta_m a (CW84 eq. 1.8): zero unless a is
 * strictly monotone through the zone */
real mc_slope(const real* a, int m) {
  real dl = a[m] - a[m - 1], dr = a[m + 1] - a[m];
  bool mono = (dl > 0.0 && dr > 0.0) || (dl < 0.0 && dr < 0.0);
  if (!mono) return 0.0;
  real da = 0.5 * (a[m + 1] - a[m - 1]);
  real lim = rmin(fabs(da), rmin(2.0 * fabs(dl), 2.0 * fabs(dr)));
  return copysign(lim, da);
}
/* interface value a_{m+1/2} between zones m and m+1 from their averages and
 * monotonised slopes (CW84 eq. 1.6 on a uniform grid) */
real face_value(real a0, real a1, real s0, real s1) { return 0.5 * (a0 + a1) - SIXTH * (s1 - s0); }
/* limited, flattened parabola of a zone with average ai and interface values
 * aM (low) and aP (high): edge values am, ap and a6 */
void ppm_limit(real ai, real aM, real aP, real chi, real* am, real* ap, real* a6) {
  /* CW84 eq. 1.10: local extremum -> constant; overshooting parabola -> steepen
   * the opposite edge.  The two tests (a+-a)(a-a-) <= 0 and D*M > D^2/6 are
   * written as sign tests, which are their exact-arithmetic meaning. */
  bool same = ((aP - ai) > 0.0 && (ai - aM) > 0.0) || ((aP - ai) < 0.0 && (ai - aM) < 0.0);
  if (!same) {
    aP = ai; aM = ai;
  } else {
    real D = aP - aM, M = ai - 0.5 * (aM + aP);
    real up = M - SIXTH * D; /* D*M > D^2/6   <=>  D*(M - D/6) > 0 */
    real dn = M + SIXTH * D; /* -D^2/6 > D*M  <=>  D*(M + D/6) < 0 */
    if ((D > 0.0 && up > 0.0) || (D < 0.0 && up < 0.0)) aM = 3.0 * ai - 2.0 * aP;
    else if ((D > 0.0 && dn < 0.0) || (D < 0.0 && dn > 0.0)) aP = 3.0 * ai - 2.0 * aM;
  }
  /* flattening blends the edges toward the zone average where chi < 1 */
  if (chi < 1.0) {
    aP = chi * aP + (1.0 - chi) * ai;
    aM = chi * aM + (1.0 - chi) * ai;
  }
  *am = aM; *ap = aP; *a6 = 6.0 * (ai - 0.5 * (aM + aP));
}
/* the same for the zone at index 3 of a 7-point line (unit pins) */
void ppm_parabola(const real* a, real chi, real* am, real* ap, real* a6) {
  real s2 = mc_slope(a, 2), s3 = mc_slope(a, 3), s4 = mc_slope(a, 4);
  ppm_limit(a[3], face_value(a[2], a[3], s2, s3), face_value(a[3], a[4], s3, s4), chi, am, ap, a6);
}
/* averages of the parabola over the domains swept by a wave of Courant number
 * sigma toward the high (I+) and low (I-) face (CW84 eqs. 1.12) */
real integ_plus(real am, real ap, real a6, real s) {
  return ap - 0.5 * s * ((ap - am) - (1.0 - TWOTHIRDS * s) * a6);
}
real integ_minus(real am, real ap, real a6, real s) {
  return am + 0.5 * s * ((ap - am) + (1.0 - TWOTHIRDS * s) * a6);
}

/* ---- Step 6 for one zone and direction d: characteristic tracing ----
 * am, ap, a6: the zone's limited parabolas of (rho, un, ut1, ut2, p);
 * zone: its averages of the same five variables; Q, id: its sound speed and
 * eigenvector coefficients.  Outputs the primitive states at the zone's low
 * face (qm) and high face (qp) at t^{n+1/2}, components in absolute order
 * (rho, u, v, w, p). */
void trace_from_parabola(const real am[5], const real ap[5], const real a6[5], const real zone[5],
                         const std::vector<real>* Q, long id, int d, const oracle_params& P, real dtdx, real dt,
                         real qm[5], real qp[5]) {
  const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
  real un = zone[1], c = Q[QC][id];
  /* eigenvectors of the primitive (rho, un, p) system at the zone state:
   *   r- = (1, -c/rho, c^2), r0 = (1, 0, 0), r+ = (1, c/rho, c^2)
   *   l- = (0, -rho/(2c), 1/(2c^2)), l0 = (1, 0, -1/c^2), l+ = (0, rho/(2c), 1/(2c^2)) */
  real rho_c = Q[QRC][id], c_rho = Q[QCR][id], inv_c2 = Q[QIC2][id], c2 = c * c;
  real lu = 0.5 * rho_c, lp = 0.5 * inv_c2;
  real lam[3] = {un - c, un, un + c};
  real sig[3];
  for (int w = 0; w < 3; ++w) sig[w] = fabs(lam[w]) * dtdx;

  for (int side = 0; side < 2; ++side) {
    /* side 1: high face, waves moving right (lam > 0) reach it, averages I+;
     * side 0: low face, waves moving left (lam < 0), averages I- */
    bool reach[3];
    for (int w = 0; w < 3; ++w) reach[w] = side ? (lam[w] > 0.0) : (lam[w] < 0.0);
    int fast = side ? 2 : 0; /* fastest wave toward that face gives the reference state */
    /* I(w, v): average of variable v's parabola over the domain swept by wave w */
    auto I = [&](int w, int v) {
      return side ? integ_plus(am[v], ap[v], a6[v], sig[w]) : integ_minus(am[v], ap[v], a6[v], sig[w]);
    };
    real ref[5];
    for (int v = 0; v < 5; ++v) ref[v] = reach[fast] ? I(fast, v) : zone[v];
    /* wave strengths beta = l . (ref - I(sigma_nu)) of the waves that reach the face */
    real bm = 0.0, b0 = 0.0, bp = 0.0, bt1 = 0.0, bt2 = 0.0;
    if (reach[0]) bm = -lu * (ref[1] - I(0, 1)) + lp * (ref[4] - I(0, 4));
    if (reach[1]) {
      b0 = (ref[0] - I(1, 0)) - inv_c2 * (ref[4] - I(1, 4));
      bt1 = ref[2] - I(1, 2);
      bt2 = ref[3] - I(1, 3);
    }
    if (reach[2]) bp = lu * (ref[1] - I(2, 1)) + lp * (ref[4] - I(2, 4));
    /* edge state = ref - sum beta_nu r_nu */
    real s_rho = ref[0] - ((bm + b0) + bp);
    real s_un = ref[1] - (bm * (-c_rho) + bp * c_rho);
    real s_p = ref[4] - (bm * c2 + bp * c2);
    real s_t1 = ref[2] - bt1, s_t2 = ref[3] - bt2;
    /* half-step gravity on every velocity component (none without gravity), then floors */
    if (P.grav[0] != 0.0 || P.grav[1] != 0.0 || P.grav[2] != 0.0) {
      real hdt = 0.5 * dt;
      s_un = s_un + hdt * P.grav[d];
      s_t1 = s_t1 + hdt * P.grav[t1];
      s_t2 = s_t2 + hdt * P.grav[t2];
    }
    s_rho = rmax(s_rho, real(P.small_dens));
    s_p = rmax(s_p, real(P.small_pres));
    real* out = side ? qp : qm;
    out[0] = s_rho; out[1 + d] = s_un; out[1 + t1] = s_t1; out[1 + t2] = s_t2; out[4] = s_p;
  }
}

struct Fields {
  /* 5-component arrays on the grown box */
  std::vector<real> a;
  long sc;
  void init(long sc_) { sc = sc_; a.assign(5 * sc_, real(0.0)); }
  void get(long id, real v[5]) const { for (int c = 0; c < 5; ++c) v[c] = a[c * sc + id]; }
  void put(long id, const real v[5]) { for (int c = 0; c < 5; ++c) a[c * sc + id] = v[c]; }
};

/* ---- Steps 4-6 along one pencil in direction d ----
 * The pencil holds zones -4 .. n_d+3 at (transverse) position `base`; every
 * flattening coefficient, slope and interface value is formed once, then
 * each zone in [-1, n_d] gets its parabolas and traced face states. */
void trace_pencil(const std::vector<real>* Q, long base, long st, int nd, int d, const oracle_params& P,
                  real dtdx, real dt, Fields& TM, Fields& TP) {
  const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
  const int vmap[5] = {QRHO, QU + d, QU + t1, QU + t2, QP}; /* rho, un, ut1, ut2, p */
  const int len = nd + 2 * NG, off = NG;                   /* index of zone j is j + off */
  std::vector<real> a[5], slope[5], face[5];
  for (int v = 0; v < 5; ++v) {
    a[v].resize(len);
    for (int m = 0; m < len; ++m) a[v][m] = Q[vmap[v]][base + (long)(m - off) * st];
  }
  /* CW84 flattening: chi~ on zones [-2, n+1], chi on zones [-1, n] */
  std::vector<real> chit(len, real(1.0)), chi(len, real(1.0));
  if (P.flatten) {
    for (int j = -2; j <= nd + 1; ++j) chit[j + off] = flat_tilde(a[4].data(), a[1].data(), j + off, P.small_pres);
    for (int j = -1; j <= nd; ++j) {
      int m = j + off;
      real dp1 = a[4][m + 1] - a[4][m - 1];
      int s = (dp1 < 0.0) ? 1 : -1; /* the neighbour on the low-pressure side, into which a shock runs */
      chi[m] = rmin(chit[m], chit[m + s]);
    }
  }
  /* slopes on zones [-2, n+1]; interface j+1/2 for j in [-2, n] stored at j */
  for (int v = 0; v < 5; ++v) {
    slope[v].assign(len, real(0.0));
    face[v].assign(len, real(0.0));
    for (int j = -2; j <= nd + 1; ++j) slope[v][j + off] = mc_slope(a[v].data(), j + off);
    for (int j = -2; j <= nd; ++j) {
      int m = j + off;
      face[v][m] = face_value(a[v][m], a[v][m + 1], slope[v][m], slope[v][m + 1]);
    }
  }
  for (int j = -1; j <= nd; ++j) {
    int m = j + off;
    real am[5], ap[5], a6[5], zone[5], qm[5], qp[5];
    for (int v = 0; v < 5; ++v) {
      zone[v] = a[v][m];
      ppm_limit(a[v][m], face[v][m - 1], face[v][m], chi[m], &am[v], &ap[v], &a6[v]);
    }
    long id = base + (long)j * st;
    trace_from_parabola(am, ap, a6, zone, Q, id, d, P, dtdx, dt, qm, qp);
    TM.put(id, qm);
    TP.put(id, qp);
  }
}

/* outer wave-speed estimates of the HLLC fan.
 * Davis: S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R).
 * Einfeldt: S_L = min(u_L - c_L, u~ - c~), S_R = max(u_R + c_R, u~ + c~) with
 * the Roe averages u~ = (sqrt(rho_L) u_L + sqrt(rho_R) u_R)/(sqrt(rho_L) + sqrt(rho_R)),
 * H~ likewise from the specific enthalpies H = (rho E + p)/rho, and
 * c~^2 = (gamma - 1)(H~ - |u~|^2/2). */
void wave_speeds(const real sL[NS], const real sR[NS], int d, double gamma, int einfeldt, real cl, real cr,
                 real* sl, real* sr) {
  real ul = sL[1 + d], ur = sR[1 + d];
  if (!einfeldt) {
    *sl = rmin(ul - cl, ur - cr);
    *sr = rmax(ul + cl, ur + cr);
    return;
  }
  real ql = sqrt(sL[S_RHO]), qr = sqrt(sR[S_RHO]);
  real iw = 1.0 / (ql + qr);
  real wl = ql * iw, wr = qr * iw;
  real ut[3];
  for (int k = 0; k < 3; ++k) ut[k] = wl * sL[1 + k] + wr * sR[1 + k];
  real hl = (sL[S_E] + sL[S_P]) * sL[S_INV], hr = (sR[S_E] + sR[S_P]) * sR[S_INV];
  real ht = wl * hl + wr * hr;
  real q2 = (ut[0] * ut[0] + ut[1] * ut[1]) + ut[2] * ut[2];
  real ct = sqrt((gamma - 1.0) * (ht - 0.5 * q2));
  *sl = rmin(ul - cl, ut[d] - ct);
  *sr = rmax(ur + cr, ut[d] + ct);
}

/* ---- Step 7: HLLC flux in direction d (Toro, Spruce & Speares 1994) ----
 * sL, sR: face states (rho, u, v, w, p, rho*E, 1/rho) left and right of the face. */
void hllc(const real sL[NS], const real sR[NS], int d, double gamma, int einfeldt, real F[5],
          int* upwind_left = nullptr) {
  real rl = sL[S_RHO], pl = sL[S_P], ul = sL[1 + d];
  real rr = sR[S_RHO], pr = sR[S_P], ur = sR[1 + d];
  real cl = sound_speed(pl, sL[S_INV], gamma), cr = sound_speed(pr, sR[S_INV], gamma);
  real sl, sr;
  wave_speeds(sL, sR, d, gamma, einfeldt, cl, cr, &sl, &sr);
  real ml = rl * (sl - ul), mr = rr * (sr - ur); /* mass fluxes through the outer waves */
  real sstar = ((pr - pl) + ml * ul - mr * ur) / (ml - mr);
  /* select the region containing x/t = 0, tested in this order:
   * 0 <= sL -> L;  0 <= S* -> L*;  0 < sR -> R*;  else R */
  int region = (sl >= 0.0) ? 0 : (sstar >= 0.0) ? 1 : (sr > 0.0) ? 2 : 3;
  bool left = region <= 1;
  if (upwind_left) *upwind_left = left ? 1 : 0;
  const real* s = left ? sL : sR;
  real rho = s[S_RHO], un = s[1 + d], p = s[S_P], E = s[S_E];
  if (region == 0 || region == 3) {
    /* physical flux of the chosen side */
    real mass = rho * un;
    F[0] = mass;
    for (int k = 0; k < 3; ++k) F[1 + k] = (k == d) ? mass * un + p : mass * s[1 + k];
    F[4] = un * (E + p);
    return;
  }
  real sk = left ? sl : sr, mk = left ? ml : mr;
  /* star state U*_K = f [1, S*, u_t, E/rho + (S* - u)(S* + p/(rho (S_K - u)))],
   * f = rho (S_K - u)/(S_K - S*).  With r = 1/(S_K - S*), f p/(rho(S_K-u)) = p r,
   * so the energy entry is f E/rho + (S* - u)(f S* + p r): one division fewer.
   * The star flux F_K + S_K (U*_K - U_K) (the Rankine-Hugoniot condition across
   * the S_K wave) is the physical flux of the star state with the star
   * pressure p* = p + rho (S_K - u)(S* - u): mass f S*, normal momentum
   * f S*^2 + p*, transverse momentum (f S*) u_t, energy S* (E* + p*). */
  real r = 1.0 / (sk - sstar);
  real f = mk * r;
  real du = sstar - un;
  real mstar = f * sstar;
  real pstar = p + mk * du;
  real Estar = f * (E * s[S_INV]) + du * (mstar + p * r);
  F[0] = mstar;
  for (int k = 0; k < 3; ++k) F[1 + k] = (k == d) ? mstar * sstar + pstar : mstar * s[1 + k];
  F[4] = sstar * (Estar + pstar);
}

/* ---- Step 8 helper: transverse correction of a traced primitive state ----
 * U(q) - coef_a (Fa_hi - Fa_lo) [- coef_b (Fb_hi - Fb_lo)], back to primitive with floors. */
void correct_state(const real q[5], const oracle_params& P, const Consts& K, real ca, const real* Fa_hi,
                   const real* Fa_lo, real cb, const real* Fb_hi, const real* Fb_lo, real out[NS]) {
  real U[5];
  prim_to_cons(q, K, U);
  for (int c = 0; c < 5; ++c) {
    U[c] = U[c] - ca * (Fa_hi[c] - Fa_lo[c]);
    if (Fb_hi) U[c] = U[c] - cb * (Fb_hi[c] - Fb_lo[c]);
  }
  state_from_cons(U, P, out);
}



/* ==== Method-of-lines step with passive species ====
 * Sec. 4: StarLord, a proxy of Castro with only the hydrodynamics and the
 * EOS, writes the hydrodynamics as a simple method of lines and advects 13
 * nuclear species.  The paper prints no scheme; this is the method-of-lines
 * reading of the same building blocks:
 *   dU/dt = L(U) = -sum_d (F_d(face hi) - F_d(face lo)) / dx_d + S(U)
 *   - F_d: HLLC fluxes of the limited, flattened PPM edge values of the
 *     primitive variables (rho, u, v, w, p, X_k) at the stage time; no
 *     characteristic tracing and no transverse terms;
 *   - species: the mass fraction X_k = (rho X_k)/rho is reconstructed like
 *     the other primitive variables and carried by the mass flux of the HLLC
 *     upwind side: F(rho X_k) = F(rho) X_k(side), side = left when S* >= 0
 *     (the region test of the hydro flux);
 *   - S(U) = (0, rho g, (rho u).g) on the stage state (skipped when g = 0);
 *   - time: the two-stage strong-stability-preserving Runge-Kutta scheme
 *     U1 = U^n + dt L(U^n);  U^{n+1} = 1/2 U^n + 1/2 (U1 + dt L(U1)).
 * Prefilled ghost layers are caller data at t^n and serve both stages;
 * derived faces are refilled from each stage's state. */

/* One stage on the interior: V = W - sum_d dtdx_d (F_d,hi - F_d,lo) + dt S(W).
 * W: the stage state on the grown box with ghosts filled, nf = 5 + nspec fields. */
void mol_stage(const std::vector<real>& W, const Grid& g, const oracle_params& P, int nspec, real dt,
               std::vector<real>& V, int* bad_out) {
  const int nf = NV + nspec, dim = g.dim;
  const long N = g.sc;
  Consts K;
  K.gamma = P.gamma;
  K.gm1inv = 1.0 / (P.gamma - 1.0);
  int bad = 0;
  /* primitive variables (rho, u, v, w, p, X_1 .. X_nspec) on the grown box */
  std::vector<std::vector<real>> q(nf, std::vector<real>(N));
#ifndef ORACLE_COUNT_FLOPS
#pragma omp parallel for reduction(| : bad)
#endif
  for (long id = 0; id < N; ++id) {
    real u[5], q5[5], inv;
    for (int c = 0; c < 5; ++c) u[c] = W[c * N + id];
    int zb = 0;
    cons_to_prim(u, P, q5, &inv, &zb);
    bad |= zb;
    for (int v = 0; v < 5; ++v) q[v][id] = q5[v];
    for (int k = 0; k < nspec; ++k) q[NV + k][id] = W[(NV + k) * N + id] * inv;
  }
  real dtdx[3];
  for (int a = 0; a < 3; ++a) dtdx[a] = (a < dim) ? dt / P.dx[a] : 0.0;
  /* fluxes through every d-face [0, n_d] at interior transverse positions
   * (face f, between zones f-1 and f, stored at zone f) */
  std::vector<std::vector<real>> F[3];
  for (int d = 0; d < dim; ++d) {
    F[d].assign(nf, std::vector<real>(N, real(0.0)));
    const int ta = (d == 0) ? 1 : 0, tb = (d == 2) ? 1 : 2;
    const int nb = (tb < dim) ? g.n[tb] : 1;
    const int nd = g.n[d], len = nd + 2 * NG, off = NG;
#ifndef ORACLE_COUNT_FLOPS
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
#endif
    for (int pb = 0; pb < nb; ++pb)
      for (int pa = 0; pa < g.n[ta]; ++pa) {
        int c0[3] = {0, 0, 0};
        c0[ta] = pa;
        c0[tb] = (tb < dim) ? pb : 0;
        const long base = g.id(c0[0], c0[1], c0[2]), st = g.str[d];
        /* the pencil's lines, zones -4 .. n_d+3 */
        std::vector<std::vector<real>> a(nf, std::vector<real>(len));
        for (int v = 0; v < nf; ++v)
          for (int m = 0; m < len; ++m) a[v][m] = q[v][base + (long)(m - off) * st];
        /* CW84 flattening with the normal velocity u_d: chi on zones [-1, n_d] */
        std::vector<real> chit(len, real(1.0)), chi(len, real(1.0));
        if (P.flatten) {
          for (int j = -2; j <= nd + 1; ++j) chit[j + off] = flat_tilde(a[4].data(), a[1 + d].data(), j + off, P.small_pres);
          for (int j = -1; j <= nd; ++j) {
            int m = j + off;
            real dp1 = a[4][m + 1] - a[4][m - 1];
            int s = (dp1 < 0.0) ? 1 : -1;
            chi[m] = rmin(chit[m], chit[m + s]);
          }
        }
        /* limited edge values of zones [-1, n_d]: am (low face), ap (high face) */
        std::vector<std::vector<real>> am(nf, std::vector<real>(len)), ap(nf, std::vector<real>(len));
        for (int v = 0; v < nf; ++v) {
          std::vector<real> slope(len, real(0.0)), face(len, real(0.0));
          for (int j = -2; j <= nd + 1; ++j) slope[j + off] = mc_slope(a[v].data(), j + off);
          for (int j = -2; j <= nd; ++j) {
            int m = j + off;
            face[m] = face_value(a[v][m], a[v][m + 1], slope[m], slope[m + 1]);
          }
          for (int j = -1; j <= nd; ++j) {
            int m = j + off;
            real a6;
            ppm_limit(a[v][m], face[m - 1], face[m], chi[m], &am[v][m], &ap[v][m], &a6);
          }
        }
        /* Riemann problems at faces [0, n_d] */
        for (int f = 0; f <= nd; ++f) {
          int m = f + off;
          real qL[5], qR[5], sL[NS], sR[NS], Fh[5];
          for (int v = 0; v < 5; ++v) {
            qL[v] = ap[v][m - 1];
            qR[v] = am[v][m];
          }
          state_from_prim(qL, K, sL);
          state_from_prim(qR, K, sR);
          int left = 1;
          hllc(sL, sR, d, P.gamma, P.wave_speeds, Fh, &left);
          long id = base + (long)f * st;
          for (int c = 0; c < 5; ++c) F[d][c][id] = Fh[c];
          for (int k = 0; k < nspec; ++k) F[d][NV + k][id] = Fh[0] * (left ? ap[NV + k][m - 1] : am[NV + k][m]);
        }
      }
  }
  /* the stage update, x then y then z flux differences, then the source */
  const bool grav = P.grav[0] != 0.0 || P.grav[1] != 0.0 || P.grav[2] != 0.0;
#ifndef ORACLE_COUNT_FLOPS
#pragma omp parallel for collapse(2)
#endif
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        long id = g.id(i, j, k);
        for (int c = 0; c < nf; ++c) {
          real v = W[c * N + id];
          for (int d = 0; d < dim; ++d) v = v - dtdx[d] * (F[d][c][id + g.str[d]] - F[d][c][id]);
          V[c * N + id] = v;
        }
        if (grav) {
          real rho = W[id];
          for (int a = 0; a < 3; ++a) V[(1 + a) * N + id] = V[(1 + a) * N + id] + dt * rho * P.grav[a];
          real e = (W[1 * N + id] * P.grav[0] + W[2 * N + id] * P.grav[1]) + W[3 * N + id] * P.grav[2];
          V[4 * N + id] = V[4 * N + id] + dt * e;
        }
      }
  *bad_out |= bad;
}

bool valid_params(const oracle_params* P) {
  if (!P || (P->dim != 2 && P->dim != 3)) return false;
  for (int a = 0; a < 3; ++a) if (P->n[a] < 1) return false;
  if (P->dim == 2 && P->n[2] != 1) return false;
  for (int a = 0; a < P->dim; ++a) {
    if (!(P->dx[a] > 0.0)) return false;
    for (int s = 0; s < 2; ++s) if (P->bc[a][s] < 0 || P->bc[a][s] > 3) return false;
    if ((P->bc[a][0] == ORACLE_BC_PERIODIC) != (P->bc[a][1] == ORACLE_BC_PERIODIC)) return false;
    if (P->bc[a][0] != ORACLE_BC_PREFILLED && P->n[a] < NG) return false; /* a ghost layer is a copy of interior zones */
  }
  return P->gamma > 1.0;
}

} /* namespace */

extern "C" {

long long oracle_grown_size(const oracle_params* P) {
  if (!valid_params(P)) return -1;
  Grid g(*P);
  return g.sc;
}

int oracle_fill_ghosts(double* U, const oracle_params* P) {
  if (!valid_params(P)) return ORACLE_EINVAL;
  Grid g(*P);
  std::vector<real> W(U, U + 5 * g.sc);
  fill_ghosts(W.data(), g, *P);
  for (long i = 0; i < 5 * g.sc; ++i) U[i] = double(W[i]);
  return ORACLE_OK;
}

/* CFL time step from the interior of U: cfl * min over zones and active
 * directions of dx_d / (|u_d| + c).  (Sec. 3.1 notes that a compressible code's
 * step is limited by the sound speed.) */
int oracle_dt(const double* U, const oracle_params* P, double* dt_out) {
  if (!valid_params(P) || !dt_out) return ORACLE_EINVAL;
  Grid g(*P);
  int bad = 0;
  std::vector<double> kmin(g.n[2], HUGE_VAL);
#ifndef ORACLE_COUNT_FLOPS
#pragma omp parallel for reduction(| : bad)
#endif
  for (int k = 0; k < g.n[2]; ++k) {
    int kbad = 0;
    real m = HUGE_VAL;
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        long id = g.id(i, j, k);
        real u[5], q[5];
        for (int c = 0; c < 5; ++c) u[c] = U[c * g.sc + id];
        real inv;
        cons_to_prim(u, *P, q, &inv, &kbad);
        real c = sound_speed(q[4], inv, P->gamma);
        for (int d = 0; d < g.dim; ++d) m = rmin(m, P->dx[d] / (fabs(q[1 + d]) + c));
      }
    kmin[k] = double(m);
    bad |= kbad;
  }
  double m = HUGE_VAL;
  for (int k = 0; k < g.n[2]; ++k) m = kmin[k] < m ? kmin[k] : m;
  *dt_out = P->cfl * m;
  return bad ? ORACLE_EBADSTATE : ORACLE_OK;
}

int oracle_step(const double* Uin, double* Uout, const oracle_params* P, double dt, oracle_debug* dbg) {
  if (!valid_params(P) || !Uin || !Uout || !(dt > 0.0)) return ORACLE_EINVAL;
  const Grid g(*P);
  const int dim = g.dim;
  const long N = g.sc;
  int bad = 0;
  Consts K;
  K.gamma = P->gamma;
  K.gm1inv = 1.0 / (P->gamma - 1.0);

  /* Step 1: working copy with ghost zones filled */
  std::vector<real> W(Uin, Uin + 5 * N);
  fill_ghosts(W.data(), g, *P);

  STAGE_MARK(0);
  /* Step 2: primitive variables and sound speed on the whole grown box */
  std::vector<real> Q[NQ];
  for (int v = 0; v < NQ; ++v) Q[v].assign(N, real(0.0));
#ifndef ORACLE_COUNT_FLOPS
#pragma omp parallel for reduction(| : bad)
#endif
  for (long id = 0; id < N; ++id) {
    real u[5], q[5];
    for (int c = 0; c < 5; ++c) u[c] = W[c * N + id];
    int zb = 0;
    real inv;
    cons_to_prim(u, *P, q, &inv, &zb);
    bad |= zb;
    for (int v = 0; v < 5; ++v) Q[v][id] = q[v];
    real c = sound_speed(q[4], inv, P->gamma);
    Q[QC][id] = c;
    Q[QRC][id] = q[0] / c;
    Q[QCR][id] = c / q[0];
    Q[QIC2][id] = 1.0 / (c * c);
  }

  real dtdx[3];
  for (int a = 0; a < 3; ++a) dtdx[a] = (a < dim) ? dt / P->dx[a] : 0.0;
  const int kz0 = (dim == 3) ? -1 : 0, kz1 = (dim == 3) ? g.n[2] : 0; /* the [-1, n] range in z, 3-D only */

  STAGE_MARK(1);
  /* Steps 4-6: traced states of every zone in [-1, n] on all active axes */
  Fields TM[3], TP[3];
  for (int d = 0; d < dim; ++d) {
    TM[d].init(N); TP[d].init(N);
    /* pencils along d through every transverse position in [-1, n] */
    int ta = (d == 0) ? 1 : 0, tb = (d == 2) ? 1 : 2;
    int a0 = -1, a1 = g.n[ta], b0 = (tb < dim) ? -1 : 0, b1 = (tb < dim) ? g.n[tb] : 0;
#ifndef ORACLE_COUNT_FLOPS
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
#endif
    for (int pb = b0; pb <= b1; ++pb)
      for (int pa = a0; pa <= a1; ++pa) {
        int c[3] = {0, 0, 0};
        c[ta] = pa;
        c[tb] = pb;
        c[d] = 0;
        trace_pencil(Q, g.id(c[0], c[1], c[2]), g.str[d], g.n[d], d, *P, dtdx[d], dt, TM[d], TP[d]);
      }
  }

  STAGE_MARK(2);
  /* Step 7a: first Riemann solves on d-faces f in [0, n_d], transverse range [-1, n].
   * Face f (between zones f-1 and f) is stored at zone index f. */
  Fields F1[3];
  for (int d = 0; d < dim; ++d) {
    F1[d].init(N);
    int lo[3] = {-1, -1, kz0}, hi[3] = {g.n[0], g.n[1], kz1};
    lo[d] = 0; hi[d] = g.n[d];
#ifndef ORACLE_COUNT_FLOPS
#pragma omp parallel for collapse(2)
#endif
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          long id = g.id(i, j, k);
          real qL[5], qR[5], sL[NS], sR[NS], F[5];
          TP[d].get(id - g.str[d], qL);
          TM[d].get(id, qR);
          state_from_prim(qL, K, sL);
          state_from_prim(qR, K, sR);
          hllc(sL, sR, d, P->gamma, P->wave_speeds, F);
          F1[d].put(id, F);
        }
  }

  STAGE_MARK(3);
  /* Step 8 (3-D only): intermediate fluxes F^{d|t}: d-states corrected by the
   * t-flux difference of their own zone with coefficient dt/(3 dx_t), on d-faces
   * [0, n_d], t-range [0, n_t), third-axis range [-1, n]. */
  Fields F2[3][3];
  if (dim == 3) {
    for (int d = 0; d < 3; ++d)
      for (int t = 0; t < 3; ++t) {
        if (t == d) continue;
        F2[d][t].init(N);
        int o = 3 - d - t;
        int lo[3], hi[3];
        lo[d] = 0; hi[d] = g.n[d];
        lo[t] = 0; hi[t] = g.n[t] - 1;
        lo[o] = -1; hi[o] = g.n[o];
        real coef = dtdx[t] * THIRD;
#ifndef ORACLE_COUNT_FLOPS
#pragma omp parallel for collapse(2)
#endif
        for (int k = lo[2]; k <= hi[2]; ++k)
          for (int j = lo[1]; j <= hi[1]; ++j)
            for (int i = lo[0]; i <= hi[0]; ++i) {
              long id = g.id(i, j, k), zl = id - g.str[d];
              real qL[5], qR[5], sL[NS], sR[NS], F[5], a[5], b[5], c5[5], e[5];
              TP[d].get(zl, qL);
              TM[d].get(id, qR);
              F1[t].get(zl + g.str[t], a); F1[t].get(zl, b);
              correct_state(qL, *P, K, coef, a, b, 0.0, nullptr, nullptr, sL);
              F1[t].get(id + g.str[t], c5); F1[t].get(id, e);
              correct_state(qR, *P, K, coef, c5, e, 0.0, nullptr, nullptr, sR);
              hllc(sL, sR, d, P->gamma, P->wave_speeds, F);
              F2[d][t].put(id, F);
            }
      }
  }

  STAGE_MARK(4);
  /* Step 8 final: d-states corrected with coefficient dt/(2 dx_t) by the
   * transverse flux differences (2-D: F^t; 3-D: F^{t1|t2} then F^{t2|t1}),
   * then the final solves on d-faces [0, n_d], transverse interior. */
  Fields F3[3];
  for (int d = 0; d < dim; ++d) {
    F3[d].init(N);
    int lo[3] = {0, 0, 0}, hi[3] = {g.n[0] - 1, g.n[1] - 1, (dim == 3) ? g.n[2] - 1 : 0};
    hi[d] = g.n[d];
    int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
#ifndef ORACLE_COUNT_FLOPS
#pragma omp parallel for collapse(2)
#endif
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          long id = g.id(i, j, k), zl = id - g.str[d];
          real qL[5], qR[5], sL[NS], sR[NS], F[5];
          TP[d].get(zl, qL);
          TM[d].get(id, qR);
          for (int side = 0; side < 2; ++side) {
            long z = side ? id : zl;
            const real* q = side ? qR : qL;
            real* s = side ? sR : sL;
            real ah[5], al[5], bh[5], bl[5];
            if (dim == 2) {
              F1[t1].get(z + g.str[t1], ah); F1[t1].get(z, al);
              correct_state(q, *P, K, 0.5 * dtdx[t1], ah, al, 0.0, nullptr, nullptr, s);
            } else {
              F2[t1][t2].get(z + g.str[t1], ah); F2[t1][t2].get(z, al);
              F2[t2][t1].get(z + g.str[t2], bh); F2[t2][t1].get(z, bl);
              correct_state(q, *P, K, 0.5 * dtdx[t1], ah, al, 0.5 * dtdx[t2], bh, bl, s);
            }
          }
          hllc(sL, sR, d, P->gamma, P->wave_speeds, F);
          F3[d].put(id, F);
        }
  }

  STAGE_MARK(5);
  /* Step 9: conservative update, x then y then z flux differences;
   * Step 10: time-centred constant-gravity source. */
  const bool grav = P->grav[0] != 0.0 || P->grav[1] != 0.0 || P->grav[2] != 0.0;
  std::vector<real> Out(W);
#ifndef ORACLE_COUNT_FLOPS
#pragma omp parallel for collapse(2) reduction(| : bad)
#endif
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        long id = g.id(i, j, k);
        real u0[5], u1[5];
        for (int c = 0; c < 5; ++c) u0[c] = W[c * N + id];
        for (int c = 0; c < 5; ++c) {
          real v = u0[c];
          for (int d = 0; d < dim; ++d) v = v - dtdx[d] * (F3[d].a[c * N + id + g.str[d]] - F3[d].a[c * N + id]);
          u1[c] = v;
        }
        if (grav) {
          real rho_mid = 0.5 * (u0[0] + u1[0]);
          for (int k2 = 0; k2 < 3; ++k2) u1[1 + k2] = u1[1 + k2] + dt * rho_mid * P->grav[k2];
          real e[3];
          if (P->grav_energy) {
            /* mass-flux form: the work gravity does on the mass crossing the
             * zone's faces, half of each face flux (exact balance with the
             * potential energy on closed domains) */
            for (int d = 0; d < 3; ++d)
              e[d] = (d < dim) ? 0.5 * (F3[d].a[id] + F3[d].a[id + g.str[d]]) * P->grav[d] : real(0.0);
          } else {
            e[0] = 0.5 * (u0[1] + u1[1]) * P->grav[0];
            e[1] = 0.5 * (u0[2] + u1[2]) * P->grav[1];
            e[2] = 0.5 * (u0[3] + u1[3]) * P->grav[2];
          }
          u1[4] = u1[4] + dt * ((e[0] + e[1]) + e[2]);
        }
        real q[5];
        int zb = 0;
        cons_to_prim(u1, *P, q, nullptr, &zb);
        bad |= zb;
        for (int c = 0; c < 5; ++c) Out[c * N + id] = u1[c];
      }
  STAGE_MARK(6);
  for (long i = 0; i < 5 * N; ++i) Uout[i] = double(Out[i]);

  if (dbg) {
    for (int d = 0; d < dim; ++d)
      for (long i = 0; i < 5 * N; ++i) {
        if (dbg->trace_m[d]) dbg->trace_m[d][i] = double(TM[d].a[i]);
        if (dbg->trace_p[d]) dbg->trace_p[d][i] = double(TP[d].a[i]);
        if (dbg->flux1[d]) dbg->flux1[d][i] = double(F1[d].a[i]);
        if (dbg->flux_final[d]) dbg->flux_final[d][i] = double(F3[d].a[i]);
      }
    if (dbg->prim)
      for (int v = 0; v < 6; ++v)
        for (long i = 0; i < N; ++i) dbg->prim[v * N + i] = double(Q[v][i]);
  }
  return bad ? ORACLE_EBADSTATE : ORACLE_OK;
}

/* ---- component entry points for unit pins ---- */
/* Method-of-lines step with nspec passive species: U holds 5 + nspec fields
 * on the grown box (rho, rho u, rho v, rho w, rho E, rho X_1 ..). */
int oracle_mol_step(const double* Uin, double* Uout, const oracle_params* P, int nspec, double dt) {
  if (!valid_params(P) || !Uin || !Uout || !(dt > 0.0) || nspec < 0 || nspec > 64) return ORACLE_EINVAL;
  const Grid g(*P);
  const int nf = NV + nspec;
  const long N = g.sc;
  int bad = 0;
  /* stage 1 from U^n with its ghosts filled */
  std::vector<real> W0(Uin, Uin + nf * N);
  fill_ghosts(W0.data(), g, *P, nf);
  std::vector<real> U1(W0);
  mol_stage(W0, g, *P, nspec, dt, U1, &bad);
  /* stage 2 from U1: its prefilled layers are still the caller's (copied from
   * W0), its derived faces are refilled from its own interior */
  fill_ghosts(U1.data(), g, *P, nf);
  std::vector<real> V2(U1);
  mol_stage(U1, g, *P, nspec, dt, V2, &bad);
  /* U^{n+1} = 1/2 U^n + 1/2 V2 on the interior; ghosts as filled at t^n */
  std::vector<real> Out(W0);
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        long id = g.id(i, j, k);
        real u[5];
        for (int c = 0; c < nf; ++c) Out[c * N + id] = 0.5 * W0[c * N + id] + 0.5 * V2[c * N + id];
        for (int c = 0; c < 5; ++c) u[c] = Out[c * N + id];
        real q5[5];
        int zb = 0;
        cons_to_prim(u, *P, q5, nullptr, &zb);
        bad |= zb;
      }
  for (long i = 0; i < nf * N; ++i) Uout[i] = double(Out[i]);
  return bad ? ORACLE_EBADSTATE : ORACLE_OK;
}

void oracle_hllc(const double* qL, const double* qR, int d, double gamma, double* F) {
  real l[5], r[5], sl[NS], sr[NS], f[5];
  for (int c = 0; c < 5; ++c) { l[c] = qL[c]; r[c] = qR[c]; }
  Consts K;
  K.gamma = gamma;
  K.gm1inv = 1.0 / (gamma - 1.0);
  state_from_prim(l, K, sl);
  state_from_prim(r, K, sr);
  hllc(sl, sr, d, gamma, 0, f);
  for (int c = 0; c < 5; ++c) F[c] = double(f[c]);
}

void oracle_wave_speeds(const double* qL, const double* qR, int d, double gamma, int einfeldt, double* out) {
  real l[5], r[5], sl[NS], sr[NS];
  for (int c = 0; c < 5; ++c) { l[c] = qL[c]; r[c] = qR[c]; }
  Consts K;
  K.gamma = gamma;
  K.gm1inv = 1.0 / (gamma - 1.0);
  state_from_prim(l, K, sl);
  state_from_prim(r, K, sr);
  real cl = sound_speed(sl[S_P], sl[S_INV], gamma), cr = sound_speed(sr[S_P], sr[S_INV], gamma);
  real a, b;
  wave_speeds(sl, sr, d, gamma, einfeldt, cl, cr, &a, &b);
  out[0] = double(a);
  out[1] = double(b);
}

void oracle_ppm_parabola(const double* line7, double chi, double* am_ap_a6) {
  real a[7], am, ap, a6;
  for (int m = 0; m < 7; ++m) a[m] = line7[m];
  ppm_parabola(a, chi, &am, &ap, &a6);
  am_ap_a6[0] = double(am); am_ap_a6[1] = double(ap); am_ap_a6[2] = double(a6);
}

double oracle_flatten(const double* p7, const double* un7, double small_pres) {
  real p[7], u[7];
  for (int m = 0; m < 7; ++m) { p[m] = p7[m]; u[m] = un7[m]; }
  return double(flat_coef(p, u, small_pres));
}

double oracle_integ(const double* am_ap_a6, double sigma, int plus) {
  real am = am_ap_a6[0], ap = am_ap_a6[1], a6 = am_ap_a6[2];
  return double(plus ? integ_plus(am, ap, a6, sigma) : integ_minus(am, ap, a6, sigma));
}

/* Trace one zone from 7-point primitive lines along direction d (rho,u,v,w,p
 * and c, each 7 values).  Used by the unit pins of the tracing step. */
void oracle_trace_lines(const double* lines6x7, int d, const oracle_params* P, double dtdx, double dt,
                        double* qm, double* qp) {
  std::vector<real> Q[NQ];
  for (int v = 0; v < 6; ++v) {
    Q[v].resize(7);
    for (int m = 0; m < 7; ++m) Q[v][m] = lines6x7[v * 7 + m];
  }
  for (int v = 6; v < NQ; ++v) Q[v].resize(7);
  for (int m = 0; m < 7; ++m) {
    real rho = Q[QRHO][m], c = Q[QC][m];
    Q[QRC][m] = rho / c;
    Q[QCR][m] = c / rho;
    Q[QIC2][m] = 1.0 / (c * c);
  }
  real m5[5], p5[5];
  const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
  const int vmap[5] = {QRHO, QU + d, QU + t1, QU + t2, QP};
  real line[5][7], am[5], ap[5], a6[5], zone[5];
  for (int v = 0; v < 5; ++v)
    for (int m = 0; m < 7; ++m) line[v][m] = Q[vmap[v]][m];
  real chi = P->flatten ? flat_coef(line[4], line[1], P->small_pres) : real(1.0);
  for (int v = 0; v < 5; ++v) {
    ppm_parabola(line[v], chi, &am[v], &ap[v], &a6[v]);
    zone[v] = line[v][3];
  }
  trace_from_parabola(am, ap, a6, zone, Q, 3, d, *P, dtdx, dt, m5, p5);
  for (int c = 0; c < 5; ++c) { qm[c] = double(m5[c]); qp[c] = double(p5[c]); }
}

void oracle_cons_to_prim(const double* U, const oracle_params* P, double* q, int* bad) {
  real u[5], r[5];
  for (int c = 0; c < 5; ++c) u[c] = U[c];
  int b = 0;
  cons_to_prim(u, *P, r, nullptr, &b);
  for (int c = 0; c < 5; ++c) q[c] = double(r[c]);
  if (bad) *bad = b;
}

void oracle_prim_to_cons(const double* q, double gamma, double* U) {
  real r[5], u[5];
  for (int c = 0; c < 5; ++c) r[c] = q[c];
  Consts K;
  K.gamma = gamma;
  K.gm1inv = 1.0 / (gamma - 1.0);
  prim_to_cons(r, K, u);
  for (int c = 0; c < 5; ++c) U[c] = double(u[c]);
}

#ifdef ORACLE_COUNT_FLOPS
void oracle_tally_reset(void) {
  g_tally = op_tally{0, 0, 0, 0, 0};
  for (auto& t : g_stage_tally) t = op_tally{0, 0, 0, 0, 0};
}
void oracle_tally_stages(long long* out30) {
  for (int k = 0; k < 6; ++k) {
    const op_tally& t = g_stage_tally[k];
    out30[5 * k + 0] = t.add; out30[5 * k + 1] = t.mul; out30[5 * k + 2] = t.div;
    out30[5 * k + 3] = t.sqrt; out30[5 * k + 4] = t.cmp;
  }
}
void oracle_tally_get(long long* out5) {
  out5[0] = g_tally.add; out5[1] = g_tally.mul; out5[2] = g_tally.div;
  out5[3] = g_tally.sqrt; out5[4] = g_tally.cmp;
}
#endif

} /* extern "C" */
