// Per-item device bodies of the staged CTU-PPM step.  Each stage is a
// function of one work item t (a zone, a face, or a pencil segment of one
// box); the single-box kernels and the batched kernels are thin wrappers
// that only differ in how they find the box and the item index.
#pragma once
#include "hydro_step.cuh"

namespace hydro {
namespace {

constexpr int BLOCK = 128;
// Resident blocks per SM of the single-box solver kernels (launch bound):
// with the Davis speeds the first, intermediate and final solves fit 56
// registers and run at nine blocks per SM (1.0 % faster per Sedov 128^3
// step than at eight with 64 registers; 66-70 registers at seven were 1-3 %
// slower); the Einfeldt speeds keep eight.  (The batched level's solver
// kernels measured the same at nine, with small spills, and keep theirs.)
__host__ __device__ constexpr int solver_blocks(bool einf) { return einf ? 8 : 9; }

__device__ __forceinline__ bool range_zone(const Range& R, long long t, int& i, int& j, int& k) {
  long long e0 = R.ext[0], e1 = R.ext[1];
  if (t >= e0 * e1 * R.ext[2]) return false;
  i = R.lo[0] + (int)(t % e0);
  long long r = t / e0;
  j = R.lo[1] + (int)(r % e1);
  k = R.lo[2] + (int)(r / e1);
  return true;
}

// map a grown-box coordinate on one axis to the interior zone whose data it holds
__device__ __forceinline__ int map_axis(int i, int n, int bclo, int bchi, bool& flip) {
  if (i < 0) {
    if (bclo == 0) return 0;                        // outflow
    if (bclo == 1) { flip = !flip; return -1 - i; } // reflect
    if (bclo == 2) return i + n;                    // periodic
    return i;                                       // prefilled
  }
  if (i >= n) {
    if (bchi == 0) return n - 1;
    if (bchi == 1) { flip = !flip; return 2 * n - 1 - i; }
    if (bchi == 2) return i - n;
    return i;
  }
  return i;
}

// ---- stage 1: conserved -> primitive on the grown box (ghosts mapped by BC kind)
__device__ __forceinline__ void prim_item(BoxGeom in, ScratchGeom sg, double* __restrict__ Q, StepConst K,
                                                Range R, DevFlags* flags, long long t) {
  int i, j, k;
  if (!range_zone(R, t, i, j, k)) return;
  bool flip[3] = {false, false, false};
  int src[3] = {i, j, k};
  src[0] = map_axis(i, in.n[0], in.bc[0][0], in.bc[0][1], flip[0]);
  src[1] = map_axis(j, in.n[1], in.bc[1][0], in.bc[1][1], flip[1]);
  if (K.dim == 3) src[2] = map_axis(k, in.n[2], in.bc[2][0], in.bc[2][1], flip[2]);
  long long si = in.id(src[0], src[1], src[2]);
  double U[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) U[c] = in.u[c * in.sc + si];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (flip[a]) U[1 + a] = -U[1 + a];
  double q[5], inv;
  bool bad = false;
  cons_to_prim_flag(U, K, q, &inv, &bad);
  if (bad) atomicOr(&flags->bad, 1);
  long long id = sg.id(i, j, k);
#pragma unroll
  for (int v = 0; v < 5; ++v) Q[v * sg.sc + id] = q[v];
  double c, rho_c, c_rho, inv_c2;
#ifndef HYDRO_IEEE_DIV_SQRT
  // product build: every sound-speed quantity from one refined
  // y = 1/sqrt(gamma p rho): c = (gamma p) y, 1/c = rho y, rho/c = rho (rho y),
  // c/rho = c (c y) with c y = 1/rho, 1/c^2 = (rho y)^2
  const double gp = mul_i(K.gamma, q[4]);
  const double x = gp * q[0];
  if (__builtin_expect(newton_range(x), 1)) {
    const double y = rsqrt_newton(x);
    const double ry = q[0] * y;
    c = gp * y;
    rho_c = q[0] * ry;
    c_rho = c * (c * y);
    inv_c2 = ry * ry;
  } else
#endif
  {
    c = dsqrt(mul_i(mul_i(K.gamma, q[4]), inv));
    rho_c = ddiv(q[0], c);
    c_rho = ddiv(c, q[0]);
    inv_c2 = drcp(mul_i(c, c));
  }
  Q[QC * sg.sc + id] = c;
  Q[QRC * sg.sc + id] = rho_c;
  Q[QCR * sg.sc + id] = c_rho;
  Q[QIC2 * sg.sc + id] = inv_c2;
}

// ---- stage 3 of a zone: characteristic tracing from its parabolas
// am/ap/dap (= ap - am)/a6/zone: (rho, un, ut1, ut2, p); outputs the zone's low- and high-face
// states to TM/TP at id in absolute component order.
// SKIP_FLAT: test for flat parabolas and skip their integrals (below); the
// sequential sweep leaves it off: on data where every zone moves the test's
// branch cost its launches 11 % (the row and tile kernels 4-5 %, which the
// zones at rest of a blast repay several times over)
template <int D, bool SKIP_FLAT = true>
__device__ __forceinline__ void trace_zone(const double am[5], const double ap[5], const double dap[5],
                                           const double a6[5], const double zone[5], double c, double rho_c,
                                           double c_rho, double inv_c2, const StepConst& K, double* __restrict__ TM,
                                           double* __restrict__ TP, long long sc, long long id) {
  constexpr int T1 = (D == 0) ? 1 : 0, T2 = (D == 2) ? 1 : 2;
  const double un = zone[1];
  const double c2 = c * c;
  const double lu = dhalf(rho_c), lp = dhalf(inv_c2);
  const double lam[3] = {un - c, un, un + c};
  double sig[3];
#pragma unroll
  for (int w = 0; w < 3; ++w) sig[w] = fabs(lam[w]) * K.dtdx[D];
  // Reference states: the fastest wave toward each face (lambda_- toward the
  // low face, lambda_+ toward the high face), else the zone average.
  // o0 / o1: the low / high face's edge state (rho, un, ut1, ut2, p).
  const bool fast_lo = lt0(lam[0]), fast_hi = gt0(lam[2]);
  // Flat parabolas (a+ - a- and a6 both +0, as the limiter leaves a zone at
  // rest or at an extremum): the swept-volume term (+-)s/2 (da +- t a6) is
  // +0 for any s, so I- is a- + (+0) = pz(a-) and I+ is a+ - (+0) = a+,
  // bit for bit in either build; the integrals are skipped.
  long long nonflat = 0;  // OR of the bit patterns: 0 only if every one is +0
#pragma unroll
  for (int v = 0; v < 5; ++v) nonflat |= dbits(dap[v]) | dbits(a6[v]);
  double o0[5], o1[5];
  if (SKIP_FLAT && !ine(nonflat, 0LL)) {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      o0[v] = fast_lo ? pz(am[v]) : zone[v];
      o1[v] = fast_hi ? ap[v] : zone[v];
    }
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      o0[v] = fast_lo ? integ_minus(am[v], ap[v], dap[v], a6[v], sig[0]) : zone[v];
      o1[v] = fast_hi ? integ_plus(am[v], ap[v], dap[v], a6[v], sig[2]) : zone[v];
    }
  }
  // Edge state = ref - sum of beta_nu r_nu over the waves that reach the
  // face: s_rho = ref - ((bm + b0) + bp), s_un = ref - (bm (-c/rho) + bp c/rho),
  // s_p = ref - (bm c^2 + bp c^2), s_t = ref - bt.  The reference wave's beta
  // is exactly +0 (ref - I(sigma_fast) == 0) and a wave that does not reach
  // contributes +0.0, so only the terms of the other waves are formed; where
  // a +0 is dropped from a sum, pz() applies what adding it does (turn -0
  // into +0), and every edge state is bitwise the full expression's.
  // The entropy and shear wave (lambda_0 = u_n) reaches the high face when
  // u_n > 0 and the low face when u_n < 0, never both, so its terms are formed
  // once, on the inputs of the face it reaches (lanes of a warp with opposite
  // signs of u_n then share one pass).  The low face's integral
  // a- + s/2 (da + (1 - 2s/3) a6) is the high face's form a+ - s/2 (da - (1 - 2s/3) a6)
  // with a+ -> a- and da -> -da, negation being exact.  The other acoustic
  // wave reaches only if the entropy wave does, and nothing but the reference
  // wave reaches if that one does not.
  const bool hi = gt0(un);
  if (hi || lt0(un)) {
    const double t = 1.0 - TWOTHIRDS * sig[1], hs = dhalf(sig[1]);
    double ref[5], i0[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      ref[v] = hi ? o1[v] : o0[v];
      const double e = hi ? ap[v] : am[v], x = hi ? dap[v] : dneg(dap[v]);
      i0[v] = e - hs * (x - t * a6[v]);  // I(sigma_0) of the reached face (unused for u_n)
    }
    const double b0 = (ref[0] - i0[0]) - inv_c2 * (ref[4] - i0[4]);
    const double bt1 = ref[2] - i0[2], bt2 = ref[3] - i0[3];
    double s[5];
    s[1] = ref[1];
    s[2] = ref[2] - bt1;
    s[3] = ref[3] - bt2;
    s[4] = ref[4];
    if (hi && gt0(lam[0])) {  // supersonic toward the high face: lambda_- reaches it too
      const double bm = -lu * (ref[1] - integ_plus(am[1], ap[1], dap[1], a6[1], sig[0])) +
                        lp * (ref[4] - integ_plus(am[4], ap[4], dap[4], a6[4], sig[0]));
      s[0] = ref[0] - pz(bm + b0);
      s[1] = ref[1] - pz(bm * (-c_rho));
      s[4] = ref[4] - pz(bm * c2);
    } else if (!hi && lt0(lam[2])) {  // supersonic toward the low face: lambda_+ reaches it too
      const double bp = lu * (ref[1] - integ_minus(am[1], ap[1], dap[1], a6[1], sig[2])) +
                        lp * (ref[4] - integ_minus(am[4], ap[4], dap[4], a6[4], sig[2]));
      s[0] = ref[0] - (pz(b0) + bp);
      s[1] = ref[1] - bp * c_rho;  // (-0) + bp c/rho is bp c/rho
      s[4] = ref[4] - pz(bp * c2);
    } else {
      s[0] = ref[0] - pz(b0);
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      o1[v] = hi ? s[v] : o1[v];
      o0[v] = hi ? o0[v] : s[v];
    }
  }
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    double* o = side ? o1 : o0;
    double s_rho = o[0], s_un = o[1], s_t1 = o[2], s_t2 = o[3], s_p = o[4];
    if (K.has_grav) {
      s_un = s_un + K.hdt * K.grav[D];
      s_t1 = s_t1 + K.hdt * K.grav[T1];
      s_t2 = s_t2 + K.hdt * K.grav[T2];
    }
    s_rho = dmax(s_rho, K.small_dens);
    s_p = dmax(s_p, K.small_pres);
    // primitive form; the first Riemann solve adds the conserved form
    double* out = side ? TP : TM;
    out[0 * sc + id] = s_rho;
    out[(1 + D) * sc + id] = s_un;
    out[(1 + T1) * sc + id] = s_t1;
    out[(1 + T2) * sc + id] = s_t2;
    out[4 * sc + id] = s_p;
  }
}

// ---- stages 2-3: flattening, PPM reconstruction and characteristic tracing
// along d.  Each thread sweeps one pencil segment, so every flattening
// coefficient, slope and interface value is formed once per zone (plus a
// two-zone warm-up per segment) from sliding register windows.
template <int D>
__device__ __forceinline__ void trace_item(ScratchGeom sg, const double* __restrict__ Q,
                                                 double* __restrict__ TM, double* __restrict__ TP, StepConst K,
                                                 SweepRange R, long long t) {
  if (t >= R.count()) return;
  constexpr int T1 = (D == 0) ? 1 : 0, T2 = (D == 2) ? 1 : 2;
  int c3[3];
  c3[T1] = R.lo1 + (int)(t % R.ext1);
  long long r = t / R.ext1;
  c3[T2] = R.lo2 + (int)(r % R.ext2);
  const int seg = (int)(r / R.ext2);
  const int i0 = R.lod + seg * R.seg;
  const int i1 = min(i0 + R.seg, R.nd + 1);
  c3[D] = i0;
  const long long sc = sg.sc;
  const long long st = (D == 0) ? 1 : (D == 1) ? sg.sy : sg.sz;
  const long long base = sg.id(c3[0], c3[1], c3[2]);
  const double* __restrict__ qv[5] = {Q + QRHO * sc, Q + (QU + D) * sc, Q + (QU + T1) * sc, Q + (QU + T2) * sc,
                                      Q + QP * sc};
  const double sp = K.small_pres;

  // windows relative to the current zone i: a0 = a_i, a1 = a_{i+1}, sl = slope_i,
  // fm = interface i-1/2; pressures pm2 = p_{i-2}, pm1 = p_{i-1}, pp2 = p_{i+2};
  // flattening ctm = chi~_{i-1}, ct0 = chi~_i
  double a0[5], a1[5], sl[5], fm[5], d01[5];  // d01 = a1 - a0
  double pm2, pm1, pp2, ctm = 1.0, ct0 = 1.0;
  {
    double am2[5], am1[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      am2[v] = qv[v][base - 2 * st];
      am1[v] = qv[v][base - st];
      a0[v] = qv[v][base];
      a1[v] = qv[v][base + st];
    }
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double dm = am1[v] - am2[v], d0 = a0[v] - am1[v];
      d01[v] = a1[v] - a0[v];
      double s_m1 = mc_slope_d(dm, d0, am2[v], a0[v]);
      sl[v] = mc_slope_d(d0, d01[v], am1[v], a1[v]);
      fm[v] = face_value(am1[v], a0[v], s_m1, sl[v]);
    }
    pm2 = am2[4];
    pm1 = am1[4];
    pp2 = qv[4][base + 2 * st];
    if (K.flatten) {
      double pm3 = qv[4][base - 3 * st];
      ctm = flat_tilde(pm3, pm2, a0[4], a1[4], am2[1], a0[1], sp);
      ct0 = flat_tilde(pm2, pm1, a1[4], pp2, am1[1], a1[1], sp);
    }
  }
  // operands that enter at each zone (a_{i+2} of rho, u_n, u_t1, u_t2; p_{i+3};
  // the sound-speed fields of zone i) are loaded one zone ahead, so that their
  // latency overlaps the arithmetic of the zone before
  double na2[4], np3, nc[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) na2[v] = qv[v][base + 2 * st];
  np3 = qv[4][base + 3 * st];
  nc[0] = Q[QC * sc + base]; nc[1] = Q[QRC * sc + base]; nc[2] = Q[QCR * sc + base]; nc[3] = Q[QIC2 * sc + base];
  for (int i = i0; i < i1; ++i) {
    const long long id = base + (long long)(i - i0) * st;
    double a2[5], cz[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) a2[v] = na2[v];
    a2[4] = pp2;
    const double p3 = np3;  // p_{i+3}
#pragma unroll
    for (int k = 0; k < 4; ++k) cz[k] = nc[k];
    if (i + 1 < i1) {
#pragma unroll
      for (int v = 0; v < 4; ++v) na2[v] = qv[v][id + 3 * st];
      np3 = qv[4][id + 4 * st];
      nc[0] = Q[QC * sc + id + st]; nc[1] = Q[QRC * sc + id + st];
      nc[2] = Q[QCR * sc + id + st]; nc[3] = Q[QIC2 * sc + id + st];
    }
    double chi = 1.0, ctp = 1.0;
    if (K.flatten) {
      ctp = flat_tilde(pm1, a0[4], a2[4], p3, a0[1], a2[1], sp);
      // p_{i+1} - p_{i-1} < 0 as an order comparison
      chi = dless(a1[4], pm1) ? dmin(ct0, ctp) : dmin(ct0, ctm);
    }
    double am[5], ap[5], dap[5], a6[5], zone[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      const double d12 = a2[v] - a1[v];
      double s1 = mc_slope_d(d01[v], d12, a0[v], a2[v]);
      d01[v] = d12;
      double fp = face_value(a0[v], a1[v], sl[v], s1);
      ppm_limit(a0[v], fm[v], fp, chi, am[v], ap[v], a6[v], &dap[v]);
      zone[v] = a0[v];
      sl[v] = s1;
      fm[v] = fp;
    }
    trace_zone<D, false>(am, ap, dap, a6, zone, cz[0], cz[1], cz[2], cz[3], K, TM, TP, sc, id);
    // slide the windows one zone
    pm2 = pm1;
    pm1 = a0[4];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      a0[v] = a1[v];
      a1[v] = a2[v];
    }
    pp2 = p3;
    ctm = ct0;
    ct0 = ctp;
  }
}

// ---- stages 2-3 along x with the lanes of a warp along the pencils.  The
// pencils' zones lie end to end in one sequence of positions, each pencil
// holding its zones [lod - 1, nd + 1]: the traced zones and one zone beyond
// each end.  Warp w takes positions [ROW_ZONES w - 1, ROW_ZONES w + 31); lane l
// holds position ROW_ZONES w - 1 + l and traces it when l is in
// [1, ROW_ZONES] and the position is a traced zone, so lanes 0 and 31 and the
// zones beyond a pencil's ends only supply the slope, the flattening
// coefficient and the interface value their neighbours need.  A warp may
// cover the end of one pencil and the start of the next: the two positions
// between them are those beyond-the-end zones, so every traced zone's
// neighbours are of its own pencil.  Every quantity of a zone is the
// tracing sweep's, by the same expressions: the slope and the flattening
// coefficient of each zone once, the interface value at its high face once,
// the neighbours' values through shuffles.  The loads of a warp are
// consecutive doubles (the sequential sweep along x reads with lanes along
// y, a cache line per lane).
constexpr int ROW_ZONES = 30;
// positions of one pencil, and warps for a range
__host__ __device__ __forceinline__ int row_positions(const SweepRange& R) { return R.nd - R.lod + 3; }
__host__ __device__ __forceinline__ long long row_warps(const SweepRange& R) {
  const long long npos = (long long)row_positions(R) * R.ext1 * R.ext2;
  return (npos + ROW_ZONES - 1) / ROW_ZONES;
}

// Zones at rest.  When, in every variable, a zone's average equals its
// neighbours' (bit for bit), its one-sided differences are +0, so every
// monotonised slope is +0 -- what mc_slope_d returns for them -- and the
// differences are not formed.  When two neighbours are equal with equal
// slopes in every variable, the interface value between them is the zone
// value: (a + a)/2 - (s - s)/6 = a - (+0) = a, bit for bit with or without
// contraction.  Each test is one OR of the operands' bit differences; in a
// region at rest whole warps take these paths.
__device__ __forceinline__ bool slopes_vanish(const double am1[5], const double a0[5], const double ap1[5]) {
  long long diff = 0;
#pragma unroll
  for (int v = 0; v < 5; ++v) diff |= (dbits(am1[v]) ^ dbits(a0[v])) | (dbits(a0[v]) ^ dbits(ap1[v]));
  return !ine(diff, 0LL);
}
__device__ __forceinline__ void zone_slopes(const double am1[5], const double a0[5], const double ap1[5], double sl[5]) {
  if (slopes_vanish(am1, a0, ap1)) {
#pragma unroll
    for (int v = 0; v < 5; ++v) sl[v] = 0.0;
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) sl[v] = mc_slope_d(a0[v] - am1[v], ap1[v] - a0[v], am1[v], ap1[v]);
  }
}
__device__ __forceinline__ bool faces_trivial(const double a0[5], const double a1[5], const double s0[5],
                                              const double s1[5]) {
  long long diff = 0;
#pragma unroll
  for (int v = 0; v < 5; ++v) diff |= (dbits(a0[v]) ^ dbits(a1[v])) | (dbits(s0[v]) ^ dbits(s1[v]));
  return !ine(diff, 0LL);
}
__device__ __forceinline__ void zone_faces(const double a0[5], const double a1[5], const double s0[5],
                                           const double s1[5], double fp[5]) {
  if (faces_trivial(a0, a1, s0, s1)) {
#pragma unroll
    for (int v = 0; v < 5; ++v) fp[v] = a0[v];
  } else {
#pragma unroll
    for (int v = 0; v < 5; ++v) fp[v] = face_value(a0[v], a1[v], s0[v], s1[v]);
  }
}

__device__ __forceinline__ double shfl_up1(double x) { return __shfl_up_sync(0xffffffffu, x, 1); }
__device__ __forceinline__ double shfl_dn1(double x) { return __shfl_down_sync(0xffffffffu, x, 1); }

// w: the warp's work item (tile fastest, then T1, then T2); all 32 lanes call
__device__ __forceinline__ void trace_row_x_item(ScratchGeom sg, const double* __restrict__ Q,
                                                 double* __restrict__ TM, double* __restrict__ TP, StepConst K,
                                                 SweepRange R, long long w) {
  const int L = row_positions(R);
  const long long npos = (long long)L * R.ext1 * R.ext2;
  const long long p0 = w * ROW_ZONES - 1;  // the warp's first position
  if (p0 >= npos) return;  // uniform over the warp
  const int lane = threadIdx.x & 31;
  const long long pos = p0 + lane;
  // positions in the range hold zones lod - 1 .. nd + 1 of their pencil,
  // whose stencils stay in the grown box; the others load nothing
  const bool live = pos >= 0 && pos < npos;
  const long long r = live ? pos / L : 0;
  const int q = live ? (int)(pos - r * L) : 0;
  const int j = R.lo1 + (int)(r % R.ext1), k = R.lo2 + (int)(r / R.ext1);
  const int i = R.lod - 1 + q;
  const long long sc = sg.sc;
  const long long id = sg.id(i, j, k);
  const double* __restrict__ qv[5] = {Q + QRHO * sc, Q + QU * sc, Q + QV * sc, Q + QW * sc, Q + QP * sc};
  double am1[5], a0[5], ap1[5], pm2 = 0.0, pp2 = 0.0;
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    am1[v] = live ? qv[v][id - 1] : 0.0;
    a0[v] = live ? qv[v][id] : 0.0;
    ap1[v] = live ? qv[v][id + 1] : 0.0;
  }
  if (live && K.flatten) {
    pm2 = qv[4][id - 2];
    pp2 = qv[4][id + 2];
  }
  // this zone's slope and flattening coefficient
  double sl[5];
  zone_slopes(am1, a0, ap1, sl);
  const double ct0 = K.flatten ? flat_tilde(pm2, am1[4], ap1[4], pp2, am1[1], ap1[1], K.small_pres) : 1.0;
  // the interface value at the high face, from the next zone's slope
  double fp[5], fm[5], sn[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) sn[v] = shfl_dn1(sl[v]);
  zone_faces(a0, ap1, sl, sn, fp);
#pragma unroll
  for (int v = 0; v < 5; ++v) fm[v] = shfl_up1(fp[v]);
  const double ctm = shfl_up1(ct0), ctp = shfl_dn1(ct0);
  if (lane == 0 || lane > ROW_ZONES || !live || q < 1 || q > L - 2) return;
  double chi = 1.0;
  if (K.flatten) chi = dless(ap1[4], am1[4]) ? dmin(ct0, ctp) : dmin(ct0, ctm);
  double am[5], ap[5], dap[5], a6[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) ppm_limit(a0[v], fm[v], fp[v], chi, am[v], ap[v], a6[v], &dap[v]);
  trace_zone<0>(am, ap, dap, a6, a0, Q[QC * sc + id], Q[QRC * sc + id], Q[QCR * sc + id], Q[QIC2 * sc + id], K, TM,
                TP, sc, id);
}

// ---- stages 2-3 along y or z in tiles: a block of TILE_W warps takes 32
// pencils (consecutive positions of the flattened transverse range, x
// fastest, so the loads of a warp are consecutive doubles) and TILE_ZONES
// zones [t0, t0 + TILE_ZONES) along D.  Three phases, each spread over the
// warps and separated by barriers: the slope and flattening coefficient of
// every zone of [t0 - 1, t0 + TILE_ZONES], the interface value at the high
// face of every zone of [t0 - 1, t0 + TILE_ZONES), then the limiter and the
// tracing of the tile's zones, exchanging the zones' values through shared
// memory.  Every quantity is formed once per zone (plus the two halo zones
// per tile) by the sweep's expressions, so the traced states are the
// sweep's bit for bit; a thread holds one zone's values instead of a
// sweep's sliding windows, so more warps fit an SM.
constexpr int TILE_ZONES = 12, TILE_W = 4;
struct TileSmem {
  double sl[5][TILE_ZONES + 2][32];  // slopes, rows t0 - 1 .. t0 + TILE_ZONES
  double ct[TILE_ZONES + 2][32];     // flattening coefficients, same rows
  double fp[5][TILE_ZONES + 1][32];  // interface value at the high face, rows t0 - 1 .. t0 + TILE_ZONES - 1
};

// blk: the block's work item (column group fastest, then the tile along D)
template <int D>
__device__ __forceinline__ void trace_tile_item(ScratchGeom sg, const double* __restrict__ Q,
                                                double* __restrict__ TM, double* __restrict__ TP, StepConst K,
                                                SweepRange R, long long blk, TileSmem& sm) {
  constexpr int T1 = (D == 0) ? 1 : 0, T2 = (D == 2) ? 1 : 2;
  const long long ncol = (long long)R.ext1 * R.ext2;
  const long long ngroup = (ncol + 31) / 32;
  const int tile = (int)(blk / ngroup);
  const long long col = (blk - tile * ngroup) * 32 + (threadIdx.x & 31);
  const int warp = threadIdx.x >> 5;
  const bool cvalid = col < ncol;
  int c3[3];
  c3[T1] = R.lo1 + (int)(cvalid ? col % R.ext1 : 0);
  c3[T2] = R.lo2 + (int)(cvalid ? col / R.ext1 : 0);
  const int t0 = R.lod + tile * TILE_ZONES;
  c3[D] = t0;
  const long long sc = sg.sc;
  const long long st = (D == 0) ? 1 : (D == 1) ? sg.sy : sg.sz;
  const long long id0 = sg.id(c3[0], c3[1], c3[2]);  // zone t0 of this pencil
  const double* __restrict__ qv[5] = {Q + QRHO * sc, Q + (QU + D) * sc, Q + (QU + T1) * sc, Q + (QU + T2) * sc,
                                      Q + QP * sc};
  // phase A: rows r = 0 .. TILE_ZONES + 1 hold zones t0 - 1 + r (live up to nd + 1)
  for (int r = warp; r < TILE_ZONES + 2; r += TILE_W) {
    const int i = t0 - 1 + r;
    if (cvalid && i <= R.nd + 1) {
      const long long id = id0 + (long long)(r - 1) * st;
      double am1[5], a0[5], ap1[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        am1[v] = qv[v][id - st];
        a0[v] = qv[v][id];
        ap1[v] = qv[v][id + st];
      }
      double sl[5];
      zone_slopes(am1, a0, ap1, sl);
#pragma unroll
      for (int v = 0; v < 5; ++v) sm.sl[v][r][threadIdx.x & 31] = sl[v];
      sm.ct[r][threadIdx.x & 31] =
          K.flatten ? flat_tilde(qv[4][id - 2 * st], am1[4], ap1[4], qv[4][id + 2 * st], am1[1], ap1[1], K.small_pres)
                    : 1.0;
    }
  }
  __syncthreads();
  // phase B: the interface value at the high face of zones t0 - 1 + r, r = 0 .. TILE_ZONES
  for (int r = warp; r < TILE_ZONES + 1; r += TILE_W) {
    const int i = t0 - 1 + r;
    if (cvalid && i <= R.nd) {
      const long long id = id0 + (long long)(r - 1) * st;
      const int l = threadIdx.x & 31;
      double a0[5], a1[5], s0[5], s1[5], fp[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        a0[v] = qv[v][id];
        a1[v] = qv[v][id + st];
        s0[v] = sm.sl[v][r][l];
        s1[v] = sm.sl[v][r + 1][l];
      }
      zone_faces(a0, a1, s0, s1, fp);
#pragma unroll
      for (int v = 0; v < 5; ++v) sm.fp[v][r][l] = fp[v];
    }
  }
  __syncthreads();
  // phase C: limiter and tracing of zones t0 + r, r = 0 .. TILE_ZONES - 1
  for (int r = warp; r < TILE_ZONES; r += TILE_W) {
    const int i = t0 + r;
    if (!cvalid || i > R.nd) continue;
    const int l = threadIdx.x & 31;
    const long long id = id0 + (long long)r * st;
    double a0[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) a0[v] = qv[v][id];
    double chi = 1.0;
    if (K.flatten) {
      const double ct0 = sm.ct[r + 1][l];
      chi = dless(qv[4][id + st], qv[4][id - st]) ? dmin(ct0, sm.ct[r + 2][l]) : dmin(ct0, sm.ct[r][l]);
    }
    double am[5], ap[5], dap[5], a6[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) ppm_limit(a0[v], sm.fp[v][r][l], sm.fp[v][r + 1][l], chi, am[v], ap[v], a6[v], &dap[v]);
    trace_zone<D>(am, ap, dap, a6, a0, Q[QC * sc + id], Q[QRC * sc + id], Q[QCR * sc + id], Q[QIC2 * sc + id], K, TM,
                  TP, sc, id);
  }
}

__device__ __forceinline__ void load5(const double* __restrict__ A, long long sc, long long id, double v[5]) {
#pragma unroll
  for (int c = 0; c < 5; ++c) v[c] = A[c * sc + id];
}
// face state (and its sound speed *cs) of a traced state for its (only)
// first Riemann solve; the conserved form (rho*u, rho*v, rho*w, rho*E) is
// stored beside the primitive fields, since the transverse corrections update
// it three more times
__device__ __forceinline__ void traced_state(double* __restrict__ T, long long sc, long long id,
                                             const StepConst& K, double s[NS], double* cs) {
  double q[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) q[v] = T[v * sc + id];
  state_from_prim_c(q, K, s, cs);
#pragma unroll
  for (int c = 1; c < 4; ++c) T[(TS_MOM + c - 1) * sc + id] = mul_i(q[0], q[c]);
  T[TS_E * sc + id] = s[S_E];
}
__device__ __forceinline__ void store5(double* __restrict__ A, long long sc, long long id, const double v[5]) {
#pragma unroll
  for (int c = 0; c < 5; ++c) A[c * sc + id] = v[c];
}

// ---- stage 4a: first Riemann solves from the traced states
// (EINF: Einfeldt outer wave speeds, else Davis; launches choose it from K.einfeldt)
template <int D, bool EINF>
__device__ __forceinline__ void flux1_item(ScratchGeom sg, double* __restrict__ TP, double* __restrict__ TM,
                                           double* __restrict__ F1, StepConst K, Range R, long long t) {
  int i, j, k;
  if (!range_zone(R, t, i, j, k)) return;
  const long long st = (D == 0) ? 1 : (D == 1) ? sg.sy : sg.sz;
  const long long id = sg.id(i, j, k);
  double sL[NS], sR[NS], F[5], cl, cr;
  traced_state(TP, sg.sc, id - st, K, sL, &cl);
  traced_state(TM, sg.sc, id, K, sR, &cr);
  hllc_flux_c<EINF>(sL, sR, cl, cr, D, K, F);
  store5(F1, sg.sc, id, F);
}

// U <- U - c (F[hi] - F[lo]), five components.  Where the two fluxes are
// equal bit for bit in every component (a region at rest), each difference
// is +0 and U - c (+0) is U with or without contraction, so the arithmetic
// is skipped; whole warps take that path outside a blast.
__device__ __forceinline__ void sub_flux_difference(double U[5], double c, const double* __restrict__ F,
                                                    long long sc, long long hi, long long lo) {
  double fh[5], fl[5];
  long long diff = 0;  // OR of the components' bit differences
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    fh[k] = F[k * sc + hi];
    fl[k] = F[k * sc + lo];
    diff |= dbits(fh[k]) ^ dbits(fl[k]);
  }
  if (ine(diff, 0LL)) {
#pragma unroll
    for (int k = 0; k < 5; ++k) U[k] = U[k] - c * (fh[k] - fl[k]);
  }
}

// transverse correction of a traced state (conserved form at T[.., id]) by
// one or two flux differences, back to a face state.  SKIP: skip the
// differences of equal fluxes (the final solves); the intermediate solves
// ran 3 % slower with it (1.686 against 1.643 ms per Sedov 128^3 step: the
// test gathers all ten flux values before any arithmetic, and its integer
// work joins the third of their products already on the integer pipe), so
// they keep the plain form.
template <bool SKIP>
__device__ __forceinline__ void correct(const double* __restrict__ T, long long id, const StepConst& K, double ca,
                                        const double* Fa, long long sc, long long ida_hi, long long ida_lo,
                                        double cb, const double* Fb, long long idb_hi, long long idb_lo,
                                        double s[NS]) {
  double U[5];
  U[0] = T[id];
  U[1] = T[TS_MOM * sc + id];
  U[2] = T[(TS_MOM + 1) * sc + id];
  U[3] = T[(TS_MOM + 2) * sc + id];
  U[4] = T[TS_E * sc + id];
  if (SKIP) {
    sub_flux_difference(U, ca, Fa, sc, ida_hi, ida_lo);
    if (Fb) sub_flux_difference(U, cb, Fb, sc, idb_hi, idb_lo);
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      U[c] = U[c] - ca * (Fa[c * sc + ida_hi] - Fa[c * sc + ida_lo]);
      if (Fb) U[c] = U[c] - cb * (Fb[c * sc + idb_hi] - Fb[c * sc + idb_lo]);
    }
  }
  state_from_cons(U, K, s);
}

// ---- stage 4b (3-D): intermediate fluxes F^{d|t}
template <int D, int T, bool EINF>
__device__ __forceinline__ void flux2_item(ScratchGeom sg, const double* __restrict__ TP,
                                                 const double* __restrict__ TM, const double* __restrict__ F1t,
                                                 double* __restrict__ F2, StepConst K, Range R, long long t) {
  int i, j, k;
  if (!range_zone(R, t, i, j, k)) return;
  const long long sd = (D == 0) ? 1 : (D == 1) ? sg.sy : sg.sz;
  const long long stt = (T == 0) ? 1 : (T == 1) ? sg.sy : sg.sz;
  const long long id = sg.id(i, j, k), zl = id - sd;
  const double coef = K.dtdx[T] * THIRD;
  double sL[NS], sR[NS], F[5];
  correct<false>(TP, zl, K, coef, F1t, sg.sc, zl + stt, zl, 0.0, nullptr, 0, 0, sL);
  correct<false>(TM, id, K, coef, F1t, sg.sc, id + stt, id, 0.0, nullptr, 0, 0, sR);
  hllc_flux<EINF>(sL, sR, D, K, F);
  store5(F2, sg.sc, id, F);
}

// ---- stage 4c: final fluxes from fully corrected states
// 2-D: Fa = F1 of the other axis, Fb = null; 3-D: Fa = F^{t1|t2}, Fb = F^{t2|t1}
template <int D, bool EINF>
__device__ __forceinline__ void flux3_item(ScratchGeom sg, const double* __restrict__ TP,
                                                 const double* __restrict__ TM, const double* __restrict__ Fa,
                                                 const double* __restrict__ Fb, double* __restrict__ F3,
                                                 StepConst K, Range R, long long t) {
  int i, j, k;
  if (!range_zone(R, t, i, j, k)) return;
  constexpr int T1 = (D == 0) ? 1 : 0, T2 = (D == 2) ? 1 : 2;
  const long long sd = (D == 0) ? 1 : (D == 1) ? sg.sy : sg.sz;
  const long long s1 = (T1 == 0) ? 1 : (T1 == 1) ? sg.sy : sg.sz;
  const long long s2 = (T2 == 0) ? 1 : (T2 == 1) ? sg.sy : sg.sz;
  const long long id = sg.id(i, j, k), zl = id - sd;
  const double ca = 0.5 * K.dtdx[T1], cb = 0.5 * K.dtdx[T2];
  double sL[NS], sR[NS], F[5];
  correct<true>(TP, zl, K, ca, Fa, sg.sc, zl + s1, zl, cb, Fb, zl + s2, zl, sL);
  correct<true>(TM, id, K, ca, Fa, sg.sc, id + s1, id, cb, Fb, id + s2, id, sR);
  hllc_flux<EINF>(sL, sR, D, K, F);
  store5(F3, sg.sc, id, F);
}

// block-wide max of three non-negative doubles, then one atomicMax per value
__device__ __forceinline__ void block_max3(double v[3], DevFlags* flags) {
  __shared__ double red[3][BLOCK / 32];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double x = v[a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = dmax_nn(x, __shfl_xor_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) red[a][threadIdx.x >> 5] = x;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double x = red[threadIdx.x][0];
    for (int w = 1; w < BLOCK / 32; ++w) x = dmax_nn(x, red[threadIdx.x][w]);
    if (gt0(x)) atomicMax(&flags->maxspeed[threadIdx.x], (unsigned long long)__double_as_longlong(x));
  }
}

// ---- stage 5: conservative update, gravity source, bad-state check, CFL partials
__device__ __forceinline__ void update_item(BoxGeom in, BoxGeom out, ScratchGeom sg, const double* __restrict__ Fx,
                                                  const double* __restrict__ Fy, const double* __restrict__ Fz,
                                                  StepConst K, Range R, DevFlags* flags, long long t) {
  int i, j, k;
  double spd[3] = {0.0, 0.0, 0.0};
  if (range_zone(R, t, i, j, k)) {
    const long long ii = in.id(i, j, k), oi = out.id(i, j, k), id = sg.id(i, j, k);
    const double* F[3] = {Fx, Fy, Fz};
    const long long st[3] = {1, sg.sy, sg.sz};
    double u0[5], u1[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) u0[c] = in.u[c * in.sc + ii];
#pragma unroll
    for (int c = 0; c < 5; ++c) u1[c] = u0[c];
    // direction by direction, each component in the order d = 0, 1, 2
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (d < K.dim) sub_flux_difference(u1, K.dtdx[d], F[d], sg.sc, id + st[d], id);
    if (K.has_grav) {
      double rho_mid = dhalf(u0[0] + u1[0]);
      const double dtr = mul_i(K.dt, rho_mid);
#pragma unroll
      for (int a = 0; a < 3; ++a) u1[1 + a] = u1[1 + a] + dtr * K.grav[a];
      double e[3];
      if (K.flux_grav) {
        // mass-flux form: gravity's work on the mass crossing the zone's faces
#pragma unroll
        for (int d = 0; d < 3; ++d)
          e[d] = (d < K.dim) ? mul_i(dhalf(F[d][id] + F[d][id + st[d]]), K.grav[d]) : 0.0;
      } else {
        e[0] = mul_i(dhalf(u0[1] + u1[1]), K.grav[0]);
        e[1] = dhalf(u0[2] + u1[2]) * K.grav[1];
        e[2] = dhalf(u0[3] + u1[3]) * K.grav[2];
      }
      u1[4] = u1[4] + K.dt * ((e[0] + e[1]) + e[2]);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) out.u[c * out.sc + oi] = u1[c];
    double q[5], inv;
    bool bad = false;
    cons_to_prim_flag(u1, K, q, &inv, &bad);
    if (bad) atomicOr(&flags->bad, 1);
    double c = dsqrt(mul_i(mul_i(K.gamma, q[4]), inv));
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (d < K.dim) spd[d] = fabs(q[1 + d]) + c;
  }
  block_max3(spd, flags);
}

// ---- CFL estimate of an existing box (interior)
__device__ __forceinline__ void dt_partial_item(BoxGeom box, StepConst K, Range R, DevFlags* flags, long long t) {
  int i, j, k;
  double spd[3] = {0.0, 0.0, 0.0};
  if (range_zone(R, t, i, j, k)) {
    long long id = box.id(i, j, k);
    double U[5], q[5], inv;
#pragma unroll
    for (int c = 0; c < 5; ++c) U[c] = box.u[c * box.sc + id];
    bool bad = false;
    cons_to_prim_flag(U, K, q, &inv, &bad);
    if (bad) atomicOr(&flags->bad, 1);
    double c = dsqrt(mul_i(mul_i(K.gamma, q[4]), inv));
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (d < K.dim) spd[d] = fabs(q[1 + d]) + c;
  }
  block_max3(spd, flags);
}

// dt = cfl * min_d dx_d / max_zones(|u_d| + c): equal to cfl * min over zones
// and d of dx_d/(|u_d| + c) because a correctly rounded quotient is monotone
// in its denominator
__device__ __forceinline__ void dt_final_item(DevFlags* flags, double dx0, double dx1, double dx2, int dim,
                                              double cfl) {
  double dx[3] = {dx0, dx1, dx2};
  double m = HUGE_VAL;
  for (int d = 0; d < dim; ++d) {
    double s = __longlong_as_double((long long)flags->maxspeed[d]);
    m = dmin(m, dx[d] / s);
  }
  flags->dt_next = cfl * m;
}

}  // namespace
}  // namespace hydro
