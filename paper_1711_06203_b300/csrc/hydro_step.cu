// Kernels of the staged CTU-PPM step and their launch sequence.
#include "hydro_step.cuh"

namespace hydro {

namespace {

constexpr int BLOCK = 128;

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
__global__ void __launch_bounds__(BLOCK) k_prim(BoxGeom in, ScratchGeom sg, double* __restrict__ Q, StepConst K,
                                                Range R, DevFlags* flags) {
  int i, j, k;
  if (!range_zone(R, (long long)blockIdx.x * BLOCK + threadIdx.x, i, j, k)) return;
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
  double c = sqrt(K.gamma * q[4] * inv);
  long long id = sg.id(i, j, k);
#pragma unroll
  for (int v = 0; v < 5; ++v) Q[v * sg.sc + id] = q[v];
  Q[QC * sg.sc + id] = c;
  Q[QRC * sg.sc + id] = q[0] / c;
  Q[QCR * sg.sc + id] = c / q[0];
  Q[QIC2 * sg.sc + id] = 1.0 / (c * c);
}

// ---- stage 3 of a zone: characteristic tracing from its parabolas
// am/ap/a6/zone: (rho, un, ut1, ut2, p); outputs the zone's low- and high-face
// states to TM/TP at id in absolute component order.
template <int D>
__device__ __forceinline__ void trace_zone(const double am[5], const double ap[5], const double a6[5],
                                           const double zone[5], double c, double rho_c, double c_rho,
                                           double inv_c2, const StepConst& K, double* __restrict__ TM,
                                           double* __restrict__ TP, long long sc, long long id) {
  constexpr int T1 = (D == 0) ? 1 : 0, T2 = (D == 2) ? 1 : 2;
  const double un = zone[1];
  const double c2 = c * c;
  const double lu = 0.5 * rho_c, lp = 0.5 * inv_c2;
  const double lam[3] = {un - c, un, un + c};
  double sig[3];
#pragma unroll
  for (int w = 0; w < 3; ++w) sig[w] = fabs(lam[w]) * K.dtdx[D];
#pragma unroll
  for (int side = 0; side < 2; ++side) {
    bool reach[3];
#pragma unroll
    for (int w = 0; w < 3; ++w) reach[w] = side ? gt0(lam[w]) : lt0(lam[w]);
    const int fast = side ? 2 : 0;
    auto I = [&](int w, int v) {
      return side ? integ_plus(am[v], ap[v], a6[v], sig[w]) : integ_minus(am[v], ap[v], a6[v], sig[w]);
    };
    double ref[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) ref[v] = reach[fast] ? I(fast, v) : zone[v];
    // the reference wave contributes exactly zero (ref - I(sigma_fast) == 0), so
    // only the other acoustic wave and the entropy/shear wave are evaluated
    double bm = 0.0, b0 = 0.0, bp = 0.0, bt1 = 0.0, bt2 = 0.0;
    if (side == 1 && reach[0]) bm = -lu * (ref[1] - I(0, 1)) + lp * (ref[4] - I(0, 4));
    if (reach[1]) {
      b0 = (ref[0] - I(1, 0)) - inv_c2 * (ref[4] - I(1, 4));
      bt1 = ref[2] - I(1, 2);
      bt2 = ref[3] - I(1, 3);
    }
    if (side == 0 && reach[2]) bp = lu * (ref[1] - I(2, 1)) + lp * (ref[4] - I(2, 4));
    double s_rho = ref[0] - ((bm + b0) + bp);
    double s_un = ref[1] - (bm * (-c_rho) + bp * c_rho);
    double s_p = ref[4] - (bm * c2 + bp * c2);
    double s_t1 = ref[2] - bt1, s_t2 = ref[3] - bt2;
    s_un = s_un + K.hdt * K.grav[D];
    s_t1 = s_t1 + K.hdt * K.grav[T1];
    s_t2 = s_t2 + K.hdt * K.grav[T2];
    s_rho = dmax(s_rho, K.small_dens);
    s_p = dmax(s_p, K.small_pres);
    double* out = side ? TP : TM;
    out[0 * sc + id] = s_rho;
    out[(1 + D) * sc + id] = s_un;
    out[(1 + T1) * sc + id] = s_t1;
    out[(1 + T2) * sc + id] = s_t2;
    out[4 * sc + id] = s_p;
  }
}

// pencil segments of the tracing sweep: zones [-1, n_d] along d cut into
// segments of TRACE_SEG, for every transverse position in [-1, n]
constexpr int TRACE_SEG = 16;
struct SweepRange {
  int lo1, ext1, lo2, ext2;  // transverse axes T1 (thread-fastest) and T2
  int nd, nseg;              // zones along d, segments per pencil
  __host__ __device__ long long count() const { return (long long)ext1 * ext2 * nseg; }
};

// ---- stages 2-3: flattening, PPM reconstruction and characteristic tracing
// along d.  Each thread sweeps one pencil segment, so every flattening
// coefficient, slope and interface value is formed once per zone (plus a
// two-zone warm-up per segment) from sliding register windows.
template <int D>
__global__ void __launch_bounds__(BLOCK) k_trace(ScratchGeom sg, const double* __restrict__ Q,
                                                 double* __restrict__ TM, double* __restrict__ TP, StepConst K,
                                                 SweepRange R) {
  long long t = (long long)blockIdx.x * BLOCK + threadIdx.x;
  if (t >= R.count()) return;
  constexpr int T1 = (D == 0) ? 1 : 0, T2 = (D == 2) ? 1 : 2;
  int c3[3];
  c3[T1] = R.lo1 + (int)(t % R.ext1);
  long long r = t / R.ext1;
  c3[T2] = R.lo2 + (int)(r % R.ext2);
  const int seg = (int)(r / R.ext2);
  const int i0 = -1 + seg * TRACE_SEG;
  const int i1 = min(i0 + TRACE_SEG, R.nd + 1);
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
  double a0[5], a1[5], sl[5], fm[5];
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
      double s_m1 = mc_slope(am2[v], am1[v], a0[v]);
      sl[v] = mc_slope(am1[v], a0[v], a1[v]);
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
  for (int i = i0; i < i1; ++i) {
    const long long id = base + (long long)(i - i0) * st;
    double a2[5];
#pragma unroll
    for (int v = 0; v < 4; ++v) a2[v] = qv[v][id + 2 * st];
    a2[4] = pp2;
    double chi = 1.0, ctp = 1.0, pp3 = 0.0;
    if (K.flatten) {
      pp3 = qv[4][id + 3 * st];
      ctp = flat_tilde(pm1, a0[4], a2[4], pp3, a0[1], a2[1], sp);
      double dp1 = a1[4] - pm1;
      chi = lt0(dp1) ? dmin(ct0, ctp) : dmin(ct0, ctm);
    }
    double am[5], ap[5], a6[5], zone[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      double s1 = mc_slope(a0[v], a1[v], a2[v]);
      double fp = face_value(a0[v], a1[v], sl[v], s1);
      ppm_limit(a0[v], fm[v], fp, chi, am[v], ap[v], a6[v]);
      zone[v] = a0[v];
      sl[v] = s1;
      fm[v] = fp;
    }
    trace_zone<D>(am, ap, a6, zone, Q[QC * sc + id], Q[QRC * sc + id], Q[QCR * sc + id], Q[QIC2 * sc + id], K,
                  TM, TP, sc, id);
    // slide the windows one zone
    pm2 = pm1;
    pm1 = a0[4];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
      a0[v] = a1[v];
      a1[v] = a2[v];
    }
    if (K.flatten) pp2 = pp3;
    else if (i + 1 < i1) pp2 = qv[4][id + 3 * st];
    ctm = ct0;
    ct0 = ctp;
  }
}

__device__ __forceinline__ void load5(const double* __restrict__ A, long long sc, long long id, double v[5]) {
#pragma unroll
  for (int c = 0; c < 5; ++c) v[c] = A[c * sc + id];
}
__device__ __forceinline__ void store5(double* __restrict__ A, long long sc, long long id, const double v[5]) {
#pragma unroll
  for (int c = 0; c < 5; ++c) A[c * sc + id] = v[c];
}

// ---- stage 4a: first Riemann solves from the traced states
template <int D>
__global__ void __launch_bounds__(BLOCK) k_flux1(ScratchGeom sg, const double* __restrict__ TP,
                                                 const double* __restrict__ TM, double* __restrict__ F1, StepConst K,
                                                 Range R) {
  int i, j, k;
  if (!range_zone(R, (long long)blockIdx.x * BLOCK + threadIdx.x, i, j, k)) return;
  const long long st = (D == 0) ? 1 : (D == 1) ? sg.sy : sg.sz;
  const long long id = sg.id(i, j, k);
  double qL[5], qR[5], sL[NS], sR[NS], F[5];
  load5(TP, sg.sc, id - st, qL);
  load5(TM, sg.sc, id, qR);
  state_from_prim(qL, K, sL);
  state_from_prim(qR, K, sR);
  hllc_flux(sL, sR, D, K, F);
  store5(F1, sg.sc, id, F);
}

// transverse correction of a traced primitive state by one or two flux differences
__device__ __forceinline__ void correct(const double q[5], const StepConst& K, double ca, const double* Fa,
                                        long long sc, long long ida_hi, long long ida_lo, double cb,
                                        const double* Fb, long long idb_hi, long long idb_lo, double s[NS]) {
  double U[5];
  U[0] = q[0];
  U[1] = q[0] * q[1];
  U[2] = q[0] * q[2];
  U[3] = q[0] * q[3];
  U[4] = energy_of(q, K);
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    U[c] = U[c] - ca * (Fa[c * sc + ida_hi] - Fa[c * sc + ida_lo]);
    if (Fb) U[c] = U[c] - cb * (Fb[c * sc + idb_hi] - Fb[c * sc + idb_lo]);
  }
  state_from_cons(U, K, s);
}

// ---- stage 4b (3-D): intermediate fluxes F^{d|t}
template <int D, int T>
__global__ void __launch_bounds__(BLOCK) k_flux2(ScratchGeom sg, const double* __restrict__ TP,
                                                 const double* __restrict__ TM, const double* __restrict__ F1t,
                                                 double* __restrict__ F2, StepConst K, Range R) {
  int i, j, k;
  if (!range_zone(R, (long long)blockIdx.x * BLOCK + threadIdx.x, i, j, k)) return;
  const long long sd = (D == 0) ? 1 : (D == 1) ? sg.sy : sg.sz;
  const long long stt = (T == 0) ? 1 : (T == 1) ? sg.sy : sg.sz;
  const long long id = sg.id(i, j, k), zl = id - sd;
  const double coef = K.dtdx[T] * THIRD;
  double qL[5], qR[5], sL[NS], sR[NS], F[5];
  load5(TP, sg.sc, zl, qL);
  load5(TM, sg.sc, id, qR);
  correct(qL, K, coef, F1t, sg.sc, zl + stt, zl, 0.0, nullptr, 0, 0, sL);
  correct(qR, K, coef, F1t, sg.sc, id + stt, id, 0.0, nullptr, 0, 0, sR);
  hllc_flux(sL, sR, D, K, F);
  store5(F2, sg.sc, id, F);
}

// ---- stage 4c: final fluxes from fully corrected states
// 2-D: Fa = F1 of the other axis, Fb = null; 3-D: Fa = F^{t1|t2}, Fb = F^{t2|t1}
template <int D>
__global__ void __launch_bounds__(BLOCK) k_flux3(ScratchGeom sg, const double* __restrict__ TP,
                                                 const double* __restrict__ TM, const double* __restrict__ Fa,
                                                 const double* __restrict__ Fb, double* __restrict__ F3,
                                                 StepConst K, Range R) {
  int i, j, k;
  if (!range_zone(R, (long long)blockIdx.x * BLOCK + threadIdx.x, i, j, k)) return;
  constexpr int T1 = (D == 0) ? 1 : 0, T2 = (D == 2) ? 1 : 2;
  const long long sd = (D == 0) ? 1 : (D == 1) ? sg.sy : sg.sz;
  const long long s1 = (T1 == 0) ? 1 : (T1 == 1) ? sg.sy : sg.sz;
  const long long s2 = (T2 == 0) ? 1 : (T2 == 1) ? sg.sy : sg.sz;
  const long long id = sg.id(i, j, k), zl = id - sd;
  const double ca = 0.5 * K.dtdx[T1], cb = 0.5 * K.dtdx[T2];
  double qL[5], qR[5], sL[NS], sR[NS], F[5];
  load5(TP, sg.sc, zl, qL);
  load5(TM, sg.sc, id, qR);
  correct(qL, K, ca, Fa, sg.sc, zl + s1, zl, cb, Fb, zl + s2, zl, sL);
  correct(qR, K, ca, Fa, sg.sc, id + s1, id, cb, Fb, id + s2, id, sR);
  hllc_flux(sL, sR, D, K, F);
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
__global__ void __launch_bounds__(BLOCK) k_update(BoxGeom in, BoxGeom out, ScratchGeom sg, const double* __restrict__ Fx,
                                                  const double* __restrict__ Fy, const double* __restrict__ Fz,
                                                  StepConst K, Range R, DevFlags* flags) {
  int i, j, k;
  double spd[3] = {0.0, 0.0, 0.0};
  if (range_zone(R, (long long)blockIdx.x * BLOCK + threadIdx.x, i, j, k)) {
    const long long ii = in.id(i, j, k), oi = out.id(i, j, k), id = sg.id(i, j, k);
    const double* F[3] = {Fx, Fy, Fz};
    const long long st[3] = {1, sg.sy, sg.sz};
    double u0[5], u1[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) u0[c] = in.u[c * in.sc + ii];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      double v = u0[c];
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (d < K.dim) v = v - K.dtdx[d] * (F[d][c * sg.sc + id + st[d]] - F[d][c * sg.sc + id]);
      u1[c] = v;
    }
    if (K.has_grav) {
      double rho_mid = 0.5 * (u0[0] + u1[0]);
#pragma unroll
      for (int a = 0; a < 3; ++a) u1[1 + a] = u1[1 + a] + K.dt * rho_mid * K.grav[a];
      double e0 = 0.5 * (u0[1] + u1[1]) * K.grav[0];
      double e1 = 0.5 * (u0[2] + u1[2]) * K.grav[1];
      double e2 = 0.5 * (u0[3] + u1[3]) * K.grav[2];
      u1[4] = u1[4] + K.dt * ((e0 + e1) + e2);
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) out.u[c * out.sc + oi] = u1[c];
    double q[5], inv;
    bool bad = false;
    cons_to_prim_flag(u1, K, q, &inv, &bad);
    if (bad) atomicOr(&flags->bad, 1);
    double c = sqrt(K.gamma * q[4] * inv);
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (d < K.dim) spd[d] = fabs(q[1 + d]) + c;
  }
  block_max3(spd, flags);
}

// ---- CFL estimate of an existing box (interior)
__global__ void __launch_bounds__(BLOCK) k_dt_partial(BoxGeom box, StepConst K, Range R, DevFlags* flags) {
  int i, j, k;
  double spd[3] = {0.0, 0.0, 0.0};
  if (range_zone(R, (long long)blockIdx.x * BLOCK + threadIdx.x, i, j, k)) {
    long long id = box.id(i, j, k);
    double U[5], q[5], inv;
#pragma unroll
    for (int c = 0; c < 5; ++c) U[c] = box.u[c * box.sc + id];
    bool bad = false;
    cons_to_prim_flag(U, K, q, &inv, &bad);
    if (bad) atomicOr(&flags->bad, 1);
    double c = sqrt(K.gamma * q[4] * inv);
#pragma unroll
    for (int d = 0; d < 3; ++d)
      if (d < K.dim) spd[d] = fabs(q[1 + d]) + c;
  }
  block_max3(spd, flags);
}

// dt = cfl * min_d dx_d / max_zones(|u_d| + c): equal to cfl * min over zones
// and d of dx_d/(|u_d| + c) because a correctly rounded quotient is monotone
// in its denominator
__global__ void k_dt_final(DevFlags* flags, double dx0, double dx1, double dx2, int dim, double cfl) {
  double dx[3] = {dx0, dx1, dx2};
  double m = HUGE_VAL;
  for (int d = 0; d < dim; ++d) {
    double s = __longlong_as_double((long long)flags->maxspeed[d]);
    m = dmin(m, dx[d] / s);
  }
  flags->dt_next = cfl * m;
}

__global__ void k_reset_speed(DevFlags* flags) {
  if (threadIdx.x < 3) flags->maxspeed[threadIdx.x] = 0ull;
}

inline unsigned blocks_for(long long n) { return (unsigned)((n + BLOCK - 1) / BLOCK); }

}  // namespace

cudaError_t launch_step(const StepArgs& a, cudaStream_t st, long long* launches) {
  const int dim = a.K.dim;
  long long nl = 0;
  auto mark = [&](int stage) {
    if (a.events) cudaEventRecord(a.events[stage], st);
  };
  mark(ST_PRIM);
  const int* n = a.in.n;
  const ScratchGeom& sg = a.sg;
  const Scratch& s = a.s;
  // stage 1: primitive state on the grown box
  Range rp;
  for (int ax = 0; ax < 3; ++ax) {
    int g = (ax < 2 || dim == 3) ? NG : 0;
    rp.lo[ax] = -g;
    rp.ext[ax] = n[ax] + 2 * g;
  }
  k_prim<<<blocks_for(rp.count()), BLOCK, 0, st>>>(a.in, sg, s.Q, a.K, rp, a.flags);
  nl += 1;
  mark(ST_TRACE);
  // stages 2-3: traced states on zones [-1, n] (pencil sweeps)
  Range rt;
  for (int ax = 0; ax < 3; ++ax) {
    bool act = ax < dim;
    rt.lo[ax] = act ? -1 : 0;
    rt.ext[ax] = act ? n[ax] + 2 : 1;
  }
  for (int d = 0; d < dim; ++d) {
    int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
    SweepRange sw;
    sw.lo1 = rt.lo[t1]; sw.ext1 = rt.ext[t1];
    sw.lo2 = rt.lo[t2]; sw.ext2 = rt.ext[t2];
    sw.nd = n[d];
    sw.nseg = (n[d] + 2 + TRACE_SEG - 1) / TRACE_SEG;
    unsigned b = blocks_for(sw.count());
    if (d == 0) k_trace<0><<<b, BLOCK, 0, st>>>(sg, s.Q, s.TM[0], s.TP[0], a.K, sw);
    if (d == 1) k_trace<1><<<b, BLOCK, 0, st>>>(sg, s.Q, s.TM[1], s.TP[1], a.K, sw);
    if (d == 2) k_trace<2><<<b, BLOCK, 0, st>>>(sg, s.Q, s.TM[2], s.TP[2], a.K, sw);
  }
  nl += dim;
  mark(ST_FLUX1);
  // stage 4a: first fluxes on d-faces [0, n_d] x transverse [-1, n]
  for (int d = 0; d < dim; ++d) {
    Range r = rt;
    r.lo[d] = 0;
    r.ext[d] = n[d] + 1;
    unsigned b = blocks_for(r.count());
    if (d == 0) k_flux1<0><<<b, BLOCK, 0, st>>>(sg, s.TP[0], s.TM[0], s.F1[0], a.K, r);
    if (d == 1) k_flux1<1><<<b, BLOCK, 0, st>>>(sg, s.TP[1], s.TM[1], s.F1[1], a.K, r);
    if (d == 2) k_flux1<2><<<b, BLOCK, 0, st>>>(sg, s.TP[2], s.TM[2], s.F1[2], a.K, r);
    nl += 1;
  }
  mark(ST_FLUX2);
  // stage 4b (3-D): intermediate fluxes F^{d|t}
  if (dim == 3) {
    for (int d = 0; d < 3; ++d)
      for (int t = 0; t < 3; ++t) {
        if (t == d) continue;
        int o = 3 - d - t;
        Range r;
        r.lo[d] = 0; r.ext[d] = n[d] + 1;
        r.lo[t] = 0; r.ext[t] = n[t];
        r.lo[o] = -1; r.ext[o] = n[o] + 2;
        unsigned b = blocks_for(r.count());
        const double* f1 = s.F1[t];
        double* f2 = s.F2[d][t];
#define F2CASE(DD, TT) \
  if (d == DD && t == TT) k_flux2<DD, TT><<<b, BLOCK, 0, st>>>(sg, s.TP[DD], s.TM[DD], f1, f2, a.K, r);
        F2CASE(0, 1) F2CASE(0, 2) F2CASE(1, 0) F2CASE(1, 2) F2CASE(2, 0) F2CASE(2, 1)
#undef F2CASE
        nl += 1;
      }
  }
  mark(ST_FLUX3);
  // stage 4c: final fluxes on d-faces [0, n_d] x transverse interior
  for (int d = 0; d < dim; ++d) {
    Range r;
    for (int ax = 0; ax < 3; ++ax) { r.lo[ax] = 0; r.ext[ax] = (ax < dim) ? n[ax] : 1; }
    r.ext[d] = n[d] + 1;
    unsigned b = blocks_for(r.count());
    int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
    const double* fa = (dim == 2) ? s.F1[t1] : s.F2[t1][t2];
    const double* fb = (dim == 2) ? nullptr : s.F2[t2][t1];
    if (d == 0) k_flux3<0><<<b, BLOCK, 0, st>>>(sg, s.TP[0], s.TM[0], fa, fb, s.F3[0], a.K, r);
    if (d == 1) k_flux3<1><<<b, BLOCK, 0, st>>>(sg, s.TP[1], s.TM[1], fa, fb, s.F3[1], a.K, r);
    if (d == 2) k_flux3<2><<<b, BLOCK, 0, st>>>(sg, s.TP[2], s.TM[2], fa, fb, s.F3[2], a.K, r);
    nl += 1;
  }
  mark(ST_UPDATE);
  // stage 5: update + CFL partials
  k_reset_speed<<<1, 32, 0, st>>>(a.flags);
  Range ru;
  for (int ax = 0; ax < 3; ++ax) { ru.lo[ax] = 0; ru.ext[ax] = (ax < dim) ? n[ax] : 1; }
  k_update<<<blocks_for(ru.count()), BLOCK, 0, st>>>(a.in, a.out, sg, s.F3[0], s.F3[1], dim == 3 ? s.F3[2] : s.F3[0],
                                                     a.K, ru, a.flags);
  k_dt_final<<<1, 1, 0, st>>>(a.flags, a.dx[0], a.dx[1], a.dx[2], dim, a.cfl);
  nl += 3;
  mark(NSTAGES);
  if (launches) *launches += nl;
  return cudaGetLastError();
}

cudaError_t launch_dt(const BoxGeom& box, const StepConst& K, const double dx[3], double cfl, DevFlags* flags,
                      cudaStream_t st, long long* launches) {
  Range ru;
  for (int ax = 0; ax < 3; ++ax) { ru.lo[ax] = 0; ru.ext[ax] = (ax < K.dim) ? box.n[ax] : 1; }
  k_reset_speed<<<1, 32, 0, st>>>(flags);
  k_dt_partial<<<blocks_for(ru.count()), BLOCK, 0, st>>>(box, K, ru, flags);
  k_dt_final<<<1, 1, 0, st>>>(flags, dx[0], dx[1], dx[2], K.dim, cfl);
  if (launches) *launches += 3;
  return cudaGetLastError();
}

}  // namespace hydro
