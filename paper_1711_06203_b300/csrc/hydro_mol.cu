// Method-of-lines hydro step with passive species (FP64, sm_103a).
//
// Sec. 4: StarLord, the GPU proxy of Castro, keeps only the hydrodynamics and
// the EOS, writes the hydrodynamics as a simple method of lines and advects 13
// nuclear species.  Its scheme is not printed; this is the method-of-lines
// reading of the CTU path's building blocks:
//   dU/dt = L(U) = -sum_d (F_d(face hi) - F_d(face lo)) / dx_d + S(U),
//   F_d = HLLC of the flattened, limited PPM edge values of the primitive
//   variables (rho, u, v, w, p, X_k) at the stage time (no characteristic
//   tracing, no transverse terms); the species flux is the mass flux times the
//   mass fraction of the HLLC upwind side; S = (0, rho g, (rho u).g);
//   two-stage SSP Runge-Kutta: U1 = U + dt L(U), U' = U/2 + (U1 + dt L(U1))/2.
//
// Kernels of one stage (all FP64-issue bound, like the CTU path):
//   km_prim      grown box: stage state -> (rho, u, v, w, p, X_k); ghosts by
//                boundary map (prefilled layers from the caller's input box)
//   km_flat<d>   zones [-1, n_d] x interior: flattening coefficient
//   km_recon<d>  (y, z) one thread per (variable, pencil segment): a
//                sliding-window sweep forms each slope, interface value and
//                limited edge once
//   km_recon_x   (x) one warp per (variable, row, run of 28 zones), lanes
//                along x: the same operations per zone, neighbours' values
//                by warp shuffles, loads and stores coalesced
//   km_flux<d>   faces [0, n_d] x interior: HLLC + species upwinding (per wave-speed choice)
//   km_update    interior: flux differences x, y, z, source, stage combination,
//                bad-state check and CFL partials (second stage)
// Scratch (grown-box fields): Q, EM, EP, U1 (nf = 5 + nspec each), F (3 nf),
// CHI (1): 7 nf + 1 fields.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "hydro.h"
#include "hydro_api_internal.cuh"
#include "hydro_items.cuh"

using namespace hydro;

namespace hydro {
namespace {

constexpr int MOL_SEG = 16;  // zones per reconstruction sweep segment
constexpr int XRUN = 28;     // zones per warp of the x reconstruction (32 lanes less a 2-zone halo each side)

struct MolScratch {
  double* Q;     // nf fields
  double* CHI;   // 1 field
  double* EM;    // nf fields: edge value at each zone's low face
  double* EP;    // nf fields: edge value at each zone's high face
  double* F[3];  // nf fields per direction, face f stored at zone f
  double* U1;    // nf fields: first-stage state (interior)
};

struct MolArgs {
  BoxGeom in, out, u1;  // u1: the first-stage state in scratch (scratch strides)
  ScratchGeom sg;
  MolScratch s;
  StepConst K;
  int nf;
  double dx[3];
  double cfl;
  DevFlags* flags;
};

template <int D>
__device__ __forceinline__ long long axis_stride(const ScratchGeom& sg) {
  return (D == 0) ? 1 : (D == 1) ? sg.sy : sg.sz;
}

// ---- stage state -> primitive variables on the grown box
__global__ void __launch_bounds__(BLOCK) km_prim(BoxGeom src, BoxGeom pre, ScratchGeom sg, double* __restrict__ Q,
                                                 int nf, StepConst K, Range R, DevFlags* flags) {
  int i, j, k;
  if (!range_zone(R, (long long)blockIdx.x * BLOCK + threadIdx.x, i, j, k)) return;
  bool flip[3] = {false, false, false};
  int c[3] = {i, j, k};
  c[0] = map_axis(i, src.n[0], src.bc[0][0], src.bc[0][1], flip[0]);
  c[1] = map_axis(j, src.n[1], src.bc[1][0], src.bc[1][1], flip[1]);
  if (K.dim == 3) c[2] = map_axis(k, src.n[2], src.bc[2][0], src.bc[2][1], flip[2]);
  // a coordinate left outside the interior lies in a prefilled ghost layer:
  // caller data at t^n, read from the input box in every stage
  bool ghost = false;
  for (int a = 0; a < K.dim; ++a) ghost |= (c[a] < 0 || c[a] >= src.n[a]);
  const BoxGeom& B = ghost ? pre : src;
  const long long si = B.id(c[0], c[1], c[2]);
  double U[5];
#pragma unroll
  for (int m = 0; m < 5; ++m) U[m] = B.u[m * B.sc + si];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (flip[a]) U[1 + a] = -U[1 + a];
  double q[5], inv;
  bool bad = false;
  cons_to_prim_flag(U, K, q, &inv, &bad);
  if (bad) atomicOr(&flags->bad, 1);
  const long long id = sg.id(i, j, k);
#pragma unroll
  for (int v = 0; v < 5; ++v) Q[v * sg.sc + id] = q[v];
  for (int v = 5; v < nf; ++v) Q[v * sg.sc + id] = mul_i(B.u[v * B.sc + si], inv);
}

// ---- flattening coefficient of zones [-1, n_d] (interior transverse)
template <int D>
__global__ void __launch_bounds__(BLOCK) km_flat(ScratchGeom sg, const double* __restrict__ Q,
                                                 double* __restrict__ CHI, StepConst K, Range R) {
  int i, j, k;
  if (!range_zone(R, (long long)blockIdx.x * BLOCK + threadIdx.x, i, j, k)) return;
  const long long id = sg.id(i, j, k), st = axis_stride<D>(sg);
  const double* p = Q + QP * sg.sc + id;
  const double* un = Q + (QU + D) * sg.sc + id;
  double chi = 1.0;
  if (K.flatten) {
    // the neighbour on the low-pressure side (p_{i+1} - p_{i-1} < 0 as an order comparison)
    const long long s = dless(p[st], p[-st]) ? st : -st;
    const double c0 = flat_tilde(p[-2 * st], p[-st], p[st], p[2 * st], un[-st], un[st], K.small_pres);
    const double c1 = flat_tilde(p[s - 2 * st], p[s - st], p[s + st], p[s + 2 * st], un[s - st], un[s + st],
                                 K.small_pres);
    chi = dmin(c0, c1);
  }
  CHI[id] = chi;
}

// ---- limited PPM edges of one variable along a pencil segment (y and z sweeps)
// item t: t1 (fastest), t2, segment, variable
template <int D>
__global__ void __launch_bounds__(BLOCK) km_recon(ScratchGeom sg, const double* __restrict__ Q,
                                                  const double* __restrict__ CHI, double* __restrict__ EM,
                                                  double* __restrict__ EP, int n1, int n2, int nd, int nseg, int nf) {
  long long t = (long long)blockIdx.x * BLOCK + threadIdx.x;
  const long long total = (long long)n1 * n2 * nseg * nf;
  if (t >= total) return;
  constexpr int T1 = (D == 0) ? 1 : 0, T2 = (D == 2) ? 1 : 2;
  const int p1 = (int)(t % n1);
  t /= n1;
  const int p2 = (int)(t % n2);
  t /= n2;
  const int seg = (int)(t % nseg);
  const int v = (int)(t / nseg);
  const int z0 = -1 + seg * MOL_SEG;
  const int z1 = min(nd + 1, z0 + MOL_SEG);  // zones [z0, z1) of [-1, nd]
  int c[3] = {0, 0, 0};
  c[T1] = p1;
  c[T2] = p2;
  c[D] = 0;
  const long long st = axis_stride<D>(sg);
  const long long base = sg.id(c[0], c[1], c[2]);
  const double* a = Q + (long long)v * sg.sc + base;
  // window a[m-2 .. m+2] for zone m, slopes s[m], s[m+1], interface value m-1/2
  double am2 = a[(z0 - 2) * st], am1 = a[(z0 - 1) * st], a0 = a[z0 * st], ap1 = a[(z0 + 1) * st];
  const double dm = am1 - am2, d0 = a0 - am1;
  double d01 = ap1 - a0;  // one-sided difference a_{m+1} - a_m, carried along the segment
  double s0 = mc_slope_d(d0, d01, am1, ap1);
  const double sm1 = mc_slope_d(dm, d0, am2, a0);
  double fm = face_value(am1, a0, sm1, s0);  // interface z0 - 1/2
  // each zone's new operands (a_{m+2}, chi_m) are loaded one zone ahead
  double nap2 = a[(z0 + 2) * st], nchi = CHI[base + z0 * st];
  for (int m = z0; m < z1; ++m) {
    const double ap2 = nap2, chi = nchi;
    if (m + 1 < z1) {
      nap2 = a[(m + 3) * st];
      nchi = CHI[base + (m + 1) * st];
    }
    const double d12 = ap2 - ap1;
    const double s1 = mc_slope_d(d01, d12, a0, ap2);
    d01 = d12;
    const double fp = face_value(a0, ap1, s0, s1);  // interface m + 1/2
    double lo, hi, a6;
    ppm_limit(a0, fm, fp, chi, lo, hi, a6);
    const long long o = (long long)v * sg.sc + base + m * st;
    EM[o] = lo;
    EP[o] = hi;
    a0 = ap1;
    ap1 = ap2;
    s0 = s1;
    fm = fp;
  }
}

// ---- limited PPM edges along x with lanes along x.  A thread per pencil
// (km_recon<0>) makes every load of a warp hit 32 rows; here warp w of a
// (variable, row) takes output zones [z0, z0 + XRUN) and lane l holds zone
// z0 - 2 + l.  Each lane forms its zone's left difference, slope, high
// interface value and limited edges; a lane takes its neighbours' values by
// shuffle (a zone's slope needs a_{m-1}, a_{m+1} and the next difference,
// its interface m + 1/2 the next slope, its low interface the previous
// lane's high one).  Lanes 2..29 hold complete stencils and store.  The
// operations and operands per zone are those of the sweep, so the edges are
// bitwise the same.
__global__ void __launch_bounds__(BLOCK) km_recon_x(ScratchGeom sg, const double* __restrict__ Q,
                                                    const double* __restrict__ CHI, double* __restrict__ EM,
                                                    double* __restrict__ EP, int n1, int n2, int nd, int nrun,
                                                    int nf) {
  const long long w = ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5;  // the same for the whole warp
  const int lane = threadIdx.x & 31;
  if (w >= (long long)n1 * n2 * nrun * nf) return;
  long long r = w;
  const int run = (int)(r % nrun);
  r /= nrun;
  const int j = (int)(r % n1);
  r /= n1;
  const int k = (int)(r % n2);
  const int v = (int)(r / n2);
  const int z0 = -1 + run * XRUN;        // first output zone; outputs are zones [-1, nd]
  const int m = z0 - 2 + lane;           // this lane's zone
  const int mr = min(m, nd + 3);         // lanes past the grown box read its last zone (never stored)
  const long long id = sg.id(mr, j, k);
  const double a = Q[(long long)v * sg.sc + id];
  const double chi = CHI[id];
  const unsigned all = 0xffffffffu;
  const double am1 = __shfl_up_sync(all, a, 1), ap1 = __shfl_down_sync(all, a, 1);
  const double dl = a - am1;                              // a_m - a_{m-1}
  const double dr = __shfl_down_sync(all, dl, 1);         // a_{m+1} - a_m
  const double s0 = mc_slope_d(dl, dr, am1, ap1);         // slope of zone m
  const double s1 = __shfl_down_sync(all, s0, 1);         // slope of zone m + 1
  const double fp = face_value(a, ap1, s0, s1);           // interface m + 1/2
  const double fm = __shfl_up_sync(all, fp, 1);           // interface m - 1/2
  if (lane >= 2 && lane < 2 + XRUN && m <= nd) {
    double lo, hi, a6;
    ppm_limit(a, fm, fp, chi, lo, hi, a6);
    const long long o = (long long)v * sg.sc + id;
    EM[o] = lo;
    EP[o] = hi;
  }
}

// ---- HLLC fluxes through d-faces [0, n_d] (interior transverse)
template <int D, bool EINF>  // EINF: Einfeldt outer wave speeds (K.einfeldt set), else Davis
__global__ void __launch_bounds__(BLOCK) km_flux(ScratchGeom sg, const double* __restrict__ EM,
                                                 const double* __restrict__ EP, double* __restrict__ F, int nf,
                                                 StepConst K, Range R) {
  int i, j, k;
  if (!range_zone(R, (long long)blockIdx.x * BLOCK + threadIdx.x, i, j, k)) return;
  const long long id = sg.id(i, j, k), zl = id - axis_stride<D>(sg);
  double qL[5], qR[5], sL[NS], sR[NS], Fh[5];
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    qL[v] = EP[v * sg.sc + zl];
    qR[v] = EM[v * sg.sc + id];
  }
  state_from_prim(qL, K, sL);
  state_from_prim(qR, K, sR);
  const bool left = hllc_flux<EINF>(sL, sR, D, K, Fh);
#pragma unroll
  for (int c = 0; c < 5; ++c) F[c * sg.sc + id] = Fh[c];
  for (int v = 5; v < nf; ++v) {
    const double x = left ? EP[v * sg.sc + zl] : EM[v * sg.sc + id];
    F[v * sg.sc + id] = mul_i(Fh[0], x);
  }
}

// ---- stage update.  stage 0: U1 = W + dt L(W) into scratch;
// stage 1: out = W0/2 + (U1 + dt L(U1))/2, bad-state check, CFL partials
__global__ void __launch_bounds__(BLOCK) km_update(BoxGeom w0, BoxGeom ws, BoxGeom dst, ScratchGeom sg,
                                                   const double* __restrict__ Fx, const double* __restrict__ Fy,
                                                   const double* __restrict__ Fz, int nf, StepConst K, Range R,
                                                   int second, DevFlags* flags) {
  int i, j, k;
  double spd[3] = {0.0, 0.0, 0.0};
  if (range_zone(R, (long long)blockIdx.x * BLOCK + threadIdx.x, i, j, k)) {
    const long long is = ws.id(i, j, k), id = sg.id(i, j, k), od = dst.id(i, j, k);
    const double* F[3] = {Fx, Fy, Fz};
    const long long st[3] = {1, sg.sy, sg.sz};
    double hyd[5];
    for (int c = 0; c < nf; ++c) {
      double v = ws.u[c * ws.sc + is];
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (d < K.dim) v = v - K.dtdx[d] * (F[d][c * sg.sc + id + st[d]] - F[d][c * sg.sc + id]);
      if (K.has_grav && c >= 1 && c <= 4) {
        const double rho = ws.u[is];
        if (c <= 3) {
          v = v + K.dt * rho * K.grav[c - 1];
        } else {
          const double e = (ws.u[1 * ws.sc + is] * K.grav[0] + ws.u[2 * ws.sc + is] * K.grav[1]) +
                           ws.u[3 * ws.sc + is] * K.grav[2];
          v = v + K.dt * e;
        }
      }
      if (second) v = dhalf(w0.u[c * w0.sc + w0.id(i, j, k)]) + dhalf(v);
      dst.u[c * dst.sc + od] = v;
      if (c < 5) hyd[c] = v;
    }
    if (second) {
      double q[5], inv;
      bool bad = false;
      cons_to_prim_flag(hyd, K, q, &inv, &bad);
      if (bad) atomicOr(&flags->bad, 1);
      const double cs = dsqrt(mul_i(mul_i(K.gamma, q[4]), inv));
#pragma unroll
      for (int d = 0; d < 3; ++d)
        if (d < K.dim) spd[d] = fabs(q[1 + d]) + cs;
    }
  }
  if (second) block_max3(spd, flags);
}

__global__ void km_reset(DevFlags* flags) {
  if (threadIdx.x < 3) flags->maxspeed[threadIdx.x] = 0ull;
}

__global__ void km_dt_final(DevFlags* flags, double dx0, double dx1, double dx2, int dim, double cfl) {
  dt_final_item(flags, dx0, dx1, dx2, dim, cfl);
}

inline unsigned blocks_of(long long n) { return (unsigned)((n + BLOCK - 1) / BLOCK); }

cudaError_t launch_mol_stage(const MolArgs& a, int second, cudaStream_t st, long long* nl) {
  const int dim = a.K.dim;
  const int* n = a.in.n;
  const BoxGeom& src = second ? a.u1 : a.in;
  Range rp;
  for (int ax = 0; ax < 3; ++ax) {
    const int g = (ax < 2 || dim == 3) ? NG : 0;
    rp.lo[ax] = -g;
    rp.ext[ax] = n[ax] + 2 * g;
  }
  km_prim<<<blocks_of(rp.count()), BLOCK, 0, st>>>(src, a.in, a.sg, a.s.Q, a.nf, a.K, rp, a.flags);
  *nl += 1;
  for (int d = 0; d < dim; ++d) {
    const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
    Range rf;  // zones [-1, n_d] along d, interior transverse
    for (int ax = 0; ax < 3; ++ax) {
      rf.lo[ax] = 0;
      rf.ext[ax] = (ax < dim) ? n[ax] : 1;
    }
    rf.lo[d] = -1;
    rf.ext[d] = n[d] + 2;
    if (d == 0) km_flat<0><<<blocks_of(rf.count()), BLOCK, 0, st>>>(a.sg, a.s.Q, a.s.CHI, a.K, rf);
    if (d == 1) km_flat<1><<<blocks_of(rf.count()), BLOCK, 0, st>>>(a.sg, a.s.Q, a.s.CHI, a.K, rf);
    if (d == 2) km_flat<2><<<blocks_of(rf.count()), BLOCK, 0, st>>>(a.sg, a.s.Q, a.s.CHI, a.K, rf);
    const int n1 = n[t1], n2 = (t2 < dim) ? n[t2] : 1;
    const int nseg = (n[d] + 2 + MOL_SEG - 1) / MOL_SEG;
    const long long items = (long long)n1 * n2 * nseg * a.nf;
    if (d == 0) {
      const int nrun = (n[0] + 2 + XRUN - 1) / XRUN;
      const long long threads = (long long)n1 * n2 * nrun * a.nf * 32;
      km_recon_x<<<blocks_of(threads), BLOCK, 0, st>>>(a.sg, a.s.Q, a.s.CHI, a.s.EM, a.s.EP, n1, n2, n[0], nrun, a.nf);
    }
    if (d == 1) km_recon<1><<<blocks_of(items), BLOCK, 0, st>>>(a.sg, a.s.Q, a.s.CHI, a.s.EM, a.s.EP, n1, n2, n[1], nseg, a.nf);
    if (d == 2) km_recon<2><<<blocks_of(items), BLOCK, 0, st>>>(a.sg, a.s.Q, a.s.CHI, a.s.EM, a.s.EP, n1, n2, n[2], nseg, a.nf);
    Range rx;  // faces [0, n_d] along d, interior transverse
    for (int ax = 0; ax < 3; ++ax) {
      rx.lo[ax] = 0;
      rx.ext[ax] = (ax < dim) ? n[ax] : 1;
    }
    rx.ext[d] = n[d] + 1;
    const unsigned g = blocks_of(rx.count());
    if (a.K.einfeldt) {
      if (d == 0) km_flux<0, true><<<g, BLOCK, 0, st>>>(a.sg, a.s.EM, a.s.EP, a.s.F[0], a.nf, a.K, rx);
      if (d == 1) km_flux<1, true><<<g, BLOCK, 0, st>>>(a.sg, a.s.EM, a.s.EP, a.s.F[1], a.nf, a.K, rx);
      if (d == 2) km_flux<2, true><<<g, BLOCK, 0, st>>>(a.sg, a.s.EM, a.s.EP, a.s.F[2], a.nf, a.K, rx);
    } else {
      if (d == 0) km_flux<0, false><<<g, BLOCK, 0, st>>>(a.sg, a.s.EM, a.s.EP, a.s.F[0], a.nf, a.K, rx);
      if (d == 1) km_flux<1, false><<<g, BLOCK, 0, st>>>(a.sg, a.s.EM, a.s.EP, a.s.F[1], a.nf, a.K, rx);
      if (d == 2) km_flux<2, false><<<g, BLOCK, 0, st>>>(a.sg, a.s.EM, a.s.EP, a.s.F[2], a.nf, a.K, rx);
    }
    *nl += 3;
  }
  Range ru;
  for (int ax = 0; ax < 3; ++ax) {
    ru.lo[ax] = 0;
    ru.ext[ax] = (ax < dim) ? n[ax] : 1;
  }
  const BoxGeom& dst = second ? a.out : a.u1;
  km_update<<<blocks_of(ru.count()), BLOCK, 0, st>>>(a.in, src, dst, a.sg, a.s.F[0], a.s.F[1],
                                                     dim == 3 ? a.s.F[2] : a.s.F[0], a.nf, a.K, ru, second, a.flags);
  *nl += 1;
  return cudaGetLastError();
}

// extent in doubles of a box with nf components
long long mol_span(const hydro_box_t* b, int dim, int nf) {
  const long long gz = (dim == 3) ? b->n[2] + 2 * NG : 1;
  return (long long)(nf - 1) * b->stride[2] + (gz - 1) * b->stride[1] + (b->n[1] + 2 * NG - 1) * b->stride[0] +
         b->n[0] + 2 * NG;
}

}  // namespace
}  // namespace hydro

extern "C" int hydro_mol_advance_box(hydro_ctx_t* ctx, const hydro_box_t* in, const hydro_box_t* out,
                                     const hydro_params_t* params, int nspec, double dt, double* dt_next_host,
                                     void* stream) {
  if (!ctx || !valid_params(params) || nspec < 0 || nspec > HYDRO_MOL_MAX_SPECIES) return HYDRO_EINVAL;
  if (params->flags & HYDRO_FLAG_FLUX_GRAV_ENERGY) return HYDRO_ENOTIMPL;
  const int dim = params->dim, nf = 5 + nspec;
  if (!valid_box(in, dim) || !out || !out->u || out->ng != NG) return HYDRO_EINVAL;
  if (reinterpret_cast<uintptr_t>(out->u) % sizeof(double)) return HYDRO_EINVAL;
  hydro_box_t o = *out;
  for (int a = 0; a < 3; ++a) {
    if (out->n[a] != in->n[a]) return HYDRO_EINVAL;
    o.dx[a] = in->dx[a];
    o.bc[a][0] = o.bc[a][1] = HYDRO_BC_PREFILLED;
  }
  if (!valid_box(&o, dim)) return HYDRO_EINVAL;
  {
    const double *a0 = in->u, *a1 = in->u + mol_span(in, dim, nf);
    const double *b0 = out->u, *b1 = out->u + mol_span(out, dim, nf);
    if (a0 < b1 && b0 < a1) return HYDRO_EINVAL;  // in and out overlap
  }
  if (!(dt > 0.0) || !std::isfinite(dt)) return HYDRO_EINVAL;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return HYDRO_ECUDA;
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return HYDRO_ECUDA;
  struct Restore {
    int dev, prev;
    ~Restore() { if (prev >= 0 && prev != dev) cudaSetDevice(prev); }
  } restore{ctx->device, prev};
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  MolArgs a;
  a.in = geom_of(in, dim);
  a.out = geom_of(out, dim);
  a.sg = scratch_geom(in->n, dim);
  a.nf = nf;
  const size_t fields = 7 * (size_t)nf + 1;
  int rc = ensure_scratch(ctx, (size_t)a.sg.sc * fields * sizeof(double));
  if (rc) return rc;
  double* p = ctx->scratch;
  auto take = [&](int k) { double* r = p; p += (long long)k * a.sg.sc; return r; };
  a.s.Q = take(nf);
  a.s.CHI = take(1);
  a.s.EM = take(nf);
  a.s.EP = take(nf);
  for (int d = 0; d < 3; ++d) a.s.F[d] = take(nf);
  a.s.U1 = take(nf);
  a.u1 = a.in;  // same n and boundary kinds, scratch strides
  a.u1.u = a.s.U1;
  a.u1.sy = a.sg.sy;
  a.u1.sz = a.sg.sz;
  a.u1.sc = a.sg.sc;
  a.K = step_const(params, in->dx, dt);
  for (int d = 0; d < 3; ++d) a.dx[d] = in->dx[d];
  a.cfl = params->cfl;
  a.flags = ctx->flags;
  long long nl = 0;
  km_reset<<<1, 32, 0, st>>>(ctx->flags);
  nl += 1;
  cudaError_t ce = launch_mol_stage(a, 0, st, &nl);
  if (ce == cudaSuccess) ce = launch_mol_stage(a, 1, st, &nl);
  if (ce == cudaSuccess) {
    km_dt_final<<<1, 1, 0, st>>>(ctx->flags, a.dx[0], a.dx[1], a.dx[2], dim, a.cfl);
    nl += 1;
    ce = cudaGetLastError();
  }
  ctx->launches += nl;
  if (ce != cudaSuccess) return HYDRO_ECUDA;
  if (dt_next_host) {
    DevFlags h;
    rc = read_flags(ctx, st, &h);
    if (rc) return rc;
    *dt_next_host = h.dt_next;
    if (h.bad) return HYDRO_EBADSTATE;
  }
  return HYDRO_OK;
}
