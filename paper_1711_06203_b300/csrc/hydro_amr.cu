// Two-level subcycled advance with flux registers (refinement ratio 2).
//
// Sec. 3: the suite rests on block-structured AMR with subcycling in time;
// Sec. 4: Castro advances a coarse level, then the finer level in several
// smaller steps until it reaches the same time, then synchronises the levels.
// The synchronisation is the Berger-Colella one:
//   1. coarse level: ghost fill (domain boundary kinds) and one batched step
//      of dt; the coarse fluxes through the coarse-fine interface faces are
//      copied from the step's scratch into a register;
//   2. fine level, twice: ghost fill (copy from a fine neighbour, else
//      interpolation from the coarse level at the substep's start -- time
//      first, then MC-limited linear in space) and a batched step of dt/2;
//      the fine fluxes through the interface faces are summed into a second
//      register;
//   3. reflux: every uncovered coarse zone at the interface has each of its
//      interface faces' coarse flux replaced by the area- and time-averaged
//      fine flux;
//   4. average down: every covered coarse zone becomes the mean of its 2^dim
//      fine children;
//   5. next step: min(CFL step of the synchronised coarse level, 2 x CFL step
//      of the fine level), left on the device.
// The batched steps are the product kernels; the kernels here are small
// gathers and scatters over ghost layers and interfaces.  Their arithmetic
// uses explicitly rounded operations in a fixed order, so the interface
// work is bitwise reproducible in every build.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <map>
#include <new>
#include <numeric>
#include <tuple>
#include <vector>

#include "hydro.h"
#include "hydro_api_internal.cuh"
#include "hydro_batch.cuh"
#include "hydro_items.cuh"

using namespace hydro;

namespace hydro {
namespace {

constexpr int RATIO = 2;
constexpr int MAX_AMR_PLANS = 4;

struct ACoarse {
  BoxGeom in, out;  // state at t (ghosts filled), state at t + dt
  int lo[3];
  Range interior;
};

struct AFine {
  BoxGeom a[3];     // state at t, after the first substep (library-owned), at t + dt
  int lo[3];        // fine index space
  long long grown;  // zones of the grown box
  long long czones; // coarse zones the box covers
};

// one coarse-fine interface face, seen from the uncovered coarse zone
struct AFace {
  int cb, ci[3];    // coarse box holding the uncovered zone; face position in it
  int fb, fi[3];    // fine box on the covered side; position of its first fine face
  int d, side;      // axis; -1 the zone's low face, +1 its high face
};

// an uncovered coarse zone with interface faces faces[f0 .. f0 + nf)
struct AZone {
  int cb, zi[3];
  int f0, nf;
};

struct AmrGeom {
  int dim;
  int Gc, cc[3];    // coarse owner map: cell size and extent
  int Gf, cf[3];    // fine owner map (fine index space, -1 = not covered)
  double dx[3];     // coarse spacing
};

__device__ __forceinline__ int owner_cell(int G, const int c[3], int x, int y, int z) {
  return ((z / G) * c[1] + y / G) * c[0] + x / G;
}

// the coarse state at zone X at the start of a fine substep: U(t), or
// 0.5 U(t) + 0.5 U(t + dt)
__device__ __forceinline__ void coarse_at(const ACoarse* __restrict__ C, const int* __restrict__ own,
                                          const AmrGeom& A, const int X[3], int half, double u[5]) {
  const ACoarse& c = C[own[owner_cell(A.Gc, A.cc, X[0], X[1], X[2])]];
  const int i = X[0] - c.lo[0], j = X[1] - c.lo[1], k = X[2] - c.lo[2];
  const long long io = c.in.id(i, j, k);
#pragma unroll
  for (int m = 0; m < 5; ++m) u[m] = c.in.u[m * c.in.sc + io];
  if (half) {
    const long long in = c.out.id(i, j, k);
#pragma unroll
    for (int m = 0; m < 5; ++m) u[m] = __dadd_rn(__dmul_rn(0.5, u[m]), __dmul_rn(0.5, c.out.u[m * c.out.sc + in]));
  }
}

// monotonised-central slope: 0 unless both one-sided differences are non-zero
// with one sign, else min(2|dl|, 2|dr|, |dl + dr| / 2) with that sign
__device__ __forceinline__ double mc_interp_slope(double ul, double u0, double ur) {
  const double dl = __dsub_rn(u0, ul), dr = __dsub_rn(ur, u0);
  const bool same = (dl > 0.0 && dr > 0.0) || (dl < 0.0 && dr < 0.0);
  const double m = fmin(fmin(2.0 * fabs(dl), 2.0 * fabs(dr)), 0.5 * fabs(__dadd_rn(dl, dr)));
  return same ? copysign(m, dl) : 0.0;
}

__global__ void ka_prep(const double* __restrict__ dt_dev, double* __restrict__ dtc, int nc, double* __restrict__ dtf,
                        int nf, DevFlags* lvl, DevFlags* ctx_flags) {
  const double dt = dt_dev[0];
  for (int b = threadIdx.x; b < nc; b += blockDim.x) dtc[b] = dt;
  for (int b = threadIdx.x; b < nf; b += blockDim.x) dtf[b] = 0.5 * dt;
  if (threadIdx.x == 0) {
    lvl->maxspeed[0] = lvl->maxspeed[1] = lvl->maxspeed[2] = 0ull;
    lvl->bad = 0;
    ctx_flags->bad = 0;
  }
}

// every ghost zone of every fine box of one stage (0: state at t, 1: after
// the first substep): a copy from the fine box that covers it, else the
// coarse interpolant
__global__ void __launch_bounds__(BLOCK) ka_fill(const AFine* __restrict__ F, const ACoarse* __restrict__ C,
                                                 const int* __restrict__ own_c, const int* __restrict__ own_f,
                                                 const int* __restrict__ blk_box, const int* __restrict__ box_first,
                                                 AmrGeom A, int stage, int half) {
  const int b = blk_box[blockIdx.x];
  const AFine& B = F[b];
  const long long t = (long long)(blockIdx.x - box_first[b]) * BLOCK + threadIdx.x;
  if (t >= B.grown) return;
  const BoxGeom& G = B.a[stage];
  const int gx = G.n[0] + 2 * NG, gy = G.n[1] + 2 * NG;
  int c[3];
  c[0] = (int)(t % gx) - NG;
  c[1] = (int)((t / gx) % gy) - NG;
  c[2] = (A.dim == 3) ? (int)(t / ((long long)gx * gy)) - NG : 0;
  bool ghost = false;
  for (int a = 0; a < A.dim; ++a) ghost |= (c[a] < 0 || c[a] >= G.n[a]);
  if (!ghost) return;
  const int g[3] = {B.lo[0] + c[0], B.lo[1] + c[1], (A.dim == 3) ? B.lo[2] + c[2] : 0};
  double v[5];
  const int o = own_f[owner_cell(A.Gf, A.cf, g[0], g[1], g[2])];
  if (o >= 0) {
    const AFine& O = F[o];
    const BoxGeom& OG = O.a[stage];
    const long long s = OG.id(g[0] - O.lo[0], g[1] - O.lo[1], g[2] - O.lo[2]);
#pragma unroll
    for (int m = 0; m < 5; ++m) v[m] = OG.u[m * OG.sc + s];
  } else {
    const int P[3] = {g[0] >> 1, g[1] >> 1, g[2] >> 1};
    double u0[5];
    coarse_at(C, own_c, A, P, half, u0);
#pragma unroll
    for (int m = 0; m < 5; ++m) v[m] = u0[m];
    for (int d = 0; d < A.dim; ++d) {
      int Pl[3] = {P[0], P[1], P[2]}, Pr[3] = {P[0], P[1], P[2]};
      Pl[d] -= 1;
      Pr[d] += 1;
      double ul[5], ur[5];
      coarse_at(C, own_c, A, Pl, half, ul);
      coarse_at(C, own_c, A, Pr, half, ur);
      const double off = (g[d] & 1) ? 0.25 : -0.25;  // child centre relative to the parent's, coarse units
#pragma unroll
      for (int m = 0; m < 5; ++m) v[m] = __dadd_rn(v[m], __dmul_rn(mc_interp_slope(ul[m], u0[m], ur[m]), off));
    }
  }
  const long long dst = G.id(c[0], c[1], c[2]);
#pragma unroll
  for (int m = 0; m < 5; ++m) G.u[m * G.sc + dst] = v[m];
}

// coarse register: the coarse step's final flux through each interface face
__global__ void ka_reg_coarse(const BatchBox* __restrict__ P, const AFace* __restrict__ faces, int nface,
                              double* __restrict__ reg_c) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 5LL * nface) return;
  const int f = (int)(t % nface), m = (int)(t / nface);
  const AFace& E = faces[f];
  const BatchBox& B = P[E.cb];
  reg_c[t] = B.s.F3[E.d][m * B.sg.sc + B.sg.id(E.ci[0], E.ci[1], E.ci[2])];
}

// fine register: add one substep's final fluxes through the 2^(dim-1) fine
// faces under each interface face (second transverse axis outer)
__global__ void ka_reg_fine(const BatchBox* __restrict__ P, const AFace* __restrict__ faces, int nface, int dim,
                            double* __restrict__ reg_f, int first) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 5LL * nface) return;
  const int f = (int)(t % nface), m = (int)(t / nface);
  const AFace& E = faces[f];
  const BatchBox& B = P[E.fb];
  const int t1 = (E.d == 0) ? 1 : 0, t2 = (E.d == 2) ? 1 : 2;
  const double* Fd = B.s.F3[E.d] + (long long)m * B.sg.sc;
  double acc = first ? 0.0 : reg_f[t];
  for (int o2 = 0; o2 < ((dim == 3) ? 2 : 1); ++o2)
    for (int o1 = 0; o1 < 2; ++o1) {
      int p[3] = {E.fi[0], E.fi[1], E.fi[2]};
      p[t1] += o1;
      if (dim == 3) p[t2] += o2;
      acc = __dadd_rn(acc, Fd[B.sg.id(p[0], p[1], p[2])]);
    }
  reg_f[t] = acc;
}

// reflux: U += (-+ dt/dx_d) (w * fine sum - coarse flux), faces in order
__global__ void ka_reflux(const ACoarse* __restrict__ C, const AZone* __restrict__ Z, int nz,
                          const AFace* __restrict__ faces, int nface, const double* __restrict__ reg_c,
                          const double* __restrict__ reg_f, const double* __restrict__ dt_dev, AmrGeom A) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 5LL * nz) return;
  const int z = (int)(t % nz), m = (int)(t / nz);
  const AZone& R = Z[z];
  const BoxGeom& O = C[R.cb].out;
  const long long id = m * O.sc + O.id(R.zi[0], R.zi[1], R.zi[2]);
  const double w = (A.dim == 3) ? 0.125 : 0.25;  // 1 / (2^(dim-1) fine faces x 2 substeps)
  const double dt = dt_dev[0];
  double u = O.u[id];
  for (int q = 0; q < R.nf; ++q) {
    const int f = R.f0 + q;
    const AFace& E = faces[f];
    const double dtdx = __ddiv_rn(dt, A.dx[E.d]);
    const double s = (E.side > 0) ? -dtdx : dtdx;
    const double delta = __dsub_rn(__dmul_rn(reg_f[(long long)m * nface + f], w), reg_c[(long long)m * nface + f]);
    u = __dadd_rn(u, __dmul_rn(s, delta));
  }
  O.u[id] = u;
}

// average down: each covered coarse zone = (sum of its children) x 2^-dim,
// children summed z outer, then y, then x
__global__ void __launch_bounds__(BLOCK) ka_avgdown(const AFine* __restrict__ F, const ACoarse* __restrict__ C,
                                                    const int* __restrict__ own_c, const int* __restrict__ blk_box,
                                                    const int* __restrict__ box_first, AmrGeom A) {
  const int b = blk_box[blockIdx.x];
  const AFine& B = F[b];
  const long long t = (long long)(blockIdx.x - box_first[b]) * BLOCK + threadIdx.x;
  if (t >= B.czones) return;
  const BoxGeom& G = B.a[2];
  const int ncx = G.n[0] / RATIO, ncy = G.n[1] / RATIO;
  const int I = (int)(t % ncx), J = (int)((t / ncx) % ncy), K = (A.dim == 3) ? (int)(t / ((long long)ncx * ncy)) : 0;
  double s[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int oz = 0; oz < ((A.dim == 3) ? 2 : 1); ++oz)
    for (int oy = 0; oy < 2; ++oy)
      for (int ox = 0; ox < 2; ++ox) {
        const long long id = G.id(RATIO * I + ox, RATIO * J + oy, (A.dim == 3) ? RATIO * K + oz : 0);
#pragma unroll
        for (int m = 0; m < 5; ++m) s[m] = __dadd_rn(s[m], G.u[m * G.sc + id]);
      }
  const double w = (A.dim == 3) ? 0.125 : 0.25;
  const int X[3] = {B.lo[0] / RATIO + I, B.lo[1] / RATIO + J, (A.dim == 3) ? B.lo[2] / RATIO + K : 0};
  const ACoarse& c = C[own_c[owner_cell(A.Gc, A.cc, X[0], X[1], X[2])]];
  const long long id = c.out.id(X[0] - c.lo[0], X[1] - c.lo[1], X[2] - c.lo[2]);
#pragma unroll
  for (int m = 0; m < 5; ++m) c.out.u[m * c.out.sc + id] = __dmul_rn(s[m], w);
}

// CFL partials of the synchronised coarse level
__global__ void __launch_bounds__(BLOCK) ka_dt_partial(const ACoarse* __restrict__ C, const int* __restrict__ blk_box,
                                                       const int* __restrict__ box_first, StepConst K, DevFlags* lvl) {
  const int b = blk_box[blockIdx.x];
  const ACoarse& c = C[b];
  dt_partial_item(c.out, K, c.interior, lvl, (long long)(blockIdx.x - box_first[b]) * BLOCK + threadIdx.x);
}

__global__ void ka_dt_final(DevFlags* lvl, const double* __restrict__ dtn_f, int nf, AmrGeom A, double cfl,
                            double* __restrict__ dt_next) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  dt_final_item(lvl, A.dx[0], A.dx[1], A.dx[2], A.dim, cfl);
  double m = lvl->dt_next;
  for (int b = 0; b < nf; ++b) m = dmin(m, 2.0 * dtn_f[b]);
  dt_next[0] = m;
}

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
  return h;
}

unsigned blocks_of(long long items, unsigned bs) { return (unsigned)((items + bs - 1) / bs); }

// block -> box map of a launch over per-box item counts
void block_map(const std::vector<long long>& items, std::vector<int>& first, std::vector<int>& blk) {
  first.assign(items.size(), 0);
  blk.clear();
  for (size_t b = 0; b < items.size(); ++b) {
    first[b] = (int)blk.size();
    blk.insert(blk.end(), blocks_of(items[b], BLOCK), (int)b);
  }
}

struct Carve {
  std::vector<std::pair<const void*, size_t>> parts;
  size_t total = 0;
  size_t add(const void* p, size_t bytes) {
    size_t off = total;
    parts.push_back({p, bytes});
    total += (bytes + 255) & ~size_t(255);
    return off;
  }
};

}  // namespace
}  // namespace hydro

struct AmrPlan {
  uint64_t key = 0;
  uint64_t last_use = 0;
  int nc = 0, nf = 0, nface = 0, nzone = 0;
  AmrGeom A{};
  char* mem = nullptr;
  ACoarse* C = nullptr;
  AFine* F = nullptr;
  AFace* faces = nullptr;
  AZone* zones = nullptr;
  int *own_c = nullptr, *own_f = nullptr;
  int *fill_blk = nullptr, *fill_first = nullptr;
  int *avg_blk = nullptr, *avg_first = nullptr;
  int *dt_blk = nullptr, *dt_first = nullptr;
  unsigned fill_nb = 0, avg_nb = 0, dt_nb = 0;
  double *reg_c = nullptr, *reg_f = nullptr;
  double *dtc = nullptr, *dtnc = nullptr, *dtf = nullptr, *dtnf = nullptr;
  DevFlags* lvl = nullptr;
  // host descriptors handed to the fill and the batched steps
  std::vector<hydro_box_t> c_in, c_out, f_in, f_tmp, f_out;
  std::vector<int> c_lo;
};

struct hydro_amr_state {
  std::vector<AmrPlan*> plans;
  double* tmp = nullptr;  // the fine level after its first substep
  size_t tmp_bytes = 0;
  uint64_t clock = 0;
};

namespace hydro {
namespace {

void destroy_amr_plan(AmrPlan* p) {
  if (!p) return;
  if (p->mem) cudaFree(p->mem);
  delete p;
}

hydro_box_t prefilled(hydro_box_t b) {
  for (int a = 0; a < 3; ++a) b.bc[a][0] = b.bc[a][1] = HYDRO_BC_PREFILLED;
  return b;
}

// Checks the hierarchy and builds its plan (host tables + one device block).
int build_plan(const hydro_amr_t* h, double* tmp_pool, AmrPlan* P) {
  const int dim = h->dim, nc = h->ncoarse, nf = h->nfine;
  AmrGeom& A = P->A;
  std::memset(&A, 0, sizeof A);
  A.dim = dim;
  int dom[3];
  for (int a = 0; a < 3; ++a) dom[a] = (a < dim) ? h->domain[a] : 1;
  for (int a = 0; a < 3; ++a) A.dx[a] = h->coarse_in[0].dx[a];
  // coarse owner map
  int G = 0;
  for (int a = 0; a < dim; ++a) G = std::gcd(G, dom[a]);
  for (int b = 0; b < nc; ++b)
    for (int a = 0; a < dim; ++a) G = std::gcd(G, std::gcd(h->coarse_lo[3 * b + a], h->coarse_in[b].n[a]));
  A.Gc = G;
  for (int a = 0; a < 3; ++a) A.cc[a] = (a < dim) ? dom[a] / G : 1;
  const long long ncell_c = (long long)A.cc[0] * A.cc[1] * A.cc[2];
  if (ncell_c > (1LL << 27)) return HYDRO_EINVAL;
  std::vector<int> own_c(ncell_c, -1);
  for (int b = 0; b < nc; ++b) {
    int c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
      c0[a] = (a < dim) ? h->coarse_lo[3 * b + a] / G : 0;
      c1[a] = (a < dim) ? (h->coarse_lo[3 * b + a] + h->coarse_in[b].n[a]) / G : 1;
    }
    for (int k = c0[2]; k < c1[2]; ++k)
      for (int j = c0[1]; j < c1[1]; ++j)
        for (int i = c0[0]; i < c1[0]; ++i) {
          int& o = own_c[((long long)k * A.cc[1] + j) * A.cc[0] + i];
          if (o != -1) return HYDRO_EINVAL;
          o = b;
        }
  }
  for (int o : own_c)
    if (o < 0) return HYDRO_EINVAL;
  // fine owner map over the refined domain
  int Gf = 0;
  for (int a = 0; a < dim; ++a) Gf = std::gcd(Gf, RATIO * dom[a]);
  for (int b = 0; b < nf; ++b)
    for (int a = 0; a < dim; ++a) Gf = std::gcd(Gf, std::gcd(h->fine_lo[3 * b + a], h->fine_in[b].n[a]));
  A.Gf = Gf;
  for (int a = 0; a < 3; ++a) A.cf[a] = (a < dim) ? RATIO * dom[a] / Gf : 1;
  const long long ncell_f = (long long)A.cf[0] * A.cf[1] * A.cf[2];
  if (ncell_f > (1LL << 27)) return HYDRO_EINVAL;
  std::vector<int> own_f(ncell_f, -1);
  for (int b = 0; b < nf; ++b) {
    int c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
      c0[a] = (a < dim) ? h->fine_lo[3 * b + a] / Gf : 0;
      c1[a] = (a < dim) ? (h->fine_lo[3 * b + a] + h->fine_in[b].n[a]) / Gf : 1;
    }
    for (int k = c0[2]; k < c1[2]; ++k)
      for (int j = c0[1]; j < c1[1]; ++j)
        for (int i = c0[0]; i < c1[0]; ++i) {
          int& o = own_f[((long long)k * A.cf[1] + j) * A.cf[0] + i];
          if (o != -1) return HYDRO_EINVAL;  // fine boxes overlap
          o = b;
        }
  }
  auto fine_owner = [&](int x, int y, int z) { return own_f[((long long)(z / Gf) * A.cf[1] + y / Gf) * A.cf[0] + x / Gf]; };
  auto coarse_owner = [&](int x, int y, int z) { return own_c[((long long)(z / G) * A.cc[1] + y / G) * A.cc[0] + x / G]; };
  auto covered = [&](int X, int Y, int Z) { return fine_owner(RATIO * X, RATIO * Y, RATIO * Z) >= 0; };

  // host descriptors
  P->c_in.resize(nc);
  P->c_out.resize(nc);
  P->f_in.resize(nf);
  P->f_tmp.resize(nf);
  P->f_out.resize(nf);
  P->c_lo.assign(h->coarse_lo, h->coarse_lo + 3 * nc);
  std::vector<ACoarse> C(nc);
  std::vector<long long> dt_items(nc);
  for (int b = 0; b < nc; ++b) {
    P->c_in[b] = prefilled(h->coarse_in[b]);
    P->c_out[b] = prefilled(h->coarse_out[b]);
    C[b].in = geom_of(&P->c_in[b], dim);
    C[b].out = geom_of(&P->c_out[b], dim);
    for (int a = 0; a < 3; ++a) {
      C[b].lo[a] = (a < dim) ? h->coarse_lo[3 * b + a] : 0;
      C[b].interior.lo[a] = 0;
      C[b].interior.ext[a] = (a < dim) ? h->coarse_in[b].n[a] : 1;
    }
    dt_items[b] = C[b].interior.count();
  }
  std::vector<AFine> F(nf);
  std::vector<long long> fill_items(nf), avg_items(nf);
  size_t toff = 0;
  for (int b = 0; b < nf; ++b) {
    const hydro_box_t& fb = h->fine_in[b];
    const long long gx = fb.n[0] + 2 * NG, gy = fb.n[1] + 2 * NG, gz = (dim == 3) ? fb.n[2] + 2 * NG : 1;
    hydro_box_t t = fb;
    t.u = tmp_pool + toff;
    t.stride[0] = gx;
    t.stride[1] = gx * gy;
    t.stride[2] = gx * gy * gz;
    toff += (size_t)(5 * gx * gy * gz + 31) & ~size_t(31);
    P->f_in[b] = prefilled(fb);
    P->f_tmp[b] = prefilled(t);
    P->f_out[b] = prefilled(h->fine_out[b]);
    F[b].a[0] = geom_of(&P->f_in[b], dim);
    F[b].a[1] = geom_of(&P->f_tmp[b], dim);
    F[b].a[2] = geom_of(&P->f_out[b], dim);
    for (int a = 0; a < 3; ++a) F[b].lo[a] = (a < dim) ? h->fine_lo[3 * b + a] : 0;
    F[b].grown = gx * gy * gz;
    F[b].czones = (long long)(fb.n[0] / RATIO) * (fb.n[1] / RATIO) * ((dim == 3) ? fb.n[2] / RATIO : 1);
    fill_items[b] = F[b].grown;
    avg_items[b] = F[b].czones;
  }

  // interface faces, grouped by uncovered coarse zone (row-major, x fastest),
  // each zone's faces in the order x-low, x-high, y-low, y-high, z-low, z-high
  std::map<std::tuple<int, int, int>, int> zone_mask;  // key (z, y, x) -> bit (2d + (side > 0))
  for (int b = 0; b < nf; ++b) {
    int c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
      c0[a] = (a < dim) ? F[b].lo[a] / RATIO : 0;
      c1[a] = (a < dim) ? (F[b].lo[a] + h->fine_in[b].n[a]) / RATIO : 1;
    }
    for (int d = 0; d < dim; ++d)
      for (int side = -1; side <= 1; side += 2) {
        // coarse zones just outside this face of the fine box; the face is
        // their high face when they lie below the box (side of the zone +1)
        int lo[3] = {c0[0], c0[1], c0[2]}, hi[3] = {c1[0], c1[1], c1[2]};
        lo[d] = (side < 0) ? c0[d] - 1 : c1[d];
        hi[d] = lo[d] + 1;
        for (int k = lo[2]; k < hi[2]; ++k)
          for (int j = lo[1]; j < hi[1]; ++j)
            for (int i = lo[0]; i < hi[0]; ++i) {
              if (covered(i, j, k)) continue;
              const int zs = (side < 0) ? 1 : 0;  // zone below the box: its high face
              zone_mask[{k, j, i}] |= 1 << (2 * d + zs);
            }
      }
  }
  std::vector<AFace> faces;
  std::vector<AZone> zones;
  for (auto& kv : zone_mask) {
    const int X[3] = {std::get<2>(kv.first), std::get<1>(kv.first), std::get<0>(kv.first)};
    AZone Zn;
    Zn.cb = coarse_owner(X[0], X[1], X[2]);
    for (int a = 0; a < 3; ++a) Zn.zi[a] = X[a] - C[Zn.cb].lo[a];
    Zn.f0 = (int)faces.size();
    for (int d = 0; d < dim; ++d)
      for (int s = 0; s < 2; ++s) {
        if (!(kv.second & (1 << (2 * d + s)))) continue;
        const int side = s ? 1 : -1;
        AFace E;
        E.cb = Zn.cb;
        E.d = d;
        E.side = side;
        for (int a = 0; a < 3; ++a) E.ci[a] = Zn.zi[a];
        if (side > 0) E.ci[d] += 1;
        // the fine faces: on the refined face, transverse children of X
        const int gf = RATIO * (X[d] + (side > 0 ? 1 : 0));
        int g[3] = {RATIO * X[0], RATIO * X[1], RATIO * X[2]};
        g[d] = (side > 0) ? gf : gf - 1;  // covered fine zone next to the face
        E.fb = fine_owner(g[0], g[1], g[2]);
        if (E.fb < 0) return HYDRO_EINVAL;  // cannot happen for a covered neighbour
        for (int a = 0; a < 3; ++a) E.fi[a] = g[a] - F[E.fb].lo[a];
        E.fi[d] = gf - F[E.fb].lo[d];
        faces.push_back(E);
      }
    Zn.nf = (int)faces.size() - Zn.f0;
    zones.push_back(Zn);
  }
  P->nc = nc;
  P->nf = nf;
  P->nface = (int)faces.size();
  P->nzone = (int)zones.size();

  std::vector<int> fill_first, fill_blk, avg_first, avg_blk, dt_first, dt_blk;
  block_map(fill_items, fill_first, fill_blk);
  block_map(avg_items, avg_first, avg_blk);
  block_map(dt_items, dt_first, dt_blk);
  P->fill_nb = (unsigned)fill_blk.size();
  P->avg_nb = (unsigned)avg_blk.size();
  P->dt_nb = (unsigned)dt_blk.size();

  Carve cv;
  const size_t oC = cv.add(C.data(), nc * sizeof(ACoarse));
  const size_t oF = cv.add(F.data(), nf * sizeof(AFine));
  const size_t oE = cv.add(faces.data(), faces.size() * sizeof(AFace));
  const size_t oZ = cv.add(zones.data(), zones.size() * sizeof(AZone));
  const size_t oOc = cv.add(own_c.data(), own_c.size() * sizeof(int));
  const size_t oOf = cv.add(own_f.data(), own_f.size() * sizeof(int));
  const size_t oFb = cv.add(fill_blk.data(), fill_blk.size() * sizeof(int));
  const size_t oFf = cv.add(fill_first.data(), fill_first.size() * sizeof(int));
  const size_t oAb = cv.add(avg_blk.data(), avg_blk.size() * sizeof(int));
  const size_t oAf = cv.add(avg_first.data(), avg_first.size() * sizeof(int));
  const size_t oDb = cv.add(dt_blk.data(), dt_blk.size() * sizeof(int));
  const size_t oDf = cv.add(dt_first.data(), dt_first.size() * sizeof(int));
  const size_t oRc = cv.add(nullptr, 5 * faces.size() * sizeof(double));
  const size_t oRf = cv.add(nullptr, 5 * faces.size() * sizeof(double));
  const size_t oTc = cv.add(nullptr, nc * sizeof(double));
  const size_t oTnc = cv.add(nullptr, nc * sizeof(double));
  const size_t oTf = cv.add(nullptr, std::max(nf, 1) * sizeof(double));
  const size_t oTnf = cv.add(nullptr, std::max(nf, 1) * sizeof(double));
  const size_t oL = cv.add(nullptr, sizeof(DevFlags));
  if (cudaMalloc(&P->mem, cv.total) != cudaSuccess) {
    cudaGetLastError();
    P->mem = nullptr;
    return HYDRO_ENOMEM;
  }
  std::vector<char> host(cv.total, 0);
  size_t off = 0;
  for (auto& pr : cv.parts) {
    if (pr.first && pr.second) std::memcpy(host.data() + off, pr.first, pr.second);
    off += (pr.second + 255) & ~size_t(255);
  }
  if (cudaMemcpy(P->mem, host.data(), cv.total, cudaMemcpyHostToDevice) != cudaSuccess) return HYDRO_ECUDA;
  char* m = P->mem;
  P->C = reinterpret_cast<ACoarse*>(m + oC);
  P->F = reinterpret_cast<AFine*>(m + oF);
  P->faces = reinterpret_cast<AFace*>(m + oE);
  P->zones = reinterpret_cast<AZone*>(m + oZ);
  P->own_c = reinterpret_cast<int*>(m + oOc);
  P->own_f = reinterpret_cast<int*>(m + oOf);
  P->fill_blk = reinterpret_cast<int*>(m + oFb);
  P->fill_first = reinterpret_cast<int*>(m + oFf);
  P->avg_blk = reinterpret_cast<int*>(m + oAb);
  P->avg_first = reinterpret_cast<int*>(m + oAf);
  P->dt_blk = reinterpret_cast<int*>(m + oDb);
  P->dt_first = reinterpret_cast<int*>(m + oDf);
  P->reg_c = reinterpret_cast<double*>(m + oRc);
  P->reg_f = reinterpret_cast<double*>(m + oRf);
  P->dtc = reinterpret_cast<double*>(m + oTc);
  P->dtnc = reinterpret_cast<double*>(m + oTnc);
  P->dtf = reinterpret_cast<double*>(m + oTf);
  P->dtnf = reinterpret_cast<double*>(m + oTnf);
  P->lvl = reinterpret_cast<DevFlags*>(m + oL);
  return HYDRO_OK;
}

size_t tmp_bytes_of(const hydro_amr_t* h) {
  size_t n = 0;
  for (int b = 0; b < h->nfine; ++b) {
    const hydro_box_t& fb = h->fine_in[b];
    const size_t g = (size_t)(fb.n[0] + 2 * NG) * (fb.n[1] + 2 * NG) * ((h->dim == 3) ? fb.n[2] + 2 * NG : 1);
    n += (5 * g + 31) & ~size_t(31);
  }
  return std::max<size_t>(n, 32) * sizeof(double);
}

// argument checks that need no plan: shapes, spacings, nesting
int check_hierarchy(const hydro_amr_t* h, const hydro_params_t* params) {
  const int dim = h->dim;
  if ((dim != 2 && dim != 3) || params->dim != dim || h->ncoarse < 1 || h->nfine < 0) return HYDRO_EINVAL;
  if (!h->coarse_in || !h->coarse_out || !h->coarse_lo || (h->nfine > 0 && (!h->fine_in || !h->fine_out || !h->fine_lo)))
    return HYDRO_EINVAL;
  for (int a = 0; a < 3; ++a) {
    const int n = (a < dim) ? h->domain[a] : 1;
    if (n < 1) return HYDRO_EINVAL;
  }
  const double* dxc = h->coarse_in[0].dx;
  for (int b = 0; b < h->ncoarse; ++b) {
    hydro_box_t x = prefilled(h->coarse_in[b]), y = prefilled(h->coarse_out[b]);
    if (!valid_box(&x, dim) || !valid_box(&y, dim)) return HYDRO_EINVAL;
    for (int a = 0; a < 3; ++a)
      if (h->coarse_out[b].n[a] != x.n[a]) return HYDRO_EINVAL;
    for (int a = 0; a < dim; ++a) {
      if (h->coarse_in[b].dx[a] != dxc[a]) return HYDRO_EINVAL;
      if (h->coarse_lo[3 * b + a] < 0 || h->coarse_lo[3 * b + a] + h->coarse_in[b].n[a] > h->domain[a])
        return HYDRO_EINVAL;
    }
  }
  for (int b = 0; b < h->nfine; ++b) {
    const hydro_box_t& fb = h->fine_in[b];
    hydro_box_t x = prefilled(fb), y = prefilled(h->fine_out[b]);
    if (!valid_box(&x, dim) || !valid_box(&y, dim)) return HYDRO_EINVAL;
    for (int a = 0; a < 3; ++a)
      if (h->fine_out[b].n[a] != fb.n[a]) return HYDRO_EINVAL;
    for (int a = 0; a < dim; ++a) {
      const int lo = h->fine_lo[3 * b + a], n = fb.n[a];
      if (lo % RATIO || n % RATIO) return HYDRO_EINVAL;
      // coarsened and grown by 2 (ghost layers) + 1 (slope): inside the domain
      if (lo / RATIO - 3 < 0 || (lo + n) / RATIO + 3 > h->domain[a]) return HYDRO_EINVAL;
      if (fb.dx[a] * RATIO != dxc[a]) return HYDRO_EINVAL;
    }
    if (dim == 2 && h->fine_lo[3 * b + 2] != 0) return HYDRO_EINVAL;
  }
  return HYDRO_OK;
}

}  // namespace
}  // namespace hydro

void hydro_amr_release(hydro_ctx* ctx) {
  if (!ctx || !ctx->amr) return;
  for (AmrPlan* p : ctx->amr->plans) destroy_amr_plan(p);
  if (ctx->amr->tmp) cudaFree(ctx->amr->tmp);
  delete ctx->amr;
  ctx->amr = nullptr;
}

extern "C" int hydro_amr_advance(hydro_ctx_t* ctx, const hydro_amr_t* h, const hydro_params_t* params,
                                 const double* dt_dev, double* dt_next_dev, int* bad_host, void* stream) {
  if (!ctx || !h || !params || !dt_dev || !dt_next_dev || !valid_params(params)) return HYDRO_EINVAL;
  if (params->flags & HYDRO_FLAG_FLUX_GRAV_ENERGY) return HYDRO_ENOTIMPL;
  int rc = check_hierarchy(h, params);
  if (rc) return rc;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return HYDRO_ECUDA;
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return HYDRO_ECUDA;
  struct Restore {
    int dev, prev;
    ~Restore() { if (prev >= 0 && prev != dev) cudaSetDevice(prev); }
  } restore{ctx->device, prev};
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  if (!ctx->amr) {
    ctx->amr = new (std::nothrow) hydro_amr_state();
    if (!ctx->amr) return HYDRO_ENOMEM;
  }
  hydro_amr_state* S = ctx->amr;
  // the library-owned fine stage (after the first substep): grow-only; plans
  // point into it, so a move drops them
  const size_t need = tmp_bytes_of(h);
  if (need > S->tmp_bytes) {
    if (cudaDeviceSynchronize() != cudaSuccess) return HYDRO_ECUDA;
    for (AmrPlan* p : S->plans) destroy_amr_plan(p);
    S->plans.clear();
    if (S->tmp) cudaFree(S->tmp);
    S->tmp = nullptr;
    S->tmp_bytes = 0;
    if (ctx->fail_alloc || cudaMalloc(&S->tmp, need) != cudaSuccess) {
      cudaGetLastError();
      return HYDRO_ENOMEM;
    }
    S->tmp_bytes = need;
  }
  uint64_t key = 1469598103934665603ull;
  key = fnv(key, h, offsetof(hydro_amr_t, ncoarse));
  key = fnv(key, &h->ncoarse, sizeof h->ncoarse);
  key = fnv(key, &h->nfine, sizeof h->nfine);
  key = fnv(key, h->coarse_in, h->ncoarse * sizeof(hydro_box_t));
  key = fnv(key, h->coarse_out, h->ncoarse * sizeof(hydro_box_t));
  key = fnv(key, h->coarse_lo, 3 * h->ncoarse * sizeof(int));
  if (h->nfine) {
    key = fnv(key, h->fine_in, h->nfine * sizeof(hydro_box_t));
    key = fnv(key, h->fine_out, h->nfine * sizeof(hydro_box_t));
    key = fnv(key, h->fine_lo, 3 * h->nfine * sizeof(int));
  }
  AmrPlan* P = nullptr;
  for (AmrPlan* p : S->plans)
    if (p->key == key) P = p;
  if (!P) {
    if (cudaStreamSynchronize(st) != cudaSuccess) return HYDRO_ECUDA;
    P = new (std::nothrow) AmrPlan();
    if (!P) return HYDRO_ENOMEM;
    rc = build_plan(h, S->tmp, P);
    if (rc) {
      destroy_amr_plan(P);
      return rc;
    }
    P->key = key;
    if ((int)S->plans.size() >= MAX_AMR_PLANS) {
      auto lru = std::min_element(S->plans.begin(), S->plans.end(),
                                  [](const AmrPlan* a, const AmrPlan* b) { return a->last_use < b->last_use; });
      destroy_amr_plan(*lru);
      S->plans.erase(lru);
    }
    S->plans.push_back(P);
  }
  P->last_use = ++S->clock;
  const int dim = h->dim, nc = P->nc, nf = P->nf;
  const unsigned rb = blocks_of(5LL * std::max(P->nface, 1), 256), zb = blocks_of(5LL * std::max(P->nzone, 1), 256);
  StepConst K = step_const(params, P->A.dx, 1.0);

  ka_prep<<<1, 256, 0, st>>>(dt_dev, P->dtc, nc, P->dtf, nf, P->lvl, ctx->flags);
  ctx->launches += 1;
  // 1. coarse level
  int dbc[6];
  for (int a = 0; a < 3; ++a)
    for (int s = 0; s < 2; ++s) dbc[2 * a + s] = h->domain_bc[a][s];
  rc = hydro_fill_boundary(ctx, P->c_in.data(), P->c_lo.data(), nc, dim, h->domain, dbc, st);
  if (rc) return rc;
  const BatchBox* pb = nullptr;
  rc = hydro_batch_run(ctx, P->c_in.data(), P->c_out.data(), nc, params, 0, P->dtc, P->dtnc, nullptr, nullptr, st, &pb);
  if (rc) return rc;
  if (P->nface) {
    ka_reg_coarse<<<rb, 256, 0, st>>>(pb, P->faces, P->nface, P->reg_c);
    ctx->launches += 1;
  }
  // 2. fine level: two substeps of dt/2
  if (nf) {
    for (int sub = 0; sub < 2; ++sub) {
      ka_fill<<<P->fill_nb, BLOCK, 0, st>>>(P->F, P->C, P->own_c, P->own_f, P->fill_blk, P->fill_first, P->A, sub, sub);
      const hydro_box_t* fin = sub ? P->f_tmp.data() : P->f_in.data();
      const hydro_box_t* fout = sub ? P->f_out.data() : P->f_tmp.data();
      rc = hydro_batch_run(ctx, fin, fout, nf, params, 0, P->dtf, P->dtnf, nullptr, nullptr, st, &pb);
      if (rc) return rc;
      ctx->launches += 1;
      if (P->nface) {
        ka_reg_fine<<<rb, 256, 0, st>>>(pb, P->faces, P->nface, dim, P->reg_f, sub == 0);
        ctx->launches += 1;
      }
    }
    // 3. reflux, 4. average down
    if (P->nzone) {
      ka_reflux<<<zb, 256, 0, st>>>(P->C, P->zones, P->nzone, P->faces, P->nface, P->reg_c, P->reg_f, dt_dev, P->A);
      ctx->launches += 1;
    }
    ka_avgdown<<<P->avg_nb, BLOCK, 0, st>>>(P->F, P->C, P->own_c, P->avg_blk, P->avg_first, P->A);
    ctx->launches += 1;
  }
  // 5. the next step
  ka_dt_partial<<<P->dt_nb, BLOCK, 0, st>>>(P->C, P->dt_blk, P->dt_first, K, P->lvl);
  ka_dt_final<<<1, 32, 0, st>>>(P->lvl, P->dtnf, nf, P->A, params->cfl, dt_next_dev);
  ctx->launches += 2;
  if (cudaGetLastError() != cudaSuccess) return HYDRO_ECUDA;
  if (bad_host) {
    int b[2] = {0, 0};
    if (cudaMemcpyAsync(&b[0], &P->lvl->bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&b[1], &ctx->flags->bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return HYDRO_ECUDA;
    *bad_host = (b[0] || b[1]) ? 1 : 0;
    if (*bad_host) return HYDRO_EBADSTATE;
  }
  return HYDRO_OK;
}
