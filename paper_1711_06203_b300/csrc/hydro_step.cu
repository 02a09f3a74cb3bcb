// Single-box kernels of the staged CTU-PPM step and their launch sequence.
#include <algorithm>

#include "hydro_items.cuh"

namespace hydro {

namespace {

__global__ void __launch_bounds__(BLOCK) k_prim(BoxGeom in, ScratchGeom sg, double* __restrict__ Q, StepConst K,
                                                Range R, DevFlags* flags) {
  prim_item(in, sg, Q, K, R, flags, (long long)blockIdx.x * BLOCK + threadIdx.x);
}

// the x tracing with the lanes of a warp along x (one warp per row segment)
__global__ void __launch_bounds__(BLOCK) k_trace_row_x(ScratchGeom sg, const double* __restrict__ Q,
                                                       double* __restrict__ TM, double* __restrict__ TP, StepConst K,
                                                       SweepRange R) {
  trace_row_x_item(sg, Q, TM, TP, K, R, ((long long)blockIdx.x * BLOCK + threadIdx.x) >> 5);
}

// the y and z tracing in tiles of 32 pencils x TILE_ZONES zones (five blocks
// per SM: 96 registers, a few bytes of spills, were 2 % faster on the Sedov
// box and 0.4 % on random data than 114 registers at four)
template <int D>
__global__ void __launch_bounds__(TILE_W * 32, 5) k_trace_tile(ScratchGeom sg, const double* __restrict__ Q,
                                                            double* __restrict__ TM, double* __restrict__ TP,
                                                            StepConst K, SweepRange R) {
  __shared__ TileSmem sm;
  trace_tile_item<D>(sg, Q, TM, TP, K, R, blockIdx.x, sm);
}

// Face sets of one direction each (first or final fluxes) in one launch:
// blocks [first[d], first[d+1]) solve direction d (empty sets allowed).
struct DirSets {
  Range r[3];
  unsigned first[4];
};
// direction of this block and its item index (constant indices only: a
// computed index into the launch parameters would copy them to local memory)
__device__ __forceinline__ int dir_of(unsigned f1, unsigned f2, long long& t) {
  const unsigned b = blockIdx.x;
  const int d = ((b >= f1) ? 1 : 0) + ((b >= f2) ? 1 : 0);
  const unsigned f = (d == 0) ? 0u : (d == 1) ? f1 : f2;
  t = (long long)(b - f) * BLOCK + threadIdx.x;
  return d;
}
// (resident blocks per SM: solver_blocks)
template <bool EINF>
__global__ void __launch_bounds__(BLOCK, solver_blocks(EINF)) k_flux1(ScratchGeom sg, Scratch s, StepConst K, DirSets S) {
  long long t;
  switch (dir_of(S.first[1], S.first[2], t)) {
    case 0: flux1_item<0, EINF>(sg, s.TP[0], s.TM[0], s.F1[0], K, S.r[0], t); break;
    case 1: flux1_item<1, EINF>(sg, s.TP[1], s.TM[1], s.F1[1], K, S.r[1], t); break;
    default: flux1_item<2, EINF>(sg, s.TP[2], s.TM[2], s.F1[2], K, S.r[2], t); break;
  }
}

// The six intermediate-flux sets F^{d|t} of a 3-D step are independent of
// one another, so they run as one launch: blocks [first[c], first[c+1])
// solve set c = (d, t) in the order (0,1), (0,2), (1,0), (1,2), (2,0), (2,1).
// (Six launches each ended on a partly filled last wave.)
struct Flux2Sets {
  Range r[6];
  unsigned first[7];
};
template <bool EINF>
__global__ void __launch_bounds__(BLOCK, solver_blocks(EINF)) k_flux2(ScratchGeom sg, Scratch s, StepConst K, Flux2Sets S) {
  const unsigned b = blockIdx.x;
  int c = 0;
  unsigned f = 0;
#pragma unroll
  for (int i = 1; i < 6; ++i)
    if (b >= S.first[i]) { c = i; f = S.first[i]; }
  const long long t = (long long)(b - f) * BLOCK + threadIdx.x;
  switch (c) {
    case 0: flux2_item<0, 1, EINF>(sg, s.TP[0], s.TM[0], s.F1[1], s.F2[0][1], K, S.r[0], t); break;
    case 1: flux2_item<0, 2, EINF>(sg, s.TP[0], s.TM[0], s.F1[2], s.F2[0][2], K, S.r[1], t); break;
    case 2: flux2_item<1, 0, EINF>(sg, s.TP[1], s.TM[1], s.F1[0], s.F2[1][0], K, S.r[2], t); break;
    case 3: flux2_item<1, 2, EINF>(sg, s.TP[1], s.TM[1], s.F1[2], s.F2[1][2], K, S.r[3], t); break;
    case 4: flux2_item<2, 0, EINF>(sg, s.TP[2], s.TM[2], s.F1[0], s.F2[2][0], K, S.r[4], t); break;
    default: flux2_item<2, 1, EINF>(sg, s.TP[2], s.TM[2], s.F1[1], s.F2[2][1], K, S.r[5], t); break;
  }
}

// final fluxes: in 3-D from the intermediate fluxes of the two other
// directions, in 2-D from the first fluxes of the other direction
// (held to the solver bound: the three-operand form otherwise takes 94
// registers and halves the resident warps)
template <bool THREE, bool EINF>
__global__ void __launch_bounds__(BLOCK, solver_blocks(EINF))
    k_flux3(ScratchGeom sg, Scratch s, StepConst K, DirSets S) {
  long long t;
  switch (dir_of(S.first[1], S.first[2], t)) {
    case 0:
      if (THREE) flux3_item<0, EINF>(sg, s.TP[0], s.TM[0], s.F2[1][2], s.F2[2][1], s.F3[0], K, S.r[0], t);
      else flux3_item<0, EINF>(sg, s.TP[0], s.TM[0], s.F1[1], nullptr, s.F3[0], K, S.r[0], t);
      break;
    case 1:
      if (THREE) flux3_item<1, EINF>(sg, s.TP[1], s.TM[1], s.F2[0][2], s.F2[2][0], s.F3[1], K, S.r[1], t);
      else flux3_item<1, EINF>(sg, s.TP[1], s.TM[1], s.F1[0], nullptr, s.F3[1], K, S.r[1], t);
      break;
    default:
      if (THREE) flux3_item<2, EINF>(sg, s.TP[2], s.TM[2], s.F2[0][1], s.F2[1][0], s.F3[2], K, S.r[2], t);
      break;
  }
}

__global__ void __launch_bounds__(BLOCK) k_update(BoxGeom in, BoxGeom out, ScratchGeom sg, const double* __restrict__ Fx,
                                                  const double* __restrict__ Fy, const double* __restrict__ Fz,
                                                  StepConst K, Range R, DevFlags* flags) {
  update_item(in, out, sg, Fx, Fy, Fz, K, R, flags, (long long)blockIdx.x * BLOCK + threadIdx.x);
}

__global__ void __launch_bounds__(BLOCK) k_dt_partial(BoxGeom box, StepConst K, Range R, DevFlags* flags) {
  dt_partial_item(box, K, R, flags, (long long)blockIdx.x * BLOCK + threadIdx.x);
}

__global__ void k_dt_final(DevFlags* flags, double dx0, double dx1, double dx2, int dim, double cfl) {
  dt_final_item(flags, dx0, dx1, dx2, dim, cfl);
}

__global__ void k_reset_speed(DevFlags* flags) {
  if (threadIdx.x < 3) flags->maxspeed[threadIdx.x] = 0ull;
}

__global__ void k_reset_step(DevFlags* flags) {
  if (threadIdx.x < 3) flags->maxspeed[threadIdx.x] = 0ull;
}

inline unsigned blocks_for(long long n) { return (unsigned)((n + BLOCK - 1) / BLOCK); }

// the y or z tracing over the pencils and zones of sw, in tiles of 32 pencils x TILE_ZONES zones
template <int D>
void launch_trace_tile(const ScratchGeom& sg, const Scratch& s, const StepConst& K, const SweepRange& sw,
                       cudaStream_t st) {
  const long long ngroup = ((long long)sw.ext1 * sw.ext2 + 31) / 32;
  const long long ntile = (sw.nd - sw.lod + TILE_ZONES) / TILE_ZONES;
  k_trace_tile<D><<<(unsigned)(ngroup * ntile), TILE_W * 32, 0, st>>>(sg, s.Q, s.TM[D], s.TP[D], K, sw);
}

// the x tracing over the pencils and zones of sw: one warp per ROW_ZONES positions of the pencils laid end to end
void launch_trace_row_x(const ScratchGeom& sg, const Scratch& s, const StepConst& K, const SweepRange& sw,
                        cudaStream_t st) {
  const long long warps = row_warps(sw);
  k_trace_row_x<<<(unsigned)((warps + BLOCK / 32 - 1) / (BLOCK / 32)), BLOCK, 0, st>>>(sg, s.Q, s.TM[0], s.TP[0], K,
                                                                                       sw);
}

// copy the final fluxes on the outer faces (face 0 and face n_d along every
// active d, transverse interior) into dst, plane after plane in (d, side)
// order, each plane 5 fields of (t1 fastest, t2) with t1 < t2 the transverse
// axes; x- and y-faces only on the planes [zlo, zhi), z-faces only when
// those planes include the first (face 0) or the last (face n_z) one
__global__ void k_record_faces(Scratch s, ScratchGeom sg, int n0, int n1, int n2, int dim, int zlo, int zhi,
                               double* __restrict__ dst) {
  const int n[3] = {n0, n1, n2};
  long long off = 0;
  for (int d = 0; d < dim; ++d) {
    const int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
    const int e1 = n[t1], e2 = (t2 < dim) ? n[t2] : 1;
    const long long A = (long long)e1 * e2;
    for (int side = 0; side < 2; ++side) {
      // rows of t2 to copy: for x- and y-faces (t2 = z) the planes given
      int r0 = 0, r1 = e2;
      if (dim == 3 && t2 == 2) { r0 = zlo; r1 = zhi; }
      if (d == 2 && !(side ? zhi == n2 : zlo == 0)) r1 = r0;  // z-face outside these planes
      const long long cnt = (long long)(r1 - r0) * e1;
      for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < 5 * cnt;
           q += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(q / cnt);
        const long long r = q - c * cnt;
        int z[3] = {0, 0, 0};
        z[d] = side ? n[d] : 0;
        z[t1] = (int)(r % e1);
        z[t2] = r0 + (int)(r / e1);
        dst[off + c * A + (long long)z[t2] * e1 + z[t1]] = s.F3[d][c * sg.sc + sg.id(z[0], z[1], z[2])];
      }
      off += 5 * A;
    }
  }
}

// the tracing along d over zones [lod, nd] of the pencils whose transverse
// coordinates are [-1, n] on the first transverse axis and [lo2, lo2 + ext2)
// on the second
void launch_trace_range(int d, const StepArgs& a, int lo2, int ext2, int lod, int nd, cudaStream_t st) {
  const int* n = a.in.n;
  const int t1 = (d == 0) ? 1 : 0;
  SweepRange sw;
  sw.lo1 = -1; sw.ext1 = n[t1] + 2;
  sw.lo2 = lo2; sw.ext2 = ext2;
  sw.lod = lod;
  sw.nd = nd;
  sw.seg = TRACE_SEG;
  sw.nseg = (nd - lod + TRACE_SEG) / TRACE_SEG;
  if (d == 0) launch_trace_row_x(a.sg, a.s, a.K, sw, st);
  if (d == 1) launch_trace_tile<1>(a.sg, a.s, a.K, sw, st);
  if (d == 2) launch_trace_tile<2>(a.sg, a.s, a.K, sw, st);
}
// ... over every zone [-1, n] along d
void launch_trace(int d, const StepArgs& a, int lo2, int ext2, cudaStream_t st) {
  launch_trace_range(d, a, lo2, ext2, -1, a.in.n[d], st);
}

// first fluxes of the directions d in dirs (bit d) over the face ranges r[d], one launch
int launch_flux1_ranges(const StepArgs& a, const Range r[3], unsigned dirs, cudaStream_t st) {
  DirSets S;
  S.first[0] = 0;
  for (int d = 0; d < 3; ++d) {
    S.r[d] = r[d];
    S.first[d + 1] = S.first[d] + (((dirs >> d) & 1u) ? blocks_for(S.r[d].count()) : 0u);
  }
  if (S.first[3] == 0) return 0;
  if (a.K.einfeldt) k_flux1<true><<<S.first[3], BLOCK, 0, st>>>(a.sg, a.s, a.K, S);
  else k_flux1<false><<<S.first[3], BLOCK, 0, st>>>(a.sg, a.s, a.K, S);
  return 1;
}

// first fluxes through d-faces [0, n_d] x the transverse zones of rt (the
// tracing range: zones [-1, n] on active axes, or a slab of z-planes) of the
// directions d in dirs (bit d), one launch
int launch_flux1_all(const StepArgs& a, const Range& rt, unsigned dirs, cudaStream_t st) {
  const int* n = a.in.n;
  Range r[3];
  for (int d = 0; d < 3; ++d) {
    r[d] = rt;
    r[d].lo[d] = 0;
    r[d].ext[d] = n[d] + 1;
  }
  return launch_flux1_ranges(a, r, dirs, st);
}

// final fluxes of the active directions d over the face ranges r[d], one launch
int launch_flux3_ranges(const StepArgs& a, int dim, const Range r[3], cudaStream_t st) {
  DirSets S;
  S.first[0] = 0;
  for (int d = 0; d < 3; ++d) {
    S.r[d] = r[d];
    S.first[d + 1] = S.first[d] + ((d < dim) ? blocks_for(r[d].count()) : 0u);
  }
  const unsigned g = S.first[3];
  if (g == 0) return 0;
  if (a.K.einfeldt) {
    if (dim == 3) k_flux3<true, true><<<g, BLOCK, 0, st>>>(a.sg, a.s, a.K, S);
    else k_flux3<false, true><<<g, BLOCK, 0, st>>>(a.sg, a.s, a.K, S);
  } else {
    if (dim == 3) k_flux3<true, false><<<g, BLOCK, 0, st>>>(a.sg, a.s, a.K, S);
    else k_flux3<false, false><<<g, BLOCK, 0, st>>>(a.sg, a.s, a.K, S);
  }
  return 1;
}

// final fluxes through d-faces [0, n_d] of every active direction d, over
// transverse zones [0, n) except the z range [zlo, zlo + zext) (in 3-D), one launch
int launch_flux3_all(const StepArgs& a, int dim, int zlo, int zext, cudaStream_t st) {
  const int* n = a.in.n;
  Range r[3];
  for (int d = 0; d < 3; ++d) {
    for (int ax = 0; ax < 3; ++ax) { r[d].lo[ax] = 0; r[d].ext[ax] = (ax < dim) ? n[ax] : 1; }
    if (dim == 3) { r[d].lo[2] = zlo; r[d].ext[2] = zext; }
    r[d].ext[d] += 1;
  }
  return launch_flux3_ranges(a, dim, r, st);
}

// 3-D intermediate fluxes F^{d|t}: d-faces [0, n_d] x t in [0, n_t) x third
// axis [-1, n], restricted along z to the interior planes [zlo, zlo + zext)
// of a slab (the ranges grow by the faces and zones the slab's final fluxes
// read: F^{x|y}, F^{y|x} on planes [zlo - 1, zlo + zext], F^{z|x}, F^{z|y} on
// z-faces [zlo, zlo + zext], F^{x|z}, F^{y|z} on the slab's planes)
// the six sets (d, t) in the order (0,1), (0,2), (1,0), (1,2), (2,0), (2,1)
// over the ranges r[c], one launch
int launch_flux2_ranges(const StepArgs& a, const Range r[6], cudaStream_t st) {
  Flux2Sets S;
  S.first[0] = 0;
  for (int c = 0; c < 6; ++c) {
    S.r[c] = r[c];
    S.first[c + 1] = S.first[c] + blocks_for(r[c].count());
  }
  if (S.first[6] == 0) return 0;
  if (a.K.einfeldt) k_flux2<true><<<S.first[6], BLOCK, 0, st>>>(a.sg, a.s, a.K, S);
  else k_flux2<false><<<S.first[6], BLOCK, 0, st>>>(a.sg, a.s, a.K, S);
  return 1;
}

// the range of set (d, t) with a z extent [zlo, zhi) of faces (d = z), zones
// (t = z) or planes of the third axis (neither)
Range flux2_range(const int n[3], int d, int t, int zlo, int zhi) {
  const int o = 3 - d - t;
  Range r;
  r.lo[d] = 0; r.ext[d] = n[d] + 1;
  r.lo[t] = 0; r.ext[t] = n[t];
  r.lo[o] = -1; r.ext[o] = n[o] + 2;
  r.lo[2] = zlo; r.ext[2] = std::max(0, zhi - zlo);
  return r;
}

int launch_flux2_all(const StepArgs& a, cudaStream_t st, int zlo = 0, int zext = -1) {
  const int* n = a.in.n;
  if (zext < 0) zext = n[2];
  Range r[6];
  int c = 0;
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < 3; ++t) {
      if (t == d) continue;
      // the z extent: faces, zones or the widened range of the slab
      if (d == 2) r[c] = flux2_range(n, d, t, zlo, zlo + zext + 1);
      else if (t == 2) r[c] = flux2_range(n, d, t, zlo, zlo + zext);
      else r[c] = flux2_range(n, d, t, zlo - 1, zlo + zext + 1);
      ++c;
    }
  return launch_flux2_ranges(a, r, st);
}

}  // namespace

cudaError_t launch_step(const StepArgs& a, cudaStream_t st, long long* launches) {
  const int dim = a.K.dim;
  long long nl = 0;
  auto mark = [&](int stage) {
    if (a.events) cudaEventRecord(a.events[stage], st);
  };
  mark(ST_PRIM);
  k_reset_step<<<1, 32, 0, st>>>(a.flags);
  nl += 1;
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
    const int t2 = (d == 2) ? 1 : 2;
    launch_trace(d, a, rt.lo[t2], rt.ext[t2], st);
  }
  nl += dim;
  mark(ST_FLUX1);
  // stage 4a: first fluxes on d-faces [0, n_d] x transverse [-1, n]
  nl += launch_flux1_all(a, rt, (1u << dim) - 1u, st);
  mark(ST_FLUX2);
  // stage 4b (3-D): intermediate fluxes F^{d|t}
  if (dim == 3) nl += launch_flux2_all(a, st);
  mark(ST_FLUX3);
  // stage 4c: final fluxes on d-faces [0, n_d] x transverse interior
  nl += launch_flux3_all(a, dim, 0, (dim == 3) ? n[2] : 1, st);
  mark(ST_UPDATE);
  // stage 5: update + CFL partials (speed maxima were reset at the start of the step)
  Range ru;
  for (int ax = 0; ax < 3; ++ax) { ru.lo[ax] = 0; ru.ext[ax] = (ax < dim) ? n[ax] : 1; }
  k_update<<<blocks_for(ru.count()), BLOCK, 0, st>>>(a.in, a.out, sg, s.F3[0], s.F3[1], dim == 3 ? s.F3[2] : s.F3[0],
                                                     a.K, ru, a.flags);
  k_dt_final<<<1, 1, 0, st>>>(a.flags, a.dx[0], a.dx[1], a.dx[2], dim, a.cfl);
  nl += 2;
  mark(NSTAGES);
  if (launches) *launches += nl;
  return cudaGetLastError();
}

Scratch shift_scratch(const Scratch& s, long long shift) {
  Scratch w = s;
  w.Q -= shift;
  for (int d = 0; d < 3; ++d) {
    w.TM[d] -= shift;
    w.TP[d] -= shift;
    w.F1[d] -= shift;
    w.F3[d] -= shift;
    for (int t = 0; t < 3; ++t)
      if (w.F2[d][t]) w.F2[d][t] -= shift;
  }
  return w;
}

cudaError_t launch_record_faces(const StepArgs& a, int zlo, int zhi, double* faces, cudaStream_t st) {
  const int dim = a.K.dim;
  k_record_faces<<<148, 256, 0, st>>>(a.s, a.sg, a.in.n[0], a.in.n[1], dim == 3 ? a.in.n[2] : 1, dim, zlo, zhi,
                                      faces);
  return cudaGetLastError();
}

cudaError_t launch_step_slabs(const StepArgs& a, int T, double* faces, cudaStream_t st, long long* launches) {
  const int* n = a.in.n;
  const int nslab = (n[2] + T - 1) / T;
  long long nl = 0;
  auto mark = [&](int stage) {
    if (a.events) cudaEventRecord(a.events[stage], st);
  };
  // a slabbed step is timed as a whole: its duration is reported as the
  // primitive-state stage, the other stages as zero
  mark(ST_PRIM);
  k_reset_step<<<1, 32, 0, st>>>(a.flags);
  nl += 1;
  for (int k = 0; k < nslab; ++k) {
    const int z0 = k * T, ze = std::min(T, n[2] - z0);
    StepArgs w = a;
    w.s = shift_scratch(a.s, (long long)z0 * a.sg.sz);
    const Scratch& s = w.s;
    // primitive state on planes [z0 - 4, z0 + ze + 4) of the grown box
    Range rp;
    for (int ax = 0; ax < 2; ++ax) { rp.lo[ax] = -NG; rp.ext[ax] = n[ax] + 2 * NG; }
    rp.lo[2] = z0 - NG; rp.ext[2] = ze + 2 * NG;
    k_prim<<<blocks_for(rp.count()), BLOCK, 0, st>>>(a.in, a.sg, s.Q, a.K, rp, a.flags);
    // traced states on zones [-1, n] in x and y and planes [z0 - 1, z0 + ze]
    launch_trace(0, w, z0 - 1, ze + 2, st);
    launch_trace(1, w, z0 - 1, ze + 2, st);
    launch_trace_range(2, w, -1, n[1] + 2, z0 - 1, z0 + ze, st);
    // first fluxes: x- and y-faces on planes [z0 - 1, z0 + ze], z-faces [z0, z0 + ze]
    Range r1[3];
    for (int d = 0; d < 3; ++d) {
      for (int ax = 0; ax < 2; ++ax) { r1[d].lo[ax] = -1; r1[d].ext[ax] = n[ax] + 2; }
      r1[d].lo[2] = z0 - 1; r1[d].ext[2] = ze + 2;
      if (d < 2) { r1[d].lo[d] = 0; r1[d].ext[d] = n[d] + 1; }
    }
    r1[2].lo[2] = z0; r1[2].ext[2] = ze + 1;
    nl += 4 + launch_flux1_ranges(w, r1, 7u, st);
    nl += launch_flux2_all(w, st, z0, ze);
    nl += launch_flux3_all(w, 3, z0, ze, st);
    Range ru;
    ru.lo[0] = 0; ru.ext[0] = n[0];
    ru.lo[1] = 0; ru.ext[1] = n[1];
    ru.lo[2] = z0; ru.ext[2] = ze;
    k_update<<<blocks_for(ru.count()), BLOCK, 0, st>>>(a.in, a.out, a.sg, s.F3[0], s.F3[1], s.F3[2], a.K, ru,
                                                       a.flags);
    nl += 1;
    if (faces) {
      if (launch_record_faces(w, z0, z0 + ze, faces, st) != cudaSuccess) return cudaGetLastError();
      nl += 1;
    }
  }
  k_dt_final<<<1, 1, 0, st>>>(a.flags, a.dx[0], a.dx[1], a.dx[2], 3, a.cfl);
  nl += 1;
  for (int stg = ST_TRACE; stg <= NSTAGES; ++stg) mark(stg);
  if (launches) *launches += nl;
  return cudaGetLastError();
}

// With the primitive state on planes [-NG, q) the frontiers (exclusive upper
// bounds) are:
//   x and y tracing, their first fluxes, F^{x|y}, F^{y|x}: planes [-1, q)
//   z tracing: zones [-1, q - 3) (its stencil reaches 3 planes up), in whole
//     tiles until the last chunk
//   first z fluxes, F^{z|x}, F^{z|y}, final z fluxes: z-faces f with zones
//     f - 1 and f traced (and the x/y quantities of planes f - 1, f)
//   F^{x|z}, F^{y|z}: zones k with z-faces k and k + 1 of the first fluxes
//   final x and y fluxes: planes k with F^{x|z}, F^{y|z} on k and
//     F^{z|y}, F^{z|x} on faces k, k + 1
//   update: planes k with the final z fluxes on faces k and k + 1
bool pipe_plan(int nz, int C, int bclo, int* pre_lo, PipeChunk* out) {
  if (nz < NG || C < 1 || C > nz || bclo < 0 || bclo > 2 || !pre_lo || !out) return false;
  auto zc = [&](int k) { return (int)((long long)nz * k / C); };  // first interior plane of chunk k
  // a periodic low face takes its ghost planes from the top NG interior
  // planes: those are copied first, so that the bottom can start with chunk 0
  const int pre = (bclo == 2) ? nz - NG : nz;
  *pre_lo = pre;
  auto low_ready = [&](int L) { return bclo == 2 || (bclo == 0 && L >= 1) || (bclo == 1 && L >= NG); };
  bool low_done = false;
  int done[PR_COUNT] = {};  // done up to
  done[PR_XY] = -1;
  done[PR_TZ] = -1;
  for (int k = 0; k < C; ++k) {
    PipeChunk& c = out[k];
    const bool last = k == C - 1;
    const int L = zc(k + 1);
    c.lo[PR_H2D] = zc(k);
    c.hi[PR_H2D] = std::max(zc(k), std::min(L, pre));
    c.lo[PR_PRIM] = zc(k);
    c.hi[PR_PRIM] = L;
    c.ghosts_low = !low_done && low_ready(L);
    low_done = low_done || c.ghosts_low;
    c.ghosts_high = last;  // every source plane has landed
    const int q = !low_done ? -NG : last ? nz + NG : L;
    int t[PR_COUNT];
    t[PR_XY] = std::max(done[PR_XY], std::min(q, nz + 1));
    t[PR_TZ] = std::max(done[PR_TZ], std::min(q - 3, nz + 1));
    if (!last) t[PR_TZ] = done[PR_TZ] + (t[PR_TZ] - done[PR_TZ]) / TILE_ZONES * TILE_ZONES;
    t[PR_F1Z] = std::max(done[PR_F1Z], std::min(t[PR_TZ], nz + 1));
    t[PR_F2XZ] = std::max(done[PR_F2XZ], std::min(t[PR_F1Z] - 1, nz));
    t[PR_F2Z] = std::max(done[PR_F2Z], std::min(std::min(t[PR_TZ], t[PR_XY]), nz + 1));
    t[PR_F3XY] = std::max(done[PR_F3XY], std::min(std::min(t[PR_F2XZ], t[PR_F2Z] - 1), nz));
    t[PR_F3Z] = std::max(done[PR_F3Z], std::min(std::min(t[PR_XY], t[PR_TZ]), nz + 1));
    t[PR_UPD] = std::max(done[PR_UPD], std::min(std::min(t[PR_F3XY], t[PR_F3Z] - 1), nz));
    for (int r = PR_XY; r < PR_COUNT; ++r) {
      c.lo[r] = done[r];
      c.hi[r] = t[r];
      done[r] = t[r];
    }
  }
  return true;
}

cudaError_t launch_step_host_piped(const StepArgs& a, const HostPipe& p, cudaStream_t st, long long* launches) {
  const int* n = a.in.n;
  const int nz = n[2];
  const ScratchGeom& sg = a.sg;
  const Scratch& s = a.s;
  const int C = p.nchunk;
  PipeChunk plan[PIPE_MAX_CHUNKS];
  int pre = nz;
  if (C > PIPE_MAX_CHUNKS || !pipe_plan(nz, C, a.in.bc[2][0], &pre, plan)) return cudaErrorInvalidValue;
  long long nl = 0;
  const size_t plane_bytes = (size_t)p.plane * sizeof(double);
  // of each plane, the interior rows: one contiguous run of n_y rows
  const long long row = p.plane / (n[1] + 2 * NG), rows_off = NG * row;
  const size_t rows_bytes = (size_t)(n[1] * row) * sizeof(double);
  auto copy = [&](double* dst, const double* src, int z0, int z1, cudaMemcpyKind kind, cudaStream_t cs) {
    const long long off = (long long)(z0 + NG) * p.plane + rows_off;
    for (int c = 0; c < 5; ++c)
      if (cudaMemcpy2DAsync(dst + c * p.field + off, plane_bytes, src + c * p.field + off, plane_bytes, rows_bytes,
                            (size_t)(z1 - z0), kind, cs) != cudaSuccess)
        return false;
    return true;
  };
  // input planes, chunk by chunk, after the work already queued on the
  // compute stream (which may still read the staging box)
  k_reset_step<<<1, 32, 0, st>>>(a.flags);
  nl += 1;
  if (cudaEventRecord(p.start, st) != cudaSuccess) return cudaGetLastError();
  if (cudaStreamWaitEvent(p.h2d, p.start, 0) != cudaSuccess) return cudaGetLastError();
  if (cudaStreamWaitEvent(p.back, p.start, 0) != cudaSuccess) return cudaGetLastError();
  if (pre < nz && !copy(a.in.u, p.h_in, pre, nz, cudaMemcpyHostToDevice, p.h2d)) return cudaGetLastError();
  for (int k = 0; k < C; ++k) {
    const PipeChunk& c = plan[k];
    if (c.hi[PR_H2D] > c.lo[PR_H2D] &&
        !copy(a.in.u, p.h_in, c.lo[PR_H2D], c.hi[PR_H2D], cudaMemcpyHostToDevice, p.h2d))
      return cudaGetLastError();
    if (cudaEventRecord(p.h2d_done[k], p.h2d) != cudaSuccess) return cudaGetLastError();
  }
  auto prim = [&](int zlo, int zext) {
    Range r;
    r.lo[0] = -NG; r.ext[0] = n[0] + 2 * NG;
    r.lo[1] = -NG; r.ext[1] = n[1] + 2 * NG;
    r.lo[2] = zlo; r.ext[2] = zext;
    k_prim<<<blocks_for(r.count()), BLOCK, 0, st>>>(a.in, sg, s.Q, a.K, r, a.flags);
    nl += 1;
  };
  // After each chunk every stage runs over the ranges of the plan (each zone
  // and face once, with the kernels of launch_step, so the result is bitwise
  // the same).  The front stages of a chunk (through the first fluxes) run
  // on `st`, its back stages on p.back once the front stages are done; the
  // front stages of later chunks write only planes and faces above those
  // the back stages of earlier chunks read, so the two streams run side by
  // side; each chunk's updated planes go back while the next computes.
  for (int k = 0; k < C; ++k) {
    const PipeChunk& c = plan[k];
    const bool last = k == C - 1;
    if (cudaStreamWaitEvent(st, p.h2d_done[k], 0) != cudaSuccess) return cudaGetLastError();
    prim(c.lo[PR_PRIM], c.hi[PR_PRIM] - c.lo[PR_PRIM]);
    if (c.ghosts_low) prim(-NG, NG);
    if (c.ghosts_high) prim(nz, NG);
    const int xy = c.lo[PR_XY], xy1 = c.hi[PR_XY];
    if (xy1 > xy) {
      launch_trace(0, a, xy, xy1 - xy, st);
      launch_trace(1, a, xy, xy1 - xy, st);
      nl += 2;
    }
    if (c.hi[PR_TZ] > c.lo[PR_TZ]) {
      launch_trace_range(2, a, -1, n[1] + 2, c.lo[PR_TZ], c.hi[PR_TZ] - 1, st);
      nl += 1;
    }
    // first fluxes: x- and y-faces on planes [xy, xy1), z-faces of PR_F1Z
    {
      Range r[3];
      for (int d = 0; d < 3; ++d) {
        for (int ax = 0; ax < 2; ++ax) { r[d].lo[ax] = -1; r[d].ext[ax] = n[ax] + 2; }
        r[d].lo[2] = xy; r[d].ext[2] = xy1 - xy;
        if (d < 2) { r[d].lo[d] = 0; r[d].ext[d] = n[d] + 1; }
      }
      r[2].lo[2] = c.lo[PR_F1Z]; r[2].ext[2] = c.hi[PR_F1Z] - c.lo[PR_F1Z];
      nl += launch_flux1_ranges(a, r, 7u, st);
    }
    if (cudaEventRecord(p.front_done[k], st) != cudaSuccess) return cudaGetLastError();
    if (cudaStreamWaitEvent(p.back, p.front_done[k], 0) != cudaSuccess) return cudaGetLastError();
    // intermediate fluxes, sets (0,1), (0,2), (1,0), (1,2), (2,0), (2,1)
    {
      const int a2 = c.lo[PR_F2XZ], b2 = c.hi[PR_F2XZ], z2 = c.lo[PR_F2Z], w2 = c.hi[PR_F2Z];
      Range r[6] = {flux2_range(n, 0, 1, xy, xy1), flux2_range(n, 0, 2, a2, b2), flux2_range(n, 1, 0, xy, xy1),
                    flux2_range(n, 1, 2, a2, b2),  flux2_range(n, 2, 0, z2, w2), flux2_range(n, 2, 1, z2, w2)};
      nl += launch_flux2_ranges(a, r, p.back);
    }
    // final fluxes (x- and y-faces on the planes of PR_F3XY, z-faces of
    // PR_F3Z) and the update; after the last chunk in pieces of p.piece
    // planes, each going back while the next computes
    const int step = last ? std::max(p.piece, 1) : nz + 1;
    const int f3xy1 = c.hi[PR_F3XY], f3z1 = c.hi[PR_F3Z], upd1 = c.hi[PR_UPD];
    for (int u0 = c.lo[PR_UPD], a3 = c.lo[PR_F3XY], z3 = c.lo[PR_F3Z]; u0 < upd1 || a3 < f3xy1 || z3 < f3z1;) {
      const int u1 = std::min(upd1, u0 + step);
      const int b3 = std::max(a3, last ? std::min(f3xy1, u1) : f3xy1);
      const int w3 = std::max(z3, last ? std::min(f3z1, u1 + 1) : f3z1);
      Range r[3];
      for (int d = 0; d < 3; ++d) {
        for (int ax = 0; ax < 2; ++ax) { r[d].lo[ax] = 0; r[d].ext[ax] = n[ax]; }
        r[d].lo[2] = a3; r[d].ext[2] = b3 - a3;
        if (d < 2) r[d].ext[d] += 1;
      }
      r[2].lo[2] = z3; r[2].ext[2] = w3 - z3;
      nl += launch_flux3_ranges(a, 3, r, p.back);
      if (u1 > u0) {
        Range ru;
        ru.lo[0] = 0; ru.ext[0] = n[0];
        ru.lo[1] = 0; ru.ext[1] = n[1];
        ru.lo[2] = u0; ru.ext[2] = u1 - u0;
        k_update<<<blocks_for(ru.count()), BLOCK, 0, p.back>>>(a.in, a.out, sg, s.F3[0], s.F3[1], s.F3[2], a.K, ru,
                                                               a.flags);
        nl += 1;
        // an event may be recorded again once a wait on it is enqueued
        if (cudaEventRecord(p.upd_done[k], p.back) != cudaSuccess) return cudaGetLastError();
        if (cudaStreamWaitEvent(p.d2h, p.upd_done[k], 0) != cudaSuccess) return cudaGetLastError();
        if (!copy(p.h_out, a.out.u, u0, u1, cudaMemcpyDeviceToHost, p.d2h)) return cudaGetLastError();
      }
      u0 = u1; a3 = b3; z3 = w3;
    }
  }
  // the CFL estimate after every update; the caller's stream then waits for
  // the back stages and the last output copy
  k_dt_final<<<1, 1, 0, p.back>>>(a.flags, a.dx[0], a.dx[1], a.dx[2], 3, a.cfl);
  nl += 1;
  if (cudaEventRecord(p.back_done, p.back) != cudaSuccess) return cudaGetLastError();
  if (cudaEventRecord(p.d2h_done, p.d2h) != cudaSuccess) return cudaGetLastError();
  if (cudaStreamWaitEvent(st, p.back_done, 0) != cudaSuccess) return cudaGetLastError();
  if (cudaStreamWaitEvent(st, p.d2h_done, 0) != cudaSuccess) return cudaGetLastError();
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
