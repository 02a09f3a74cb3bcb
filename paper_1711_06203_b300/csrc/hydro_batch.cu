// Batched advance of the boxes of one AMR level (paper Sec. 3 and Fig. 1:
// a level is a set of non-uniform boxes that a box iterator hands to the
// compute kernel one by one; Sec. 4 StarLord paragraph).  Here every stage of
// the CTU-PPM step is ONE launch over all boxes of the level: each block
// belongs to one box (found through a per-launch block table) and processes
// that box's work items with the same device bodies as the single-box path.
// The launch sequence of a given set of boxes (a plan) is captured once in a
// CUDA graph and replayed; per-box time steps are read from device memory at
// run time, so one graph serves every step.  The tracing kernel along each
// axis -- a pencil sweep with a given segment length, or the warp-row (x) and
// shared-memory tile (y, z) kernels of the single-box step -- is autotuned
// per box extent.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <vector>

#include "hydro.h"
#include "hydro_api_internal.cuh"
#include "hydro_batch.cuh"
#include "hydro_items.cuh"

namespace hydro {

namespace {

// ---- batched kernels: block -> (box, first block of the box)
__device__ __forceinline__ long long item_of(const int* box_first, int b) {
  return (long long)(blockIdx.x - box_first[b]) * BLOCK + threadIdx.x;
}

// the box of this block: from the per-block table when the plan has one
// (captured plans), else by binary search over the boxes' first blocks
// (direct launches, which then upload nbox ints per launch instead of one
// per block; a box with no blocks in this launch shares its first block
// with the next one, and the search takes the last such box)
__device__ __forceinline__ int box_of_block(const int* __restrict__ blk_box, const int* __restrict__ box_first,
                                            int nbox) {
  if (blk_box) return blk_box[blockIdx.x];
  int lo = 0, hi = nbox - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (box_first[mid] <= (int)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void kb_prepare(BatchBox* boxes, int nbox, const double* __restrict__ dt_dev) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  BatchBox& B = boxes[b];
  const double dt = dt_dev[b];
  B.K.dt = dt;
  B.K.hdt = 0.5 * dt;
  for (int a = 0; a < 3; ++a) B.K.dtdx[a] = (a < B.K.dim) ? dt / B.dx[a] : 0.0;
  B.flags.maxspeed[0] = B.flags.maxspeed[1] = B.flags.maxspeed[2] = 0ull;
  B.flags.bad = 0;
}

__global__ void __launch_bounds__(BLOCK) kb_prim(BatchBox* boxes, const int* __restrict__ blk_box,
                                                 const int* __restrict__ box_first, int nbox) {
  const int b = box_of_block(blk_box, box_first, nbox);
  BatchBox& B = boxes[b];
  prim_item(B.in, B.sg, B.s.Q, B.K, B.rp, &B.flags, item_of(box_first, b));
}

// (three blocks per SM: 168 registers and a few bytes of spills, against
// 195 registers at two; the 512-box level's step 76.6 -> 75.6 ms)
template <int D>
__global__ void __launch_bounds__(BLOCK, 3) kb_trace(const BatchBox* __restrict__ boxes, const int* __restrict__ blk_box,
                                                  const int* __restrict__ box_first, int nbox) {
  const int b = box_of_block(blk_box, box_first, nbox);
  const BatchBox& B = boxes[b];
  trace_item<D>(B.sg, B.s.Q, B.s.TM[D], B.s.TP[D], B.K, B.tr[D], item_of(box_first, b));
}

// the x tracing by warp rows (one warp per ROW_ZONES positions of the pencils laid end to end)
__global__ void __launch_bounds__(BLOCK) kb_trace_row_x(const BatchBox* __restrict__ boxes,
                                                        const int* __restrict__ blk_box,
                                                        const int* __restrict__ box_first, int nbox) {
  const int b = box_of_block(blk_box, box_first, nbox);
  const BatchBox& B = boxes[b];
  trace_row_x_item(B.sg, B.s.Q, B.s.TM[0], B.s.TP[0], B.K, B.tr[0], item_of(box_first, b) >> 5);
}

// the y or z tracing by tiles of 32 pencils x TILE_ZONES zones (one block per tile)
template <int D>
__global__ void __launch_bounds__(BLOCK, 5) kb_trace_tile(const BatchBox* __restrict__ boxes,
                                                          const int* __restrict__ blk_box,
                                                          const int* __restrict__ box_first, int nbox) {
  static_assert(TILE_W * 32 == BLOCK, "a tile is one block");
  __shared__ TileSmem sm;
  const int b = box_of_block(blk_box, box_first, nbox);
  const BatchBox& B = boxes[b];
  trace_tile_item<D>(B.sg, B.s.Q, B.s.TM[D], B.s.TP[D], B.K, B.tr[D], blockIdx.x - box_first[b], sm);
}

template <int D, bool EINF>
__global__ void __launch_bounds__(BLOCK) kb_flux1(const BatchBox* __restrict__ boxes, const int* __restrict__ blk_box,
                                                  const int* __restrict__ box_first, int nbox) {
  const int b = box_of_block(blk_box, box_first, nbox);
  const BatchBox& B = boxes[b];  // the traced-state arrays are written through B.s pointers
  flux1_item<D, EINF>(B.sg, B.s.TP[D], B.s.TM[D], B.s.F1[D], B.K, B.r1[D], item_of(box_first, b));
}

template <int D, int T, bool EINF>
__global__ void __launch_bounds__(BLOCK) kb_flux2(const BatchBox* __restrict__ boxes, const int* __restrict__ blk_box,
                                                  const int* __restrict__ box_first, int nbox) {
  const int b = box_of_block(blk_box, box_first, nbox);
  const BatchBox& B = boxes[b];
  flux2_item<D, T, EINF>(B.sg, B.s.TP[D], B.s.TM[D], B.s.F1[T], B.s.F2[D][T], B.K, B.r2[D][T], item_of(box_first, b));
}

// (held to 64 registers, like the single-box final fluxes: the x-face form
// otherwise takes 94 and loses a third of its resident warps)
template <int D, bool THREE, bool EINF>
__global__ void __launch_bounds__(BLOCK, 65536 / (64 * BLOCK)) kb_flux3(const BatchBox* __restrict__ boxes, const int* __restrict__ blk_box,
                                                  const int* __restrict__ box_first, int nbox) {
  const int b = box_of_block(blk_box, box_first, nbox);
  const BatchBox& B = boxes[b];
  constexpr int T1 = (D == 0) ? 1 : 0, T2 = (D == 2) ? 1 : 2;
  const double* fa = THREE ? B.s.F2[T1][T2] : B.s.F1[T1];
  const double* fb = THREE ? B.s.F2[T2][T1] : nullptr;
  flux3_item<D, EINF>(B.sg, B.s.TP[D], B.s.TM[D], fa, fb, B.s.F3[D], B.K, B.r3[D], item_of(box_first, b));
}

// (held to 64 registers: 100 unbounded; a bound of 6 blocks per SM was no faster)
__global__ void __launch_bounds__(BLOCK, 65536 / (64 * BLOCK))
    kb_update(BatchBox* boxes, const int* __restrict__ blk_box, const int* __restrict__ box_first, int nbox) {
  const int b = box_of_block(blk_box, box_first, nbox);
  BatchBox& B = boxes[b];
  update_item(B.in, B.out, B.sg, B.s.F3[0], B.s.F3[1], B.K.dim == 3 ? B.s.F3[2] : B.s.F3[0], B.K, B.ru, &B.flags,
              item_of(box_first, b));
}

// per box: CFL step of the new state, bad-state flags
__global__ void kb_finalize(BatchBox* boxes, int nbox, double* __restrict__ dt_next_dev, int* __restrict__ bad_out,
                            DevFlags* ctx_flags) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbox) return;
  BatchBox& B = boxes[b];
  dt_final_item(&B.flags, B.dx[0], B.dx[1], B.dx[2], B.K.dim, B.cfl);
  if (dt_next_dev) dt_next_dev[b] = B.flags.dt_next;
  bad_out[b] = B.flags.bad;
  if (B.flags.bad) atomicOr(&ctx_flags->bad, 1);
}

// ---- host side: plans
// L_TRACE: the pencil sweep of the boxes whose tmode[d] is 0; L_TRACE_T: the
// warp rows / tiles of the boxes whose tmode[d] is 1
enum LaunchKind { L_PRIM, L_TRACE, L_TRACE_T, L_FLUX1, L_FLUX2, L_FLUX3, L_UPDATE };

struct LaunchSpec {
  LaunchKind kind;
  int d, t;
  int nblocks;
  size_t map_off;    // offset of blk_box in the plan's map array (ints)
  size_t first_off;  // offset of box_first (nbox ints)
};

struct Plan {
  uint64_t key = 0;
  int nbox = 0, dim = 0;
  bool tables = true;     // per-block box tables in d_maps (else kernels search box_first)
  bool einfeldt = false;  // Einfeldt outer wave speeds (every box shares the flags)
  BatchBox* d_boxes = nullptr;
  int* d_maps = nullptr;
  int* d_bad = nullptr;
  std::vector<LaunchSpec> launches;
  cudaGraphExec_t exec = nullptr;
  uint64_t last_use = 0;
};

uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
  return h;
}

unsigned nblk(long long items) { return (unsigned)((items + BLOCK - 1) / BLOCK); }

void destroy_plan(Plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->d_boxes) cudaFree(p->d_boxes);
  if (p->d_maps) cudaFree(p->d_maps);
  if (p->d_bad) cudaFree(p->d_bad);
  delete p;
}

}  // namespace
}  // namespace hydro

using namespace hydro;

struct hydro_batch_state {
  std::vector<Plan*> plans;
  double* scratch = nullptr;
  size_t scratch_bytes = 0;
  cudaStream_t capture = nullptr;
  uint64_t clock = 0;
  // autotuned tracing kernel per axis and box extent along it (key: tune_key):
  // segments per pencil of the sweep, or 0 for the warp rows / tiles
  std::map<int, int> seg_parts;
  bool tune_loaded = false;
  // direct (uncaptured) launches: descriptors, block tables and flags of the
  // call in flight, rewritten by every call
  BatchBox* d_direct_boxes = nullptr;
  int* d_direct_maps = nullptr;
  int* d_direct_bad = nullptr;
  size_t direct_box_cap = 0, direct_map_cap = 0;
};

namespace {

constexpr int MAX_PLANS = 8;
// tuner candidates per extent: the sweep with 1-4 segments per pencil, or
// (0) the warp-row / tile kernels
const int SEG_PARTS[] = {1, 2, 3, 4, 0};

int tune_key(int d, int nd) { return d * 65536 + nd; }

int segment_length(hydro_batch_state* S, int d, int nd) {
  auto it = S->seg_parts.find(tune_key(d, nd));
  int parts = (it == S->seg_parts.end()) ? -1 : it->second;
  if (parts <= 0) return TRACE_SEG;
  return (nd + 2 + parts - 1) / parts;
}

// the tracing kernel of an extent: 1 the warp rows / tiles, 0 the sweep (also untuned extents)
int trace_mode(hydro_batch_state* S, int d, int nd) {
  auto it = S->seg_parts.find(tune_key(d, nd));
  return (it != S->seg_parts.end() && it->second == 0) ? 1 : 0;
}

// per-box ranges of every stage (same ranges as the single-box launch sequence)
void fill_ranges(BatchBox& B, int dim, hydro_batch_state* S) {
  const int* n = B.in.n;
  for (int ax = 0; ax < 3; ++ax) {
    int g = (ax < 2 || dim == 3) ? NG : 0;
    B.rp.lo[ax] = -g;
    B.rp.ext[ax] = n[ax] + 2 * g;
  }
  Range rt;
  for (int ax = 0; ax < 3; ++ax) {
    bool act = ax < dim;
    rt.lo[ax] = act ? -1 : 0;
    rt.ext[ax] = act ? n[ax] + 2 : 1;
  }
  for (int d = 0; d < 3; ++d) {
    int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
    SweepRange& sw = B.tr[d];
    sw.lo1 = rt.lo[t1]; sw.ext1 = rt.ext[t1];
    sw.lo2 = rt.lo[t2]; sw.ext2 = rt.ext[t2];
    sw.nd = n[d];
    sw.lod = -1;
    sw.seg = (d < dim) ? segment_length(S, d, n[d]) : TRACE_SEG;
    sw.nseg = (n[d] + 2 + sw.seg - 1) / sw.seg;
    B.tmode[d] = (d < dim) ? trace_mode(S, d, n[d]) : 0;
    Range r = rt;
    r.lo[d] = 0;
    r.ext[d] = n[d] + 1;
    B.r1[d] = r;
    Range f;
    for (int ax = 0; ax < 3; ++ax) { f.lo[ax] = 0; f.ext[ax] = (ax < dim) ? n[ax] : 1; }
    f.ext[d] = n[d] + 1;
    B.r3[d] = f;
    for (int t = 0; t < 3; ++t) {
      if (t == d) continue;
      int o = 3 - d - t;
      Range q;
      q.lo[d] = 0; q.ext[d] = n[d] + 1;
      q.lo[t] = 0; q.ext[t] = n[t];
      q.lo[o] = -1; q.ext[o] = n[o] + 2;
      B.r2[d][t] = q;
    }
  }
  for (int ax = 0; ax < 3; ++ax) { B.ru.lo[ax] = 0; B.ru.ext[ax] = (ax < dim) ? n[ax] : 1; }
}

// threads (blocks x BLOCK) of the warp-row / tile tracing of a box along d
long long tile_items(const BatchBox& B, int d) {
  const SweepRange& R = B.tr[d];
  if (d == 0) {
    const long long warps = row_warps(R);
    return (warps + BLOCK / 32 - 1) / (BLOCK / 32) * BLOCK;
  }
  const long long ngroup = ((long long)R.ext1 * R.ext2 + 31) / 32;
  return ngroup * ((R.nd - R.lod + TILE_ZONES) / TILE_ZONES) * BLOCK;
}

long long items_of(const BatchBox& B, LaunchKind k, int d, int t) {
  switch (k) {
    case L_PRIM: return B.rp.count();
    case L_TRACE: return B.tmode[d] ? 0 : B.tr[d].count();
    case L_TRACE_T: return B.tmode[d] ? tile_items(B, d) : 0;
    case L_FLUX1: return B.r1[d].count();
    case L_FLUX2: return B.r2[d][t].count();
    case L_FLUX3: return B.r3[d].count();
    default: return B.ru.count();
  }
}

// solver launches, per wave-speed choice (EINF: Einfeldt, else Davis)
template <bool EINF>
void launch_flux1(int d, unsigned g, const BatchBox* B, const int* bb, const int* bf, int nb, cudaStream_t st) {
  if (d == 0) kb_flux1<0, EINF><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
  if (d == 1) kb_flux1<1, EINF><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
  if (d == 2) kb_flux1<2, EINF><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
}
template <bool EINF>
void launch_flux2(int d, int t, unsigned g, const BatchBox* B, const int* bb, const int* bf, int nb,
                  cudaStream_t st) {
#define F2(DD, TT) \
  if (d == DD && t == TT) kb_flux2<DD, TT, EINF><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
  F2(0, 1) F2(0, 2) F2(1, 0) F2(1, 2) F2(2, 0) F2(2, 1)
#undef F2
}
template <bool EINF>
void launch_flux3(int d, int dim, unsigned g, const BatchBox* B, const int* bb, const int* bf, int nb,
                  cudaStream_t st) {
  if (dim == 3) {
    if (d == 0) kb_flux3<0, true, EINF><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
    if (d == 1) kb_flux3<1, true, EINF><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
    if (d == 2) kb_flux3<2, true, EINF><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
  } else {
    if (d == 0) kb_flux3<0, false, EINF><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
    if (d == 1) kb_flux3<1, false, EINF><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
  }
}

void enqueue_launch(const Plan* p, const LaunchSpec& L, cudaStream_t st) {
  const int* bb = p->tables ? p->d_maps + L.map_off : nullptr;
  const int* bf = p->d_maps + L.first_off;
  const int nb = p->nbox;
  BatchBox* B = p->d_boxes;
  const unsigned g = (unsigned)L.nblocks;
  if (g == 0) return;  // no box of the set takes this kernel
  switch (L.kind) {
    case L_PRIM: kb_prim<<<g, BLOCK, 0, st>>>(B, bb, bf, nb); break;
    case L_TRACE:
      if (L.d == 0) kb_trace<0><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
      if (L.d == 1) kb_trace<1><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
      if (L.d == 2) kb_trace<2><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
      break;
    case L_TRACE_T:
      if (L.d == 0) kb_trace_row_x<<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
      if (L.d == 1) kb_trace_tile<1><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
      if (L.d == 2) kb_trace_tile<2><<<g, BLOCK, 0, st>>>(B, bb, bf, nb);
      break;
    case L_FLUX1:
      if (p->einfeldt) launch_flux1<true>(L.d, g, B, bb, bf, nb, st);
      else launch_flux1<false>(L.d, g, B, bb, bf, nb, st);
      break;
    case L_FLUX2:
      if (p->einfeldt) launch_flux2<true>(L.d, L.t, g, B, bb, bf, nb, st);
      else launch_flux2<false>(L.d, L.t, g, B, bb, bf, nb, st);
      break;
    case L_FLUX3:
      if (p->einfeldt) launch_flux3<true>(L.d, p->dim, g, B, bb, bf, nb, st);
      else launch_flux3<false>(L.d, p->dim, g, B, bb, bf, nb, st);
      break;
    case L_UPDATE: kb_update<<<g, BLOCK, 0, st>>>(B, bb, bf, nb); break;
  }
}

// kernels a launch list enqueues (launches without blocks are skipped)
long long kernels_of(const std::vector<LaunchSpec>& L) {
  long long k = 0;
  for (auto& l : L) k += l.nblocks > 0;
  return k;
}

// the stage launches of a step, in order
std::vector<LaunchSpec> launch_list(int dim) {
  std::vector<LaunchSpec> v;
  v.push_back({L_PRIM, 0, 0, 0, 0, 0});
  for (int d = 0; d < dim; ++d) {
    v.push_back({L_TRACE, d, 0, 0, 0, 0});
    v.push_back({L_TRACE_T, d, 0, 0, 0, 0});
  }
  for (int d = 0; d < dim; ++d) v.push_back({L_FLUX1, d, 0, 0, 0, 0});
  if (dim == 3)
    for (int d = 0; d < 3; ++d)
      for (int t = 0; t < 3; ++t)
        if (t != d) v.push_back({L_FLUX2, d, t, 0, 0, 0});
  for (int d = 0; d < dim; ++d) v.push_back({L_FLUX3, d, 0, 0, 0, 0});
  v.push_back({L_UPDATE, 0, 0, 0, 0, 0});
  return v;
}

// block tables of every launch for the given box descriptors (host): each
// box's first block, and with `blocks` the box of every block
void build_maps(const std::vector<BatchBox>& boxes, std::vector<LaunchSpec>& L, std::vector<int>& maps,
                bool blocks = true) {
  const int nbox = (int)boxes.size();
  maps.clear();
  for (auto& l : L) {
    l.first_off = maps.size();
    maps.resize(maps.size() + nbox);
    long long total = 0;
    for (int b = 0; b < nbox; ++b) {
      maps[l.first_off + b] = (int)total;
      total += nblk(items_of(boxes[b], l.kind, l.d, l.t));
    }
    l.nblocks = (int)total;
    l.map_off = maps.size();
    if (!blocks) continue;
    maps.resize(maps.size() + total);
    for (int b = 0; b < nbox; ++b) {
      long long nb = nblk(items_of(boxes[b], l.kind, l.d, l.t));
      std::fill(maps.begin() + l.map_off + maps[l.first_off + b], maps.begin() + l.map_off + maps[l.first_off + b] + nb,
                b);
    }
  }
}

int ensure_batch_scratch(hydro_ctx* ctx, size_t bytes) {
  hydro_batch_state* S = ctx->batch;
  if (bytes <= S->scratch_bytes) return HYDRO_OK;
  // the pool moves: every plan points into it, so drop them all
  if (cudaDeviceSynchronize() != cudaSuccess) return HYDRO_ECUDA;
  for (Plan* p : S->plans) destroy_plan(p);
  S->plans.clear();
  if (S->scratch) cudaFree(S->scratch);
  S->scratch = nullptr;
  S->scratch_bytes = 0;
  if (ctx->fail_alloc) return HYDRO_ENOMEM;
  if (cudaMalloc(&S->scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    return HYDRO_ENOMEM;
  }
  S->scratch_bytes = bytes;
  return HYDRO_OK;
}

// optional persisted tuning: "axis extent parts" lines in the file named by
// HYDRO_TUNE_CACHE (parts: segments per pencil of the sweep, 0 for the warp
// rows / tiles)
void load_tuning(hydro_batch_state* S) {
  S->tune_loaded = true;
  const char* path = std::getenv("HYDRO_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  int d, nd, parts;
  while (std::fscanf(f, "%d %d %d", &d, &nd, &parts) == 3)
    if (d >= 0 && d < 3 && nd > 0 && nd < 65536 && parts >= 0 && parts <= 8) S->seg_parts[tune_key(d, nd)] = parts;
  std::fclose(f);
}

void save_tuning(const hydro_batch_state* S) {
  const char* path = std::getenv("HYDRO_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "w");
  if (!f) return;
  for (auto& kv : S->seg_parts) std::fprintf(f, "%d %d %d\n", kv.first / 65536, kv.first % 65536, kv.second);
  std::fclose(f);
}

// time the tracing along axis ad over the boxes of sub (one warm-up pass,
// then three), with each box's own choice of kernel along ad
int time_tracing(const std::vector<BatchBox>& sub, int ad, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1,
                 float* ms) {
  std::vector<BatchBox> boxes = sub;
  std::vector<LaunchSpec> L = {{L_TRACE, ad, 0, 0, 0, 0}, {L_TRACE_T, ad, 0, 0, 0, 0}};
  std::vector<int> maps;
  build_maps(boxes, L, maps);
  Plan p;
  p.nbox = (int)boxes.size();
  if (cudaMalloc(&p.d_boxes, boxes.size() * sizeof(BatchBox)) != cudaSuccess ||
      cudaMalloc(&p.d_maps, maps.size() * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (p.d_boxes) cudaFree(p.d_boxes);
    p.d_boxes = nullptr;
    return HYDRO_ENOMEM;
  }
  cudaMemcpyAsync(p.d_boxes, boxes.data(), boxes.size() * sizeof(BatchBox), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(p.d_maps, maps.data(), maps.size() * sizeof(int), cudaMemcpyHostToDevice, st);
  p.launches = L;
  for (int rep = 0; rep < 4; ++rep) {
    if (rep == 1) cudaEventRecord(e0, st);
    for (auto& l : p.launches) enqueue_launch(&p, l, st);
  }
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  *ms = 0.f;
  cudaEventElapsedTime(ms, e0, e1);
  cudaFree(p.d_boxes);
  cudaFree(p.d_maps);
  p.d_boxes = nullptr;
  p.d_maps = nullptr;
  return HYDRO_OK;
}

// the box with tracing kernel `parts` along axis ad (0: warp rows / tiles,
// else the sweep with its pencils cut into that many segments)
BatchBox with_tracing(BatchBox B, int ad, int parts) {
  const int nd = B.in.n[ad];
  B.tmode[ad] = parts == 0 ? 1 : 0;
  if (parts > 0) {
    B.tr[ad].seg = (nd + 2 + parts - 1) / parts;
    B.tr[ad].nseg = (nd + 2 + B.tr[ad].seg - 1) / B.tr[ad].seg;
  }
  return B;
}

// Choose the tracing kernel per (axis d, extent nd) class of untuned boxes.
// The sweep's segment count is timed per class (1-4 segments per pencil).
// The choice between the sweep and the warp-row (x) / tile (y, z) kernels
// is then made per axis, timing all of the axis's untuned boxes both ways:
// a class alone can be a launch of one or two waves, whose tail ranks the
// kernels differently from the step's launch, where all classes run
// together (on the 64-box level the per-class timing kept the sweep for
// y/z classes where the tiles are 20-30 % faster per zone-direction).
// Runs the primitive stage first so the tracing reads real data; writes
// scratch only.
int autotune(hydro_ctx* ctx, std::vector<BatchBox>& boxes, Plan* tmp, int dim) {
  hydro_batch_state* S = ctx->batch;
  std::map<int, std::vector<int>> cls;  // tune_key -> boxes
  for (int b = 0; b < (int)boxes.size(); ++b)
    for (int d = 0; d < dim; ++d) {
      const int key = tune_key(d, boxes[b].in.n[d]);
      if (!S->seg_parts.count(key)) cls[key].push_back(b);
    }
  if (cls.empty()) return HYDRO_OK;
  cudaStream_t st = S->capture;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return HYDRO_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return HYDRO_ECUDA; }
  // primitive state of every box (the plan's first launch)
  enqueue_launch(tmp, tmp->launches[0], st);
  int rc = HYDRO_OK;
  std::map<int, int> sweep_parts;  // tune_key -> best segment count of the sweep
  for (auto& kv : cls) {
    const int ad = kv.first / 65536, nd = kv.first % 65536;
    float best_ms = 1e30f;
    int best = 1;
    for (int parts : SEG_PARTS) {
      if (parts == 0 || (parts > 1 && (nd + 2 + parts - 1) / parts < 4)) continue;
      std::vector<BatchBox> sub;
      for (int b : kv.second) sub.push_back(with_tracing(boxes[b], ad, parts));
      float ms = 0.f;
      rc = time_tracing(sub, ad, st, e0, e1, &ms);
      if (rc) break;
      if (ms < best_ms) { best_ms = ms; best = parts; }
    }
    if (rc) break;
    sweep_parts[kv.first] = best;
  }
  for (int ad = 0; ad < dim && rc == HYDRO_OK; ++ad) {
    std::vector<BatchBox> sweep, rows;
    std::vector<int> keys;
    for (auto& kv : cls) {
      if (kv.first / 65536 != ad) continue;
      keys.push_back(kv.first);
      for (int b : kv.second) {
        sweep.push_back(with_tracing(boxes[b], ad, sweep_parts[kv.first]));
        rows.push_back(with_tracing(boxes[b], ad, 0));
      }
    }
    if (keys.empty()) continue;
    float ms_sweep = 0.f, ms_rows = 0.f;
    rc = time_tracing(sweep, ad, st, e0, e1, &ms_sweep);
    if (rc == HYDRO_OK) rc = time_tracing(rows, ad, st, e0, e1, &ms_rows);
    if (rc) break;
    for (int key : keys) S->seg_parts[key] = (ms_rows < ms_sweep) ? 0 : sweep_parts[key];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess && rc == HYDRO_OK) rc = HYDRO_ECUDA;
  if (rc == HYDRO_OK) save_tuning(S);
  return rc;
}

}  // namespace

size_t hydro_batch_pool_bytes(const hydro_ctx* ctx) { return ctx && ctx->batch ? ctx->batch->scratch_bytes : 0; }

void hydro_batch_release(hydro_ctx* ctx) {
  if (!ctx || !ctx->batch) return;
  hydro_batch_state* S = ctx->batch;
  for (Plan* p : S->plans) destroy_plan(p);
  if (S->scratch) cudaFree(S->scratch);
  if (S->capture) cudaStreamDestroy(S->capture);
  if (S->d_direct_boxes) cudaFree(S->d_direct_boxes);
  if (S->d_direct_maps) cudaFree(S->d_direct_maps);
  if (S->d_direct_bad) cudaFree(S->d_direct_bad);
  delete S;
  ctx->batch = nullptr;
}

// Device descriptors of every box of a batched call: the scratch pool (one
// block per box), per-box constants and stage ranges, sweep segments (tuned
// per size class unless `tune` is off).  Waits for the work queued on `st`.
static int build_boxes(hydro_ctx* ctx, const hydro_box_t* in, const hydro_box_t* out, int nbox,
                       const hydro_params_t* params, int pstride, int dim, bool tune, cudaStream_t st,
                       std::vector<BatchBox>& boxes) {
  hydro_batch_state* S = ctx->batch;
  // the tuner and the pool below write scratch from another stream: let the
  // work already queued on `st` (which may still read scratch) finish first
  if (cudaStreamSynchronize(st) != cudaSuccess) return HYDRO_ECUDA;
  // scratch pool: one scratch block per box
  std::vector<ScratchGeom> sgs(nbox);
  size_t total = 0;
  for (int b = 0; b < nbox; ++b) {
    sgs[b] = scratch_geom(in[b].n, dim);
    total += (size_t)sgs[b].sc * SCRATCH_FIELDS;
  }
  int rc = ensure_batch_scratch(ctx, total * sizeof(double));
  if (rc) return rc;
  boxes.resize(nbox);
  size_t off = 0;
  for (int b = 0; b < nbox; ++b) {
    BatchBox& B = boxes[b];
    std::memset(&B, 0, sizeof B);
    B.in = geom_of(&in[b], dim);
    B.out = geom_of(&out[b], dim);
    B.sg = sgs[b];
    B.s = carve_scratch(S->scratch + off, sgs[b].sc);
    off += (size_t)sgs[b].sc * SCRATCH_FIELDS;
    const hydro_params_t* pb = &params[(size_t)b * pstride];
    B.K = step_const(pb, in[b].dx, 1.0);  // dt fields are set on the device every call
    for (int a = 0; a < 3; ++a) B.dx[a] = in[b].dx[a];
    B.cfl = pb->cfl;
  }
  for (int b = 0; b < nbox; ++b) fill_ranges(boxes[b], dim, S);
  if (tune) {
    // a throw-away plan holding only the primitive stage, for the tuner's input
    Plan tmp;
    tmp.nbox = nbox;
    std::vector<LaunchSpec> L = {{L_PRIM, 0, 0, 0, 0, 0}};
    std::vector<int> maps;
    build_maps(boxes, L, maps);
    tmp.launches = L;
    if (cudaMalloc(&tmp.d_boxes, nbox * sizeof(BatchBox)) != cudaSuccess ||
        cudaMalloc(&tmp.d_maps, maps.size() * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      if (tmp.d_boxes) cudaFree(tmp.d_boxes);
      return HYDRO_ENOMEM;
    }
    cudaMemcpyAsync(tmp.d_boxes, boxes.data(), nbox * sizeof(BatchBox), cudaMemcpyHostToDevice, S->capture);
    cudaMemcpyAsync(tmp.d_maps, maps.data(), maps.size() * sizeof(int), cudaMemcpyHostToDevice, S->capture);
    rc = autotune(ctx, boxes, &tmp, dim);
    cudaStreamSynchronize(S->capture);
    cudaFree(tmp.d_boxes);
    cudaFree(tmp.d_maps);
    if (rc) return rc;
    for (int b = 0; b < nbox; ++b) fill_ranges(boxes[b], dim, S);
  } else {
    for (int b = 0; b < nbox; ++b)
      for (int d = 0; d < 3; ++d) {
        boxes[b].tr[d].seg = TRACE_SEG;
        boxes[b].tr[d].nseg = (boxes[b].in.n[d] + 2 + TRACE_SEG - 1) / TRACE_SEG;
      }
  }
  return HYDRO_OK;
}

// per-box bad-state flags of the call just enqueued (waits for it) when asked for
static int read_bad(const int* d_bad, int nbox, int* bad_first_host, int* bad_all_host, cudaStream_t st) {
  if (!bad_first_host && !bad_all_host) return HYDRO_OK;
  std::vector<int> tmp;
  int* bad = bad_all_host;
  if (!bad) {
    tmp.resize(nbox);
    bad = tmp.data();
  }
  if (cudaMemcpyAsync(bad, d_bad, nbox * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return HYDRO_ECUDA;
  int first = -1;
  for (int b = 0; b < nbox; ++b)
    if (bad[b]) { first = b; break; }
  if (bad_first_host) *bad_first_host = first;
  return first >= 0 ? HYDRO_EBADSTATE : HYDRO_OK;
}

// The same launch sequence enqueued directly, without a graph or a cached
// plan: for callers whose set of boxes changes from call to call (a server
// stepping a different subset of its requests every iteration), where a
// capture per set would cost more than the launches it saves.  Descriptors
// and block tables go to device buffers reused by every direct call, so the
// caller must not overlap two direct calls on one context.
static int run_direct(hydro_ctx* ctx, const hydro_box_t* in, const hydro_box_t* out, int nbox,
                      const hydro_params_t* params, int pstride, int dim, bool tune, const double* dt_dev,
                      double* dt_next_dev, int* bad_first_host, int* bad_all_host, cudaStream_t st,
                      const hydro::BatchBox** plan_boxes, std::chrono::steady_clock::time_point t_entry,
                      double* enqueue_ms) {
  hydro_batch_state* S = ctx->batch;
  std::vector<BatchBox> boxes;
  int rc = build_boxes(ctx, in, out, nbox, params, pstride, dim, tune, st, boxes);
  if (rc) return rc;
  Plan p;  // launch list and first blocks only; the buffers belong to S
  p.nbox = nbox;
  p.dim = dim;
  p.tables = false;
  p.einfeldt = (params[0].flags & HYDRO_FLAG_EINFELDT) != 0;
  p.launches = launch_list(dim);
  std::vector<int> maps;
  build_maps(boxes, p.launches, maps, false);
  if ((size_t)nbox > S->direct_box_cap || maps.size() > S->direct_map_cap) {
    if (S->d_direct_boxes) cudaFree(S->d_direct_boxes);
    if (S->d_direct_maps) cudaFree(S->d_direct_maps);
    if (S->d_direct_bad) cudaFree(S->d_direct_bad);
    S->d_direct_boxes = nullptr;
    S->d_direct_maps = nullptr;
    S->d_direct_bad = nullptr;
    S->direct_box_cap = S->direct_map_cap = 0;
    const size_t nb = std::max<size_t>(2 * (size_t)nbox, 64), nm = std::max<size_t>(2 * maps.size(), 1 << 16);
    if (cudaMalloc(&S->d_direct_boxes, nb * sizeof(BatchBox)) != cudaSuccess ||
        cudaMalloc(&S->d_direct_maps, nm * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&S->d_direct_bad, nb * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return HYDRO_ENOMEM;
    }
    S->direct_box_cap = nb;
    S->direct_map_cap = nm;
  }
  // pageable sources: each copy has left the host vector when the call returns
  if (cudaMemcpyAsync(S->d_direct_boxes, boxes.data(), nbox * sizeof(BatchBox), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(S->d_direct_maps, maps.data(), maps.size() * sizeof(int), cudaMemcpyHostToDevice, st) !=
          cudaSuccess)
    return HYDRO_ECUDA;
  p.d_boxes = S->d_direct_boxes;
  p.d_maps = S->d_direct_maps;
  p.d_bad = S->d_direct_bad;
  const unsigned gb = (unsigned)((nbox + 127) / 128);
  kb_prepare<<<gb, 128, 0, st>>>(p.d_boxes, nbox, dt_dev);
  for (auto& l : p.launches) enqueue_launch(&p, l, st);
  kb_finalize<<<gb, 128, 0, st>>>(p.d_boxes, nbox, dt_next_dev, p.d_bad, ctx->flags);
  if (cudaGetLastError() != cudaSuccess) return HYDRO_ECUDA;
  if (enqueue_ms)
    *enqueue_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_entry).count();
  ctx->launches += kernels_of(p.launches) + 2;
  if (plan_boxes) *plan_boxes = S->d_direct_boxes;
  return read_bad(S->d_direct_bad, nbox, bad_first_host, bad_all_host, st);
}

// Batched step with per-box parameters (params[b * pstride]); all boxes
// share params[0].dim.  bad_all_host (nullable, nbox ints) receives every
// box's bad-state flag, bad_first_host the first bad box index.
int hydro_batch_run(hydro_ctx_t* ctx, const hydro_box_t* in, const hydro_box_t* out, int nbox,
                    const hydro_params_t* params, int pstride, const double* dt_dev, double* dt_next_dev,
                    int* bad_first_host, int* bad_all_host, cudaStream_t st, const hydro::BatchBox** plan_boxes,
                    bool direct, double* enqueue_ms) {
  const auto t_entry = std::chrono::steady_clock::now();
  if (!ctx || !in || !out || nbox < 1 || !dt_dev || !params) return HYDRO_EINVAL;
  const int dim = params[0].dim;
  for (int b = 0; b < nbox; ++b) {
    const hydro_params_t* pb = &params[(size_t)b * pstride];
    if (!valid_params(pb) || pb->dim != dim || pb->flags != params[0].flags) return HYDRO_EINVAL;
  }
  for (int b = 0; b < nbox; ++b) {
    if (!valid_box(&in[b], dim) || !out[b].u || out[b].ng != NG) return HYDRO_EINVAL;
    if (reinterpret_cast<uintptr_t>(out[b].u) % sizeof(double)) return HYDRO_EINVAL;
    hydro_box_t o = out[b];
    for (int a = 0; a < 3; ++a) {
      if (o.n[a] != in[b].n[a]) return HYDRO_EINVAL;
      o.dx[a] = in[b].dx[a];
      o.bc[a][0] = o.bc[a][1] = HYDRO_BC_PREFILLED;
    }
    if (!valid_box(&o, dim) || boxes_overlap(&in[b], &o, dim)) return HYDRO_EINVAL;
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return HYDRO_ECUDA;
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return HYDRO_ECUDA;
  struct Restore {
    int dev, prev;
    ~Restore() { if (prev >= 0 && prev != dev) cudaSetDevice(prev); }
  } restore{ctx->device, prev};

  if (!ctx->batch) {
    ctx->batch = new (std::nothrow) hydro_batch_state();
    if (!ctx->batch) return HYDRO_ENOMEM;
    if (cudaStreamCreateWithFlags(&ctx->batch->capture, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx->batch;
      ctx->batch = nullptr;
      return HYDRO_ECUDA;
    }
  }
  hydro_batch_state* S = ctx->batch;
  if (!S->tune_loaded) load_tuning(S);
  const hydro_params_t* params0 = params;

  // plan key: every box's geometry and pointers, the params, the dt arrays
  uint64_t key = 1469598103934665603ull;
  key = fnv(key, &nbox, sizeof nbox);
  key = fnv(key, in, sizeof(hydro_box_t) * nbox);
  key = fnv(key, out, sizeof(hydro_box_t) * nbox);
  for (int b = 0; b < (pstride ? nbox : 1); ++b) key = fnv(key, &params[(size_t)b * pstride], sizeof(hydro_params_t));
  key = fnv(key, &dt_dev, sizeof dt_dev);
  key = fnv(key, &dt_next_dev, sizeof dt_next_dev);
  const bool tune = !(params0->flags & HYDRO_FLAG_NO_AUTOTUNE);
  key = fnv(key, &tune, sizeof tune);
  if (direct) return run_direct(ctx, in, out, nbox, params, pstride, dim, tune, dt_dev, dt_next_dev,
                                bad_first_host, bad_all_host, st, plan_boxes, t_entry, enqueue_ms);
  Plan* plan = nullptr;
  for (Plan* p : S->plans)
    if (p->key == key) plan = p;

  if (!plan) {
    std::vector<BatchBox> boxes;
    int rc = build_boxes(ctx, in, out, nbox, params, pstride, dim, tune, st, boxes);
    if (rc) return rc;
    plan = new (std::nothrow) Plan();
    if (!plan) return HYDRO_ENOMEM;
    plan->key = key;
    plan->nbox = nbox;
    plan->dim = dim;
    plan->einfeldt = (params0->flags & HYDRO_FLAG_EINFELDT) != 0;
    plan->launches = launch_list(dim);
    std::vector<int> maps;
    build_maps(boxes, plan->launches, maps);
    if (cudaMalloc(&plan->d_boxes, nbox * sizeof(BatchBox)) != cudaSuccess ||
        cudaMalloc(&plan->d_maps, maps.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&plan->d_bad, nbox * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      destroy_plan(plan);
      return HYDRO_ENOMEM;
    }
    if (cudaMemcpyAsync(plan->d_boxes, boxes.data(), nbox * sizeof(BatchBox), cudaMemcpyHostToDevice, S->capture) !=
            cudaSuccess ||
        cudaMemcpyAsync(plan->d_maps, maps.data(), maps.size() * sizeof(int), cudaMemcpyHostToDevice, S->capture) !=
            cudaSuccess ||
        cudaStreamSynchronize(S->capture) != cudaSuccess) {
      destroy_plan(plan);
      return HYDRO_ECUDA;
    }
    // capture the whole step as a graph
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(S->capture, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      destroy_plan(plan);
      return HYDRO_ECUDA;
    }
    const unsigned gb = (unsigned)((nbox + 127) / 128);
    kb_prepare<<<gb, 128, 0, S->capture>>>(plan->d_boxes, nbox, dt_dev);
    for (auto& l : plan->launches) enqueue_launch(plan, l, S->capture);
    kb_finalize<<<gb, 128, 0, S->capture>>>(plan->d_boxes, nbox, dt_next_dev, plan->d_bad, ctx->flags);
    cudaError_t ce = cudaStreamEndCapture(S->capture, &graph);
    if (ce != cudaSuccess || !graph || cudaGraphInstantiate(&plan->exec, graph, 0) != cudaSuccess) {
      cudaGetLastError();
      if (graph) cudaGraphDestroy(graph);
      destroy_plan(plan);
      return HYDRO_ECUDA;
    }
    cudaGraphDestroy(graph);
    if ((int)S->plans.size() >= MAX_PLANS) {
      auto lru = std::min_element(S->plans.begin(), S->plans.end(),
                                  [](const Plan* a, const Plan* b) { return a->last_use < b->last_use; });
      if (cudaStreamSynchronize(st) != cudaSuccess) return HYDRO_ECUDA;
      destroy_plan(*lru);
      S->plans.erase(lru);
    }
    S->plans.push_back(plan);
  }
  plan->last_use = ++S->clock;
  if (plan_boxes) *plan_boxes = plan->d_boxes;
  if (cudaGraphLaunch(plan->exec, st) != cudaSuccess) return HYDRO_ECUDA;
  if (enqueue_ms)
    *enqueue_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_entry).count();
  ctx->launches += kernels_of(plan->launches) + 2;
  return read_bad(plan->d_bad, nbox, bad_first_host, bad_all_host, st);
}

extern "C" int hydro_advance_batch(hydro_ctx_t* ctx, const hydro_box_t* in, const hydro_box_t* out, int nbox,
                                   const hydro_params_t* params, const double* dt_dev, double* dt_next_dev,
                                   int* bad_box_host, void* stream) {
  return hydro_batch_run(ctx, in, out, nbox, params, 0, dt_dev, dt_next_dev, bad_box_host, nullptr,
                         static_cast<cudaStream_t>(stream), nullptr, false);
}

static __global__ void kb_accumulate(double* __restrict__ t, const double* __restrict__ dt) { *t += *dt; }

extern "C" int hydro_advance_box_steps(hydro_ctx_t* ctx, const hydro_box_t* a, const hydro_box_t* b,
                                       const hydro_params_t* params, int nsteps, double* dt_dev, double* t_dev,
                                       void* stream) {
  if (!ctx || !a || !b || !params || !dt_dev || nsteps < 0 || !valid_params(params)) return HYDRO_EINVAL;
  for (int ax = 0; ax < params->dim; ++ax)
    for (int side = 0; side < 2; ++side)
      if (a->bc[ax][side] == HYDRO_BC_PREFILLED || b->bc[ax][side] == HYDRO_BC_PREFILLED) return HYDRO_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < nsteps; ++k) {
    const hydro_box_t* in = (k % 2) ? b : a;
    const hydro_box_t* out = (k % 2) ? a : b;
    double* dt_in = dt_dev + (k % 2);
    double* dt_out = dt_dev + ((k + 1) % 2);
    int rc = hydro_batch_run(ctx, in, out, 1, params, 0, dt_in, dt_out, nullptr, nullptr, st, nullptr);
    if (rc) return rc;
    if (t_dev) {
      kb_accumulate<<<1, 1, 0, st>>>(t_dev, dt_in);
      if (cudaGetLastError() != cudaSuccess) return HYDRO_ECUDA;
      ctx->launches += 1;
    }
  }
  return HYDRO_OK;
}

extern "C" int hydro_batch_tuning(hydro_ctx_t* ctx, int* axis, int* extent, int* segment, int nmax) {
  if (!ctx || nmax < 0 || (nmax > 0 && (!axis || !extent || !segment))) return HYDRO_EINVAL;
  if (!ctx->batch) return 0;
  int k = 0;
  for (auto& kv : ctx->batch->seg_parts) {
    if (k < nmax) {
      axis[k] = kv.first / 65536;
      extent[k] = kv.first % 65536;
      segment[k] = kv.second ? (extent[k] + 2 + kv.second - 1) / kv.second : 0;
    }
    ++k;
  }
  return k;
}
