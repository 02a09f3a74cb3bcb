// Ghost-zone fill of a level of boxes that tile a rectangular domain, and the
// level time step.  The paper's box iterator works on a level whose boxes
// exchange ghost data through the AMR library (Sec. 3: AMReX manages the grid
// data and parallel communication; Fig. 1 shows a level of uneven boxes).
// Here every ghost zone of every box is filled on the device in one launch:
// its global index is mapped through the domain boundary kind on each axis
// (outflow: nearest domain zone; reflect: mirror image with the normal
// momentum negated; periodic: wrap), and the zone it lands on is copied from
// the box that owns it.  Interior zones are never written, so reads and
// writes cannot collide.  With the boxes' ghosts filled, a batched step
// (hydro_advance_batch with PREFILLED boxes) advances the whole level.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <cstdint>
#include <new>
#include <numeric>
#include <vector>

#include "hydro.h"
#include "hydro_api_internal.cuh"

using namespace hydro;

namespace {

constexpr int FBLOCK = 256;

struct FillBox {
  BoxGeom g;
  int lo[3];       // global index of interior zone (0,0,0)
  long long grown; // zones of the grown box
};

struct FillGeom {
  int dim;
  int domain[3];
  int bc[3][2];
  int G;           // owner-map cell size (divides every box corner and the domain)
  int cells[3];    // owner-map extent
};

__device__ __forceinline__ int domain_map(int i, int n, int bclo, int bchi, bool& flip) {
  if (i < 0) {
    if (bclo == HYDRO_BC_OUTFLOW) return 0;
    if (bclo == HYDRO_BC_REFLECT) { flip = true; return -1 - i; }
    return ((i % n) + n) % n;  // periodic
  }
  if (i >= n) {
    if (bchi == HYDRO_BC_OUTFLOW) return n - 1;
    if (bchi == HYDRO_BC_REFLECT) { flip = true; return 2 * n - 1 - i; }
    return i % n;
  }
  return i;
}

__global__ void __launch_bounds__(FBLOCK) kf_fill(const FillBox* __restrict__ boxes, const int* __restrict__ blk_box,
                                                   const int* __restrict__ box_first, const int* __restrict__ owner,
                                                   FillGeom F) {
  const int b = blk_box[blockIdx.x];
  const FillBox& B = boxes[b];
  const long long t = (long long)(blockIdx.x - box_first[b]) * FBLOCK + threadIdx.x;
  if (t >= B.grown) return;
  const int gx = B.g.n[0] + 2 * NG, gy = B.g.n[1] + 2 * NG;
  int c[3];
  c[0] = (int)(t % gx) - NG;
  c[1] = (int)((t / gx) % gy) - NG;
  c[2] = (F.dim == 3) ? (int)(t / ((long long)gx * gy)) - NG : 0;
  bool ghost = false;
  for (int a = 0; a < F.dim; ++a) ghost |= (c[a] < 0 || c[a] >= B.g.n[a]);
  if (!ghost) return;
  int gi[3] = {0, 0, 0};
  bool flip[3] = {false, false, false};
  for (int a = 0; a < 3; ++a) {
    gi[a] = (a < F.dim) ? domain_map(B.lo[a] + c[a], F.domain[a], F.bc[a][0], F.bc[a][1], flip[a]) : 0;
  }
  const int cell = ((gi[2] / F.G) * F.cells[1] + gi[1] / F.G) * F.cells[0] + gi[0] / F.G;
  const FillBox& O = boxes[owner[F.dim == 3 ? cell : (gi[1] / F.G) * F.cells[0] + gi[0] / F.G]];
  const long long src = O.g.id(gi[0] - O.lo[0], gi[1] - O.lo[1], F.dim == 3 ? gi[2] - O.lo[2] : 0);
  const long long dst = B.g.id(c[0], c[1], c[2]);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    double v = O.g.u[q * O.g.sc + src];
    if (q >= 1 && q <= 3 && flip[q - 1]) v = -v;
    B.g.u[q * B.g.sc + dst] = v;
  }
}

__global__ void k_level_min_dt(const double* __restrict__ dt_next, double* __restrict__ dt, int nbox) {
  __shared__ double red[32];
  double m = HUGE_VAL;
  for (int b = threadIdx.x; b < nbox; b += blockDim.x) m = dmin_nn(m, dt_next[b]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = dmin_nn(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : HUGE_VAL;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = dmin_nn(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) red[0] = m;
  }
  __syncthreads();
  m = red[0];
  for (int b = threadIdx.x; b < nbox; b += blockDim.x) dt[b] = m;
}

}  // namespace

struct FillPlan {
  uint64_t key = 0;
  char* mem = nullptr;  // FillBox[nbox], box_first[nbox], blk_box[nblocks], owner map
  int nbox = 0;
  unsigned nblocks = 0;
  size_t nown = 0;
  FillGeom F{};
  uint64_t last_use = 0;
};

struct hydro_level_state {
  std::vector<FillPlan> plans;
  uint64_t clock = 0;
};

extern "C" int hydro_fill_boundary(hydro_ctx_t* ctx, const hydro_box_t* boxes, const int* lo, int nbox, int dim,
                                   const int* domain, const int* domain_bc, void* stream) {
  if (!ctx || !boxes || !lo || !domain || !domain_bc || nbox < 1 || (dim != 2 && dim != 3)) return HYDRO_EINVAL;
  FillGeom F;
  std::memset(&F, 0, sizeof F);
  F.dim = dim;
  int G = 0;
  for (int a = 0; a < 3; ++a) {
    F.domain[a] = (a < dim) ? domain[a] : 1;
    if (F.domain[a] < 1) return HYDRO_EINVAL;
    for (int s = 0; s < 2; ++s) {
      F.bc[a][s] = (a < dim) ? domain_bc[2 * a + s] : HYDRO_BC_OUTFLOW;
      if (F.bc[a][s] != HYDRO_BC_OUTFLOW && F.bc[a][s] != HYDRO_BC_REFLECT && F.bc[a][s] != HYDRO_BC_PERIODIC)
        return HYDRO_EINVAL;
    }
    if ((F.bc[a][0] == HYDRO_BC_PERIODIC) != (F.bc[a][1] == HYDRO_BC_PERIODIC)) return HYDRO_EINVAL;
    if (a < dim) G = std::gcd(G, F.domain[a]);
  }
  for (int b = 0; b < nbox; ++b) {
    hydro_box_t x = boxes[b];
    for (int a = 0; a < 3; ++a) x.bc[a][0] = x.bc[a][1] = HYDRO_BC_PREFILLED;
    if (!valid_box(&x, dim)) return HYDRO_EINVAL;
    for (int a = 0; a < dim; ++a) {
      if (lo[3 * b + a] < 0 || lo[3 * b + a] + boxes[b].n[a] > F.domain[a]) return HYDRO_EINVAL;
      G = std::gcd(G, std::gcd(lo[3 * b + a], boxes[b].n[a]));
    }
  }
  // a reflected ghost layer mirrors the first NG zones of the domain
  for (int a = 0; a < dim; ++a)
    if ((F.bc[a][0] == HYDRO_BC_REFLECT || F.bc[a][1] == HYDRO_BC_REFLECT) && F.domain[a] < NG) return HYDRO_EINVAL;
  F.G = G;
  for (int a = 0; a < 3; ++a) F.cells[a] = (a < dim) ? F.domain[a] / G : 1;
  // owner map: every cell covered by exactly one box
  const long long ncell = (long long)F.cells[0] * F.cells[1] * F.cells[2];
  if (ncell > (1LL << 27)) return HYDRO_EINVAL;
  std::vector<int> own(ncell, -1);
  for (int b = 0; b < nbox; ++b) {
    int c0[3], c1[3];
    for (int a = 0; a < 3; ++a) {
      c0[a] = (a < dim) ? lo[3 * b + a] / G : 0;
      c1[a] = (a < dim) ? (lo[3 * b + a] + boxes[b].n[a]) / G : 1;
    }
    for (int k = c0[2]; k < c1[2]; ++k)
      for (int j = c0[1]; j < c1[1]; ++j)
        for (int i = c0[0]; i < c1[0]; ++i) {
          int& o = own[((long long)k * F.cells[1] + j) * F.cells[0] + i];
          if (o != -1) return HYDRO_EINVAL;  // overlap
          o = b;
        }
  }
  for (int o : own)
    if (o < 0) return HYDRO_EINVAL;  // the boxes do not cover the domain
  std::vector<FillBox> fb(nbox);
  std::vector<int> first(nbox), blk;
  for (int b = 0; b < nbox; ++b) {
    fb[b].g = geom_of(&boxes[b], dim);
    for (int a = 0; a < 3; ++a) fb[b].lo[a] = (a < dim) ? lo[3 * b + a] : 0;
    fb[b].grown = (long long)(boxes[b].n[0] + 2 * NG) * (boxes[b].n[1] + 2 * NG) *
                  ((dim == 3) ? boxes[b].n[2] + 2 * NG : 1);
    first[b] = (int)blk.size();
    long long nb = (fb[b].grown + FBLOCK - 1) / FBLOCK;
    blk.insert(blk.end(), nb, b);
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return HYDRO_ECUDA;
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return HYDRO_ECUDA;
  struct Restore {
    int dev, prev;
    ~Restore() { if (prev >= 0 && prev != dev) cudaSetDevice(prev); }
  } restore{ctx->device, prev};
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // the fill tables of a level (a plan) are kept on the device and reused by
  // later calls with the same boxes, corners and domain
  if (!ctx->level) {
    ctx->level = new (std::nothrow) hydro_level_state();
    if (!ctx->level) return HYDRO_ENOMEM;
  }
  hydro_level_state* L = ctx->level;
  uint64_t key = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) key = (key ^ c[i]) * 1099511628211ull;
  };
  mix(&nbox, sizeof nbox);
  mix(boxes, nbox * sizeof(hydro_box_t));
  mix(lo, 3 * nbox * sizeof(int));
  mix(&F, sizeof F);
  FillPlan* plan = nullptr;
  for (FillPlan& p : L->plans)
    if (p.key == key) plan = &p;
  if (!plan) {
    const size_t bytes = nbox * sizeof(FillBox) + (nbox + blk.size() + own.size()) * sizeof(int);
    char* mem = nullptr;
    if (cudaMalloc(&mem, bytes) != cudaSuccess) {
      cudaGetLastError();
      return HYDRO_ENOMEM;
    }
    std::vector<char> host(bytes);
    std::memcpy(host.data(), fb.data(), nbox * sizeof(FillBox));
    std::memcpy(host.data() + nbox * sizeof(FillBox), first.data(), nbox * sizeof(int));
    std::memcpy(host.data() + nbox * sizeof(FillBox) + nbox * sizeof(int), blk.data(), blk.size() * sizeof(int));
    std::memcpy(host.data() + nbox * sizeof(FillBox) + (nbox + blk.size()) * sizeof(int), own.data(),
                own.size() * sizeof(int));
    if (cudaMemcpy(mem, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(mem);
      return HYDRO_ECUDA;
    }
    if (L->plans.size() >= 8) {
      // drop the least recently used plan once the device is done with it
      auto lru = std::min_element(L->plans.begin(), L->plans.end(),
                                  [](const FillPlan& x, const FillPlan& y) { return x.last_use < y.last_use; });
      if (cudaDeviceSynchronize() != cudaSuccess) return HYDRO_ECUDA;
      cudaFree(lru->mem);
      L->plans.erase(lru);
    }
    FillPlan np;
    np.key = key;
    np.mem = mem;
    np.nbox = nbox;
    np.nblocks = (unsigned)blk.size();
    np.nown = own.size();
    np.F = F;
    L->plans.push_back(np);
    plan = &L->plans.back();
  }
  plan->last_use = ++L->clock;
  FillBox* d_boxes = reinterpret_cast<FillBox*>(plan->mem);
  int* d_first = reinterpret_cast<int*>(plan->mem + plan->nbox * sizeof(FillBox));
  int* d_blk = d_first + plan->nbox;
  int* d_own = d_blk + plan->nblocks;
  kf_fill<<<plan->nblocks, FBLOCK, 0, st>>>(d_boxes, d_blk, d_first, d_own, plan->F);
  ctx->launches += 1;
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

void hydro_level_release(hydro_ctx* ctx) {
  if (!ctx || !ctx->level) return;
  for (FillPlan& p : ctx->level->plans) cudaFree(p.mem);
  delete ctx->level;
  ctx->level = nullptr;
}

extern "C" int hydro_level_min_dt(const double* dt_next_dev, double* dt_dev, int nbox, void* stream) {
  if (!dt_next_dev || !dt_dev || nbox < 1) return HYDRO_EINVAL;
  k_level_min_dt<<<1, 256, 0, static_cast<cudaStream_t>(stream)>>>(dt_next_dev, dt_dev, nbox);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}
