// C ABI of the CTU-PPM step: context, argument validation, scratch
// management and the box-level entry points declared in include/hydro.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "hydro.h"
#include "hydro_api_internal.cuh"

using namespace hydro;

namespace {
// restores the calling thread's current device on scope exit
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = (prev == dev) || cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

namespace hydro {

bool valid_params(const hydro_params_t* p) {
  if (!p) return false;
  if (p->dim != 2 && p->dim != 3) return false;
  if (!(p->gamma > 1.0) || !std::isfinite(p->gamma)) return false;
  if (!(p->cfl > 0.0) || !(p->cfl <= 1.0)) return false;
  if (!(p->small_dens > 0.0) || !(p->small_pres > 0.0)) return false;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(p->grav[a])) return false;
  return true;
}

bool valid_box(const hydro_box_t* b, int dim) {
  if (!b || !b->u) return false;
  if (reinterpret_cast<uintptr_t>(b->u) % sizeof(double)) return false;
  if (b->ng != NG) return false;
  for (int a = 0; a < 3; ++a)
    if (b->n[a] < 1 || b->n[a] > (1 << 20)) return false;
  if (dim == 2 && b->n[2] != 1) return false;
  const long long gx = b->n[0] + 2 * NG, gy = b->n[1] + 2 * NG;
  const long long gz = (dim == 3) ? b->n[2] + 2 * NG : 1;
  if (b->stride[0] < gx || b->stride[1] < b->stride[0] * gy || b->stride[2] < b->stride[1] * gz) return false;
  for (int a = 0; a < dim; ++a) {
    if (!(b->dx[a] > 0.0) || !std::isfinite(b->dx[a])) return false;
    for (int s = 0; s < 2; ++s)
      if (b->bc[a][s] < HYDRO_BC_OUTFLOW || b->bc[a][s] > HYDRO_BC_PREFILLED) return false;
    if ((b->bc[a][0] == HYDRO_BC_PERIODIC) != (b->bc[a][1] == HYDRO_BC_PERIODIC)) return false;
    // a derived ghost layer copies interior zones, so the axis needs at least NG of them
    bool derived = b->bc[a][0] != HYDRO_BC_PREFILLED || b->bc[a][1] != HYDRO_BC_PREFILLED;
    if (derived && b->n[a] < NG) return false;
  }
  return true;
}

long long box_span(const hydro_box_t* b, int dim) {
  const long long gz = (dim == 3) ? b->n[2] + 2 * NG : 1;
  return 4 * b->stride[2] + (gz - 1) * b->stride[1] + (b->n[1] + 2 * NG - 1) * b->stride[0] + b->n[0] + 2 * NG;
}

bool boxes_overlap(const hydro_box_t* a, const hydro_box_t* b, int dim) {
  const char* a0 = reinterpret_cast<const char*>(a->u);
  const char* b0 = reinterpret_cast<const char*>(b->u);
  const char* a1 = a0 + box_span(a, dim) * (long long)sizeof(double);
  const char* b1 = b0 + box_span(b, dim) * (long long)sizeof(double);
  return a0 < b1 && b0 < a1;
}

BoxGeom geom_of(const hydro_box_t* b, int dim) {
  BoxGeom g;
  g.u = b->u;
  g.sy = b->stride[0];
  g.sz = b->stride[1];
  g.sc = b->stride[2];
  for (int a = 0; a < 3; ++a) {
    g.n[a] = b->n[a];
    g.bc[a][0] = b->bc[a][0];
    g.bc[a][1] = b->bc[a][1];
  }
  g.gz = (dim == 3) ? NG : 0;
  return g;
}

StepConst step_const(const hydro_params_t* p, const double dx[3], double dt) {
  StepConst K;
  K.gamma = p->gamma;
  K.gm1 = p->gamma - 1.0;
  K.gm1inv = 1.0 / (p->gamma - 1.0);
  K.small_dens = p->small_dens;
  K.small_pres = p->small_pres;
  for (int a = 0; a < 3; ++a) K.grav[a] = p->grav[a];
  K.dt = dt;
  K.hdt = 0.5 * dt;
  for (int a = 0; a < 3; ++a) K.dtdx[a] = (a < p->dim) ? dt / dx[a] : 0.0;
  K.dim = p->dim;
  K.flatten = (p->flags & HYDRO_FLAG_NO_FLATTEN) ? 0 : 1;
  K.has_grav = (p->grav[0] != 0.0 || p->grav[1] != 0.0 || p->grav[2] != 0.0) ? 1 : 0;
  K.einfeldt = (p->flags & HYDRO_FLAG_EINFELDT) ? 1 : 0;
  K.flux_grav = (p->flags & HYDRO_FLAG_FLUX_GRAV_ENERGY) ? 1 : 0;
  return K;
}

// scratch geometry of a box of interior n (contiguous, rows padded to even length)
ScratchGeom scratch_geom(const int n[3], int dim) {
  ScratchGeom sg;
  long long gx = n[0] + 2 * NG, gy = n[1] + 2 * NG, gz = (dim == 3) ? n[2] + 2 * NG : 1;
  sg.sy = (gx + 1) & ~1LL;
  sg.sz = sg.sy * gy;
  sg.sc = sg.sz * gz;
  sg.gz = (dim == 3) ? NG : 0;
  return sg;
}

Scratch carve_scratch(double* base, long long sc) {
  Scratch s;
  double* p = base;
  auto take = [&](int nf) { double* r = p; p += (long long)nf * sc; return r; };
  s.Q = take(NQ);
  for (int d = 0; d < 3; ++d) s.TM[d] = take(TS_FIELDS);
  for (int d = 0; d < 3; ++d) s.TP[d] = take(TS_FIELDS);
  for (int d = 0; d < 3; ++d) s.F1[d] = take(5);
  for (int d = 0; d < 3; ++d)
    for (int t = 0; t < 3; ++t) s.F2[d][t] = (t == d) ? nullptr : take(5);
  for (int d = 0; d < 3; ++d) s.F3[d] = take(5);
  return s;
}

int ensure_scratch(hydro_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->scratch_bytes) return HYDRO_OK;
  if (ctx->scratch) {
    if (cudaDeviceSynchronize() != cudaSuccess) return HYDRO_ECUDA;
    cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_bytes = 0;
  }
  if (ctx->fail_alloc) return HYDRO_ENOMEM;
  if (cudaMalloc(&ctx->scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    ctx->scratch = nullptr;
    return HYDRO_ENOMEM;
  }
  ctx->scratch_bytes = bytes;
  return HYDRO_OK;
}

// copy the flag block to the host after the stream drains; clears the bad flag
int read_flags(hydro_ctx* ctx, cudaStream_t st, DevFlags* host) {
  if (cudaMemcpyAsync(host, ctx->flags, sizeof(DevFlags), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return HYDRO_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HYDRO_ECUDA;
  if (host->bad) {
    if (cudaMemsetAsync(&ctx->flags->bad, 0, sizeof(int), st) != cudaSuccess) return HYDRO_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HYDRO_ECUDA;
  }
  return HYDRO_OK;
}

// zones of the transverse interior of a d-face plane
long long face_area(const int n[3], int dim, int d) {
  long long A = 1;
  for (int t = 0; t < dim; ++t)
    if (t != d) A *= n[t];
  return A;
}


int ensure_faces(hydro_ctx* ctx, const int n[3], int dim) {
  size_t need = 0;
  for (int d = 0; d < dim; ++d) need += 2 * 5 * (size_t)face_area(n, dim, d) * sizeof(double);
  ctx->faces_dim = 0;
  if (need > ctx->faces_bytes) {
    if (ctx->faces) cudaFree(ctx->faces);
    ctx->faces = nullptr;
    ctx->faces_bytes = 0;
    if (cudaMalloc(&ctx->faces, need) != cudaSuccess) {
      cudaGetLastError();
      return HYDRO_ENOMEM;
    }
    ctx->faces_bytes = need;
  }
  return HYDRO_OK;
}

// interior planes per slab of a 3-D step whose whole-box scratch exceeds
// the context's limit (balanced slabs of at most the planes the limit
// holds), or 0 to step the box whole
int slab_planes(const hydro_ctx* ctx, const ScratchGeom& sg, const int n[3], int dim) {
  if (dim != 3 || ctx->scratch_limit == 0) return 0;
  const size_t per_plane = (size_t)sg.sz * SCRATCH_FIELDS * sizeof(double);
  if ((size_t)sg.sc * SCRATCH_FIELDS * sizeof(double) <= ctx->scratch_limit) return 0;
  long long tmax = (long long)(ctx->scratch_limit / per_plane) - 2 * NG;
  if (tmax < 1) tmax = 1;
  const long long nslab = (n[2] + tmax - 1) / tmax;
  return (int)((n[2] + nslab - 1) / nslab);
}

int record_face_fluxes(hydro_ctx* ctx, const StepArgs& a, const int n[3], int dim, cudaStream_t st) {
  int rc = ensure_faces(ctx, n, dim);
  if (rc) return rc;
  if (launch_record_faces(a, 0, dim == 3 ? n[2] : 1, ctx->faces, st) != cudaSuccess) return HYDRO_ECUDA;
  ctx->launches += 1;
  ctx->faces_dim = dim;
  for (int t = 0; t < 3; ++t) ctx->faces_n[t] = n[t];
  return HYDRO_OK;
}

// after a profiled step: wait for it and add its stage durations
int collect_stage_times(hydro_ctx* ctx, cudaStream_t st) {
  if (cudaEventSynchronize(ctx->events[NSTAGES]) != cudaSuccess) return HYDRO_ECUDA;
  for (int s = 0; s < NSTAGES; ++s) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->events[s], ctx->events[s + 1]) != cudaSuccess) return HYDRO_ECUDA;
    ctx->stage_ms[s] += ms;
  }
  ctx->stage_calls += 1;
  (void)st;
  return HYDRO_OK;
}

}  // namespace hydro

namespace {
__global__ void k_selftest_scale2(const double* __restrict__ x, double* __restrict__ twice, double* __restrict__ half,
                                  long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  twice[i] = dtwice(x[i]);
  half[i] = dhalf(x[i]);
}
__global__ void k_selftest_divsqrt(const double* __restrict__ x, const double* __restrict__ y,
                                   double* __restrict__ rcp, double* __restrict__ quo, double* __restrict__ sq,
                                   long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  rcp[i] = drcp(x[i]);
  quo[i] = ddiv(y[i], x[i]);
  sq[i] = dsqrt(x[i]);
}
__global__ void k_selftest_rsqrt(const double* __restrict__ x, double* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#ifdef HYDRO_IEEE_DIV_SQRT
  out[i] = 1.0 / sqrt(x[i]);
#else
  out[i] = newton_range(x[i]) ? rsqrt_newton(x[i]) : 1.0 / sqrt(x[i]);
#endif
}
// FP64 issue rate: eight independent multiply-add chains per thread
__global__ void k_selftest_fp64_rate(double* __restrict__ out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += x[c];
  out[(long long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}
__global__ void k_selftest_intpipe(const double* __restrict__ x, const double* __restrict__ y,
                                   double* __restrict__ prod, double* __restrict__ sum, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  prod[i] = mul_i(x[i], y[i]);
  sum[i] = add_i(x[i], y[i]);
}
// z-chunks of the overlapped host-buffer step, and planes per piece of the
// last chunk's final fluxes and update (Sedov 128^3 initial state per call,
// 3.59 ms on the device alone: 4.56 ms with 6 chunks, 4.49 with 8, 4.62
// with 10, 4.81 with 12; pieces of 2, 4, 8 planes with 8 chunks: 4.51,
// 4.49, 4.50; one piece, before the at-rest shortcuts: +0.15 ms)
constexpr int PIPE_CHUNKS = 8, PIPE_PIECE = 4;

// copy and back-stage streams and events of the overlapped host-buffer step
int ensure_pipe(hydro_ctx* ctx) {
  if (ctx->pipe_ready) return HYDRO_OK;
  bool ok = cudaStreamCreateWithFlags(&ctx->pipe_h2d, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&ctx->pipe_d2h, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&ctx->pipe_back, cudaStreamNonBlocking) == cudaSuccess;
  for (auto& e : ctx->pipe_events) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (ctx->pipe_h2d) cudaStreamDestroy(ctx->pipe_h2d);
    if (ctx->pipe_d2h) cudaStreamDestroy(ctx->pipe_d2h);
    if (ctx->pipe_back) cudaStreamDestroy(ctx->pipe_back);
    for (auto& e : ctx->pipe_events) {
      if (e) cudaEventDestroy(e);
      e = nullptr;
    }
    ctx->pipe_h2d = ctx->pipe_d2h = ctx->pipe_back = nullptr;
    return HYDRO_ENOMEM;
  }
  ctx->pipe_ready = true;
  return HYDRO_OK;
}

}  // namespace

extern "C" {

const char* hydro_strerror(int s) {
  switch (s) {
    case HYDRO_OK: return "ok";
    case HYDRO_EINVAL: return "invalid argument";
    case HYDRO_ENOMEM: return "out of memory";
    case HYDRO_ECUDA: return "CUDA runtime error";
    case HYDRO_EBADSTATE: return "non-physical state (rho <= 0, p <= 0 or non-finite)";
    case HYDRO_EAGAIN: return "not ready";
    case HYDRO_ETIMEDOUT: return "timed out";
    case HYDRO_ENOTIMPL: return "not implemented";
    case HYDRO_ETOOBIG: return "box exceeds the fixed storage of the allocation-free step (HYDRO_NOALLOC_MAX_ZONES)";
    case HYDRO_ECANCELED: return "cancelled";
    default: return "unknown status";
  }
}

int hydro_ctx_create(hydro_ctx_t** out, int device) {
  if (!out) return HYDRO_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return HYDRO_ECUDA;
  }
  DeviceGuard g(device);
  if (!g.ok) return HYDRO_ECUDA;
  hydro_ctx* ctx = new (std::nothrow) hydro_ctx();
  if (!ctx) return HYDRO_ENOMEM;
  ctx->device = device;
  if (cudaMalloc(&ctx->flags, sizeof(DevFlags)) != cudaSuccess ||
      cudaMemset(ctx->flags, 0, sizeof(DevFlags)) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->flags) cudaFree(ctx->flags);
    delete ctx;
    return HYDRO_ENOMEM;
  }
  *out = ctx;
  return HYDRO_OK;
}

void hydro_ctx_destroy(hydro_ctx_t* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->flags) cudaFree(ctx->flags);
  for (auto& e : ctx->events)
    if (e) cudaEventDestroy(e);
  hydro_batch_release(ctx);
  hydro_level_release(ctx);
  hydro_amr_release(ctx);
  if (ctx->host_stage) cudaFree(ctx->host_stage);
  if (ctx->pipe_h2d) cudaStreamDestroy(ctx->pipe_h2d);
  if (ctx->pipe_d2h) cudaStreamDestroy(ctx->pipe_d2h);
  if (ctx->pipe_back) cudaStreamDestroy(ctx->pipe_back);
  for (auto& e : ctx->pipe_events)
    if (e) cudaEventDestroy(e);
  if (ctx->faces) cudaFree(ctx->faces);
  delete ctx;
}

int hydro_ctx_check(hydro_ctx_t* ctx) {
  if (!ctx) return HYDRO_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HYDRO_ECUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return HYDRO_ECUDA;
  int bad = 0;
  if (cudaMemcpy(&bad, &ctx->flags->bad, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return HYDRO_ECUDA;
  if (bad) {
    if (cudaMemset(&ctx->flags->bad, 0, sizeof(int)) != cudaSuccess) return HYDRO_ECUDA;
    return HYDRO_EBADSTATE;
  }
  return HYDRO_OK;
}

int hydro_dt(hydro_ctx_t* ctx, const hydro_box_t* box, const hydro_params_t* params, double* dt_host,
             void* stream) {
  if (!ctx || !dt_host || !valid_params(params) || !valid_box(box, params->dim)) return HYDRO_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HYDRO_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  StepConst K = step_const(params, box->dx, 1.0);
  BoxGeom bg = geom_of(box, params->dim);
  if (launch_dt(bg, K, box->dx, params->cfl, ctx->flags, st, &ctx->launches) != cudaSuccess) return HYDRO_ECUDA;
  DevFlags h;
  int rc = read_flags(ctx, st, &h);
  if (rc) return rc;
  *dt_host = h.dt_next;
  return h.bad ? HYDRO_EBADSTATE : HYDRO_OK;
}

int hydro_advance_box(hydro_ctx_t* ctx, const hydro_box_t* in, const hydro_box_t* out,
                      const hydro_params_t* params, double dt, double* dt_next_host, void* stream) {
  if (!ctx || !valid_params(params)) return HYDRO_EINVAL;
  const int dim = params->dim;
  if (!valid_box(in, dim) || !out || !out->u || out->ng != NG) return HYDRO_EINVAL;
  if (reinterpret_cast<uintptr_t>(out->u) % sizeof(double)) return HYDRO_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (out->n[a] != in->n[a]) return HYDRO_EINVAL;
  {
    hydro_box_t o = *out;
    for (int a = 0; a < 3; ++a) { o.dx[a] = in->dx[a]; o.bc[a][0] = o.bc[a][1] = HYDRO_BC_PREFILLED; }
    if (!valid_box(&o, dim)) return HYDRO_EINVAL;
    if (boxes_overlap(in, &o, dim)) return HYDRO_EINVAL;
  }
  if (!(dt > 0.0) || !std::isfinite(dt)) return HYDRO_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HYDRO_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  StepArgs a;
  a.in = geom_of(in, dim);
  a.out = geom_of(out, dim);
  a.sg = scratch_geom(in->n, dim);
  a.K = step_const(params, in->dx, dt);
  for (int d = 0; d < 3; ++d) a.dx[d] = in->dx[d];
  a.cfl = params->cfl;
  a.flags = ctx->flags;
  a.events = ctx->profiling ? ctx->events : nullptr;
  const int T = slab_planes(ctx, a.sg, in->n, dim);
  int rc;
  if (T > 0) {
    // scratch larger than the context's limit: slab by slab along z
    a.sg.sc = a.sg.sz * (T + 2 * NG);
    rc = ensure_scratch(ctx, (size_t)a.sg.sc * SCRATCH_FIELDS * sizeof(double));
    if (rc) return rc;
    a.s = carve_scratch(ctx->scratch, a.sg.sc);
    double* faces = nullptr;
    if (ctx->record_faces) {
      rc = ensure_faces(ctx, in->n, dim);
      if (rc) return rc;
      faces = ctx->faces;
    }
    if (launch_step_slabs(a, T, faces, st, &ctx->launches) != cudaSuccess) return HYDRO_ECUDA;
    if (faces) {
      ctx->faces_dim = dim;
      for (int t = 0; t < 3; ++t) ctx->faces_n[t] = in->n[t];
    }
  } else {
    size_t bytes = (size_t)a.sg.sc * SCRATCH_FIELDS * sizeof(double);
    rc = ensure_scratch(ctx, bytes);
    if (rc) return rc;
    a.s = carve_scratch(ctx->scratch, a.sg.sc);
    if (launch_step(a, st, &ctx->launches) != cudaSuccess) return HYDRO_ECUDA;
    if (ctx->record_faces) {
      rc = record_face_fluxes(ctx, a, in->n, dim, st);
      if (rc) return rc;
    }
  }
  if (ctx->profiling) {
    rc = collect_stage_times(ctx, st);
    if (rc) return rc;
  }
  if (dt_next_host) {
    DevFlags h;
    rc = read_flags(ctx, st, &h);
    if (rc) return rc;
    *dt_next_host = h.dt_next;
    if (h.bad) return HYDRO_EBADSTATE;
  }
  return HYDRO_OK;
}

int hydro_advance_box_host(hydro_ctx_t* ctx, const hydro_box_t* in, const hydro_box_t* out,
                           const hydro_params_t* params, double dt, double* dt_next_host, void* stream) {
  if (!ctx || !in || !out || !in->u || !out->u || !valid_params(params)) return HYDRO_EINVAL;
  const int dim = params->dim;
  if (!valid_box(in, dim)) return HYDRO_EINVAL;
  const long long gx = in->n[0] + 2 * NG, gy = in->n[1] + 2 * NG, gz = (dim == 3) ? in->n[2] + 2 * NG : 1;
  for (const hydro_box_t* b : {in, out}) {
    if (b->stride[0] != gx || b->stride[1] != gx * gy || b->stride[2] != gx * gy * gz || b->ng != NG) return HYDRO_EINVAL;
    for (int a = 0; a < 3; ++a)
      if (b->n[a] != in->n[a]) return HYDRO_EINVAL;
  }
  const size_t elems = (size_t)5 * gx * gy * gz, bytes = elems * sizeof(double);
  {
    const char *a0 = reinterpret_cast<const char*>(in->u), *b0 = reinterpret_cast<const char*>(out->u);
    if (a0 < b0 + bytes && b0 < a0 + bytes) return HYDRO_EINVAL;  // host buffers overlap
  }
  if (!(dt > 0.0) || !std::isfinite(dt)) return HYDRO_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HYDRO_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (2 * bytes > ctx->host_stage_bytes) {
    if (cudaStreamSynchronize(st) != cudaSuccess) return HYDRO_ECUDA;
    if (ctx->host_stage) cudaFree(ctx->host_stage);
    ctx->host_stage = nullptr;
    ctx->host_stage_bytes = 0;
    if (ctx->fail_alloc || cudaMalloc(&ctx->host_stage, 2 * bytes) != cudaSuccess) {
      cudaGetLastError();
      return HYDRO_ENOMEM;
    }
    ctx->host_stage_bytes = 2 * bytes;
  }
  hydro_box_t din = *in, dout = *out;
  din.u = ctx->host_stage;
  dout.u = ctx->host_stage + elems;
  for (int a = 0; a < 3; ++a) dout.dx[a] = in->dx[a];
  // Only the planes the step reads and defines cross the host link: the
  // input's ghost zones are read only on prefilled faces (derived faces map
  // their ghosts onto interior zones), and the output's ghost zones are
  // unspecified.  Each field's interior planes along the slowest axis (z in
  // 3-D, y in 2-D) are one contiguous range, copied flat (strided copies of
  // single rows run far below the link's bandwidth).
  bool prefilled = false;
  for (int a = 0; a < dim; ++a) prefilled |= in->bc[a][0] == HYDRO_BC_PREFILLED || in->bc[a][1] == HYDRO_BC_PREFILLED;
  const long long field = gx * gy * gz;
  const long long plane = (dim == 3) ? gx * gy : gx, nplanes = (dim == 3) ? in->n[2] : in->n[1];
  auto copy_planes = [&](double* dst, const double* src, cudaMemcpyKind kind) {
    for (int c = 0; c < 5; ++c) {
      const long long off = c * field + NG * plane;
      if (cudaMemcpyAsync(dst + off, src + off, (size_t)(nplanes * plane) * sizeof(double), kind, st) != cudaSuccess)
        return false;
    }
    return true;
  };
  int rc;
  const ScratchGeom whole = scratch_geom(in->n, dim);
  if (dim == 3 && !prefilled && !ctx->profiling && slab_planes(ctx, whole, in->n, dim) == 0) {
    // 3-D with derived faces: copies overlap the kernels (launch_step_host_piped)
    rc = ensure_pipe(ctx);
    if (rc) return rc;
    StepArgs a;
    a.in = geom_of(&din, dim);
    a.out = geom_of(&dout, dim);
    a.sg = scratch_geom(in->n, dim);
    rc = ensure_scratch(ctx, (size_t)a.sg.sc * SCRATCH_FIELDS * sizeof(double));
    if (rc) return rc;
    a.s = carve_scratch(ctx->scratch, a.sg.sc);
    a.K = step_const(params, in->dx, dt);
    for (int d = 0; d < 3; ++d) a.dx[d] = in->dx[d];
    a.cfl = params->cfl;
    a.flags = ctx->flags;
    a.events = nullptr;
    HostPipe hp;
    hp.h_in = in->u;
    hp.h_out = out->u;
    hp.field = field;
    hp.plane = plane;
    hp.nchunk = (int)std::min<long long>(PIPE_CHUNKS, in->n[2]);
    hp.piece = PIPE_PIECE;
    hp.h2d = ctx->pipe_h2d;
    hp.d2h = ctx->pipe_d2h;
    hp.back = ctx->pipe_back;
    hp.start = ctx->pipe_events[0];
    hp.d2h_done = ctx->pipe_events[1];
    hp.back_done = ctx->pipe_events[2];
    for (int k = 0; k < PIPE_MAX_CHUNKS; ++k) {
      hp.h2d_done[k] = ctx->pipe_events[3 + k];
      hp.front_done[k] = ctx->pipe_events[3 + PIPE_MAX_CHUNKS + k];
      hp.upd_done[k] = ctx->pipe_events[3 + 2 * PIPE_MAX_CHUNKS + k];
    }
    if (launch_step_host_piped(a, hp, st, &ctx->launches) != cudaSuccess) return HYDRO_ECUDA;
    if (ctx->record_faces) {
      rc = record_face_fluxes(ctx, a, in->n, dim, st);
      if (rc) return rc;
    }
  } else {
    if (prefilled) {
      if (cudaMemcpyAsync(din.u, in->u, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) return HYDRO_ECUDA;
    } else if (!copy_planes(din.u, in->u, cudaMemcpyHostToDevice)) {
      return HYDRO_ECUDA;
    }
    rc = hydro_advance_box(ctx, &din, &dout, params, dt, nullptr, st);
    if (rc) return rc;
    if (!copy_planes(out->u, dout.u, cudaMemcpyDeviceToHost)) return HYDRO_ECUDA;
  }
  DevFlags h;
  rc = read_flags(ctx, st, &h);  // synchronises: the host output is complete on return
  if (rc) return rc;
  if (dt_next_host) *dt_next_host = h.dt_next;
  return h.bad ? HYDRO_EBADSTATE : HYDRO_OK;
}

int hydro_advance_box_retry(hydro_ctx_t* ctx, const hydro_box_t* in, const hydro_box_t* out,
                            const hydro_params_t* params, double dt, int max_retries, double* dt_taken_host,
                            double* dt_next_host, void* stream) {
  if (max_retries < 0 || max_retries > 60) return HYDRO_EINVAL;
  double d = dt;
  for (int attempt = 0; attempt <= max_retries; ++attempt) {
    double next = 0.0;
    int rc = hydro_advance_box(ctx, in, out, params, d, &next, stream);
    if (rc == HYDRO_OK) {
      if (dt_taken_host) *dt_taken_host = d;
      if (dt_next_host) *dt_next_host = next;
      return HYDRO_OK;
    }
    if (rc != HYDRO_EBADSTATE) return rc;
    d *= 0.5;  // the input is untouched (out-of-place step): redo from it
  }
  return HYDRO_EBADSTATE;
}

int hydro_ctx_set_profiling(hydro_ctx_t* ctx, int enable) {
  if (!ctx) return HYDRO_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HYDRO_ECUDA;
  if (enable && !ctx->events[0]) {
    for (auto& e : ctx->events)
      if (cudaEventCreate(&e) != cudaSuccess) return HYDRO_ECUDA;
  }
  ctx->profiling = enable ? 1 : 0;
  for (double& m : ctx->stage_ms) m = 0.0;
  ctx->stage_calls = 0;
  return HYDRO_OK;
}

int hydro_ctx_stage_times(hydro_ctx_t* ctx, double* ms, int nmax, long long* calls) {
  if (!ctx || !ms || nmax < 0) return HYDRO_EINVAL;
  for (int s = 0; s < nmax && s < NSTAGES; ++s) ms[s] = ctx->stage_ms[s];
  if (calls) *calls = ctx->stage_calls;
  return NSTAGES;
}

long long hydro_ctx_launches(const hydro_ctx_t* ctx) { return ctx ? ctx->launches : -1; }

int hydro_ctx_set_scratch_limit(hydro_ctx_t* ctx, size_t bytes) {
  if (!ctx) return HYDRO_EINVAL;
  ctx->scratch_limit = bytes;
  return HYDRO_OK;
}

int hydro_ctx_fail_allocations(hydro_ctx_t* ctx, int enable) {
  if (!ctx) return HYDRO_EINVAL;
  ctx->fail_alloc = enable ? 1 : 0;
  return HYDRO_OK;
}

int hydro_ctx_record_face_fluxes(hydro_ctx_t* ctx, int enable) {
  if (!ctx) return HYDRO_EINVAL;
  ctx->record_faces = enable ? 1 : 0;
  ctx->faces_dim = 0;
  return HYDRO_OK;
}

int hydro_ctx_face_flux(hydro_ctx_t* ctx, int d, int side, double* dst, void* stream) {
  if (!ctx || !dst || side < 0 || side > 1 || ctx->faces_dim == 0 || d < 0 || d >= ctx->faces_dim)
    return HYDRO_EINVAL;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HYDRO_ECUDA;
  long long off = 0;
  for (int e = 0; e < d; ++e) off += 2 * 5 * face_area(ctx->faces_n, ctx->faces_dim, e);
  const long long A = 5 * face_area(ctx->faces_n, ctx->faces_dim, d);
  off += side * A;
  if (cudaMemcpyAsync(dst, ctx->faces + off, (size_t)A * sizeof(double), cudaMemcpyDeviceToDevice,
                      static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return HYDRO_ECUDA;
  return HYDRO_OK;
}

int hydro_selftest_divsqrt(const double* x, const double* y, double* rcp, double* quo, double* sq, long long n,
                           void* stream) {
  if (!x || !y || !rcp || !quo || !sq || n < 0) return HYDRO_EINVAL;
  if (n == 0) return HYDRO_OK;
  k_selftest_divsqrt<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, rcp, quo, sq,
                                                                                                  n);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

int hydro_selftest_intpipe(const double* x, const double* y, double* prod, double* sum, long long n, void* stream) {
  if (!x || !y || !prod || !sum || n < 0) return HYDRO_EINVAL;
  if (n == 0) return HYDRO_OK;
  k_selftest_intpipe<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, y, prod, sum, n);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

int hydro_selftest_rsqrt(const double* x, double* out, long long n, void* stream) {
  if (!x || !out || n < 0) return HYDRO_EINVAL;
  if (n == 0) return HYDRO_OK;
  k_selftest_rsqrt<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, out, n);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

int hydro_pipe_plan(int nz, int nchunk, int bc_low, int* pre_lo, int* out) {
  if (!pre_lo || !out || nchunk < 1 || nchunk > PIPE_MAX_CHUNKS) return HYDRO_EINVAL;
  PipeChunk plan[PIPE_MAX_CHUNKS];
  if (!pipe_plan(nz, nchunk, bc_low, pre_lo, plan)) return HYDRO_EINVAL;
  for (int k = 0; k < nchunk; ++k) {
    int* o = out + 22 * k;
    for (int r = 0; r < PR_COUNT; ++r) {
      o[2 * r] = plan[k].lo[r];
      o[2 * r + 1] = plan[k].hi[r];
    }
    o[20] = plan[k].ghosts_low;
    o[21] = plan[k].ghosts_high;
  }
  return HYDRO_OK;
}

int hydro_selftest_fp64_rate(double* out, int nblocks, int iters, void* stream) {
  if (!out || nblocks < 1 || iters < 1) return HYDRO_EINVAL;
  k_selftest_fp64_rate<<<(unsigned)nblocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(out, iters, 0.999999,
                                                                                        1e-6);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

int hydro_selftest_scale2(const double* x, double* twice, double* half, long long n, void* stream) {
  if (!x || !twice || !half || n < 0) return HYDRO_EINVAL;
  if (n == 0) return HYDRO_OK;
  k_selftest_scale2<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, twice, half, n);
  return cudaGetLastError() == cudaSuccess ? HYDRO_OK : HYDRO_ECUDA;
}

}  // extern "C"
