// Allocation-free variant of the box step: the same staged kernels, with
// their scratch and flag block in fixed device storage of this file instead of
// memory a context allocates.
//
// Who needs it: code that must not allocate device memory at all while it
// runs: a host that has already reserved the whole GPU, a real-time loop that
// cannot tolerate the synchronisation a cudaMalloc/cudaFree may imply, or a
// plug-in whose host application owns every allocation.  Such callers still
// pass their own input and output boxes.
//
// The storage below is a file-scope __device__ array: every GPU on which this
// library is loaded holds it (60.1 MiB) until the process exits.  Host code
// must not use the array's name as a pointer (in host code it is only a
// stand-in symbol); the device address is fetched once per device with
// cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "hydro.h"
#include "hydro_api_internal.cuh"

using namespace hydro;

namespace {

constexpr long long NOALLOC_ZONES = HYDRO_NOALLOC_MAX_ZONES;
constexpr long long NOALLOC_DOUBLES = NOALLOC_ZONES * SCRATCH_FIELDS;

// scratch of the staged step followed by the flag block
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES + 8];
static_assert(sizeof(DevFlags) <= 8 * sizeof(double), "flag block must fit the reserved tail");

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mutex;
double* g_dev_scratch[MAX_DEVICES] = {};  // device address of g_noalloc_scratch per device

// once per device, with that device current: fetch the array's device
// address and clear its flag block (the bad-state flag then stays set from
// the call that raised it until a call with dt_next_host reports it)
int noalloc_setup(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_dev_scratch[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return HYDRO_ECUDA;
    }
    if (cudaMemset(static_cast<double*>(p) + NOALLOC_DOUBLES, 0, sizeof(DevFlags)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
      cudaGetLastError();
      return HYDRO_ECUDA;
    }
    g_dev_scratch[device] = static_cast<double*>(p);
  }
  *out = g_dev_scratch[device];
  return HYDRO_OK;
}

}  // namespace

extern "C" int hydro_advance_box_noalloc(const hydro_box_t* in, const hydro_box_t* out,
                                         const hydro_params_t* params, double dt, double* dt_next_host,
                                         void* stream) {
  if (!valid_params(params)) return HYDRO_EINVAL;
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
  ScratchGeom sg = scratch_geom(in->n, dim);
  if (sg.sc > NOALLOC_ZONES) return HYDRO_ETOOBIG;

  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= MAX_DEVICES) {
    cudaGetLastError();
    return HYDRO_ECUDA;
  }
  double* base = nullptr;
  int rc = noalloc_setup(device, &base);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  StepArgs a;
  a.in = geom_of(in, dim);
  a.out = geom_of(out, dim);
  a.sg = sg;
  a.s = carve_scratch(base, sg.sc);
  a.K = step_const(params, in->dx, dt);
  for (int d = 0; d < 3; ++d) a.dx[d] = in->dx[d];
  a.cfl = params->cfl;
  a.flags = reinterpret_cast<DevFlags*>(base + NOALLOC_DOUBLES);
  a.events = nullptr;
  // the flag block keeps the previous call's contents: the step itself resets
  // the speed maxima; the bad-state flag is sticky, so a
  // bad state of a call without dt_next_host is reported by the next call
  // that passes one, which clears it
  if (launch_step(a, st, nullptr) != cudaSuccess) return HYDRO_ECUDA;
  if (dt_next_host) {
    DevFlags h;
    if (cudaMemcpyAsync(&h, a.flags, sizeof(DevFlags), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return HYDRO_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return HYDRO_ECUDA;
    *dt_next_host = h.dt_next;
    if (h.bad) {
      if (cudaMemsetAsync(&a.flags->bad, 0, sizeof(int), st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return HYDRO_ECUDA;
      return HYDRO_EBADSTATE;
    }
  }
  return HYDRO_OK;
}
