// Internal declarations shared by the C-ABI translation units.
#pragma once
#include <cstddef>

#include "hydro.h"
#include "hydro_step.cuh"

struct hydro_batch_state;
struct hydro_level_state;
struct hydro_amr_state;

struct hydro_ctx {
  int device = 0;
  double* scratch = nullptr;      // staged-step intermediates (grown on demand)
  size_t scratch_bytes = 0;
  hydro::DevFlags* flags = nullptr;
  int fail_alloc = 0;             // hydro_ctx_fail_allocations: every scratch allocation fails while set
  hydro_batch_state* batch = nullptr;
  hydro_level_state* level = nullptr;
  hydro_amr_state* amr = nullptr;
  long long launches = 0;         // kernels enqueued by this context
  int profiling = 0;              // record stage events around each step
  cudaEvent_t events[hydro::NSTAGES + 1] = {};
  double stage_ms[hydro::NSTAGES] = {};
  long long stage_calls = 0;
  double* host_stage = nullptr;   // device in/out boxes of hydro_advance_box_host (grown on demand)
  size_t host_stage_bytes = 0;
  // copy and back-stage streams and events of the overlapped host-buffer step (made on first use)
  cudaStream_t pipe_h2d = nullptr, pipe_d2h = nullptr, pipe_back = nullptr;
  cudaEvent_t pipe_events[3 * hydro::PIPE_MAX_CHUNKS + 3] = {};
  bool pipe_ready = false;
  // final fluxes through the outer faces of the last recorded box step
  int record_faces = 0;
  double* faces = nullptr;        // 2 * dim face planes, 5 fields each, in (d, side) order
  size_t faces_bytes = 0;
  int faces_dim = 0;              // 0: nothing recorded
  int faces_n[3] = {0, 0, 0};
  // a 3-D box whose whole-box step scratch exceeds this is stepped slab by slab along z (0: never)
  size_t scratch_limit = (size_t)16 << 30;
};

void hydro_batch_release(hydro_ctx* ctx);
void hydro_level_release(hydro_ctx* ctx);
void hydro_amr_release(hydro_ctx* ctx);
size_t hydro_batch_pool_bytes(const hydro_ctx* ctx);
namespace hydro { struct BatchBox; }
// batched step with per-box params; *plan_boxes (nullable) receives the device
// descriptors of the plan that ran (valid until the next batched call).
// direct: enqueue the launches without capturing or caching a plan (for box
// sets that change from call to call).  *enqueue_ms (nullable): host time
// from entry until the step was enqueued (plan or descriptors, tuning, launch)
int hydro_batch_run(hydro_ctx_t* ctx, const hydro_box_t* in, const hydro_box_t* out, int nbox,
                    const hydro_params_t* params, int pstride, const double* dt_dev, double* dt_next_dev,
                    int* bad_first_host, int* bad_all_host, cudaStream_t st, const hydro::BatchBox** plan_boxes,
                    bool direct = false, double* enqueue_ms = nullptr);

namespace hydro {
bool valid_params(const hydro_params_t* p);
bool valid_box(const hydro_box_t* b, int dim);
bool boxes_overlap(const hydro_box_t* a, const hydro_box_t* b, int dim);
BoxGeom geom_of(const hydro_box_t* b, int dim);
StepConst step_const(const hydro_params_t* p, const double dx[3], double dt);
ScratchGeom scratch_geom(const int n[3], int dim);
Scratch carve_scratch(double* base, long long sc);
int ensure_scratch(hydro_ctx* ctx, size_t bytes);
int read_flags(hydro_ctx* ctx, cudaStream_t st, DevFlags* host);
int collect_stage_times(hydro_ctx* ctx, cudaStream_t st);
int record_face_fluxes(hydro_ctx* ctx, const StepArgs& a, const int n[3], int dim, cudaStream_t st);
int ensure_faces(hydro_ctx* ctx, const int n[3], int dim);
int slab_planes(const hydro_ctx* ctx, const ScratchGeom& sg, const int n[3], int dim);
}  // namespace hydro
