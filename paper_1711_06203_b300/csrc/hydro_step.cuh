// Staged CTU-PPM step kernels (FP64, sm_103a).
//
// B300's FP64 pipe issues roughly 1.6 lane-operations per clock per SM (a
// divide or square root costs about 8.6 of those slots) while the FP32/INT
// pipes and HBM have ~75x and ~100x more headroom.  The step is therefore
// laid out for zero redundant FP64 work rather than minimum memory traffic:
// every intermediate (primitive state, traced face states, first,
// intermediate and final fluxes) is computed exactly once over the range its
// consumers need and kept in device scratch (L2-resident for small boxes).
//
// Ranges (zone coordinates, interior [0, n) per axis, ghosts to [-4, n+4)):
//   prim            grown box (ghost zones mapped from the interior by BC kind)
//   trace (per d)   zones [-1, n] on every active axis
//   F1_d            d-faces [0, n_d] x transverse [-1, n]
//   F2_{d|t} (3-D)  d-faces [0, n_d] x t in [0, n_t) x third axis [-1, n]
//   F3_d            d-faces [0, n_d] x transverse interior
//   update          interior
// A face f along d is stored at the position of zone f (between f-1 and f).
#pragma once
#include "hydro_device.cuh"

namespace hydro {

// geometry of a grown box with arbitrary element strides
struct BoxGeom {
  double* u;
  long long sy, sz, sc;  // row, plane, component strides (elements)
  int n[3];
  int gz;                // ghost zones in z: 4 in 3-D, 0 in 2-D
  int bc[3][2];
  __host__ __device__ long long id(int i, int j, int k) const {
    return (long long)(k + gz) * sz + (long long)(j + NG) * sy + (i + NG);
  }
};

// geometry of the contiguous scratch arrays (same zone indexing)
struct ScratchGeom {
  long long sy, sz, sc;
  int gz;
  __host__ __device__ long long id(int i, int j, int k) const {
    return (long long)(k + gz) * sz + (long long)(j + NG) * sy + (i + NG);
  }
};

struct Range {
  int lo[3];
  int ext[3];
  long long count() const { return (long long)ext[0] * ext[1] * ext[2]; }
};

// pencil segments of the tracing sweep: zones [lod, nd] along d (lod = -1:
// the whole range [-1, n_d]) cut into segments of TRACE_SEG, for every
// transverse position in the given ranges
constexpr int TRACE_SEG = 16;
struct SweepRange {
  int lo1, ext1, lo2, ext2;  // transverse axes T1 (thread-fastest) and T2
  int nd, nseg, seg;         // last zone along d, segments per pencil, zones per segment
  int lod;                   // first zone along d
  __host__ __device__ long long count() const { return (long long)ext1 * ext2 * nseg; }
};

// fields of a traced face state: rho, u, v, w, p, then rho*u, rho*v, rho*w, rho*E
enum { TS_MOM = 5, TS_E = 8, TS_FIELDS = 9 };

// scratch field bases
struct Scratch {
  double* Q;          // NQ fields
  double* TM[3];      // traced state at each zone's low face, TS_FIELDS fields
  double* TP[3];      // traced state at each zone's high face, TS_FIELDS fields
  double* F1[3];      // first fluxes
  double* F2[3][3];   // intermediate fluxes F^{d|t}
  double* F3[3];      // final fluxes
};

// number of scratch fields (each one grown box of doubles)
constexpr int SCRATCH_FIELDS = NQ + 3 * TS_FIELDS + 3 * TS_FIELDS + 3 * 5 + 6 * 5 + 3 * 5;

// device reduction / flag block owned by a context
struct DevFlags {
  unsigned long long maxspeed[3];  // bit patterns of max over zones of |u_d| + c (non-negative doubles)
  int bad;                         // sticky non-physical-state flag
  int pad;
  double dt_next;                  // cfl * min_d dx_d / maxspeed_d
};

// stages of a step, timed separately when a context profiles
enum Stage { ST_PRIM = 0, ST_TRACE = 1, ST_FLUX1 = 2, ST_FLUX2 = 3, ST_FLUX3 = 4, ST_UPDATE = 5, NSTAGES = 6 };

struct StepArgs {
  BoxGeom in, out;
  ScratchGeom sg;
  Scratch s;
  StepConst K;
  double dx[3];
  double cfl;
  DevFlags* flags;
  cudaEvent_t* events;   // NSTAGES + 1 events recorded at stage boundaries, or null
};

// enqueue one step (all kernels) on `stream`; adds the number of kernels
// launched to *launches
cudaError_t launch_step(const StepArgs& a, cudaStream_t stream, long long* launches);

// The same step of a 3-D box computed slab by slab along z, T interior planes
// at a time, with scratch for T + 8 planes only (a.sg, a.s: that window,
// unshifted).  Each slab computes every intermediate its planes need from
// the input box itself (the ghost mapping is the whole box's), so planes
// next to a slab boundary are computed by both slabs with the same values:
// the result is bitwise that of launch_step.  `faces` (nullable): record the
// outer-face fluxes slab by slab into this buffer (layout of
// hydro_ctx_face_flux).
cudaError_t launch_step_slabs(const StepArgs& a, int T, double* faces, cudaStream_t stream, long long* launches);
// scratch pointers that index a window of planes starting at plane z0 with
// the whole box's zone coordinates (every pointer moves down by z0 * sz)
Scratch shift_scratch(const Scratch& s, long long shift);
// copy the final fluxes on the outer faces into `faces` (layout of
// hydro_ctx_face_flux): d-faces along x and y over the planes [zlo, zhi),
// the z-faces at 0 and n_z when the planes include the first or last one
cudaError_t launch_record_faces(const StepArgs& a, int zlo, int zhi, double* faces, cudaStream_t stream);

// A 3-D step whose input arrives from, and whose output returns to, host
// memory, with the copies overlapping the kernels: the interior z-planes
// arrive in chunks on one copy stream; after each chunk every stage runs
// over the planes whose inputs have become ready (the z stencils trail the
// landed planes by a few planes), and the planes it finishes go back on a
// second copy stream while the next chunk computes.  The front stages
// (primitive state, tracing, first fluxes) run on the caller's stream and
// the back stages (intermediate and final fluxes, update) on a second
// compute stream, one chunk behind, so that the two fill each other's
// launch tails; they touch disjoint planes.  Every face has a derived
// boundary (ghost zones come from interior zones).  Every zone and face is
// computed once, by the kernels and per-zone arithmetic of launch_step, so
// the result is bitwise the same.
constexpr int PIPE_MAX_CHUNKS = 16;
struct HostPipe {
  const double* h_in;            // host grown boxes in the natural layout
  double* h_out;
  long long field, plane;        // elements per field and per z-plane of the grown box
  int nchunk;                    // z-chunks of the interior, 1..PIPE_MAX_CHUNKS
  int piece;                     // planes per piece of the last chunk's final fluxes and update
  cudaStream_t h2d, d2h;         // copy streams
  cudaStream_t back;             // compute stream of the back stages
  cudaEvent_t start, d2h_done, back_done;
  cudaEvent_t h2d_done[PIPE_MAX_CHUNKS], front_done[PIPE_MAX_CHUNKS], upd_done[PIPE_MAX_CHUNKS];
};
cudaError_t launch_step_host_piped(const StepArgs& a, const HostPipe& p, cudaStream_t stream, long long* launches);

// The plan of launch_step_host_piped: what runs after each input chunk.
// Half-open ranges along z, of planes (x/y quantities, z tracing zones,
// F^{x|z}, F^{y|z}, final x/y fluxes, update) or of z-faces (first,
// intermediate and final z fluxes).  Front stages: primitive state,
// tracing, first fluxes; back stages: intermediate and final fluxes,
// update.
enum PipeRange {
  PR_H2D,   // interior planes copied in with the chunk
  PR_PRIM,  // interior planes whose primitive state is formed
  PR_XY,    // x/y tracing, first x/y fluxes, F^{x|y}, F^{y|x}: planes from -1
  PR_TZ,    // z tracing: zones from -1
  PR_F1Z,   // first z fluxes: z-faces
  PR_F2XZ,  // F^{x|z}, F^{y|z}: planes
  PR_F2Z,   // F^{z|x}, F^{z|y}: z-faces
  PR_F3XY,  // final x and y fluxes: planes
  PR_F3Z,   // final z fluxes: z-faces
  PR_UPD,   // update: planes
  PR_COUNT
};
struct PipeChunk {
  int lo[PR_COUNT], hi[PR_COUNT];
  int ghosts_low, ghosts_high;  // 1: the low (high) ghost planes' primitive state is formed with this chunk
};
// Fills out[0..nchunk) and *pre_lo (the interior planes [pre_lo, nz) are
// copied ahead of chunk 0: the sources of a periodic low face's ghost
// planes).  nz >= NG, 1 <= nchunk <= nz, bc_low in {0 outflow, 1 reflect,
// 2 periodic}.  Returns false on other arguments.
bool pipe_plan(int nz, int nchunk, int bc_low, int* pre_lo, PipeChunk* out);
// enqueue a CFL estimate of the interior of a box into flags->dt_next
cudaError_t launch_dt(const BoxGeom& box, const StepConst& K, const double dx[3], double cfl, DevFlags* flags,
                      cudaStream_t stream, long long* launches);

}  // namespace hydro
