/* hydro.h — C ABI of the B300-native CTU-PPM hydrodynamics step.
 *
 * One unsplit corner-transport-upwind (CTU) piecewise-parabolic (PPM) Godunov
 * step of the gamma-law Euler equations, with an optional constant-gravity
 * source, on block-structured boxes with ghost zones.  The paper (Sec. 3.2)
 * names Castro's hydrodynamics scheme "an unsplit piecewise parabolic
 * method"; its Sec. 4 GPU paragraph states the execution model kept here: an
 * iterator hands each box's data pointer to a compute kernel that operates on
 * data already resident on the device.  Every stage of the step runs in this
 * library's CUDA kernels (sm_103a, FP64 throughout).
 *
 * Conventions shared by every call
 *  - Pointers marked "device" are CUDA device pointers on the context's
 *    device; "host" pointers are ordinary host memory.  The caller owns every
 *    buffer it passes; the library never frees or retains them after return.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Device work is enqueued on it in order; calls return before it
 *    completes unless a host output (dt_next_host, bad_box_host) is requested,
 *    in which case the call synchronises that stream.
 *  - Return values are hydro_status codes; no call throws or aborts.
 *    Argument errors are reported synchronously and enqueue nothing.
 *  - A context is not thread-safe: use one per host thread.
 *
 * Box layout (hydro_box_t)
 *  - 5 conserved FP64 fields U = (rho, rho*u, rho*v, rho*w, rho*E), each a 3-D
 *    array over the GROWN box: n[a] interior zones plus ng = 4 ghost zones on
 *    both sides of every active axis (x, y; and z when dim = 3).  In 2-D,
 *    n[2] = 1 and z has no ghost zones.
 *  - `u` points at field 0, zone (-4, -4, -4) (2-D: (-4, -4, 0)); zone (i,j,k)
 *    of field c lives at u[c*stride[2] + (k+gz)*stride[1] + (j+4)*stride[0] + (i+4)]
 *    with gz = 4 in 3-D and 0 in 2-D: x is contiguous, stride[0] is the row
 *    pitch (>= n[0]+8), stride[1] the plane pitch (>= stride[0]*(n[1]+8)),
 *    stride[2] the component pitch (>= stride[1]*(n[2]+2*gz)).  Strides are
 *    in elements.
 *  - Ghost zones of an input box are either filled by the caller
 *    (HYDRO_BC_PREFILLED) or derived on the fly from the interior by the
 *    boundary kind of that face; the input box is never written.
 *  - The output box receives the interior of U^{n+1}; its ghost zones are
 *    left unspecified.  Input and output must not overlap.
 */
#ifndef HYDRO_H
#define HYDRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HYDRO_OK = 0,
  HYDRO_EINVAL = -1,     /* invalid argument (nothing enqueued) */
  HYDRO_ENOMEM = -2,     /* device or host allocation failed */
  HYDRO_ECUDA = -3,      /* a CUDA runtime call failed */
  HYDRO_EBADSTATE = -4,  /* a zone held rho <= 0, p <= 0 or a non-finite value */
  HYDRO_EAGAIN = -5,     /* result not ready yet (serve_poll) */
  HYDRO_ETIMEDOUT = -6,  /* a bounded wait ran out */
  HYDRO_ENOTIMPL = -7,   /* not supported by this build */
  HYDRO_ETOOBIG = -8,    /* box larger than the fixed storage of hydro_advance_box_noalloc */
  HYDRO_ECANCELED = -9   /* a served request was cancelled (serve_cancel) */
} hydro_status;

/* boundary kind of one face of a box */
enum {
  HYDRO_BC_OUTFLOW = 0,   /* zero-gradient: ghost = nearest interior zone */
  HYDRO_BC_REFLECT = 1,   /* mirror image, normal momentum negated */
  HYDRO_BC_PERIODIC = 2,  /* wrap around the same box (both faces of the axis) */
  HYDRO_BC_PREFILLED = 3  /* ghost zones hold valid data supplied by the caller */
};

/* hydro_params_t.flags */
#define HYDRO_FLAG_NO_FLATTEN 1u  /* disable Colella-Woodward flattening */
#define HYDRO_FLAG_NO_AUTOTUNE 2u /* hydro_advance_batch: fixed 16-zone sweep segments, no timing runs */
#define HYDRO_FLAG_EINFELDT 4u     /* HLLC outer speeds from Roe averages (Einfeldt) instead of Davis */
#define HYDRO_FLAG_FLUX_GRAV_ENERGY 8u /* gravity energy source from the face mass fluxes (balances the
                                          potential energy exactly) instead of the cell-centred form */

typedef struct {
  double gamma;       /* gamma-law EOS exponent, > 1 */
  double cfl;         /* Courant number for the time-step estimate, in (0, 1] */
  double grav[3];     /* constant gravitational acceleration (0 = none) */
  double small_dens;  /* density floor (> 0), e.g. 1e-200 */
  double small_pres;  /* pressure floor (> 0), e.g. 1e-200 */
  int dim;            /* 2 or 3 */
  unsigned flags;     /* HYDRO_FLAG_* */
} hydro_params_t;

typedef struct {
  double* u;            /* device: field 0 at the first grown zone (see layout above) */
  int n[3];             /* interior zones per axis, >= 1; n[2] = 1 when dim = 2 */
  int ng;               /* ghost zones per side on active axes: must be 4 */
  long long stride[3];  /* element strides: row, plane, component */
  double dx[3];         /* zone widths, > 0 on active axes */
  int bc[3][2];         /* boundary kind per axis (x, y, z) and side (low, high) */
} hydro_box_t;

typedef struct hydro_ctx hydro_ctx_t;

/* Create a context on CUDA device `device`.  The context owns the scratch
 * memory of the staged step (grown on demand to the largest box seen), the
 * device flags for bad-state detection and the reduction buffers of the CFL
 * estimate.  Returns HYDRO_ECUDA if the device cannot be used. */
int hydro_ctx_create(hydro_ctx_t** ctx, int device);

/* Release a context and everything it owns.  Synchronises its device. NULL is a no-op. */
void hydro_ctx_destroy(hydro_ctx_t* ctx);

/* Human-readable name of a status code (static storage). */
const char* hydro_strerror(int status);

/* CFL time step of a box (paper Sec. 3.1: a compressible step is limited by
 * the sound speed): dt = cfl * min over interior zones and active directions
 * d of dx_d / (|u_d| + c), c = sqrt(gamma p / rho).  Writes the value to
 * *dt_host (host) after synchronising `stream`.  HYDRO_EBADSTATE if any
 * interior zone is non-physical. */
int hydro_dt(hydro_ctx_t* ctx, const hydro_box_t* box, const hydro_params_t* params, double* dt_host,
             void* stream);

/* Advance one box by dt with one CTU-PPM step (paper Sec. 3.2's unsplit PPM;
 * Sec. 4's box-at-a-time kernel call): in -> out, out of place.
 *  - in, out: boxes of identical interior size on the same device (strides may
 *    differ); `in` is only read.
 *  - dt: the step, > 0.
 *  - dt_next_host: NULL, or host memory that receives the CFL step of U^{n+1}
 *    (the call then synchronises `stream` and also reports HYDRO_EBADSTATE
 *    for a non-physical input or result).  With NULL the call is fully
 *    asynchronous; a bad state is then recorded in the context and reported by
 *    the next hydro_ctx_check().
 *  - Every grown-box zone of `in` that the stencil reads must hold a physical
 *    state. */
int hydro_advance_box(hydro_ctx_t* ctx, const hydro_box_t* in, const hydro_box_t* out,
                      const hydro_params_t* params, double dt, double* dt_next_host, void* stream);

/* Advance every box of a level by one CTU-PPM step in one batched, graph-
 * captured launch sequence (paper Sec. 3: a level is a set of boxes of uneven
 * sizes that the box iterator hands to the kernel one by one; Fig. 1).
 *  - in[b], out[b] (host arrays of nbox descriptors): as for hydro_advance_box,
 *    box by box; all boxes share `params` (dim, gamma, gravity, flags).
 *  - dt_dev: device array of nbox steps, read when the step runs (an AMR
 *    level passes its level dt replicated); values are not checked.
 *  - dt_next_dev: NULL or a device array receiving each box's CFL step of
 *    U^{n+1}.
 *  - bad_box_host: NULL, or host memory receiving the index of the first box
 *    that met a non-physical zone (-1 if none); the call then synchronises
 *    `stream` and returns HYDRO_EBADSTATE for a bad box.  Without it a bad
 *    state is recorded in the context (hydro_ctx_check).
 *  - The first call for a given set of descriptors, params and dt arrays
 *    builds a plan: per-box work tables, scratch for all boxes in one
 *    context-owned pool, the tracing kernel per axis and box extent (a
 *    pencil sweep with 1-4 segments per pencil, or the warp-row / tile
 *    kernels; timed on
 *    the boxes unless HYDRO_FLAG_NO_AUTOTUNE, which takes 16-zone sweep
 *    segments; remembered in the context, and in the file named by the
 *    environment variable HYDRO_TUNE_CACHE if set) and a CUDA graph of the
 *    whole step.  Later
 *    calls with the same descriptors replay the graph; the context keeps the
 *    8 most recent plans.  Plans of one context share the scratch pool: do not
 *    run two batched steps of one context concurrently. */
int hydro_advance_batch(hydro_ctx_t* ctx, const hydro_box_t* in, const hydro_box_t* out, int nbox,
                        const hydro_params_t* params, const double* dt_dev, double* dt_next_dev, int* bad_box_host,
                        void* stream);

/* Advance one box nsteps CTU-PPM steps with the time step kept on the device,
 * with no host synchronisation between steps (paper Sec. 3: the time loop of a
 * level; here it runs as replays of two captured step graphs, which removes
 * the per-step host round trip that bounds small boxes).
 *  - a, b: two device boxes of the same interior size (as for
 *    hydro_advance_box); step k goes a -> b for even k, b -> a for odd k, so
 *    the result is in b after an odd number of steps and in a after an even
 *    one.  No face may be HYDRO_BC_PREFILLED (its ghosts would be stale after
 *    the first step): HYDRO_EINVAL.
 *  - dt_dev: device array of 2 doubles; dt_dev[0] holds the first step's dt
 *    on entry (e.g. from hydro_dt).  Step k takes dt_dev[k % 2] and writes
 *    the CFL step of its result to dt_dev[(k + 1) % 2], so after the call
 *    dt_dev[nsteps % 2] is the next step's dt.
 *  - t_dev: NULL, or a device double to which every step's dt is added.
 *  - A non-physical state is recorded in the context (hydro_ctx_check).
 *  - Asynchronous on `stream`; shares the batched step's plans and scratch
 *    pool (do not overlap with hydro_advance_batch on the same context). */
int hydro_advance_box_steps(hydro_ctx_t* ctx, const hydro_box_t* a, const hydro_box_t* b,
                            const hydro_params_t* params, int nsteps, double* dt_dev, double* t_dev, void* stream);

/* Fill every ghost zone of a level of boxes that tile a rectangular domain
 * (paper Sec. 3: the AMR library manages a level's grid data and ghost
 * exchange; Fig. 1: a level of uneven boxes).
 *  - boxes[b] (host array): the level's boxes (device data); their bc fields
 *    are ignored.  lo (host, 3*nbox ints): global index of each box's interior
 *    zone (0,0,0); the boxes must cover [0, domain) exactly, without overlap.
 *  - domain (host, dim ints): zones per axis; domain_bc (host, 2*dim ints):
 *    HYDRO_BC_OUTFLOW / REFLECT / PERIODIC for the low and high face of each
 *    axis (periodic on both faces or neither).
 *  - Each ghost zone's global index is mapped through the domain boundary kind
 *    per axis (the same per-axis maps as a single box's derived ghosts) and
 *    copied from the box owning the zone it lands on.  Only ghost zones are
 *    written.  Asynchronous on `stream`; the fill tables of a level are built
 *    on the first call and kept in the context (the 8 most recent levels).
 *  After the fill, advance the level with hydro_advance_batch on the same
 *  boxes marked HYDRO_BC_PREFILLED. */
int hydro_fill_boundary(hydro_ctx_t* ctx, const hydro_box_t* boxes, const int* lo, int nbox, int dim,
                        const int* domain, const int* domain_bc, void* stream);

/* Level time step: dt_dev[b] = min over all boxes of dt_next_dev[b'] (the AMR
 * level advances every box with the same dt).  Device arrays of nbox doubles;
 * enqueued on `stream`. */
int hydro_level_min_dt(const double* dt_next_dev, double* dt_dev, int nbox, void* stream);

/* The autotuned tracing kernels of a context: up to nmax triples (axis, box
 * extent along it, zones per pencil segment of the sweep or 0 for the
 * warp-row (x) / shared-memory tile (y, z) kernels) into the host arrays
 * axis/extent/segment.  Returns the number of tuned (axis, extent) classes. */
int hydro_batch_tuning(hydro_ctx_t* ctx, int* axis, int* extent, int* segment, int nmax);

/* hydro_advance_box on host buffers: in->u and out->u point to host memory
 * (pinned or pageable) holding grown boxes in the natural layout (stride[0]
 * = nx+8, stride[1] = stride[0]*(ny+8), stride[2] = stride[1]*(nz+8, or 1
 * in 2-D), 5 components).  The call copies the input to context-owned device
 * memory, runs the step, copies the result back and returns once the host
 * output is complete.  Only what the step reads and defines crosses the host
 * link: with a HYDRO_BC_PREFILLED face the whole input box goes over (its
 * ghost layers are data); otherwise only interior zones are read (derived
 * faces map their ghosts onto the interior), so each field's interior planes
 * along the slowest axis -- in 3-D only their interior rows -- go over.  The
 * output comes back the same way; the host output's ghost zones outside the
 * copied rows and planes are not written, and those inside are unspecified.
 * In 3-D with no prefilled face the copies run on two context-owned copy
 * streams in z-chunks that overlap the kernels (fully so with pinned host
 * buffers): the front stages run on `stream`, the back stages on a third
 * context-owned stream, and `stream` waits for all of them before the call
 * returns; otherwise everything runs on `stream`.
 * dt_next_host (nullable) receives the CFL step of the result; a
 * non-physical state returns HYDRO_EBADSTATE.  HYDRO_EINVAL for other
 * layouts or overlapping host buffers. */
int hydro_advance_box_host(hydro_ctx_t* ctx, const hydro_box_t* in, const hydro_box_t* out,
                           const hydro_params_t* params, double dt, double* dt_next_host, void* stream);

/* hydro_advance_box with the retry mechanism of paper Sec. 3.2 (Castro can
 * redo a step based on criteria evaluated during the integration): if the
 * step meets a non-physical state (rho <= 0, p <= 0 or non-finite, in the
 * input or the result), it is redone from the untouched input with half the
 * time step, up to max_retries (0..60) times.  *dt_taken_host (host,
 * nullable) receives the step that succeeded, *dt_next_host (nullable) the
 * CFL step of its result.  Synchronises `stream` after every attempt.
 * HYDRO_EBADSTATE if every attempt failed (e.g. a bad input state). */
int hydro_advance_box_retry(hydro_ctx_t* ctx, const hydro_box_t* in, const hydro_box_t* out,
                            const hydro_params_t* params, double dt, int max_retries, double* dt_taken_host,
                            double* dt_next_host, void* stream);

/* A two-level hierarchy, refinement ratio 2 in space and time (paper Sec. 3:
 * block-structured AMR with subcycling in time; Castro advances the coarse
 * level, then the fine level in smaller steps to the same time, then
 * synchronises the two).  All arrays are host arrays of descriptors; box data
 * live on the device. */
typedef struct {
  int dim;                        /* 2 or 3 */
  int domain[3];                  /* coarse zones per axis (unused axes: 1) */
  int domain_bc[3][2];            /* OUTFLOW / REFLECT / PERIODIC, low and high face per axis */
  int ncoarse;                    /* coarse boxes, tiling [0, domain) exactly */
  const hydro_box_t* coarse_in;   /* state at t; ghost zones are overwritten */
  const hydro_box_t* coarse_out;  /* receives the synchronised state at t + dt */
  const int* coarse_lo;           /* 3 ints per box: global index of interior zone (0,0,0) */
  int nfine;                      /* fine boxes (0 allowed) */
  const hydro_box_t* fine_in;     /* fine state at t; ghost zones are overwritten */
  const hydro_box_t* fine_out;    /* receives the fine state at t + dt */
  const int* fine_lo;             /* 3 ints per box, in the fine index space (2x the coarse) */
} hydro_amr_t;

/* One coarse step of a two-level hierarchy (Berger-Colella subcycling):
 *   1. coarse ghost fill (domain boundary kinds) and a batched step of dt;
 *   2. two fine steps of dt/2, each after a fine ghost fill: a ghost zone is
 *      copied from the fine box that covers it, else interpolated from the
 *      coarse level -- in time first (the coarse state at t for the first
 *      step, 0.5 U(t) + 0.5 U(t+dt) for the second), then in space (linear
 *      with a monotonised-central slope per axis, conservative);
 *   3. reflux: each uncovered coarse zone next to the fine region gets the
 *      coarse flux through each shared face replaced by the fine fluxes
 *      through it, averaged over the 2^(dim-1) fine faces and both fine steps;
 *   4. average down: each covered coarse zone becomes the mean of its children.
 * Coarse boxes share one spacing dx; fine boxes have dx/2 exactly.  Fine boxes
 * have even corners and sizes, do not overlap, and lie, coarsened and grown by
 * 3 coarse zones, inside the domain (so their ghosts and the interpolation
 * stencil only see coarse interior zones).  The box descriptors' bc fields
 * are ignored.  dt_dev (device, 1 double): the coarse step.  dt_next_dev
 * (device, 1 double): receives min(CFL step of the synchronised coarse level,
 * 2 x CFL step of the fine level).  bad_host (host, nullable): if given, the
 * call synchronises `stream` and stores 1 if any step met a non-physical
 * state (then returns HYDRO_EBADSTATE), else 0.  The fine state after the
 * first step lives in context-owned memory.  The tables of a hierarchy are
 * built on the first call and kept (the 4 most recent).  HYDRO_EINVAL for a
 * hierarchy that breaks the rules above; HYDRO_ENOTIMPL with
 * HYDRO_FLAG_FLUX_GRAV_ENERGY (the reflux corrects hydrodynamic fluxes only).
 * Asynchronous on `stream` otherwise. */
int hydro_amr_advance(hydro_ctx_t* ctx, const hydro_amr_t* h, const hydro_params_t* params, const double* dt_dev,
                      double* dt_next_dev, int* bad_host, void* stream);

/* One method-of-lines step of a box carrying nspec passive species (paper
 * Sec. 4: StarLord, the GPU proxy of Castro, keeps the hydrodynamics and the
 * EOS, writes the hydrodynamics as a simple method of lines and advects 13
 * nuclear species).
 *  - Semi-discrete form dU/dt = -sum_d (F_d(hi face) - F_d(lo face))/dx_d + S:
 *    F_d is the HLLC flux of the flattened, limited PPM edge values of the
 *    primitive variables (rho, u, v, w, p, X_k) at the stage time, without
 *    characteristic tracing or transverse terms; the species flux is the mass
 *    flux times the mass fraction of the HLLC upwind side (S* >= 0: left);
 *    S = (0, rho g, (rho u).g).  Time: two-stage SSP Runge-Kutta,
 *    U1 = U + dt L(U), U' = U/2 + (U1 + dt L(U1))/2.
 *  - in/out: boxes of 5 + nspec components (stride[2] apart): rho, rho u,
 *    rho v, rho w, rho E, then rho X_1 .. rho X_nspec.  Derived boundary faces
 *    are refilled from each stage's state; prefilled ghost layers are the
 *    caller's data at t and serve both stages.
 *  - 0 <= nspec <= HYDRO_MOL_MAX_SPECIES.  dt_next_host (nullable) as in
 *    hydro_advance_box (CFL step of the result; synchronises the stream; a
 *    non-physical state returns HYDRO_EBADSTATE).  HYDRO_ENOTIMPL with
 *    HYDRO_FLAG_FLUX_GRAV_ENERGY.  Scratch: 7 (5 + nspec) + 1 grown-box
 *    fields of the context's scratch. */
#define HYDRO_MOL_MAX_SPECIES 32
int hydro_mol_advance_box(hydro_ctx_t* ctx, const hydro_box_t* in, const hydro_box_t* out,
                          const hydro_params_t* params, int nspec, double dt, double* dt_next_host, void* stream);

/* Report and clear the context's sticky bad-state flag: synchronises the
 * context's device, returns HYDRO_EBADSTATE if any step since the last check
 * met a non-physical zone, else HYDRO_OK. */
int hydro_ctx_check(hydro_ctx_t* ctx);

/* ---- serving: continuous batching of independent problems ----
 * A server owns a context, a stream and a scheduler thread.  Requests are
 * admitted in arrival order while their device footprint (two copies of the
 * grown state, plus the step scratch the scheduling policy can need) fits the
 * HBM budget and a slot is free.  Every scheduler iteration then advances a
 * set of admitted requests by one CTU-PPM step in a single batched step
 * (hydro_advance_batch's engine), each with its own gamma and CFL time step,
 * so requests that arrive while others run join the next iteration.  Which
 * requests step is the policy's choice (serve_set_policy).  Finished requests
 * are retired and their memory released.  All serve_* calls are
 * thread-safe. */
enum { HYDRO_PROB_SOD = 0, HYDRO_PROB_SEDOV = 1, HYDRO_PROB_TWO_STATE = 2 };

typedef struct {
  int kind;             /* HYDRO_PROB_*: 3-D problem on the unit cube, outflow boundaries */
  int n;                /* zones per side (cubic box), 4..1024 */
  int steps;            /* CTU-PPM steps to take, >= 1 */
  double gamma;         /* gamma-law exponent, > 1 */
  double cfl;           /* Courant number, (0, 1] */
  double rho_l, p_l;    /* Sod / two-state: state at x < 0.5 (at rest) */
  double rho_r, p_r;    /*                  state at x >= 0.5 (at rest) */
  double energy;        /* Sedov: blast energy, deposited as pressure within 4 zones of the centre */
  double p_ambient;     /* Sedov: ambient pressure (density 1) */
  double* result_host;  /* NULL, or host memory for 5*(n+8)^3 doubles: the final grown state (interior
                           valid), written before the request completes; owned by the caller */
} hydro_request_t;

typedef struct {
  int status;              /* HYDRO_OK, or the error that retired the request */
  int steps_done;
  double t_final;          /* simulated time reached */
  double latency_ms;       /* submit -> result ready */
  double queue_ms;         /* submit -> admitted */
  long long zone_updates;  /* steps_done * n^3 */
} hydro_result_t;

typedef struct {
  int queued, active;
  long long admitted, completed, iterations, zone_updates;
  double busy_ms;           /* time the scheduler spent in batched steps (enqueue + device) */
  size_t hbm_budget, hbm_states, hbm_scratch_pool;
  long long box_steps;      /* box steps taken (a batched iteration of k boxes counts k) */
  double enqueue_ms;        /* host time choosing sets, building descriptors, tuning, enqueueing */
  double ms_per_unit;       /* measured cost of one step per (n+3)^3 zones, ms */
} hydro_serve_stats_t;

/* Scheduling policies (serve_set_policy). */
enum {
  HYDRO_SERVE_ALL = 0,            /* every admitted request steps every iteration */
  HYDRO_SERVE_RESPONSE_RATIO = 1  /* default: highest (waited + remaining work) / remaining work first,
                                     within a per-iteration GPU-time quantum */
};

typedef struct serve serve_t;

/* Create a server on `device` with an HBM budget in bytes (0: 80% of the free
 * memory at creation) and at most max_slots concurrently active requests. */
int serve_create(serve_t** s, int device, size_t hbm_budget_bytes, int max_slots);
/* Queue a request (copied); *id receives its handle.  HYDRO_ETOOBIG if it can
 * never fit the budget, HYDRO_EINVAL for bad parameters. */
int serve_submit(serve_t* s, const hydro_request_t* req, uint64_t* id);
/* Wait up to timeout_ms (0: do not wait, < 0: forever) for request `id`.
 * HYDRO_OK: *res filled and the handle released; HYDRO_EAGAIN (timeout 0) or
 * HYDRO_ETIMEDOUT: not finished yet; HYDRO_EINVAL: unknown handle. */
int serve_poll(serve_t* s, uint64_t id, hydro_result_t* res, int timeout_ms);
/* Cancel request `id`.  A request still queued leaves the queue at once; an
 * admitted one is retired before the scheduler's next iteration (its memory
 * freed, the steps done so far reported); either way its result, collected
 * by serve_poll as usual, carries status HYDRO_ECANCELED and no state is
 * copied to result_host.  A request that has already finished keeps its
 * result.  HYDRO_EINVAL: unknown (or already collected) handle. */
int serve_cancel(serve_t* s, uint64_t id);
/* Snapshot of the server's counters. */
int serve_stats(serve_t* s, hydro_serve_stats_t* st);
/* Choose the scheduling policy while the server is idle (nothing queued or
 * active; else HYDRO_EAGAIN).  HYDRO_SERVE_RESPONSE_RATIO: each iteration
 * steps the requests in decreasing order of (time since submission +
 * remaining work) / remaining work, where remaining work = steps left x the
 * measured cost of one step of that box size, adding requests while the
 * iteration's estimated GPU time stays within quantum_ms (the first request
 * always steps); only the stepped set needs step scratch, so the admission
 * reserve is the largest box's scratch plus what a quantum can hold.
 * HYDRO_SERVE_ALL: every admitted request steps every iteration (quantum_ms
 * ignored) and the reserve is the scratch of every admitted request.  The
 * default is HYDRO_SERVE_RESPONSE_RATIO with a 2.5 ms quantum.  Either way a
 * request's result does not depend on the policy or on the other requests. */
int serve_set_policy(serve_t* s, int policy, double quantum_ms);
/* Stop the scheduler (the step in flight completes), release everything;
 * requests not yet polled are dropped.  NULL is a no-op. */
void serve_destroy(serve_t* s);

/* ---- allocation-free step (the paper has no counterpart) ----
 * For callers that cannot allocate device memory while they run: a host that
 * has reserved the whole GPU for itself, a real-time loop that cannot afford
 * the device-wide synchronisation an allocation or free may cause, or a
 * plug-in whose host owns every allocation.  The step is the same as
 * hydro_advance_box, but its scratch lives in fixed device storage of the
 * library: no context, no cudaMalloc/cudaFree, no allocating library call.
 *  - Maximum box: the scratch grid of the box (its grown extent, rows padded
 *    to even length: ((n0+8+1)&~1) * (n1+8) * (n2+8 in 3-D, else 1)) must
 *    hold at most HYDRO_NOALLOC_MAX_ZONES zones, e.g. a 32^3 3-D box or a
 *    244^2 2-D box; larger boxes return HYDRO_ETOOBIG and enqueue nothing.
 *  - The storage (64,000 zones x 123 fields x 8 B = 60.1 MiB) is held on
 *    every GPU that loads this library until the process exits, and is
 *    shared by every call on that device: calls
 *    whose work overlaps on the GPU (different streams, or threads) race and
 *    must be serialised by the caller.  Each step resets the scratch state
 *    it needs; only the bad-state flag carries over (see below).
 *  - Runs on the calling thread's current device.  The first call on a device
 *    looks up the storage's device address (cudaGetSymbolAddress); make that
 *    first call outside any stream capture.
 *  - in, out, params, dt, dt_next_host, stream: as for hydro_advance_box.
 *    A bad state is reported only by a call that passes dt_next_host: the
 *    device's bad-state flag stays set from the call that raised it until
 *    such a call returns HYDRO_EBADSTATE, which clears it. */
#define HYDRO_NOALLOC_MAX_ZONES 64000
int hydro_advance_box_noalloc(const hydro_box_t* in, const hydro_box_t* out, const hydro_params_t* params,
                              double dt, double* dt_next_host, void* stream);

/* ---- instrumentation (paper: no profiler is named; this is the build's own tracing) ----
 * Stages of a step, in order: 0 primitive state, 1 characteristic tracing,
 * 2 first Riemann solves, 3 intermediate (3-D) solves, 4 final solves,
 * 5 update + CFL reduction. */
#define HYDRO_NSTAGES 6

/* Enable (1) or disable (0) per-stage CUDA-event timing of hydro_advance_box
 * on the stream it is called with, and reset the accumulated times.  While
 * enabled every hydro_advance_box call synchronises its stream after the step. */
int hydro_ctx_set_profiling(hydro_ctx_t* ctx, int enable);

/* Copy up to nmax accumulated stage durations (milliseconds, summed over the
 * profiled calls) into ms (host) and the number of profiled calls into *calls
 * (host, nullable).  Returns the number of stages (HYDRO_NSTAGES) or a
 * negative status. */
int hydro_ctx_stage_times(hydro_ctx_t* ctx, double* ms, int nmax, long long* calls);

/* Total number of CUDA kernels this context has enqueued (host counter). */
long long hydro_ctx_launches(const hydro_ctx_t* ctx);

/* Scratch limit of a context's single-box step (hydro_advance_box and
 * hydro_advance_box_host).  The staged step keeps every intermediate of a box
 * (123 fields of the grown box, 984 bytes per grown zone: 2.5 GB at 128^3,
 * 137 GB at 512^3).  A 3-D box whose whole-box scratch exceeds `bytes` is
 * stepped slab by slab along z instead, with scratch for one slab and its
 * 4-plane halos (balanced slabs of as many planes as fit): the result is
 * bitwise the same, at the cost of recomputing the few planes where slabs
 * meet.  0: never slab.  Default 16 GiB.  Takes effect at the next step. */
int hydro_ctx_set_scratch_limit(hydro_ctx_t* ctx, size_t bytes);

/* Diagnostics (no counterpart in the paper): fault injection on the host.
 * While enabled, the context's large device allocations -- the step scratch,
 * the host-buffer step's staging boxes, the batched level's scratch pool and
 * the two-level temporaries -- fail as if the device were out of memory, so
 * callers can test their HYDRO_ENOMEM handling: a call that needs one of
 * them returns HYDRO_ENOMEM and enqueues no step.  Memory the context
 * already holds is still used.
 * Disabling restores normal allocation; the context stays usable. */
int hydro_ctx_fail_allocations(hydro_ctx_t* ctx, int enable);

/* ---- boundary fluxes of a box step (paper Sec. 3: a level's coarse-fine
 * synchronisation corrects coarse zones with the fluxes of the fine level, so
 * the fluxes through a box's outer faces are part of what a step produces;
 * they are also the boundary term of its conservation balance) ----
 * Enable (1) or disable (0) recording: while enabled, every hydro_advance_box
 * and hydro_advance_box_host call on this context also keeps the final
 * Riemann fluxes (the ones the update differences) through the 2*dim outer
 * faces of its box, in context-owned device memory (one extra kernel).
 * Disabling forgets what was recorded. */
int hydro_ctx_record_face_fluxes(hydro_ctx_t* ctx, int enable);

/* Copy the recorded fluxes through face `side` (0: the low face, face 0; 1:
 * the high face, face n[d]) of axis d of the most recent recorded step into
 * dst (device, caller-owned): 5 fields (mass, momentum x/y/z, energy flux per
 * unit area and time), each n[t1] x n[t2] values with t1 < t2 the two other
 * axes and t1 fastest (in 2-D t2 has extent 1).  Enqueued on `stream`, after
 * the step in stream order.  HYDRO_EINVAL if nothing is recorded (recording
 * off, or no step since it was enabled) or d is not an axis of that step. */
int hydro_ctx_face_flux(hydro_ctx_t* ctx, int d, int side, double* dst, void* stream);

/* Diagnostics (no counterpart in the paper): the kernels scale by 2 and by
 * 1/2 on the integer pipe instead of the FP64 multiplier; this runs those two
 * helpers over x[0..n) (device arrays of n doubles) into twice[] and half[],
 * asynchronously on `stream`, so a test can compare them bit for bit with
 * IEEE 2.0*x and 0.5*x. */
int hydro_selftest_scale2(const double* x, double* twice, double* half, long long n, void* stream);

/* Diagnostics (no counterpart in the paper): the product build forms the
 * sound speed and 1/rho of a first-solve face state from one refined
 * reciprocal square root; this runs that helper over x[0..n) (device) into
 * out[] (device), asynchronously on `stream`, so a test can bound its error
 * against 1/sqrt(x).  The contraction-free build returns IEEE 1.0/sqrt(x). */
int hydro_selftest_rsqrt(const double* x, double* out, long long n, void* stream);

/* Diagnostics (no counterpart in the paper): the device's FP64 issue rate,
 * the denominator of the step's FP64 roofline.  Launches nblocks blocks of
 * 256 threads, each thread running 8 independent chains of `iters` FP64
 * multiply-adds (nblocks * 256 * 8 * iters FMAs, 2 flops each), and writes
 * one double per thread to out (device, nblocks * 256 doubles); time it with
 * events on `stream`. */
int hydro_selftest_fp64_rate(double* out, int nblocks, int iters, void* stream);

/* Diagnostics (no counterpart in the paper): the kernels' reciprocal,
 * quotient and square root -- IEEE in the contraction-free build, Newton
 * refinements of the hardware's approximations in the product build -- over
 * x[0..n), y[0..n) (device arrays): rcp = 1/x, quo = y/x, sq = sqrt(x),
 * asynchronously on `stream`, so a test can bound their error against IEEE. */
int hydro_selftest_divsqrt(const double* x, const double* y, double* rcp, double* quo, double* sq, long long n,
                           void* stream);

/* Diagnostics (no counterpart in the paper): the kernels form part of their
 * FP64 products and sums from the operands' bit patterns on the integer
 * pipe; this runs those two routines over x[0..n), y[0..n) (device arrays):
 * prod = x*y, sum = x+y, asynchronously on `stream`, so a test can compare
 * them bit for bit with the IEEE operations (round to nearest even). */
int hydro_selftest_intpipe(const double* x, const double* y, double* prod, double* sum, long long n, void* stream);

/* Diagnostics (no counterpart in the paper; host only, no device needed):
 * the schedule hydro_advance_box_host runs for a 3-D box of nz interior
 * planes with derived faces, input copied in nchunk z-chunks
 * (1 <= nchunk <= min(nz, 16), nz >= 4), low z face of kind bc_low
 * (HYDRO_BC_OUTFLOW, _REFLECT or _PERIODIC).  Writes *pre_lo (interior
 * planes [*pre_lo, nz) are copied ahead of the chunks) and, per chunk k,
 * 22 ints at out[22 k]: ten half-open [lo, hi) ranges along z -- interior
 * planes copied in, interior planes whose primitive state is formed, then
 * planes of the x/y tracing, first x/y fluxes and F^{x|y}, F^{y|x} (from
 * -1), zones of the z tracing (from -1), z-faces of the first z fluxes,
 * planes of F^{x|z}, F^{y|z}, z-faces of F^{z|x}, F^{z|y}, planes of the
 * final x/y fluxes, z-faces of the final z fluxes, planes of the update --
 * then two flags: the low and the high ghost planes' primitive state is
 * formed with this chunk.  HYDRO_EINVAL for other arguments. */
int hydro_pipe_plan(int nz, int nchunk, int bc_low, int* pre_lo, int* out);

#ifdef __cplusplus
}
#endif
#endif /* HYDRO_H */
