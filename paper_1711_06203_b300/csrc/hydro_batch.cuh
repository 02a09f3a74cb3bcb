// Device descriptor of one box of a batched step (shared by the batch engine
// and the kernels that read a batched step's scratch, e.g. flux registers).
#pragma once
#include "hydro_step.cuh"

namespace hydro {

// everything a batched kernel needs about one box (device resident)
struct BatchBox {
  BoxGeom in, out;
  ScratchGeom sg;
  Scratch s;
  StepConst K;  // dt, hdt, dtdx refreshed on the device from dt_dev every call
  double dx[3];
  double cfl;
  Range rp, ru;
  SweepRange tr[3];
  int tmode[3];  // tracing along d: 0 the pencil sweep (tr[d].seg zones per segment), 1 warp rows (x) / tiles (y, z)
  Range r1[3], r2[3][3], r3[3];
  DevFlags flags;
};

}  // namespace hydro
