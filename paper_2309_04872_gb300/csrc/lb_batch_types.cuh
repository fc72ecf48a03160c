// Launch records of the batched step (shared by the kernel and the runtime).
#pragma once

#include "lb_common.cuh"

namespace lbp {

struct BatchRun {
  StepParams P[2];  // by parity of the step counter: in/out buffers swapped
  double z0, dt;    // driver centre at t = 0, time step
  long long prev_from;  // WARMC backward differences restart: active when step > prev_from
  int closure;      // CL_LEC or CL_WARMC
  int ntz, ntx;     // tiles along z and x
  int axi;          // 1: axisymmetric (z, r) run
};

struct BatchArgs {
  const BatchRun* runs;
  const int2* items;         // (run, tile index)
  int nitems;
  const long long* step;     // device step counter
};

}  // namespace lbp
