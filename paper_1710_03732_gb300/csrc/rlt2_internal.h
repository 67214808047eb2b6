// Internal interfaces shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "rlt2.h"

namespace rlt2 {

// One launch solves `batch` LAPs of size m; LAP b has cost A[b*m*m..] (+ Badd[b*m*m..]).
struct LapArgs {
  long long batch;
  int m;
  const double* A;
  const double* Badd;        // nullable: cost = A + Badd (the Z->Y and Y->X folds)
  const double* u0;          // nullable: starting row duals (batch*m)
  const int* warm_gate;      // nullable: if set and *warm_gate == 0 the start is cold
  double* value;             // batch
  double* u;                 // nullable, batch*m
  double* v;                 // nullable, batch*m
  int* r2c;                  // nullable, batch*m
  int* naug;                 // nullable, batch
  double* pi;                // nullable, batch*m*m reduced costs ((cost - u_r) - v_c)
  int dual_mode;             // 0 raw, 1 canonical
  unsigned long long* stats; // nullable, [0] += augmentations, [1] += relaxations
  const int* skip;           // nullable: kernel does nothing when *skip != 0
};

// Configure the LAP kernel for size m (shared-memory limit, occupancy); call
// outside stream capture before the first launch of that size.
cudaError_t prepare_lap(int m);

// Enqueue the batched LAP kernel (grid sized for the device); returns the CUDA error.
cudaError_t launch_lap(const LapArgs& a, cudaStream_t s);

// Thread-local last error text.
void set_error(const std::string& msg);
rlt2_status cuda_fail(cudaError_t e, const char* what);

}  // namespace rlt2
