// dirac_internal.h -- what the library's translation units share (not part of
// the public ABI): error reporting and a read-only view of a single-problem
// context.
#pragma once

#include "dirac.h"

#include <cuda_runtime.h>

namespace dirac {

// Records a printf-style message for dirac_last_error() and returns `s`.
dirac_status fail(dirac_status s, const char* fmt, ...);

// The operator and fields of a context as set by dirac_create / dirac_set_fields.
struct CtxView {
  int nx, ny;
  double dx, dy, mass, c;
  int order, boundary;
  const double* V;        // FP64 potential energy on the grid (device), or null for V = 0
  double vmin, vmax;      // range of V (0, 0 when V = 0)
  double ax, ay;          // uniform vector potential (static fields)
  double shift;           // energy shift s: the operator is H - s
  bool fields_set;
  cudaStream_t stream;
  long long* launches;    // the context's kernel-launch counter
  bool profiling;         // dirac_profile_enable is on: time kernels with CUDA events
};

dirac_status ctx_view(dirac_ctx* ctx, CtxView* v);

}  // namespace dirac
