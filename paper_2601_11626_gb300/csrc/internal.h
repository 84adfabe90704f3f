// Library-internal definitions shared by the host translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "csvd.h"

// A rank-r incremental state (Lemma 1 / Cor. 3): basis U (m x r row-major,
// ld r, double-buffered for the rotation and re-orthonormalisation),
// retained singular values, FP64 scalars {energy, discarded} and a device
// status word, all owned by the state.
struct csvd_state_s {
  int64_t m = 0;
  int r = 0;
  int prec = 0;
  cudaStream_t stream = nullptr;
  int rt = 0;
  int nblocks = 0;
  float* U[2] = {nullptr, nullptr};
  int cur = 0;
  float* sigma = nullptr;
  double* scal = nullptr;
  int* status = nullptr;
};

namespace csvd {
// Records the thread-local error message and returns st.
csvd_status set_error(csvd_status st, const char* msg);
// Streaming multiprocessors of the current device.
int device_sm_count();
}  // namespace csvd
