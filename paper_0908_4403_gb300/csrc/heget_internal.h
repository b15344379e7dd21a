// heget_internal.h -- host-side constants and error helpers shared by the
// C-ABI translation units.
#pragma once

#include <cstdarg>

#include <cuda_runtime.h>

namespace heget {

constexpr int kBlockThreads = 256;   // amplitude kernels: threads per block
constexpr int kMaxGrid = 65536;      // block partials held by a context

// Records a message for heget_last_error() and returns `code`.
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

}  // namespace heget
