// Definition of the opaque mgmlmc_ctx handle shared by the extern "C" files.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "engine.h"

struct mgmlmc_ctx {
  mg::Engine *eng = nullptr;
  std::string err;
  // per-sample values of every term of the last mgmlmc_estimate_trace call
  std::vector<std::vector<std::complex<double>>> last_samples;
};

// in and out of an operator call must not share any byte: the transfer and
// projection kernels read their input after writing parts of the output
inline void require_disjoint(const void *a, size_t abytes, const void *b, size_t bbytes) {
  const uintptr_t a0 = (uintptr_t)a, b0 = (uintptr_t)b;
  if (a0 < b0 + bbytes && b0 < a0 + abytes)
    throw mg::Error(MGMLMC_ERR_ARG, "in and out overlap (they must be distinct buffers)");
}
