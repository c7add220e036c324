// Definition of the opaque mgmlmc_ctx handle shared by the extern "C" files.
#pragma once

#include <string>

#include "engine.h"

struct mgmlmc_ctx {
  mg::Engine *eng = nullptr;
  std::string err;
};
