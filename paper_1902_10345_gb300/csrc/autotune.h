// Autotuner cache: the best (kernel, k, seg_rows, warps) per dtype and shape
// class, measured by sdfg_autotune and optionally persisted to a file named by
// the SDFG_AUTOTUNE_CACHE environment variable.
#pragma once

#include "../../include/sdfg_jacobi.h"

namespace sdfg {

// Shape class: dtype and the power-of-two buckets of rows and cols.
bool autotune_lookup(int rows, int cols, int dtype, sdfg_config *out);
void autotune_store(int rows, int cols, int dtype, const sdfg_config &c);

}  // namespace sdfg
