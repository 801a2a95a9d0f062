// stokes_mlp_internal.cuh -- what the time stepper uses of the warm-start network.
#pragma once
#include <cuda_runtime.h>

#include "../../include/stokes.h"

namespace stokes {
// Predictions y (B x n_out, de-standardised) of inputs x (B x n_in), both device FP32, on s.
int mlp_infer(stokes_mlp *m, int B, const float *x, float *y, cudaStream_t s);
int mlp_dims(const stokes_mlp *m, int *n_in, int *n_out);
}  // namespace stokes
