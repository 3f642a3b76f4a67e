// Library-internal access to the predictor from the network's step loop.
#pragma once
#include <cuda_runtime.h>

#include "eprop_predictor.h"

// Issues the forward pass on `st` for rows of FP32 inputs already on the
// device; returns the device pointer of the FP32 outputs [rows][n_out].
const float *predictor_issue_forward(eprop_predictor *p, const float *x_dev, int rows, cudaStream_t st);
void predictor_dims(const eprop_predictor *p, int *n_in, int *n_out, int *max_rows);
