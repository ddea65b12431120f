// fec_batch.h -- batched execution behind fec_cluster_batch.
#pragma once

#include <cuda_runtime.h>

#include "fec.h"

namespace fec {

struct BatchEngine;

BatchEngine *batch_create(int device, int sms, const char *tune_path);
void batch_destroy(BatchEngine *e);

// Cluster nb frames (device or host buffers) on `main`; synchronous.
fec_status batch_run(BatchEngine *e, cudaStream_t main, size_t budget, const float *xyz,
                     const int64_t *offsets, int32_t nb, const float *d, const int64_t *mn,
                     const int64_t *mx, int32_t *labels, int32_t *num_clusters);

// Device bytes held by the engine's lanes.
size_t batch_bytes(const BatchEngine *e);

}  // namespace fec
