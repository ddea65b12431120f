// fec_serve.h -- serving engine behind fec_serve_submit / fec_serve_poll.
#pragma once

#include "fec.h"

namespace fec {

struct ServeEngine;

ServeEngine *serve_create(fec_ctx *owner, const char *tune_cache);
void serve_destroy(ServeEngine *e);

// One cloud on ctx (caller holds ctx's lock).  Defined in fec_api.cu.
fec_status cluster_locked(fec_ctx *ctx, const float *xyz, int64_t n, float d, int64_t min_size,
                          int64_t max_size, int32_t *labels, int32_t *num_clusters);

}  // namespace fec
