// Batched advance of many boxes (placeholder until the batch engine lands).
#include "hydro_api_internal.cuh"

void hydro_batch_release(hydro_ctx* ctx) { (void)ctx; }
