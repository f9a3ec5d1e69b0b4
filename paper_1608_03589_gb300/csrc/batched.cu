// Persistent batched R* -- placeholder.
#include "common.cuh"

namespace bp {

bp_status launch_batched(bp_plan *const *, const void *const *, const bp_dtype *, float *const *, int, cudaStream_t) {
    return fail(BP_ERR_UNSUPPORTED, "batched path not built yet");
}

}  // namespace bp
