// Fourier (Backprojection Slice Theorem) path -- placeholder until the gridding kernels land.
#include "common.cuh"

namespace bp {

bp_status ensure_fourier(bp_plan *) { return fail(BP_ERR_UNSUPPORTED, "Fourier path not built yet"); }
void free_fourier(bp_plan *) {}
bp_status launch_fourier(bp_plan *, const void *, bp_dtype, float *, int, cudaStream_t) {
    return fail(BP_ERR_UNSUPPORTED, "Fourier path not built yet");
}
bp_status launch_radon_fourier(bp_plan *, const float *, float *, int, cudaStream_t) {
    return fail(BP_ERR_UNSUPPORTED, "Fourier adjoint not built yet");
}

}  // namespace bp
