// bp_fbp_static: filtered backprojection that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a reconstruction:
// code embedded in a host framework that owns every device allocation (a fixed memory
// pool or budget, where a private cudaMalloc can fail or break the budget), or
// real-time acquisition loops in which allocating is not allowed (cudaMalloc may
// synchronise the device and its latency is unbounded).  For them this entry point keeps
// its scratch -- the filtered sinogram of one slice -- in one file-scope static device
// array of fixed size, which every GPU that loads the library holds until the process
// exits.  The filter's frequency response is the plan's own (FP64 on the host, made by
// bp_plan_create for Ram-Lak and Shepp-Logan), so a call only reads it.  The caller still
// passes its own input and output buffers.
#include <mutex>

#include "common.cuh"

namespace bp {

namespace {

constexpr size_t kStaticFloats = BP_STATIC_SCRATCH_BYTES / sizeof(float);
constexpr int kMaxDevices = 128;

// The scratch itself.  In host code the symbol is only a host-side stand-in, never a
// device address: host code must use the address that cudaGetSymbolAddress returns.
static __device__ __align__(256) float g_static_scratch[kStaticFloats];

std::mutex g_setup_mutex;
float *g_scratch_addr[kMaxDevices] = {};

// Once per device, with that device current: look up the device address of the array.
bp_status scratch_address(int device, float **out) {
    if (device < 0 || device >= kMaxDevices) return fail(BP_ERR_UNSUPPORTED, "bp_fbp_static: device index too large");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)");
        g_scratch_addr[device] = static_cast<float *>(ptr);
    }
    *out = g_scratch_addr[device];
    return BP_OK;
}

}  // namespace

}  // namespace bp

using namespace bp;

extern "C" bp_status bp_fbp_static(bp_plan *p, const void *sino, bp_dtype dtype, float *img, bp_filter_kind kind,
                                   int batch, void *stream) {
    set_error("");
    bp_status st = check_plan(p);
    if (st != BP_OK) return st;
    if (!sino || !img) return fail(BP_ERR_INVALID_ARG, "data pointer is NULL");
    if (!aligned16(sino) || !aligned16(img)) return fail(BP_ERR_INVALID_ARG, "data pointers must be 16-byte aligned");
    if (batch < 1 || batch > 65535) return fail(BP_ERR_INVALID_ARG, "batch out of range [1, 65535]");
    if (dtype != BP_F32 && dtype != BP_BF16 && dtype != BP_F16) return fail(BP_ERR_INVALID_ARG, "invalid dtype");
    if (kind != BP_RAMLAK && kind != BP_SHEPP_LOGAN)
        return fail(BP_ERR_UNSUPPORTED, "bp_fbp_static supports BP_RAMLAK and BP_SHEPP_LOGAN only");
    const size_t slice = (size_t)p->n_theta * p->n_det;
    if (slice > kStaticFloats)
        return fail(BP_ERR_UNSUPPORTED, "bp_fbp_static: n_theta * n_det exceeds the static scratch of "
                                        "BP_STATIC_SCRATCH_BYTES / 4 floats");
    const float *H = p->d_H[kind];
    if (!H) return fail(BP_ERR_INVALID_ARG, "bp_fbp_static: the plan has no filter response for this kind");
    float *q = nullptr;
    st = scratch_address(p->device, &q);
    if (st != BP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // Every value the kernels read from the scratch is written earlier in this call, so
    // nothing needs clearing.
    const size_t esz = dtype == BP_F32 ? 4 : 2;
    for (int b = 0; b < batch; ++b) {
        const char *sb = (const char *)sino + esz * slice * b;
        st = launch_filter_response(p, sb, dtype, q, H, 1, s);
        if (st != BP_OK) return st;
        DirectShape shape = direct_shape(p, BP_F32, 1);
        shape.workspace = 0;  // the forms that need a plan workspace would allocate it
        st = launch_direct_shape(p, q, BP_F32, img + (size_t)b * p->N * p->N, 1, 0, s, 0.f, shape);
        if (st != BP_OK) return st;
    }
    return BP_OK;
}
