// Persistent batched R*: independent slices with different geometries (image size, bins,
// angle sets, storage type) in one kernel launch (Section 2, eq "bp_app", per slice).
//
// Every slice is split into 64 x 64 pixel tiles; the (slice, tile) work items are numbered
// slice after slice.  A grid of (SM count x resident CTAs) CTAs pulls items from a device
// counter until the list is exhausted, so large and small slices mix without a tail of idle
// SMs.  The per-slice descriptors travel by value in the kernel parameters (captured with
// the launch, so the call can be recorded in a CUDA graph); the counter is reset by a
// stream-ordered memset before each launch.  Each tile is the direct kernel's tile
// (direct_tile.cuh): the 2 x 2-block form for slices whose pixels are no larger than their
// detector bins, else the pair-table form.  No thread ever waits on another: the queue is one atomicAdd per item.
#include <algorithm>

#include "common.cuh"
#include "direct_tile.cuh"

namespace bp {

namespace {

constexpr int kMaxSlices = 256;  // descriptors per launch (larger batches use several launches)

struct SliceDesc {
    const void *sino;
    float *img;
    const AngleParam *ap;
    int N, n_det, n_theta, W, C, dtype, tiles1, item0;  // tiles1: tiles per side; item0: first item
    int quad;  // |c|, |s| <= 1: the 2 x 2-block tile
};
struct BatchParams {
    SliceDesc d[kMaxSlices];
    int n, items;
};
static_assert(sizeof(BatchParams) <= 31 * 1024, "kernel parameter block too large");

__global__ void __launch_bounds__(kThreads, 4)
bp_batched_kernel(const __grid_constant__ BatchParams bpm, int *__restrict__ counter) {
    extern __shared__ __align__(16) float4 tab4[];  // [kStage][W] float4 (2 x 2-block tile) or float2 (pair tile)
    float2 *tab = reinterpret_cast<float2 *>(tab4);
    __shared__ DirectStageSmem sm;
    __shared__ QuadStageSmem<> qsm;
    __shared__ int item_s;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item_s = atomicAdd(counter, 1);
        __syncthreads();
        const int item = item_s;
        if (item >= bpm.items) break;
        // slice of this item: last descriptor whose first item <= item (binary search)
        int lo = 0, hi = bpm.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bpm.d[mid].item0 <= item) lo = mid;
            else hi = mid - 1;
        }
        const SliceDesc &d = bpm.d[lo];
        const int t = item - d.item0;
        const int ty = t / d.tiles1, tx = t - ty * d.tiles1;
        if (d.quad) {
            switch (d.dtype) {
                case BP_F32:
                    direct_tile_quad_sync<float>((const float *)d.sino, d.img, d.ap, d.N, d.n_det, 0, d.n_theta, d.W,
                                                 d.C, tx, ty, 0, 0, 0.f, tab4, qsm);
                    break;
                case BP_BF16:
                    direct_tile_quad_sync<__nv_bfloat16>((const __nv_bfloat16 *)d.sino, d.img, d.ap, d.N, d.n_det, 0,
                                                         d.n_theta, d.W, d.C, tx, ty, 0, 0, 0.f, tab4, qsm);
                    break;
                default:
                    direct_tile_quad_sync<__half>((const __half *)d.sino, d.img, d.ap, d.N, d.n_det, 0, d.n_theta,
                                                  d.W, d.C, tx, ty, 0, 0, 0.f, tab4, qsm);
                    break;
            }
            continue;
        }
        switch (d.dtype) {
            case BP_F32:
                direct_tile_sync<float>((const float *)d.sino, d.img, d.ap, d.N, d.n_det, 0, d.n_theta, d.W, d.C, tx,
                                        ty, 0, 0, 0.f, tab, sm);
                break;
            case BP_BF16:
                direct_tile_sync<__nv_bfloat16>((const __nv_bfloat16 *)d.sino, d.img, d.ap, d.N, d.n_det, 0,
                                                d.n_theta, d.W, d.C, tx, ty, 0, 0, 0.f, tab, sm);
                break;
            default:
                direct_tile_sync<__half>((const __half *)d.sino, d.img, d.ap, d.N, d.n_det, 0, d.n_theta, d.W, d.C,
                                         tx, ty, 0, 0, 0.f, tab, sm);
                break;
        }
    }
}

}  // namespace

bp_status launch_batched(bp_plan *const *plans, const void *const *sinos, const bp_dtype *dtypes, float *const *imgs,
                         int n, cudaStream_t st) {
    if (klein_mixed_eligible(plans, imgs, n)) return launch_klein_mixed(plans, sinos, dtypes, imgs, n, st);
    bp_plan *p0 = plans[0];
    if (!p0->d_counter) BP_CUDA_TRY(cudaMalloc(&p0->d_counter, sizeof(int)));
    static int sms = 0, dev_of_sms = -1;
    if (dev_of_sms != p0->device) {
        BP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p0->device));
        dev_of_sms = p0->device;
    }
    stage_begin(p0, st);
    for (int base = 0; base < n; base += kMaxSlices) {
        const int cnt = std::min(kMaxSlices, n - base);
        BatchParams bpm;
        int items = 0, Wmax = 0;
        for (int i = 0; i < cnt; ++i) {
            const bp_plan *p = plans[base + i];
            SliceDesc &d = bpm.d[i];
            d.sino = sinos[base + i];
            d.img = imgs[base + i];
            d.ap = p->d_ang;
            d.N = p->N;
            d.n_det = p->n_det;
            d.n_theta = p->n_theta;
            d.W = p->W;
            d.C = p->C;
            d.dtype = (int)dtypes[base + i];
            d.tiles1 = (p->N + kTile - 1) / kTile;
            d.item0 = items;
            d.quad = p->step_max <= 1.0f ? 1 : 0;
            items += d.tiles1 * d.tiles1;
            Wmax = std::max(Wmax, p->W * (d.quad ? 2 : 1));  // float4 entries count twice
        }
        bpm.n = cnt;
        bpm.items = items;
        const size_t smem = sizeof(float2) * (size_t)kStage * Wmax;
        BP_CUDA_TRY(cudaFuncSetAttribute(bp_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bp_batched_kernel, kThreads, smem));
        const int grid = std::max(1, std::min(items, sms * std::max(1, per_sm)));
        BP_CUDA_TRY(cudaMemsetAsync(p0->d_counter, 0, sizeof(int), st));
        bp_batched_kernel<<<grid, kThreads, smem, st>>>(bpm, p0->d_counter);
        BP_CUDA_TRY(cudaGetLastError());
        stage_mark(p0, st, "bp_batched_kernel");
    }
    return BP_OK;
}

}  // namespace bp
