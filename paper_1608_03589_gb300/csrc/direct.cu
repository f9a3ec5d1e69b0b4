// Pixel-driven direct backprojection R* (Section 2, eq "bp_app") for sm_103a.
//
// b(x_p) = sum_k w_k [ (1 - f) g_{k,j} + f g_{k,j+1} ],  u = x_p . xi_k / dt + (n_det-1)/2,
// j = floor(u), f = u - j, zero outside the detector.
//
// Design (GB300): a CTA owns a 64 x 64 pixel tile (16 pixels per thread) and walks the
// angles in stages.  For each (tile, angle) it stages the W detector bins the tile can touch
// into shared memory as a pre-weighted table, in one of two forms.
//
// 2 x 2-block form (bp_direct_quad_sync_kernel; pixels no larger than detector bins, i.e.
// |c|, |s| <= 1, every benchmark workload): a thread owns four 2 x 2 pixel blocks; over a
// block u spans |c| + |s| <= 2 bins, so with j = floor(u at the block's lowest corner) and
// r = u - j the four pixels need only g_j .. g_{j+3}, and the linear interpolant is exactly
// the sum of clamped ramps
//     w g(u) = w g_j + sum_{i=0..2} w (g_{j+i+1} - g_{j+i}) sat(r - i),   sat = clamp to [0, 1]
// (ramps above r vanish, those below are 1).  One 16-byte entry (w g_j, w dg_j, w dg_{j+1},
// w dg_{j+2}) serves all four pixels of a block; the common w g_j is summed once per block;
// the lowest corner needs one FFMA, the side corners two ramps, the far corner two or three
// (FADD.SAT clamps).  j comes from a paired add rounded toward minus infinity of the magic
// constant 1.5 * 2^23, whose bits index shared memory.  The corner roles follow the signs of
// (c, s): the accumulators are kept per role and exchanged when the signs change; stages
// whose angles share the signs skip the per-angle tests.  The table is built from global
// memory each stage (the single float4 table takes 24 KB, so four CTAs share an SM and
// cover the loads' latency); the stage arithmetic lives in direct_tile.cuh.
//
// Pair form (other geometries): entries
//     d_m = w_k (g_{J0+m+1} - g_{J0+m}),   e_m = w_k g_{J0+m} + (1/2 - (m - C)) d_m,
// so that with the tile-local, half-bin-shifted coordinate q = u - J0 - C - 1/2 the
// interpolated, weighted sample is the single FMA  e_m + q d_m  with m - C = rint(q)
// (magic-number rounding again).  bp_direct_tma_kernel (16-byte strided rows): the raw
// windows of stage s+2 are fetched by TMA (one 3D box per angle, zero-filled off the
// detector) into a double buffer while stage s computes; the (e, d) table is double buffered
// too, so each stage has a single block barrier; coordinates and the rounding of two pixels
// share one packed f32x2 instruction.  bp_direct_kernel: synchronous window loads for other
// strides.
//
// In both forms the per-tile window origin J0 and base coordinate come from exact 32.32
// fixed-point tile stepping, so float32 only ever holds tile-local coordinates (|q| <= W/2).
//
// When N is even, pixels are no larger than bins and the angle set is closed under
// theta -> pi - theta (every uniform set), launch_direct_shape takes the four-image form of
// direct_klein.cu instead (it needs a plan workspace; calls that must not allocate keep the forms
// here).
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>
#include <type_traits>

#include "common.cuh"
#include "direct_tile.cuh"
#include "f32x2.cuh"
#include "tma.cuh"

namespace bp {

namespace {

constexpr size_t kMaxDirectSmem = 200 * 1024;

// Stage range [s0, s1) of angle group g out of `asplit` over S stages (balanced, non-empty
// when asplit <= S).
__device__ __forceinline__ int group_stage(int g, int S, int asplit) { return (int)((long long)g * S / asplit); }

template <typename Tin>
__global__ void __launch_bounds__(kThreads, 2)
bp_direct_kernel(const Tin *__restrict__ sino, float *__restrict__ img, const AngleParam *__restrict__ ap,
                 int N, int n_det, int n_theta, int W, int C, int accumulate, int tiles, int asplit,
                 long long sino_stride, long long img_stride, float wuni) {
    extern __shared__ __align__(16) float2 tab[];  // [kStage][W] (e, d) pairs
    __shared__ DirectStageSmem sm;
    const int ty = blockIdx.y % tiles, grp = blockIdx.y / tiles;
    const int S = (n_theta + kStage - 1) / kStage;
    const int k_begin = group_stage(grp, S, asplit) * kStage;
    const int k_end = min(n_theta, group_stage(grp + 1, S, asplit) * kStage);
    direct_tile_sync<Tin>(sino + (long long)blockIdx.z * sino_stride, img + (long long)blockIdx.z * img_stride, ap,
                          N, n_det, k_begin, k_end, W, C, blockIdx.x, ty, accumulate, asplit > 1, wuni, tab, sm);
}

// The 2 x 2-block form with synchronous window loads (|c|, |s| <= 1): STAGE angles per stage,
// MINB CTAs per SM.
template <typename Tin, int STAGE, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
bp_direct_quad_sync_kernel(const Tin *__restrict__ sino, float *__restrict__ img, const AngleParam *__restrict__ ap,
                           int N, int n_det, int n_theta, int W, int C, int accumulate, int tiles, int asplit,
                           long long sino_stride, long long img_stride, float wuni) {
    extern __shared__ __align__(16) float4 qtab[];  // [STAGE][W]
    __shared__ QuadStageSmem<STAGE> qsm;
    const int ty = blockIdx.y % tiles, grp = blockIdx.y / tiles;
    const int S = (n_theta + STAGE - 1) / STAGE;
    const int k_begin = group_stage(grp, S, asplit) * STAGE;
    const int k_end = min(n_theta, group_stage(grp + 1, S, asplit) * STAGE);
    direct_tile_quad_sync<Tin, STAGE>(sino + (long long)blockIdx.z * sino_stride,
                                      img + (long long)blockIdx.z * img_stride, ap, N, n_det, k_begin, k_end, W, C,
                                      blockIdx.x, ty, accumulate, asplit > 1, wuni, qtab, qsm);
}

template <typename T> __device__ __forceinline__ float smem_f(const unsigned char *p, int i);
template <> __device__ __forceinline__ float smem_f<float>(const unsigned char *p, int i) {
    return reinterpret_cast<const float *>(p)[i];
}
template <> __device__ __forceinline__ float smem_f<__nv_bfloat16>(const unsigned char *p, int i) {
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[i]);
}
template <> __device__ __forceinline__ float smem_f<__half>(const unsigned char *p, int i) {
    return __half2float(reinterpret_cast<const __half *>(p)[i]);
}

// STAGE angles per stage; the table of each angle is built by kThreads / STAGE threads.
template <typename Tin, int STAGE>
__global__ void __launch_bounds__(kThreads, 3)
bp_direct_tma_kernel(const __grid_constant__ CUtensorMap tmap, float *__restrict__ img,
                     const AngleParam *__restrict__ ap, int N, int n_theta, int W, int C, int Wb, int RS,
                     int accumulate, int tiles, int asplit, long long img_stride, int *__restrict__ err, float wuni) {
    constexpr int TPA = kThreads / STAGE;
    extern __shared__ __align__(128) unsigned char dsm[];
    unsigned char *raw = dsm;                                              // [2][STAGE] rows of RS bytes
    float2 *tab = reinterpret_cast<float2 *>(dsm + 2 * STAGE * RS);      // [2][STAGE][W]
    __shared__ float4 sp[3][STAGE];   // q0, c, s, table base bits
    __shared__ int sof[3][STAGE];     // J0 - J0r (TMA box starts at the 8-aligned J0r)
    __shared__ float sw[3][STAGE];
    __shared__ __align__(8) unsigned long long bars[2];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int lx = lane & 7;
    const int ly = warp * 8 + (lane >> 3);
    const int tx = blockIdx.x, ty = blockIdx.y % tiles, grp = blockIdx.y / tiles, bz = blockIdx.z;
    img += (long long)bz * img_stride;
    const uint32_t bar0 = smem_u32(&bars[0]);
    const unsigned tab_u32 = smem_u32(tab);
    // this CTA's stages: [s0, s0 + S) of the (n_theta / STAGE) stages
    const int S_all = (n_theta + STAGE - 1) / STAGE;
    const int s0 = group_stage(grp, S_all, asplit);
    const int S = group_stage(grp + 1, S_all, asplit) - s0;

    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        mbar_fence_init();
    }
    __syncthreads();

    // Stage parameters and TMA issue for local stage i: thread kk < kn handles angle k0 + kk.
    auto prepare = [&](int i) {
        const int k0 = (s0 + i) * STAGE, kn = min(STAGE, n_theta - k0), b = i & 1, slot = i % 3;
        if (tid == 0) mbar_expect_tx(bar0 + 8 * b, (uint32_t)(kn * Wb * (int)sizeof(Tin)));
        if (tid < kn) {
            const AngleParam p = ap[k0 + tid];
            const long long U = p.U00 + (long long)tx * p.CT + (long long)ty * p.ST;
            const int Ji = (int)(U >> 32);
            const float frac = (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f;
            const float emin = (float)(kTile - 1) * (fminf(p.c, 0.f) + fminf(p.s, 0.f));
            const int J0 = Ji + (int)floorf(emin) - 1;
            const int J0r = J0 & ~7;
            const float q0 = (float)(Ji - J0 - C) + (frac - 0.5f);
            const unsigned base = tab_u32 + (unsigned)((b * STAGE + tid) * W) * 8u + 8u * (unsigned)C -
                                  (kMagicBits << 3);
            sp[slot][tid] = make_float4(q0, p.c, p.s, __uint_as_float(base));
            sof[slot][tid] = J0 - J0r;
            sw[slot][tid] = wuni > 0.f ? wuni : p.w;
            tma_load_3d(smem_u32(raw + (b * STAGE + tid) * RS), &tmap, J0r, k0 + tid, bz, bar0 + 8 * b);
        }
    };

    float acc[2][8];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 8; ++a) acc[b][a] = 0.f;
    const float fx = (float)lx, fy = (float)ly;
    const unsigned long long MM = pk2(kMagic, kMagic);

    prepare(0);
    if (S > 1) prepare(1);
    __syncthreads();
    bool ok = true;
    for (int i = 0; i < S; ++i) {
        const int b = i & 1, slot = i % 3;
        const int kn = min(STAGE, n_theta - (s0 + i) * STAGE);
        ok &= mbar_wait(bar0 + 8 * b, (uint32_t)((i >> 1) & 1));
        {
            // build the (e, d) table of stage i from its raw windows: TPA threads per angle
            const int kk = tid / TPA, r = tid % TPA;
            if (kk < kn) {
                const unsigned char *row = raw + (b * STAGE + kk) * RS;
                const int off = sof[slot][kk];
                const float w = sw[slot][kk];
                float2 *dst = tab + (b * STAGE + kk) * W;
                for (int m = r; m < W; m += TPA) {
                    const float g0 = smem_f<Tin>(row, off + m);
                    const float g1 = smem_f<Tin>(row, off + m + 1);
                    const float d = w * (g1 - g0);
                    dst[m] = make_float2(fmaf(0.5f - (float)(m - C), d, w * g0), d);
                }
            }
        }
        if (__syncthreads_or(!ok)) {
            // a copy did not complete in time: record it, issue no further copy, wait (bounded)
            // for the copies still in flight (stages i and i + 1) and leave without writing
            if (tid == 0) atomicExch(err, 1);
            mbar_wait(bar0 + 8 * b, (uint32_t)((i >> 1) & 1));
            if (i + 1 < S) mbar_wait(bar0 + 8 * (b ^ 1), (uint32_t)(((i + 1) >> 1) & 1));
            return;
        }
        if (i + 2 < S) {
            if (tid < STAGE) fence_proxy_async_smem();
            prepare(i + 2);
        }
        for (int kk = 0; kk < kn; ++kk) {
            const float4 P = sp[slot][kk];
            const float qt = fmaf(fy, P.z, fmaf(fx, P.y, P.x));
            const unsigned long long Q = pk2(qt, fmaf(4.f, P.z, qt));
            const unsigned long long CC = pk2(P.y, P.y);
            const unsigned base = __float_as_uint(P.w);
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const unsigned long long qa = ffma2(pk2(8.f * a, 8.f * a), CC, Q);
                const unsigned long long va = fadd2(qa, MM);
                float q0, q1, v0, v1;
                upk2(qa, q0, q1);
                upk2(va, v0, v1);
                const float2 e0 = lds64(base + (__float_as_uint(v0) << 3));
                const float2 e1 = lds64(base + (__float_as_uint(v1) << 3));
                acc[0][a] += fmaf(q0, e0.y, e0.x);
                acc[1][a] += fmaf(q1, e1.y, e1.x);
            }
        }
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int y = ty * kTile + ly + 4 * b;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int x = tx * kTile + lx + 8 * a;
            if (x < N && y < N) {
                float *dst = img + (long long)y * N + x;
                if (asplit > 1) atomicAdd(dst, acc[b][a]);
                else *dst = accumulate ? (*dst + acc[b][a]) : acc[b][a];
            }
        }
    }
}

template <typename Tin> constexpr CUtensorMapDataType tmap_type();
template <> constexpr CUtensorMapDataType tmap_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> constexpr CUtensorMapDataType tmap_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }
template <> constexpr CUtensorMapDataType tmap_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }

// Dynamic shared memory of the TMA kernel for `stage` angles per stage.
size_t tma_smem(const bp_plan *p, int stage, int esz) {
    const int Wb = (p->W + 8 + 7) & ~7;
    const size_t RS = ((size_t)Wb * esz + 127) & ~(size_t)127;
    return 2 * (size_t)stage * RS + 2 * sizeof(float2) * (size_t)stage * p->W;
}

bool tma_eligible(const bp_plan *p, int esz) {
    const int Wb = (p->W + 8 + 7) & ~7;
    return ((long long)p->n_det * esz) % 16 == 0 && Wb <= 256;
}

// The 2 x 2-block form needs |c|, |s| <= 1 (a block spans at most g_j .. g_{j+3}) and its
// float4 table of kStage x W entries in shared memory.
bool quad_form(const bp_plan *p) {
    return p->step_max <= 1.0f && sizeof(float4) * (size_t)kStage * p->W <= kMaxDirectSmem;
}

// The shape a direct launch really uses: on the TMA path the stage is lowered until its
// shared memory fits; the synchronous path always stages kStage angles; groups are clamped.
DirectShape direct_effective(const bp_plan *p, int esz, bool tma, DirectShape shape) {
    DirectShape e;
    e.stage = kStage;
    e.workspace = shape.workspace;
    if (shape.workspace && p->klein.eligible) {
        e.stage = (shape.stage == 8 || shape.stage == 32) ? shape.stage : kStage;  // four-image variants
        e.asplit = klein_clamp_groups(p, shape.asplit);
        return e;
    }
    if (tma && !quad_form(p)) {
        e.stage = (shape.stage == 8 || shape.stage == 32) ? shape.stage : kStage;
        while (e.stage > 8 && tma_smem(p, e.stage, esz) > kMaxDirectSmem) e.stage >>= 1;
        if (tma_smem(p, e.stage, esz) > kMaxDirectSmem) e.stage = kStage;
    }
    e.asplit = std::max(1, std::min(shape.asplit, direct_max_asplit(p, e.stage)));
    return e;
}

template <typename Tin, int STAGE>
bp_status launch_tma(bp_plan *p, const CUtensorMap &map, float *img, int batch, int accumulate, int asplit,
                     cudaStream_t st, float wuni) {
    const int tiles = (p->N + kTile - 1) / kTile;
    const int esz = (int)sizeof(Tin);
    const int Wb = (p->W + 8 + 7) & ~7;
    const int RS = (Wb * esz + 127) & ~127;
    const size_t smem = tma_smem(p, STAGE, esz);
    auto kern = bp_direct_tma_kernel<Tin, STAGE>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(tiles, tiles * asplit, batch);
    kern<<<grid, kThreads, smem, st>>>(map, img, p->d_ang, p->N, p->n_theta, p->W, p->C, Wb, RS, accumulate, tiles,
                                       asplit, (long long)p->N * p->N, p->d_err, wuni);
    BP_CUDA_TRY(cudaGetLastError());
    stage_mark(p, st, "bp_direct_tma_kernel");
    return BP_OK;
}

template <typename Tin>
bool encode_rows(const bp_plan *p, const Tin *sino, int batch, int box, CUtensorMap *map) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const int esz = (int)sizeof(Tin);
    const cuuint64_t dims[3] = {(cuuint64_t)p->n_det, (cuuint64_t)p->n_theta, (cuuint64_t)batch};
    const cuuint64_t strides[2] = {(cuuint64_t)p->n_det * esz, (cuuint64_t)p->n_det * p->n_theta * esz};
    const cuuint32_t boxd[3] = {(cuuint32_t)box, 1, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, tmap_type<Tin>(), 3, const_cast<Tin *>(sino), dims, strides, boxd, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename Tin>
bp_status launch_direct_t(bp_plan *p, const Tin *sino, float *img, int batch, int accumulate, cudaStream_t st,
                          float wuni, DirectShape shape) {
    const int tiles = (p->N + kTile - 1) / kTile;
    const int esz = (int)sizeof(Tin);
    const bool have_enc = tensor_map_encoder() != nullptr;
    const bool quad = quad_form(p);
    const DirectShape eff = direct_effective(p, esz, !quad && have_enc && tma_eligible(p, esz), shape);
    const int stage = eff.stage, asplit = eff.asplit;
    stage_begin(p, st);
    if (asplit > 1 && !accumulate) {
        BP_CUDA_TRY(cudaMemsetAsync(img, 0, sizeof(float) * (size_t)p->N * p->N * batch, st));
        stage_mark(p, st, "memset (direct R* angle groups)");
    }
    dim3 grid(tiles, tiles * asplit, batch);
    if (quad) {
        const size_t qsmem = sizeof(float4) * (size_t)kStage * p->W;
        auto qk = bp_direct_quad_sync_kernel<Tin, kStage, 4>;
        BP_CUDA_TRY(cudaFuncSetAttribute(qk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsmem));
        qk<<<grid, kThreads, qsmem, st>>>(sino, img, p->d_ang, p->N, p->n_det, p->n_theta, p->W, p->C, accumulate,
                                          tiles, asplit, (long long)p->n_theta * p->n_det, (long long)p->N * p->N,
                                          wuni);
        BP_CUDA_TRY(cudaGetLastError());
        stage_mark(p, st, "bp_direct_quad_sync_kernel");
        return BP_OK;
    }
    CUtensorMap map;
    const bool tma = have_enc && tma_eligible(p, esz) && tma_smem(p, stage, esz) <= kMaxDirectSmem &&
                     encode_rows(p, sino, batch, (p->W + 8 + 7) & ~7, &map);
    if (tma) {
        switch (stage) {
            case 8: return launch_tma<Tin, 8>(p, map, img, batch, accumulate, asplit, st, wuni);
            case 32: return launch_tma<Tin, 32>(p, map, img, batch, accumulate, asplit, st, wuni);
            default: return launch_tma<Tin, 16>(p, map, img, batch, accumulate, asplit, st, wuni);
        }
    }
    const size_t smem = sizeof(float2) * (size_t)kStage * p->W;
    if (smem > kMaxDirectSmem) return fail(BP_ERR_UNSUPPORTED, "direct R*: window too large for shared memory");
    auto kern = bp_direct_kernel<Tin>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, kThreads, smem, st>>>(sino, img, p->d_ang, p->N, p->n_det, p->n_theta, p->W, p->C, accumulate,
                                       tiles, asplit, (long long)p->n_theta * p->n_det, (long long)p->N * p->N,
                                       wuni);
    BP_CUDA_TRY(cudaGetLastError());
    stage_mark(p, st, "bp_direct_kernel");
    return BP_OK;
}

}  // namespace

bp_status launch_direct_shape(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, int accumulate,
                              cudaStream_t st, float wuni, DirectShape shape) {
    if (dt != BP_F32 && dt != BP_BF16 && dt != BP_F16) return fail(BP_ERR_INVALID_ARG, "invalid dtype");
    if (shape.workspace && p->klein.eligible)
        return launch_direct_klein(p, sino, dt, img, batch, accumulate, st, wuni, shape.stage, shape.asplit);
    switch (dt) {
        case BP_F32: return launch_direct_t(p, (const float *)sino, img, batch, accumulate, st, wuni, shape);
        case BP_BF16:
            return launch_direct_t(p, (const __nv_bfloat16 *)sino, img, batch, accumulate, st, wuni, shape);
        case BP_F16: return launch_direct_t(p, (const __half *)sino, img, batch, accumulate, st, wuni, shape);
    }
    return fail(BP_ERR_INVALID_ARG, "invalid dtype");
}

bp_status launch_direct(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, int accumulate,
                        cudaStream_t st, float wuni) {
    return launch_direct_shape(p, sino, dt, img, batch, accumulate, st, wuni, direct_shape(p, dt, batch));
}

// Filter + direct R* (bp_fbp_direct).  With the four-image form and the persistent filter
// transform, each slice's filtered rows go straight into the row tables (one launch, the
// filtered sinogram never leaves the chip); otherwise the slices are filtered into a plan-owned
// array and backprojected from it.  The launch shape is the one of BP_F32 sinograms (what the
// tables and the array hold).
bp_status launch_fbp_direct(bp_plan *p, const void *sino, bp_dtype dt, float *img, int kind, float param, int batch,
                            cudaStream_t st) {
    bp_status s = ensure_filter(p, kind, param);
    if (s != BP_OK) return s;
    const DirectShape shape = direct_shape(p, BP_F32, batch);
    if (shape.workspace && p->klein.eligible && p->d_twpass)
        return launch_direct_klein(p, sino, dt, img, batch, 0, st, 0.f, shape.stage, shape.asplit, p->d_H[kind]);
    const size_t n = (size_t)batch * p->n_theta * p->n_det;
    if (n > p->fbp_n) {
        BP_CUDA_TRY(cudaStreamSynchronize(st));  // no queued call may still read the old array
        cudaFree(p->d_fbp);
        p->d_fbp = nullptr;
        p->fbp_n = 0;
        BP_CUDA_TRY(cudaMalloc(&p->d_fbp, sizeof(float) * n));
        p->fbp_n = n;
    }
    s = launch_filter(p, sino, dt, p->d_fbp, kind, param, batch, st);
    if (s != BP_OK) return s;
    return launch_direct_shape(p, p->d_fbp, BP_F32, img, batch, 0, st, 0.f, shape);
}

DirectShape direct_clamp(const bp_plan *p, bp_dtype dt, DirectShape shape) {
    const int esz = dt == BP_F32 ? 4 : 2;
    return direct_effective(p, esz, tensor_map_encoder() != nullptr && tma_eligible(p, esz), shape);
}

DirectShape direct_shape_used(const bp_plan *p, bp_dtype dt, int batch) {
    return direct_clamp(p, dt, direct_shape(p, dt, batch));
}

// Largest useful angle split: every group keeps at least one stage, and the grid's y
// dimension (tiles x asplit) stays within 65535.
int direct_max_asplit(const bp_plan *p, int stage) {
    const int tiles = (p->N + kTile - 1) / kTile;
    const int S = (p->n_theta + stage - 1) / stage;
    return std::max(1, std::min(S, 65535 / tiles));
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    });
    return fn;
}

}  // namespace bp
