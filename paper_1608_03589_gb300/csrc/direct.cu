// Pixel-driven direct backprojection R* (Section 2, eq "bp_app") for sm_103a.
//
// b(x_p) = sum_k w_k [ (1 - f) g_{k,j} + f g_{k,j+1} ],  u = x_p . xi_k / dt + (n_det-1)/2,
// j = floor(u), f = u - j, zero outside the detector.
//
// Design (GB300): a CTA owns a 64 x 64 pixel tile (16 pixels per thread) and walks the
// angles in stages of kStage.  For each (tile, angle) it stages the W detector bins the
// tile can touch into shared memory, pre-weighted and pre-differenced as pairs
//     d_m = w_k (g_{J0+m+1} - g_{J0+m}),   e_m = w_k g_{J0+m} + (1/2 - (m - C)) d_m,
// so that with the tile-local, half-bin-shifted coordinate q = u - J0 - C - 1/2 the
// interpolated, weighted sample is the single FMA  e_m + q d_m  with m - C = rint(q).
// rint(q) comes from the float "magic number" rounding (q + 1.5 * 2^23 keeps the integer
// in its low mantissa bits), whose bit pattern indexes shared memory directly.  Per
// pixel-angle update: FFMA (coordinate), FADD (rounding), LEA (address), LDS.64, FFMA,
// FADD.  The per-tile window origin J0 and base coordinate come from exact 32.32 fixed-
// point tile stepping, so float32 only ever holds tile-local coordinates (|q| <= W/2).
//
// Two variants.  bp_direct_tma_kernel (used whenever the sinogram rows are 16-byte strided):
// the raw windows of stage s+2 are fetched by TMA (one 3D box per angle, zero-filled off the
// detector) into a double buffer while stage s computes; the (e, d) table is double
// buffered too, so each stage has a single block barrier; coordinates and the magic-number
// rounding of two pixels share one packed f32x2 instruction.  bp_direct_kernel is the plain
// fallback (synchronous window loads) for other strides.
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "direct_tile.cuh"
#include "tma.cuh"

namespace bp {

namespace {

template <typename Tin>
__global__ void __launch_bounds__(kThreads, 2)
bp_direct_kernel(const Tin *__restrict__ sino, float *__restrict__ img, const AngleParam *__restrict__ ap,
                 int N, int n_det, int n_theta, int W, int C, int accumulate,
                 long long sino_stride, long long img_stride, float wuni) {
    extern __shared__ __align__(16) float2 tab[];  // [kStage][W] (e, d) pairs
    __shared__ DirectStageSmem sm;
    direct_tile_sync<Tin>(sino + (long long)blockIdx.z * sino_stride, img + (long long)blockIdx.z * img_stride, ap,
                          N, n_det, n_theta, W, C, blockIdx.x, blockIdx.y, accumulate, wuni, tab, sm);
}

__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
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

template <typename Tin>
__global__ void __launch_bounds__(kThreads, 3)
bp_direct_tma_kernel(const __grid_constant__ CUtensorMap tmap, float *__restrict__ img,
                     const AngleParam *__restrict__ ap, int N, int n_theta, int W, int C, int Wb, int RS,
                     int accumulate, long long img_stride, int *__restrict__ err, float wuni) {
    extern __shared__ __align__(128) unsigned char dsm[];
    unsigned char *raw = dsm;                                              // [2][kStage] rows of RS bytes
    float2 *tab = reinterpret_cast<float2 *>(dsm + 2 * kStage * RS);     // [2][kStage][W]
    __shared__ float4 sp[3][kStage];   // q0, c, s, table base bits
    __shared__ int sof[3][kStage];     // J0 - J0r (TMA box starts at the 8-aligned J0r)
    __shared__ float sw[3][kStage];
    __shared__ __align__(8) unsigned long long bars[2];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int lx = lane & 7;
    const int ly = warp * 8 + (lane >> 3);
    const int tx = blockIdx.x, ty = blockIdx.y, bz = blockIdx.z;
    img += (long long)bz * img_stride;
    const uint32_t bar0 = smem_u32(&bars[0]);
    const unsigned tab_u32 = smem_u32(tab);
    const int S = (n_theta + kStage - 1) / kStage;

    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        mbar_fence_init();
    }
    __syncthreads();

    // Stage parameters and TMA issue for stage s: thread kk < kn handles angle k0 + kk.
    auto prepare = [&](int s) {
        const int k0 = s * kStage, kn = min(kStage, n_theta - k0), b = s & 1, slot = s % 3;
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
            const unsigned base = tab_u32 + (unsigned)((b * kStage + tid) * W) * 8u + 8u * (unsigned)C -
                                  (kMagicBits << 3);
            sp[slot][tid] = make_float4(q0, p.c, p.s, __uint_as_float(base));
            sof[slot][tid] = J0 - J0r;
            sw[slot][tid] = wuni > 0.f ? wuni : p.w;
            tma_load_3d(smem_u32(raw + (b * kStage + tid) * RS), &tmap, J0r, k0 + tid, bz, bar0 + 8 * b);
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
    for (int s = 0; s < S; ++s) {
        const int b = s & 1, slot = s % 3;
        const int kn = min(kStage, n_theta - s * kStage);
        ok &= mbar_wait(bar0 + 8 * b, (uint32_t)((s >> 1) & 1));
        {
            // build the (e, d) table of stage s from its raw windows: 16 threads per angle
            const int kk = tid >> 4, r = tid & 15;
            if (kk < kn) {
                const unsigned char *row = raw + (b * kStage + kk) * RS;
                const int off = sof[slot][kk];
                const float w = sw[slot][kk];
                float2 *dst = tab + (b * kStage + kk) * W;
                for (int m = r; m < W; m += 16) {
                    const float g0 = smem_f<Tin>(row, off + m);
                    const float g1 = smem_f<Tin>(row, off + m + 1);
                    const float d = w * (g1 - g0);
                    dst[m] = make_float2(fmaf(0.5f - (float)(m - C), d, w * g0), d);
                }
            }
        }
        __syncthreads();
        if (s + 2 < S) {
            if (tid < kStage) fence_proxy_async_smem();
            prepare(s + 2);
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
    if (!ok && lane == 0) atomicExch(err, 1);

#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int y = ty * kTile + ly + 4 * b;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int x = tx * kTile + lx + 8 * a;
            if (x < N && y < N) {
                float *dst = img + (long long)y * N + x;
                *dst = accumulate ? (*dst + acc[b][a]) : acc[b][a];
            }
        }
    }
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

template <typename Tin> constexpr CUtensorMapDataType tmap_type();
template <> constexpr CUtensorMapDataType tmap_type<float>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT32; }
template <> constexpr CUtensorMapDataType tmap_type<__nv_bfloat16>() { return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; }
template <> constexpr CUtensorMapDataType tmap_type<__half>() { return CU_TENSOR_MAP_DATA_TYPE_FLOAT16; }

template <typename Tin>
bp_status launch_direct_t(bp_plan *p, const Tin *sino, float *img, int batch, int accumulate, cudaStream_t st,
                          float wuni) {
    const int tiles = (p->N + kTile - 1) / kTile;
    const int esz = (int)sizeof(Tin);
    const int Wb = (p->W + 8 + 7) & ~7;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (enc && ((long long)p->n_det * esz) % 16 == 0 && Wb <= 256) {
        CUtensorMap map;
        const cuuint64_t dims[3] = {(cuuint64_t)p->n_det, (cuuint64_t)p->n_theta, (cuuint64_t)batch};
        const cuuint64_t strides[2] = {(cuuint64_t)p->n_det * esz, (cuuint64_t)p->n_det * p->n_theta * esz};
        const cuuint32_t box[3] = {(cuuint32_t)Wb, 1, 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = enc(&map, tmap_type<Tin>(), 3, const_cast<Tin *>(sino), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS) {
            const int RS = (Wb * esz + 127) & ~127;
            const size_t smem = 2 * (size_t)kStage * RS + 2 * sizeof(float2) * (size_t)kStage * p->W;
            auto kern = bp_direct_tma_kernel<Tin>;
            BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            dim3 grid(tiles, tiles, batch);
            kern<<<grid, kThreads, smem, st>>>(map, img, p->d_ang, p->N, p->n_theta, p->W, p->C, Wb, RS, accumulate,
                                               (long long)p->N * p->N, p->d_err, wuni);
            BP_CUDA_TRY(cudaGetLastError());
            return BP_OK;
        }
    }
    const size_t smem = sizeof(float2) * (size_t)kStage * p->W;
    auto kern = bp_direct_kernel<Tin>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(tiles, tiles, batch);
    kern<<<grid, kThreads, smem, st>>>(sino, img, p->d_ang, p->N, p->n_det, p->n_theta, p->W, p->C, accumulate,
                                       (long long)p->n_theta * p->n_det, (long long)p->N * p->N, wuni);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

}  // namespace

bp_status launch_direct(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, int accumulate,
                        cudaStream_t st, float wuni) {
    switch (dt) {
        case BP_F32: return launch_direct_t(p, (const float *)sino, img, batch, accumulate, st, wuni);
        case BP_BF16: return launch_direct_t(p, (const __nv_bfloat16 *)sino, img, batch, accumulate, st, wuni);
        case BP_F16: return launch_direct_t(p, (const __half *)sino, img, batch, accumulate, st, wuni);
    }
    return fail(BP_ERR_INVALID_ARG, "invalid dtype");
}

}  // namespace bp
