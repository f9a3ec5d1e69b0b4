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
#include "common.cuh"

namespace bp {

namespace {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr unsigned kMagicBits = 0x4B400000u;

template <typename Tin>
__global__ void __launch_bounds__(kThreads, 2)
bp_direct_kernel(const Tin *__restrict__ sino, float *__restrict__ img, const AngleParam *__restrict__ ap,
                 int N, int n_det, int n_theta, int W, int C, int accumulate,
                 long long sino_stride, long long img_stride) {
    extern __shared__ __align__(16) float2 tab[];  // [kStage][W] (e, d) pairs
    __shared__ float4 sp[kStage];                  // q0, c, s, table base (bits)
    __shared__ int sJ0[kStage];
    __shared__ float sw[kStage];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int lx = lane & 7;
    const int ly = warp * 8 + (lane >> 3);
    const int tx = blockIdx.x, ty = blockIdx.y;
    sino += (long long)blockIdx.z * sino_stride;
    img += (long long)blockIdx.z * img_stride;

    float acc[2][8];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 8; ++a) acc[b][a] = 0.f;

    const float fx = (float)lx, fy = (float)ly;
    const unsigned tab_u32 = smem_u32(tab);

    for (int k0 = 0; k0 < n_theta; k0 += kStage) {
        const int kn = min(kStage, n_theta - k0);
        __syncthreads();
        if (tid < kn) {
            const AngleParam p = ap[k0 + tid];
            const long long U = p.U00 + (long long)tx * p.CT + (long long)ty * p.ST;
            const int Ji = (int)(U >> 32);
            const float frac = (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f;
            const float emin = (float)(kTile - 1) * (fminf(p.c, 0.f) + fminf(p.s, 0.f));
            const int J0 = Ji + (int)floorf(emin) - 1;
            const float q0 = (float)(Ji - J0 - C) + (frac - 0.5f);
            sJ0[tid] = J0;
            sw[tid] = p.w;
            const unsigned base = tab_u32 + (unsigned)(tid * W) * 8u + 8u * (unsigned)C - (kMagicBits << 3);
            sp[tid] = make_float4(q0, p.c, p.s, __uint_as_float(base));
        }
        __syncthreads();
        {
            // 16 threads per angle build its (e, d) window.
            const int kk = tid >> 4, r = tid & 15;
            if (kk < kn) {
                const Tin *row = sino + (long long)(k0 + kk) * n_det;
                const int J0 = sJ0[kk];
                const float w = sw[kk];
                for (int m = r; m < W; m += 16) {
                    const int j = J0 + m;
                    const float g0 = (j >= 0 && j < n_det) ? load_f(row + j) : 0.f;
                    const float g1 = (j + 1 >= 0 && j + 1 < n_det) ? load_f(row + j + 1) : 0.f;
                    const float d = w * (g1 - g0);
                    const float e = fmaf(0.5f - (float)(m - C), d, w * g0);
                    tab[kk * W + m] = make_float2(e, d);
                }
            }
        }
        __syncthreads();
        for (int kk = 0; kk < kn; ++kk) {
            const float4 P = sp[kk];
            const float qt = fmaf(fy, P.z, fmaf(fx, P.y, P.x));
            const unsigned base = __float_as_uint(P.w);
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float qb = fmaf(4.f * b, P.z, qt);
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const float q = fmaf(8.f * a, P.y, qb);
                    const float v = q + kMagic;
                    const float2 ed = lds64(base + (__float_as_uint(v) << 3));
                    acc[b][a] += fmaf(q, ed.y, ed.x);
                }
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
                *dst = accumulate ? (*dst + acc[b][a]) : acc[b][a];
            }
        }
    }
}

template <typename Tin>
bp_status launch_direct_t(bp_plan *p, const Tin *sino, float *img, int batch, int accumulate, cudaStream_t st) {
    const int tiles = (p->N + kTile - 1) / kTile;
    const size_t smem = sizeof(float2) * (size_t)kStage * p->W;
    auto kern = bp_direct_kernel<Tin>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(tiles, tiles, batch);
    kern<<<grid, kThreads, smem, st>>>(sino, img, p->d_ang, p->N, p->n_det, p->n_theta, p->W, p->C, accumulate,
                                       (long long)p->n_theta * p->n_det, (long long)p->N * p->N);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

}  // namespace

bp_status launch_direct(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, int accumulate,
                        cudaStream_t st) {
    switch (dt) {
        case BP_F32: return launch_direct_t(p, (const float *)sino, img, batch, accumulate, st);
        case BP_BF16: return launch_direct_t(p, (const __nv_bfloat16 *)sino, img, batch, accumulate, st);
        case BP_F16: return launch_direct_t(p, (const __half *)sino, img, batch, accumulate, st);
    }
    return fail(BP_ERR_INVALID_ARG, "invalid dtype");
}

}  // namespace bp
