// One 64 x 64 tile of the direct R* with synchronous window loads (internal).  Shared by
// the plain direct kernel and the persistent batched kernel; the arithmetic is described in
// direct.cu.
#pragma once

#include "common.cuh"

namespace bp {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr unsigned kMagicBits = 0x4B400000u;

struct DirectStageSmem {
    float4 sp[kStage];  // q0, c, s, table base (bits)
    int J0[kStage];
    float w[kStage];
};

// Angles [k_begin, k_end) of tile (tx, ty); the partial sum is added atomically when
// atomic_out (angle-split launches), else stored (or added, with accumulate).
// tab: kStage * W float2 of shared memory.  All threads of the block must call it.
template <typename Tin>
__device__ __forceinline__ void direct_tile_sync(const Tin *__restrict__ sino, float *__restrict__ img,
                                                 const AngleParam *__restrict__ ap, int N, int n_det, int k_begin,
                                                 int k_end, int W, int C, int tx, int ty, int accumulate,
                                                 int atomic_out, float wuni, float2 *tab, DirectStageSmem &sm) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int lx = lane & 7;
    const int ly = warp * 8 + (lane >> 3);

    float acc[2][8];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 8; ++a) acc[b][a] = 0.f;

    const float fx = (float)lx, fy = (float)ly;
    const unsigned tab_u32 = smem_u32(tab);

    for (int k0 = k_begin; k0 < k_end; k0 += kStage) {
        const int kn = min(kStage, k_end - k0);
        __syncthreads();
        if (tid < kn) {
            const AngleParam p = ap[k0 + tid];
            const long long U = p.U00 + (long long)tx * p.CT + (long long)ty * p.ST;
            const int Ji = (int)(U >> 32);
            const float frac = (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f;
            const float emin = (float)(kTile - 1) * (fminf(p.c, 0.f) + fminf(p.s, 0.f));
            const int J0 = Ji + (int)floorf(emin) - 1;
            const float q0 = (float)(Ji - J0 - C) + (frac - 0.5f);
            sm.J0[tid] = J0;
            sm.w[tid] = wuni > 0.f ? wuni : p.w;
            const unsigned base = tab_u32 + (unsigned)(tid * W) * 8u + 8u * (unsigned)C - (kMagicBits << 3);
            sm.sp[tid] = make_float4(q0, p.c, p.s, __uint_as_float(base));
        }
        __syncthreads();
        {
            // 16 threads per angle build its (e, d) window.
            const int kk = tid >> 4, r = tid & 15;
            if (kk < kn) {
                const Tin *row = sino + (long long)(k0 + kk) * n_det;
                const int J0 = sm.J0[kk];
                const float w = sm.w[kk];
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
            const float4 P = sm.sp[kk];
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
                if (atomic_out) atomicAdd(dst, acc[b][a]);
                else *dst = accumulate ? (*dst + acc[b][a]) : acc[b][a];
            }
        }
    }
}

}  // namespace bp
