// Shared-memory radix-2 FFT building blocks (internal).
//
// Forward transforms are decimation-in-frequency (natural order in, bit-reversed out);
// inverse transforms are decimation-in-time (bit-reversed in, natural out, conjugate
// twiddles, unnormalised).  A pointwise product between the two therefore needs no
// explicit bit reversal as long as the multiplier is stored bit-reversed.
// Twiddles: tw[r] = exp(-2 pi i r / P0), r < P0/2, for a table built for length P0;
// a length-P transform (P <= P0, both powers of two) reads tw with stride P0/P.
#pragma once

#include <cuda_runtime.h>

namespace bp {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}

// z: shared memory, length P = 2^logP.  All threads of the block participate; ends synchronised.
__device__ __forceinline__ void fft_dif_fwd(float2 *z, int logP, const float2 *__restrict__ tw, int twstride) {
    const int P = 1 << logP;
    for (int ls = logP - 1; ls >= 0; --ls) {
        const int s = 1 << ls;
        const int step = (P >> (ls + 1)) * twstride;  // twiddle index step = P0 / (2s)
        for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
            const int i = t & (s - 1);
            const int i0 = ((t >> ls) << (ls + 1)) + i;
            const int i1 = i0 + s;
            const float2 a = z[i0], b = z[i1];
            z[i0] = cadd(a, b);
            z[i1] = cmul(csub(a, b), __ldg(tw + i * step));
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void fft_dit_inv(float2 *z, int logP, const float2 *__restrict__ tw, int twstride) {
    const int P = 1 << logP;
    for (int ls = 0; ls < logP; ++ls) {
        const int s = 1 << ls;
        const int step = (P >> (ls + 1)) * twstride;
        for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
            const int i = t & (s - 1);
            const int i0 = ((t >> ls) << (ls + 1)) + i;
            const int i1 = i0 + s;
            const float2 a = z[i0];
            const float2 b = cmulc(z[i1], __ldg(tw + i * step));
            z[i0] = cadd(a, b);
            z[i1] = csub(a, b);
        }
        __syncthreads();
    }
}

// Forward DIT (bit-reversed in, natural out) and inverse DIF (natural in, bit-reversed out).
__device__ __forceinline__ void fft_dit_fwd(float2 *z, int logP, const float2 *__restrict__ tw, int twstride) {
    const int P = 1 << logP;
    for (int ls = 0; ls < logP; ++ls) {
        const int s = 1 << ls;
        const int step = (P >> (ls + 1)) * twstride;
        for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
            const int i = t & (s - 1);
            const int i0 = ((t >> ls) << (ls + 1)) + i;
            const int i1 = i0 + s;
            const float2 a = z[i0];
            const float2 b = cmul(z[i1], __ldg(tw + i * step));
            z[i0] = cadd(a, b);
            z[i1] = csub(a, b);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ void fft_dif_inv(float2 *z, int logP, const float2 *__restrict__ tw, int twstride) {
    const int P = 1 << logP;
    for (int ls = logP - 1; ls >= 0; --ls) {
        const int s = 1 << ls;
        const int step = (P >> (ls + 1)) * twstride;
        for (int t = threadIdx.x; t < (P >> 1); t += blockDim.x) {
            const int i = t & (s - 1);
            const int i0 = ((t >> ls) << (ls + 1)) + i;
            const int i1 = i0 + s;
            const float2 a = z[i0], b = z[i1];
            z[i0] = cadd(a, b);
            z[i1] = cmulc(csub(a, b), __ldg(tw + i * step));
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int bitrev(int v, int logP) { return (int)(__brev((unsigned)v) >> (32 - logP)); }

}  // namespace bp
