// Shared-memory FFT building blocks (internal).
//
// stockham_fft: a length-P = 2^logP complex transform of one shared-memory array, computed
// as a sequence of Stockham (self-sorting) radix-16/8/4/2 passes.  In each pass a thread
// loads R elements at stride P/R into registers, applies the pass twiddles, performs an
// R-point DFT in registers and writes the R results to their sorted positions; two block
// barriers per pass separate the loads from the stores, so the transform runs in place.
// Natural order in, natural order out.  Forward = exp(-2 pi i jk/P), inverse = exp(+...),
// both unnormalised.  Twiddles: tw[r] = exp(-2 pi i r / P0), r < P0/2, built in FP64 on the
// host for a length P0 >= P (both powers of two); the transform reads stride P0/P.
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

// exp(-+2 pi i r / P) from the half table (r in [0, P)), sign: forward (-) or inverse (+).
__device__ __forceinline__ float2 twiddle(const float2 *__restrict__ tw, int r, int logP, int twstride, bool inverse) {
    const int half = 1 << (logP - 1);
    float2 w = __ldg(tw + (r & (half - 1)) * twstride);
    if (r & half) w = make_float2(-w.x, -w.y);
    if (inverse) w.y = -w.y;
    return w;
}

// cos / sin of 2 pi k / 16, k = 0..7 (the twiddles of every in-register DFT up to 16 points).
__device__ __constant__ const float kC16[8] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                                               0.0f, -0.38268343236508977f, -0.70710678118654752f,
                                               -0.92387953251128674f};
__device__ __constant__ const float kS16[8] = {0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f,
                                               1.0f, 0.92387953251128674f, 0.70710678118654752f,
                                               0.38268343236508977f};

// In-register R-point DFT (R = 2, 4, 8, 16), iterative radix-2 on the register array,
// natural order in and out.
template <int R>
__device__ __forceinline__ void dft_reg(float2 *a, bool inverse) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
        int j = 0;
#pragma unroll
        for (int b = 1, t = i; b < R; b <<= 1, t >>= 1) j = (j << 1) | (t & 1);
        if (j > i) {
            const float2 tmp = a[i];
            a[i] = a[j];
            a[j] = tmp;
        }
    }
#pragma unroll
    for (int len = 2; len <= R; len <<= 1) {
        const int h = len >> 1;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const int idx = k * (16 / len);
            const float2 w = make_float2(kC16[idx], inverse ? kS16[idx] : -kS16[idx]);
#pragma unroll
            for (int i = k; i < R; i += len) {
                const float2 u = a[i];
                const float2 v = (k == 0) ? a[i + h] : cmul(a[i + h], w);
                a[i] = cadd(u, v);
                a[i + h] = csub(u, v);
            }
        }
    }
}

// One Stockham pass of radix R over sub-transforms of length L (L R <= P).  Each thread
// handles G = 16 / R butterflies groups; the block must have at least P / 16 threads.
template <int R>
__device__ __forceinline__ void stockham_pass(float2 *z, int logP, int L, const float2 *__restrict__ tw, int twstride,
                                              bool inverse) {
    constexpr int G = 16 / R;
    const int P = 1 << logP;
    const int m = P / R;
    float2 a[G][R];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int t = threadIdx.x + g * blockDim.x;
        if (t < m) {
#pragma unroll
            for (int r = 0; r < R; ++r) a[g][r] = z[t + r * m];
        }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int t = threadIdx.x + g * blockDim.x;
        if (t < m) {
            const int k = t & (L - 1);
            const int j = t / L;
            // pass twiddles W_{L R}^{r k} = exp(-+2 pi i r k / (L R)) = tw index r k P / (L R)
            const int step = k * (P / (L * R));
#pragma unroll
            for (int r = 1; r < R; ++r) a[g][r] = cmul(a[g][r], twiddle(tw, r * step, logP, twstride, inverse));
            dft_reg<R>(a[g], inverse);
            const int base = j * L * R + k;
#pragma unroll
            for (int q = 0; q < R; ++q) z[base + q * L] = a[g][q];
        }
    }
    __syncthreads();
}

// Threads per block for a length-P transform.
__host__ __device__ inline int fft_threads(int P) {
    const int t = P / 16;
    return t < 32 ? 32 : (t > 1024 ? 1024 : t);
}

// Whole transform (blockDim.x >= P/16, see fft_threads); z ends synchronised.
__device__ __forceinline__ void stockham_fft(float2 *z, int logP, const float2 *__restrict__ tw, int twstride,
                                             bool inverse) {
    int L = 1, rem = logP;
    while (rem > 0) {
        if (rem >= 4) {
            stockham_pass<16>(z, logP, L, tw, twstride, inverse);
            L <<= 4;
            rem -= 4;
        } else if (rem == 3) {
            stockham_pass<8>(z, logP, L, tw, twstride, inverse);
            L <<= 3;
            rem -= 3;
        } else if (rem == 2) {
            stockham_pass<4>(z, logP, L, tw, twstride, inverse);
            L <<= 2;
            rem -= 2;
        } else {
            stockham_pass<2>(z, logP, L, tw, twstride, inverse);
            L <<= 1;
            rem -= 1;
        }
    }
}

__device__ __forceinline__ int bitrev(int v, int logP) { return (int)(__brev((unsigned)v) >> (32 - logP)); }

}  // namespace bp
