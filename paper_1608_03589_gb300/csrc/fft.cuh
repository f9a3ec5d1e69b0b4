// Shared-memory FFT building blocks (internal).
//
// stockham_fft: a length-P = 2^logP complex transform of one shared-memory array, computed
// as a sequence of Stockham (self-sorting) radix-16/8/4/2 passes.  In each pass a thread
// loads R elements at stride P/R into registers, applies the pass twiddles, performs an
// R-point DFT in registers and writes the R results to their sorted positions; two block
// barriers per pass separate the loads from the stores, so the transform runs in place.
// Natural order in, natural order out.  Forward = exp(-2 pi i jk/P), inverse = exp(+...),
// both unnormalised.  Twiddles: tw[r] = exp(-2 pi i r / P0), r < P0/2, built in FP64 on the
// host for a length P0 >= P (both powers of two) and staged in shared memory; the transform
// reads stride P0/P.
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
// The table lives in shared memory (stage_twiddles), next to the transformed rows.
__device__ __forceinline__ float2 twiddle(const float2 *tw, int r, int logP, int twstride, bool inverse) {
    const int half = 1 << (logP - 1);
    float2 w = tw[(r & (half - 1)) * twstride];
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

template <int R> struct Log2R;
template <> struct Log2R<2> { static constexpr int v = 1; };
template <> struct Log2R<4> { static constexpr int v = 2; };
template <> struct Log2R<8> { static constexpr int v = 3; };
template <> struct Log2R<16> { static constexpr int v = 4; };

// In-register R-point DFT (R = 2, 4, 8, 16), iterative radix-2 on the register array,
// natural order in and out.  All loops have compile-time trip counts (fully unrolled).
template <int R>
__device__ __forceinline__ void dft_reg(float2 (&a)[R], bool inverse) {
    constexpr int LR = Log2R<R>::v;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        int j = 0;
#pragma unroll
        for (int b = 0; b < LR; ++b) j |= ((i >> b) & 1) << (LR - 1 - b);
        if (j > i) {
            const float2 tmp = a[i];
            a[i] = a[j];
            a[j] = tmp;
        }
    }
#pragma unroll
    for (int st = 0; st < LR; ++st) {
        const int h = 1 << st;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const int idx = k * (8 >> st);
            const float2 w = make_float2(kC16[idx], inverse ? kS16[idx] : -kS16[idx]);
#pragma unroll
            for (int i = k; i < R; i += 2 * h) {
                const float2 u = a[i];
                const float2 v = (k == 0) ? a[i + h] : cmul(a[i + h], w);
                a[i] = cadd(u, v);
                a[i + h] = csub(u, v);
            }
        }
    }
}

// Shared-memory bank swizzle of the intermediate passes.  A float2 covers two of the 32
// banks, so a half warp is conflict-free when its 16 indices differ mod 16.  The stores of
// the first passes go to stride-R indices (and, for radix 8, to groups of 8 contiguous
// entries 8 R apart), which all fall on a few banks; XOR-ing the low four index bits with a
// function of the 16-entry row spreads them over all banks, while contiguous runs of 16
// stay contiguous within their row.  The first pass reads and the last pass writes the
// plain layout, so callers never see the swizzle.
template <int E>
__device__ __forceinline__ int fft_swz(int i) {
    const int row = i >> 4;
    const int f = (E >= 16) ? (row & 15) : ((row & 7) | ((row & 4) << 1));
    return i ^ f;
}

// One Stockham pass of radix R over sub-transforms of length L (L R <= P).  Each of the nthr
// threads handles G = E / R butterfly groups (E elements per thread); nthr = P / E.
// in_sw / out_sw: the input / output array uses the swizzled layout.
template <int R, int E>
__device__ __forceinline__ void stockham_pass(float2 *z, int logP, int L, const float2 *tw, int twstride,
                                              bool inverse, int tid, int nthr, bool in_sw, bool out_sw) {
    constexpr int G = E / R;
    const int P = 1 << logP;
    const int m = P / R;
    float2 a[G][R];
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int t = tid + g * nthr;
        if (t < m) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = t + r * m;
                a[g][r] = z[in_sw ? fft_swz<E>(i) : i];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int t = tid + g * nthr;
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
            for (int q = 0; q < R; ++q) {
                const int i = base + q * L;
                z[out_sw ? fft_swz<E>(i) : i] = a[g][q];
            }
        }
    }
    __syncthreads();
}

// Elements per thread and threads per transform of length P: 8 per thread (radix <= 8
// passes, fits 64 registers) up to P = 8192, 16 per thread above.
__host__ __device__ inline int fft_elems(int P) { return P > 8192 ? 16 : 8; }
__host__ __device__ inline int fft_threads(int P) {
    const int t = P / fft_elems(P);
    return t < 32 ? 32 : t;
}

template <int E>
__device__ __forceinline__ void stockham_fft_e(float2 *z, int logP, const float2 *tw, int twstride,
                                               bool inverse, int tid, int nthr) {
    int L = 1, rem = logP;
    bool in_sw = false;
    while (rem > 0) {
        if constexpr (E >= 16) {
            if (rem >= 4) {
                stockham_pass<16, E>(z, logP, L, tw, twstride, inverse, tid, nthr, in_sw, rem > 4);
                L <<= 4;
                rem -= 4;
                in_sw = true;
                continue;
            }
        }
        if (rem >= 3) {
            stockham_pass<8, E>(z, logP, L, tw, twstride, inverse, tid, nthr, in_sw, rem > 3);
            L <<= 3;
            rem -= 3;
        } else if (rem == 2) {
            stockham_pass<4, E>(z, logP, L, tw, twstride, inverse, tid, nthr, in_sw, false);
            L <<= 2;
            rem -= 2;
        } else {
            stockham_pass<2, E>(z, logP, L, tw, twstride, inverse, tid, nthr, in_sw, false);
            L <<= 1;
            rem -= 1;
        }
        in_sw = true;
    }
}

// Whole transform by a group of nthr = fft_threads(P) threads (tid in [0, nthr)), E =
// fft_elems(P).  Every thread of the block must make the same sequence of calls (block
// barriers inside: several groups can transform several arrays of the same length
// together).  z ends synchronised.
template <int E>
__device__ __forceinline__ void stockham_fft(float2 *z, int logP, const float2 *tw, int twstride,
                                             bool inverse, int tid, int nthr) {
    stockham_fft_e<E>(z, logP, tw, twstride, inverse, tid, nthr);
}

// Copy n twiddles from global to shared memory (all threads of the block; a block barrier
// must separate it from the first transform).
__device__ __forceinline__ void stage_twiddles(float2 *dst, const float2 *__restrict__ src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __ldg(src + i);
}

__device__ __forceinline__ int bitrev(int v, int logP) { return (int)(__brev((unsigned)v) >> (32 - logP)); }

}  // namespace bp
