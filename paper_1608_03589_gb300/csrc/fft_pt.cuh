// Register-blocked Stockham passes with per-pass twiddle tables (internal), shared by the
// persistent row kernels: the FBP row filter (filter.cu) and the inverse-FFT passes of the
// Fourier path (fourier.cu).  A length-2^LOGP transform runs radix-8 passes, then one of radix
// 2^(LOGP % 3); P / kPassE threads each hold kPassE elements.  Pass twiddles come from a table
// laid out per pass as T[(r - 1) L + k] = W_{LR}^{rk} (build_pass_twiddles), so that the lanes
// of a warp (consecutive k) read consecutive entries, free of bank conflicts.
#pragma once

#include "fft.cuh"

namespace bp {

constexpr int kPassE = 8;  // elements per thread

template <int R>
__device__ __forceinline__ void pt_twiddle_dft(float2 (&a)[R], const float2 *__restrict__ T, int L, int k,
                                               bool inverse) {
    if (L > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
            float2 w = T[(r - 1) * L + k];
            if (inverse) w.y = -w.y;
            a[r] = cmul(a[r], w);
        }
    }
    dft_reg<R>(a, inverse);
}

// One middle pass, shared memory to shared memory (swizzled layout both ways).
template <int R, int LOGP>
__device__ __forceinline__ void pt_pass(float2 *z, const float2 *T, int L, int t, bool inverse) {
    constexpr int P = 1 << LOGP, NT = P / kPassE, G = kPassE / R, m = P / R;
    float2 a[G][R];
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int r = 0; r < R; ++r) a[g][r] = z[fft_swz<kPassE>(t + g * NT + r * m)];
    __syncthreads();
#pragma unroll
    for (int g = 0; g < G; ++g) {
        const int tg = t + g * NT, k = tg & (L - 1), j = tg / L;
        pt_twiddle_dft<R>(a[g], T, L, k, inverse);
#pragma unroll
        for (int q = 0; q < R; ++q) z[fft_swz<kPassE>(j * L * R + k + q * L)] = a[g][q];
    }
    __syncthreads();
}

// Pass structure of a length-2^LOGP transform: radix-8 passes, then one of radix 2^(LOGP % 3).
template <int LOGP> struct PtPlan {
    static constexpr int n8 = LOGP / 3;
    static constexpr int rb = LOGP % 3;
    static constexpr int Rl = rb == 0 ? 8 : (1 << rb);           // radix of the last pass
    static constexpr int npass = n8 + (rb ? 1 : 0);
};

// Offset of pass p's twiddles in the table (passes with L = 1 have none).
template <int LOGP>
__host__ __device__ constexpr int pt_offset(int p) {
    int off = 0, L = 1;
    for (int i = 0; i < p; ++i) {
        const int R = (i < PtPlan<LOGP>::n8) ? 8 : PtPlan<LOGP>::Rl;
        if (L > 1) off += (R - 1) * L;
        L *= R;
    }
    return off;
}

// One transform (inverse when INV) of the row whose first-pass inputs x[t + r NT] are in a:
// outputs t + (g + q Gl) NT of the last pass in c[g][q].  Begins with a block barrier (the
// previous row's reads of z are done).
template <int LOGM, bool INV>
__device__ __forceinline__ void pt_row(float2 (&a)[kPassE], float2 *z, const float2 *T, int t,
                                       float2 (&c)[kPassE / PtPlan<LOGM>::Rl][PtPlan<LOGM>::Rl]) {
    using PL = PtPlan<LOGM>;
    constexpr int M = 1 << LOGM, NT = M / kPassE, Rl = PL::Rl, Gl = kPassE / Rl;
    __syncthreads();
    dft_reg<8>(a, INV);  // pass 0 (L = 1, radix 8)
#pragma unroll
    for (int q = 0; q < 8; ++q) z[fft_swz<kPassE>(t * 8 + q)] = a[q];
    __syncthreads();
    int L = 8;
#pragma unroll
    for (int p = 1; p < PL::n8; ++p) {
        if (p == PL::npass - 1) break;
        pt_pass<8, LOGM>(z, T + pt_offset<LOGM>(p), L, t, INV);
        L *= 8;
    }
    constexpr int lp = PL::npass - 1, m = M / Rl;
#pragma unroll
    for (int g = 0; g < Gl; ++g)
#pragma unroll
        for (int r = 0; r < Rl; ++r) c[g][r] = z[fft_swz<kPassE>(t + g * NT + r * m)];
#pragma unroll
    for (int g = 0; g < Gl; ++g) pt_twiddle_dft<Rl>(c[g], T + pt_offset<LOGM>(lp), L, t + g * NT, INV);
}

}  // namespace bp
