// Persistent row transforms of the log-polar paths (internal): a length-L = 2H transform of a
// complex row as two register-first length-H transforms (fft_pt.cuh: per-pass twiddles in
// shared memory, first and last passes in registers) of its even and odd entries, combined by
// one radix-2 step in registers (decimation in time: X[k] = E[k] + w^k O[k],
// X[k + H] = E[k] - w^k O[k], w = exp(-+2 pi i / L)); a thread's E outputs wait in shared
// memory while O is transformed.  H / kPassE threads; thread t holds k = t + m H / kPassE.
#pragma once

#include "fft_pt.cuh"

namespace bp {

template <int LOGH>
__host__ __device__ constexpr int lp_rows_pt_tw_off() {
    return ((1 << LOGH) + 15) & ~15;  // after the work array
}
template <int LOGH>
__host__ __device__ constexpr int lp_rows_pt_twn() {
    return (pt_offset<LOGH>(PtPlan<LOGH>::npass) + 1) & ~1;  // even-padded per-pass twiddles
}
template <int LOGH>
constexpr size_t lp_rows_pt_smem() {
    // work array, per-pass twiddles, held E outputs
    return sizeof(float2) * ((size_t)lp_rows_pt_tw_off<LOGH>() + lp_rows_pt_twn<LOGH>() + (size_t)(1 << LOGH));
}

template <int LOGH>
__device__ __forceinline__ void lp_stage_pass_twiddles(float2 *Tw, const float2 *__restrict__ twp, int t) {
    constexpr int NT = (1 << LOGH) / kPassE, n4t = lp_rows_pt_twn<LOGH>() / 2;
    const float4 *ts = reinterpret_cast<const float4 *>(twp);
    float4 *td = reinterpret_cast<float4 *>(Tw);
    for (int i = t; i < n4t; i += NT) td[i] = __ldg(ts + i);
}

// X[k] -> xl[m], X[k + H] -> xu[m] (k = t + m NT) from the even entries ae[r] = x[2(t + r NT)]
// and odd ones ao[r] = x[2(t + r NT) + 1]; twL[k] = exp(-2 pi i k / L), k < H.
template <int LOGH, bool INV>
__device__ __forceinline__ void lp_dit_row(float2 (&ae)[kPassE], float2 (&ao)[kPassE], float2 *z, const float2 *Tw,
                                           float2 *sE, const float2 *__restrict__ twL, int t, float2 (&xl)[kPassE],
                                           float2 (&xu)[kPassE]) {
    using PL = PtPlan<LOGH>;
    constexpr int NT = (1 << LOGH) / kPassE, Rl = PL::Rl, Gl = kPassE / Rl;
    float2 c[Gl][Rl];
    pt_row<LOGH, INV>(ae, z, Tw, t, c);
#pragma unroll
    for (int g = 0; g < Gl; ++g)
#pragma unroll
        for (int q = 0; q < Rl; ++q) sE[t + (g + q * Gl) * NT] = c[g][q];
    pt_row<LOGH, INV>(ao, z, Tw, t, c);
#pragma unroll
    for (int g = 0; g < Gl; ++g)
#pragma unroll
        for (int q = 0; q < Rl; ++q) {
            const int m = g + q * Gl, k = t + m * NT;
            float2 w = __ldg(twL + k);
            if (INV) w.y = -w.y;
            const float2 e = sE[k], o = cmul(c[g][q], w);
            xl[m] = make_float2(e.x + o.x, e.y + o.y);
            xu[m] = make_float2(e.x - o.x, e.y - o.y);
        }
}

// The spectra of the two real rows packed in X = FFT(a + i b): A[k] = (X[k] + conj X[L - k]) / 2
// to ta, B[k] = (X[k] - conj X[L - k]) / (2i) to tb (skipped when null), through the work array
// in two halves (X[L - k] belongs to another thread).
template <int LOGH>
__device__ __forceinline__ void lp_separate_store(const float2 (&xl)[kPassE], const float2 (&xu)[kPassE], float2 *z,
                                                  int t, float2 *__restrict__ ta, float2 *__restrict__ tb) {
    constexpr int H = 1 << LOGH, NT = H / kPassE;
    __syncthreads();  // every thread is done with z (the second transform)
#pragma unroll
    for (int m = 0; m < kPassE; ++m) z[t + m * NT] = xu[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kPassE; ++m) {  // lower k: X[L - k] = X[H + (H - k)] (k > 0), X[0] for k = 0
        const int k = t + m * NT;
        const float2 zm = xl[m], zc = k == 0 ? xl[m] : z[H - k];
        ta[k] = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
        if (tb) tb[k] = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kPassE; ++m) z[t + m * NT] = xl[m];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kPassE; ++m) {  // upper k' = H + k: X[L - k'] = X[H - k] (X[H] itself for k = 0)
        const int k = t + m * NT;
        const float2 zm = xu[m], zc = k == 0 ? xu[m] : z[H - k];
        ta[H + k] = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
        if (tb) tb[H + k] = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
    }
}

}  // namespace bp
