// The persistent FBP row filter (Section 3, Remark 1 (ii), eq "fbp"; internal), shared by the
// plain filter (filter.cu, filtered rows to global memory) and the four-image direct R*
// (direct_klein.cu, whose fused form turns each filtered row pair straight into its row tables).
//
// Transform lengths P = 2^9 .. 2^12 (n_det <= 2048): each CTA stages H and a per-pass twiddle
// table in shared memory once and then walks row pairs (two real rows as one complex row).  The
// passes are the Stockham radix-8 passes of fft.cuh (a radix-4 or radix-2 pass last when
// log2 P is not a multiple of 3) with P / 8 threads, but
//  * pass twiddles come from a table laid out per pass as T[(r - 1) L + k] = W_{LR}^{rk}, so
//    the lanes of a warp (consecutive k) read consecutive entries, free of bank conflicts;
//  * the first forward pass reads the two rows straight from global memory (the upper half
//    of the zero-padded row is known to be zero) and the next pair's loads are in flight
//    while the current pair is transformed;
//  * the outputs of the last forward pass that a thread holds are exactly the inputs of its
//    first inverse pass, so H is applied and that pass computed in registers;
//  * the last inverse pass hands the first n_det outputs to the output policy Epi:
//      Epi::kStaged false: epi.put(r0, has1, n_det, i, v) per output i < n_det from registers
//        (v.x of row r0, v.y of row r0 + 1);
//      Epi::kStaged true: the pair is staged in shared memory (rows r0 and r0 + 1 at
//        sg[4 + i] and sg[n_det + 12 + i], four zeros on each side of each row) and every thread
//        calls epi.rows(sg, r0, has1, n_det) after a barrier.
// Shared memory: P float2 work array (which also holds the staging: 2 (n_det + 8) <= 2 P
// floats), the twiddles, P floats of H.
#pragma once

#include "common.cuh"
#include "fft.cuh"
#include "fft_pt.cuh"

namespace bp {

template <int LOGP>
constexpr size_t filter_pt_smem() {
    constexpr int P = 1 << LOGP, TWN = pt_offset<LOGP>(PtPlan<LOGP>::npass);
    return sizeof(float2) * (P + ((TWN + 1) & ~1)) + sizeof(float) * P;
}

template <typename Tin, int LOGP, typename Epi>
__device__ __forceinline__ void filter_pt_body(const Tin *__restrict__ in, const Epi &epi,
                                               const float *__restrict__ H, const float2 *__restrict__ twp,
                                               long long rows, int n_det) {
    using PL = PtPlan<LOGP>;
    constexpr int P = 1 << LOGP, NT = P / kPassE, Rl = PL::Rl, Gl = kPassE / Rl;
    constexpr int TWN = pt_offset<LOGP>(PL::npass);
    static_assert(TWN % 2 == 0, "per-pass twiddle count");
    extern __shared__ __align__(16) float2 pz[];
    float2 *z = pz;                                           // [P] work array
    float2 *T = z + P;                                        // [TWN] per-pass twiddles
    float *Hs = reinterpret_cast<float *>(T + ((TWN + 1) & ~1));  // [P] response
    const int t = threadIdx.x;
    const long long npairs = (rows + 1) / 2;
    // inputs of the first forward pass: x[t + r NT], r < 4 (r >= 4 lies in the zero padding)
    float2 nxt[4];
    auto fetch = [&](long long pair) {
        const long long r0 = 2 * pair;
        const bool has1 = r0 + 1 < rows;
        const Tin *a = in + r0 * n_det, *b = a + n_det;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = t + r * NT;
            float va = 0.f, vb = 0.f;
            if (i < n_det) {
                va = load_f(a + i);
                if (has1) vb = load_f(b + i);
            }
            nxt[r] = make_float2(va, vb);
        }
    };
    long long pair = blockIdx.x;
    if (pair < npairs) fetch(pair);
    // stage the twiddles and H (16-byte loads, all in flight together; T and Hs start
    // 16-byte aligned, TWN is even and P a multiple of 4)
    {
        constexpr int n4t = TWN / 2, n4h = P / 4;
        const float4 *ts = reinterpret_cast<const float4 *>(twp);
        const float4 *hs = reinterpret_cast<const float4 *>(H);
        float4 *td = reinterpret_cast<float4 *>(T);
        float4 *hd = reinterpret_cast<float4 *>(Hs);
#pragma unroll
        for (int i = 0; i < (n4t + NT - 1) / NT; ++i)
            if (t + i * NT < n4t) td[t + i * NT] = __ldg(ts + t + i * NT);
#pragma unroll
        for (int i = 0; i < (n4h + NT - 1) / NT; ++i)
            if (t + i * NT < n4h) hd[t + i * NT] = __ldg(hs + t + i * NT);
    }
    for (; pair < npairs; pair += gridDim.x) {
        float2 a[8];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = nxt[r];
#pragma unroll
        for (int r = 4; r < 8; ++r) a[r] = make_float2(0.f, 0.f);
        if (pair + gridDim.x < npairs) fetch(pair + gridDim.x);
        __syncthreads();  // previous pair's last reads of z (and the staged tables) are done
        // forward pass 0 (L = 1, radix 8) from registers
        dft_reg<8>(a, false);
#pragma unroll
        for (int q = 0; q < 8; ++q) z[fft_swz<kPassE>(t * 8 + q)] = a[q];
        __syncthreads();
        int L = 8;
#pragma unroll
        for (int p = 1; p < PL::n8; ++p) {
            if (p == PL::npass - 1) break;
            pt_pass<8, LOGP>(z, T + pt_offset<LOGP>(p), L, t, false);
            L *= 8;
        }
        // last forward pass into registers, times H, first inverse pass (L = 1, radix 8)
        float2 b[8];
        {
            constexpr int lp = PL::npass - 1, m = P / Rl;
            float2 c[Gl][Rl];
#pragma unroll
            for (int g = 0; g < Gl; ++g)
#pragma unroll
                for (int r = 0; r < Rl; ++r) c[g][r] = z[fft_swz<kPassE>(t + g * NT + r * m)];
#pragma unroll
            for (int g = 0; g < Gl; ++g) {
                // here L * Rl = P: k = t + g NT, j = 0, outputs at k + q L = t + (g + q Gl) NT
                pt_twiddle_dft<Rl>(c[g], T + pt_offset<LOGP>(lp), L, t + g * NT, false);
#pragma unroll
                for (int q = 0; q < Rl; ++q) {
                    const int r = g + q * Gl;
                    const float h = Hs[t + r * NT];
                    b[r] = make_float2(c[g][q].x * h, c[g][q].y * h);
                }
            }
        }
        dft_reg<8>(b, true);
        __syncthreads();  // all reads of the last forward pass done before z is overwritten
#pragma unroll
        for (int q = 0; q < 8; ++q) z[fft_swz<kPassE>(t * 8 + q)] = b[q];
        __syncthreads();
        L = 8;
#pragma unroll
        for (int p = 1; p < PL::n8; ++p) {
            if (p == PL::npass - 1) break;
            pt_pass<8, LOGP>(z, T + pt_offset<LOGP>(p), L, t, true);
            L *= 8;
        }
        // last inverse pass: outputs t + (g + q Gl) NT
        {
            constexpr int lp = PL::npass - 1, m = P / Rl;
            float2 c[Gl][Rl];
#pragma unroll
            for (int g = 0; g < Gl; ++g)
#pragma unroll
                for (int r = 0; r < Rl; ++r) c[g][r] = z[fft_swz<kPassE>(t + g * NT + r * m)];
            const long long r0 = 2 * pair;
            const bool has1 = r0 + 1 < rows;
            if constexpr (Epi::kStaged) __syncthreads();  // every read of z done: it becomes the staging
            float *sg = reinterpret_cast<float *>(z);
#pragma unroll
            for (int g = 0; g < Gl; ++g) {
                pt_twiddle_dft<Rl>(c[g], T + pt_offset<LOGP>(lp), L, t + g * NT, true);
#pragma unroll
                for (int q = 0; q < Rl; ++q) {
                    const int i = t + (g + q * Gl) * NT;
                    if (i < n_det) {
                        if constexpr (Epi::kStaged) {
                            sg[4 + i] = c[g][q].x;
                            sg[n_det + 12 + i] = c[g][q].y;
                        } else {
                            epi.put(r0, has1, n_det, i, c[g][q]);
                        }
                    }
                }
            }
            if constexpr (Epi::kStaged) {
                if (t < 16) {
                    const int i = (t & 7) < 4 ? (t & 7) : n_det + (t & 7);  // 0..3, n_det + 4 .. n_det + 7
                    sg[(t >> 3) * (n_det + 8) + i] = 0.f;
                }
                __syncthreads();
                epi.rows(sg, r0, has1, n_det);
            }
        }
    }
}

}  // namespace bp
