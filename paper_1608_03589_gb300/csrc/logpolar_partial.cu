// Partial (sector) log-polar backprojection (Section 5.2, "Partial Backprojections", with the
// shifting property eq "sh_prop"; per sector Andersson's convolution of Section 5.1 Steps 1-4,
// eq "andersson", kernel eq "and_kernel").
//
// The half-line angles phi in [0, pi) count every line once; they are split into Q sectors of
// K nodes (phi_j = j dphi, dphi = pi / n_half, n_half = 2^ceil(log2 n_theta)).  Sector q, centre
// phi_c, moves the origin to -d xi_{phi_c} (d = R (1 - a_r) / a_r, R = sqrt 2 the radius of the
// image disk): the shifted sinogram g(s - d cos(phi - phi_c), phi) has every line of the
// sector at s > 0, so its log-polar mesh mu_i = rho_0 + i drho starts at a finite rho_0 (the
// lowest line any output node sees, ln((d - R) cos gamma) - 2 drho) and ends at ln(d + R),
// with the outermost step at most the detector pitch (eq "N_rho").  Per sector:
//   Step 1 (fused into the first transform): the shifted sinogram on the (mu, phi) mesh by
//   linear interpolation along the detector and between the bracketing projections; the
//   detector coordinate is split on the host (FP64) into integer and fraction per mu node and
//   per sector row, so float32 only adds fractions;
//   Step 2: the unit-mass hat of the point mass at -ln cos(b dphi) / drho per angular lag b,
//   transformed once per plan (same kernels), scaled by dphi / (Lp Lr);
//   Step 3: linear convolution in rho and in angle by zero-padded 2D FFTs: rows along rho
//   (two real rows packed per complex transform), columns along phi (only the K sector rows
//   are read; only the output angle rows are written back), rows along rho inverse (only the
//   output rho window is kept);
//   Step 4: bilinear interpolation at the pixel centres from per-sector FP64-built tables,
//   summed over the sectors.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "fft.cuh"
#include "fft_pt.cuh"
#include "lp_rows.cuh"
#include "tma.cuh"

namespace bp {

namespace {

constexpr int kLppBatch = 8;  // column-segment loads in flight per thread

constexpr int kMaxLPP = 16384;  // longest transform held in shared memory

__device__ __forceinline__ void norm_frac(int &k, float &f) {
    if (f >= 1.f) {
        k += 1;
        f -= 1.f;
    }
}

// g at detector index u = k + f of row `row` (zero off the detector), linear interpolation.
template <typename Tin>
__device__ __forceinline__ float lpp_lerp(const Tin *__restrict__ row, int n_det, int k, float f) {
    const float g0 = (k >= 0 && k < n_det) ? load_f(row + k) : 0.f;
    const float g1 = (k + 1 >= 0 && k + 1 < n_det) ? load_f(row + k + 1) : 0.f;
    return fmaf(f, g1 - g0, g0);
}

// Step 1 sample of sector row j (bracket a, row split r) at mu node i (split s):
// u = +(s_i/dt) + (-D_j + c0) for an unflipped projection, -(s_i/dt) + (D_j + c0) for a flipped one.
template <typename Tin>
__device__ __forceinline__ float lpp_sample(const Tin *__restrict__ sino, int n_det, const int4 a, const int4 r,
                                            const int2 s) {
    const float sf = __int_as_float(s.y);
    float v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int code = e == 0 ? a.x : a.y;
        const int kproj = code & 0x3fffffff;
        const bool neg = (code >> 30) & 1;
        int k;
        float f;
        if (!neg) {
            k = s.x + r.x;
            f = sf + __int_as_float(r.y);
        } else {
            k = r.z - s.x - 1;
            f = (1.f - sf) + __int_as_float(r.w);
        }
        norm_frac(k, f);
        v[e] = lpp_lerp(sino + (long long)kproj * n_det, n_det, k, f);
    }
    const float w = __int_as_float(a.z);
    return fmaf(w, v[1] - v[0], v[0]);
}

// Forward transform along rho of rows (2b, 2b+1) < n_rows: the sector's Step 1 samples
// (kernel_src = 0) or the kernel hat rows (kernel_src = 1).
template <typename Tin, int E>
__global__ void __launch_bounds__(1024, 1)
lpp_rows_fwd_kernel(const Tin *__restrict__ sino, int n_det, const int4 *__restrict__ atab,
                    const int4 *__restrict__ rowtab, const int2 *__restrict__ stab, const float2 *__restrict__ kfrac,
                    int kernel_src, int n_rho, int n_rows, float2 *__restrict__ T, const float2 *__restrict__ tw,
                    int logL) {
    extern __shared__ __align__(128) float2 z[];
    const int L = 1 << logL;
    float2 *tws = z + L;
    stage_twiddles(tws, tw, L / 2);
    const int q0 = 2 * blockIdx.x, q1 = q0 + 1;
    const bool has1 = q1 < n_rows;
    if (kernel_src) {
        const float2 k0 = __ldg(kfrac + q0), k1 = has1 ? __ldg(kfrac + q1) : make_float2(-1.f, 0.f);
        const int a0 = (int)k0.x, a1 = (int)k1.x;
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            float va = 0.f, vb = 0.f;
            if (k0.x >= 0.f) va = (i == a0) ? 1.f - k0.y : ((i == a0 + 1) ? k0.y : 0.f);
            if (k1.x >= 0.f) vb = (i == a1) ? 1.f - k1.y : ((i == a1 + 1) ? k1.y : 0.f);
            z[i] = make_float2(va, vb);
        }
    } else {
        const int4 a0 = __ldg(atab + q0), r0 = __ldg(rowtab + q0);
        const int4 a1 = has1 ? __ldg(atab + q1) : a0, r1 = has1 ? __ldg(rowtab + q1) : r0;
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            float va = 0.f, vb = 0.f;
            if (i < n_rho) {
                const int2 s = __ldg(stab + i);
                va = lpp_sample(sino, n_det, a0, r0, s);
                if (has1) vb = lpp_sample(sino, n_det, a1, r1, s);
            }
            z[i] = make_float2(va, vb);
        }
    }
    __syncthreads();
    stockham_fft<E>(z, logL, tws, 1, false, threadIdx.x, blockDim.x);
    float2 *ta = T + (long long)q0 * L, *tb = T + (long long)q1 * L;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        const float2 zm = z[k];
        const float2 zc = z[(L - k) & (L - 1)];
        ta[k] = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
        if (has1) tb[k] = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
    }
}

// Transforms along phi (length Lp) of columns [k0, k0 + C) of T (rows of length Lr): rows
// >= n_in are zero.  prep = 1: forward, times `scale`, into Khat (all Lp rows).  prep = 0:
// forward, times Khat, inverse; output row a_lo + r (mod Lp) goes to row r of T, r < n_aout.
template <int E>
__global__ void __launch_bounds__(1024, 1)
lpp_cols_kernel(float2 *__restrict__ T, float2 *__restrict__ Khat, const float2 *__restrict__ tw, int logLp, int Lr,
                int C, int n_in, int prep, float scale, int a_lo, int n_aout) {
    extern __shared__ __align__(128) float2 z[];
    const int Lp = 1 << logLp;
    float2 *tws = z + (size_t)C * Lp;
    stage_twiddles(tws, tw, Lp / 2);
    const long long k0 = (long long)blockIdx.x * C;
    const int nel = C * Lp, bd = (int)blockDim.x;
    // column segments of 8 C bytes from the n_in rows: eight loads in flight per thread
    for (int e0 = threadIdx.x; e0 < nel; e0 += kLppBatch * bd) {
        float2 v[kLppBatch];
#pragma unroll
        for (int u = 0; u < kLppBatch; ++u) {
            const int e = e0 + u * bd, q = e / C, c = e - q * C;
            v[u] = (e < nel && q < n_in) ? T[(long long)q * Lr + k0 + c] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kLppBatch; ++u) {
            const int e = e0 + u * bd, q = e / C, c = e - q * C;
            if (e < nel) z[c * Lp + q] = v[u];
        }
    }
    __syncthreads();
    const int nthr = fft_threads(Lp), groups = blockDim.x / nthr;
    const int g = threadIdx.x / nthr, tid = threadIdx.x - g * nthr;
    for (int c0 = 0; c0 < C; c0 += groups) stockham_fft<E>(z + (c0 + g) * Lp, logLp, tws, 1, false, tid, nthr);
    if (prep) {
        for (int e = threadIdx.x; e < C * Lp; e += blockDim.x) {
            const int q = e / C, c = e - q * C;
            const float2 v = z[c * Lp + q];
            Khat[(long long)q * Lr + k0 + c] = make_float2(scale * v.x, scale * v.y);
        }
        return;
    }
    for (int e0 = threadIdx.x; e0 < nel; e0 += kLppBatch * bd) {
        float2 kv[kLppBatch];
#pragma unroll
        for (int u = 0; u < kLppBatch; ++u) {
            const int e = e0 + u * bd, q = e / C, c = e - q * C;
            if (e < nel) kv[u] = __ldg(Khat + (long long)q * Lr + k0 + c);
        }
#pragma unroll
        for (int u = 0; u < kLppBatch; ++u) {
            const int e = e0 + u * bd, q = e / C, c = e - q * C;
            if (e < nel) z[c * Lp + q] = cmul(z[c * Lp + q], kv[u]);
        }
    }
    __syncthreads();
    for (int c0 = 0; c0 < C; c0 += groups) stockham_fft<E>(z + (c0 + g) * Lp, logLp, tws, 1, true, tid, nthr);
    for (int e = threadIdx.x; e < C * n_aout; e += blockDim.x) {
        const int r = e / C, c = e - r * C;
        const int q = (a_lo + r) & (Lp - 1);
        T[(long long)r * Lr + k0 + c] = z[c * Lp + q];
    }
}

// The column pass over column pairs through the TMA with the persistent transform (as the full
// log-polar column pass): the pair's n_in input rows arrive by 2D TMA loads (rows beyond n_in
// of the last box read as zero; those beyond the boxes are zero in registers), both columns'
// inputs go to registers, the pair of Khat arrives during the forward transforms and is
// multiplied into their outputs, the next pair is requested before the inverse transforms, and
// the n_aout output rows (a_lo + r) mod Lp leave through a staging buffer by 2D TMA stores.
// Every wait is bounded: on expiry the kernel sets *err, waits (bounded) for its copy once more
// and returns.
template <int LOGP>
__host__ __device__ constexpr int lpp_cols_stage_off() {
    return ((1 << LOGP) + pt_offset<LOGP>(PtPlan<LOGP>::npass) + 15) & ~15;
}
template <int LOGP>
constexpr size_t lpp_cols_pt_smem() {
    return sizeof(float2) * ((size_t)lpp_cols_stage_off<LOGP>() + 4 * (size_t)(1 << LOGP));
}

template <int LOGP>
__global__ void __launch_bounds__((1 << LOGP) / kPassE)
lpp_cols_pt_kernel(const __grid_constant__ CUtensorMap imap, const __grid_constant__ CUtensorMap omap,
                   const __grid_constant__ CUtensorMap kmap, const float2 *__restrict__ twp, int Lr, int n_in,
                   int a_lo, int n_aout, int BR, int *__restrict__ err) {
    using PL = PtPlan<LOGP>;
    constexpr int NP = 1 << LOGP, NT = NP / kPassE, Rl = PL::Rl, Gl = kPassE / Rl;
    constexpr int TWN = pt_offset<LOGP>(PL::npass);
    extern __shared__ __align__(128) float2 z[];  // [NP] work | [TWN] twiddles | [NP] pairs in | [NP] pairs out
    __shared__ __align__(8) unsigned long long bar;
    float2 *T = z + NP;
    float4 *sin = reinterpret_cast<float4 *>(z + lpp_cols_stage_off<LOGP>());
    float4 *sout = sin + NP;
    const int t = threadIdx.x;
    const int nb_in = (n_in + BR - 1) / BR, nb_k = NP / BR, nb_out = (n_aout + BR - 1) / BR;
    const uint32_t b = smem_u32(&bar);
    auto issue = [&](const CUtensorMap *map, int nb, int pr) {  // thread 0: nb boxes of one column pair
        mbar_expect_tx(b, (uint32_t)(nb * BR * sizeof(float4)));
        for (int k = 0; k < nb; ++k) tma_load_2d(smem_u32(sin + k * BR), map, 4 * pr, k * BR, b);
    };
    if (t == 0) {
        mbar_init(b, 1);
        mbar_fence_init();
    }
    {
        constexpr int n4t = (TWN + 1) / 2;  // float4 loads of the (even-padded) table
        const float4 *ts = reinterpret_cast<const float4 *>(twp);
        float4 *td = reinterpret_cast<float4 *>(T);
        for (int i = t; i < n4t; i += NT) td[i] = __ldg(ts + i);
    }
    __syncthreads();
    const int npairs = Lr / 2;
    int pair = blockIdx.x;
    if (t == 0 && pair < npairs) issue(&imap, nb_in, pair);
    uint32_t parity = 0;
    auto wait = [&]() -> bool {
        if (__syncthreads_or(!mbar_wait(b, parity))) {
            if (t == 0) atomicExch(err, 1);
            mbar_wait(b, parity);
            return false;
        }
        parity ^= 1u;
        return true;
    };
    for (; pair < npairs; pair += gridDim.x) {
        if (!wait()) return;  // the input rows of the pair
        float2 a0[kPassE], a1[kPassE];
#pragma unroll
        for (int r = 0; r < kPassE; ++r) {
            const int q = t + r * NT;
            const float4 v = q < n_in ? sin[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            a0[r] = make_float2(v.x, v.y);
            a1[r] = make_float2(v.z, v.w);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (t == 0) issue(&kmap, nb_k, pair);
        float2 c0[Gl][Rl], c1[Gl][Rl];
        pt_row<LOGP, false>(a0, z, T, t, c0);
        pt_row<LOGP, false>(a1, z, T, t, c1);
        if (!wait()) return;  // Khat's pair
#pragma unroll
        for (int g = 0; g < Gl; ++g)
#pragma unroll
            for (int q = 0; q < Rl; ++q) {
                const float4 k = sin[t + (g + q * Gl) * NT];
                a0[g + q * Gl] = cmul(c0[g][q], make_float2(k.x, k.y));
                a1[g + q * Gl] = cmul(c1[g][q], make_float2(k.z, k.w));
            }
        fence_proxy_async_smem();
        __syncthreads();
        if (t == 0) {
            if (pair + (int)gridDim.x < npairs) issue(&imap, nb_in, pair + gridDim.x);
            bulk_wait_read<0>();  // the previous pair's stores have read the out buffer
        }
        // (the barrier at the start of each transform orders that wait before the writes below)
        pt_row<LOGP, true>(a0, z, T, t, c0);
#pragma unroll
        for (int g = 0; g < Gl; ++g)
#pragma unroll
            for (int q = 0; q < Rl; ++q) {
                const int r = (t + (g + q * Gl) * NT - a_lo) & (NP - 1);
                if (r < n_aout) reinterpret_cast<float2 *>(sout + r)[0] = c0[g][q];
            }
        pt_row<LOGP, true>(a1, z, T, t, c1);
#pragma unroll
        for (int g = 0; g < Gl; ++g)
#pragma unroll
            for (int q = 0; q < Rl; ++q) {
                const int r = (t + (g + q * Gl) * NT - a_lo) & (NP - 1);
                if (r < n_aout) reinterpret_cast<float2 *>(sout + r)[1] = c1[g][q];
            }
        fence_proxy_async_smem();
        __syncthreads();
        if (t == 0) {
            for (int k = 0; k < nb_out; ++k) tma_store_2d(&omap, 4 * pair, k * BR, smem_u32(sout + k * BR));
            bulk_commit();
        }
    }
    if (t == 0) bulk_wait_all();
}

// Persistent forms of the two row passes for Lr = 2^(LOGH + 1), LOGH = 9 .. 13 (lp_rows.cuh).
// Forward along rho of rows (2b, 2b + 1) < n_rows: the sector's Step 1 samples go straight to
// registers (the second row is zero when n_rows is odd).
template <typename Tin, int LOGH>
__global__ void __launch_bounds__((1 << LOGH) / kPassE, 1)
lpp_rows_fwd_pt_kernel(const Tin *__restrict__ sino, int n_det, const int4 *__restrict__ atab,
                       const int4 *__restrict__ rowtab, const int2 *__restrict__ stab, int n_rho, int n_rows,
                       float2 *__restrict__ Tout, const float2 *__restrict__ twp, const float2 *__restrict__ twL) {
    constexpr int H = 1 << LOGH, L = 2 * H, NT = H / kPassE;
    extern __shared__ __align__(128) float2 z[];  // [H] work | per-pass twiddles | [H] E outputs
    float2 *Tw = z + lp_rows_pt_tw_off<LOGH>();
    float2 *sE = Tw + lp_rows_pt_twn<LOGH>();
    const int t = threadIdx.x;
    lp_stage_pass_twiddles<LOGH>(Tw, twp, t);
    for (int pr = blockIdx.x; 2 * pr < n_rows; pr += gridDim.x) {
        const int q0 = 2 * pr, q1 = q0 + 1;
        const bool has1 = q1 < n_rows;
        const int4 a0 = __ldg(atab + q0), r0 = __ldg(rowtab + q0);
        const int4 a1 = has1 ? __ldg(atab + q1) : a0, r1 = has1 ? __ldg(rowtab + q1) : r0;
        float2 ae[kPassE], ao[kPassE];
#pragma unroll
        for (int r = 0; r < kPassE; ++r) {
            const int i = 2 * (t + r * NT);  // even sample i, odd sample i + 1
            float2 ve = make_float2(0.f, 0.f), vo = ve;
            if (i < n_rho) {
                const int2 s = __ldg(stab + i);
                ve.x = lpp_sample(sino, n_det, a0, r0, s);
                if (has1) ve.y = lpp_sample(sino, n_det, a1, r1, s);
            }
            if (i + 1 < n_rho) {
                const int2 s = __ldg(stab + i + 1);
                vo.x = lpp_sample(sino, n_det, a0, r0, s);
                if (has1) vo.y = lpp_sample(sino, n_det, a1, r1, s);
            }
            ae[r] = ve;
            ao[r] = vo;
        }
        float2 xl[kPassE], xu[kPassE];
        lp_dit_row<LOGH, false>(ae, ao, z, Tw, sE, twL, t, xl, xu);
        lp_separate_store<LOGH>(xl, xu, z, t, Tout + (long long)q0 * L, has1 ? Tout + (long long)q1 * L : nullptr);
    }
}

// Inverse along rho of output rows (2b, 2b + 1) < n_rows: outputs c_lo .. c_lo + n_out - 1 to B.
template <int LOGH>
__global__ void __launch_bounds__((1 << LOGH) / kPassE, 1)
lpp_rows_inv_pt_kernel(const float2 *__restrict__ Tin, float *__restrict__ B, const float2 *__restrict__ twp,
                       const float2 *__restrict__ twL, int n_rows, int c_lo, int n_out) {
    constexpr int H = 1 << LOGH, L = 2 * H, NT = H / kPassE;
    extern __shared__ __align__(128) float2 z[];  // [H] work | per-pass twiddles | [H] E outputs
    float2 *Tw = z + lp_rows_pt_tw_off<LOGH>();
    float2 *sE = Tw + lp_rows_pt_twn<LOGH>();
    const int t = threadIdx.x;
    lp_stage_pass_twiddles<LOGH>(Tw, twp, t);
    for (int pr = blockIdx.x; 2 * pr < n_rows; pr += gridDim.x) {
        const int q0 = 2 * pr, q1 = q0 + 1;
        const bool has1 = q1 < n_rows;
        const float4 *ta = reinterpret_cast<const float4 *>(Tin + (long long)q0 * L);
        const float4 *tb = reinterpret_cast<const float4 *>(Tin + (long long)q1 * L);
        float2 ae[kPassE], ao[kPassE];
#pragma unroll
        for (int r = 0; r < kPassE; ++r) {
            const int j = t + r * NT;  // entries 2j, 2j + 1 of both rows
            const float4 va = __ldg(ta + j), vb = has1 ? __ldg(tb + j) : make_float4(0.f, 0.f, 0.f, 0.f);
            ae[r] = make_float2(va.x - vb.y, va.y + vb.x);
            ao[r] = make_float2(va.z - vb.w, va.w + vb.z);
        }
        float2 xl[kPassE], xu[kPassE];
        lp_dit_row<LOGH, true>(ae, ao, z, Tw, sE, twL, t, xl, xu);
        float *b0 = B + (long long)q0 * n_out, *b1 = B + (long long)q1 * n_out;
#pragma unroll
        for (int m = 0; m < kPassE; ++m) {
            const int n = t + m * NT - c_lo, nu = n + H;
            if (n >= 0 && n < n_out) {
                b0[n] = xl[m].x;
                if (has1) b1[n] = xl[m].y;
            }
            if (nu >= 0 && nu < n_out) {
                b0[nu] = xu[m].x;
                if (has1) b1[nu] = xu[m].y;
            }
        }
    }
}

// Inverse transform along rho of output rows (2b, 2b+1) < n_rows (both real, packed as
// T_a + i T_b); outputs c_lo .. c_lo + n_out - 1 go to B.
template <int E>
__global__ void __launch_bounds__(1024, 1)
lpp_rows_inv_kernel(const float2 *__restrict__ T, float *__restrict__ B, const float2 *__restrict__ tw, int logL,
                    int n_rows, int c_lo, int n_out) {
    extern __shared__ __align__(128) float2 z[];
    const int L = 1 << logL;
    float2 *tws = z + L;
    stage_twiddles(tws, tw, L / 2);
    const int q0 = 2 * blockIdx.x, q1 = q0 + 1;
    const bool has1 = q1 < n_rows;
    const float2 *ta = T + (long long)q0 * L, *tb = T + (long long)q1 * L;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        const float2 a = ta[k], b = has1 ? tb[k] : make_float2(0.f, 0.f);
        z[k] = make_float2(a.x - b.y, a.y + b.x);
    }
    __syncthreads();
    stockham_fft<E>(z, logL, tws, 1, true, threadIdx.x, blockDim.x);
    for (int c = threadIdx.x; c < n_out; c += blockDim.x) {
        const float2 v = z[c_lo + c];
        B[(long long)q0 * n_out + c] = v.x;
        if (has1) B[(long long)q1 * n_out + c] = v.y;
    }
}

// Step 4 for one sector: pixel p adds B at its (rho node + fraction, angle node + fraction).
__global__ void __launch_bounds__(256)
lpp_cart_kernel(const float *__restrict__ B, const int4 *__restrict__ pix, float *__restrict__ img, int NN, int n_out,
                int accumulate) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NN) return;
    const int4 t = __ldg(pix + p);
    const float fc = __int_as_float(t.y), fa = __int_as_float(t.w);
    const float *r0 = B + (long long)t.z * n_out + t.x, *r1 = r0 + n_out;
    const float v0 = fmaf(fc, __ldg(r0 + 1) - __ldg(r0), __ldg(r0));
    const float v1 = fmaf(fc, __ldg(r1 + 1) - __ldg(r1), __ldg(r1));
    const float v = fmaf(fa, v1 - v0, v0);
    img[p] = accumulate ? img[p] + v : v;
}

// Per-sector pixel tables in FP64: (c0, fc, a0, fa) of ln |x - O'| and of the angle of x - O'.
struct PixGeom {
    double dx, d, rho0, drho, dphi;
    int N, K, c_lo, a_lo, n_out, n_aout, Q;
};

__global__ void __launch_bounds__(256)
lpp_pix_kernel(int4 *__restrict__ pix, PixGeom G) {
    const long long NN = (long long)G.N * G.N;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= NN * G.Q) return;
    const int q = (int)(e / NN);
    const long long p = e - (long long)q * NN;
    const int iy = (int)(p / G.N), ix = (int)(p - (long long)iy * G.N);
    const double x = -1.0 + (ix + 0.5) * G.dx, y = -1.0 + (iy + 0.5) * G.dx;
    const double phic = (q * (double)G.K + 0.5 * (G.K - 1)) * G.dphi;
    const double ux = cos(phic), uy = sin(phic);
    const double px = x + G.d * ux, py = y + G.d * uy;
    const double rho = 0.5 * log(px * px + py * py);
    const double ang = phic + atan2(-uy * px + ux * py, ux * px + uy * py);
    const double c = (rho - G.rho0) / G.drho - G.c_lo;
    const double a = ang / G.dphi - ((double)q * G.K + G.a_lo);
    double c0 = floor(c), a0 = floor(a);
    c0 = fmin(fmax(c0, 0.0), (double)(G.n_out - 2));
    a0 = fmin(fmax(a0, 0.0), (double)(G.n_aout - 2));
    pix[e] = make_int4((int)c0, __float_as_int((float)(c - c0)), (int)a0, __float_as_int((float)(a - a0)));
}

int pow2_ge(long long n) {
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

std::vector<float2> half_twiddles(int n) {
    std::vector<float2> tw(std::max(1, n / 2));
    for (int i = 0; i < n / 2; ++i) {
        const double an = -2.0 * M_PI * (double)i / (double)n;
        tw[i] = make_float2((float)std::cos(an), (float)std::sin(an));
    }
    return tw;
}

int fbits(float f) {
    int i;
    std::memcpy(&i, &f, sizeof i);
    return i;
}

// value = k + f with integer k and f in [0, 1)
void split(double v, int &k, float &f) {
    const double fl = std::floor(v);
    k = (int)fl;
    f = (float)(v - fl);
    if (f >= 1.0f) {  // rounding up to 1
        k += 1;
        f = 0.f;
    }
}

int cols_per_cta_lpp(int Lp) { return std::max(1, std::min(8, (int)(131072 / (sizeof(float2) * Lp)))); }

template <typename Tin, int LOGH>
bp_status rows_fwd_lpp_pt(bp_plan *p, const Tin *sino, int q, cudaStream_t st) {
    LppWork &w = p->lpp;
    constexpr size_t smem = lp_rows_pt_smem<LOGH>();
    auto kern = lpp_rows_fwd_pt_kernel<Tin, LOGH>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (1 << LOGH) / kPassE, smem));
    const int ctas = std::min((w.K + 1) / 2, std::max(1, per_sm) * std::max(1, p->sm_count));
    kern<<<ctas, (1 << LOGH) / kPassE, smem, st>>>(sino, p->n_det, w.atab + (size_t)q * w.K, w.rowtab, w.stab,
                                                    w.n_rho, w.K, w.T, w.twPassH, w.twLr);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

template <int LOGH>
bp_status rows_inv_lpp_pt(bp_plan *p, cudaStream_t st) {
    LppWork &w = p->lpp;
    constexpr size_t smem = lp_rows_pt_smem<LOGH>();
    auto kern = lpp_rows_inv_pt_kernel<LOGH>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (1 << LOGH) / kPassE, smem));
    const int ctas = std::min((w.n_aout + 1) / 2, std::max(1, per_sm) * std::max(1, p->sm_count));
    kern<<<ctas, (1 << LOGH) / kPassE, smem, st>>>(w.T, w.B, w.twPassH, w.twLr, w.n_aout, w.c_lo, w.n_out);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

template <typename Tin>
bp_status rows_fwd_lpp(bp_plan *p, const Tin *sino, int q, int kernel_src, cudaStream_t st) {
    LppWork &w = p->lpp;
    if (!kernel_src && w.twPassH) {
        switch (ilog2(w.Lr) - 1) {
            case 9: return rows_fwd_lpp_pt<Tin, 9>(p, sino, q, st);
            case 10: return rows_fwd_lpp_pt<Tin, 10>(p, sino, q, st);
            case 11: return rows_fwd_lpp_pt<Tin, 11>(p, sino, q, st);
            case 12: return rows_fwd_lpp_pt<Tin, 12>(p, sino, q, st);
            case 13: return rows_fwd_lpp_pt<Tin, 13>(p, sino, q, st);
            default: break;
        }
    }
    const size_t smem = sizeof(float2) * ((size_t)w.Lr + w.Lr / 2);
    auto kern = fft_elems(w.Lr) == 16 ? lpp_rows_fwd_kernel<Tin, 16> : lpp_rows_fwd_kernel<Tin, 8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int n_rows = kernel_src ? w.Lp : w.K;
    kern<<<(n_rows + 1) / 2, fft_threads(w.Lr), smem, st>>>(sino, p->n_det, w.atab + (size_t)q * w.K, w.rowtab,
                                                            w.stab, w.kfrac, kernel_src, w.n_rho, n_rows, w.T, w.twLr,
                                                            ilog2(w.Lr));
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

template <int LOGP>
bp_status cols_lpp_pt(bp_plan *p, cudaStream_t st) {
    LppWork &w = p->lpp;
    constexpr size_t smem = lpp_cols_pt_smem<LOGP>();
    auto kern = lpp_cols_pt_kernel<LOGP>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (1 << LOGP) / kPassE, smem));
    const int ctas = std::min(w.Lr / 2, std::max(1, per_sm) * std::max(1, p->sm_count));
    kern<<<ctas, (1 << LOGP) / kPassE, smem, st>>>(w.Tin_map, w.Tout_map, w.K_map, w.twPassLp, w.Lr, w.K, w.a_lo,
                                                    w.n_aout, std::min(256, w.Lp), p->d_err);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

bp_status cols_lpp(bp_plan *p, int prep, float scale, cudaStream_t st) {
    LppWork &w = p->lpp;
    if (!prep && w.maps_ok && w.twPassLp) {
        switch (ilog2(w.Lp)) {
            case 9: return cols_lpp_pt<9>(p, st);
            case 10: return cols_lpp_pt<10>(p, st);
            case 11: return cols_lpp_pt<11>(p, st);
            case 12: return cols_lpp_pt<12>(p, st);
            default: break;
        }
    }
    const int C = cols_per_cta_lpp(w.Lp);
    const size_t smem = sizeof(float2) * ((size_t)C * w.Lp + w.Lp / 2);
    auto kern = fft_elems(w.Lp) == 16 ? lpp_cols_kernel<16> : lpp_cols_kernel<8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nthr = fft_threads(w.Lp);
    int groups = 1;
    while (groups * 2 <= C && nthr * groups * 2 <= 1024) groups *= 2;
    kern<<<w.Lr / C, nthr * groups, smem, st>>>(w.T, w.Khat, w.twLp, ilog2(w.Lp), w.Lr, C, prep ? w.Lp : w.K, prep,
                                                scale, w.a_lo, w.n_aout);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

bp_status ensure_lpp(bp_plan *p, int Q, float a_r, cudaStream_t st) {
    LppWork &w = p->lpp;
    if (w.T && w.Q == Q && w.a_r == a_r) return BP_OK;
    free_logpolar_partial(p);
    const int N = p->N, n_det = p->n_det, n_theta = p->n_theta;
    const double dx = 2.0 / N, dt = p->dt, R = std::sqrt(2.0);
    const int n_half = pow2_ge(std::max(n_theta, 1));
    if (Q < 1 || n_half % Q) return fail(BP_ERR_INVALID_ARG, "sectors must be a power of two dividing the angle nodes");
    const int K = n_half / Q;
    const double dphi = M_PI / n_half, d = R * (1.0 - a_r) / a_r;
    const double beta = 0.5 * (K - 1) * dphi, alpha = std::asin(R / d), gamma = alpha + beta + 3.0 * dphi;
    if (!(gamma < 0.5 * M_PI))
        return fail(BP_ERR_INVALID_ARG, "sector too wide for the shift: use more sectors or a smaller a_r");
    const double step = -std::log(1.0 - dt / (d + R));
    const double rho0 = std::log((d - R) * std::cos(gamma)) - 2.0 * step, top = std::log(d + R);
    const long long n_rho = (long long)std::ceil((top - rho0) / step) + 1;
    const double drho = (top - rho0) / (double)(n_rho - 1);
    const int c_lo = (int)std::floor((std::log(d - R) - rho0) / drho);
    const long long n_out = n_rho - c_lo;
    const double A = alpha / dphi;
    const int a_lo = (int)std::floor(0.5 * (K - 1) - A) - 1, a_hi = (int)std::ceil(0.5 * (K - 1) + A) + 1;
    const int n_aout = a_hi - a_lo + 1;
    const int b_lo = a_lo - (K - 1), b_hi = a_hi;
    const int kmax = (int)std::floor(-std::log(std::cos(std::max(-b_lo, b_hi) * dphi)) / drho) + 1;
    const long long Lr_req = n_rho + kmax + 1;
    const long long Lp_req = std::max<long long>({(long long)(b_hi - b_lo + 1), (long long)n_aout, (long long)K});
    if (Lr_req > kMaxLPP || Lp_req > kMaxLPP)
        return fail(BP_ERR_UNSUPPORTED, "partial log-polar: mesh too fine for the shared-memory transforms");
    w.Q = Q;
    w.a_r = a_r;
    w.K = K;
    w.n_half = n_half;
    w.n_rho = (int)n_rho;
    w.c_lo = c_lo;
    w.n_out = (int)n_out;
    w.a_lo = a_lo;
    w.n_aout = n_aout;
    w.Lr = pow2_ge(Lr_req);
    w.Lp = pow2_ge(Lp_req);
    // Step 1 tables: s_i / dt split per mu node; the shift d cos(phi_j - phi_c) / dt split per
    // sector row (the same for every sector); bracketing projections per angle node
    const double c0 = 0.5 * (n_det - 1);
    std::vector<int2> stab(n_rho);
    for (long long i = 0; i < n_rho; ++i) {
        int k;
        float f;
        split(std::exp(rho0 + (double)i * drho) / dt, k, f);
        stab[i] = make_int2(k, fbits(f));
    }
    std::vector<int4> rowtab(K);
    for (int jp = 0; jp < K; ++jp) {
        const double D = d * std::cos((jp - 0.5 * (K - 1)) * dphi) / dt;
        int kp, kn;
        float fp, fn;
        split(-D + c0, kp, fp);
        split(D + c0, kn, fn);
        rowtab[jp] = make_int4(kp, fbits(fp), kn, fbits(fn));
    }
    std::vector<std::pair<double, int>> th(n_theta);
    for (int k = 0; k < n_theta; ++k) {
        double a = std::fmod(p->theta[k], M_PI);
        if (a < 0) a += M_PI;
        if (a >= M_PI) a = 0.0;
        th[k] = {a, k};
    }
    std::stable_sort(th.begin(), th.end(),
                     [](const std::pair<double, int> &x, const std::pair<double, int> &y) { return x.first < y.first; });
    std::vector<int4> atab(n_half);
    for (int j = 0; j < n_half; ++j) {
        const double tq = j * dphi;  // in [0, pi)
        const int a = (int)(std::upper_bound(th.begin(), th.end(), std::make_pair(tq, 0x7fffffff),
                                             [](const std::pair<double, int> &x, const std::pair<double, int> &y) {
                                                 return x.first < y.first;
                                             }) - th.begin()) - 1;
        int lo, hi, slo, shi;
        double alo, ahi;
        if (a < 0) {
            lo = n_theta - 1; alo = th[lo].first - M_PI; slo = 1;
            hi = 0; ahi = th[0].first; shi = 0;
        } else if (a == n_theta - 1) {
            lo = n_theta - 1; alo = th[lo].first; slo = 0;
            hi = 0; ahi = th[0].first + M_PI; shi = 1;
        } else {
            lo = a; alo = th[a].first; slo = 0;
            hi = a + 1; ahi = th[a + 1].first; shi = 0;
        }
        atab[j] = make_int4(th[lo].second | (slo << 30), th[hi].second | (shi << 30),
                            fbits((float)((tq - alo) / (ahi - alo))), 0);
    }
    // Step 2: kernel node and fraction per row of the angular transform (lag b at row b mod Lp)
    std::vector<float2> kfrac(w.Lp, make_float2(-1.f, 0.f));
    for (int b = b_lo; b <= b_hi; ++b) {
        const double r = -std::log(std::cos(b * dphi)) / drho;
        const double a0 = std::floor(r);
        kfrac[((b % w.Lp) + w.Lp) % w.Lp] = make_float2((float)a0, (float)(r - a0));
    }
    const std::vector<float2> twr = half_twiddles(w.Lr), twp = half_twiddles(w.Lp);
    const size_t NN = (size_t)N * N;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess) w.bytes += bytes;
    };
    alloc((void **)&w.stab, sizeof(int2) * stab.size());
    alloc((void **)&w.rowtab, sizeof(int4) * rowtab.size());
    alloc((void **)&w.atab, sizeof(int4) * atab.size());
    alloc((void **)&w.kfrac, sizeof(float2) * kfrac.size());
    alloc((void **)&w.twLr, sizeof(float2) * twr.size());
    alloc((void **)&w.twLp, sizeof(float2) * twp.size());
    std::vector<float2> twph;  // per-pass twiddles of the Lr/2-point transform (the persistent row passes)
    if (w.Lr / 2 >= 512 && w.Lr / 2 <= 8192) {
        build_pass_twiddles(ilog2(w.Lr / 2), twph);
        twph.resize((twph.size() + 1) & ~(size_t)1);
        alloc((void **)&w.twPassH, sizeof(float2) * twph.size());
    }
    std::vector<float2> twpp;  // per-pass twiddles of the Lp-point transform (the persistent column pass)
    if (w.Lp >= 512 && w.Lp <= 4096) {
        build_pass_twiddles(ilog2(w.Lp), twpp);
        twpp.resize((twpp.size() + 1) & ~(size_t)1);
        alloc((void **)&w.twPassLp, sizeof(float2) * twpp.size());
    }
    alloc((void **)&w.T, sizeof(float2) * (size_t)w.Lp * w.Lr);
    alloc((void **)&w.Khat, sizeof(float2) * (size_t)w.Lp * w.Lr);
    alloc((void **)&w.B, sizeof(float) * (size_t)(n_aout + 1) * w.n_out);
    alloc((void **)&w.pix, sizeof(int4) * NN * Q);
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up(w.stab, stab.data(), sizeof(int2) * stab.size());
    up(w.rowtab, rowtab.data(), sizeof(int4) * rowtab.size());
    up(w.atab, atab.data(), sizeof(int4) * atab.size());
    up(w.kfrac, kfrac.data(), sizeof(float2) * kfrac.size());
    up(w.twLr, twr.data(), sizeof(float2) * twr.size());
    up(w.twLp, twp.data(), sizeof(float2) * twp.size());
    if (!twpp.empty()) up(w.twPassLp, twpp.data(), sizeof(float2) * twpp.size());
    if (!twph.empty()) up(w.twPassH, twph.data(), sizeof(float2) * twph.size());
    if (e != cudaSuccess) {
        free_logpolar_partial(p);
        return cuda_fail(e, "partial log-polar workspace");
    }
    // T (its first K rows as input, its first n_aout rows as output) and Khat as FP32
    // [rows][2 Lr] for the column pass's TMA copies (one column pair per box)
    w.maps_ok = false;
    if (PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder()) {
        const cuuint64_t gstride[1] = {(cuuint64_t)w.Lr * sizeof(float2)};
        const cuuint32_t box[2] = {4, (cuuint32_t)std::min(256, w.Lp)};
        const cuuint32_t estr[2] = {1, 1};
        auto encode = [&](CUtensorMap *m, void *base, int rows) {
            const cuuint64_t gdim[2] = {(cuuint64_t)2 * w.Lr, (cuuint64_t)rows};
            return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, gdim, gstride, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        };
        w.maps_ok = n_aout <= w.Lp && K <= w.Lp && encode(&w.Tin_map, w.T, K) && encode(&w.Tout_map, w.T, n_aout) &&
                    encode(&w.K_map, w.Khat, w.Lp);
    }
    PixGeom G{dx, d, rho0, drho, dphi, N, K, c_lo, a_lo, (int)n_out, n_aout, Q};
    const long long total = (long long)NN * Q;
    lpp_pix_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(w.pix, G);
    bp_status s = cudaGetLastError() == cudaSuccess ? BP_OK : fail(BP_ERR_CUDA, "partial log-polar pixel tables");
    // kernel transform, scaled by dphi / (Lp Lr) (the two inverse transforms are unnormalised)
    if (s == BP_OK) s = rows_fwd_lpp<float>(p, nullptr, 0, 1, st);
    if (s == BP_OK) s = cols_lpp(p, 1, (float)(dphi / ((double)w.Lp * w.Lr)), st);
    if (s != BP_OK) {
        free_logpolar_partial(p);
        return s;
    }
    return BP_OK;
}

}  // namespace

void free_logpolar_partial(bp_plan *p) {
    LppWork &w = p->lpp;
    cudaFree(w.stab);
    cudaFree(w.rowtab);
    cudaFree(w.atab);
    cudaFree(w.kfrac);
    cudaFree(w.twLr);
    cudaFree(w.twLp);
    cudaFree(w.twPassLp);
    cudaFree(w.twPassH);
    cudaFree(w.T);
    cudaFree(w.Khat);
    cudaFree(w.B);
    cudaFree(w.pix);
    w = LppWork();
}

bp_status launch_logpolar_partial(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, int sectors,
                                  float a_r, cudaStream_t st) {
    bp_status s = ensure_lpp(p, sectors, a_r, st);
    if (s != BP_OK) return s;
    LppWork &w = p->lpp;
    const int N = p->N, NN = N * N;
    const size_t esz = dt == BP_F32 ? 4 : 2;
    const size_t smemL = sizeof(float2) * ((size_t)w.Lr + w.Lr / 2);
    auto kinv = fft_elems(w.Lr) == 16 ? lpp_rows_inv_kernel<16> : lpp_rows_inv_kernel<8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemL));
    stage_begin(p, st);
    for (int b = 0; b < batch; ++b) {
        const char *sb = (const char *)sino + esz * (size_t)b * p->n_theta * p->n_det;
        float *ib = img + (size_t)b * NN;
        for (int q = 0; q < w.Q; ++q) {
            switch (dt) {
                case BP_F32: s = rows_fwd_lpp(p, (const float *)sb, q, 0, st); break;
                case BP_BF16: s = rows_fwd_lpp(p, (const __nv_bfloat16 *)sb, q, 0, st); break;
                case BP_F16: s = rows_fwd_lpp(p, (const __half *)sb, q, 0, st); break;
            }
            if (s != BP_OK) return s;
            stage_mark(p, st, "lpp_rows_fwd_kernel");
            if ((s = cols_lpp(p, 0, 1.f, st)) != BP_OK) return s;
            stage_mark(p, st, "lpp_cols_kernel");
            switch (w.twPassH ? ilog2(w.Lr) - 1 : 0) {
                case 9: s = rows_inv_lpp_pt<9>(p, st); break;
                case 10: s = rows_inv_lpp_pt<10>(p, st); break;
                case 11: s = rows_inv_lpp_pt<11>(p, st); break;
                case 12: s = rows_inv_lpp_pt<12>(p, st); break;
                case 13: s = rows_inv_lpp_pt<13>(p, st); break;
                default:
                    kinv<<<(w.n_aout + 1) / 2, fft_threads(w.Lr), smemL, st>>>(w.T, w.B, w.twLr, ilog2(w.Lr),
                                                                               w.n_aout, w.c_lo, w.n_out);
            }
            if (s != BP_OK) return s;
            stage_mark(p, st, "lpp_rows_inv_kernel");
            lpp_cart_kernel<<<(NN + 255) / 256, 256, 0, st>>>(w.B, w.pix + (size_t)q * NN, ib, NN, w.n_out, q > 0);
            BP_CUDA_TRY(cudaGetLastError());
            stage_mark(p, st, "lpp_cart_kernel");
        }
    }
    return BP_OK;
}

}  // namespace bp
