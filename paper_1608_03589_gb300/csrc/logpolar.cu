// Andersson's log-polar backprojection as the paper implements it (Section 5.1, Steps 1-4,
// with the adaptive rho_0 of Section 5.2): in log-polar coordinates x = e^rho xi_theta,
// s = e^mu the backprojection is a convolution (eq "andersson"),
//     [R* g]_L(rho, theta) = int int g_L(mu, phi) delta(1 - e^{rho - mu} cos(theta - phi)) dmu dphi,
// so it is computed by 2D FFTs on a uniform (mu, phi) mesh.
//
// Meshes (image [-1, 1]^2, N pixels, dx = 2/N; detector pitch dt): rho_0 = ln(dx/2);
// s_max = t_{n_det-1} + dt; N_rho = ceil((ln s_max - rho_0) / -ln(1 - dt/s_max)) + 1 nodes
// mu_i = rho_0 + i drho (the outermost step at most the detector pitch, eq "N_rho");
// N_phi = 2^ceil(log2(2 n_theta)) angles phi_j = 2 pi j / N_phi; output nodes rho_0 + c drho,
// c < N_out, reaching the farthest pixel centre; convolution length L = 2^ceil(log2(N_rho +
// N_out)) along rho (linear), N_phi along phi (circular).
//
// Step 1 (fused into the first transform): g_L(mu_i, phi_j) by linear interpolation along the
// detector (zero off it) and between the two projections bracketing the angle (cyclic, with
// g(t, theta + pi) = g(-t, theta)); every weight comes from FP64 host tables.
// Step 2: delta(1 - e^{rho'} cos theta') is a unit point mass at rho' = -ln cos theta' for
// cos theta' > 0, the hat of unit mass on the two nodes around it (the printed indicator of
// eq "calc_and_kernel" has twice the mass); its 2D transform is built once per plan by the
// same transform kernels, scaled by dphi / (N_phi L).
// Step 3: rows along rho (two real rows packed in one complex transform, then separated),
// columns along phi (C adjacent columns per CTA: forward, times the kernel transform,
// inverse, in place), rows along rho inverse (two real outputs packed).
// Step 4: bilinear interpolation at the pixel centres from an FP64 per-pixel table (cyclic
// in theta); the centre of an odd image takes the mean over the angles at rho_0.
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

constexpr int kMaxLP = 16384;  // longest transform held in shared memory
constexpr int kLpBatch = 8;    // column-segment loads in flight per thread

// Row source of the first transform: the log-polar resampled sinogram, or the kernel.
template <typename Tin>
__device__ __forceinline__ float lp_sample(const Tin *__restrict__ sino, int n_det, const int4 a, const int4 *rtab,
                                           int i) {
    // a = (ka | sign_a << 30, kb | sign_b << 30, bits(w), 0); rtab[i] = (j+, bits(f+), j-, bits(f-))
    const int4 r = __ldg(rtab + i);
    float v[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int code = e == 0 ? a.x : a.y;
        const int k = code & 0x3fffffff;
        const bool neg = (code >> 30) & 1;
        const int j = neg ? r.z : r.x;
        const float f = __int_as_float(neg ? r.w : r.y);
        const Tin *row = sino + (long long)k * n_det;
        const float g0 = (j >= 0 && j < n_det) ? load_f(row + j) : 0.f;
        const float g1 = (j + 1 >= 0 && j + 1 < n_det) ? load_f(row + j + 1) : 0.f;
        v[e] = fmaf(f, g1 - g0, g0);
    }
    const float w = __int_as_float(a.z);
    return fmaf(w, v[1] - v[0], v[0]);
}

// Forward transform along rho of row pair (2b, 2b+1): rows from the sinogram (kernel_src = 0)
// or the kernel hat (kernel_src = 1); the two spectra are separated and written to T.
template <typename Tin, int E>
__global__ void __launch_bounds__(1024, 1)
lp_rows_fwd_kernel(const Tin *__restrict__ sino, int n_det, const int4 *__restrict__ atab,
                   const int4 *__restrict__ rtab, const float2 *__restrict__ kfrac, int kernel_src, int n_rho,
                   float2 *__restrict__ T, const float2 *__restrict__ tw, int logL) {
    extern __shared__ __align__(128) float2 z[];
    const int L = 1 << logL;
    float2 *tws = z + L;
    stage_twiddles(tws, tw, L / 2);
    const int q0 = 2 * blockIdx.x, q1 = q0 + 1;
    if (kernel_src) {
        const float2 k0 = __ldg(kfrac + q0), k1 = __ldg(kfrac + q1);  // (node, fraction); node < 0: none
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            const int a0 = (int)k0.x, a1 = (int)k1.x;
            float va = 0.f, vb = 0.f;
            if (k0.x >= 0.f) va = (i == a0) ? 1.f - k0.y : ((i == a0 + 1) ? k0.y : 0.f);
            if (k1.x >= 0.f) vb = (i == a1) ? 1.f - k1.y : ((i == a1 + 1) ? k1.y : 0.f);
            z[i] = make_float2(va, vb);
        }
    } else {
        const int4 a0 = __ldg(atab + q0), a1 = __ldg(atab + q1);
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            float va = 0.f, vb = 0.f;
            if (i < n_rho) {
                va = lp_sample(sino, n_det, a0, rtab, i);
                vb = lp_sample(sino, n_det, a1, rtab, i);
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
        tb[k] = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
    }
}

// Transforms along phi of C adjacent columns [k0, k0 + C) of T (n_phi rows of length L).
// prep = 1: forward transform, times `scale`, written to Khat (the kernel's 2D transform);
// prep = 0: forward, times Khat, inverse, written back to T.
template <int E>
__global__ void __launch_bounds__(1024, 1)
lp_cols_kernel(float2 *__restrict__ T, float2 *__restrict__ Khat, const float2 *__restrict__ tw, int logPhi,
               int L, int C, int prep, float scale) {
    extern __shared__ __align__(128) float2 z[];
    const int n_phi = 1 << logPhi;
    float2 *tws = z + (size_t)C * n_phi;
    stage_twiddles(tws, tw, n_phi / 2);
    const long long k0 = (long long)blockIdx.x * C;
    const int nel = C * n_phi, bd = (int)blockDim.x;
    // column segments of 8 C bytes from n_phi rows: eight loads in flight per thread
    for (int e0 = threadIdx.x; e0 < nel; e0 += kLpBatch * bd) {
        float2 v[kLpBatch];
#pragma unroll
        for (int u = 0; u < kLpBatch; ++u) {
            const int e = e0 + u * bd, q = e / C, c = e - q * C;
            if (e < nel) v[u] = T[(long long)q * L + k0 + c];
        }
#pragma unroll
        for (int u = 0; u < kLpBatch; ++u) {
            const int e = e0 + u * bd, q = e / C, c = e - q * C;
            if (e < nel) z[c * n_phi + q] = v[u];
        }
    }
    __syncthreads();
    const int nthr = fft_threads(n_phi), groups = blockDim.x / nthr;
    const int g = threadIdx.x / nthr, tid = threadIdx.x - g * nthr;
    for (int c0 = 0; c0 < C; c0 += groups) stockham_fft<E>(z + (c0 + g) * n_phi, logPhi, tws, 1, false, tid, nthr);
    if (prep) {
        for (int e = threadIdx.x; e < C * n_phi; e += blockDim.x) {
            const int q = e / C, c = e - q * C;
            const float2 v = z[c * n_phi + q];
            Khat[(long long)q * L + k0 + c] = make_float2(scale * v.x, scale * v.y);
        }
        return;
    }
    for (int e0 = threadIdx.x; e0 < nel; e0 += kLpBatch * bd) {
        float2 kv[kLpBatch];
#pragma unroll
        for (int u = 0; u < kLpBatch; ++u) {
            const int e = e0 + u * bd, q = e / C, c = e - q * C;
            if (e < nel) kv[u] = __ldg(Khat + (long long)q * L + k0 + c);
        }
#pragma unroll
        for (int u = 0; u < kLpBatch; ++u) {
            const int e = e0 + u * bd, q = e / C, c = e - q * C;
            if (e < nel) z[c * n_phi + q] = cmul(z[c * n_phi + q], kv[u]);
        }
    }
    __syncthreads();
    for (int c0 = 0; c0 < C; c0 += groups) stockham_fft<E>(z + (c0 + g) * n_phi, logPhi, tws, 1, true, tid, nthr);
    for (int e = threadIdx.x; e < C * n_phi; e += blockDim.x) {
        const int q = e / C, c = e - q * C;
        T[(long long)q * L + k0 + c] = z[c * n_phi + q];
    }
}

// The same column pass (prep = 0) over column pairs through the TMA, with the persistent
// transform (first and last passes in registers, per-pass twiddles in shared memory): the pair
// of T arrives by 2D TMA loads (boxes of 16 bytes x BR rows) in a staging buffer and both
// columns' inputs go to registers; the pair of Khat then arrives in the same buffer during the
// forward transforms and is multiplied into their register outputs, which are the inverse
// transforms' inputs; the next pair of T is requested before the inverse transforms, and the
// result leaves through a second staging buffer by 2D TMA stores.  Every wait is bounded: on
// expiry the kernel sets *err, waits (bounded) for its copy once more and returns.
template <int LOGP>
__host__ __device__ constexpr int lp_cols_stage_off() {
    return ((1 << LOGP) + pt_offset<LOGP>(PtPlan<LOGP>::npass) + 15) & ~15;
}
template <int LOGP>
constexpr size_t lp_cols_pt_smem() {
    return sizeof(float2) * ((size_t)lp_cols_stage_off<LOGP>() + 4 * (size_t)(1 << LOGP));
}

template <int LOGP>
__global__ void __launch_bounds__((1 << LOGP) / kPassE, 1)
lp_cols_pt_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap kmap,
                  const float2 *__restrict__ twp, int L, int BR, int *__restrict__ err) {
    using PL = PtPlan<LOGP>;
    constexpr int NP = 1 << LOGP, NT = NP / kPassE, Rl = PL::Rl, Gl = kPassE / Rl;
    constexpr int TWN = pt_offset<LOGP>(PL::npass);
    extern __shared__ __align__(128) float2 z[];  // [NP] work | [TWN] twiddles | [NP] pairs in | [NP] pairs out
    __shared__ __align__(8) unsigned long long bar;
    float2 *T = z + NP;
    float4 *sin = reinterpret_cast<float4 *>(z + lp_cols_stage_off<LOGP>());
    float4 *sout = sin + NP;
    const int t = threadIdx.x, nbox = NP / BR;
    const uint32_t b = smem_u32(&bar);
    auto issue = [&](const CUtensorMap *map, int pr) {  // thread 0: one column pair of map
        mbar_expect_tx(b, (uint32_t)(NP * sizeof(float4)));
        for (int k = 0; k < nbox; ++k) tma_load_2d(smem_u32(sin + k * BR), map, 4 * pr, k * BR, b);
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
    const int npairs = L / 2;
    int pair = blockIdx.x;
    if (t == 0 && pair < npairs) issue(&tmap, pair);
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
        if (!wait()) return;  // T's pair
        float2 a0[kPassE], a1[kPassE];
#pragma unroll
        for (int r = 0; r < kPassE; ++r) {
            const float4 v = sin[t + r * NT];
            a0[r] = make_float2(v.x, v.y);
            a1[r] = make_float2(v.z, v.w);
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (t == 0) issue(&kmap, pair);
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
            if (pair + (int)gridDim.x < npairs) issue(&tmap, pair + gridDim.x);
            bulk_wait_read<0>();  // the previous pair's stores have read the out buffer
        }
        // (the barrier at the start of each transform orders that wait before the writes below)
        pt_row<LOGP, true>(a0, z, T, t, c0);
#pragma unroll
        for (int g = 0; g < Gl; ++g)
#pragma unroll
            for (int q = 0; q < Rl; ++q) reinterpret_cast<float2 *>(sout + t + (g + q * Gl) * NT)[0] = c0[g][q];
        pt_row<LOGP, true>(a1, z, T, t, c1);
#pragma unroll
        for (int g = 0; g < Gl; ++g)
#pragma unroll
            for (int q = 0; q < Rl; ++q) reinterpret_cast<float2 *>(sout + t + (g + q * Gl) * NT)[1] = c1[g][q];
        fence_proxy_async_smem();
        __syncthreads();
        if (t == 0) {
            for (int k = 0; k < nbox; ++k) tma_store_2d(&tmap, 4 * pair, k * BR, smem_u32(sout + k * BR));
            bulk_commit();
        }
    }
    if (t == 0) bulk_wait_all();
}

// Inverse transform along rho of row pair (2b, 2b+1), both real: packed as T_a + i T_b; the
// first n_out outputs of each go to B.
template <int E>
__global__ void __launch_bounds__(1024, 1)
lp_rows_inv_kernel(const float2 *__restrict__ T, float *__restrict__ B, const float2 *__restrict__ tw, int logL,
                   int n_out) {
    extern __shared__ __align__(128) float2 z[];
    const int L = 1 << logL;
    float2 *tws = z + L;
    stage_twiddles(tws, tw, L / 2);
    const int q0 = 2 * blockIdx.x, q1 = q0 + 1;
    const float2 *ta = T + (long long)q0 * L, *tb = T + (long long)q1 * L;
    for (int k = threadIdx.x; k < L; k += blockDim.x) {
        const float2 a = ta[k], b = tb[k];
        z[k] = make_float2(a.x - b.y, a.y + b.x);
    }
    __syncthreads();
    stockham_fft<E>(z, logL, tws, 1, true, threadIdx.x, blockDim.x);
    for (int c = threadIdx.x; c < n_out; c += blockDim.x) {
        const float2 v = z[c];
        B[(long long)q0 * n_out + c] = v.x;
        B[(long long)q1 * n_out + c] = v.y;
    }
}

// Persistent forms of the two row passes for L = 2^(LOGH + 1), LOGH = 9 .. 13 (lp_rows.cuh).
// Forward along rho of row pairs (2b, 2b + 1): the log-polar samples of the two rows (packed as
// one complex row, zero from n_rho on) go straight to registers.
template <typename Tin, int LOGH>
__global__ void __launch_bounds__((1 << LOGH) / kPassE, 1)
lp_rows_fwd_pt_kernel(const Tin *__restrict__ sino, int n_det, const int4 *__restrict__ atab,
                      const int4 *__restrict__ rtab, int n_rho, int n_rows, float2 *__restrict__ Tout,
                      const float2 *__restrict__ twp, const float2 *__restrict__ twL) {
    constexpr int H = 1 << LOGH, L = 2 * H, NT = H / kPassE;
    extern __shared__ __align__(128) float2 z[];  // [H] work | per-pass twiddles | [H] E outputs
    float2 *Tw = z + lp_rows_pt_tw_off<LOGH>();
    float2 *sE = Tw + lp_rows_pt_twn<LOGH>();
    const int t = threadIdx.x;
    lp_stage_pass_twiddles<LOGH>(Tw, twp, t);
    for (int pr = blockIdx.x; 2 * pr < n_rows; pr += gridDim.x) {
        const int q0 = 2 * pr, q1 = q0 + 1;
        const int4 a0 = __ldg(atab + q0), a1 = __ldg(atab + q1);
        float2 ae[kPassE], ao[kPassE];
#pragma unroll
        for (int r = 0; r < kPassE; ++r) {
            const int i = 2 * (t + r * NT);  // even sample i, odd sample i + 1
            ae[r] = i < n_rho ? make_float2(lp_sample(sino, n_det, a0, rtab, i), lp_sample(sino, n_det, a1, rtab, i))
                              : make_float2(0.f, 0.f);
            ao[r] = i + 1 < n_rho
                        ? make_float2(lp_sample(sino, n_det, a0, rtab, i + 1), lp_sample(sino, n_det, a1, rtab, i + 1))
                        : make_float2(0.f, 0.f);
        }
        float2 xl[kPassE], xu[kPassE];
        lp_dit_row<LOGH, false>(ae, ao, z, Tw, sE, twL, t, xl, xu);
        lp_separate_store<LOGH>(xl, xu, z, t, Tout + (long long)q0 * L, Tout + (long long)q1 * L);
    }
}

// Inverse along rho of row pairs (2b, 2b + 1): Z = T_a + i T_b split into even and odd entries
// at the load (16-byte pairs), the first n_out outputs of each real row to B.
template <int LOGH>
__global__ void __launch_bounds__((1 << LOGH) / kPassE, 1)
lp_rows_inv_pt_kernel(const float2 *__restrict__ Tin, float *__restrict__ B, const float2 *__restrict__ twp,
                      const float2 *__restrict__ twL, int n_rows, int n_out) {
    constexpr int H = 1 << LOGH, L = 2 * H, NT = H / kPassE;
    extern __shared__ __align__(128) float2 z[];  // [H] work | per-pass twiddles | [H] E outputs
    float2 *Tw = z + lp_rows_pt_tw_off<LOGH>();
    float2 *sE = Tw + lp_rows_pt_twn<LOGH>();
    const int t = threadIdx.x;
    lp_stage_pass_twiddles<LOGH>(Tw, twp, t);
    for (int pr = blockIdx.x; 2 * pr < n_rows; pr += gridDim.x) {
        const int q0 = 2 * pr, q1 = q0 + 1;
        const float4 *ta = reinterpret_cast<const float4 *>(Tin + (long long)q0 * L);
        const float4 *tb = reinterpret_cast<const float4 *>(Tin + (long long)q1 * L);
        float2 ae[kPassE], ao[kPassE];
#pragma unroll
        for (int r = 0; r < kPassE; ++r) {
            const int j = t + r * NT;  // entries 2j, 2j + 1 of both rows
            const float4 va = __ldg(ta + j), vb = __ldg(tb + j);
            ae[r] = make_float2(va.x - vb.y, va.y + vb.x);
            ao[r] = make_float2(va.z - vb.w, va.w + vb.z);
        }
        float2 xl[kPassE], xu[kPassE];
        lp_dit_row<LOGH, true>(ae, ao, z, Tw, sE, twL, t, xl, xu);
        float *b0 = B + (long long)q0 * n_out, *b1 = B + (long long)q1 * n_out;
#pragma unroll
        for (int m = 0; m < kPassE; ++m) {
            const int n = t + m * NT;
            if (n < n_out) {
                b0[n] = xl[m].x;
                b1[n] = xl[m].y;
            }
            if (n + H < n_out) {
                b0[n + H] = xu[m].x;
                b1[n + H] = xu[m].y;
            }
        }
    }
}

// Step 4: pixel p takes B at its (rho node + fraction, theta node + fraction).
__global__ void __launch_bounds__(256)
lp_cart_kernel(const float *__restrict__ B, const int4 *__restrict__ pix, float *__restrict__ img, int NN, int n_phi,
               int n_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NN) return;
    const int4 t = __ldg(pix + p);
    if (t.x < 0) return;  // the centre of an odd image (lp_centre_kernel)
    const float fc = __int_as_float(t.y), fb = __int_as_float(t.w);
    const int b1 = (t.z + 1 == n_phi) ? 0 : t.z + 1;
    const float *r0 = B + (long long)t.z * n_out + t.x, *r1 = B + (long long)b1 * n_out + t.x;
    const float v0 = fmaf(fc, __ldg(r0 + 1) - __ldg(r0), __ldg(r0));
    const float v1 = fmaf(fc, __ldg(r1 + 1) - __ldg(r1), __ldg(r1));
    img[p] = fmaf(fb, v1 - v0, v0);
}

// The centre pixel of an odd image: mean of B over the angles at rho_0 (fixed-order block sum).
__global__ void __launch_bounds__(256)
lp_centre_kernel(const float *__restrict__ B, float *__restrict__ img, int centre, int n_phi, int n_out) {
    __shared__ float red[256];
    float s = 0.f;
    for (int q = threadIdx.x; q < n_phi; q += blockDim.x) s += __ldg(B + (long long)q * n_out);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) img[centre] = red[0] / (float)n_phi;
}

int pow2_at_least(long long n) {
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

template <typename Tin, int LOGH>
bp_status rows_fwd_pt(bp_plan *p, const Tin *sino, cudaStream_t st) {
    LogPolarWork &w = p->lp;
    constexpr size_t smem = lp_rows_pt_smem<LOGH>();
    auto kern = lp_rows_fwd_pt_kernel<Tin, LOGH>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (1 << LOGH) / kPassE, smem));
    const int ctas = std::min(w.n_phi / 2, std::max(1, per_sm) * std::max(1, p->sm_count));
    kern<<<ctas, (1 << LOGH) / kPassE, smem, st>>>(sino, p->n_det, w.atab, w.rtab, w.n_rho, w.n_phi, w.T, w.twPassH,
                                                    w.twL);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

template <int LOGH>
bp_status rows_inv_pt(bp_plan *p, cudaStream_t st) {
    LogPolarWork &w = p->lp;
    constexpr size_t smem = lp_rows_pt_smem<LOGH>();
    auto kern = lp_rows_inv_pt_kernel<LOGH>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (1 << LOGH) / kPassE, smem));
    const int ctas = std::min(w.n_phi / 2, std::max(1, per_sm) * std::max(1, p->sm_count));
    kern<<<ctas, (1 << LOGH) / kPassE, smem, st>>>(w.T, w.B, w.twPassH, w.twL, w.n_phi, w.n_out);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

template <typename Tin>
bp_status rows_fwd(bp_plan *p, const Tin *sino, int kernel_src, cudaStream_t st) {
    LogPolarWork &w = p->lp;
    if (!kernel_src && w.twPassH) {
        switch (ilog2(w.L) - 1) {
            case 9: return rows_fwd_pt<Tin, 9>(p, sino, st);
            case 10: return rows_fwd_pt<Tin, 10>(p, sino, st);
            case 11: return rows_fwd_pt<Tin, 11>(p, sino, st);
            case 12: return rows_fwd_pt<Tin, 12>(p, sino, st);
            case 13: return rows_fwd_pt<Tin, 13>(p, sino, st);
            default: break;
        }
    }
    const size_t smem = sizeof(float2) * ((size_t)w.L + w.L / 2);
    auto kern = fft_elems(w.L) == 16 ? lp_rows_fwd_kernel<Tin, 16> : lp_rows_fwd_kernel<Tin, 8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<w.n_phi / 2, fft_threads(w.L), smem, st>>>(sino, p->n_det, w.atab, w.rtab, w.kfrac, kernel_src, w.n_rho,
                                                      w.T, w.twL, ilog2(w.L));
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

int cols_per_cta(int n_phi) { return std::max(1, std::min(4, (int)(131072 / (sizeof(float2) * n_phi)))); }

template <int LOGP>
bp_status cols_pt(bp_plan *p, cudaStream_t st) {
    LogPolarWork &w = p->lp;
    constexpr size_t smem = lp_cols_pt_smem<LOGP>();
    auto kern = lp_cols_pt_kernel<LOGP>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int ctas = std::min(w.L / 2, std::max(1, p->sm_count));
    kern<<<ctas, (1 << LOGP) / kPassE, smem, st>>>(w.T_map, w.K_map, w.twPassPhi, w.L, std::min(256, w.n_phi),
                                                    p->d_err);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

bp_status cols(bp_plan *p, int prep, float scale, cudaStream_t st) {
    LogPolarWork &w = p->lp;
    if (!prep && w.maps_ok && w.twPassPhi) {
        switch (ilog2(w.n_phi)) {
            case 9: return cols_pt<9>(p, st);
            case 10: return cols_pt<10>(p, st);
            case 11: return cols_pt<11>(p, st);
            case 12: return cols_pt<12>(p, st);
            default: break;
        }
    }
    const int C = cols_per_cta(w.n_phi);
    const size_t smem = sizeof(float2) * ((size_t)C * w.n_phi + w.n_phi / 2);
    auto kern = fft_elems(w.n_phi) == 16 ? lp_cols_kernel<16> : lp_cols_kernel<8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nthr = fft_threads(w.n_phi);
    int groups = 1;
    while (groups * 2 <= C && nthr * groups * 2 <= 1024) groups *= 2;
    kern<<<w.L / C, nthr * groups, smem, st>>>(w.T, w.Khat, w.twPhi, ilog2(w.n_phi), w.L, C, prep, scale);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

std::vector<float2> twiddles(int n) {
    std::vector<float2> tw(std::max(1, n / 2));
    for (int i = 0; i < n / 2; ++i) {
        const double an = -2.0 * M_PI * (double)i / (double)n;
        tw[i] = make_float2((float)std::cos(an), (float)std::sin(an));
    }
    return tw;
}

int f2i(float f) {
    int i;
    std::memcpy(&i, &f, sizeof i);
    return i;
}

bp_status ensure_logpolar(bp_plan *p, cudaStream_t st) {
    LogPolarWork &w = p->lp;
    if (w.T) return BP_OK;
    const int N = p->N, n_det = p->n_det, n_theta = p->n_theta;
    const double dx = 2.0 / N, dt = p->dt;
    const double s_max = 0.5 * (n_det - 1) * dt + dt;
    const double rho0 = std::log(0.5 * dx), top = std::log(s_max);
    if (n_det < 2 || !(top > rho0)) return fail(BP_ERR_UNSUPPORTED, "log-polar: needs n_det >= 2 and a detector wider than half a pixel");
    const double step = -std::log(1.0 - dt / s_max);
    const long long n_rho = (long long)std::ceil((top - rho0) / step) + 1;
    const double drho = (top - rho0) / (double)(n_rho - 1);
    const double r_far = std::sqrt(2.0) * (1.0 - 0.5 * dx);
    const long long n_out = (long long)std::ceil((std::log(std::max(r_far, 0.5 * dx)) - rho0) / drho) + 2;
    const int n_phi = pow2_at_least(2LL * n_theta);
    const long long Lreq = n_rho + n_out;
    if (Lreq > kMaxLP || n_phi > kMaxLP)
        return fail(BP_ERR_UNSUPPORTED, "log-polar: mesh too fine for the shared-memory transforms (N up to about 2048)");
    const int L = pow2_at_least(Lreq);
    w.n_rho = (int)n_rho;
    w.n_out = (int)n_out;
    w.n_phi = n_phi;
    w.L = L;
    w.rho0 = rho0;
    w.drho = drho;
    // Step 1 tables: detector bin and fraction of +-s_i, bracketing projections per phi_j
    std::vector<int4> rtab(n_rho);
    for (long long i = 0; i < n_rho; ++i) {
        const double s = std::exp(rho0 + (double)i * drho);
        int4 r;
        const double up = s / dt + 0.5 * (n_det - 1), un = -s / dt + 0.5 * (n_det - 1);
        const double jp = std::floor(up), jn = std::floor(un);
        r.x = (int)jp;
        r.y = f2i((float)(up - jp));
        r.z = (int)jn;
        r.w = f2i((float)(un - jn));
        rtab[i] = r;
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
    std::vector<int4> atab(n_phi);
    for (int q = 0; q < n_phi; ++q) {
        const double phi = 2.0 * M_PI * q / n_phi;
        double tq = std::fmod(phi, M_PI);
        const int sq = phi < M_PI ? 0 : 1;  // 1: negative detector coordinate
        // last sorted angle <= tq
        int a = (int)(std::upper_bound(th.begin(), th.end(), std::make_pair(tq, 0x7fffffff),
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
        int4 e;
        e.x = th[lo].second | ((slo ^ sq) << 30);
        e.y = th[hi].second | ((shi ^ sq) << 30);
        e.z = f2i((float)((tq - alo) / (ahi - alo)));
        e.w = 0;
        atab[q] = e;
    }
    // Step 2: kernel node and fraction per angle offset
    std::vector<float2> kfrac(n_phi);
    for (int b = 0; b < n_phi; ++b) {
        const double c = std::cos(2.0 * M_PI * b / n_phi);
        kfrac[b] = make_float2(-1.f, 0.f);
        if (c <= 0.0) continue;
        const double r = -std::log(c) / drho;
        const double a0 = std::floor(r);
        if (a0 >= (double)n_out) continue;
        kfrac[b] = make_float2((float)a0, (float)(r - a0));
    }
    // Step 4: per-pixel table
    const size_t NN = (size_t)N * N;
    std::vector<int4> pix(NN);
    for (int iy = 0; iy < N; ++iy) {
        const double y = -1.0 + (iy + 0.5) * dx;
        for (int ix = 0; ix < N; ++ix) {
            const double x = -1.0 + (ix + 0.5) * dx;
            const double r = std::hypot(x, y);
            int4 e;
            if (r <= 0.0) {
                e = make_int4(-1, 0, 0, 0);
            } else {
                double c = (std::log(r) - rho0) / drho;
                c = std::min(std::max(c, 0.0), (double)n_out - 1.0);
                double c0 = std::min(std::floor(c), (double)n_out - 2.0);
                double ph = std::atan2(y, x);
                if (ph < 0) ph += 2.0 * M_PI;
                const double pb = ph / (2.0 * M_PI / n_phi);
                double b0 = std::floor(pb);
                const double fb = pb - b0;
                int bi = (int)b0 % n_phi;
                e = make_int4((int)c0, f2i((float)(c - c0)), bi, f2i((float)fb));
            }
            pix[(size_t)iy * N + ix] = e;
        }
    }
    const std::vector<float2> twL = twiddles(L), twP = twiddles(n_phi);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess) w.bytes += bytes;
    };
    alloc((void **)&w.rtab, sizeof(int4) * rtab.size());
    alloc((void **)&w.atab, sizeof(int4) * atab.size());
    alloc((void **)&w.kfrac, sizeof(float2) * kfrac.size());
    alloc((void **)&w.pix, sizeof(int4) * pix.size());
    alloc((void **)&w.twL, sizeof(float2) * twL.size());
    alloc((void **)&w.twPhi, sizeof(float2) * twP.size());
    std::vector<float2> twph;  // per-pass twiddles of the L/2-point transform (the persistent row passes)
    if (L / 2 >= 512 && L / 2 <= 8192) {
        build_pass_twiddles(ilog2(L / 2), twph);
        twph.resize((twph.size() + 1) & ~(size_t)1);
        alloc((void **)&w.twPassH, sizeof(float2) * twph.size());
    }
    std::vector<float2> twpp;  // per-pass twiddles of the n_phi-point transform (the persistent column pass)
    if (n_phi >= 512 && n_phi <= 4096) {
        build_pass_twiddles(ilog2(n_phi), twpp);
        twpp.resize((twpp.size() + 1) & ~(size_t)1);
        alloc((void **)&w.twPassPhi, sizeof(float2) * twpp.size());
    }
    alloc((void **)&w.T, sizeof(float2) * (size_t)n_phi * L);
    alloc((void **)&w.Khat, sizeof(float2) * (size_t)n_phi * L);
    alloc((void **)&w.B, sizeof(float) * (size_t)n_phi * n_out);
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up(w.rtab, rtab.data(), sizeof(int4) * rtab.size());
    up(w.atab, atab.data(), sizeof(int4) * atab.size());
    up(w.kfrac, kfrac.data(), sizeof(float2) * kfrac.size());
    up(w.pix, pix.data(), sizeof(int4) * pix.size());
    up(w.twL, twL.data(), sizeof(float2) * twL.size());
    up(w.twPhi, twP.data(), sizeof(float2) * twP.size());
    if (!twpp.empty()) up(w.twPassPhi, twpp.data(), sizeof(float2) * twpp.size());
    if (!twph.empty()) up(w.twPassH, twph.data(), sizeof(float2) * twph.size());
    if (e != cudaSuccess) {
        free_logpolar(p);
        return cuda_fail(e, "log-polar workspace");
    }
    // T and Khat as FP32 [n_phi][2L] for the column pass's TMA copies (one column pair per box)
    w.maps_ok = false;
    if (PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder()) {
        const cuuint64_t gdim[2] = {(cuuint64_t)2 * L, (cuuint64_t)n_phi};
        const cuuint64_t gstride[1] = {(cuuint64_t)L * sizeof(float2)};
        const cuuint32_t box[2] = {4, (cuuint32_t)std::min(256, n_phi)};
        const cuuint32_t estr[2] = {1, 1};
        auto encode = [&](CUtensorMap *m, void *base) {
            return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, gdim, gstride, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
        };
        w.maps_ok = encode(&w.T_map, w.T) && encode(&w.K_map, w.Khat);
    }
    // kernel transform, scaled by dphi / (N_phi L) (the two inverse transforms are unnormalised)
    bp_status s = rows_fwd<float>(p, nullptr, 1, st);
    if (s == BP_OK) s = cols(p, 1, (float)((2.0 * M_PI / n_phi) / ((double)n_phi * L)), st);
    if (s != BP_OK) {
        free_logpolar(p);
        return s;
    }
    return BP_OK;
}

}  // namespace

void free_logpolar(bp_plan *p) {
    LogPolarWork &w = p->lp;
    cudaFree(w.rtab);
    cudaFree(w.atab);
    cudaFree(w.kfrac);
    cudaFree(w.pix);
    cudaFree(w.twL);
    cudaFree(w.twPhi);
    cudaFree(w.twPassPhi);
    cudaFree(w.twPassH);
    cudaFree(w.T);
    cudaFree(w.Khat);
    cudaFree(w.B);
    w = LogPolarWork();
}

bp_status launch_logpolar(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, cudaStream_t st) {
    bp_status s = ensure_logpolar(p, st);
    if (s != BP_OK) return s;
    LogPolarWork &w = p->lp;
    const int N = p->N;
    const size_t esz = dt == BP_F32 ? 4 : 2;
    const size_t smemL = sizeof(float2) * ((size_t)w.L + w.L / 2);
    auto kinv = fft_elems(w.L) == 16 ? lp_rows_inv_kernel<16> : lp_rows_inv_kernel<8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemL));
    stage_begin(p, st);
    for (int b = 0; b < batch; ++b) {
        const char *sb = (const char *)sino + esz * (size_t)b * p->n_theta * p->n_det;
        switch (dt) {
            case BP_F32: s = rows_fwd(p, (const float *)sb, 0, st); break;
            case BP_BF16: s = rows_fwd(p, (const __nv_bfloat16 *)sb, 0, st); break;
            case BP_F16: s = rows_fwd(p, (const __half *)sb, 0, st); break;
        }
        if (s != BP_OK) return s;
        stage_mark(p, st, "lp_rows_fwd_kernel");
        if ((s = cols(p, 0, 1.f, st)) != BP_OK) return s;
        stage_mark(p, st, "lp_cols_kernel");
        switch (w.twPassH ? ilog2(w.L) - 1 : 0) {
            case 9: s = rows_inv_pt<9>(p, st); break;
            case 10: s = rows_inv_pt<10>(p, st); break;
            case 11: s = rows_inv_pt<11>(p, st); break;
            case 12: s = rows_inv_pt<12>(p, st); break;
            case 13: s = rows_inv_pt<13>(p, st); break;
            default: kinv<<<w.n_phi / 2, fft_threads(w.L), smemL, st>>>(w.T, w.B, w.twL, ilog2(w.L), w.n_out);
        }
        if (s != BP_OK) return s;
        stage_mark(p, st, "lp_rows_inv_kernel");
        float *ib = img + (size_t)b * N * N;
        const int NN = N * N;
        lp_cart_kernel<<<(NN + 255) / 256, 256, 0, st>>>(w.B, w.pix, ib, NN, w.n_phi, w.n_out);
        if (N % 2 == 1) lp_centre_kernel<<<1, 256, 0, st>>>(w.B, ib, (N / 2) * N + N / 2, w.n_phi, w.n_out);
        BP_CUDA_TRY(cudaGetLastError());
        stage_mark(p, st, "lp_cart_kernel");
    }
    return BP_OK;
}

}  // namespace bp
