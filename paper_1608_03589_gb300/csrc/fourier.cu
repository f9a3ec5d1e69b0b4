// Fourier form of R*: the Backprojection Slice Theorem (Section 3, eq "bst") evaluated as a
// type-1 non-uniform FFT (Section 5.3, Steps 2.2-4, with Step 3 realised as gridding).
//
// With G_k[m] the P-point DFT of projection k (zero-padded, Step 2.2) and the Nyquist bin
// dropped, the backprojection of the band-limited interpolant of every projection is
//     b(x) = Re sum_k sum_{m=0}^{P/2-1} c_{k,m} exp(2 pi i kappa_m xi_k . x),
//     c_{k,m} = (w_k / P) (m ? 2 : 1) G_k[m] exp(i pi m (n_det-1) / P),  kappa_m = m / (P dt).
// The BST's 1/sigma is cancelled by the polar area element |sigma| (Section 6, eq
// "reg_fbp"), so the samples carry plain quadrature weights.  In grid units of an
// M x M oversampled frequency grid (M = 2^ceil(log2(2N))), sample (k, m) sits at
//     z = m rho xi_k,   rho = M dx / (P dt),
// and the image is  b(i) = Re sum_s c'_s exp(2 pi i z_s . i' / M),  i' = i - floor(N/2),
// c'_s = c_s exp(2 pi i delta (z_x + z_y) / M), delta = floor(N/2) - (N-1)/2.
// Gridding spreads every c'_s onto the grid with a separable Kaiser-Bessel kernel of
// width W = 6 (Beatty et al.'s beta for the actual oversampling M/N), two pruned 1D
// inverse FFT passes produce the N x N output, and dividing by the kernel's Fourier
// transform (deapodisation) removes the kernel.
//
// Kernels: (1) the projection spectra: P-point FFTs of projection pairs in shared memory
// (persistent, per-pass twiddles, for P = 512 ... 4096), the two half spectra scaled into
// c'_{k,m} (quadrature weight, Hermitian factor, detector and half-pixel phases);
// (2) gridding as a gather: one thread per pair of adjacent grid cells walks only the rays
// whose angle falls in the pair's footprint as seen from the origin (O(1) lookup for uniform
// angle sets, else binary search in the sorted angles), and on each ray only the samples
// inside the footprint, sharing the sample value and the x weight between the two cells; the
// separable kernel comes from an FP64-built table with linear interpolation.  A cell's work
// grows as it nears the origin, so blocks are dispatched from the origin outwards and the
// core square (where nearly every ray passes) takes one to eight warps per cell in ring order.
// No atomics, deterministic, one store per cell;  (3) the two pruned inverse-FFT passes
// (persistent, per-pass twiddles, for M = 512 ... 8192): rows l_x in pairs into a transposed
// intermediate, then rows i_y with deapodisation and the real part.  The adjoint R_F mirrors
// them: forward passes (the padding never loaded), interpolation at the polar samples by
// 64 x 64 grid tiles staged in shared memory, and the Hermitian inverse row transforms.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "fft.cuh"
#include "fft_pt.cuh"
#include "lp_rows.cuh"
#include "tma.cuh"

namespace bp {

namespace {

constexpr int kKB = 2048;         // kernel table intervals on [0, W/2]
constexpr int kCore = 64;         // cells with max(|u_x|, |u_y|) < kCore are gathered by a warp each

struct SortedRay {                // one ray, in increasing angle order
    long long ax, ay;             // rho cos(phi), rho sin(phi) in 32.32 fixed point (grid cells per sample)
    float isx, isy;               // 1 / (rho cos), 1 / (rho sin) (infinite for a zero component)
    float sx, sy;                 // ax, ay as float (per-sample steps)
    int k;                        // original projection index
    int pad;
};

// Kaiser-Bessel kernel phi(d) = I0(beta sqrt(1 - (2d/W)^2)) on |d| <= W/2 = HW from the table
// tab[i] = (phi(i h), phi((i+1) h) - phi(i h)), h = HW/kKB, built in FP64 on the host.  The
// width W = 2 HW is 6 (the default) or 4 (bp_set_fourier_width).
template <int HW>
__device__ __forceinline__ float kb_tab(const float2 *__restrict__ tab, float d) {
    const float x = fminf(fabsf(d) * ((float)kKB / (float)HW), (float)kKB - 1e-3f);
    const int i = (int)x;
    const float2 v = __ldg(tab + i);
    return fmaf(x - (float)i, v.y, v.x);
}

// The same lookup from a copy of the table in shared memory.
template <int HW>
__device__ __forceinline__ float kb_tab_s(const float2 *tab, float d) {
    const float x = fminf(fabsf(d) * ((float)kKB / (float)HW), (float)kKB - 1e-3f);
    const int i = (int)x;
    const float2 v = tab[i];
    return fmaf(x - (float)i, v.y, v.x);
}

__device__ __forceinline__ float2 half_pixel_phase(const long long *__restrict__ r, int m, float delta2_over_M) {
    const long long zx = (long long)m * r[0], zy = (long long)m * r[1];
    const float rx = (float)(unsigned)(zx & 0xffffffffLL) * 2.3283064365386963e-10f;
    const float ry = (float)(unsigned)(zy & 0xffffffffLL) * 2.3283064365386963e-10f;
    float sn, cs;
    sincospif(((float)((int)(zx >> 32) + (int)(zy >> 32)) + (rx + ry)) * delta2_over_M, &sn, &cs);
    return make_float2(cs, sn);
}

// ---------------------------------------------------------------------------------- (1) spectra
template <typename Tin, int E>
__global__ void __launch_bounds__(1024, 1)
fourier_spectra_kernel(const Tin *__restrict__ sino, float2 *__restrict__ spec, const float *__restrict__ wk,
                       const float2 *__restrict__ tw, int n_theta, int n_det, int logP, float wuni,
                       const long long *__restrict__ ray, float delta2_over_M, const float *__restrict__ Hf) {
    extern __shared__ __align__(128) float2 z[];
    const int P = 1 << logP, H = P >> 1;
    float2 *tws = z + P;  // P/2 twiddles
    stage_twiddles(tws, tw, H);
    const int k0 = 2 * blockIdx.x, k1 = k0 + 1;
    const bool has1 = k1 < n_theta;
    const Tin *a = sino + (long long)k0 * n_det;
    const Tin *b = sino + (long long)k1 * n_det;
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        float va = 0.f, vb = 0.f;
        if (j < n_det) {
            va = load_f(a + j);
            if (has1) vb = load_f(b + j);
        }
        z[j] = make_float2(va, vb);
    }
    __syncthreads();
    stockham_fft<E>(z, logP, tws, 1, false, threadIdx.x, blockDim.x);
    if (Hf) {
        // fused FBP filter, the same steps as bp_filter: times the response (dt/P included),
        // inverse transform, the filtered rows cut to the detector, transformed again
        for (int j = threadIdx.x; j < P; j += blockDim.x) {
            const float h = __ldg(Hf + j);
            const float2 v = z[j];
            z[j] = make_float2(v.x * h, v.y * h);
        }
        __syncthreads();
        stockham_fft<E>(z, logP, tws, 1, true, threadIdx.x, blockDim.x);
        // an unpaired last projection keeps an exactly zero partner row, as when reloaded
        for (int j = threadIdx.x; j < P; j += blockDim.x) {
            if (j >= n_det) z[j] = make_float2(0.f, 0.f);
            else if (!has1) z[j].y = 0.f;
        }
        __syncthreads();
        stockham_fft<E>(z, logP, tws, 1, false, threadIdx.x, blockDim.x);
    }
    // A[m] = (Z[m] + conj Z[P-m]) / 2,  B[m] = (Z[m] - conj Z[P-m]) / (2i)
    const float wa = (wuni > 0.f ? wuni : __ldg(wk + k0)) / (float)P;
    const float wb = has1 ? (wuni > 0.f ? wuni : __ldg(wk + k1)) / (float)P : 0.f;
    const long long twoP = 2LL * P;
    for (int m = threadIdx.x; m < H; m += blockDim.x) {
        const float2 zm = z[m];
        const float2 zc = z[(P - m) & (P - 1)];
        const float2 A = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
        const float2 B = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
        // detector-centre phase exp(i pi m (n_det-1)/P), argument reduced exactly mod 2P
        const long long r = ((long long)m * (n_det - 1)) % twoP;
        float sn, cs;
        sincospif((float)r / (float)P, &sn, &cs);
        float2 pa = make_float2(cs, sn), pb = pa;
        if (delta2_over_M != 0.f) {
            // half-pixel phase exp(2 pi i delta (z_x + z_y) / M) of sample (k, m), z = m rho xi_k
            pa = cmul(pa, half_pixel_phase(ray + 2 * k0, m, delta2_over_M));
            if (has1) pb = cmul(pb, half_pixel_phase(ray + 2 * k1, m, delta2_over_M));
        }
        const float f = (m == 0) ? 1.f : 2.f;
        const float2 ca = cmul(A, pa), cb = cmul(B, pb);
        spec[(long long)k0 * H + m] = make_float2(f * wa * ca.x, f * wa * ca.y);
        if (has1) spec[(long long)k1 * H + m] = make_float2(f * wb * cb.x, f * wb * cb.y);
    }
}

// Persistent form of (1) for P = 2^9 .. 2^12 (per-pass twiddles, next pair's loads in flight
// during the current transforms).  The rows fill the first half of the zero-padded row, so
// only the first-pass inputs x[t + r NT], r < 4, are loaded.  With the fused filter the
// forward transform's outputs, times H, are the inverse transform's first-pass inputs in
// registers, and the inverse's outputs, cut to the detector, those of the second forward
// transform.  The last transform's outputs go to shared memory for the split into the two
// half spectra (as in (1)).
template <int LOGP>
__device__ __forceinline__ void pt_regs_to_inputs(float2 (&c)[kPassE / PtPlan<LOGP>::Rl][PtPlan<LOGP>::Rl],
                                                  float2 (&a)[kPassE]) {
    constexpr int Rl = PtPlan<LOGP>::Rl, Gl = kPassE / Rl;
    // last-pass output t + (g + q Gl) NT is first-pass input r = g + q Gl
#pragma unroll
    for (int g = 0; g < Gl; ++g)
#pragma unroll
        for (int q = 0; q < Rl; ++q) a[g + q * Gl] = c[g][q];
}

template <typename Tin, int LOGP>
__global__ void __launch_bounds__((1 << LOGP) / kPassE, 1024 / ((1 << LOGP) / kPassE))
fourier_spectra_pt_kernel(const Tin *__restrict__ sino, float2 *__restrict__ spec, const float *__restrict__ wk,
                          const float2 *__restrict__ twp, int n_theta, int n_det, float wuni,
                          const long long *__restrict__ ray, float delta2_over_M, const float *__restrict__ Hf) {
    using PL = PtPlan<LOGP>;
    constexpr int P = 1 << LOGP, H = P / 2, NT = P / kPassE;
    constexpr int TWN = pt_offset<LOGP>(PL::npass);
    extern __shared__ __align__(16) float2 sp_sm[];
    float2 *z = sp_sm;     // [P]
    float2 *T = z + P;     // [TWN]
    const int t = threadIdx.x;
    const int npairs = (n_theta + 1) / 2;
    float2 nxt[4];
    auto fetch = [&](int pair) {
        const int k0 = 2 * pair;
        const bool has1 = k0 + 1 < n_theta;
        const Tin *a = sino + (long long)k0 * n_det, *b = a + n_det;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int j = t + r * NT;
            float va = 0.f, vb = 0.f;
            if (j < n_det) {
                va = load_f(a + j);
                if (has1) vb = load_f(b + j);
            }
            nxt[r] = make_float2(va, vb);
        }
    };
    int pair = blockIdx.x;
    if (pair < npairs) fetch(pair);
    {
        constexpr int n4t = TWN / 2;
        const float4 *ts = reinterpret_cast<const float4 *>(twp);
        float4 *td = reinterpret_cast<float4 *>(T);
#pragma unroll
        for (int i = 0; i < (n4t + NT - 1) / NT; ++i)
            if (t + i * NT < n4t) td[t + i * NT] = __ldg(ts + t + i * NT);
    }
    constexpr int Rl = PL::Rl, Gl = kPassE / Rl;
    for (; pair < npairs; pair += gridDim.x) {
        const int k0 = 2 * pair, k1 = k0 + 1;
        const bool has1 = k1 < n_theta;
        float2 a[kPassE];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = nxt[r];
#pragma unroll
        for (int r = 4; r < kPassE; ++r) a[r] = make_float2(0.f, 0.f);
        if (pair + (int)gridDim.x < npairs) fetch(pair + gridDim.x);
        float2 c[Gl][Rl];
        pt_row<LOGP, false>(a, z, T, t, c);
        if (Hf) {
            // times the response (dt/P included), inverse transform, cut to the detector (an
            // unpaired last projection keeps a zero partner row), transformed again
#pragma unroll
            for (int g = 0; g < Gl; ++g)
#pragma unroll
                for (int q = 0; q < Rl; ++q) {
                    const float hv = __ldg(Hf + t + (g + q * Gl) * NT);
                    c[g][q] = make_float2(c[g][q].x * hv, c[g][q].y * hv);
                }
            pt_regs_to_inputs<LOGP>(c, a);
            pt_row<LOGP, true>(a, z, T, t, c);
            pt_regs_to_inputs<LOGP>(c, a);
#pragma unroll
            for (int r = 0; r < kPassE; ++r) {
                const int j = t + r * NT;
                if (j >= n_det) a[r] = make_float2(0.f, 0.f);
                else if (!has1) a[r].y = 0.f;
            }
            pt_row<LOGP, false>(a, z, T, t, c);
        }
        __syncthreads();  // every thread's last-pass reads of z are done
#pragma unroll
        for (int g = 0; g < Gl; ++g)
#pragma unroll
            for (int q = 0; q < Rl; ++q) z[t + (g + q * Gl) * NT] = c[g][q];
        __syncthreads();
        // A[m] = (Z[m] + conj Z[P-m]) / 2,  B[m] = (Z[m] - conj Z[P-m]) / (2i)
        const float wa = (wuni > 0.f ? wuni : __ldg(wk + k0)) / (float)P;
        const float wb = has1 ? (wuni > 0.f ? wuni : __ldg(wk + k1)) / (float)P : 0.f;
        const long long twoP = 2LL * P;
        for (int m = t; m < H; m += NT) {
            const float2 zm = z[m];
            const float2 zc = z[(P - m) & (P - 1)];
            const float2 A = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
            const float2 B = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
            const long long r = ((long long)m * (n_det - 1)) % twoP;
            float sn, cs;
            sincospif((float)r / (float)P, &sn, &cs);
            float2 pa = make_float2(cs, sn), pb = pa;
            if (delta2_over_M != 0.f) {
                pa = cmul(pa, half_pixel_phase(ray + 2 * k0, m, delta2_over_M));
                if (has1) pb = cmul(pb, half_pixel_phase(ray + 2 * k1, m, delta2_over_M));
            }
            const float f = (m == 0) ? 1.f : 2.f;
            const float2 ca = cmul(A, pa), cb = cmul(B, pb);
            spec[(long long)k0 * H + m] = make_float2(f * wa * ca.x, f * wa * ca.y);
            if (has1) spec[(long long)k1 * H + m] = make_float2(f * wb * cb.x, f * wb * cb.y);
        }
    }
}

// ---------------------------------------------------------------------------------- (2) gridding
// Cell l (G[l_x][l_y], l mod M) sums c'_s phi(u_x - z_x) phi(u_y - z_y) over the samples z
// with floor(z) in [u - 3, u + 2] per axis (the 6-cell footprint of the spreading form),
// u ranging over the periodic images of the cell's centred coordinate.

// Sorted-ray index range [lo, lo + count) (indices taken mod n) whose angle lies within the
// angular window of the cell's footprint box [ux - 3, ux + 3) x [uy - 3, uy + 3): the disc of
// radius 3 sqrt(2) around u seen from the origin; all rays if that disc holds the origin.
__device__ __forceinline__ int first_at_least(const float *__restrict__ sphi, const RayIndex &ri, float a) {
    if (ri.uniform) return min(ri.n, max(0, (int)ceilf((a - ri.phi0) / ri.dphi - 1e-4f)));
    int l = 0, h = ri.n;
    while (l < h) {
        const int mid = (l + h) >> 1;
        if (__ldg(sphi + mid) < a) l = mid + 1;
        else h = mid;
    }
    return l;
}

__device__ __forceinline__ void ray_range(const float *__restrict__ sphi, const RayIndex &ri, float ux, float uy,
                                          int &lo, int &count, float R = 4.2427f /* 3 sqrt(2) + margin */) {
    const float r2 = ux * ux + uy * uy;
    if (r2 <= R * R) {
        lo = 0;
        count = ri.n;
        return;
    }
    const float twopi = 6.2831853071795865f;
    const float half = asinf(R * rsqrtf(r2)) + 1e-4f;
    float a = atan2f(uy, ux) - half;
    a -= twopi * floorf(a * (1.f / twopi));  // [0, 2 pi)
    const float e = a + 2.f * half;
    lo = first_at_least(sphi, ri, a);
    count = first_at_least(sphi, ri, fminf(e, twopi) + 1e-7f) - lo;
    if (e > twopi) count += min(lo, first_at_least(sphi, ri, e - twopi + 1e-7f));
}

// Sum of the contributions of sorted rays lo + j (j = j0, j0 + dj, ...) < lo + count to
// the cell image (ux, uy).
template <int HW>
__device__ __forceinline__ float2 gather_rays(const float2 *__restrict__ spec, const SortedRay *__restrict__ sray,
                                              const float2 *__restrict__ tab, int n, int H, int ux, int uy, int lo,
                                              int count, int j0, int dj) {
    float2 acc = make_float2(0.f, 0.f);
    const float h = (float)HW;
    const float fx0 = (float)ux - h, fx1 = (float)ux + h, fy0 = (float)uy - h, fy1 = (float)uy + h;
    for (int j = j0; j < count; j += dj) {
        int i = lo + j;
        if (i >= n) i -= n;
        const SortedRay r = sray[i];
        // samples m with z = m (sx, sy) inside the box (one spare sample each side)
        const float ax0 = fx0 * r.isx, ax1 = fx1 * r.isx, ay0 = fy0 * r.isy, ay1 = fy1 * r.isy;
        float mlo = fmaxf(0.f, fmaxf(fminf(ax0, ax1), fminf(ay0, ay1)));
        float mhi = fminf((float)(H - 1), fminf(fmaxf(ax0, ax1), fmaxf(ay0, ay1)));
        if (!(mlo <= mhi + 2.f)) continue;  // also rejects NaN (0 * inf on a zero component)
        const int m0 = max(0, (int)mlo - 1), m1 = min(H - 1, (int)mhi + 1);
        const float2 *sk = spec + (long long)r.k * H;
        // exact offsets d = u - z at m0 from the fixed-point ray, then float steps (|m - m0| small)
        const long long zx = (long long)m0 * r.ax, zy = (long long)m0 * r.ay;
        const float dx0 = (float)(ux - (int)(zx >> 32)) - (float)(unsigned)(zx & 0xffffffffLL) * 2.3283064365386963e-10f;
        const float dy0 = (float)(uy - (int)(zy >> 32)) - (float)(unsigned)(zy & 0xffffffffLL) * 2.3283064365386963e-10f;
        const float sx = r.sx, sy = r.sy;
        for (int m = m0; m <= m1; ++m) {
            const float t = (float)(m - m0);
            const float dx = fmaf(-t, sx, dx0), dy = fmaf(-t, sy, dy0);
            // footprint rule of the spreading form: u - z in (-HW, HW] per axis
            if (!(dx > -h && dx <= h && dy > -h && dy <= h)) continue;
            const float2 v = __ldg(sk + m);
            const float w = kb_tab<HW>(tab, dx) * kb_tab<HW>(tab, dy);
            acc.x = fmaf(w, v.x, acc.x);
            acc.y = fmaf(w, v.y, acc.y);
        }
    }
    return acc;
}

// The pair of cells (u_x, u_y) and (u_x, u_y + 1): they share the rays of the angular window
// of their union box [u_x - HW, u_x + HW) x [u_y - HW, u_y + HW + 1) and, per sample, the
// spectrum value and the x weight.
template <int HW>
__device__ __forceinline__ void gather_rays_pair(const float2 *__restrict__ spec,
                                                 const SortedRay *__restrict__ sray, const float2 *__restrict__ tab,
                                                 int n, int H, int ux, int uy, int lo, int count, float2 &acc0,
                                                 float2 &acc1) {
    const float h = (float)HW;
    const float fx0 = (float)ux - h, fx1 = (float)ux + h, fy0 = (float)uy - h, fy1 = (float)uy + h + 1.f;
    for (int j = 0; j < count; ++j) {
        int i = lo + j;
        if (i >= n) i -= n;
        const SortedRay r = sray[i];
        // samples m with z = m (sx, sy) inside the union box (one spare sample each side)
        const float ax0 = fx0 * r.isx, ax1 = fx1 * r.isx, ay0 = fy0 * r.isy, ay1 = fy1 * r.isy;
        float mlo = fmaxf(0.f, fmaxf(fminf(ax0, ax1), fminf(ay0, ay1)));
        float mhi = fminf((float)(H - 1), fminf(fmaxf(ax0, ax1), fmaxf(ay0, ay1)));
        if (!(mlo <= mhi + 2.f)) continue;  // also rejects NaN (0 * inf on a zero component)
        const int m0 = max(0, (int)mlo - 1), m1 = min(H - 1, (int)mhi + 1);
        const float2 *sk = spec + (long long)r.k * H;
        // exact offsets d = u - z at m0 from the fixed-point ray, then float steps (|m - m0| small)
        const long long zx = (long long)m0 * r.ax, zy = (long long)m0 * r.ay;
        const float dx0 = (float)(ux - (int)(zx >> 32)) - (float)(unsigned)(zx & 0xffffffffLL) * 2.3283064365386963e-10f;
        const float dy0 = (float)(uy - (int)(zy >> 32)) - (float)(unsigned)(zy & 0xffffffffLL) * 2.3283064365386963e-10f;
        const float sx = r.sx, sy = r.sy;
        for (int m = m0; m <= m1; ++m) {
            const float t = (float)(m - m0);
            const float dx = fmaf(-t, sx, dx0), dy = fmaf(-t, sy, dy0), dy1 = dy + 1.f;
            // footprint rule of the spreading form: u - z in (-HW, HW] per axis
            if (!(dx > -h && dx <= h)) continue;
            const bool in0 = dy > -h && dy <= h, in1 = dy1 > -h && dy1 <= h;
            if (!(in0 || in1)) continue;
            const float2 v = __ldg(sk + m);
            const float kx = kb_tab<HW>(tab, dx);
            if (in0) {
                const float w = kx * kb_tab<HW>(tab, dy);
                acc0.x = fmaf(w, v.x, acc0.x);
                acc0.y = fmaf(w, v.y, acc0.y);
            }
            if (in1) {
                const float w = kx * kb_tab<HW>(tab, dy1);
                acc1.x = fmaf(w, v.x, acc1.x);
                acc1.y = fmaf(w, v.y, acc1.y);
            }
        }
    }
}

// One thread per pair of cells (l_y even, l_y + 1) outside the core square; 64 x 8 cells per
// block (stores along l_y).  A pair never straddles the l_y = M/2 wrap (M/2 is even).  The work
// of a cell grows as it nears the origin (more rays cross its footprint), so blocks are
// dispatched from the origin outwards: even block indices take chunks from the low end of
// each axis, odd ones from the high (wrapped, negative) end, and the costly blocks start first.
template <int HW>
__global__ void __launch_bounds__(256, 6)
grid_gather_pair_kernel(const float2 *__restrict__ spec, const SortedRay *__restrict__ sray,
                        const float *__restrict__ sphi, const float2 *__restrict__ tab, float2 *__restrict__ grid,
                        int M, int H, RayIndex ri, float rmax, int amax, int core) {
    const int bx = blockIdx.x, by = blockIdx.y;
    const int ly0 = (bx & 1) ? M - 64 * (1 + (bx >> 1)) : 64 * (bx >> 1);
    const int lx0 = (by & 1) ? M - 8 * (1 + (by >> 1)) : 8 * (by >> 1);
    const int ly = ly0 + 2 * (threadIdx.x & 31);
    const int lx = lx0 + (threadIdx.x >> 5);
    if (lx >= M || ly >= M) return;
    const int cx = lx < M / 2 ? lx : lx - M, cy = ly < M / 2 ? ly : ly - M;
    const bool own0 = max(abs(cx), abs(cy)) >= core, own1 = max(abs(cx), abs(cy + 1)) >= core;
    if (!own0 && !own1) return;  // the core kernel owns both cells
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
    // periodic images whose union box can reach the sample disc |z| <= rmax; with every ray
    // in the upper half plane (z_y >= 0) also u_y + 1 > -HW
    const float h = (float)HW;
    const float lim = rmax + h + 1.f, iM = 1.f / (float)M;
    const int a_lo = max(-amax, (int)ceilf((-lim - (float)cx) * iM));
    const int a_hi = min(amax, (int)floorf((lim - (float)cx) * iM));
    const int b_lo = max(-amax, (int)ceilf(((ri.upper ? -h : -lim) - (float)cy) * iM));
    const int b_hi = min(amax, (int)floorf((lim - (float)cy) * iM));
    // the disc of radius sqrt(HW^2 + (HW + 1/2)^2) (+ margin) around the pair's centre holds both boxes
    const float R = sqrtf(h * h + (h + 0.5f) * (h + 0.5f)) + 0.01f;
    for (int a = a_lo; a <= a_hi; ++a) {
        for (int b = b_lo; b <= b_hi; ++b) {
            const int ux = cx + a * M, uy = cy + b * M;
            if (ri.upper && uy <= -HW - 1) continue;  // no sample has z_y < u_y + HW + 1
            const float qx = fmaxf(0.f, fmaxf((float)ux - h, -h - (float)ux));
            const float qy = fmaxf(0.f, fmaxf((float)uy - h, -h - 1.f - (float)uy));
            if (qx * qx + qy * qy > rmax * rmax) continue;
            int lo, count;
            ray_range(sphi, ri, (float)ux, (float)uy + 0.5f, lo, count, R);
            gather_rays_pair<HW>(spec, sray, tab, ri.n, H, ux, uy, lo, count, acc0, acc1);
        }
    }
    if (own0) grid[(long long)lx * M + ly] = acc0;
    if (own1) grid[(long long)lx * M + ly + 1] = acc1;
}

// WPC warps per core cell (max(|u_x|, |u_y|) < kCore), cells [cell_begin, cell_end) of the ring
// order: lanes split the rays, warp sums, then (WPC > 1) a sum over the cell's warps.
template <int HW, int WPC>
__global__ void __launch_bounds__(256)
grid_gather_core_kernel(const float2 *__restrict__ spec, const SortedRay *__restrict__ sray,
                        const float *__restrict__ sphi, const float2 *__restrict__ tab, float2 *__restrict__ grid,
                        int M, int H, RayIndex ri, float rmax, int amax, int cell_begin, int cell_end) {
    static_assert(WPC == 1 || WPC == 2 || WPC == 4 || WPC == 8, "warps per cell");
    __shared__ float2 part[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cell = cell_begin + blockIdx.x * (8 / WPC) + warp / WPC;
    const int sub = warp % WPC;  // this warp's share of the cell's rays
    const bool live = cell < cell_end;
    // cells in square rings max(|c_x|, |c_y|) = r from the origin outwards (the inner cells,
    // crossed by every ray, start first): ring r >= 1 holds cells (2r - 1)^2 .. (2r + 1)^2 - 1
    int cx = 0, cy = 0;
    if (live && cell > 0) {
        const int r = (int)ceilf((sqrtf((float)cell + 1.f) - 1.f) * 0.5f);
        const int pidx = cell - (2 * r - 1) * (2 * r - 1), sd = pidx / (2 * r), q = pidx - sd * (2 * r);
        cx = sd == 0 ? -r + q : sd == 1 ? r : sd == 2 ? r - q : -r;
        cy = sd == 0 ? -r : sd == 1 ? -r + q : sd == 2 ? r : r - q;
    }
    float2 acc = make_float2(0.f, 0.f);
    if (live) {
        for (int a = -amax; a <= amax; ++a) {
            for (int b = -amax; b <= amax; ++b) {
                const int ux = cx + a * M, uy = cy + b * M;
                const float h = (float)HW;
                if (ri.upper && uy <= -HW) continue;  // no sample has z_y < u_y + HW
                const float qx = fmaxf(0.f, fmaxf((float)ux - h, -h - (float)ux));
                const float qy = fmaxf(0.f, fmaxf((float)uy - h, -h - (float)uy));
                if (qx * qx + qy * qy > rmax * rmax) continue;
                int lo, count;
                // the disc of radius HW sqrt(2) (+ margin) around the cell holds its box
                ray_range(sphi, ri, (float)ux, (float)uy, lo, count, h * 1.41421356f + 0.0002f);
                const float2 v = gather_rays<HW>(spec, sray, tab, ri.n, H, ux, uy, lo, count, sub * 32 + lane,
                                                 32 * WPC);
                acc.x += v.x;
                acc.y += v.y;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (WPC > 1) {
        if (lane == 0) part[warp] = acc;
        __syncthreads();
        if (sub == 0 && lane == 0) {
#pragma unroll
            for (int w = 1; w < WPC; ++w) {
                acc.x += part[warp + w].x;
                acc.y += part[warp + w].y;
            }
        }
    }
    if (live && sub == 0 && lane == 0) grid[(long long)(cx & (M - 1)) * M + (cy & (M - 1))] = acc;
}

// ---------------------------------------------------------------------------------- (3) inverse FFT passes
// R contiguous rows per CTA arrive with one bulk asynchronous copy; blockDim / fft_threads(M)
// thread groups transform them in rounds.
__device__ __forceinline__ bool load_rows_async(float2 *z, const float2 *src, int count, unsigned long long *bar) {
    const uint32_t b = smem_u32(bar);
    if (threadIdx.x == 0) {
        mbar_init(b, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(b, (uint32_t)(count * sizeof(float2)));
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
            ::"r"(smem_u32(z)), "l"(src), "r"((uint32_t)(count * sizeof(float2))), "r"(b)
            : "memory");
    }
    return mbar_wait(b, 0);
}

// Pass along y: rows l_x of G (contiguous in l_y), keep i_y in [0, N), write inter[i_y][l_x] * dy[i_y].
template <int E>
__global__ void __launch_bounds__(1024, 1)
ifft_pass_y_kernel(const float2 *__restrict__ grid, float2 *__restrict__ inter, const float *__restrict__ deap,
                   const float2 *__restrict__ tw, int M, int logM, int N, int R, int *__restrict__ err) {
    extern __shared__ __align__(128) float2 z[];
    __shared__ __align__(8) unsigned long long bar;
    float2 *tws = z + R * M;  // M/2 twiddles
    stage_twiddles(tws, tw, M / 2);
    const int lx0 = blockIdx.x * R;
    const int nthr = fft_threads(M), groups = blockDim.x / nthr;
    const int g = threadIdx.x / nthr, tid = threadIdx.x - g * nthr;
    if (__syncthreads_or(!load_rows_async(z, grid + (long long)lx0 * M, R * M, &bar))) {
        // the copy did not complete in time: record it, wait (bounded) for it once more so that
        // no copy is left in flight, and leave without computing
        if (threadIdx.x == 0) atomicExch(err, 1);
        mbar_wait(smem_u32(&bar), 0);
        return;
    }
    for (int r0 = 0; r0 < R; r0 += groups) stockham_fft<E>(z + (r0 + g) * M, logM, tws, 1, true, tid, nthr);
    const int h = N / 2;
    for (int i = threadIdx.x; i < N * R; i += blockDim.x) {
        const int iy = i / R, r = i - iy * R;
        const int pos = (iy - h) & (M - 1);
        const float d = __ldg(deap + iy);
        const float2 v = z[r * M + pos];
        inter[(long long)iy * M + lx0 + r] = make_float2(v.x * d, v.y * d);
    }
}

// Pass along x: rows i_y of inter (contiguous in l_x), keep i_x in [0, N), img = Re * dx[i_x].
template <int E>
__global__ void __launch_bounds__(1024, 1)
ifft_pass_x_kernel(const float2 *__restrict__ inter, float *__restrict__ img, const float *__restrict__ deap,
                   const float2 *__restrict__ tw, int M, int logM, int N, int R, int *__restrict__ err) {
    extern __shared__ __align__(128) float2 z[];
    __shared__ __align__(8) unsigned long long bar;
    float2 *tws = z + R * M;  // M/2 twiddles
    stage_twiddles(tws, tw, M / 2);
    const int iy0 = blockIdx.x * R;
    const int rows = min(R, N - iy0);
    const int nthr = fft_threads(M), groups = blockDim.x / nthr;
    const int g = threadIdx.x / nthr, tid = threadIdx.x - g * nthr;
    if (__syncthreads_or(!load_rows_async(z, inter + (long long)iy0 * M, rows * M, &bar))) {
        if (threadIdx.x == 0) atomicExch(err, 1);  // as in ifft_pass_y_kernel
        mbar_wait(smem_u32(&bar), 0);
        return;
    }
    // rows beyond the last image row hold stale data that is transformed but never written out
    for (int r0 = 0; r0 < R; r0 += groups) stockham_fft<E>(z + (r0 + g) * M, logM, tws, 1, true, tid, nthr);
    const int h = N / 2;
    for (int i = threadIdx.x; i < rows * N; i += blockDim.x) {
        const int r = i / N, ix = i - r * N;
        const int pos = (ix - h) & (M - 1);
        img[(long long)(iy0 + r) * N + ix] = z[r * M + pos].x * __ldg(deap + ix);
    }
}

// The spectra for P = 2^14 (no fused filter) from a persistent kernel: each P-point transform of
// a packed projection pair as two register-first P/2-point transforms combined in registers
// (lp_rows.cuh); Z[P - m] for the two rows' separation comes from the upper half through the
// work array; then the detector-centre and half-pixel phases and the weights as above.
template <typename Tin>
__global__ void __launch_bounds__(1024, 1)
fourier_spectra_split_kernel(const Tin *__restrict__ sino, float2 *__restrict__ spec, const float *__restrict__ wk,
                             const float2 *__restrict__ twp, const float2 *__restrict__ twP, int n_theta, int n_det,
                             float wuni, const long long *__restrict__ ray, float delta2_over_M) {
    constexpr int LOGH = 13, H = 1 << LOGH, P = 2 * H, NT = H / kPassE;
    extern __shared__ __align__(128) float2 z[];  // [H] work | per-pass twiddles | [H] E outputs
    float2 *Tw = z + lp_rows_pt_tw_off<LOGH>();
    float2 *sE = Tw + lp_rows_pt_twn<LOGH>();
    const int t = threadIdx.x;
    lp_stage_pass_twiddles<LOGH>(Tw, twp, t);
    const long long twoP = 2LL * P;
    for (int pr = blockIdx.x; 2 * pr < n_theta; pr += gridDim.x) {
        const int k0 = 2 * pr, k1 = k0 + 1;
        const bool has1 = k1 < n_theta;
        const Tin *a = sino + (long long)k0 * n_det;
        const Tin *b = sino + (long long)k1 * n_det;
        float2 ae[kPassE], ao[kPassE];
#pragma unroll
        for (int r = 0; r < kPassE; ++r) {
            const int i = 2 * (t + r * NT);  // even sample i, odd sample i + 1
            ae[r] = make_float2(i < n_det ? load_f(a + i) : 0.f, (has1 && i < n_det) ? load_f(b + i) : 0.f);
            ao[r] = make_float2(i + 1 < n_det ? load_f(a + i + 1) : 0.f,
                                (has1 && i + 1 < n_det) ? load_f(b + i + 1) : 0.f);
        }
        float2 xl[kPassE], xu[kPassE];
        lp_dit_row<LOGH, false>(ae, ao, z, Tw, sE, twP, t, xl, xu);
        __syncthreads();  // every thread is done with z (the second transform)
#pragma unroll
        for (int m = 0; m < kPassE; ++m) z[t + m * NT] = xu[m];
        __syncthreads();
        const float wa = (wuni > 0.f ? wuni : __ldg(wk + k0)) / (float)P;
        const float wb = has1 ? (wuni > 0.f ? wuni : __ldg(wk + k1)) / (float)P : 0.f;
#pragma unroll
        for (int mi = 0; mi < kPassE; ++mi) {
            const int m = t + mi * NT;  // Z[P - m] = X[H + (H - m)] (m > 0), X[0] for m = 0
            const float2 zm = xl[mi], zc = m == 0 ? xl[mi] : z[H - m];
            const float2 A = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
            const float2 B = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
            const long long r = ((long long)m * (n_det - 1)) % twoP;
            float sn, cs;
            sincospif((float)r / (float)P, &sn, &cs);
            float2 pa = make_float2(cs, sn), pb = pa;
            if (delta2_over_M != 0.f) {
                pa = cmul(pa, half_pixel_phase(ray + 2 * k0, m, delta2_over_M));
                if (has1) pb = cmul(pb, half_pixel_phase(ray + 2 * k1, m, delta2_over_M));
            }
            const float f = (m == 0) ? 1.f : 2.f;
            const float2 ca = cmul(A, pa), cb = cmul(B, pb);
            spec[(long long)k0 * H + m] = make_float2(f * wa * ca.x, f * wa * ca.y);
            if (has1) spec[(long long)k1 * H + m] = make_float2(f * wb * cb.x, f * wb * cb.y);
        }
    }
}

// Persistent form of the two passes for M = 2^14: each M-point transform as two register-first
// M/2-point transforms of its even and odd entries combined in registers (lp_rows.cuh); rows
// arrive as 16-byte (even, odd) pairs.  XPASS false: rows l_x of G, outputs
// inter[i_y][l_x] = z * deap[i_y] (8-byte stores); true: rows i_y of inter,
// img[i_y][i_x] = Re z * deap[i_x].  Output position pos is image index
// (pos + floor(N/2)) mod M when that is below N.
template <bool XPASS>
__global__ void __launch_bounds__(1024, 1)
ifft_split_kernel(const float2 *__restrict__ in, float2 *__restrict__ inter, float *__restrict__ img,
                  const float *__restrict__ deap, const float2 *__restrict__ twp, const float2 *__restrict__ twM,
                  int rows, int N) {
    constexpr int LOGH = 13, H = 1 << LOGH, M = 2 * H, NT = H / kPassE;
    extern __shared__ __align__(128) float2 z[];  // [H] work | per-pass twiddles | [H] E outputs
    float2 *Tw = z + lp_rows_pt_tw_off<LOGH>();
    float2 *sE = Tw + lp_rows_pt_twn<LOGH>();
    const int t = threadIdx.x, h = N / 2;
    lp_stage_pass_twiddles<LOGH>(Tw, twp, t);
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const float4 *src = reinterpret_cast<const float4 *>(in + (long long)row * M);
        float2 ae[kPassE], ao[kPassE];
#pragma unroll
        for (int r = 0; r < kPassE; ++r) {
            const float4 v = __ldg(src + t + r * NT);
            ae[r] = make_float2(v.x, v.y);
            ao[r] = make_float2(v.z, v.w);
        }
        float2 xl[kPassE], xu[kPassE];
        lp_dit_row<LOGH, true>(ae, ao, z, Tw, sE, twM, t, xl, xu);
#pragma unroll
        for (int m = 0; m < kPassE; ++m) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int pos = t + m * NT + half * H;
                const int o = pos < N - h ? pos + h : pos - (M - h);
                if (o < 0 || o >= N) continue;
                const float2 v = half ? xu[m] : xl[m];
                const float d = __ldg(deap + o);
                if (XPASS) img[(long long)row * N + o] = v.x * d;
                else inter[(long long)o * M + row] = make_float2(v.x * d, v.y * d);
            }
        }
    }
}

// Persistent form of the two passes for M = 2^9 .. 2^13: each CTA stages the per-pass twiddle
// table of the M-point transform once and walks rows; the next row's loads are in flight while
// the current row is transformed (first pass from registers, radix-8 passes in shared memory,
// last pass from registers straight to the pruned outputs).  Output i of a row is position
// pos = i of the transform, i.e. image index (i + floor(N/2)) mod M when that is below N.
//   XPASS false: rows l_x of G in pairs (2p, 2p + 1); the first row's outputs wait in shared
//                memory and leave with the second's as 16-byte pairs,
//                inter[i_y][2p .. 2p + 1] = z * deap[i_y] (TST: the pairs are staged in shared
//                memory and written by 2D TMA stores of 256 rows, off the load/store path);
//   XPASS true:  rows i_y of inter, img[i_y][i_x] = Re z * deap[i_x].
// 128-byte aligned start (in float2) of the y pass's output staging after the work array and
// twiddles
template <int LOGM>
__host__ __device__ constexpr int ifft_pt_stage_off() {
    return ((1 << LOGM) + pt_offset<LOGM>(PtPlan<LOGM>::npass) + 15) & ~15;
}
template <int LOGM, bool XPASS, bool TST = false>
__host__ __device__ constexpr int ifft_pt_smem_elems() {
    // work array, per-pass twiddles (even count); y pass: the held first-row outputs (N <= M/2),
    // or with TMA stores a staging buffer of M/2 16-byte pairs
    return XPASS ? (1 << LOGM) + pt_offset<LOGM>(PtPlan<LOGM>::npass)
                 : ifft_pt_stage_off<LOGM>() + (TST ? (1 << LOGM) : (1 << LOGM) / 2);
}
// the TMA-store y pass: 256-row boxes tile M/2, and two CTAs of its shared memory fit an SM
template <int LOGM>
constexpr bool ifft_tst_ok() {
    return (1 << LOGM) >= 512 && sizeof(float2) * ifft_pt_smem_elems<LOGM, false, true>() <= 110u * 1024u;
}

template <int LOGM, bool XPASS, bool TST = false>
__global__ void __launch_bounds__((1 << LOGM) / kPassE, 1024 / ((1 << LOGM) / kPassE))
ifft_pt_kernel(const float2 *__restrict__ in, float2 *__restrict__ inter, float *__restrict__ img,
               const float *__restrict__ deap, const float2 *__restrict__ twp, int rows, int N,
               const __grid_constant__ CUtensorMap omap) {
    using PL = PtPlan<LOGM>;
    constexpr int M = 1 << LOGM, NT = M / kPassE, Rl = PL::Rl, Gl = kPassE / Rl;
    constexpr int TWN = pt_offset<LOGM>(PL::npass);
    static_assert(TWN % 2 == 0, "per-pass twiddle count");
    extern __shared__ __align__(128) float2 pz[];
    float2 *z = pz;                                 // [M] work array
    float2 *T = z + M;                              // [TWN] per-pass twiddles
    float2 *hold = pz + ifft_pt_stage_off<LOGM>();  // y pass: [M/2] first row's outputs, by image index;
                                                    // TST: [M/2] 16-byte output pairs
    const int t = threadIdx.x;
    const int h = N / 2;
    float2 nxt[kPassE];  // inputs of the first pass: x[t + r NT]
    auto fetch = [&](int row) {
        const float2 *src = in + (long long)row * M;
#pragma unroll
        for (int r = 0; r < kPassE; ++r) nxt[r] = __ldg(src + t + r * NT);
    };
    // the first row's loads are in flight while the twiddle table is staged
    int row = XPASS ? blockIdx.x : 2 * blockIdx.x;
    if (row < rows) fetch(row);
    {
        constexpr int n4t = TWN / 2;  // float4 loads; T starts 16-byte aligned (M even)
        const float4 *ts = reinterpret_cast<const float4 *>(twp);
        float4 *td = reinterpret_cast<float4 *>(T);
#pragma unroll
        for (int i = 0; i < (n4t + NT - 1) / NT; ++i)
            if (t + i * NT < n4t) td[t + i * NT] = __ldg(ts + t + i * NT);
    }
    if constexpr (XPASS) {
        for (; row < rows; row += gridDim.x) {
            float2 a[kPassE];
#pragma unroll
            for (int r = 0; r < kPassE; ++r) a[r] = nxt[r];
            if (row + (int)gridDim.x < rows) fetch(row + gridDim.x);
            float2 c[Gl][Rl];
            pt_row<LOGM, true>(a, z, T, t, c);
#pragma unroll
            for (int g = 0; g < Gl; ++g)
#pragma unroll
                for (int q = 0; q < Rl; ++q) {
                    const int i = t + (g + q * Gl) * NT;
                    const int o = i < N - h ? i + h : i - (M - h);  // image index, valid in [0, N)
                    if (o >= 0 && o < N) img[(long long)row * N + o] = c[g][q].x * __ldg(deap + o);
                }
        }
    } else if constexpr (TST) {
        // rows 2p, 2p + 1: each output pair (first row .xy, second .zw) is staged in shared
        // memory and the staged column pair leaves as 2D TMA stores of 256 rows
        // inter[o0 .. o0 + 255][2p .. 2p + 1] (the tensor map clips rows >= N); the staging
        // buffer is rewritten once the previous pair's stores have read it
        float4 *sb = reinterpret_cast<float4 *>(hold);
        for (; row < rows; row = (row & 1) ? row - 1 + 2 * (int)gridDim.x : row + 1) {
            float2 a[kPassE];
#pragma unroll
            for (int r = 0; r < kPassE; ++r) a[r] = nxt[r];
            const int nr = (row & 1) ? row - 1 + 2 * (int)gridDim.x : row + 1;
            if (nr < rows) fetch(nr);
            // the previous pair's stores have read the buffer (the barriers inside the transform
            // order this wait before every thread's staging writes)
            if (!(row & 1) && t == 0) bulk_wait_read<0>();
            float2 c[Gl][Rl];
            pt_row<LOGM, true>(a, z, T, t, c);
#pragma unroll
            for (int g = 0; g < Gl; ++g)
#pragma unroll
                for (int q = 0; q < Rl; ++q) {
                    const int i = t + (g + q * Gl) * NT;
                    const int o = i < N - h ? i + h : i - (M - h);
                    if (o >= 0 && o < N) {
                        const float d = __ldg(deap + o);
                        reinterpret_cast<float2 *>(sb + o)[row & 1] = make_float2(c[g][q].x * d, c[g][q].y * d);
                    }
                }
            if (row & 1) {
                fence_proxy_async_smem();  // this thread's staging writes, before the async-proxy reads
                __syncthreads();           // the pair is staged
                if (t == 0) {
                    for (int o0 = 0; o0 < N; o0 += 256) tma_store_2d(&omap, 2 * (row - 1), o0, smem_u32(sb + o0));
                    bulk_commit();
                }
            }
        }
        if (t == 0) bulk_wait_all();
    } else {
        // rows 2p, 2p + 1 (p = b, b + G, ...): the first row's outputs wait in shared memory
        // (read back by the same thread) and leave with the second's as 16-byte pairs
        for (; row < rows; row = (row & 1) ? row - 1 + 2 * (int)gridDim.x : row + 1) {
            float2 a[kPassE];
#pragma unroll
            for (int r = 0; r < kPassE; ++r) a[r] = nxt[r];
            const int nr = (row & 1) ? row - 1 + 2 * (int)gridDim.x : row + 1;
            if (nr < rows) fetch(nr);
            float2 c[Gl][Rl];
            pt_row<LOGM, true>(a, z, T, t, c);
#pragma unroll
            for (int g = 0; g < Gl; ++g)
#pragma unroll
                for (int q = 0; q < Rl; ++q) {
                    const int i = t + (g + q * Gl) * NT;
                    const int o = i < N - h ? i + h : i - (M - h);
                    if (o >= 0 && o < N) {
                        const float d = __ldg(deap + o);
                        const float2 v = make_float2(c[g][q].x * d, c[g][q].y * d);
                        if (!(row & 1)) {
                            hold[o] = v;
                        } else {
                            const float2 u = hold[o];
                            *reinterpret_cast<float4 *>(inter + (long long)o * M + row - 1) =
                                make_float4(u.x, u.y, v.x, v.y);
                        }
                    }
                }
        }
    }
}

// ---------------------------------------------------------------------------------- adjoint (R_F)
// R_F = (dx^2/dt) diag(1/w) A_F^T with A_F the Fourier-path R* above.  Transposing every
// linear step in reverse order: deapodise and embed the image, forward 2D FFT (pruned:
// N nonzero input rows and columns), Kaiser-Bessel interpolation at the polar samples
// (the transpose of spreading), conjugate sample factors, and per angle the Hermitian
// inverse P-point FFT whose first n_det outputs are the projection.

// Pass along x: image rows i_y (R per CTA) embedded at (i - floor(N/2)) mod M, times the
// deapodisation, forward FFT, written to T[i_y][l_x].
template <int E>
__global__ void __launch_bounds__(1024, 1)
adj_fft_x_kernel(const float *__restrict__ img, float2 *__restrict__ T, const float *__restrict__ deap,
                 const float2 *__restrict__ tw, int M, int logM, int N, int R) {
    extern __shared__ __align__(128) float2 z[];
    float2 *tws = z + R * M;  // M/2 twiddles
    stage_twiddles(tws, tw, M / 2);
    const int iy0 = blockIdx.x * R;
    const int rows = min(R, N - iy0);
    const int nthr = fft_threads(M), groups = blockDim.x / nthr;
    const int g = threadIdx.x / nthr, tid = threadIdx.x - g * nthr;
    const int h = N / 2;
    for (int i = threadIdx.x; i < R * M; i += blockDim.x) z[i] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int i = threadIdx.x; i < rows * N; i += blockDim.x) {
        const int r = i / N, ix = i - r * N;
        const float v = __ldg(img + (long long)(iy0 + r) * N + ix) * __ldg(deap + ix) * __ldg(deap + iy0 + r);
        z[r * M + ((ix - h) & (M - 1))] = make_float2(v, 0.f);
    }
    __syncthreads();
    for (int r0 = 0; r0 < R; r0 += groups) stockham_fft<E>(z + (r0 + g) * M, logM, tws, 1, false, tid, nthr);
    for (int i = threadIdx.x; i < rows * M; i += blockDim.x) T[(long long)iy0 * M + i] = z[i];
}

// Pass along y: columns l_x (R per CTA) of T, embedded at (i_y - floor(N/2)) mod M, forward
// FFT, written to G[l_x][l_y].
template <int E>
__global__ void __launch_bounds__(1024, 1)
adj_fft_y_kernel(const float2 *__restrict__ T, float2 *__restrict__ grid, const float2 *__restrict__ tw, int M,
                 int logM, int N, int R) {
    extern __shared__ __align__(128) float2 z[];
    float2 *tws = z + R * M;  // M/2 twiddles
    stage_twiddles(tws, tw, M / 2);
    const int lx0 = blockIdx.x * R;
    const int nthr = fft_threads(M), groups = blockDim.x / nthr;
    const int g = threadIdx.x / nthr, tid = threadIdx.x - g * nthr;
    const int h = N / 2;
    for (int i = threadIdx.x; i < R * M; i += blockDim.x) z[i] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int i = threadIdx.x; i < N * R; i += blockDim.x) {
        const int iy = i / R, r = i - iy * R;
        z[r * M + ((iy - h) & (M - 1))] = T[(long long)iy * M + lx0 + r];
    }
    __syncthreads();
    for (int r0 = 0; r0 < R; r0 += groups) stockham_fft<E>(z + (r0 + g) * M, logM, tws, 1, false, tid, nthr);
    for (int i = threadIdx.x; i < R * M; i += blockDim.x) grid[(long long)lx0 * M + i] = z[i];
}

// Persistent form of the two adjoint passes for M = 2^9 .. 2^13 (the transpose of
// ifft_pt_kernel; same row walk, table and pass structure, forward transforms).  Input
// position pos of a row holds image index (pos + floor(N/2)) mod M when that is below N, else
// zero (the padding is never loaded); all M outputs are written.
//   YPASS false: rows i_y of the image times deap[i_x] deap[i_y] -> T[i_y][l_x];
//   YPASS true:  columns l_x of T -> G[l_x][l_y].
template <int LOGM, bool YPASS>
__global__ void __launch_bounds__((1 << LOGM) / kPassE, 1024 / ((1 << LOGM) / kPassE))
fft_pt_fwd_kernel(const float *__restrict__ img, const float2 *__restrict__ Tin, float2 *__restrict__ out,
                  const float *__restrict__ deap, const float2 *__restrict__ twp, int rows, int N) {
    using PL = PtPlan<LOGM>;
    constexpr int M = 1 << LOGM, NT = M / kPassE, Rl = PL::Rl, Gl = kPassE / Rl;
    constexpr int TWN = pt_offset<LOGM>(PL::npass);
    static_assert(TWN % 2 == 0, "per-pass twiddle count");
    extern __shared__ __align__(128) float2 pz[];
    float2 *z = pz;      // [M] work array
    float2 *T = z + M;   // [TWN] per-pass twiddles
    const int t = threadIdx.x;
    const int h = N / 2;
    float2 nxt[kPassE];  // inputs of the first pass: x[t + r NT]
    auto fetch = [&](int row) {
        const float dy = YPASS ? 1.f : __ldg(deap + row);
#pragma unroll
        for (int r = 0; r < kPassE; ++r) {
            const int pos = t + r * NT;
            const int o = pos < N - h ? pos + h : pos - (M - h);  // image index, valid in [0, N)
            float2 v = make_float2(0.f, 0.f);
            if (o >= 0 && o < N) {
                if (YPASS) v = __ldg(Tin + (long long)o * M + row);
                else v.x = __ldg(img + (long long)row * N + o) * __ldg(deap + o) * dy;
            }
            nxt[r] = v;
        }
    };
    int row = blockIdx.x;
    if (row < rows) fetch(row);
    {
        constexpr int n4t = TWN / 2;
        const float4 *ts = reinterpret_cast<const float4 *>(twp);
        float4 *td = reinterpret_cast<float4 *>(T);
#pragma unroll
        for (int i = 0; i < (n4t + NT - 1) / NT; ++i)
            if (t + i * NT < n4t) td[t + i * NT] = __ldg(ts + t + i * NT);
    }
    for (; row < rows; row += gridDim.x) {
        float2 a[kPassE];
#pragma unroll
        for (int r = 0; r < kPassE; ++r) a[r] = nxt[r];
        if (row + gridDim.x < rows) fetch(row + gridDim.x);
        __syncthreads();  // previous row's last reads of z (and the staged table) are done
        dft_reg<8>(a, false);
#pragma unroll
        for (int q = 0; q < 8; ++q) z[fft_swz<kPassE>(t * 8 + q)] = a[q];
        __syncthreads();
        int L = 8;
#pragma unroll
        for (int p = 1; p < PL::n8; ++p) {
            if (p == PL::npass - 1) break;
            pt_pass<8, LOGM>(z, T + pt_offset<LOGM>(p), L, t, false);
            L *= 8;
        }
        constexpr int lp = PL::npass - 1, m = M / Rl;
        float2 c[Gl][Rl];
#pragma unroll
        for (int g = 0; g < Gl; ++g)
#pragma unroll
            for (int r = 0; r < Rl; ++r) c[g][r] = z[fft_swz<kPassE>(t + g * NT + r * m)];
        float2 *dst = out + (long long)row * M;
#pragma unroll
        for (int g = 0; g < Gl; ++g) {
            pt_twiddle_dft<Rl>(c[g], T + pt_offset<LOGM>(lp), L, t + g * NT, false);
#pragma unroll
            for (int q = 0; q < Rl; ++q) dst[t + (g + q * Gl) * NT] = c[g][q];
        }
    }
}

// The adjoint's column pass when N = M/2 (the usual power-of-two case): columns in pairs
// (2p, 2p + 1), read as 16-byte pairs T[i_y][2p .. 2p + 1].  Then only the first-pass inputs
// r = 0, 1, 6, 7 of a thread are inside the image (positions t + r NT below M/4 or from 3M/4
// on); the second column's values wait in shared memory (the thread's own slots) while the
// first column is transformed, and the next pair's loads are in flight during both.
template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) / kPassE, 1024 / ((1 << LOGM) / kPassE))
fft_pt_fwd_cols_kernel(const float2 *__restrict__ Tin, float2 *__restrict__ out, const float2 *__restrict__ twp,
                       int rows) {
    using PL = PtPlan<LOGM>;
    constexpr int M = 1 << LOGM, NT = M / kPassE, Rl = PL::Rl, Gl = kPassE / Rl;
    constexpr int TWN = pt_offset<LOGM>(PL::npass);
    constexpr int N = M / 2, h = N / 2;
    constexpr int RV[4] = {0, 1, kPassE - 2, kPassE - 1};  // the inputs inside the image
    static_assert(TWN % 2 == 0, "per-pass twiddle count");
    extern __shared__ __align__(128) float2 pz[];
    float2 *z = pz;          // [M] work array
    float2 *T = z + M;       // [TWN] per-pass twiddles
    float2 *hold = T + TWN;  // [4 NT] second column's inputs
    const int t = threadIdx.x;
    float4 nxt[4];
    auto fetch = [&](int pair) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int pos = t + RV[j] * NT;
            const int o = pos < N - h ? pos + h : pos - (M - h);
            nxt[j] = __ldg(reinterpret_cast<const float4 *>(Tin + (long long)o * M + 2 * pair));
        }
    };
    const int npairs = rows / 2;
    int pair = blockIdx.x;
    if (pair < npairs) fetch(pair);
    {
        constexpr int n4t = TWN / 2;
        const float4 *ts = reinterpret_cast<const float4 *>(twp);
        float4 *td = reinterpret_cast<float4 *>(T);
#pragma unroll
        for (int i = 0; i < (n4t + NT - 1) / NT; ++i)
            if (t + i * NT < n4t) td[t + i * NT] = __ldg(ts + t + i * NT);
    }
    for (; pair < npairs; pair += gridDim.x) {
        float2 a[kPassE];
#pragma unroll
        for (int r = 0; r < kPassE; ++r) a[r] = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            a[RV[j]] = make_float2(nxt[j].x, nxt[j].y);
            hold[j * NT + t] = make_float2(nxt[j].z, nxt[j].w);
        }
        if (pair + (int)gridDim.x < npairs) fetch(pair + gridDim.x);
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            if (half) {
#pragma unroll
                for (int r = 0; r < kPassE; ++r) a[r] = make_float2(0.f, 0.f);
#pragma unroll
                for (int j = 0; j < 4; ++j) a[RV[j]] = hold[j * NT + t];
            }
            float2 c[Gl][Rl];
            pt_row<LOGM, false>(a, z, T, t, c);
            float2 *dst = out + (long long)(2 * pair + half) * M;
#pragma unroll
            for (int g = 0; g < Gl; ++g)
#pragma unroll
                for (int q = 0; q < Rl; ++q) dst[t + (g + q * Gl) * NT] = c[g][q];
        }
    }
}

// The same column pass with the column pairs brought in by 2D TMA loads (boxes of one column
// pair x 256 rows of the intermediate, through its tensor map) into a shared staging buffer:
// the first column's inputs are read as .xy, the second's as .zw, and once the second's are in
// registers the next pair's loads are issued, in flight during the second transform.  Every
// wait is bounded: on expiry the kernel sets *err, waits (bounded) for its copy once more and
// returns.
template <int LOGM>
__global__ void __launch_bounds__((1 << LOGM) / kPassE, 1024 / ((1 << LOGM) / kPassE))
fft_pt_fwd_cols_tma_kernel(const __grid_constant__ CUtensorMap imap, float2 *__restrict__ out,
                           const float2 *__restrict__ twp, int rows, int *__restrict__ err) {
    using PL = PtPlan<LOGM>;
    constexpr int M = 1 << LOGM, NT = M / kPassE, Rl = PL::Rl, Gl = kPassE / Rl;
    constexpr int TWN = pt_offset<LOGM>(PL::npass);
    constexpr int N = M / 2, h = N / 2;
    constexpr int NBOX = (N + 255) / 256;
    constexpr int RV[4] = {0, 1, kPassE - 2, kPassE - 1};  // the inputs inside the image
    static_assert(TWN % 2 == 0, "per-pass twiddle count");
    extern __shared__ __align__(128) float2 pz[];
    __shared__ __align__(8) unsigned long long bar;
    float2 *z = pz;  // [M] work array
    float2 *T = z + M;  // [TWN] per-pass twiddles
    float4 *stg = reinterpret_cast<float4 *>(pz + ifft_pt_stage_off<LOGM>());  // [NBOX 256] staged pairs
    const int t = threadIdx.x;
    const uint32_t b = smem_u32(&bar);
    const int npairs = rows / 2;
    auto issue = [&](int pr) {  // thread 0: the column pair's boxes
        mbar_expect_tx(b, (uint32_t)(NBOX * 256 * sizeof(float4)));
        for (int k = 0; k < NBOX; ++k) tma_load_2d(smem_u32(stg + 256 * k), &imap, 4 * pr, 256 * k, b);
    };
    if (t == 0) {
        mbar_init(b, 1);
        mbar_fence_init();
    }
    __syncthreads();
    int pair = blockIdx.x;
    if (t == 0 && pair < npairs) issue(pair);
    {
        constexpr int n4t = TWN / 2;
        const float4 *ts = reinterpret_cast<const float4 *>(twp);
        float4 *td = reinterpret_cast<float4 *>(T);
#pragma unroll
        for (int i = 0; i < (n4t + NT - 1) / NT; ++i)
            if (t + i * NT < n4t) td[t + i * NT] = __ldg(ts + t + i * NT);
    }
    int o[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int pos = t + RV[j] * NT;
        o[j] = pos < N - h ? pos + h : pos - (M - h);
    }
    uint32_t parity = 0;
    for (; pair < npairs; pair += gridDim.x) {
        if (__syncthreads_or(!mbar_wait(b, parity))) {
            if (t == 0) atomicExch(err, 1);
            mbar_wait(b, parity);
            return;
        }
        parity ^= 1u;
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            float2 a[kPassE];
#pragma unroll
            for (int r = 0; r < kPassE; ++r) a[r] = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 v = stg[o[j]];
                a[RV[j]] = half ? make_float2(v.z, v.w) : make_float2(v.x, v.y);
            }
            if (half) {
                // every thread holds its inputs: the staging buffer takes the next pair
                fence_proxy_async_smem();
                __syncthreads();
                if (t == 0 && pair + (int)gridDim.x < npairs) issue(pair + gridDim.x);
            }
            float2 c[Gl][Rl];
            pt_row<LOGM, false>(a, z, T, t, c);
            float2 *dst = out + (long long)(2 * pair + half) * M;
#pragma unroll
            for (int g = 0; g < Gl; ++g)
#pragma unroll
                for (int q = 0; q < Rl; ++q) dst[t + (g + q * Gl) * NT] = c[g][q];
        }
    }
}

// Interpolation at the polar samples (the transpose of the spreading) by grid tiles
// (after ensure_adj_items): sample (k, m) belongs to the kAdjTile x kAdjTile tile holding its lowest cell
// floor(z) (the same 32.32 fixed-point floor as below); one CTA per work item (a run of ray
// segments of one tile, at most kAdjItemSamples samples) stages the tile and its kernel halo in
// shared memory with coalesced row loads, and its threads read the 2 HW x 2 HW neighbourhoods
// from there.  Per sample: the interpolation weights (the transpose of the spreading), then the
// conjugate sample factor (1/P)(m ? 2 : 1) exp(-i pi m (n_det-1)/P) exp(-2 pi i delta (z_x + z_y)/M)
// and dx^2/dt (or the quadrature weight).
constexpr int kAdjTile = 64;
constexpr int kAdjItemSamples = 2048;
constexpr int kAdjItemSegs = 256;

// Dynamic shared memory of adj_interp_tiled_kernel<HW>: segments, tile with halo, kernel
// table, sample -> segment index.
__host__ __device__ constexpr size_t adj_tiled_smem(int HW) {
    return sizeof(int4) * kAdjItemSegs + sizeof(float2) * ((size_t)(kAdjTile + 2 * HW - 1) * (kAdjTile + 2 * HW - 1)) +
           sizeof(float2) * (kKB + 1) + sizeof(unsigned short) * kAdjItemSamples;
}

template <int HW>
__global__ void __launch_bounds__(256)
adj_interp_tiled_kernel(const float2 *__restrict__ grid, float2 *__restrict__ spec, const long long *__restrict__ ray,
                        const int4 *__restrict__ items, const int4 *__restrict__ segs, int M, int H, int P, int n_det,
                        const float2 *__restrict__ tab, float delta2_over_M, float scale,
                        const float *__restrict__ wk) {
    constexpr int W = 2 * HW, S = kAdjTile + W - 1;
    extern __shared__ __align__(16) float2 adj_sm[];
    int4 *sseg = reinterpret_cast<int4 *>(adj_sm);            // [kAdjItemSegs]
    float2 *tile = adj_sm + 2 * kAdjItemSegs;                 // [S * S] cells x0.., y0.. (mod M)
    float2 *stab = tile + S * S;                              // [kKB + 1] the kernel table (scattered lookups)
    unsigned short *seg_of = reinterpret_cast<unsigned short *>(stab + kKB + 1);  // [kAdjItemSamples]
    const int4 it = __ldg(items + blockIdx.x);  // tile (tx nt + ty), first segment, segments, samples
    const int nt = M / kAdjTile;
    const int tx = it.x / nt, ty = it.x - tx * nt;
    const int Mmask = M - 1;
    const int x0 = tx * kAdjTile - (HW - 1), y0 = ty * kAdjTile - (HW - 1);
    for (int i = threadIdx.x; i < S * S; i += blockDim.x) {
        const int xi = i / S, yi = i - xi * S;
        tile[i] = __ldg(grid + (long long)((x0 + xi) & Mmask) * M + ((y0 + yi) & Mmask));
    }
    for (int i = threadIdx.x; i < it.z; i += blockDim.x) sseg[i] = __ldg(segs + it.y + i);
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int j = warp; j < it.z; j += nw) {
            const int4 sg = __ldg(segs + it.y + j);
            for (int i = lane; i < sg.z; i += 32) seg_of[sg.w + i] = (unsigned short)j;
        }
    }
    for (int i = threadIdx.x; i <= kKB; i += blockDim.x) stab[i] = __ldg(tab + i);
    __syncthreads();
    for (int sidx = threadIdx.x; sidx < it.w; sidx += blockDim.x) {
        const int4 sg = sseg[seg_of[sidx]];
        const int k = sg.x, m = sg.y + (sidx - sg.w);
        const long long zx = (long long)m * __ldg(ray + 2 * k), zy = (long long)m * __ldg(ray + 2 * k + 1);
        const int fx = (int)(zx >> 32), fy = (int)(zy >> 32);
        const float rx = (float)(unsigned)(zx & 0xffffffffLL) * 2.3283064365386963e-10f;
        const float ry = (float)(unsigned)(zy & 0xffffffffLL) * 2.3283064365386963e-10f;
        float wy[W];
#pragma unroll
        for (int t = 0; t < W; ++t) wy[t] = kb_tab_s<HW>(stab, (float)(t - (HW - 1)) - ry);
        // tile-local row and column of the window's first cell, in [0, kAdjTile)
        const int lxl = (fx & Mmask) - tx * kAdjTile, lyl = (fy & Mmask) - ty * kAdjTile;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int t = 0; t < W; ++t) {
            const float wx = kb_tab_s<HW>(stab, (float)(t - (HW - 1)) - rx);
            const float2 *row = tile + (lxl + t) * S + lyl;
            float2 r = make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < W; ++u) {
                const float2 v = row[u];
                r.x = fmaf(wy[u], v.x, r.x);
                r.y = fmaf(wy[u], v.y, r.y);
            }
            acc.x = fmaf(wx, r.x, acc.x);
            acc.y = fmaf(wx, r.y, acc.y);
        }
        float sn, cs;
        sincospif(-((float)(fx + fy) + (rx + ry)) * delta2_over_M, &sn, &cs);
        acc = cmul(acc, make_float2(cs, sn));
        const long long ph = ((long long)m * (n_det - 1)) % (2LL * P);
        sincospif(-(float)ph / (float)P, &sn, &cs);
        acc = cmul(acc, make_float2(cs, sn));
        const float f = (m == 0 ? 1.f : 2.f) * (wk ? __ldg(wk + k) : scale) / (float)P;
        spec[(long long)k * H + m] = make_float2(f * acc.x, f * acc.y);
    }
}


// Per projection pair: y_j = Re sum_{m < P/2} s_m exp(2 pi i m j / P) = (1/2) IFFT(Hermitian(s))_j;
// two real outputs share one complex transform (Z = H_a + i H_b).
template <int E>
__global__ void __launch_bounds__(1024, 1)
adj_rows_kernel(const float2 *__restrict__ spec, float *__restrict__ sino, const float2 *__restrict__ tw,
                int n_theta, int n_det, int logP) {
    extern __shared__ __align__(128) float2 z[];
    const int P = 1 << logP, H = P >> 1;
    float2 *tws = z + P;  // P/2 twiddles
    stage_twiddles(tws, tw, H);
    const int k0 = 2 * blockIdx.x, k1 = k0 + 1;
    const bool has1 = k1 < n_theta;
    const float2 *sa = spec + (long long)k0 * H, *sb = spec + (long long)k1 * H;
    for (int m = threadIdx.x; m < P; m += blockDim.x) {
        float2 ha, hb;  // Hermitian completions
        if (m == 0) {
            ha = make_float2(2.f * sa[0].x, 0.f);
            hb = make_float2(has1 ? 2.f * sb[0].x : 0.f, 0.f);
        } else if (m < H) {
            ha = sa[m];
            hb = has1 ? sb[m] : make_float2(0.f, 0.f);
        } else if (m == H) {
            ha = hb = make_float2(0.f, 0.f);
        } else {
            const float2 a = sa[P - m];
            const float2 b = has1 ? sb[P - m] : make_float2(0.f, 0.f);
            ha = make_float2(a.x, -a.y);
            hb = make_float2(b.x, -b.y);
        }
        z[m] = make_float2(ha.x - hb.y, ha.y + hb.x);  // H_a + i H_b
    }
    __syncthreads();
    stockham_fft<E>(z, logP, tws, 1, true, threadIdx.x, blockDim.x);
    for (int j = threadIdx.x; j < n_det; j += blockDim.x) {
        sino[(long long)k0 * n_det + j] = 0.5f * z[j].x;
        if (has1) sino[(long long)k1 * n_det + j] = 0.5f * z[j].y;
    }
}

// Persistent form of adj_rows_kernel for P = 2^9 .. 2^12: the Hermitian completions of the
// pair's half spectra are built while loading the first-pass inputs, the last pass writes
// the first n_det outputs straight to the sinogram.
template <int LOGP>
__global__ void __launch_bounds__((1 << LOGP) / kPassE, 1024 / ((1 << LOGP) / kPassE))
adj_rows_pt_kernel(const float2 *__restrict__ spec, float *__restrict__ sino, const float2 *__restrict__ twp,
                   int n_theta, int n_det) {
    using PL = PtPlan<LOGP>;
    constexpr int P = 1 << LOGP, H = P / 2, NT = P / kPassE;
    constexpr int TWN = pt_offset<LOGP>(PL::npass);
    constexpr int Rl = PL::Rl, Gl = kPassE / Rl;
    extern __shared__ __align__(16) float2 ar_sm[];
    float2 *z = ar_sm;     // [P]
    float2 *T = z + P;     // [TWN]
    const int t = threadIdx.x;
    const int npairs = (n_theta + 1) / 2;
    float2 nxt[kPassE];
    auto fetch = [&](int pair) {
        const int k0 = 2 * pair;
        const bool has1 = k0 + 1 < n_theta;
        const float2 *sa = spec + (long long)k0 * H, *sb = sa + H;
#pragma unroll
        for (int r = 0; r < kPassE; ++r) {
            const int j = t + r * NT;
            float2 ha, hb;  // Hermitian completions
            if (j == 0) {
                ha = make_float2(2.f * __ldg(&sa[0].x), 0.f);
                hb = make_float2(has1 ? 2.f * __ldg(&sb[0].x) : 0.f, 0.f);
            } else if (j < H) {
                ha = __ldg(sa + j);
                hb = has1 ? __ldg(sb + j) : make_float2(0.f, 0.f);
            } else if (j == H) {
                ha = hb = make_float2(0.f, 0.f);
            } else {
                const float2 va = __ldg(sa + P - j);
                const float2 vb = has1 ? __ldg(sb + P - j) : make_float2(0.f, 0.f);
                ha = make_float2(va.x, -va.y);
                hb = make_float2(vb.x, -vb.y);
            }
            nxt[r] = make_float2(ha.x - hb.y, ha.y + hb.x);  // H_a + i H_b
        }
    };
    int pair = blockIdx.x;
    if (pair < npairs) fetch(pair);
    {
        constexpr int n4t = TWN / 2;
        const float4 *ts = reinterpret_cast<const float4 *>(twp);
        float4 *td = reinterpret_cast<float4 *>(T);
#pragma unroll
        for (int i = 0; i < (n4t + NT - 1) / NT; ++i)
            if (t + i * NT < n4t) td[t + i * NT] = __ldg(ts + t + i * NT);
    }
    for (; pair < npairs; pair += gridDim.x) {
        const int k0 = 2 * pair;
        const bool has1 = k0 + 1 < n_theta;
        float2 a[kPassE];
#pragma unroll
        for (int r = 0; r < kPassE; ++r) a[r] = nxt[r];
        if (pair + (int)gridDim.x < npairs) fetch(pair + gridDim.x);
        float2 c[Gl][Rl];
        pt_row<LOGP, true>(a, z, T, t, c);
        float *oa = sino + (long long)k0 * n_det, *ob = oa + n_det;
#pragma unroll
        for (int g = 0; g < Gl; ++g)
#pragma unroll
            for (int q = 0; q < Rl; ++q) {
                const int j = t + (g + q * Gl) * NT;
                if (j < n_det) {
                    oa[j] = 0.5f * c[g][q].x;
                    if (has1) ob[j] = 0.5f * c[g][q].y;
                }
            }
    }
}

double kb_hat(double f, double beta, int width) {
    // Fourier transform of I0(beta sqrt(1 - (2t/W)^2)) on |t| <= W/2 at frequency f (cycles per cell)
    const double kW = width;
    const double x = M_PI * kW * f;
    const double a2 = beta * beta - x * x;
    if (a2 > 0) {
        const double a = std::sqrt(a2);
        return a < 1e-8 ? kW : kW * std::sinh(a) / a;
    }
    const double a = std::sqrt(-a2);
    return a < 1e-8 ? kW : kW * std::sin(a) / a;
}

}  // namespace

void free_fourier(bp_plan *p) {
    FourierWork &f = p->four;
    cudaFree(f.spec);
    cudaFree(f.grid);
    cudaFree(f.mid);
    cudaFree(f.deapod);
    cudaFree(f.wk);
    cudaFree(f.twM);
    cudaFree(f.twpassM);
    cudaFree(f.twpassH);
    cudaFree(f.ray);
    cudaFree(f.sray);
    cudaFree(f.sphi);
    cudaFree(f.kbtab);
    cudaFree(f.adj_items);
    cudaFree(f.adj_segs);
    f = FourierWork();
}

// Host (FP64) tables of the Fourier path: per-angle ray steps in 32.32 fixed point (original
// order, for the spectra and the adjoint) and sorted by ray angle (for the gather), the
// Kaiser-Bessel table and the deapodisation.
bp_status ensure_fourier(bp_plan *p) {
    FourierWork &f = p->four;
    if (f.grid) return BP_OK;
    const int N = p->N, n_theta = p->n_theta, P = p->P, H = P / 2;
    int M = 1;
    while (M < 2 * N) M <<= 1;
    M = std::max(M, 64);  // the core square (side 2 min(kCore, M/2) - 1) and a 64-cell tile fit
    if ((size_t)M * sizeof(float2) > 128u * 1024u)
        return fail(BP_ERR_UNSUPPORTED, "Fourier path: N too large for the shared-memory FFT (N <= 8192)");
    if ((size_t)P * sizeof(float2) > 200u * 1024u)
        return fail(BP_ERR_UNSUPPORTED, "Fourier path: n_det too large for the shared-memory FFT (n_det <= 8192)");
    const int kW = p->fourier_W;  // kernel width, 6 or 4
    const double sigma = (double)M / N;
    double b2 = (kW / sigma) * (kW / sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8;
    const double beta = M_PI * std::sqrt(std::max(b2, 1.0));
    const double rho = (double)M * p->dx / ((double)P * p->dt);

    std::vector<long long> ray(2 * (size_t)n_theta);
    std::vector<std::pair<double, int>> order(n_theta);
    for (int k = 0; k < n_theta; ++k) {
        const double c = std::cos(p->theta[k]), sn = std::sin(p->theta[k]);
        ray[2 * k] = (long long)std::llround(std::ldexp(rho * c, 32));
        ray[2 * k + 1] = (long long)std::llround(std::ldexp(rho * sn, 32));
        double phi = std::atan2(sn, c);
        if (phi < 0) phi += 2.0 * M_PI;
        if (phi >= 2.0 * M_PI) phi = 0.0;
        order[k] = {phi, k};
    }
    std::sort(order.begin(), order.end());
    std::vector<SortedRay> sray(n_theta);
    std::vector<float> sphi(n_theta);
    for (int i = 0; i < n_theta; ++i) {
        const int k = order[i].second;
        sray[i].ax = ray[2 * k];
        sray[i].ay = ray[2 * k + 1];
        const double sxd = std::ldexp((double)ray[2 * k], -32), syd = std::ldexp((double)ray[2 * k + 1], -32);
        sray[i].isx = sxd != 0.0 ? (float)(1.0 / sxd) : INFINITY;
        sray[i].isy = syd != 0.0 ? (float)(1.0 / syd) : INFINITY;
        sray[i].sx = (float)sxd;
        sray[i].sy = (float)syd;
        sray[i].k = k;
        sray[i].pad = 0;
        // the float angle must stay sorted and in [0, 2 pi) after rounding
        sphi[i] = std::min((float)order[i].first, std::nextafter((float)(2.0 * M_PI), 0.f));
        if (i > 0 && sphi[i] < sphi[i - 1]) sphi[i] = sphi[i - 1];
    }
    // uniform spacing of the sorted angles gives an O(1) index lookup
    f.ri.n = n_theta;
    f.ri.upper = 1;
    for (int k = 0; k < n_theta; ++k)
        if (ray[2 * k + 1] < 0) f.ri.upper = 0;
    f.ri.uniform = 0;
    if (n_theta > 1) {
        const double d = (order[n_theta - 1].first - order[0].first) / (n_theta - 1);
        bool uni = d > 0;
        for (int i = 0; i < n_theta && uni; ++i)
            uni = std::fabs(order[i].first - (order[0].first + i * d)) < 1e-9;
        if (uni) {
            f.ri.uniform = 1;
            f.ri.phi0 = (float)order[0].first;
            f.ri.dphi = (float)d;
        }
    }
    // kernel table: (phi(i h), phi((i+1) h) - phi(i h)), h = (W/2) / kKB
    std::vector<float2> tab(kKB + 1);
    auto phi = [&](double d) {
        const double a = 2.0 * d / kW;
        return std::cyl_bessel_i(0.0, beta * std::sqrt(std::max(0.0, 1.0 - a * a)));
    };
    for (int i = 0; i <= kKB; ++i) {
        const double d0 = 0.5 * kW * i / kKB, d1 = 0.5 * kW * (i + 1) / kKB;
        const double v0 = phi(d0), v1 = i < kKB ? phi(d1) : v0;
        tab[i] = make_float2((float)v0, (float)(v1 - v0));
    }
    // deapodisation 1 / phi_hat(i - floor(N/2)) (separable), weights, twiddles
    std::vector<float> deap(N), wk(n_theta);
    for (int i = 0; i < N; ++i) deap[i] = (float)(1.0 / kb_hat((double)(i - N / 2) / M, beta, kW));
    for (int k = 0; k < n_theta; ++k) wk[k] = (float)p->w[k];
    std::vector<float2> tw(M / 2);
    for (int i = 0; i < M / 2; ++i) {
        const double an = -2.0 * M_PI * (double)i / (double)M;
        tw[i] = make_float2((float)std::cos(an), (float)std::sin(an));
    }

    std::vector<float2> twp, twh;
    build_pass_twiddles(ilog2(M), twp);
    twp.resize((twp.size() + 1) & ~(size_t)1);  // a whole number of float4 loads
    if (M == 16384) {  // the split M-point transforms (two M/2-point ones)
        build_pass_twiddles(ilog2(M) - 1, twh);
        twh.resize((twh.size() + 1) & ~(size_t)1);
    }

    f.M = M;
    f.W = kW;
    f.logM = ilog2(M);
    f.beta = (float)beta;
    f.rho = (float)rho;
    f.rmax = (float)(rho * (H - 1)) + 1.0f;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess) f.bytes += bytes;
    };
    alloc((void **)&f.spec, sizeof(float2) * (size_t)n_theta * H);
    alloc((void **)&f.grid, sizeof(float2) * (size_t)M * M);
    alloc((void **)&f.mid, sizeof(float2) * (size_t)N * M);
    alloc((void **)&f.deapod, sizeof(float) * N);
    alloc((void **)&f.wk, sizeof(float) * n_theta);
    alloc((void **)&f.twM, sizeof(float2) * tw.size());
    alloc((void **)&f.twpassM, sizeof(float2) * twp.size());
    if (!twh.empty()) alloc((void **)&f.twpassH, sizeof(float2) * twh.size());
    alloc((void **)&f.ray, sizeof(long long) * ray.size());
    alloc(&f.sray, sizeof(SortedRay) * sray.size());
    alloc((void **)&f.sphi, sizeof(float) * sphi.size());
    alloc((void **)&f.kbtab, sizeof(float2) * tab.size());
    if (e == cudaSuccess) e = cudaMemcpy(f.deapod, deap.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f.wk, wk.data(), sizeof(float) * n_theta, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f.twM, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(f.twpassM, twp.data(), sizeof(float2) * twp.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !twh.empty())
        e = cudaMemcpy(f.twpassH, twh.data(), sizeof(float2) * twh.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f.ray, ray.data(), sizeof(long long) * ray.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(f.sray, sray.data(), sizeof(SortedRay) * sray.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f.sphi, sphi.data(), sizeof(float) * sphi.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f.kbtab, tab.data(), sizeof(float2) * tab.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_fourier(p);
        return cuda_fail(e, "Fourier workspace");
    }
    // mid as FP32 [N][2M] for the y pass's TMA stores: boxes of 4 floats (one column pair) x
    // 256 rows
    f.mid_map_ok = false;
    if (PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder()) {
        const cuuint64_t gdim[2] = {(cuuint64_t)2 * M, (cuuint64_t)N};
        const cuuint64_t gstride[1] = {(cuuint64_t)M * sizeof(float2)};
        const cuuint32_t box[2] = {4, 256};
        const cuuint32_t estr[2] = {1, 1};
        f.mid_map_ok = enc(&f.mid_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, f.mid, gdim, gstride, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    return BP_OK;
}

template <typename Tin, int LOGP>
static bp_status spectra_pt(bp_plan *p, const Tin *sino, cudaStream_t st, float wuni, float delta2, const float *Hf) {
    constexpr int NT = (1 << LOGP) / kPassE;
    constexpr size_t smem = sizeof(float2) * ((1 << LOGP) + pt_offset<LOGP>(PtPlan<LOGP>::npass));
    auto kern = fourier_spectra_pt_kernel<Tin, LOGP>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    const int npairs = (p->n_theta + 1) / 2;
    const int ctas = std::min(npairs, std::max(1, per_sm) * std::max(1, p->sm_count));
    kern<<<ctas, NT, smem, st>>>(sino, p->four.spec, p->four.wk, p->d_twpass, p->n_theta, p->n_det, wuni,
                                 p->four.ray, delta2, Hf);
    stage_mark(p, st, "fourier_spectra_pt_kernel");
    return BP_OK;
}

template <typename Tin>
static bp_status spectra_t(bp_plan *p, const Tin *sino, cudaStream_t st, float wuni, float delta2, const float *Hf) {
    const int logP = ilog2(p->P);
    if (p->d_twpass) {
        switch (logP) {
            case 9: return spectra_pt<Tin, 9>(p, sino, st, wuni, delta2, Hf);
            case 10: return spectra_pt<Tin, 10>(p, sino, st, wuni, delta2, Hf);
            case 11: return spectra_pt<Tin, 11>(p, sino, st, wuni, delta2, Hf);
            case 12: return spectra_pt<Tin, 12>(p, sino, st, wuni, delta2, Hf);
            default: break;
        }
    }
    const FourierWork &f = p->four;
    if (!Hf && p->P == 16384 && f.M == 16384 && f.twpassH) {  // the split transforms (twiddles of M = P)
        constexpr size_t smem = lp_rows_pt_smem<13>();
        auto kern = fourier_spectra_split_kernel<Tin>;
        BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int ctas = std::min((p->n_theta + 1) / 2, std::max(1, p->sm_count));
        kern<<<ctas, 1024, smem, st>>>(sino, f.spec, f.wk, f.twpassH, f.twM, p->n_theta, p->n_det, wuni, f.ray, delta2);
        stage_mark(p, st, "fourier_spectra_kernel");
        return BP_OK;
    }
    const size_t smem = sizeof(float2) * (p->P + p->P / 2);
    const int threads = fft_threads(p->P);
    auto kern = fft_elems(p->P) == 16 ? fourier_spectra_kernel<Tin, 16> : fourier_spectra_kernel<Tin, 8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(p->n_theta + 1) / 2, threads, smem, st>>>(sino, p->four.spec, p->four.wk, p->d_twP, p->n_theta, p->n_det,
                                                      logP, wuni, p->four.ray, delta2, Hf);
    stage_mark(p, st, "fourier_spectra_kernel");
    return BP_OK;
}

// Row passes of the 2D transforms: two rows per CTA transformed one after the other by
// fft_threads(M) threads, so that two CTAs (2 x 32 KB rows + twiddles, 2 x 512 threads at 64
// registers for M = 4096) share an SM and one's loads overlap the other's transforms.
static int rows_per_cta(int M) { return M <= 8192 ? 2 : 1; }

// Inverse 2D FFT of the M x M grid (f.grid), pruned to the N x N image, times deap[i_x]
// deap[i_y] (the deapodisation; ones for no correction), real part into img.
static bp_status launch_grid_to_image_rows(bp_plan *p, const float *deap, float *img, cudaStream_t st) {
    FourierWork &f = p->four;
    const int N = p->N, M = f.M;
    if (M == 16384 && f.twpassH) {
        constexpr size_t smem = lp_rows_pt_smem<13>();
        auto ky = ifft_split_kernel<false>;
        auto kx = ifft_split_kernel<true>;
        BP_CUDA_TRY(cudaFuncSetAttribute(ky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        BP_CUDA_TRY(cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        const int sms = std::max(1, p->sm_count);
        ky<<<std::min(sms, M), 1024, smem, st>>>(f.grid, f.mid, nullptr, deap, f.twpassH, f.twM, M, N);
        stage_mark(p, st, "ifft_pass_y_kernel");
        kx<<<std::min(sms, N), 1024, smem, st>>>(f.mid, nullptr, img, deap, f.twpassH, f.twM, N, N);
        stage_mark(p, st, "ifft_pass_x_kernel");
        BP_CUDA_TRY(cudaGetLastError());
        return BP_OK;
    }
    const int R = rows_per_cta(M);
    const size_t smemR = sizeof(float2) * ((size_t)R * M + M / 2);
    auto pass_y = fft_elems(M) == 16 ? ifft_pass_y_kernel<16> : ifft_pass_y_kernel<8>;
    auto pass_x = fft_elems(M) == 16 ? ifft_pass_x_kernel<16> : ifft_pass_x_kernel<8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(pass_y, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemR));
    BP_CUDA_TRY(cudaFuncSetAttribute(pass_x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemR));
    const int nthr = fft_threads(M);
    const int groups = 1;
    pass_y<<<M / R, nthr * groups, smemR, st>>>(f.grid, f.mid, deap, f.twM, M, f.logM, N, R, p->d_err);
    stage_mark(p, st, "ifft_pass_y_kernel");
    pass_x<<<(N + R - 1) / R, nthr * groups, smemR, st>>>(f.mid, img, deap, f.twM, M, f.logM, N, R, p->d_err);
    stage_mark(p, st, "ifft_pass_x_kernel");
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

// The persistent passes for one M: grid of (CTAs per SM) x SMs, capped by the rows.
template <int LOGM>
static bp_status launch_ifft_pt(bp_plan *p, const float *deap, float *img, cudaStream_t st) {
    FourierWork &f = p->four;
    constexpr int M = 1 << LOGM, NT = M / kPassE;
    constexpr bool TST = ifft_tst_ok<LOGM>();
    const bool tst = TST && f.mid_map_ok;
    const size_t smem_y =
        sizeof(float2) * (tst ? ifft_pt_smem_elems<LOGM, false, true>() : ifft_pt_smem_elems<LOGM, false>());
    constexpr size_t smem_x = sizeof(float2) * ifft_pt_smem_elems<LOGM, true>();
    auto ky = tst ? ifft_pt_kernel<LOGM, false, TST> : ifft_pt_kernel<LOGM, false>;
    auto kx = ifft_pt_kernel<LOGM, true>;
    BP_CUDA_TRY(cudaFuncSetAttribute(ky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_y));
    BP_CUDA_TRY(cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_x));
    int per_sm_y = 0, per_sm_x = 0;
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_y, ky, NT, smem_y));
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_x, kx, NT, smem_x));
    const int sms = std::max(1, p->sm_count);
    // the y pass takes rows in pairs (M is even)
    ky<<<std::min(std::max(1, per_sm_y) * sms, M / 2), NT, smem_y, st>>>(f.grid, f.mid, nullptr, deap, f.twpassM, M,
                                                                        p->N, f.mid_map);
    stage_mark(p, st, "ifft_pt_kernel (y pass)");
    kx<<<std::min(std::max(1, per_sm_x) * sms, p->N), NT, smem_x, st>>>(f.mid, nullptr, img, deap, f.twpassM, p->N,
                                                                       p->N, f.mid_map);
    stage_mark(p, st, "ifft_pt_kernel (x pass)");
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

bp_status launch_grid_to_image(bp_plan *p, const float *deap, float *img, cudaStream_t st) {
    switch (p->four.logM) {
        case 9: return launch_ifft_pt<9>(p, deap, img, st);
        case 10: return launch_ifft_pt<10>(p, deap, img, st);
        case 11: return launch_ifft_pt<11>(p, deap, img, st);
        case 12: return launch_ifft_pt<12>(p, deap, img, st);
        case 13: return launch_ifft_pt<13>(p, deap, img, st);
        default: return launch_grid_to_image_rows(p, deap, img, st);
    }
}

// The core square in ring order: cells inside ring kCoreInner (crossed by nearly every ray) take
// eight warps each, the others one.
constexpr int kCoreInner = 16;
template <int HW>
static void launch_core(FourierWork &f, const SortedRay *sr, int M, int H, int amax, int core, cudaStream_t st) {
    const int n = (2 * core - 1) * (2 * core - 1);
    const int ri = std::min(kCoreInner, core);
    const int n_in = (2 * ri - 1) * (2 * ri - 1);
    grid_gather_core_kernel<HW, 8><<<n_in, 256, 0, st>>>(f.spec, sr, f.sphi, f.kbtab, f.grid, M, H, f.ri, f.rmax,
                                                         amax, 0, n_in);
    if (n > n_in)
        grid_gather_core_kernel<HW, 1><<<(n - n_in + 7) / 8, 256, 0, st>>>(f.spec, sr, f.sphi, f.kbtab, f.grid, M, H,
                                                                           f.ri, f.rmax, amax, n_in, n);
}

bp_status launch_fourier(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, cudaStream_t st,
                         float wuni, int filter_kind, float filter_param) {
    bp_status s = ensure_fourier(p);
    if (s != BP_OK) return s;
    const float *Hf = nullptr;
    if (filter_kind >= 0) {
        if ((s = ensure_filter(p, filter_kind, filter_param)) != BP_OK) return s;
        Hf = p->d_H[filter_kind];
    }
    FourierWork &f = p->four;
    const int N = p->N, M = f.M, H = p->P / 2;
    const size_t esz = dt == BP_F32 ? 4 : 2;
    stage_begin(p, st);
    const float delta2 = (N % 2 == 0) ? 1.0f / (float)M : 0.0f;  // 2 delta / M
    for (int b = 0; b < batch; ++b) {
        const char *sb = (const char *)sino + esz * (size_t)b * p->n_theta * p->n_det;
        switch (dt) {
            case BP_F32: s = spectra_t(p, (const float *)sb, st, wuni, delta2, Hf); break;
            case BP_BF16: s = spectra_t(p, (const __nv_bfloat16 *)sb, st, wuni, delta2, Hf); break;
            case BP_F16: s = spectra_t(p, (const __half *)sb, st, wuni, delta2, Hf); break;
        }
        if (s != BP_OK) return s;
        const dim3 g((M + 63) / 64, (M + 7) / 8);
        const int amax = (int)std::ceil((f.rmax + 4.25 + M / 2) / M);
        const int core = std::min(kCore, M / 2);
        const SortedRay *sr = (const SortedRay *)f.sray;
        if (f.W == 4) {
            grid_gather_pair_kernel<2><<<g, 256, 0, st>>>(f.spec, sr, f.sphi, f.kbtab, f.grid, M, H, f.ri, f.rmax,
                                                          amax, core);
            stage_mark(p, st, "grid_gather_pair_kernel");
            launch_core<2>(f, sr, M, H, amax, core, st);
            stage_mark(p, st, "grid_gather_core_kernel");
        } else {
            grid_gather_pair_kernel<3><<<g, 256, 0, st>>>(f.spec, sr, f.sphi, f.kbtab, f.grid, M, H, f.ri, f.rmax,
                                                          amax, core);
            stage_mark(p, st, "grid_gather_pair_kernel");
            launch_core<3>(f, sr, M, H, amax, core, st);
            stage_mark(p, st, "grid_gather_core_kernel");
        }
        BP_CUDA_TRY(cudaGetLastError());
        if ((s = launch_grid_to_image(p, f.deapod, img + (size_t)b * N * N, st)) != BP_OK) return s;
    }
    return BP_OK;
}

// Work items of adj_interp_tiled_kernel (once per plan, after ensure_fourier): every sample
// (k, m), m < H, binned by the tile of floor(z) with the device's fixed-point products, runs
// of consecutive m on one ray in one tile as segments, a tile's segments cut into items of at
// most kAdjItemSamples samples and kAdjItemSegs segments.
static bp_status ensure_adj_items(bp_plan *p) {
    FourierWork &f = p->four;
    if (f.adj_items) return BP_OK;
    const int M = f.M, H = p->P / 2, n = p->n_theta;
    static_assert(64 % kAdjTile == 0, "the grid side (a power of two >= 64) is a whole number of tiles");
    const int nt = M / kAdjTile;
    std::vector<long long> ray(2 * (size_t)n);
    BP_CUDA_TRY(cudaMemcpy(ray.data(), f.ray, sizeof(long long) * ray.size(), cudaMemcpyDeviceToHost));
    std::vector<std::vector<int4>> per_tile((size_t)nt * nt);  // (k, m0, count, -)
    for (int k = 0; k < n; ++k) {
        int cur = -1, m0 = 0;
        for (int m = 0; m <= H; ++m) {
            int tile = -1;
            if (m < H) {
                const long long zx = (long long)m * ray[2 * k], zy = (long long)m * ray[2 * k + 1];
                const int fx = (int)(zx >> 32) & (M - 1), fy = (int)(zy >> 32) & (M - 1);
                tile = (fx / kAdjTile) * nt + fy / kAdjTile;
            }
            if (tile != cur) {
                if (cur >= 0) per_tile[cur].push_back(make_int4(k, m0, m - m0, 0));
                cur = tile;
                m0 = m;
            }
        }
    }
    std::vector<int4> items, segs;
    for (int t = 0; t < nt * nt; ++t) {
        int4 item = make_int4(t, (int)segs.size(), 0, 0);
        auto close = [&]() {
            if (item.z > 0) items.push_back(item);
            item = make_int4(t, (int)segs.size(), 0, 0);
        };
        for (int4 sg : per_tile[t]) {
            while (sg.z > 0) {
                if (item.z == kAdjItemSegs || item.w == kAdjItemSamples) close();
                const int take = std::min(sg.z, kAdjItemSamples - item.w);
                segs.push_back(make_int4(sg.x, sg.y, take, item.w));
                item.z += 1;
                item.w += take;
                sg.y += take;
                sg.z -= take;
            }
        }
        close();
    }
    cudaError_t e = cudaMalloc(&f.adj_items, sizeof(int4) * std::max<size_t>(items.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&f.adj_segs, sizeof(int4) * std::max<size_t>(segs.size(), 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(f.adj_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f.adj_segs, segs.data(), sizeof(int4) * segs.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(f.adj_items);
        cudaFree(f.adj_segs);
        f.adj_items = f.adj_segs = nullptr;
        return cuda_fail(e, "adjoint interpolation work items");
    }
    f.adj_n_items = (int)items.size();
    f.bytes += sizeof(int4) * (items.size() + segs.size());
    return BP_OK;
}

// The persistent adjoint passes for one M (grid as in launch_ifft_pt).
template <int LOGM>
static bp_status launch_fft_pt_fwd(bp_plan *p, const float *img, cudaStream_t st) {
    FourierWork &f = p->four;
    constexpr int M = 1 << LOGM, NT = M / kPassE;
    constexpr size_t smem = sizeof(float2) * (M + pt_offset<LOGM>(PtPlan<LOGM>::npass));
    auto kx = fft_pt_fwd_kernel<LOGM, false>;
    auto ky = fft_pt_fwd_kernel<LOGM, true>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    BP_CUDA_TRY(cudaFuncSetAttribute(ky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kx, NT, smem));
    const int ctas = std::max(1, per_sm) * std::max(1, p->sm_count);
    kx<<<std::min(ctas, p->N), NT, smem, st>>>(img, nullptr, f.mid, f.deapod, f.twpassM, p->N, p->N);
    stage_mark(p, st, "fft_pt_fwd_kernel (x pass)");
    if (2 * p->N == M && f.mid_map_ok && ifft_tst_ok<LOGM>()) {
        // columns in pairs through 2D TMA loads
        constexpr size_t smem2 = sizeof(float2) * (ifft_pt_stage_off<LOGM>() + M);
        auto kc = fft_pt_fwd_cols_tma_kernel<LOGM>;
        BP_CUDA_TRY(cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
        int per_sm2 = 0;
        BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, kc, NT, smem2));
        kc<<<std::min(std::max(1, per_sm2) * std::max(1, p->sm_count), M / 2), NT, smem2, st>>>(
            f.mid_map, f.grid, f.twpassM, M, p->d_err);
        stage_mark(p, st, "fft_pt_fwd_cols_kernel");
    } else if (2 * p->N == M) {
        // columns in pairs, 16-byte loads
        constexpr size_t smem2 = smem + sizeof(float2) * (M / 2);
        auto kc = fft_pt_fwd_cols_kernel<LOGM>;
        BP_CUDA_TRY(cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
        int per_sm2 = 0;
        BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, kc, NT, smem2));
        kc<<<std::min(std::max(1, per_sm2) * std::max(1, p->sm_count), M / 2), NT, smem2, st>>>(f.mid, f.grid,
                                                                                               f.twpassM, M);
        stage_mark(p, st, "fft_pt_fwd_cols_kernel");
    } else {
        ky<<<std::min(ctas, M), NT, smem, st>>>(nullptr, f.mid, f.grid, f.deapod, f.twpassM, M, p->N);
        stage_mark(p, st, "fft_pt_fwd_kernel (y pass)");
    }
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

template <int LOGP>
static bp_status launch_adj_rows_pt(bp_plan *p, float *sino, cudaStream_t st) {
    constexpr int NT = (1 << LOGP) / kPassE;
    constexpr size_t smem = sizeof(float2) * ((1 << LOGP) + pt_offset<LOGP>(PtPlan<LOGP>::npass));
    auto kern = adj_rows_pt_kernel<LOGP>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    const int npairs = (p->n_theta + 1) / 2;
    const int ctas = std::min(npairs, std::max(1, per_sm) * std::max(1, p->sm_count));
    kern<<<ctas, NT, smem, st>>>(p->four.spec, sino, p->d_twpass, p->n_theta, p->n_det);
    stage_mark(p, st, "adj_rows_pt_kernel");
    return BP_OK;
}

bp_status launch_radon_fourier(bp_plan *p, const float *img, float *sino, int batch, cudaStream_t st,
                               int per_angle_w) {
    bp_status s = ensure_fourier(p);
    if (s != BP_OK) return s;
    if ((s = ensure_adj_items(p)) != BP_OK) return s;
    FourierWork &f = p->four;
    const int N = p->N, M = f.M, P = p->P, H = P / 2;
    const int R = rows_per_cta(M);
    const size_t smemR = sizeof(float2) * ((size_t)R * M + M / 2);
    const int nthr = fft_threads(M);
    const int groups = 1;
    const bool e16 = fft_elems(M) == 16;
    auto kx = e16 ? adj_fft_x_kernel<16> : adj_fft_x_kernel<8>;
    auto ky = e16 ? adj_fft_y_kernel<16> : adj_fft_y_kernel<8>;
    auto kr = fft_elems(P) == 16 ? adj_rows_kernel<16> : adj_rows_kernel<8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemR));
    BP_CUDA_TRY(cudaFuncSetAttribute(ky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemR));
    BP_CUDA_TRY(cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float2) * (P + P / 2))));
    const float delta2 = (N % 2 == 0) ? 1.0f / (float)M : 0.0f;
    const float scale = (float)(p->dx * p->dx / p->dt);
    stage_begin(p, st);
    for (int b = 0; b < batch; ++b) {
        const float *ib = img + (size_t)b * N * N;
        switch (f.logM) {
            case 9: s = launch_fft_pt_fwd<9>(p, ib, st); break;
            case 10: s = launch_fft_pt_fwd<10>(p, ib, st); break;
            case 11: s = launch_fft_pt_fwd<11>(p, ib, st); break;
            case 12: s = launch_fft_pt_fwd<12>(p, ib, st); break;
            case 13: s = launch_fft_pt_fwd<13>(p, ib, st); break;
            default:
                kx<<<(N + R - 1) / R, nthr * groups, smemR, st>>>(ib, f.mid, f.deapod, f.twM, M, f.logM, N, R);
                stage_mark(p, st, "adj_fft_x_kernel");
                ky<<<M / R, nthr * groups, smemR, st>>>(f.mid, f.grid, f.twM, M, f.logM, N, R);
                stage_mark(p, st, "adj_fft_y_kernel");
        }
        if (s != BP_OK) return s;
        {
            auto kt = f.W == 4 ? adj_interp_tiled_kernel<2> : adj_interp_tiled_kernel<3>;
            const size_t sm = adj_tiled_smem(f.W / 2);
            BP_CUDA_TRY(cudaFuncSetAttribute(kt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            kt<<<f.adj_n_items, 256, sm, st>>>(f.grid, f.spec, f.ray, f.adj_items, f.adj_segs, M, H, P, p->n_det,
                                               f.kbtab, delta2, scale, per_angle_w ? f.wk : nullptr);
            stage_mark(p, st, "adj_interp_tiled_kernel");
        }
        float *sb = sino + (size_t)b * p->n_theta * p->n_det;
        switch (p->d_twpass ? ilog2(P) : 0) {
            case 9: s = launch_adj_rows_pt<9>(p, sb, st); break;
            case 10: s = launch_adj_rows_pt<10>(p, sb, st); break;
            case 11: s = launch_adj_rows_pt<11>(p, sb, st); break;
            case 12: s = launch_adj_rows_pt<12>(p, sb, st); break;
            default:
                kr<<<(p->n_theta + 1) / 2, fft_threads(P), sizeof(float2) * (P + P / 2), st>>>(
                    f.spec, sb, p->d_twP, p->n_theta, p->n_det, ilog2(P));
                stage_mark(p, st, "adj_rows_kernel");
        }
        if (s != BP_OK) return s;
        BP_CUDA_TRY(cudaGetLastError());
    }
    return BP_OK;
}

}  // namespace bp
