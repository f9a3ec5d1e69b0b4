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
// Kernels: (1) fourier_spectra: one CTA per projection pair, P-point FFT in shared memory,
// the two half spectra scaled into c_{k,m};  (2) grid_spread: one CTA per work item of a
// 32 x 32 grid tile (host-built list of ray segments that touch the tile, split so no
// item exceeds a fixed sample count), warp groups of 6 lanes spread one sample each into
// the shared-memory tile; the tile's first item stores it, later items add with global
// reductions (second launch);  (3) ifft_pass_y / ifft_pass_x: M-point inverse FFTs of R
// rows per CTA with output pruning to N points, transposed intermediate, fused
// deapodisation and real part.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "fft.cuh"
#include "tma.cuh"

namespace bp {

namespace {

constexpr int kW = 6;          // kernel width (grid cells)
constexpr int kTS = 32;        // grid tile side
constexpr int kMaxItem = 1024; // samples per gridding work item
constexpr int kGridThreads = 128;

struct GridSeg {
    int k, m_lo, m_hi, pad;
};
struct GridItem {
    int x0, y0, seg_begin, seg_end;
};

// Modified Bessel function I0 for x >= 0 by the polynomial approximations of Abramowitz &
// Stegun, Handbook of Mathematical Functions, 9.8.1 (x <= 3.75) and 9.8.2 (x >= 3.75),
// relative error below 2e-7.  Both branches are evaluated (no divergence).
__device__ __forceinline__ float bessel_i0(float x) {
    const float a = x * (1.0f / 3.75f);
    const float a2 = a * a;
    const float small =
        1.0f + a2 * (3.5156229f + a2 * (3.0899424f + a2 * (1.2067492f + a2 * (0.2659732f + a2 * (0.0360768f +
        a2 * 0.0045813f)))));
    const float t = 3.75f / fmaxf(x, 3.75f);
    const float p = 0.39894228f + t * (0.01328592f + t * (0.00225319f + t * (-0.00157565f + t * (0.00916281f +
                    t * (-0.02057706f + t * (0.02635537f + t * (-0.01647633f + t * 0.00392377f)))))));
    const float large = p * __expf(x) * rsqrtf(fmaxf(x, 3.75f));
    return x < 3.75f ? small : large;
}

__device__ __forceinline__ float kb_weight(float t, float beta) {
    // I0(beta sqrt(1 - (2t/W)^2)) for |t| <= W/2
    const float a = t * (2.0f / kW);
    const float r = fmaxf(0.f, 1.f - a * a);
    return bessel_i0(beta * sqrtf(r));
}

// ---------------------------------------------------------------------------------- (1) spectra
template <typename Tin, int E>
__global__ void __launch_bounds__(1024, 1)
fourier_spectra_kernel(const Tin *__restrict__ sino, float2 *__restrict__ spec, const float *__restrict__ wk,
                       const float2 *__restrict__ tw, int n_theta, int n_det, int logP, float wuni) {
    extern __shared__ __align__(16) float2 z[];
    const int P = 1 << logP, H = P >> 1;
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
    stockham_fft<E>(z, logP, tw, 1, false, threadIdx.x, blockDim.x);
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
        const float2 ph = make_float2(cs, sn);
        const float f = (m == 0) ? 1.f : 2.f;
        const float2 ca = cmul(A, ph), cb = cmul(B, ph);
        spec[(long long)k0 * H + m] = make_float2(f * wa * ca.x, f * wa * ca.y);
        if (has1) spec[(long long)k1 * H + m] = make_float2(f * wb * cb.x, f * wb * cb.y);
    }
}

// ---------------------------------------------------------------------------------- (2) gridding
// G[l_x][l_y] (l mod M).  One CTA per work item (segments of rays crossing one 32 x 32
// tile).  Each warp accumulates into its own copy of the tile with plain read-modify-writes:
// it takes one ray segment at a time, its lanes holding samples S apart on the ray, where
// S * rho * max(|cos|, |sin|) > 1 so that the lanes' base cells differ along the ray's
// dominant axis; for every footprint offset (tx, ty) the 32 lanes then touch 32 different
// cells.  The warp copies are summed at the end; the tile's first item stores the sum, later
// items add it with global reductions (second launch).
__global__ void __launch_bounds__(kGridThreads, 3)
grid_spread_kernel(const float2 *__restrict__ spec, const long long *__restrict__ ray, const GridSeg *__restrict__ segs,
                   const GridItem *__restrict__ items, float2 *__restrict__ grid, int M, int H, float beta,
                   float delta2_over_M, float rho, int accumulate) {
    __shared__ float2 acc[kGridThreads / 32][kTS][kTS + 1];
    const GridItem it = items[blockIdx.x];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float2(*mine)[kTS + 1] = acc[warp];
    for (int i = lane; i < kTS * kTS; i += 32) mine[i / kTS][i % kTS] = make_float2(0.f, 0.f);
    __syncwarp();
    const int Mmask = M - 1;
    for (int j = it.seg_begin + warp; j < it.seg_end; j += kGridThreads / 32) {
        const GridSeg sg = segs[j];
        const long long ax = ray[2 * sg.k], ay = ray[2 * sg.k + 1];
        const float2 *sk = spec + (long long)sg.k * H;
        const float step = fmaxf(fabsf((float)ax), fabsf((float)ay)) * 2.3283064365386963e-10f;  // rho max(|c|,|s|)
        const int S = (int)floorf(1.0f / fmaxf(step, 1e-6f)) + 1;
        for (int base = sg.m_lo; base <= sg.m_hi; base += 32 * S) {
            for (int ph = 0; ph < S; ++ph) {
                const int m = base + ph + S * lane;
                const bool act = m <= sg.m_hi;
                float wy[kW], wx[kW];
                float2 v = make_float2(0.f, 0.f);
                int fx = 0, fy = 0;
                if (act) {
                    const long long zx = (long long)m * ax, zy = (long long)m * ay;
                    fx = (int)(zx >> 32);
                    fy = (int)(zy >> 32);
                    const float rx = (float)(unsigned)(zx & 0xffffffffLL) * 2.3283064365386963e-10f;
                    const float ry = (float)(unsigned)(zy & 0xffffffffLL) * 2.3283064365386963e-10f;
                    v = __ldg(sk + m);
                    float sn, cs;
                    sincospif(((float)(fx + fy) + (rx + ry)) * delta2_over_M, &sn, &cs);
                    v = cmul(v, make_float2(cs, sn));
#pragma unroll
                    for (int t = 0; t < kW; ++t) {
                        wy[t] = kb_weight((float)(t - 2) - ry, beta);
                        wx[t] = kb_weight((float)(t - 2) - rx, beta);
                    }
                }
#pragma unroll
                for (int tx = 0; tx < kW; ++tx) {
                    const int lx = ((fx - 2 + tx) & Mmask) - it.x0;
                    const bool inx = act && lx >= 0 && lx < kTS;
                    const float2 vx = make_float2(wx[tx] * v.x, wx[tx] * v.y);
#pragma unroll
                    for (int ty = 0; ty < kW; ++ty) {
                        const int ly = ((fy - 2 + ty) & Mmask) - it.y0;
                        if (inx && ly >= 0 && ly < kTS) {
                            float2 c = mine[lx][ly];
                            c.x = fmaf(wy[ty], vx.x, c.x);
                            c.y = fmaf(wy[ty], vx.y, c.y);
                            mine[lx][ly] = c;
                        }
                        __syncwarp();
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTS * kTS; i += kGridThreads) {
        const int lx = i / kTS, ly = i % kTS;
        float2 v = acc[0][lx][ly];
#pragma unroll
        for (int w = 1; w < kGridThreads / 32; ++w) {
            v.x += acc[w][lx][ly].x;
            v.y += acc[w][lx][ly].y;
        }
        float2 *dst = grid + (long long)(it.x0 + lx) * M + (it.y0 + ly);
        if (accumulate) {
            if (v.x != 0.f) atomicAdd(&dst->x, v.x);
            if (v.y != 0.f) atomicAdd(&dst->y, v.y);
        } else {
            *dst = v;
        }
    }
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
    const int lx0 = blockIdx.x * R;
    const int nthr = fft_threads(M), groups = blockDim.x / nthr;
    const int g = threadIdx.x / nthr, tid = threadIdx.x - g * nthr;
    if (!load_rows_async(z, grid + (long long)lx0 * M, R * M, &bar) && threadIdx.x == 0) atomicExch(err, 1);
    for (int r0 = 0; r0 < R; r0 += groups) stockham_fft<E>(z + (r0 + g) * M, logM, tw, 1, true, tid, nthr);
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
    const int iy0 = blockIdx.x * R;
    const int rows = min(R, N - iy0);
    const int nthr = fft_threads(M), groups = blockDim.x / nthr;
    const int g = threadIdx.x / nthr, tid = threadIdx.x - g * nthr;
    if (!load_rows_async(z, inter + (long long)iy0 * M, rows * M, &bar) && threadIdx.x == 0) atomicExch(err, 1);
    // rows beyond the last image row hold stale data that is transformed but never written out
    for (int r0 = 0; r0 < R; r0 += groups) stockham_fft<E>(z + (r0 + g) * M, logM, tw, 1, true, tid, nthr);
    const int h = N / 2;
    for (int i = threadIdx.x; i < rows * N; i += blockDim.x) {
        const int r = i / N, ix = i - r * N;
        const int pos = (ix - h) & (M - 1);
        img[(long long)(iy0 + r) * N + ix] = z[r * M + pos].x * __ldg(deap + ix);
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
    for (int r0 = 0; r0 < R; r0 += groups) stockham_fft<E>(z + (r0 + g) * M, logM, tw, 1, false, tid, nthr);
    for (int i = threadIdx.x; i < rows * M; i += blockDim.x) T[(long long)iy0 * M + i] = z[i];
}

// Pass along y: columns l_x (R per CTA) of T, embedded at (i_y - floor(N/2)) mod M, forward
// FFT, written to G[l_x][l_y].
template <int E>
__global__ void __launch_bounds__(1024, 1)
adj_fft_y_kernel(const float2 *__restrict__ T, float2 *__restrict__ grid, const float2 *__restrict__ tw, int M,
                 int logM, int N, int R) {
    extern __shared__ __align__(128) float2 z[];
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
    for (int r0 = 0; r0 < R; r0 += groups) stockham_fft<E>(z + (r0 + g) * M, logM, tw, 1, false, tid, nthr);
    for (int i = threadIdx.x; i < R * M; i += blockDim.x) grid[(long long)lx0 * M + i] = z[i];
}

// Interpolation at the polar samples (transpose of the spreading): one thread per sample,
// consecutive samples of one ray in consecutive lanes; result times the conjugate sample
// factor (1/P)(m ? 2 : 1) exp(-i pi m (n_det-1)/P) exp(-2 pi i delta (z_x + z_y)/M) and dx^2/dt.
__global__ void __launch_bounds__(256)
adj_interp_kernel(const float2 *__restrict__ grid, float2 *__restrict__ spec, const long long *__restrict__ ray,
                  int M, int H, int P, int n_det, float beta, float delta2_over_M, float scale,
                  const float *__restrict__ wk) {
    const int k = blockIdx.y;
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= H) return;
    const long long zx = (long long)m * ray[2 * k], zy = (long long)m * ray[2 * k + 1];
    const int fx = (int)(zx >> 32), fy = (int)(zy >> 32);
    const float rx = (float)(unsigned)(zx & 0xffffffffLL) * 2.3283064365386963e-10f;
    const float ry = (float)(unsigned)(zy & 0xffffffffLL) * 2.3283064365386963e-10f;
    const int Mmask = M - 1;
    float wy[kW];
#pragma unroll
    for (int t = 0; t < kW; ++t) wy[t] = kb_weight((float)(t - 2) - ry, beta);
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int tx = 0; tx < kW; ++tx) {
        const float wx = kb_weight((float)(tx - 2) - rx, beta);
        const float2 *row = grid + (long long)((fx - 2 + tx) & Mmask) * M;
        float2 r = make_float2(0.f, 0.f);
#pragma unroll
        for (int ty = 0; ty < kW; ++ty) {
            const float2 v = __ldg(row + ((fy - 2 + ty) & Mmask));
            r.x = fmaf(wy[ty], v.x, r.x);
            r.y = fmaf(wy[ty], v.y, r.y);
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

// Per projection pair: y_j = Re sum_{m < P/2} s_m exp(2 pi i m j / P) = (1/2) IFFT(Hermitian(s))_j;
// two real outputs share one complex transform (Z = H_a + i H_b).
template <int E>
__global__ void __launch_bounds__(1024, 1)
adj_rows_kernel(const float2 *__restrict__ spec, float *__restrict__ sino, const float2 *__restrict__ tw,
                int n_theta, int n_det, int logP) {
    extern __shared__ __align__(16) float2 z[];
    const int P = 1 << logP, H = P >> 1;
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
    stockham_fft<E>(z, logP, tw, 1, true, threadIdx.x, blockDim.x);
    for (int j = threadIdx.x; j < n_det; j += blockDim.x) {
        sino[(long long)k0 * n_det + j] = 0.5f * z[j].x;
        if (has1) sino[(long long)k1 * n_det + j] = 0.5f * z[j].y;
    }
}

double kb_hat(double f, double beta) {
    // Fourier transform of I0(beta sqrt(1 - (2t/W)^2)) on |t| <= W/2 at frequency f (cycles per cell)
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
    cudaFree(f.ray);
    cudaFree(f.segs);
    cudaFree(f.items);
    f = FourierWork();
}

// Host (FP64) geometry of the gridding step: per-angle ray steps in 32.32 fixed point,
// the ray segments that touch every 32 x 32 grid tile, and balanced work items.
bp_status ensure_fourier(bp_plan *p) {
    FourierWork &f = p->four;
    if (f.grid) return BP_OK;
    const int N = p->N, n_theta = p->n_theta, P = p->P, H = P / 2;
    int M = 1;
    while (M < 2 * N) M <<= 1;
    M = std::max(M, kTS);
    if ((size_t)M * sizeof(float2) > 128u * 1024u)
        return fail(BP_ERR_UNSUPPORTED, "Fourier path: N too large for the shared-memory FFT (N <= 8192)");
    if ((size_t)P * sizeof(float2) > 200u * 1024u)
        return fail(BP_ERR_UNSUPPORTED, "Fourier path: n_det too large for the shared-memory FFT (n_det <= 8192)");
    const double sigma = (double)M / N;
    double b2 = (kW / sigma) * (kW / sigma) * (sigma - 0.5) * (sigma - 0.5) - 0.8;
    const double beta = M_PI * std::sqrt(std::max(b2, 1.0));
    const double rho = (double)M * p->dx / ((double)P * p->dt);

    // ray steps and the sample walk that builds the tile segments
    std::vector<long long> ray(2 * (size_t)n_theta);
    const int tiles1 = M / kTS;
    std::vector<int> last(tiles1 * tiles1, -1);
    std::vector<GridSeg> segs;
    std::vector<int> seg_tile;
    segs.reserve((size_t)n_theta * 4 * (H / kTS + 2));
    for (int k = 0; k < n_theta; ++k) {
        const long long ax = (long long)std::llround(std::ldexp(rho * std::cos(p->theta[k]), 32));
        const long long ay = (long long)std::llround(std::ldexp(rho * std::sin(p->theta[k]), 32));
        ray[2 * k] = ax;
        ray[2 * k + 1] = ay;
        for (int m = 0; m < H; ++m) {
            const int fx = (int)(((long long)m * ax) >> 32), fy = (int)(((long long)m * ay) >> 32);
            const int tx0 = ((fx - 2) & (M - 1)) / kTS, tx1 = ((fx + 3) & (M - 1)) / kTS;
            const int ty0 = ((fy - 2) & (M - 1)) / kTS, ty1 = ((fy + 3) & (M - 1)) / kTS;
            const int txs[2] = {tx0, tx1}, tys[2] = {ty0, ty1};
            for (int a = 0; a < (tx0 == tx1 ? 1 : 2); ++a)
                for (int b = 0; b < (ty0 == ty1 ? 1 : 2); ++b) {
                    const int t = txs[a] * tiles1 + tys[b];
                    const int li = last[t];
                    if (li >= 0 && segs[li].k == k && segs[li].m_hi == m - 1) {
                        segs[li].m_hi = m;
                    } else {
                        last[t] = (int)segs.size();
                        segs.push_back(GridSeg{k, m, m, 0});
                        seg_tile.push_back(t);
                    }
                }
        }
    }
    // group segments by tile (counting sort), split each tile's list into items
    const int ntiles = tiles1 * tiles1;
    std::vector<int> cnt(ntiles + 1, 0);
    for (int t : seg_tile) cnt[t + 1]++;
    for (int t = 0; t < ntiles; ++t) cnt[t + 1] += cnt[t];
    std::vector<GridSeg> sorted(segs.size());
    {
        std::vector<int> pos(cnt.begin(), cnt.end() - 1);
        for (size_t i = 0; i < segs.size(); ++i) sorted[pos[seg_tile[i]]++] = segs[i];
    }
    std::vector<GridItem> owners, extras;
    owners.reserve(ntiles);
    for (int t = 0; t < ntiles; ++t) {
        const int x0 = (t / tiles1) * kTS, y0 = (t % tiles1) * kTS;
        int b = cnt[t], e = cnt[t + 1];
        bool first = true;
        do {
            int s = b, load = 0;
            while (s < e && (load == 0 || load + (sorted[s].m_hi - sorted[s].m_lo + 1) <= kMaxItem)) {
                load += sorted[s].m_hi - sorted[s].m_lo + 1;
                ++s;
            }
            (first ? owners : extras).push_back(GridItem{x0, y0, b, s});
            first = false;
            b = s;
        } while (b < e);
    }
    // deapodisation 1 / phi_hat(i - floor(N/2)) (separable), weights, twiddles
    std::vector<float> deap(N), wk(n_theta);
    for (int i = 0; i < N; ++i) deap[i] = (float)(1.0 / kb_hat((double)(i - N / 2) / M, beta));
    for (int k = 0; k < n_theta; ++k) wk[k] = (float)p->w[k];
    std::vector<float2> tw(M / 2);
    for (int i = 0; i < M / 2; ++i) {
        const double a = -2.0 * M_PI * (double)i / (double)M;
        tw[i] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    std::vector<GridItem> all(owners);
    all.insert(all.end(), extras.begin(), extras.end());

    f.M = M;
    f.logM = ilog2(M);
    f.beta = (float)beta;
    f.rho = (float)rho;
    f.n_segs = (int)sorted.size();
    f.n_owner = (int)owners.size();
    f.n_extra = (int)extras.size();
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
    alloc((void **)&f.ray, sizeof(long long) * ray.size());
    alloc(&f.segs, sizeof(GridSeg) * sorted.size());
    alloc(&f.items, sizeof(GridItem) * all.size());
    if (e == cudaSuccess) e = cudaMemcpy(f.deapod, deap.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f.wk, wk.data(), sizeof(float) * n_theta, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f.twM, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f.ray, ray.data(), sizeof(long long) * ray.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !sorted.empty())
        e = cudaMemcpy(f.segs, sorted.data(), sizeof(GridSeg) * sorted.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f.items, all.data(), sizeof(GridItem) * all.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_fourier(p);
        return cuda_fail(e, "Fourier workspace");
    }
    return BP_OK;
}

template <typename Tin>
static bp_status spectra_t(bp_plan *p, const Tin *sino, cudaStream_t st, float wuni) {
    const int logP = ilog2(p->P);
    const size_t smem = sizeof(float2) * p->P;
    const int threads = fft_threads(p->P);
    auto kern = fft_elems(p->P) == 16 ? fourier_spectra_kernel<Tin, 16> : fourier_spectra_kernel<Tin, 8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(p->n_theta + 1) / 2, threads, smem, st>>>(sino, p->four.spec, p->four.wk, p->d_twP, p->n_theta, p->n_det,
                                                      logP, wuni);
    return BP_OK;
}

static int rows_per_cta(int M) { return std::max(1, std::min(4, (int)(131072 / (sizeof(float2) * M)))); }

bp_status launch_fourier(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, cudaStream_t st,
                         float wuni) {
    bp_status s = ensure_fourier(p);
    if (s != BP_OK) return s;
    FourierWork &f = p->four;
    const int N = p->N, M = f.M, H = p->P / 2;
    const size_t esz = dt == BP_F32 ? 4 : 2;
    const int R = rows_per_cta(M);
    const size_t smemR = sizeof(float2) * (size_t)R * M;
    auto pass_y = fft_elems(M) == 16 ? ifft_pass_y_kernel<16> : ifft_pass_y_kernel<8>;
    auto pass_x = fft_elems(M) == 16 ? ifft_pass_x_kernel<16> : ifft_pass_x_kernel<8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(pass_y, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemR));
    BP_CUDA_TRY(cudaFuncSetAttribute(pass_x, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemR));
    const int nthr = fft_threads(M);
    int groups = 1;
    while (groups * 2 <= R && nthr * groups * 2 <= 1024) groups *= 2;
    const float delta2 = (N % 2 == 0) ? 1.0f / (float)M : 0.0f;  // 2 delta / M
    for (int b = 0; b < batch; ++b) {
        const char *sb = (const char *)sino + esz * (size_t)b * p->n_theta * p->n_det;
        switch (dt) {
            case BP_F32: s = spectra_t(p, (const float *)sb, st, wuni); break;
            case BP_BF16: s = spectra_t(p, (const __nv_bfloat16 *)sb, st, wuni); break;
            case BP_F16: s = spectra_t(p, (const __half *)sb, st, wuni); break;
        }
        if (s != BP_OK) return s;
        const GridItem *items = (const GridItem *)f.items;
        grid_spread_kernel<<<f.n_owner, kGridThreads, 0, st>>>(f.spec, f.ray, (const GridSeg *)f.segs, items, f.grid,
                                                               M, H, f.beta, delta2, f.rho, 0);
        if (f.n_extra > 0)
            grid_spread_kernel<<<f.n_extra, kGridThreads, 0, st>>>(f.spec, f.ray, (const GridSeg *)f.segs,
                                                                   items + f.n_owner, f.grid, M, H, f.beta, delta2,
                                                                   f.rho, 1);
        pass_y<<<M / R, nthr * groups, smemR, st>>>(f.grid, f.mid, f.deapod, f.twM, M, f.logM, N, R,
                                                           p->d_err);
        pass_x<<<(N + R - 1) / R, nthr * groups, smemR, st>>>(f.mid, img + (size_t)b * N * N, f.deapod,
                                                                     f.twM, M, f.logM, N, R, p->d_err);
        BP_CUDA_TRY(cudaGetLastError());
    }
    return BP_OK;
}

bp_status launch_radon_fourier(bp_plan *p, const float *img, float *sino, int batch, cudaStream_t st,
                               int per_angle_w) {
    bp_status s = ensure_fourier(p);
    if (s != BP_OK) return s;
    FourierWork &f = p->four;
    const int N = p->N, M = f.M, P = p->P, H = P / 2;
    const int R = rows_per_cta(M);
    const size_t smemR = sizeof(float2) * (size_t)R * M;
    const int nthr = fft_threads(M);
    int groups = 1;
    while (groups * 2 <= R && nthr * groups * 2 <= 1024) groups *= 2;
    const bool e16 = fft_elems(M) == 16;
    auto kx = e16 ? adj_fft_x_kernel<16> : adj_fft_x_kernel<8>;
    auto ky = e16 ? adj_fft_y_kernel<16> : adj_fft_y_kernel<8>;
    auto kr = fft_elems(P) == 16 ? adj_rows_kernel<16> : adj_rows_kernel<8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemR));
    BP_CUDA_TRY(cudaFuncSetAttribute(ky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemR));
    BP_CUDA_TRY(cudaFuncSetAttribute(kr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(float2) * P)));
    const float delta2 = (N % 2 == 0) ? 1.0f / (float)M : 0.0f;
    const float scale = (float)(p->dx * p->dx / p->dt);
    for (int b = 0; b < batch; ++b) {
        kx<<<(N + R - 1) / R, nthr * groups, smemR, st>>>(img + (size_t)b * N * N, f.mid, f.deapod, f.twM, M, f.logM,
                                                         N, R);
        ky<<<M / R, nthr * groups, smemR, st>>>(f.mid, f.grid, f.twM, M, f.logM, N, R);
        adj_interp_kernel<<<dim3((H + 255) / 256, p->n_theta), 256, 0, st>>>(f.grid, f.spec, f.ray, M, H, P, p->n_det,
                                                                              f.beta, delta2, scale,
                                                                              per_angle_w ? f.wk : nullptr);
        kr<<<(p->n_theta + 1) / 2, fft_threads(P), sizeof(float2) * P, st>>>(
            f.spec, sino + (size_t)b * p->n_theta * p->n_det, p->d_twP, p->n_theta, p->n_det, ilog2(P));
        BP_CUDA_TRY(cudaGetLastError());
    }
    return BP_OK;
}

}  // namespace bp
