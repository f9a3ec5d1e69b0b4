// The paper's own Backprojection-Slice-Theorem algorithm (Section 5.3, Steps 1-4; the
// theorem is eq "bst" of Section 3, the kernel K^sigma at the origin eq "kernel"): the
// backprojection's 2D transform is read off the projections' 1D transforms on a polar grid
// and interpolated linearly to a Cartesian grid, then inverted by a 2D inverse FFT.
//
// Conventions (shared with the gridding form in fourier.cu): each projection is zero-padded
// to Pb = os P points (os = radial oversampling, P = 2^ceil(log2(2 n_det))); its transform at
// kappa_m = m / (Pb dt) is ghat_k = dt e^{i pi m (n_det-1)/Pb} G_k[m]; by the BST the
// backprojection's transform on ray theta_k is bhat = ghat_k K^sigma with K^sigma =
// 1/|kappa| (1/dkappa at kappa = 0), i.e.
//     bhat_k[m] = Pb dt^2 e^{i pi m (n_det-1)/Pb} G_k[m] / max(m, 1),   m < Pb/2,
// and on the opposite ray theta_k + pi its complex conjugate (Step 1: the full lines of
// theta in [0, pi) are the semi-polar half-lines of theta in [0, 2 pi), so there is no s = 0
// boundary and the window of Step 2.1 is not needed).  The Cartesian node l (frequency
// l / (M dx), M = max(2^ceil(log2(2N)), 64)) takes the value interpolated linearly in the
// fractional sample index |l| / rho (rho = M dx / (Pb dt) grid cells per sample) and in angle
// between the two bracketing rays (Step 3); the image is the Riemann sum of the inverse
// transform, (1/(M dx))^2 Re sum_l bhat(l) e^{2 pi i l . x / (M dx)} (Step 4), computed by the
// pruned inverse-FFT passes of the Fourier path without deapodisation.
//
// Kernels: bst_polar_kernel (one CTA per projection pair, Pb-point shared-memory FFT);
// bst_interp_kernel (one thread per Cartesian node: angle bracket by O(1) lookup for uniform
// angle sets, else binary search; four complex loads; the origin node, shared by every ray,
// takes the mean of the rays' values); the inverse passes of fourier.cu.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "fft.cuh"
#include "lp_rows.cuh"

namespace bp {

namespace {

constexpr int kConjBit = 1 << 30;

template <typename Tin, int E>
__global__ void __launch_bounds__(1024, 1)
bst_polar_kernel(const Tin *__restrict__ sino, float2 *__restrict__ polar, const float2 *__restrict__ tw,
                 int n_theta, int n_det, int logP, float scale) {
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
    const long long twoP = 2LL * P;
    for (int m = threadIdx.x; m < H; m += blockDim.x) {
        // the two rows' transforms from the packed one: A = (Z[m] + conj Z[P-m]) / 2, B = (Z[m] - conj Z[P-m]) / 2i
        const float2 zm = z[m];
        const float2 zc = z[(P - m) & (P - 1)];
        const float2 A = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
        const float2 B = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
        const long long r = ((long long)m * (n_det - 1)) % twoP;  // detector-centre phase, reduced mod 2P
        float sn, cs;
        sincospif((float)r / (float)P, &sn, &cs);
        const float2 ph = make_float2(cs, sn);
        const float f = scale / (float)max(m, 1);  // K^sigma
        const float2 ca = cmul(A, ph);
        polar[(long long)k0 * H + m] = make_float2(f * ca.x, f * ca.y);
        if (has1) {
            const float2 cb = cmul(B, ph);
            polar[(long long)k1 * H + m] = make_float2(f * cb.x, f * cb.y);
        }
    }
}

// Steps 1 and 2.1 on semi-polar half-lines with the window of eq "w": the half-lines of
// projection k sampled at s_i = i dt (linear interpolation between detector centres, zero
// off the detector) times w_i, joined into one line t = i dt, |i| < ns, whose centre sample
// is shared by the two half-lines.  By linearity the transform of this line is the sum of the
// two half-lines' one-sided transforms (conjugated for the opposite one), which is what
// Step 2.2 needs on each ray, so the full-line kernels below do the rest.
// The same polar values from a persistent kernel for Pb = 2^(LOGH + 1), LOGH = 9 .. 13: each
// Pb-point transform of a packed projection pair as two register-first Pb/2-point transforms
// of its even and odd samples combined in registers (lp_rows.cuh); X[Pb - m] for the two
// rows' separation comes from the upper half through the work array.
template <typename Tin, int LOGH>
__global__ void __launch_bounds__((1 << LOGH) / kPassE, 1)
bst_polar_pt_kernel(const Tin *__restrict__ sino, float2 *__restrict__ polar, const float2 *__restrict__ twp,
                    const float2 *__restrict__ twPb, int n_theta, int n_det, float scale) {
    constexpr int H = 1 << LOGH, P = 2 * H, NT = H / kPassE;
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
        lp_dit_row<LOGH, false>(ae, ao, z, Tw, sE, twPb, t, xl, xu);
        __syncthreads();  // every thread is done with z (the second transform)
#pragma unroll
        for (int m = 0; m < kPassE; ++m) z[t + m * NT] = xu[m];
        __syncthreads();
#pragma unroll
        for (int mi = 0; mi < kPassE; ++mi) {
            const int m = t + mi * NT;  // Z[Pb - m] = X[H + (H - m)] (m > 0), X[0] for m = 0
            const float2 zm = xl[mi], zc = m == 0 ? xl[mi] : z[H - m];
            const float2 A = make_float2(0.5f * (zm.x + zc.x), 0.5f * (zm.y - zc.y));
            const float2 B = make_float2(0.5f * (zm.y + zc.y), -0.5f * (zm.x - zc.x));
            const long long r = ((long long)m * (n_det - 1)) % twoP;  // detector-centre phase, reduced mod 2P
            float sn, cs;
            sincospif((float)r / (float)P, &sn, &cs);
            const float2 ph = make_float2(cs, sn);
            const float f = scale / (float)max(m, 1);  // K^sigma
            const float2 ca = cmul(A, ph);
            polar[(long long)k0 * H + m] = make_float2(f * ca.x, f * ca.y);
            if (has1) {
                const float2 cb = cmul(B, ph);
                polar[(long long)k1 * H + m] = make_float2(f * cb.x, f * cb.y);
            }
        }
    }
}

template <typename Tin>
__global__ void __launch_bounds__(256)
bst_window_rows_kernel(const Tin *__restrict__ sino, float *__restrict__ rows, const float *__restrict__ win,
                       int n_theta, int n_det, int ns) {
    const int np = 2 * ns - 1;
    const long long total = (long long)n_theta * np;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(idx / np), i = (int)(idx - (long long)k * np) - (ns - 1);  // t = i dt
        const Tin *row = sino + (long long)k * n_det;
        float v;
        if (n_det & 1) {  // u = i + (n_det - 1) / 2 is a detector centre
            const int j = i + (n_det - 1) / 2;
            v = (j >= 0 && j < n_det) ? load_f(row + j) : 0.f;
        } else {          // u is half-way between centres j0 and j0 + 1
            const int j0 = i + n_det / 2 - 1;
            const float a = (j0 >= 0 && j0 < n_det) ? load_f(row + j0) : 0.f;
            const float b = (j0 + 1 >= 0 && j0 + 1 < n_det) ? load_f(row + j0 + 1) : 0.f;
            v = 0.5f * (a + b);
        }
        rows[idx] = v * __ldg(win + (i < 0 ? -i : i));
    }
}

// Index of the last sorted angle <= phi (-1 if none).
__device__ __forceinline__ int last_at_most(const float *__restrict__ ang, const RayIndex &ri, float phi) {
    if (ri.uniform) return min(ri.n - 1, max(-1, (int)floorf((phi - ri.phi0) / ri.dphi)));
    int l = 0, h = ri.n;
    while (l < h) {
        const int mid = (l + h) >> 1;
        if (__ldg(ang + mid) <= phi) l = mid + 1;
        else h = mid;
    }
    return l - 1;
}

__device__ __forceinline__ float2 ray_sample(const float2 *__restrict__ polar, int code, int m, int H) {
    if (m >= H) return make_float2(0.f, 0.f);
    const float2 v = __ldg(polar + (long long)(code & (kConjBit - 1)) * H + m);
    return (code & kConjBit) ? make_float2(v.x, -v.y) : v;
}

// Interpolation weights to float rounding of the weights themselves: at radius m' ~ Pb/2
// samples or angle ~ 2 pi a plain float position would lose ~1e-3 of the fractions, so the
// radius is a two-float sqrt times a two-float 1/rho, and the angle is measured from ray a
// (its direction as two floats) through an exact cross product.
__global__ void __launch_bounds__(256)
bst_interp_kernel(const float2 *__restrict__ polar, const float *__restrict__ ang, const int *__restrict__ ray,
                  const float4 *__restrict__ dir, const float *__restrict__ inv_gap, RayIndex ri,
                  float2 *__restrict__ grid, int M, int H, float ih, float il, float scale, float delta2_over_M,
                  int n_theta) {
    const int ly = blockIdx.x * 32 + (threadIdx.x & 31);
    const int lx = blockIdx.y * 8 + (threadIdx.x >> 5);
    __shared__ float red[256];
    if (blockIdx.x == 0 && blockIdx.y == 0) {
        // the origin node belongs to every ray: the mean of their (real) values there, by a
        // fixed-order block reduction
        float s = 0.f;
        for (int k = threadIdx.x; k < n_theta; k += blockDim.x) s += __ldg(polar + (long long)k * H).x;
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) grid[0] = make_float2(scale * red[0] / (float)n_theta, 0.f);
        if (lx == 0 && ly == 0) return;
    }
    if (lx >= M || ly >= M) return;
    const int cx = lx < M / 2 ? lx : lx - M, cy = ly < M / 2 ? ly : ly - M;
    const float fx = (float)cx, fy = (float)cy;
    // fractional radial sample index m' = |l| / rho: |l| = s + slo (two floats), u = |l|^2 exact;
    // nodes beyond the last radial sample are zero (no angle needed)
    const int u = cx * cx + cy * cy;
    const float uh = (float)(u & ~0xff), ul = (float)(u & 0xff);
    const float sq = sqrtf(uh + ul);
    const float slo = (fmaf(-sq, sq, uh) + ul) / (2.f * sq);
    const float mh = sq * ih;
    const float ml = fmaf(sq, ih, -mh) + fmaf(slo, ih, sq * il);
    int m0 = (int)floorf(mh);
    float tm = (mh - (float)m0) + ml;
    if (tm < 0.f) {
        m0 -= 1;
        tm += 1.f;
    } else if (tm >= 1.f) {
        m0 += 1;
        tm -= 1.f;
    }
    if (m0 >= H) {
        grid[(long long)lx * M + ly] = make_float2(0.f, 0.f);
        return;
    }
    const float twopi = 6.2831853071795865f;
    float phi = atan2f(fy, fx);
    if (phi < 0.f) phi += twopi;
    // bracketing rays a, b (cyclic in angle); t = angle from ray a / angular gap a -> b
    const int n = ri.n;
    int a = last_at_most(ang, ri, phi);
    if (a < 0) a = n - 1;
    const int b = (a + 1 == n) ? 0 : a + 1;
    const float4 d = __ldg(dir + a);  // (cos, sin) of ray a: high parts, low parts
    const float p1 = d.x * fy, p2 = d.y * fx;
    const float e1 = fmaf(d.x, fy, -p1), e2 = fmaf(d.y, fx, -p2);
    const float cr = (p1 - p2) + ((e1 - e2) + fmaf(d.z, fy, -d.w * fx));  // xi_a x l
    const float dt = fmaf(d.x, fx, d.y * fy);                              // xi_a . l
    const float t = (n > 1) ? atan2f(cr, dt) * __ldg(inv_gap + a) : 0.f;
    float2 v = make_float2(0.f, 0.f);
    {
        const int ca = __ldg(ray + a), cb = __ldg(ray + b);
        const float2 a0 = ray_sample(polar, ca, m0, H), a1 = ray_sample(polar, ca, m0 + 1, H);
        const float2 b0 = ray_sample(polar, cb, m0, H), b1 = ray_sample(polar, cb, m0 + 1, H);
        const float2 va = make_float2(fmaf(tm, a1.x - a0.x, a0.x), fmaf(tm, a1.y - a0.y, a0.y));
        const float2 vb = make_float2(fmaf(tm, b1.x - b0.x, b0.x), fmaf(tm, b1.y - b0.y, b0.y));
        v = make_float2(scale * fmaf(t, vb.x - va.x, va.x), scale * fmaf(t, vb.y - va.y, va.y));
        if (delta2_over_M != 0.f) {
            // half-pixel phase exp(2 pi i delta (l_x + l_y) / M) of the pixel-centre offset
            float sn, cs;
            sincospif(delta2_over_M * (float)(cx + cy), &sn, &cs);
            v = cmul(v, make_float2(cs, sn));
        }
    }
    grid[(long long)lx * M + ly] = v;
}

// Rows of n_det samples (n_det <= Pb) centred on t = 0.
template <typename Tin, int LOGH>
bp_status polar_pt(bp_plan *p, const Tin *sino, int n_det, float scale, cudaStream_t st) {
    BstWork &w = p->bst;
    constexpr size_t smem = lp_rows_pt_smem<LOGH>();
    auto kern = bst_polar_pt_kernel<Tin, LOGH>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (1 << LOGH) / kPassE, smem));
    const int ctas = std::min((p->n_theta + 1) / 2, std::max(1, per_sm) * std::max(1, p->sm_count));
    kern<<<ctas, (1 << LOGH) / kPassE, smem, st>>>(sino, w.polar, w.twPassH, w.twPb, p->n_theta, n_det, scale);
    BP_CUDA_TRY(cudaGetLastError());
    stage_mark(p, st, "bst_polar_kernel");
    return BP_OK;
}

template <typename Tin>
bp_status polar_t(bp_plan *p, const Tin *sino, int n_det, cudaStream_t st) {
    BstWork &w = p->bst;
    if (w.twPassH) {
        const float scale = (float)((double)w.Pb * p->dt * p->dt);
        switch (ilog2(w.Pb) - 1) {
            case 9: return polar_pt<Tin, 9>(p, sino, n_det, scale, st);
            case 10: return polar_pt<Tin, 10>(p, sino, n_det, scale, st);
            case 11: return polar_pt<Tin, 11>(p, sino, n_det, scale, st);
            case 12: return polar_pt<Tin, 12>(p, sino, n_det, scale, st);
            case 13: return polar_pt<Tin, 13>(p, sino, n_det, scale, st);
            default: break;
        }
    }
    const int logP = ilog2(w.Pb);
    const size_t smem = sizeof(float2) * (w.Pb + w.Pb / 2);
    auto kern = fft_elems(w.Pb) == 16 ? bst_polar_kernel<Tin, 16> : bst_polar_kernel<Tin, 8>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const float scale = (float)((double)w.Pb * p->dt * p->dt);
    kern<<<(p->n_theta + 1) / 2, fft_threads(w.Pb), smem, st>>>(sino, w.polar, w.twPb, p->n_theta, n_det, logP,
                                                                scale);
    BP_CUDA_TRY(cudaGetLastError());
    stage_mark(p, st, "bst_polar_kernel");
    return BP_OK;
}

bp_status ensure_bst(bp_plan *p, int os) {
    BstWork &w = p->bst;
    if (w.polar && w.os == os) return BP_OK;
    free_bst(p);  // (also the windowed form's rows: ensure_bst_window makes them again)
    bp_status s = ensure_fourier(p);
    if (s != BP_OK) return s;
    const int n = p->n_theta, Pb = p->P * os, H = Pb / 2;
    // ray directions theta_k (the m >= 0 half) and theta_k + pi (conjugate values), sorted
    std::vector<std::pair<double, int>> r(2 * (size_t)n);
    for (int k = 0; k < n; ++k) {
        double a = std::fmod(p->theta[k], 2.0 * M_PI);
        if (a < 0) a += 2.0 * M_PI;
        double b = std::fmod(a + M_PI, 2.0 * M_PI);
        if (a >= 2.0 * M_PI) a = 0.0;
        if (b >= 2.0 * M_PI) b = 0.0;
        r[2 * (size_t)k] = {a, k};
        r[2 * (size_t)k + 1] = {b, k | kConjBit};
    }
    std::stable_sort(r.begin(), r.end(),
                     [](const std::pair<double, int> &x, const std::pair<double, int> &y) { return x.first < y.first; });
    const int R = 2 * n;
    std::vector<float> ang(R);
    std::vector<int> code(R);
    for (int i = 0; i < R; ++i) {
        ang[i] = std::min((float)r[i].first, std::nextafter((float)(2.0 * M_PI), 0.f));
        if (i > 0 && ang[i] < ang[i - 1]) ang[i] = ang[i - 1];
        code[i] = r[i].second;
    }
    // ray directions as two floats (high, low) and 1 / the angular gap to the next ray
    std::vector<float4> dirs(R);
    std::vector<float> igap(R);
    for (int i = 0; i < R; ++i) {
        const double c = std::cos(r[i].first), sn = std::sin(r[i].first);
        const float ch = (float)c, sh = (float)sn;
        dirs[i] = make_float4(ch, sh, (float)(c - ch), (float)(sn - sh));
        const double next = (i + 1 < R) ? r[i + 1].first : r[0].first + 2.0 * M_PI;
        const double gap = next - r[i].first;
        igap[i] = gap > 0 ? (float)(1.0 / gap) : 0.f;
    }
    w.ri = RayIndex();
    w.ri.n = R;
    if (R > 1) {
        const double d = (r[R - 1].first - r[0].first) / (R - 1);
        bool uni = d > 0;
        for (int i = 0; i < R && uni; ++i) uni = std::fabs(r[i].first - (r[0].first + i * d)) < 1e-9;
        if (uni) {
            w.ri.uniform = 1;
            w.ri.phi0 = (float)r[0].first;
            w.ri.dphi = (float)d;
        }
    }
    std::vector<float2> tw(H);
    for (int i = 0; i < H; ++i) {
        const double an = -2.0 * M_PI * (double)i / (double)Pb;
        tw[i] = make_float2((float)std::cos(an), (float)std::sin(an));
    }
    std::vector<float> ones(p->N, 1.0f);
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void **ptr, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(ptr, std::max<size_t>(bytes, 16));
        if (e == cudaSuccess) w.bytes += bytes;
    };
    std::vector<float2> twph;  // per-pass twiddles of the Pb/2-point transform (the persistent polar kernel)
    if (H >= 512 && H <= 8192) {
        build_pass_twiddles(ilog2(H), twph);
        twph.resize((twph.size() + 1) & ~(size_t)1);
        alloc((void **)&w.twPassH, sizeof(float2) * twph.size());
    }
    alloc((void **)&w.polar, sizeof(float2) * (size_t)n * H);
    alloc((void **)&w.twPb, sizeof(float2) * tw.size());
    alloc((void **)&w.ang, sizeof(float) * R);
    alloc((void **)&w.ray, sizeof(int) * R);
    alloc((void **)&w.ones, sizeof(float) * p->N);
    alloc((void **)&w.dir, sizeof(float4) * R);
    alloc((void **)&w.igap, sizeof(float) * R);
    if (e == cudaSuccess) e = cudaMemcpy(w.dir, dirs.data(), sizeof(float4) * R, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.igap, igap.data(), sizeof(float) * R, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.twPb, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.ang, ang.data(), sizeof(float) * R, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.ray, code.data(), sizeof(int) * R, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(w.ones, ones.data(), sizeof(float) * p->N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !twph.empty())
        e = cudaMemcpy(w.twPassH, twph.data(), sizeof(float2) * twph.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_bst(p);
        return cuda_fail(e, "BST workspace");
    }
    w.os = os;
    w.Pb = Pb;
    return BP_OK;
}

// Window of eq "w" on the ns = floor(n_det/2) + 1 half-line samples (FP64) and the joined
// rows of the windowed semi-polar form.
bp_status ensure_bst_window(bp_plan *p, float beta) {
    BstWork &w = p->bst;
    const int ns = p->n_det / 2 + 1, np = 2 * ns - 1;
    if (!w.wrows) {
        cudaError_t e = cudaMalloc(&w.wrows, sizeof(float) * (size_t)p->n_theta * np);
        if (e == cudaSuccess) e = cudaMalloc(&w.win, sizeof(float) * ns);
        if (e != cudaSuccess) {
            cudaFree(w.wrows);
            cudaFree(w.win);
            w.wrows = nullptr;
            w.win = nullptr;
            return cuda_fail(e, "windowed BST workspace");
        }
        w.bytes += sizeof(float) * ((size_t)p->n_theta * np + ns);
        w.beta = -1.f;
    }
    if (w.beta == beta) return BP_OK;
    std::vector<float> win(ns, 1.0f);
    const double b = beta, i0b = std::cyl_bessel_i(0.0, b);
    for (int i = 0; i < ns && ns > 1; ++i) {
        const double x = (2.0 * i - ns + 1.0) / (ns - 1.0);
        win[i] = (float)(std::cyl_bessel_i(0.0, b * std::sqrt(std::max(0.0, 1.0 - x * x))) / i0b);
    }
    BP_CUDA_TRY(cudaMemcpy(w.win, win.data(), sizeof(float) * ns, cudaMemcpyHostToDevice));
    w.beta = beta;
    return BP_OK;
}

}  // namespace

void free_bst(bp_plan *p) {
    BstWork &w = p->bst;
    cudaFree(w.wrows);
    cudaFree(w.win);
    cudaFree(w.polar);
    cudaFree(w.twPb);
    cudaFree(w.twPassH);
    cudaFree(w.ang);
    cudaFree(w.ray);
    cudaFree(w.ones);
    cudaFree(w.dir);
    cudaFree(w.igap);
    w = BstWork();
}

bp_status launch_bst(bp_plan *p, const void *sino, bp_dtype dt, float *img, int os, int batch, cudaStream_t st) {
    if ((size_t)p->P * os * sizeof(float2) * 3 / 2 > 200u * 1024u)
        return fail(BP_ERR_UNSUPPORTED, "BST: n_det x oversampling too large for the shared-memory FFT");
    bp_status s = ensure_bst(p, os);
    if (s == BP_OK) s = ensure_fourier(p);  // its grid may have been released (bp_set_fourier_width)
    if (s != BP_OK) return s;
    BstWork &w = p->bst;
    FourierWork &f = p->four;
    const int N = p->N, M = f.M, H = w.Pb / 2;
    const size_t esz = dt == BP_F32 ? 4 : 2;
    const double inv_rho = (double)w.Pb * p->dt / ((double)M * p->dx);
    const float ih = (float)inv_rho, il = (float)(inv_rho - (double)ih);
    const float scale = (float)(1.0 / (((double)M * p->dx) * ((double)M * p->dx)));
    const float delta2 = (N % 2 == 0) ? 1.0f / (float)M : 0.0f;  // 2 delta / M
    stage_begin(p, st);
    for (int b = 0; b < batch; ++b) {
        const char *sb = (const char *)sino + esz * (size_t)b * p->n_theta * p->n_det;
        switch (dt) {
            case BP_F32: s = polar_t(p, (const float *)sb, p->n_det, st); break;
            case BP_BF16: s = polar_t(p, (const __nv_bfloat16 *)sb, p->n_det, st); break;
            case BP_F16: s = polar_t(p, (const __half *)sb, p->n_det, st); break;
        }
        if (s != BP_OK) return s;
        const dim3 g((M + 31) / 32, (M + 7) / 8);
        bst_interp_kernel<<<g, 256, 0, st>>>(w.polar, w.ang, w.ray, w.dir, w.igap, w.ri, f.grid, M, H, ih, il, scale,
                                             delta2, p->n_theta);
        BP_CUDA_TRY(cudaGetLastError());
        stage_mark(p, st, "bst_interp_kernel");
        if ((s = launch_grid_to_image(p, w.ones, img + (size_t)b * N * N, st)) != BP_OK) return s;
    }
    return BP_OK;
}

bp_status launch_bst_windowed(bp_plan *p, const void *sino, bp_dtype dt, float *img, int os, float beta, int batch,
                              cudaStream_t st) {
    if ((size_t)p->P * os * sizeof(float2) * 3 / 2 > 200u * 1024u)
        return fail(BP_ERR_UNSUPPORTED, "BST: n_det x oversampling too large for the shared-memory FFT");
    bp_status s = ensure_bst(p, os);
    if (s == BP_OK) s = ensure_fourier(p);
    if (s == BP_OK) s = ensure_bst_window(p, beta);
    if (s != BP_OK) return s;
    BstWork &w = p->bst;
    FourierWork &f = p->four;
    const int N = p->N, M = f.M, H = w.Pb / 2;
    const int ns = p->n_det / 2 + 1, np = 2 * ns - 1;  // np <= n_det + 1 <= P
    const size_t esz = dt == BP_F32 ? 4 : 2;
    const double inv_rho = (double)w.Pb * p->dt / ((double)M * p->dx);
    const float ih = (float)inv_rho, il = (float)(inv_rho - (double)ih);
    const float scale = (float)(1.0 / (((double)M * p->dx) * ((double)M * p->dx)));
    const float delta2 = (N % 2 == 0) ? 1.0f / (float)M : 0.0f;
    const long long total = (long long)p->n_theta * np;
    const unsigned blocks = (unsigned)std::min<long long>((total + 255) / 256, 8LL * std::max(1, p->sm_count));
    stage_begin(p, st);
    for (int b = 0; b < batch; ++b) {
        const char *sb = (const char *)sino + esz * (size_t)b * p->n_theta * p->n_det;
        switch (dt) {
            case BP_F32:
                bst_window_rows_kernel<<<blocks, 256, 0, st>>>((const float *)sb, w.wrows, w.win, p->n_theta, p->n_det, ns);
                break;
            case BP_BF16:
                bst_window_rows_kernel<<<blocks, 256, 0, st>>>((const __nv_bfloat16 *)sb, w.wrows, w.win, p->n_theta,
                                                               p->n_det, ns);
                break;
            case BP_F16:
                bst_window_rows_kernel<<<blocks, 256, 0, st>>>((const __half *)sb, w.wrows, w.win, p->n_theta, p->n_det,
                                                               ns);
                break;
        }
        BP_CUDA_TRY(cudaGetLastError());
        stage_mark(p, st, "bst_window_rows_kernel");
        if ((s = polar_t(p, (const float *)w.wrows, np, st)) != BP_OK) return s;
        const dim3 g((M + 31) / 32, (M + 7) / 8);
        bst_interp_kernel<<<g, 256, 0, st>>>(w.polar, w.ang, w.ray, w.dir, w.igap, w.ri, f.grid, M, H, ih, il, scale,
                                             delta2, p->n_theta);
        BP_CUDA_TRY(cudaGetLastError());
        stage_mark(p, st, "bst_interp_kernel");
        if ((s = launch_grid_to_image(p, w.ones, img + (size_t)b * N * N, st)) != BP_OK) return s;
    }
    return BP_OK;
}

}  // namespace bp
