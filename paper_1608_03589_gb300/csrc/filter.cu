// FBP row filter (Section 3, Remark 1 (ii), eq "fbp"; Section 6 for the Tikhonov filter).
//
// q_j = dt * sum_{i<n_det} h(j - i) g_i  (linear convolution with the band-limited spatial
// kernel h of the filter's frequency response) computed as a circular convolution of
// length P >= 2 n_det - 1:  q = IFFT( FFT(g zero-padded) * H ),  H = (dt/P) DFT_P(h_circ),
// h_circ[r] = h(r) for r < n_det, h_circ[P - r] = h(-r).  H is real and even, so two real
// rows travel together as one complex row (a + i b): the real and imaginary parts of the
// result are the two filtered rows.  One CTA per row pair, the whole P-point transform in
// shared memory (register-blocked Stockham passes, natural order throughout).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "fft.cuh"
#include "fft_pt.cuh"
#include "filter_pt.cuh"

namespace bp {

namespace {

template <typename Tin, int E>
__global__ void __launch_bounds__(1024, 1)
filter_kernel(const Tin *__restrict__ in, float *__restrict__ out, const float *__restrict__ H,
              const float2 *__restrict__ tw, long long rows, int n_det, int logP) {
    extern __shared__ __align__(16) float2 z[];
    const int P = 1 << logP;
    float2 *tws = z + P;  // P/2 twiddles
    stage_twiddles(tws, tw, P / 2);
    const long long r0 = 2 * (long long)blockIdx.x, r1 = r0 + 1;
    const bool has1 = r1 < rows;
    const Tin *a = in + r0 * n_det;
    const Tin *b = in + r1 * n_det;
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
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        const float h = __ldg(H + j);
        const float2 v = z[j];
        z[j] = make_float2(v.x * h, v.y * h);
    }
    __syncthreads();
    stockham_fft<E>(z, logP, tws, 1, true, threadIdx.x, blockDim.x);
    float *oa = out + r0 * n_det;
    float *ob = out + r1 * n_det;
    for (int j = threadIdx.x; j < n_det; j += blockDim.x) {
        const float2 v = z[j];
        oa[j] = v.x;
        if (has1) ob[j] = v.y;
    }
}

// Transform lengths P = 2^9 .. 2^12 (n_det <= 2048) take the persistent kernel of filter_pt.cuh
// instead, its filtered rows written straight from registers.
struct RowsOut {
    static constexpr bool kStaged = false;
    float *out;
    __device__ __forceinline__ void put(long long r0, bool has1, int n_det, int i, float2 v) const {
        float *oa = out + r0 * n_det;
        oa[i] = v.x;
        if (has1) oa[n_det + i] = v.y;
    }
};

template <typename Tin, int LOGP>
__global__ void __launch_bounds__((1 << LOGP) / kPassE, 1024 / ((1 << LOGP) / kPassE))
filter_pt_kernel(const Tin *__restrict__ in, float *__restrict__ out, const float *__restrict__ H,
                 const float2 *__restrict__ twp, long long rows, int n_det) {
    filter_pt_body<Tin, LOGP>(in, RowsOut{out}, H, twp, rows, n_det);
}

// Spatial taps h(n), |n| < n_det, of the three filters (host, FP64).
void filter_taps(int kind, double dt, double lam, int n_det, std::vector<double> &h /* index n + n_det - 1 */) {
    h.assign(2 * n_det - 1, 0.0);
    if (kind == BP_RAMLAK) {
        for (int n = -(n_det - 1); n <= n_det - 1; ++n) {
            double v = 0.0;
            if (n == 0) v = 1.0 / (4.0 * dt * dt);
            else if (n & 1) v = -1.0 / (M_PI * M_PI * (double)n * (double)n * dt * dt);
            h[n + n_det - 1] = v;
        }
    } else if (kind == BP_SHEPP_LOGAN) {
        for (int n = -(n_det - 1); n <= n_det - 1; ++n)
            h[n + n_det - 1] = -2.0 / (M_PI * M_PI * dt * dt * (4.0 * (double)n * (double)n - 1.0));
    } else {
        // h(n) = 2 int_0^{W} nu/(1 + lam nu) cos(2 pi nu n dt) d nu, W = 1/(2 dt), by composite
        // Simpson on 2^16 panels.  With nu_i = i W / M the cosine is cos(pi i n / M), so all taps
        // are one DCT-I of the weighted samples, evaluated with a 2M-point FFT.
        const int M = 1 << 16;
        const double Wn = 0.5 / dt, hs = Wn / M;
        std::vector<double> re(2 * M, 0.0), im(2 * M, 0.0), a(M + 1);
        for (int i = 0; i <= M; ++i) {
            const double nu = i * hs;
            const double c = (i == 0 || i == M) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
            a[i] = c * nu / (1.0 + lam * nu);
        }
        for (int i = 0; i <= M; ++i) re[i] = a[i];
        for (int i = 1; i < M; ++i) re[2 * M - i] = a[i];
        host_fft(re, im, false);
        for (int n = -(n_det - 1); n <= n_det - 1; ++n) {
            const int an = n < 0 ? -n : n;
            const double sgn = (an & 1) ? -1.0 : 1.0;
            const double s = 0.5 * (re[an] + a[0] + sgn * a[M]);
            h[n + n_det - 1] = 2.0 * s * hs / 3.0;
        }
    }
}

}  // namespace

// Per-pass twiddle table of filter_pt_kernel for P = 2^logP (FP64 -> float):
// for each pass with L > 1, T[(r - 1) L + k] = exp(-2 pi i r k / (L R)).
void build_pass_twiddles(int logP, std::vector<float2> &T) {
    T.clear();
    int L = 1, rem = logP;
    while (rem > 0) {
        const int R = rem >= 3 ? 8 : (1 << rem);
        rem -= rem >= 3 ? 3 : rem;
        if (L > 1)
            for (int r = 1; r < R; ++r)
                for (int k = 0; k < L; ++k) {
                    const double a = -2.0 * M_PI * (double)r * (double)k / ((double)L * R);
                    T.push_back(make_float2((float)std::cos(a), (float)std::sin(a)));
                }
        L *= R;
    }
}

bool filter_pt_supported(int P) { return P >= 512 && P <= 4096; }

bp_status ensure_filter(bp_plan *p, int kind, float param) {
    if (p->d_H[kind] && (kind != BP_TIKHONOV || p->H_param[kind] == param)) return BP_OK;
    const int P = p->P, n = p->n_det, logP = ilog2(P);
    std::vector<double> h;
    filter_taps(kind, p->dt, (double)param, n, h);
    std::vector<double> re(P, 0.0), im(P, 0.0);
    for (int r = 0; r < n; ++r) re[r] = h[r + n - 1];
    for (int r = 1; r < n; ++r) re[P - r] = h[-r + n - 1];
    host_fft(re, im, false);
    std::vector<float> H(P);
    const double scale = p->dt / P;
    for (int i = 0; i < P; ++i) H[i] = (float)(re[i] * scale);
    (void)logP;
    if (!p->d_H[kind]) BP_CUDA_TRY(cudaMalloc(&p->d_H[kind], sizeof(float) * P));
    BP_CUDA_TRY(cudaMemcpy(p->d_H[kind], H.data(), sizeof(float) * P, cudaMemcpyHostToDevice));
    p->H_param[kind] = param;
    return BP_OK;
}

namespace {

template <typename Tin, int LOGP>
bp_status launch_pt(bp_plan *p, const Tin *in, float *out, const float *H, long long rows, cudaStream_t st) {
    constexpr int P = 1 << LOGP, NT = P / kPassE;
    constexpr size_t smem = filter_pt_smem<LOGP>();
    auto kern = filter_pt_kernel<Tin, LOGP>;
    BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    const long long npairs = (rows + 1) / 2;
    const long long grid = std::max(1LL, std::min(npairs, (long long)std::max(1, per_sm) * std::max(1, p->sm_count)));
    kern<<<(unsigned)grid, NT, smem, st>>>(in, out, H, p->d_twpass, rows, p->n_det);
    BP_CUDA_TRY(cudaGetLastError());
    stage_mark(p, st, "filter_pt_kernel");
    return BP_OK;
}

template <typename Tin>
bp_status launch_pt_t(bp_plan *p, const Tin *in, float *out, const float *H, long long rows, cudaStream_t st) {
    switch (ilog2(p->P)) {
        case 9: return launch_pt<Tin, 9>(p, in, out, H, rows, st);
        case 10: return launch_pt<Tin, 10>(p, in, out, H, rows, st);
        case 11: return launch_pt<Tin, 11>(p, in, out, H, rows, st);
        default: return launch_pt<Tin, 12>(p, in, out, H, rows, st);
    }
}

bp_status launch_pt_any(bp_plan *p, const void *in, bp_dtype dt, float *out, const float *H, long long rows,
                        cudaStream_t st) {
    if (!aligned16(H) || !aligned16(p->d_twpass)) return fail(BP_ERR_INVALID_ARG, "filter response not 16-byte aligned");
    switch (dt) {
        case BP_F32: return launch_pt_t(p, (const float *)in, out, H, rows, st);
        case BP_BF16: return launch_pt_t(p, (const __nv_bfloat16 *)in, out, H, rows, st);
        case BP_F16: return launch_pt_t(p, (const __half *)in, out, H, rows, st);
    }
    return fail(BP_ERR_INVALID_ARG, "invalid dtype");
}

}  // namespace

bp_status launch_filter(bp_plan *p, const void *in, bp_dtype dt, float *out, int kind, float param, int batch,
                        cudaStream_t st) {
    if ((size_t)(p->P + p->P / 2) * sizeof(float2) > 200u * 1024u)
        return fail(BP_ERR_UNSUPPORTED, "filter: n_det too large for the shared-memory FFT (n_det <= 8192)");
    bp_status s = ensure_filter(p, kind, param);
    if (s != BP_OK) return s;
    stage_begin(p, st);
    const long long rows = (long long)batch * p->n_theta;
    if (p->d_twpass) return launch_pt_any(p, in, dt, out, p->d_H[kind], rows, st);
    const int logP = ilog2(p->P);
    const int threads = fft_threads(p->P);
    const size_t smem = sizeof(float2) * (p->P + p->P / 2);
    const unsigned blocks = (unsigned)((rows + 1) / 2);
#define BP_FILTER_LAUNCH(T)                                                                               \
    do {                                                                                                  \
        if (fft_elems(p->P) == 16) {                                                                      \
            BP_CUDA_TRY(cudaFuncSetAttribute(filter_kernel<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)smem));                                                 \
            filter_kernel<T, 16><<<blocks, threads, smem, st>>>((const T *)in, out, p->d_H[kind], p->d_twP, \
                                                                rows, p->n_det, logP);                    \
        } else {                                                                                          \
            BP_CUDA_TRY(cudaFuncSetAttribute(filter_kernel<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)smem));                                                 \
            filter_kernel<T, 8><<<blocks, threads, smem, st>>>((const T *)in, out, p->d_H[kind], p->d_twP,  \
                                                               rows, p->n_det, logP);                     \
        }                                                                                                 \
    } while (0)
    switch (dt) {
        case BP_F32: BP_FILTER_LAUNCH(float); break;
        case BP_BF16: BP_FILTER_LAUNCH(__nv_bfloat16); break;
        case BP_F16: BP_FILTER_LAUNCH(__half); break;
    }
#undef BP_FILTER_LAUNCH
    BP_CUDA_TRY(cudaGetLastError());
    stage_mark(p, st, "filter_kernel");
    return BP_OK;
}

// Row filter with a caller-supplied response (P floats, natural order, already scaled by dt/P).
bp_status launch_filter_response(bp_plan *p, const void *in, bp_dtype dt, float *out, const float *H, int batch,
                                 cudaStream_t st) {
    if ((size_t)(p->P + p->P / 2) * sizeof(float2) > 200u * 1024u)
        return fail(BP_ERR_UNSUPPORTED, "filter: n_det too large for the shared-memory FFT (n_det <= 8192)");
    stage_begin(p, st);
    const long long rows = (long long)batch * p->n_theta;
    if (p->d_twpass) return launch_pt_any(p, in, dt, out, H, rows, st);
    const int logP = ilog2(p->P);
    const int threads = fft_threads(p->P);
    const size_t smem = sizeof(float2) * (p->P + p->P / 2);
    const unsigned blocks = (unsigned)((rows + 1) / 2);
#define BP_FILTER_LAUNCH_H(T)                                                                             \
    do {                                                                                                  \
        if (fft_elems(p->P) == 16) {                                                                      \
            BP_CUDA_TRY(cudaFuncSetAttribute(filter_kernel<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)smem));                                                 \
            filter_kernel<T, 16><<<blocks, threads, smem, st>>>((const T *)in, out, H, p->d_twP, rows,     \
                                                                p->n_det, logP);                          \
        } else {                                                                                          \
            BP_CUDA_TRY(cudaFuncSetAttribute(filter_kernel<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                             (int)smem));                                                 \
            filter_kernel<T, 8><<<blocks, threads, smem, st>>>((const T *)in, out, H, p->d_twP, rows,      \
                                                               p->n_det, logP);                           \
        }                                                                                                 \
    } while (0)
    switch (dt) {
        case BP_F32: BP_FILTER_LAUNCH_H(float); break;
        case BP_BF16: BP_FILTER_LAUNCH_H(__nv_bfloat16); break;
        case BP_F16: BP_FILTER_LAUNCH_H(__half); break;
    }
#undef BP_FILTER_LAUNCH_H
    BP_CUDA_TRY(cudaGetLastError());
    stage_mark(p, st, "filter_kernel");
    return BP_OK;
}

}  // namespace bp
