// Plan creation / destruction, FP64 host tables, error reporting and the host-buffer entry point.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

namespace bp {

static thread_local std::string g_last_error;
const char *last_error_cstr() { return g_last_error.c_str(); }

void set_error(const std::string &msg) { g_last_error = msg; }

bp_status fail(bp_status st, const std::string &msg) {
    set_error(msg);
    return st;
}

bp_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e));
    return (e == cudaErrorMemoryAllocation) ? BP_ERR_OOM : BP_ERR_CUDA;
}

bool aligned16(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

bp_status check_plan(const bp_plan *p) {
    if (!p) return fail(BP_ERR_INVALID_ARG, "plan is NULL");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device)
        return fail(BP_ERR_INVALID_ARG, "the current device differs from the plan's device");
    return BP_OK;
}

// Iterative radix-2 FFT in double precision (host tables only).  Sign -1 forward.
void host_fft(std::vector<double> &re, std::vector<double> &im, bool inverse) {
    const size_t n = re.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            std::swap(re[i], re[j]);
            std::swap(im[i], im[j]);
        }
    }
    const double sgn = inverse ? 1.0 : -1.0;
    for (size_t len = 2; len <= n; len <<= 1) {
        const size_t half = len >> 1;
        for (size_t k = 0; k < half; ++k) {
            const double ang = sgn * 2.0 * M_PI * (double)k / (double)len;
            const double wr = std::cos(ang), wi = std::sin(ang);
            for (size_t i = k; i < n; i += len) {
                const size_t j = i + half;
                const double xr = re[j] * wr - im[j] * wi;
                const double xi = re[j] * wi + im[j] * wr;
                re[j] = re[i] - xr;
                im[j] = im[i] - xi;
                re[i] += xr;
                im[i] += xi;
            }
        }
    }
}

// Quadrature weights of eq "bp_app" (Section 2) for an arbitrary angle set: sort mod pi,
// w_k = (next gap + previous gap) / 2 with period-pi wrap-around.
static void angle_weights(const std::vector<double> &theta, std::vector<double> &w) {
    const int n = (int)theta.size();
    w.assign(n, 0.0);
    if (n == 1) {
        w[0] = M_PI;
        return;
    }
    std::vector<std::pair<double, int>> s(n);
    for (int k = 0; k < n; ++k) {
        double a = std::fmod(theta[k], M_PI);
        if (a < 0) a += M_PI;
        s[k] = {a, k};
    }
    std::sort(s.begin(), s.end());
    for (int i = 0; i < n; ++i) {
        const double prev = (i == 0) ? s[n - 1].first - M_PI : s[i - 1].first;
        const double next = (i == n - 1) ? s[0].first + M_PI : s[i + 1].first;
        w[s[i].second] = 0.5 * (next - prev);
    }
}

static void timer_record(bp_plan *p, cudaStream_t st, const char *name) {
    StageTimer &t = p->timer;
    if (!t.on) return;
    if (t.used >= kStageTimerCap) {
        t.overflow = true;
        return;
    }
    if (t.used == (int)t.ev.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            t.overflow = true;
            return;
        }
        t.ev.push_back(e);
        t.name.push_back(nullptr);
    }
    if (cudaEventRecord(t.ev[t.used], st) != cudaSuccess) {
        t.overflow = true;
        return;
    }
    t.name[t.used++] = name;
}

void stage_begin(bp_plan *p, cudaStream_t st) { timer_record(p, st, nullptr); }
void stage_mark(bp_plan *p, cudaStream_t st, const char *name) { timer_record(p, st, name); }

static long long to_fix32(double v) { return (long long)std::llround(std::ldexp(v, 32)); }

}  // namespace bp


using namespace bp;

extern "C" const char *bp_last_error(void) { return last_error_cstr(); }

extern "C" const char *bp_version(void) { return "bp 0.1 sm_103a"; }

static void plan_free_device(bp_plan *p) {
    for (cudaEvent_t e : p->timer.ev) cudaEventDestroy(e);
    p->timer.ev.clear();
    cudaFree(p->d_ang);
    cudaFree(p->d_twP);
    cudaFree(p->d_twpass);
    for (auto &h : p->d_H) cudaFree(h);
    free_fourier(p);
    free_bst(p);
    free_logpolar(p);
    free_logpolar_partial(p);
    free_klein(p);
    cudaFree(p->d_stage);
    cudaFree(p->d_fbp);
    for (int k = 0; k < kHostSlots; ++k) {
        if (p->ev_h2d[k]) cudaEventDestroy(p->ev_h2d[k]);
        if (p->ev_comp[k]) cudaEventDestroy(p->ev_comp[k]);
        if (p->ev_d2h[k]) cudaEventDestroy(p->ev_d2h[k]);
    }
    if (p->s_h2d) cudaStreamDestroy(p->s_h2d);
    if (p->s_d2h) cudaStreamDestroy(p->s_d2h);
    cudaFree(p->d_desc);
    cudaFree(p->d_counter);
    cudaFree(p->d_status);
    cudaFree(p->d_err);
}

extern "C" bp_plan *bp_plan_create(int N, int n_det, int n_theta, const double *theta, double det_spacing) {
    set_error("");
    if (N < 1 || N > BP_MAX_N) { fail(BP_ERR_UNSUPPORTED, "N out of range [1, BP_MAX_N]"); return nullptr; }
    if (n_det < 1 || n_det > BP_MAX_NDET) { fail(BP_ERR_UNSUPPORTED, "n_det out of range [1, BP_MAX_NDET]"); return nullptr; }
    if (n_theta < 1 || n_theta > BP_MAX_NTHETA) { fail(BP_ERR_UNSUPPORTED, "n_theta out of range [1, BP_MAX_NTHETA]"); return nullptr; }
    if (!theta) { fail(BP_ERR_INVALID_ARG, "theta is NULL"); return nullptr; }
    if (!(det_spacing > 0.0) || !std::isfinite(det_spacing)) { fail(BP_ERR_INVALID_ARG, "det_spacing must be finite and > 0"); return nullptr; }
    for (int k = 0; k < n_theta; ++k)
        if (!std::isfinite(theta[k])) { fail(BP_ERR_INVALID_ARG, "theta contains a non-finite value"); return nullptr; }

    bp_plan *p = new (std::nothrow) bp_plan();
    if (!p) { fail(BP_ERR_OOM, "host allocation of the plan failed"); return nullptr; }
    p->N = N; p->n_det = n_det; p->n_theta = n_theta;
    p->dt = det_spacing; p->dx = 2.0 / N;
    if (cudaGetDevice(&p->device) != cudaSuccess) { fail(BP_ERR_CUDA, "cudaGetDevice failed"); delete p; return nullptr; }
    if (cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
        p->sm_count = 0;
    p->theta.assign(theta, theta + n_theta);
    angle_weights(p->theta, p->w);

    // Per-angle coordinate tables (eq "bp_app"): u(ix, iy) = c (ix - N/2 + 1/2) + s (iy - N/2 + 1/2) + (n_det-1)/2
    // with c = cos(theta) dx/dt and s = sin(theta) dx/dt.  Tile steps are kept exact in 32.32 fixed point.
    std::vector<AngleParam> ap(n_theta);
    const double r = p->dx / p->dt;
    double ext = 0.0;
    for (int k = 0; k < n_theta; ++k) {
        const double c = std::cos(theta[k]) * r, s = std::sin(theta[k]) * r;
        const double u00 = c * (0.5 - 0.5 * N) + s * (0.5 - 0.5 * N) + 0.5 * (n_det - 1);
        ap[k].U00 = to_fix32(u00);
        ap[k].CT = to_fix32(c * kTile);
        ap[k].ST = to_fix32(s * kTile);
        ap[k].c = (float)c;
        ap[k].s = (float)s;
        ap[k].w = (float)p->w[k];
        ap[k].pad = 0.f;
        ext = std::max(ext, std::fabs((double)ap[k].c) + std::fabs((double)ap[k].s));
        p->step_max = std::max(p->step_max, std::max(std::fabs(ap[k].c), std::fabs(ap[k].s)));
    }
    // Window: all bins touched by a kTile x kTile tile plus a rounding margin on each side.
    int W = (int)std::ceil((kTile - 1) * ext) + 4;
    W = (W + 3) & ~3;
    if ((double)W * kStage * 8.0 > 96.0 * 1024.0) {
        fail(BP_ERR_UNSUPPORTED, "dx/det_spacing too large: direct-kernel window exceeds shared memory");
        delete p;
        return nullptr;
    }
    p->W = W;
    p->C = W / 2;
    // Fixed-point range: |u| must stay well inside 2^31 bins.
    if (std::fabs(0.5 * (n_det - 1)) + 2.0 * N * r > 1.0e9) {
        fail(BP_ERR_UNSUPPORTED, "geometry out of fixed-point range");
        delete p;
        return nullptr;
    }
    p->P = 1 << ilog2(2 * n_det);
    klein_plan(p);

    cudaError_t e = cudaMalloc(&p->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_ang, sizeof(AngleParam) * n_theta);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_ang, ap.data(), sizeof(AngleParam) * n_theta, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        // filter twiddles exp(-2 pi i r / P), r < P/2, from FP64
        std::vector<float2> tw(p->P / 2);
        for (int i = 0; i < p->P / 2; ++i) {
            const double a = -2.0 * M_PI * (double)i / (double)p->P;
            tw[i] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        e = cudaMalloc(&p->d_twP, sizeof(float2) * tw.size());
        if (e == cudaSuccess) e = cudaMemcpy(p->d_twP, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && filter_pt_supported(p->P)) {
        std::vector<float2> tp;
        build_pass_twiddles(ilog2(p->P), tp);
        e = cudaMalloc(&p->d_twpass, sizeof(float2) * tp.size());
        if (e == cudaSuccess) e = cudaMemcpy(p->d_twpass, tp.data(), sizeof(float2) * tp.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cuda_fail(e, "bp_plan_create device tables");
        plan_free_device(p);
        delete p;
        return nullptr;
    }
    // Ram-Lak and Shepp-Logan responses (FP64 on the host, eq "fbp"), made here so that
    // bp_fbp_static only reads them (the Tikhonov response depends on lambda: made on use)
    for (int kind : {(int)BP_RAMLAK, (int)BP_SHEPP_LOGAN}) {
        if (ensure_filter(p, kind, 0.f) != BP_OK) {
            plan_free_device(p);
            delete p;
            return nullptr;
        }
    }
    return p;
}

extern "C" void bp_destroy(bp_plan *p) {
    if (!p) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    plan_free_device(p);
    if (cur >= 0 && cur != p->device) cudaSetDevice(cur);
    delete p;
}

static bp_status check_common(bp_plan *p, const void *a, const void *b, int batch) {
    bp_status st = check_plan(p);
    if (st != BP_OK) return st;
    if (!a || !b) return fail(BP_ERR_INVALID_ARG, "data pointer is NULL");
    if (!aligned16(a) || !aligned16(b)) return fail(BP_ERR_INVALID_ARG, "data pointers must be 16-byte aligned");
    if (batch < 1 || batch > 65535) return fail(BP_ERR_INVALID_ARG, "batch out of range [1, 65535]");
    return BP_OK;
}

static bool valid_dtype(bp_dtype d) { return d == BP_F32 || d == BP_BF16 || d == BP_F16; }

extern "C" bp_status bp_filter(bp_plan *p, const void *in, bp_dtype dtype, float *out, bp_filter_kind kind,
                               float param, int batch, void *stream) {
    set_error("");
    bp_status st = check_common(p, in, out, batch);
    if (st != BP_OK) return st;
    if (!valid_dtype(dtype)) return fail(BP_ERR_INVALID_ARG, "invalid dtype");
    if (kind != BP_RAMLAK && kind != BP_SHEPP_LOGAN && kind != BP_TIKHONOV)
        return fail(BP_ERR_INVALID_ARG, "invalid filter kind");
    if (kind == BP_TIKHONOV && !(param >= 0.f && std::isfinite(param)))
        return fail(BP_ERR_INVALID_ARG, "Tikhonov lambda must be finite and >= 0");
    if (dtype != BP_F32 && (const void *)out == in)
        return fail(BP_ERR_INVALID_ARG, "in-place filtering needs BP_F32 input");
    return launch_filter(p, in, dtype, out, (int)kind, param, batch, (cudaStream_t)stream);
}

extern "C" bp_status bp_backproject_direct(bp_plan *p, const void *sino, bp_dtype dtype, float *img, int batch,
                                           int accumulate, void *stream) {
    set_error("");
    bp_status st = check_common(p, sino, img, batch);
    if (st != BP_OK) return st;
    if (!valid_dtype(dtype)) return fail(BP_ERR_INVALID_ARG, "invalid dtype");
    return launch_direct(p, sino, dtype, img, batch, accumulate ? 1 : 0, (cudaStream_t)stream);
}

extern "C" bp_status bp_backproject_fourier(bp_plan *p, const void *sino, bp_dtype dtype, float *img, int batch,
                                            void *stream) {
    set_error("");
    bp_status st = check_common(p, sino, img, batch);
    if (st != BP_OK) return st;
    if (!valid_dtype(dtype)) return fail(BP_ERR_INVALID_ARG, "invalid dtype");
    return launch_fourier(p, sino, dtype, img, batch, (cudaStream_t)stream);
}

extern "C" bp_status bp_fbp_fourier(bp_plan *p, const void *sino, bp_dtype dtype, float *img, bp_filter_kind kind,
                                    float param, int batch, void *stream) {
    set_error("");
    bp_status st = check_common(p, sino, img, batch);
    if (st != BP_OK) return st;
    if (!valid_dtype(dtype)) return fail(BP_ERR_INVALID_ARG, "invalid dtype");
    if (kind != BP_RAMLAK && kind != BP_SHEPP_LOGAN && kind != BP_TIKHONOV)
        return fail(BP_ERR_INVALID_ARG, "invalid filter kind");
    if (kind == BP_TIKHONOV && !(param >= 0.f && std::isfinite(param)))
        return fail(BP_ERR_INVALID_ARG, "Tikhonov lambda must be finite and >= 0");
    return launch_fourier(p, sino, dtype, img, batch, (cudaStream_t)stream, 0.f, (int)kind, param);
}

extern "C" bp_status bp_fbp_direct(bp_plan *p, const void *sino, bp_dtype dtype, float *img, bp_filter_kind kind,
                                   float param, int batch, void *stream) {
    set_error("");
    bp_status st = check_common(p, sino, img, batch);
    if (st != BP_OK) return st;
    if (!valid_dtype(dtype)) return fail(BP_ERR_INVALID_ARG, "invalid dtype");
    if (kind != BP_RAMLAK && kind != BP_SHEPP_LOGAN && kind != BP_TIKHONOV)
        return fail(BP_ERR_INVALID_ARG, "invalid filter kind");
    if (kind == BP_TIKHONOV && !(param >= 0.f && std::isfinite(param)))
        return fail(BP_ERR_INVALID_ARG, "Tikhonov lambda must be finite and >= 0");
    return launch_fbp_direct(p, sino, dtype, img, (int)kind, param, batch, (cudaStream_t)stream);
}

extern "C" bp_status bp_backproject_bst(bp_plan *p, const void *sino, bp_dtype dtype, float *img,
                                        int radial_oversampling, int batch, void *stream) {
    set_error("");
    bp_status st = check_common(p, sino, img, batch);
    if (st != BP_OK) return st;
    if (!valid_dtype(dtype)) return fail(BP_ERR_INVALID_ARG, "invalid dtype");
    const int os = radial_oversampling;
    if (os != 1 && os != 2 && os != 4 && os != 8)
        return fail(BP_ERR_INVALID_ARG, "radial_oversampling must be 1, 2, 4 or 8");
    return launch_bst(p, sino, dtype, img, os, batch, (cudaStream_t)stream);
}

extern "C" bp_status bp_backproject_bst_windowed(bp_plan *p, const void *sino, bp_dtype dtype, float *img,
                                                 int radial_oversampling, float beta, int batch, void *stream) {
    set_error("");
    bp_status st = check_common(p, sino, img, batch);
    if (st != BP_OK) return st;
    if (!valid_dtype(dtype)) return fail(BP_ERR_INVALID_ARG, "invalid dtype");
    const int os = radial_oversampling;
    if (os != 1 && os != 2 && os != 4 && os != 8)
        return fail(BP_ERR_INVALID_ARG, "radial_oversampling must be 1, 2, 4 or 8");
    if (!(beta >= 0.f) || !std::isfinite(beta)) return fail(BP_ERR_INVALID_ARG, "beta must be finite and >= 0");
    return launch_bst_windowed(p, sino, dtype, img, os, beta, batch, (cudaStream_t)stream);
}

extern "C" bp_status bp_backproject_logpolar(bp_plan *p, const void *sino, bp_dtype dtype, float *img, int batch,
                                             void *stream) {
    set_error("");
    bp_status st = check_common(p, sino, img, batch);
    if (st != BP_OK) return st;
    if (!valid_dtype(dtype)) return fail(BP_ERR_INVALID_ARG, "invalid dtype");
    return launch_logpolar(p, sino, dtype, img, batch, (cudaStream_t)stream);
}

extern "C" bp_status bp_backproject_logpolar_partial(bp_plan *p, const void *sino, bp_dtype dtype, float *img,
                                                     int sectors, float a_r, int batch, void *stream) {
    set_error("");
    bp_status st = check_common(p, sino, img, batch);
    if (st != BP_OK) return st;
    if (!valid_dtype(dtype)) return fail(BP_ERR_INVALID_ARG, "invalid dtype");
    if (sectors < 1 || (sectors & (sectors - 1))) return fail(BP_ERR_INVALID_ARG, "sectors must be a power of two");
    if (!(a_r > 0.f && a_r < 0.5f)) return fail(BP_ERR_INVALID_ARG, "a_r must lie in (0, 1/2)");
    return launch_logpolar_partial(p, sino, dtype, img, batch, sectors, a_r, (cudaStream_t)stream);
}

extern "C" bp_status bp_set_direct_workspace(bp_plan *p, unsigned long long bytes) {
    set_error("");
    bp_status st = check_plan(p);
    if (st != BP_OK) return st;
    return klein_set_workspace(p, (size_t)bytes);
}

extern "C" bp_status bp_set_fourier_width(bp_plan *p, int width) {
    set_error("");
    bp_status st = check_plan(p);
    if (st != BP_OK) return st;
    if (width != 4 && width != 6) return fail(BP_ERR_INVALID_ARG, "Fourier kernel width must be 4 or 6");
    if (width == p->fourier_W) return BP_OK;
    BP_CUDA_TRY(cudaDeviceSynchronize());  // no call of this plan may still use the workspace
    free_fourier(p);
    p->fourier_W = width;
    return BP_OK;
}

extern "C" bp_status bp_radon(bp_plan *p, const float *img, float *sino, int batch, int fourier_adjoint,
                              void *stream) {
    set_error("");
    bp_status st = check_common(p, img, sino, batch);
    if (st != BP_OK) return st;
    if ((const void *)img == (const void *)sino) return fail(BP_ERR_INVALID_ARG, "img and sino must not alias");
    if (fourier_adjoint) return launch_radon_fourier(p, img, sino, batch, (cudaStream_t)stream);
    return launch_radon_direct(p, img, sino, batch, (cudaStream_t)stream);
}

// Slices go through a ring of kHostSlots device slots: slice i's sinogram is copied in on
// s_h2d, filtered and backprojected on the caller's stream, and its image copied out on s_d2h,
// so that the copies of slices i + 1 and i - 1 overlap the kernels of slice i.  Events order
// the reuse of a slot: its next copy-in waits for its kernels, its next kernels for its
// copy-out.
extern "C" bp_status bp_fbp_host(bp_plan *p, const float *sino, float *img, bp_filter_kind kind, float param,
                                 int batch, void *stream) {
    set_error("");
    bp_status st = check_plan(p);
    if (st != BP_OK) return st;
    if (!sino || !img) return fail(BP_ERR_INVALID_ARG, "host pointer is NULL");
    if (batch < 1 || batch > 65535) return fail(BP_ERR_INVALID_ARG, "batch out of range [1, 65535]");
    // everything the per-slice calls check is checked here, before any copy is queued
    if (kind != BP_RAMLAK && kind != BP_SHEPP_LOGAN && kind != BP_TIKHONOV)
        return fail(BP_ERR_INVALID_ARG, "invalid filter kind");
    if (kind == BP_TIKHONOV && !(param >= 0.f && std::isfinite(param)))
        return fail(BP_ERR_INVALID_ARG, "Tikhonov lambda must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t sino_n = (size_t)p->n_theta * p->n_det, img_n = (size_t)p->N * p->N;
    const size_t sino_pad = (sino_n + 3) & ~(size_t)3, img_pad = (img_n + 3) & ~(size_t)3;
    const int S = std::min(batch, kHostSlots);
    if ((size_t)S > p->stage_batch) {
        BP_CUDA_TRY(cudaStreamSynchronize(s));
        cudaFree(p->d_stage);
        p->d_stage = nullptr;
        p->stage_batch = 0;
        BP_CUDA_TRY(cudaMalloc(&p->d_stage, sizeof(float) * (sino_pad + img_pad) * S));
        p->stage_batch = (size_t)S;
    }
    if (!p->s_h2d) {
        BP_CUDA_TRY(cudaStreamCreateWithFlags(&p->s_h2d, cudaStreamNonBlocking));
        BP_CUDA_TRY(cudaStreamCreateWithFlags(&p->s_d2h, cudaStreamNonBlocking));
        for (int k = 0; k < kHostSlots; ++k) {
            BP_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_h2d[k], cudaEventDisableTiming));
            BP_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_comp[k], cudaEventDisableTiming));
            BP_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_d2h[k], cudaEventDisableTiming));
        }
    }
    // on a failure the copies already queued still read or write the caller's buffers: drain
    // the streams before returning, so that the caller may release them
    auto drain = [&](bp_status fst) {
        cudaStreamSynchronize(p->s_h2d);
        cudaStreamSynchronize(p->s_d2h);
        cudaStreamSynchronize(s);
        return fst;
    };
#define BP_HOST_TRY(expr)                                                  \
    do {                                                                   \
        cudaError_t _e = (expr);                                           \
        if (_e != cudaSuccess) return drain(cuda_fail(_e, #expr));         \
    } while (0)
    for (int i = 0; i < batch; ++i) {
        const int k = i % S;
        float *d_sino = p->d_stage + (sino_pad + img_pad) * k;
        float *d_img = d_sino + sino_pad;
        if (i >= S) BP_HOST_TRY(cudaStreamWaitEvent(p->s_h2d, p->ev_comp[k], 0));
        BP_HOST_TRY(cudaMemcpyAsync(d_sino, sino + sino_n * i, sizeof(float) * sino_n, cudaMemcpyHostToDevice,
                                    p->s_h2d));
        BP_HOST_TRY(cudaEventRecord(p->ev_h2d[k], p->s_h2d));
        BP_HOST_TRY(cudaStreamWaitEvent(s, p->ev_h2d[k], 0));
        if (i >= S) BP_HOST_TRY(cudaStreamWaitEvent(s, p->ev_d2h[k], 0));
        st = bp_fbp_direct(p, d_sino, BP_F32, d_img, kind, param, 1, stream);
        if (st != BP_OK) return drain(st);
        BP_HOST_TRY(cudaEventRecord(p->ev_comp[k], s));
        BP_HOST_TRY(cudaStreamWaitEvent(p->s_d2h, p->ev_comp[k], 0));
        BP_HOST_TRY(cudaMemcpyAsync(img + img_n * i, d_img, sizeof(float) * img_n, cudaMemcpyDeviceToHost, p->s_d2h));
        BP_HOST_TRY(cudaEventRecord(p->ev_d2h[k], p->s_d2h));
    }
#undef BP_HOST_TRY
    BP_CUDA_TRY(cudaStreamSynchronize(p->s_d2h));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    return BP_OK;
}

extern "C" bp_status bp_backproject_batched(bp_plan *const *plans, const void *const *sinos, const bp_dtype *dtypes,
                                            float *const *imgs, int n, void *stream) {
    set_error("");
    if (!plans || !sinos || !dtypes || !imgs) return fail(BP_ERR_INVALID_ARG, "NULL array argument");
    if (n < 1) return fail(BP_ERR_INVALID_ARG, "n must be >= 1");
    for (int i = 0; i < n; ++i) {
        bp_status st = check_common(plans[i], sinos[i], imgs[i], 1);
        if (st != BP_OK) return st;
        if (!valid_dtype(dtypes[i])) return fail(BP_ERR_INVALID_ARG, "invalid dtype");
        if (plans[i]->device != plans[0]->device) return fail(BP_ERR_INVALID_ARG, "plans on different devices");
    }
    return launch_batched(plans, sinos, dtypes, imgs, n, (cudaStream_t)stream);
}

extern "C" bp_status bp_check(bp_plan *p, void *stream) {
    set_error("");
    bp_status st = check_plan(p);
    if (st != BP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    BP_CUDA_TRY(cudaMemcpyAsync(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BP_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) {
        BP_CUDA_TRY(cudaMemset(p->d_err, 0, sizeof(int)));
        return fail(BP_ERR_TIMEOUT, "a device-side bounded wait gave up (results of the affected call are invalid)");
    }
    return BP_OK;
}

extern "C" bp_status bp_radon_transpose(bp_plan *p, const float *sino, float *img, int batch, int fourier,
                                        void *stream) {
    set_error("");
    bp_status st = check_common(p, sino, img, batch);
    if (st != BP_OK) return st;
    if ((const void *)img == (const void *)sino) return fail(BP_ERR_INVALID_ARG, "img and sino must not alias");
    // R = (dx^2/dt) diag(1/w) A^T  =>  R^T = (dx^2/dt) A diag(1/w): R* with every weight dx^2/dt
    const float wu = (float)(p->dx * p->dx / p->dt);
    if (fourier) return launch_fourier(p, sino, BP_F32, img, batch, (cudaStream_t)stream, wu);
    return launch_direct(p, sino, BP_F32, img, batch, 0, (cudaStream_t)stream, wu);
}

extern "C" bp_status bp_backproject_transpose(bp_plan *p, const float *img, float *sino, int batch, int fourier,
                                              void *stream) {
    set_error("");
    bp_status st = check_common(p, img, sino, batch);
    if (st != BP_OK) return st;
    if ((const void *)img == (const void *)sino) return fail(BP_ERR_INVALID_ARG, "img and sino must not alias");
    // A^T = (dt/dx^2) diag(w) R: R with angle k scaled by w_k instead of dx^2/dt
    if (fourier) return launch_radon_fourier(p, img, sino, batch, (cudaStream_t)stream, 1);
    return launch_radon_direct(p, img, sino, batch, (cudaStream_t)stream, 1);
}

extern "C" bp_status bp_stage_timing(bp_plan *p, int on) {
    set_error("");
    bp_status st = check_plan(p);
    if (st != BP_OK) return st;
    p->timer.on = on != 0;
    p->timer.used = 0;
    p->timer.overflow = false;
    return BP_OK;
}

extern "C" bp_status bp_stage_times(bp_plan *p, int cap, const char **names, float *ms, int *launches, int *count) {
    set_error("");
    bp_status st = check_plan(p);
    if (st != BP_OK) return st;
    if (!count || (cap > 0 && (!names || !ms || !launches)) || cap < 0)
        return fail(BP_ERR_INVALID_ARG, "bp_stage_times: NULL output or negative capacity");
    StageTimer &t = p->timer;
    if (t.overflow) {
        t.used = 0;
        t.overflow = false;
        return fail(BP_ERR_UNSUPPORTED, "bp_stage_times: more launches than the timer records; read it more often");
    }
    struct Agg {
        const char *name;
        double ms;
        int launches;
    };
    std::vector<Agg> agg;
    if (t.used > 0) BP_CUDA_TRY(cudaEventSynchronize(t.ev[t.used - 1]));
    for (int i = 1; i < t.used; ++i) {
        if (!t.name[i]) continue;
        float dt_ms = 0.f;
        BP_CUDA_TRY(cudaEventElapsedTime(&dt_ms, t.ev[i - 1], t.ev[i]));
        size_t j = 0;
        while (j < agg.size() && std::strcmp(agg[j].name, t.name[i]) != 0) ++j;
        if (j == agg.size()) agg.push_back({t.name[i], 0.0, 0});
        agg[j].ms += dt_ms;
        agg[j].launches += 1;
    }
    const int n = (int)agg.size();
    for (int j = 0; j < n && j < cap; ++j) {
        names[j] = agg[j].name;
        ms[j] = (float)agg[j].ms;
        launches[j] = agg[j].launches;
    }
    t.used = 0;
    *count = n;
    return BP_OK;
}
