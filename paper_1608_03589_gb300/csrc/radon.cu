// Forward Radon transform R as the exact scaled transpose of the direct R* (Section 1,
// eqs "P_theta" and "adjoint"):
//     (R f)_{kj} = (dx^2 / dt) * sum_p hat(u_pk - j) f_p,
// i.e. every pixel deposits (1 - f) f_p into bin floor(u) and f f_p into bin floor(u) + 1.
//
// Design: the same 64 x 64 tile / 16-angle stage decomposition and the same fixed-point
// tile coordinates as the direct R* kernel.  Each CTA holds its tile's pixel values in
// registers, deposits into a per-(tile, angle) shared-memory window with shared atomics,
// and adds each window to the sinogram with one global reduction per touched bin.
#include "common.cuh"

namespace bp {

namespace {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagicInt = 0x4B400000;

__global__ void __launch_bounds__(kThreads)
radon_direct_kernel(const float *__restrict__ img, float *__restrict__ sino, const AngleParam *__restrict__ ap,
                    int N, int n_det, int n_theta, int W, int C, float scale,
                    long long img_stride, long long sino_stride) {
    extern __shared__ __align__(16) float win[];  // [kStage][W]
    __shared__ float4 sp[kStage];                 // q0, c, s, -
    __shared__ int sJ0[kStage];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int lx = lane & 7;
    const int ly = warp * 8 + (lane >> 3);
    const int tx = blockIdx.x, ty = blockIdx.y;
    img += (long long)blockIdx.z * img_stride;
    sino += (long long)blockIdx.z * sino_stride;

    float f[2][8];
    bool any = false;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int y = ty * kTile + ly + 4 * b;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int x = tx * kTile + lx + 8 * a;
            f[b][a] = (x < N && y < N) ? __ldg(img + (long long)y * N + x) : 0.f;
            any |= (f[b][a] != 0.f);
        }
    }
    // A tile of zeros contributes nothing.
    if (!__syncthreads_or(any)) return;

    const float fx = (float)lx, fy = (float)ly;
    for (int k0 = 0; k0 < n_theta; k0 += kStage) {
        const int kn = min(kStage, n_theta - k0);
        for (int i = tid; i < kStage * W; i += kThreads) win[i] = 0.f;
        if (tid < kn) {
            const AngleParam p = ap[k0 + tid];
            const long long U = p.U00 + (long long)tx * p.CT + (long long)ty * p.ST;
            const int Ji = (int)(U >> 32);
            const float frac = (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f;
            const float emin = (float)(kTile - 1) * (fminf(p.c, 0.f) + fminf(p.s, 0.f));
            const int J0 = Ji + (int)floorf(emin) - 1;
            sJ0[tid] = J0;
            sp[tid] = make_float4((float)(Ji - J0 - C) + (frac - 0.5f), p.c, p.s, 0.f);
        }
        __syncthreads();
        for (int kk = 0; kk < kn; ++kk) {
            const float4 P = sp[kk];
            const float qt = fmaf(fy, P.z, fmaf(fx, P.y, P.x));
            float *wk = win + kk * W + C;
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float qb = fmaf(4.f * b, P.z, qt);
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const float v = f[b][a];
                    if (v != 0.f) {
                        const float q = fmaf(8.f * a, P.y, qb);
                        const float r = q + kMagic;
                        const int m = __float_as_int(r) - kMagicInt;  // rint(q): bin offset from the window centre
                        const float fr = (q - (r - kMagic)) + 0.5f;   // u - floor(u)
                        atomicAdd(wk + m, v - fr * v);
                        atomicAdd(wk + m + 1, fr * v);
                    }
                }
            }
        }
        __syncthreads();
        for (int i = tid; i < kn * W; i += kThreads) {
            const int kk = i / W, m = i - kk * W;
            const float v = win[i];
            const int j = sJ0[kk] + m;
            if (v != 0.f && j >= 0 && j < n_det) atomicAdd(sino + (long long)(k0 + kk) * n_det + j, scale * v);
        }
        __syncthreads();
    }
}

}  // namespace

bp_status launch_radon_direct(bp_plan *p, const float *img, float *sino, int batch, cudaStream_t st) {
    const size_t sino_n = (size_t)p->n_theta * p->n_det;
    BP_CUDA_TRY(cudaMemsetAsync(sino, 0, sizeof(float) * sino_n * batch, st));
    const int tiles = (p->N + kTile - 1) / kTile;
    const size_t smem = sizeof(float) * (size_t)kStage * p->W;
    BP_CUDA_TRY(cudaFuncSetAttribute(radon_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const float scale = (float)(p->dx * p->dx / p->dt);
    dim3 grid(tiles, tiles, batch);
    radon_direct_kernel<<<grid, kThreads, smem, st>>>(img, sino, p->d_ang, p->N, p->n_det, p->n_theta, p->W, p->C,
                                                      scale, (long long)p->N * p->N, (long long)sino_n);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

}  // namespace bp
