// Forward Radon transform R as the exact scaled transpose of the direct R* (Section 1,
// eqs "P_theta" and "adjoint"):
//     (R f)_{kj} = (dx^2 / dt) * sum_p hat(u_pk - j) f_p,
// i.e. every pixel deposits (1 - fr) f_p into bin floor(u) and fr f_p into bin floor(u) + 1.
//
// Design (GB300): a CTA owns kAng consecutive angles and one band of the image; it walks
// the band's 64 x 64 pixel tiles (the next tile is prefetched into registers while the
// current one is processed) and keeps the full detector rows of its angles in shared
// memory, so each sinogram bin is written to global memory once per band.  Within a tile
// each warp owns a private window of bins per angle.  Lanes of a warp take pixels that
// are S_k pixels apart along the angle's dominant axis, with S_k |dominant step| > 1 bin,
// so the 32 lanes of one instruction always hit 32 different bins: the deposits are plain
// shared-memory read-modify-writes, no atomics.  After each tile the warp windows are
// summed into the detector rows (each bin owned by one thread).  The window origin J0 and
// the tile-local coordinate come from the same 32.32 fixed-point tile stepping as R*.
#include <algorithm>

#include "common.cuh"

namespace bp {

namespace {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagicInt = 0x4B400000;
constexpr int kRThreads = 256;
constexpr int kRWarps = kRThreads / 32;
constexpr int kAngMax = 4;

__global__ void __launch_bounds__(kRThreads, 2)
radon_direct_kernel(const float *__restrict__ img, float *__restrict__ sino, const AngleParam *__restrict__ ap,
                    int N, int n_det, int n_theta, int W, int C, int kAng, int tiles_per_band, float scale,
                    int use_atomic, long long img_stride, long long sino_stride) {
    extern __shared__ __align__(16) float rsm[];
    float *rows = rsm;                                   // [kAng][n_det] detector rows of this CTA
    float *tile = rows + kAng * n_det;                   // [64][65] current pixel tile
    float *win = tile + kTile * (kTile + 1);             // [warps][kAng][W] private bin windows
    __shared__ float4 sp[kAngMax];                       // q0, c, s, dominant step
    __shared__ int sJ0[kAngMax], sS[kAngMax], sX[kAngMax];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k0 = blockIdx.x * kAng;
    const int kn = min(kAng, n_theta - k0);
    const int tiles = (N + kTile - 1) / kTile;
    const int t_begin = blockIdx.y * tiles_per_band;
    const int t_end = min(tiles * tiles, t_begin + tiles_per_band);
    img += (long long)blockIdx.z * img_stride;
    sino += (long long)blockIdx.z * sino_stride;

    for (int i = tid; i < kAng * n_det; i += kRThreads) rows[i] = 0.f;
    float *mywin = win + warp * kAng * W;
    for (int i = lane; i < kAng * W; i += 32) mywin[i] = 0.f;

    // register prefetch of a tile: thread covers rows (tid/64) + 4i, column tid%64
    float pre[16];
    auto fetch = [&](int t) {
        const int ty = t / tiles, tx = t % tiles;
        const int x = tx * kTile + (tid & 63);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int y = ty * kTile + (tid >> 6) + 4 * i;
            pre[i] = (x < N && y < N) ? __ldg(img + (long long)y * N + x) : 0.f;
        }
    };
    if (t_begin < t_end) fetch(t_begin);

    for (int t = t_begin; t < t_end; ++t) {
        const int ty = t / tiles, tx = t % tiles;
        __syncthreads();  // previous tile fully consumed (tile buffer, params, windows reduced)
#pragma unroll
        for (int i = 0; i < 16; ++i) tile[((tid >> 6) + 4 * i) * (kTile + 1) + (tid & 63)] = pre[i];
        if (tid < kn) {
            const AngleParam p = ap[k0 + tid];
            const long long U = p.U00 + (long long)tx * p.CT + (long long)ty * p.ST;
            const int Ji = (int)(U >> 32);
            const float frac = (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f;
            const float emin = (float)(kTile - 1) * (fminf(p.c, 0.f) + fminf(p.s, 0.f));
            const int J0 = Ji + (int)floorf(emin) - 1;
            const float q0 = (float)(Ji - J0 - C) + (frac - 0.5f);
            const bool xdom = fabsf(p.c) >= fabsf(p.s);
            const float dom = xdom ? fabsf(p.c) : fabsf(p.s);
            sJ0[tid] = J0;
            sS[tid] = (int)floorf(1.0f / dom) + 1;  // S * |dominant step| > 1 bin
            sX[tid] = xdom ? 1 : 0;
            sp[tid] = make_float4(q0, p.c, p.s, 0.f);
        }
        __syncthreads();
        if (t + 1 < t_end) fetch(t + 1);

        for (int a = 0; a < kn; ++a) {
            const float4 P = sp[a];
            const int S = sS[a];
            const bool xdom = sX[a] != 0;
            float *wa = mywin + a * W + C;
            // lines along the dominant axis: warp w takes lines w, w+8, ...; lane l takes
            // positions phase + S*l on the line.
            for (int line = warp; line < kTile; line += kRWarps) {
                for (int ph = 0; ph < S; ++ph) {
                    const int pos = ph + S * lane;
                    const bool act = pos < kTile;  // all lanes reach both __syncwarp calls
                    const int x = xdom ? pos : line, y = xdom ? line : pos;
                    const float f = act ? tile[y * (kTile + 1) + x] : 0.f;
                    const float q = fmaf((float)y, P.z, fmaf((float)x, P.y, P.x));
                    const float r = q + kMagic;
                    const int m = __float_as_int(r) - kMagicInt;  // rint(q)
                    const float fr = (q - (r - kMagic)) + 0.5f;    // u - floor(u)
                    const float hi = fr * f;
                    if (act) wa[m] += f - hi;
                    __syncwarp();
                    if (act) wa[m + 1] += hi;
                    __syncwarp();
                }
            }
        }
        __syncthreads();
        // sum the warp windows into the detector rows and clear them
        for (int i = tid; i < kn * W; i += kRThreads) {
            const int a = i / W, m = i - a * W;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < kRWarps; ++w) {
                float *cell = win + (w * kAng + a) * W + m;
                s += *cell;
                *cell = 0.f;
            }
            const int j = sJ0[a] + m;
            if (j >= 0 && j < n_det) rows[a * n_det + j] += s;
        }
    }
    __syncthreads();
    for (int i = tid; i < kn * n_det; i += kRThreads) {
        const int a = i / n_det, j = i - a * n_det;
        float *dst = sino + (long long)(k0 + a) * n_det + j;
        const float v = scale * rows[i];
        if (use_atomic) {
            if (v != 0.f) atomicAdd(dst, v);
        } else {
            *dst = v;
        }
    }
}

}  // namespace

bp_status launch_radon_direct(bp_plan *p, const float *img, float *sino, int batch, cudaStream_t st) {
    const size_t sino_n = (size_t)p->n_theta * p->n_det;
    const int tiles = (p->N + kTile - 1) / kTile;
    const int ntiles = tiles * tiles;
    int kAng = kAngMax;
    while (kAng > 1 && (size_t)kAng * p->n_det * 4 > 64 * 1024) kAng >>= 1;
    const size_t smem = sizeof(float) * ((size_t)kAng * p->n_det + kTile * (kTile + 1) + (size_t)kRWarps * kAng * p->W);
    if (smem > 200 * 1024) return fail(BP_ERR_UNSUPPORTED, "radon: n_det or window too large for shared memory");
    // bands: enough CTAs to fill the GPU about twice, at most one band per tile
    const int ablocks = (p->n_theta + kAng - 1) / kAng;
    int bands = std::max(1, std::min(ntiles, (2 * 152 * 2 + ablocks - 1) / ablocks));
    const int per_band = (ntiles + bands - 1) / bands;
    bands = (ntiles + per_band - 1) / per_band;
    const int use_atomic = bands > 1;
    if (use_atomic) BP_CUDA_TRY(cudaMemsetAsync(sino, 0, sizeof(float) * sino_n * batch, st));
    BP_CUDA_TRY(cudaFuncSetAttribute(radon_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const float scale = (float)(p->dx * p->dx / p->dt);
    dim3 grid(ablocks, bands, batch);
    radon_direct_kernel<<<grid, kRThreads, smem, st>>>(img, sino, p->d_ang, p->N, p->n_det, p->n_theta, p->W, p->C,
                                                       kAng, per_band, scale, use_atomic, (long long)p->N * p->N,
                                                       (long long)sino_n);
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

}  // namespace bp
