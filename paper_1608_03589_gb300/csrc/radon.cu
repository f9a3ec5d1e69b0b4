// Forward Radon transform R as the exact scaled transpose of the direct R* (Section 1,
// eqs "P_theta" and "adjoint"):
//     (R f)_{kj} = (dx^2 / dt) * sum_p hat(u_pk - j) f_p,
// i.e. every pixel deposits (1 - fr) f_p into bin floor(u) and fr f_p into bin floor(u) + 1.
//
// Two forms share the launch structure (GB300): a CTA owns kAng consecutive angles and one
// band of the image; it walks the band's 64 x 64 pixel tiles (the next tile is prefetched into
// registers while the current one is processed) and keeps the full detector rows of its angles
// in shared memory, so each sinogram bin is written to global memory once per band.  When
// pixels are no larger than bins (|c|, |s| <= 1) the 2 x 2-block form below runs (the
// transpose of the 2 x 2-block R*); otherwise the per-pixel form described here.
//
// Per-pixel form: within a tile each warp owns a private window per angle of interval sums (A_m, B_m) = (sum f,
// sum f (q - m)) over the pixels whose tile-local coordinate q rounds to m; the two bins
// around interval m then receive A/2 - B and A/2 + B (exactly (1 - fr) f and fr f summed),
// with no cancellation because |q - m| <= 1/2.  Lanes of a warp take pixels S pixels apart
// along the dominant axis of the block's angles, with S |dominant step| > 1 bin, so the 32
// lanes of one instruction always hit 32 different intervals: each deposit is one plain
// float2 shared-memory read-modify-write, no atomics; a pixel value is read once and
// deposited for all angles of the block (independent windows: the reads of all angles are
// issued before the writes, and the coordinates of two angles share one packed f32x2
// instruction).  After each tile the warp windows are folded into the detector rows (each bin
// owned by one thread).  The window origin J0 and the tile-local coordinate come from the
// same 32.32 fixed-point tile stepping as R*.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "f32x2.cuh"

namespace bp {

namespace {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagicInt = 0x4B400000;
constexpr int kRThreads = 256;
constexpr int kRWarps = kRThreads / 32;
constexpr int kAngMax = 4;
constexpr size_t kMaxRadonSmem = 200 * 1024;

__global__ void __launch_bounds__(kRThreads, 3)
radon_direct_kernel(const float *__restrict__ img, float *__restrict__ sino, const AngleParam *__restrict__ ap,
                    int N, int n_det, int n_theta, int W, int C, int kAng, int tiles_per_band, float scale,
                    int use_atomic, long long img_stride, long long sino_stride, int per_angle_w) {
    extern __shared__ __align__(16) float rsm[];
    float *rows = rsm;                                                   // [kAng][n_det] detector rows
    float2 *win = reinterpret_cast<float2 *>(rows + ((kAng * n_det + 3) & ~3));  // [warps][kAng][W] (A, B)
    float *tile = reinterpret_cast<float *>(win + kRWarps * kAng * W);  // [64][65] pixel tile
    __shared__ float4 sp[kAngMax];  // q0, c, s, -
    __shared__ int sJ0[kAngMax];
    __shared__ int sMode[2];        // common (x-dominant, S) of the block's angles, or S = 0 if mixed

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k0 = blockIdx.x * kAng;
    const int kn = min(kAng, n_theta - k0);
    const int tiles = (N + kTile - 1) / kTile;
    const int t_begin = blockIdx.y * tiles_per_band;
    const int t_end = min(tiles * tiles, t_begin + tiles_per_band);
    img += (long long)blockIdx.z * img_stride;
    sino += (long long)blockIdx.z * sino_stride;

    for (int i = tid; i < kAng * n_det; i += kRThreads) rows[i] = 0.f;
    float2 *mywin = win + warp * kAng * W;
    for (int i = lane; i < kAng * W; i += 32) mywin[i] = make_float2(0.f, 0.f);
    if (tid == 0) {
        // one lane spacing for all angles of the block when they share a dominant axis
        int xd = -1, S = 0;
        bool mixed = false;  // once two axes are seen, the block stays mixed
        for (int a = 0; a < kn; ++a) {
            const AngleParam p = ap[k0 + a];
            const bool x = fabsf(p.c) >= fabsf(p.s);
            const float dom = x ? fabsf(p.c) : fabsf(p.s);
            const int Sa = (int)floorf(1.0f / dom) + 1;  // Sa * |dominant step| > 1 bin
            if (a == 0) { xd = x; S = Sa; }
            else if (xd != (int)x) mixed = true;
            else S = max(S, Sa);
        }
        sMode[0] = xd;
        sMode[1] = mixed ? 0 : S;
    }

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

    // deposit the pixels of lines warp, warp + 8, ... of the tile for angles [a0, a1)
    const unsigned win_u32 = smem_u32(mywin);
    const unsigned long long MM = pk2(kMagic, kMagic);
    auto deposit = [&](int a0, int a1, bool xdom, int S) {
        // per pair of angles (2p, 2p + 1): base coordinates and steps packed for the paired
        // FP32 instructions, and the window byte addresses offset so that the rounding's bit
        // pattern (magic + m) indexes the window directly
        unsigned long long Q0[kAngMax / 2], CX[kAngMax / 2], SY[kAngMax / 2];
        unsigned wb[kAngMax];
#pragma unroll
        for (int p2 = 0; p2 < kAngMax / 2; ++p2) {
            const float4 Pa = (a0 + 2 * p2 < a1) ? sp[a0 + 2 * p2] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 Pb = (a0 + 2 * p2 + 1 < a1) ? sp[a0 + 2 * p2 + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            Q0[p2] = pk2(Pa.x, Pb.x);
            CX[p2] = pk2(Pa.y, Pb.y);
            SY[p2] = pk2(Pa.z, Pb.z);
        }
#pragma unroll
        for (int a = 0; a < kAngMax; ++a)
            wb[a] = win_u32 + 8u * (unsigned)((a0 + a) * W + C) - ((unsigned)kMagicInt << 3);
        for (int line = warp; line < kTile; line += kRWarps) {
            for (int base = 0; base < kTile; base += 32 * S) {
                for (int ph = 0; ph < S; ++ph) {
                    const int pos = base + ph + S * lane;
                    const bool act = pos < kTile;
                    const int x = xdom ? pos : line, y = xdom ? line : pos;
                    const float f = act ? tile[y * (kTile + 1) + x] : 0.f;
                    const unsigned long long X2 = pk2((float)x, (float)x), Y2 = pk2((float)y, (float)y);
                    // all angles' window cells are read before any is written back (different
                    // angles never share a cell), so the reads are in flight together
                    unsigned cell[kAngMax];
                    float dq[kAngMax];
#pragma unroll
                    for (int p2 = 0; p2 < kAngMax / 2; ++p2) {
                        const unsigned long long Q = ffma2(Y2, SY[p2], ffma2(X2, CX[p2], Q0[p2]));
                        const unsigned long long R = fadd2(Q, MM);            // magic + rint(q)
                        const unsigned long long D = fsub2(Q, fsub2(R, MM));  // q - rint(q)
                        float r0, r1;
                        upk2(R, r0, r1);
                        upk2(D, dq[2 * p2], dq[2 * p2 + 1]);
                        cell[2 * p2] = wb[2 * p2] + (__float_as_uint(r0) << 3);
                        cell[2 * p2 + 1] = wb[2 * p2 + 1] + (__float_as_uint(r1) << 3);
                    }
                    const int na = act ? a1 - a0 : 0;
                    float2 v[kAngMax];
#pragma unroll
                    for (int a = 0; a < kAngMax; ++a)
                        if (a < na) v[a] = lds64(cell[a]);
#pragma unroll
                    for (int a = 0; a < kAngMax; ++a) {
                        if (a < na) {
                            v[a].x += f;
                            v[a].y = fmaf(f, dq[a], v[a].y);
                            sts64(cell[a], v[a]);
                        }
                    }
                    __syncwarp();
                }
            }
        }
    };

    // The common case: a full block of kAngMax angles sharing a dominant axis whose step
    // exceeds half a bin, so lanes sit S = 2 pixels apart and the 64-pixel line is exactly two
    // phases of 32 active lanes.  The same deposits as `deposit`, fully unrolled, without the
    // per-lane and per-angle predicates.
    auto deposit_full = [&](auto xdom_tag) {
        constexpr bool XDOM = decltype(xdom_tag)::value;
        unsigned long long Q0[kAngMax / 2], CX[kAngMax / 2], SY[kAngMax / 2];
        unsigned wb[kAngMax];
#pragma unroll
        for (int p2 = 0; p2 < kAngMax / 2; ++p2) {
            const float4 Pa = sp[2 * p2], Pb = sp[2 * p2 + 1];
            Q0[p2] = pk2(Pa.x, Pb.x);
            CX[p2] = pk2(Pa.y, Pb.y);
            SY[p2] = pk2(Pa.z, Pb.z);
        }
#pragma unroll
        for (int a = 0; a < kAngMax; ++a) wb[a] = win_u32 + 8u * (unsigned)(a * W + C) - ((unsigned)kMagicInt << 3);
        for (int line = warp; line < kTile; line += kRWarps) {
#pragma unroll
            for (int ph = 0; ph < 2; ++ph) {
                const int pos = ph + 2 * lane;
                const int x = XDOM ? pos : line, y = XDOM ? line : pos;
                const float f = tile[y * (kTile + 1) + x];
                const unsigned long long X2 = pk2((float)x, (float)x), Y2 = pk2((float)y, (float)y);
                unsigned cell[kAngMax];
                float dq[kAngMax];
#pragma unroll
                for (int p2 = 0; p2 < kAngMax / 2; ++p2) {
                    const unsigned long long Q = ffma2(Y2, SY[p2], ffma2(X2, CX[p2], Q0[p2]));
                    const unsigned long long R = fadd2(Q, MM);
                    const unsigned long long D = fsub2(Q, fsub2(R, MM));
                    float r0, r1;
                    upk2(R, r0, r1);
                    upk2(D, dq[2 * p2], dq[2 * p2 + 1]);
                    cell[2 * p2] = wb[2 * p2] + (__float_as_uint(r0) << 3);
                    cell[2 * p2 + 1] = wb[2 * p2 + 1] + (__float_as_uint(r1) << 3);
                }
                float2 v[kAngMax];
#pragma unroll
                for (int a = 0; a < kAngMax; ++a) v[a] = lds64(cell[a]);
#pragma unroll
                for (int a = 0; a < kAngMax; ++a) {
                    v[a].x += f;
                    v[a].y = fmaf(f, dq[a], v[a].y);
                    sts64(cell[a], v[a]);
                }
                __syncwarp();
            }
        }
    };

    for (int t = t_begin; t < t_end; ++t) {
        const int ty = t / tiles, tx = t % tiles;
        __syncthreads();  // previous tile fully consumed (tile buffer, params, windows folded)
#pragma unroll
        for (int i = 0; i < 16; ++i) tile[((tid >> 6) + 4 * i) * (kTile + 1) + (tid & 63)] = pre[i];
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
        if (t + 1 < t_end) fetch(t + 1);

        if (sMode[1] == 2 && kn == kAngMax && kAng == kAngMax) {
            if (sMode[0] != 0) deposit_full(std::integral_constant<bool, true>());
            else deposit_full(std::integral_constant<bool, false>());
        } else if (sMode[1] > 0) {
            deposit(0, kn, sMode[0] != 0, sMode[1]);
        } else {
            for (int a = 0; a < kn; ++a) {  // mixed dominant axes: one angle at a time
                const float4 P = sp[a];
                const bool x = fabsf(P.y) >= fabsf(P.z);
                const float dom = x ? fabsf(P.y) : fabsf(P.z);
                deposit(a, a + 1, x, (int)floorf(1.0f / dom) + 1);
            }
        }
        __syncthreads();
        // fold the warp windows into the detector rows: bin m takes interval m (lower part)
        // and interval m - 1 (upper part); clear the windows
        for (int i = tid; i < kn * W; i += kRThreads) {
            const int a = i / W, m = i - a * W;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < kRWarps; ++w) {
                const float2 *wa = win + (w * kAng + a) * W;
                const float2 lo = wa[m];
                s += 0.5f * lo.x - lo.y;
                if (m > 0) {
                    const float2 up = wa[m - 1];
                    s += 0.5f * up.x + up.y;
                }
            }
            const int j = sJ0[a] + m;
            if (j >= 0 && j < n_det) rows[a * n_det + j] += s;
        }
        __syncthreads();
        for (int i = tid; i < kRWarps * kn * W; i += kRThreads) {
            const int w = i / (kn * W), r = i - w * kn * W;
            win[w * kAng * W + r] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    for (int i = tid; i < kn * n_det; i += kRThreads) {
        const int a = i / n_det, j = i - a * n_det;
        float *dst = sino + (long long)(k0 + a) * n_det + j;
        const float v = (per_angle_w ? __ldg(&ap[k0 + a].w) : scale) * rows[i];
        if (use_atomic) {
            if (v != 0.f) atomicAdd(dst, v);
        } else {
            *dst = v;
        }
    }
}

// ---------------------------------------------------------------- 2 x 2-block form
// Transpose of the 2 x 2-block R* (|c|, |s| <= 1).  In the forward form each corner of a block
// whose lowest corner sits at window coordinate q (entry e = floor(q) + C, r = q - floor(q))
// takes g_j + sum_k ramp_k dg_{j+k}, ramp_k = sat(r + o - k), o the corner's offset in
// {0, |c|, |s|, |c| + |s|}.  The transpose adds the block's four pixels into entry e of a
// window table as
//     (X, Y, Z, V) += (sum f, sum f ramp_0, sum f ramp_1, sum f ramp_2),
// and once the tile is done, bin J0 + m takes X_m - Y_m + Y_{m-1} - Z_{m-1} + Z_{m-2} - V_{m-2}
// + V_{m-3} (dg_{j+k} = g_{j+k+1} - g_{j+k}).  The 8 / kAng warps of an angle each own a table
// and take interleaved lines of blocks along the angle's minor axis; lanes take blocks S apart
// along the dominant axis with 2 S |dominant step| > 1 bin, so the 32 entries of one
// read-modify-write are distinct: one float4 read-modify-write per block and angle.  The
// pixel tile keeps its 8-byte pairs XOR-swizzled per line pair (slot = pair ^ (line / 2 mod
// 16)), so that lanes walking a row or a column of blocks read it without bank conflicts.  Each
// warp folds its own table into bins with three warp shuffles per 32 bins and adds them into
// the angle's detector row (shared-memory atomics: the angle's warps fold at the same time).
constexpr int kQGuard = 1;  // unused guard entries on each side of a warp table

__device__ __forceinline__ float add_sat(float a, float b) {  // min(max(a + b, 0), 1)
    float d;
    asm("add.sat.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}
// a + b rounded toward minus infinity: with b = 1.5 * 2^23 the low mantissa bits hold floor(a)
__device__ __forceinline__ float add_rm(float a, float b) {
    float d;
    asm("add.rm.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

struct QuadRamp {
    float ac, ac1, as, as1, af, af1, af2;  // |c|, |c| - 1, |s|, |s| - 1, |c| + |s|, minus 1, minus 2
};

// The warp's lines of blocks for one angle: block (L, I) along (dominant, minor) axes with
// I = h + wpa i; lanes with act false compute but do not deposit.
template <bool SX, bool FAR2>
__device__ __forceinline__ void radon_quad_lines(unsigned tile_u32, unsigned tab, float qL, float qstep, int n_it,
                                                 int h, int wpa, int L, bool xdom, int rowoff, int rowdelta,
                                                 const QuadRamp &k, bool act) {
#pragma unroll 2
    for (int i = 0; i < n_it; ++i) {
        const int I = h + wpa * i;
        const int bx = xdom ? L : I, by = xdom ? I : L;
        const unsigned pa = tile_u32 + 4u * (unsigned)((by << 7) + ((bx ^ (by & 15)) << 1) + rowoff);
        const float2 plo = lds64(pa), phi = lds64(pa + (unsigned)rowdelta);
        const float f0 = SX ? plo.y : plo.x, fc = SX ? plo.x : plo.y;  // lowest corner, x neighbour
        const float fs = SX ? phi.y : phi.x, ff = SX ? phi.x : phi.y;  // y neighbour, far corner
        const float q = fmaf((float)i, qstep, qL);
        const float Rf = add_rm(q, kMagic);
        const float r = q - (Rf - kMagic);
        const unsigned ea = tab + (__float_as_uint(Rf) << 4);
        float dy = fmaf(fc, add_sat(r, k.ac), fmaf(fs, add_sat(r, k.as), f0 * r));
        float dz = fmaf(fc, add_sat(r, k.ac1), fs * add_sat(r, k.as1));
        float dw = 0.f;
        if (FAR2) {  // |c| + |s| >= 1: the far corner's first ramp is 1
            dy += ff;
            dz = fmaf(ff, add_sat(r, k.af1), dz);
            dw = ff * add_sat(r, k.af2);
        } else {     // |c| + |s| < 1: its third ramp is 0
            dy = fmaf(ff, add_sat(r, k.af), dy);
            dz = fmaf(ff, add_sat(r, k.af1), dz);
        }
        const float F = (f0 + fc) + (fs + ff);
        if (act) {
            float4 t = lds128(ea);
            t.x += F;
            t.y += dy;
            t.z += dz;
            if (FAR2) t.w += dw;
            sts128(ea, t);
        }
        __syncwarp();  // the next line's read-modify-writes see this line's
    }
}

__global__ void __launch_bounds__(kRThreads, 3)
radon_quad_kernel(const float *__restrict__ img, float *__restrict__ sino, const AngleParam *__restrict__ ap, int N,
                  int n_det, int n_theta, int W, int C, int kAng, int tiles_per_band, float scale, int use_atomic,
                  long long img_stride, long long sino_stride, int per_angle_w) {
    extern __shared__ __align__(16) float rsm[];
    const int rows_n = (kAng * n_det + 3) & ~3;
    const int Wt = W + 2 * kQGuard;
    float *rows = rsm;                                                       // [kAng][n_det] detector rows
    float4 *tabs = reinterpret_cast<float4 *>(rsm + rows_n);                 // [warps][Wt] window tables
    float *tile = reinterpret_cast<float *>(tabs + kRWarps * Wt);           // [64 * 64] swizzled pixel tile

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k0 = blockIdx.x * kAng;
    const int kn = min(kAng, n_theta - k0);
    const int tiles = (N + kTile - 1) / kTile;
    const int t_begin = blockIdx.y * tiles_per_band;
    const int t_end = min(tiles * tiles, t_begin + tiles_per_band);
    img += (long long)blockIdx.z * img_stride;
    sino += (long long)blockIdx.z * sino_stride;

    for (int i = tid; i < rows_n; i += kRThreads) rows[i] = 0.f;
    for (int i = tid; i < kRWarps * Wt; i += kRThreads) tabs[i] = make_float4(0.f, 0.f, 0.f, 0.f);

    // the warp's angle a (of the block's kAng) and its share h of the angle's block lines
    const int wpa = kRWarps / kAng;
    const int a = warp % kAng, h = warp / kAng;
    const bool live = a < kn;
    AngleParam P = {};
    if (live) P = ap[k0 + a];
    const float c = P.c, s = P.s;
    QuadRamp k;
    k.ac = fabsf(c);
    k.as = fabsf(s);
    k.ac1 = k.ac - 1.f;
    k.as1 = k.as - 1.f;
    k.af = k.ac + k.as;
    k.af1 = k.af - 1.f;
    k.af2 = k.af - 2.f;
    const bool xdom = k.ac >= k.as;
    const float d1 = xdom ? c : s, d2 = xdom ? s : c;  // u steps per pixel along the dominant, minor axes
    const int S = live ? max(1, min(32, (int)ceilf(1.001f / (2.f * fabsf(d1))))) : 1;
    const bool SX = c < 0.f, SY = s < 0.f, FAR2 = k.af1 >= 0.f;
    const float lo = fminf(c, 0.f) + fminf(s, 0.f);
    const int F63 = (int)floorf((float)(kTile - 1) * lo);
    const int rowoff = SY ? kTile : 0;           // line of the lowest corner within the block (floats)
    const int rowdelta = SY ? -4 * kTile : 4 * kTile;  // bytes to the block's other line
    const int n_it = kTile / 2 / wpa;
    const float qstep = (float)(2 * wpa) * d2;
    const unsigned tile_u32 = smem_u32(tile);
    const unsigned tab = smem_u32(tabs + warp * Wt + kQGuard) + 16u * (unsigned)C - ((unsigned)kMagicInt << 4);

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

    // the warp's table -> bins J0 .. J0 + m_end - 1 of the angle's row (added atomically: the
    // angle's warps fold together), table cleared.  Entries above 3 + 62 (|c| + |s|) stay zero (a
    // margin of two bins is kept).
    const int m_end = min(W + 3, (int)(62.f * k.af) + 9);
    const unsigned tab0 = smem_u32(tabs + warp * Wt + kQGuard);
    auto fold = [&](int J0) {
        float k1 = 0.f, k2 = 0.f, k3 = 0.f;  // c1, c2, c3 of the previous 32 entries' last lanes
        for (int m0 = 0; m0 < m_end; m0 += 32) {
            const int m = m0 + lane;
            float4 T = make_float4(0.f, 0.f, 0.f, 0.f);
            if (m < W) {
                T = lds128(tab0 + 16u * (unsigned)m);
                sts128(tab0 + 16u * (unsigned)m, make_float4(0.f, 0.f, 0.f, 0.f));
            }
            // entry m adds (X - Y, Y - Z, Z - V, V) to bins m .. m + 3
            const float c0 = T.x - T.y, c1 = T.y - T.z, c2 = T.z - T.w, c3 = T.w;
            const float s1 = __shfl_sync(0xffffffffu, c1, (lane + 31) & 31);
            const float s2 = __shfl_sync(0xffffffffu, c2, (lane + 30) & 31);
            const float s3 = __shfl_sync(0xffffffffu, c3, (lane + 29) & 31);
            const float v = c0 + (lane >= 1 ? s1 : k1) + (lane >= 2 ? s2 : k2) + (lane >= 3 ? s3 : k3);
            k1 = s1;
            k2 = s2;
            k3 = s3;
            const int j = J0 + m;
            if (m < m_end && j >= 0 && j < n_det) atomicAdd(rows + a * n_det + j, v);
        }
    };

    int J0prev = 0;
    for (int t = t_begin; t < t_end; ++t) {
        const int ty = t / tiles, tx = t % tiles;
        __syncthreads();  // every block of the previous tile deposited; initial clears done
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int y = (tid >> 6) + 4 * i, x = tid & 63;
            tile[y * kTile + 2 * ((x >> 1) ^ ((y >> 1) & 15)) + (x & 1)] = pre[i];
        }
        if (live && t > t_begin) fold(J0prev);
        __syncthreads();  // tile stored, tables cleared
        if (t + 1 < t_end) fetch(t + 1);
        if (live) {
            const long long U = P.U00 + (long long)tx * P.CT + (long long)ty * P.ST;
            const int Ji = (int)(U >> 32);
            const float frac = (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f;
            J0prev = Ji + F63 - 1;  // window start: entry e is bin J0 + e
            const float q0 = (float)(1 - F63 - C) + frac + lo;
            for (int ph = 0; ph < S; ++ph) {
                const int L = ph + S * lane;
                const bool act = L < kTile / 2;
                const int Lc = act ? L : kTile / 2 - 1;
                const float qL = fmaf(2.f * (float)Lc, d1, fmaf(2.f * (float)h, d2, q0));
                if (SX) {
                    if (FAR2) radon_quad_lines<true, true>(tile_u32, tab, qL, qstep, n_it, h, wpa, Lc, xdom, rowoff, rowdelta, k, act);
                    else radon_quad_lines<true, false>(tile_u32, tab, qL, qstep, n_it, h, wpa, Lc, xdom, rowoff, rowdelta, k, act);
                } else {
                    if (FAR2) radon_quad_lines<false, true>(tile_u32, tab, qL, qstep, n_it, h, wpa, Lc, xdom, rowoff, rowdelta, k, act);
                    else radon_quad_lines<false, false>(tile_u32, tab, qL, qstep, n_it, h, wpa, Lc, xdom, rowoff, rowdelta, k, act);
                }
            }
        }
    }
    __syncthreads();
    if (live && t_begin < t_end) fold(J0prev);
    __syncthreads();
    for (int i = tid; i < kn * n_det; i += kRThreads) {
        const int aa = i / n_det, j = i - aa * n_det;
        float *dst = sino + (long long)(k0 + aa) * n_det + j;
        const float v = (per_angle_w ? __ldg(&ap[k0 + aa].w) : scale) * rows[i];
        if (use_atomic) {
            if (v != 0.f) atomicAdd(dst, v);
        } else {
            *dst = v;
        }
    }
}

}  // namespace

// The 2 x 2-block form needs |c|, |s| <= 1 (a block spans at most four bins).
static bool radon_quad_form(const bp_plan *p) { return p->step_max <= 1.0f; }

static size_t radon_pair_smem(const bp_plan *p, int kAng) {
    return sizeof(float) * ((((size_t)kAng * p->n_det + 3) & ~(size_t)3) + kTile * (kTile + 1)) +
           sizeof(float2) * (size_t)kRWarps * kAng * p->W;
}

static size_t radon_quad_smem(const bp_plan *p, int kAng) {
    return sizeof(float) * ((((size_t)kAng * p->n_det + 3) & ~(size_t)3) + (size_t)kTile * kTile) +
           sizeof(float4) * (size_t)kRWarps * (p->W + 2 * kQGuard);
}

size_t radon_smem(const bp_plan *p, int kAng) {
    return radon_quad_form(p) ? radon_quad_smem(p, kAng) : radon_pair_smem(p, kAng);
}

int radon_max_kang(const bp_plan *p) {
    int kAng = kAngMax;
    while (kAng > 1 && radon_smem(p, kAng) > kMaxRadonSmem) kAng >>= 1;
    return kAng;
}

// The shape a launch really uses (defaults resolved, values clamped); bands is the number
// of bands after rounding the tiles per band up.
RadonShape radon_effective(const bp_plan *p, RadonShape shape) {
    const int tiles = (p->N + kTile - 1) / kTile;
    const int ntiles = tiles * tiles;
    int kAng = kAngMax;
    if (shape.kang == 1 || shape.kang == 2 || shape.kang == 4) {
        kAng = shape.kang;
    } else {  // default: detector rows of the block's angles within 64 KB
        while (kAng > 1 && (size_t)kAng * p->n_det * 4 > 64 * 1024) kAng >>= 1;
    }
    kAng = std::min(kAng, radon_max_kang(p));
    const int ablocks = (p->n_theta + kAng - 1) / kAng;
    int bands = shape.bands;
    if (bands <= 0) {
        // default: enough CTAs to fill the GPU about twice (2 CTAs per SM)
        const int target = 2 * 2 * std::max(1, p->sm_count);
        bands = (target + ablocks - 1) / ablocks;
    }
    bands = std::max(1, std::min(ntiles, bands));
    const int per_band = (ntiles + bands - 1) / bands;
    RadonShape e;
    e.kang = kAng;
    e.bands = (ntiles + per_band - 1) / per_band;
    return e;
}

RadonShape radon_clamp(const bp_plan *p, RadonShape shape) { return radon_effective(p, shape); }
RadonShape radon_shape_used(const bp_plan *p, int batch) { return radon_effective(p, radon_shape(p, batch)); }

bp_status launch_radon_shape(bp_plan *p, const float *img, float *sino, int batch, cudaStream_t st, int per_angle_w,
                             RadonShape shape) {
    const size_t sino_n = (size_t)p->n_theta * p->n_det;
    const int tiles = (p->N + kTile - 1) / kTile;
    const int ntiles = tiles * tiles;
    const RadonShape eff = radon_effective(p, shape);
    const int kAng = eff.kang, bands = eff.bands;
    const size_t smem = radon_smem(p, kAng);
    if (smem > kMaxRadonSmem) return fail(BP_ERR_UNSUPPORTED, "radon: n_det or window too large for shared memory");
    const int ablocks = (p->n_theta + kAng - 1) / kAng;
    const int per_band = (ntiles + bands - 1) / bands;
    const int use_atomic = bands > 1;
    stage_begin(p, st);
    if (use_atomic) {
        BP_CUDA_TRY(cudaMemsetAsync(sino, 0, sizeof(float) * sino_n * batch, st));
        stage_mark(p, st, "memset (R image bands)");
    }
    const float scale = (float)(p->dx * p->dx / p->dt);
    dim3 grid(ablocks, bands, batch);
    if (radon_quad_form(p)) {
        BP_CUDA_TRY(cudaFuncSetAttribute(radon_quad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        radon_quad_kernel<<<grid, kRThreads, smem, st>>>(img, sino, p->d_ang, p->N, p->n_det, p->n_theta, p->W, p->C,
                                                         kAng, per_band, scale, use_atomic, (long long)p->N * p->N,
                                                         (long long)sino_n, per_angle_w);
        stage_mark(p, st, "radon_quad_kernel");
    } else {
        BP_CUDA_TRY(cudaFuncSetAttribute(radon_direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        radon_direct_kernel<<<grid, kRThreads, smem, st>>>(img, sino, p->d_ang, p->N, p->n_det, p->n_theta, p->W,
                                                           p->C, kAng, per_band, scale, use_atomic,
                                                           (long long)p->N * p->N, (long long)sino_n, per_angle_w);
        stage_mark(p, st, "radon_direct_kernel");
    }
    BP_CUDA_TRY(cudaGetLastError());
    return BP_OK;
}

bp_status launch_radon_direct(bp_plan *p, const float *img, float *sino, int batch, cudaStream_t st, int per_angle_w) {
    return launch_radon_shape(p, img, sino, batch, st, per_angle_w, radon_shape(p, batch));
}

}  // namespace bp
