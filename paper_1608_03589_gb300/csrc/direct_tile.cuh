// Pieces of the direct R* shared by the kernels of direct.cu and batched.cu (internal): one
// 64 x 64 tile with synchronous window loads, in the pair-table form (direct_tile_sync) and in
// the 2 x 2-block form (direct_tile_quad_sync), and the stage arithmetic of the 2 x 2-block
// form (quad_*), which the TMA kernel uses too.  The arithmetic is described in direct.cu.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "f32x2.cuh"

namespace bp {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr unsigned kMagicBits = 0x4B400000u;

struct DirectStageSmem {
    float4 sp[kStage];  // q0, c, s, table base (bits)
    int J0[kStage];
    float w[kStage];
};

// Angles [k_begin, k_end) of tile (tx, ty); the partial sum is added atomically when
// atomic_out (angle-split launches), else stored (or added, with accumulate).
// tab: kStage * W float2 of shared memory.  All threads of the block must call it.
template <typename Tin>
__device__ __forceinline__ void direct_tile_sync(const Tin *__restrict__ sino, float *__restrict__ img,
                                                 const AngleParam *__restrict__ ap, int N, int n_det, int k_begin,
                                                 int k_end, int W, int C, int tx, int ty, int accumulate,
                                                 int atomic_out, float wuni, float2 *tab, DirectStageSmem &sm) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int lx = lane & 7;
    const int ly = warp * 8 + (lane >> 3);

    float acc[2][8];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 8; ++a) acc[b][a] = 0.f;

    const float fx = (float)lx, fy = (float)ly;
    const unsigned tab_u32 = smem_u32(tab);

    for (int k0 = k_begin; k0 < k_end; k0 += kStage) {
        const int kn = min(kStage, k_end - k0);
        __syncthreads();
        if (tid < kn) {
            const AngleParam p = ap[k0 + tid];
            const long long U = p.U00 + (long long)tx * p.CT + (long long)ty * p.ST;
            const int Ji = (int)(U >> 32);
            const float frac = (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f;
            const float emin = (float)(kTile - 1) * (fminf(p.c, 0.f) + fminf(p.s, 0.f));
            const int J0 = Ji + (int)floorf(emin) - 1;
            const float q0 = (float)(Ji - J0 - C) + (frac - 0.5f);
            sm.J0[tid] = J0;
            sm.w[tid] = wuni > 0.f ? wuni : p.w;
            const unsigned base = tab_u32 + (unsigned)(tid * W) * 8u + 8u * (unsigned)C - (kMagicBits << 3);
            sm.sp[tid] = make_float4(q0, p.c, p.s, __uint_as_float(base));
        }
        __syncthreads();
        {
            // 16 threads per angle build its (e, d) window.
            const int kk = tid >> 4, r = tid & 15;
            if (kk < kn) {
                const Tin *row = sino + (long long)(k0 + kk) * n_det;
                const int J0 = sm.J0[kk];
                const float w = sm.w[kk];
                for (int m = r; m < W; m += 16) {
                    const int j = J0 + m;
                    const float g0 = (j >= 0 && j < n_det) ? load_f(row + j) : 0.f;
                    const float g1 = (j + 1 >= 0 && j + 1 < n_det) ? load_f(row + j + 1) : 0.f;
                    const float d = w * (g1 - g0);
                    const float e = fmaf(0.5f - (float)(m - C), d, w * g0);
                    tab[kk * W + m] = make_float2(e, d);
                }
            }
        }
        __syncthreads();
        for (int kk = 0; kk < kn; ++kk) {
            const float4 P = sm.sp[kk];
            const float qt = fmaf(fy, P.z, fmaf(fx, P.y, P.x));
            const unsigned base = __float_as_uint(P.w);
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float qb = fmaf(4.f * b, P.z, qt);
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const float q = fmaf(8.f * a, P.y, qb);
                    const float v = q + kMagic;
                    const float2 ed = lds64(base + (__float_as_uint(v) << 3));
                    acc[b][a] += fmaf(q, ed.y, ed.x);
                }
            }
        }
    }

#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const int y = ty * kTile + ly + 4 * b;
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int x = tx * kTile + lx + 8 * a;
            if (x < N && y < N) {
                float *dst = img + (long long)y * N + x;
                if (atomic_out) atomicAdd(dst, acc[b][a]);
                else *dst = accumulate ? (*dst + acc[b][a]) : acc[b][a];
            }
        }
    }
}

// ------------------------------------------------------------------ 2 x 2-block form
// Saturated add: min(max(a + b, 0), 1).
__device__ __forceinline__ float add_sat(float a, float b) {
    float d;
    asm("add.sat.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// v[i] <- v[i ^ m] for the four corner roles of a block (bit 0: x flipped, bit 1: y flipped),
// with compile-time indices only.
__device__ __forceinline__ void xor_permute(float (&v)[4], int m) {
    if (m & 1) {
        float t = v[0]; v[0] = v[1]; v[1] = t;
        t = v[2]; v[2] = v[3]; v[3] = t;
    }
    if (m & 2) {
        float t = v[0]; v[0] = v[2]; v[2] = t;
        t = v[1]; v[1] = v[3]; v[3] = t;
    }
}

// Thread -> blocks: each group of 8 lanes covers 4 x 2 blocks (8 x 4 pixels), so the table
// entries of a quarter warp lie within 8 consecutive bins and its 128-bit loads are
// conflict-free; the thread's blocks are (X0 + 8 a, Y0), a < 4, in 2-pixel units.
__device__ __forceinline__ void quad_thread_blocks(int tid, int &X0, int &Y0) {
    const int lane = tid & 31, warp = tid >> 5, qtr = lane >> 3;
    X0 = (lane & 3) + 4 * (qtr & 1);
    Y0 = ((lane >> 2) & 1) + 2 * (qtr >> 1) + 4 * warp;
}

// Per-angle stage parameters of tile (tx, ty): sq = (q at the lowest corner of block (0,0), c,
// s, table base bits), sr = ramp offsets of the side corners, sf = far corner's offsets and
// the corner-role bits; J0 = first bin of the window.  tab_entry0 = shared address of the
// angle's first table entry.
struct QuadAngle {
    float4 sq, sr, sf;
    int J0, role;
    bool far2;
};
__device__ __forceinline__ QuadAngle quad_angle(const AngleParam &p, int tx, int ty, int C, unsigned tab_entry0) {
    QuadAngle o;
    const long long U = p.U00 + (long long)tx * p.CT + (long long)ty * p.ST;
    const int Ji = (int)(U >> 32);
    const float frac = (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f;
    const float lo = fminf(p.c, 0.f) + fminf(p.s, 0.f);
    o.J0 = Ji + (int)floorf((float)(kTile - 1) * lo) - 1;
    const float q0 = (float)(Ji - o.J0 - C) + frac + lo;
    const unsigned base = tab_entry0 + 16u * (unsigned)C - (kMagicBits << 4);
    const float ac = fabsf(p.c), as = fabsf(p.s), af = ac + as;
    o.role = (p.c < 0.f ? 1 : 0) | (p.s < 0.f ? 2 : 0);
    o.far2 = af - 1.f >= 0.f;
    o.sq = make_float4(q0, p.c, p.s, __uint_as_float(base));
    o.sr = make_float4(ac, ac - 1.f, as, as - 1.f);
    o.sf = make_float4(af, af - 1.f, af - 2.f, __int_as_float(o.role));
    return o;
}

// Stage-uniformity word from lanes < kn of one warp (all 32 lanes call it): role | 4 when
// every angle has the same corner roles, plus 8 when every far corner needs two ramps.
__device__ __forceinline__ int quad_uniform(bool act, int role, bool far2) {
    const int r0 = __shfl_sync(0xffffffffu, role, 0);
    const bool same = __all_sync(0xffffffffu, !act || role == r0);
    const bool all2 = __all_sync(0xffffffffu, !act || far2);
    return same ? (r0 | 4 | (all2 ? 8 : 0)) : 0;
}

// One stage of kn angles for the thread's four blocks (tables and parameters in shared
// memory).  acc[a][role], G[a]: see direct.cu.
__device__ __forceinline__ void quad_stage(float (&acc)[4][4], float (&G)[4], int &role, const float4 *__restrict__ sq,
                                           const float4 *__restrict__ sr, const float4 *__restrict__ sf, int u,
                                           int kn, float fx, float fy) {
    const unsigned long long MM = pk2(kMagic, kMagic);
    // one angle: CHECK = per-angle role check, FAR = 0 per-angle far-corner test, 1 two ramps,
    // 2 three ramps
    auto angle = [&](int kk, auto check_tag, auto far_tag) {
        constexpr bool CHECK = decltype(check_tag)::value;
        constexpr int FAR = decltype(far_tag)::value;
        const float4 A = sq[kk];
        const float4 R2 = sr[kk];
        const float4 F = sf[kk];
        if (CHECK) {
            const int rl = __float_as_int(F.w);
            if (rl != role) {
                // the corner roles follow the signs of (c, s): move each pixel's sum to its new role
#pragma unroll
                for (int a = 0; a < 4; ++a) xor_permute(acc[a], rl ^ role);
                role = rl;
            }
        }
        const float qt = fmaf(fy, A.z, fmaf(fx, A.y, A.x));
        const unsigned long long Q = pk2(qt, fmaf(16.f, A.y, qt));
        const unsigned long long CC = pk2(A.y, A.y);
        const unsigned base = __float_as_uint(A.w);
        // far corner: with |c| + |s| >= 1 its lowest ramp is always 1 (two ramps suffice)
        const bool far2 = FAR == 1 || (FAR == 0 && F.y >= 0.f);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const unsigned long long qa = h ? ffma2(pk2(32.f, 32.f), CC, Q) : Q;  // blocks 2h, 2h + 1
            const unsigned long long Rf = fadd2_rm(qa, MM);                      // magic + floor(q)
            const unsigned long long RB = fsub2(qa, fsub2(Rf, MM));              // r = q - floor(q)
            float v0, v1, rb[2];
            upk2(Rf, v0, v1);
            upk2(RB, rb[0], rb[1]);
            float4 T[2];
            T[0] = lds128(base + (__float_as_uint(v0) << 4));
            T[1] = lds128(base + (__float_as_uint(v1) << 4));
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                float(&q)[4] = acc[2 * h + e];
                const float r = rb[e];
                const float4 t = T[e];  // w g_j, w dg_j, w dg_{j+1}, w dg_{j+2}
                G[2 * h + e] += t.x;
                q[0] = fmaf(t.y, r, q[0]);
                q[1] = fmaf(t.z, add_sat(r, R2.y), fmaf(t.y, add_sat(r, R2.x), q[1]));
                q[2] = fmaf(t.z, add_sat(r, R2.w), fmaf(t.y, add_sat(r, R2.z), q[2]));
                if (far2)
                    q[3] = fmaf(t.w, add_sat(r, F.z), fmaf(t.z, add_sat(r, F.y), q[3] + t.y));
                else
                    q[3] = fmaf(t.w, add_sat(r, F.z), fmaf(t.z, add_sat(r, F.y), fmaf(t.y, add_sat(r, F.x), q[3])));
            }
        }
    };
    using True_ = std::integral_constant<bool, true>;
    using False_ = std::integral_constant<bool, false>;
    if (u & 4) {
        // every angle of the stage has the same corner roles: exchange once, no checks
        const int rl = u & 3;
        if (rl != role) {
#pragma unroll
            for (int a = 0; a < 4; ++a) xor_permute(acc[a], rl ^ role);
            role = rl;
        }
        if (u & 8) {
            for (int kk = 0; kk < kn; ++kk) angle(kk, False_(), std::integral_constant<int, 1>());
        } else {
            for (int kk = 0; kk < kn; ++kk) angle(kk, False_(), std::integral_constant<int, 2>());
        }
    } else {
        for (int kk = 0; kk < kn; ++kk) angle(kk, True_(), std::integral_constant<int, 0>());
    }
}

// The thread's 16 pixels, back in position order: pixel px + 2 py of block a has role
// (px + 2 py) ^ role.  Stored, added (accumulate) or added atomically (atomic_out).
__device__ __forceinline__ void quad_write(float (&acc)[4][4], const float (&G)[4], int role, float *__restrict__ img,
                                           int N, int tx, int ty, int X0, int Y0, int accumulate, int atomic_out) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        xor_permute(acc[a], role);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int x = tx * kTile + 2 * X0 + 16 * a + (r & 1);
            const int y = ty * kTile + 2 * Y0 + (r >> 1);
            if (x < N && y < N) {
                float *dst = img + (long long)y * N + x;
                const float val = acc[a][r] + G[a];
                if (atomic_out) atomicAdd(dst, val);
                else *dst = accumulate ? (*dst + val) : val;
            }
        }
    }
}

template <int STAGE = kStage>
struct QuadStageSmem {
    float4 sq[STAGE], sr[STAGE], sf[STAGE];
    int J0[STAGE];
    float w[STAGE];
    int u;
};

// 2 x 2-block form of direct_tile_sync (|c|, |s| <= 1): angles [k_begin, k_end) of tile
// (tx, ty) in stages of STAGE; each stage's float4 table (w g_j, w dg_j, w dg_{j+1},
// w dg_{j+2}) is built from global memory by kThreads / STAGE threads per angle, each a run of
// entries.  tab: STAGE * W float4 of shared memory.  All threads of the block must call it.
template <typename Tin, int STAGE = kStage>
__device__ __forceinline__ void direct_tile_quad_sync(const Tin *__restrict__ sino, float *__restrict__ img,
                                                      const AngleParam *__restrict__ ap, int N, int n_det,
                                                      int k_begin, int k_end, int W, int C, int tx, int ty,
                                                      int accumulate, int atomic_out, float wuni, float4 *tab,
                                                      QuadStageSmem<STAGE> &sm) {
    const int tid = threadIdx.x, warp = tid >> 5;
    int X0, Y0;
    quad_thread_blocks(tid, X0, Y0);
    float acc[4][4], G[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        G[a] = 0.f;
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[a][r] = 0.f;
    }
    int role = 0;
    const float fx = (float)(2 * X0), fy = (float)(2 * Y0);
    const unsigned tab_u32 = smem_u32(tab);
    constexpr int TPA = kThreads / STAGE;
    const int run = (W + TPA - 1) / TPA;
    for (int k0 = k_begin; k0 < k_end; k0 += STAGE) {
        const int kn = min(STAGE, k_end - k0);
        __syncthreads();  // the previous stage's table and parameters are no longer read
        if (warp == 0) {
            const bool act = tid < kn;
            int rl = 0;
            bool f2 = true;
            if (act) {
                const AngleParam p = ap[k0 + tid];
                const QuadAngle o = quad_angle(p, tx, ty, C, tab_u32 + (unsigned)(tid * W) * 16u);
                sm.sq[tid] = o.sq;
                sm.sr[tid] = o.sr;
                sm.sf[tid] = o.sf;
                sm.J0[tid] = o.J0;
                sm.w[tid] = wuni > 0.f ? wuni : p.w;
                rl = o.role;
                f2 = o.far2;
            }
            const int u = quad_uniform(act, rl, f2);
            if (tid == 0) sm.u = u;
        }
        __syncthreads();
        {
            const int kk = tid / TPA, r = tid % TPA;
            if (kk < kn) {
                const Tin *row = sino + (long long)(k0 + kk) * n_det;
                const int J0 = sm.J0[kk];
                const float w = sm.w[kk];
                float4 *dst = tab + kk * W;
                const int m0 = r * run, m1 = min(W, m0 + run);
                auto g_at = [&](int m) {
                    const int j = J0 + m;
                    return (j >= 0 && j < n_det) ? load_f(row + j) : 0.f;
                };
                if (m0 < m1) {
                    float g0 = g_at(m0), g1 = g_at(m0 + 1), g2 = g_at(m0 + 2);
                    float d0 = w * (g1 - g0), d1 = w * (g2 - g1);
                    for (int m = m0; m < m1; ++m) {
                        const float g3 = g_at(m + 3);
                        const float d2 = w * (g3 - g2);
                        dst[m] = make_float4(w * g0, d0, d1, d2);
                        g0 = g1;
                        g1 = g2;
                        g2 = g3;
                        d0 = d1;
                        d1 = d2;
                    }
                }
            }
        }
        __syncthreads();
        quad_stage(acc, G, role, sm.sq, sm.sr, sm.sf, sm.u, kn, fx, fy);
    }
    quad_write(acc, G, role, img, N, tx, ty, X0, Y0, accumulate, atomic_out);
}

}  // namespace bp
