// Direct R* (Section 2, eq "bp_app") for mirror-symmetric geometries: the four-image form.
//
// b(x_p) = sum_k w_k [ (1 - f) g_{k,j} + f g_{k,j+1} ],  u = x_p . xi_k / dt + (n_det-1)/2,
// j = floor(u), f = u - j, zero outside the detector.
//
// Symmetry (the four mirrors of the square: identity, x -> -x, y -> -y, and both).  With the
// pixel grid centred (N even) and the angle set closed under theta -> pi - theta (every uniform
// set is), the pixel P = (X, Y) at angle theta_k and
//   M_x P = (-X,  Y) at the partner angle theta_k' = pi - theta_k,
//   M_y P = ( X, -Y) at theta_k' with the detector read backwards,
//   -P         at theta_k  with the detector read backwards
// all sit at the same detector coordinate u (exactly, in the mathematics), because
// xi_k' = (-cos, sin) and reading a row backwards maps u to n_det - 1 - u.  So one thread owns a
// 2 x 2 pixel block of the quadrant X, Y < 0 and its three mirror images, computes the block's
// floor, fraction and clamped ramps once per angle, and applies them to all four images.  Every
// (pixel, angle) pair of the image is visited exactly once, because k -> k' is a bijection of
// the angle set.
//
// Arithmetic per block and angle is that of the 2 x 2-block form of direct.cu: with
// j = floor(u at the block's lowest corner) and r = u - j, the interpolants of the four pixels
// are  w g_j + sum_{i<3} w dg_{j+i} sat(r + offset_p - i)  with dg_j = g_{j+1} - g_j; the offsets
// depend only on (|c|, |s|), so the six clamped ramps serve all four images.  The images come in
// two pairs that each read one row forwards and backwards (row k: P and -P; row k': M_x P and
// M_y P); a row's table interleaves the forward and backward entries, so each pair is updated
// with paired f32x2 instructions whose operands arrive in adjacent registers.
//
// Tables.  One launch (klein_tables_kernel, or the row filter of the fused FBP) writes each row's
// entries once per call to a global workspace, over the bins any block can reach, for a chunk of
// slices at once (as many as a quarter of the free device memory holds).  The main kernel copies
// 48-entry windows of them (one per plane, row and angle: 768 bytes) into shared memory with
// cp.async.bulk, three stages of 8 angles in flight, so its block barriers and table builds
// disappear; the warps take turns issuing the copies of the stage two ahead.
//
// Schedule.  The quadrant is cut into 32 x 32-pixel regions (one 2 x 2 block per thread, 256
// threads), and the angles (in runs of 32 followed by their 32 partners) into S groups.  A
// persistent grid sweeps the chunk's slices and, within each, the groups in order; each group's
// (region, angle) pairs, region-major, are split evenly over all CTAs, so every CTA does the same
// amount of work and only one group's table rows are in use at a time (they stay in L2).  A CTA
// adds its partial sums with vector atomic adds whenever it leaves a region.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "direct_tile.cuh"
#include "tma.cuh"
#include "f32x2.cuh"
#include "filter_pt.cuh"

namespace bp {

namespace {

constexpr int kKRegion = 32;          // region side (pixels)
constexpr int kKThreads = 256;        // one 2 x 2 block per thread
constexpr int kKW = 48;               // table entries per region window: 31 (|c| + |s|) + 4 <= 48
constexpr int kKWin = kKW * 16;       // bytes of one window of one plane
constexpr int kKMargin = 4;           // extra table entries beyond the reachable bins

// Table of one row, forward and backward interleaved, in two planes of 16-byte entries: entry
// m (bin j = jlo + m) is (w g_j, w g'_j, w dg_j, w dg'_j) in plane 0 and (w dg_{j+1},
// w dg'_{j+1}, w dg_{j+2}, w dg'_{j+2}) in plane 1, g'_j = g_{n_det - 1 - j} the reversed row,
// dg_j = g_{j+1} - g_j, zero outside the detector: the two images that read a row (forwards and
// backwards) find their operands in adjacent registers of two 16-byte loads, and the loads of a
// quarter warp (8 consecutive entries of a plane) are free of bank conflicts.  One CTA per row r
// of a chunk of slices (angle k = r mod n_theta); the row is staged in shared memory with four
// zeros on each side.  A plane holds RS >= L + kKW entries, so a window copied from any reachable
// bin stays inside it; row r's planes start at entry 2 r RS.  zero (unless null): the chunk's
// images, N^2 / 4 float4 each, cleared for the main kernel's atomic adds, each row's CTA its
// share of its slice's image.
// The table entries m < L of one row (planes p0 and p0 + RS) from its values staged in shared
// memory at sr[4 + j] with four zeros on each side, weight w; by the CTA's threads.
__device__ __forceinline__ void klein_write_row(float4 *__restrict__ p0, const float *sr, int n_det, int jlo, int L,
                                                int RS, float w) {
    auto g = [&](int j) { return (j >= -4 && j < n_det + 4) ? sr[j + 4] : 0.f; };
    float4 *p1 = p0 + RS;
    for (int m = threadIdx.x; m < L; m += blockDim.x) {
        const int j = jlo + m, jr = n_det - 1 - j;
        const float a0 = g(j), a1 = g(j + 1), a2 = g(j + 2), a3 = g(j + 3);
        const float b0 = g(jr), b1 = g(jr - 1), b2 = g(jr - 2), b3 = g(jr - 3);
        p0[m] = make_float4(w * a0, w * b0, w * (a1 - a0), w * (b1 - b0));
        p1[m] = make_float4(w * (a2 - a1), w * (b2 - b1), w * (a3 - a2), w * (b3 - b2));
    }
}

template <typename Tin>
__global__ void __launch_bounds__(256)
klein_tables_kernel(const Tin *__restrict__ sino, float4 *__restrict__ tab, const AngleParam *__restrict__ ap,
                    int n_theta, int n_det, int jlo, int L, int RS, float wuni, float4 *__restrict__ zero, long long n4) {
    extern __shared__ float sg[];  // [n_det + 8]
    const long long r = blockIdx.x;
    const int k = (int)(r % n_theta);
    const Tin *row = sino + r * n_det;
    for (int i = threadIdx.x; i < n_det + 8; i += blockDim.x) {
        const int j = i - 4;
        sg[i] = (j >= 0 && j < n_det) ? load_f(row + j) : 0.f;
    }
    if (zero) {
        float4 *im = zero + (r / n_theta) * n4;
        const long long per = (n4 + n_theta - 1) / n_theta, z1 = min(n4, (k + 1) * per);
        for (long long i = k * per + threadIdx.x; i < z1; i += blockDim.x) im[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    klein_write_row(tab + 2 * r * RS, sg, n_det, jlo, L, RS, wuni > 0.f ? wuni : ap[k].w);
}

// Mixed batches (bp_backproject_batched): one CTA per row of every slice (rows d.row0 ..
// d.row0 + n_theta - 1 of slice d), each slice's own geometry, element type and table block; a
// row's CTA also clears its share of the slice's image (the main kernel adds into it).
struct KleinTabSlice {
    const void *sino;
    float4 *tab;
    const AngleParam *ap;
    float4 *img;
    int N, n_det, n_theta, jlo, L, RS, dtype, row0;
};
struct KleinTabBatch {
    KleinTabSlice d[256];
    int n;
};
static_assert(sizeof(KleinTabBatch) <= 31 * 1024, "kernel parameter block too large");

__device__ __forceinline__ float load_any(const void *p, int dtype, long long i) {
    if (dtype == BP_BF16) return load_f((const __nv_bfloat16 *)p + i);
    if (dtype == BP_F16) return load_f((const __half *)p + i);
    return load_f((const float *)p + i);
}

__global__ void __launch_bounds__(256) klein_tables_mixed_kernel(const __grid_constant__ KleinTabBatch tb) {
    extern __shared__ float sg[];  // [max n_det + 8]
    const int r = blockIdx.x;
    int lo = 0, hi = tb.n - 1;  // the last slice with row0 <= r
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tb.d[mid].row0 <= r) lo = mid;
        else hi = mid - 1;
    }
    const KleinTabSlice &d = tb.d[lo];
    const int k = r - d.row0, n_det = d.n_det;
    const long long base = (long long)k * n_det;
    for (int i = threadIdx.x; i < n_det + 8; i += blockDim.x) {
        const int j = i - 4;
        sg[i] = (j >= 0 && j < n_det) ? load_any(d.sino, d.dtype, base + j) : 0.f;
    }
    const long long n4 = (long long)d.N * d.N / 4, per = (n4 + d.n_theta - 1) / d.n_theta;
    const long long z1 = min(n4, (k + 1) * per);
    for (long long i = k * per + threadIdx.x; i < z1; i += blockDim.x) d.img[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    klein_write_row(d.tab + 2LL * k * d.RS, sg, n_det, d.jlo, d.L, d.RS, __ldg(&d.ap[k].w));
}

// The fused FBP form of the tables: the persistent row filter of filter_pt.cuh turns each row
// pair into its filtered values in shared memory, and the pair's table entries (the layout of
// klein_tables_kernel, the same arithmetic on the same values) are written from there, so the
// filtered sinogram never goes through global memory.  Rows r of a chunk of slices, angle
// k = r mod n_theta.
struct KleinTabOut {
    static constexpr bool kStaged = true;
    float4 *tab;
    const AngleParam *ap;
    int n_theta, jlo, L, RS;
    float wuni;
    __device__ __forceinline__ void rows(const float *sg, long long r0, bool has1, int n_det) const {
        for (int h = 0; h < 2; ++h) {
            if (h == 1 && !has1) break;
            const long long r = r0 + h;
            klein_write_row(tab + 2 * r * RS, sg + h * (n_det + 8), n_det, jlo, L, RS,
                            wuni > 0.f ? wuni : ap[r % n_theta].w);
        }
    }
};

// rows: the chunk's rows; zero: the chunk's images (n4 float4), cleared here for the main
// kernel's atomic adds (null when it accumulates), in place of a memset launch.
template <typename Tin, int LOGP>
__global__ void __launch_bounds__((1 << LOGP) / kPassE, 1024 / ((1 << LOGP) / kPassE))
klein_filter_tables_kernel(const Tin *__restrict__ sino, KleinTabOut out, const float *__restrict__ H,
                           const float2 *__restrict__ twp, long long rows, int n_det, float4 *__restrict__ zero,
                           long long n4) {
    if (zero)
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x)
            zero[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    filter_pt_body<Tin, LOGP>(sino, out, H, twp, rows, n_det);
}

// Add (or store) two horizontally adjacent pixels; x even, so the pair is 8-byte aligned.
__device__ __forceinline__ void put_pair(float *__restrict__ p, float a, float b, bool both, int mode) {
    if (both) {
        float2 *q = reinterpret_cast<float2 *>(p);
        if (mode == 0) *q = make_float2(a, b);
        else atomicAdd(q, make_float2(a, b));
    } else {
        if (mode == 0) *p = a;
        else atomicAdd(p, a);
    }
}

// Per schedule slot (angles ordered so that each angle and its mirror partner are adjacent):
// the pixel coordinate tables of direct.cu (u of pixel (0, 0) and its steps per pixel in 32.32
// fixed point), the row k of the slot's angle and its partner k' | (d << 31), d = 1 when row k'
// must be read backwards for the x-mirror image.
struct KleinAngle {
    long long U00, CP, SP;
    float c, s;
    unsigned partner;
    int row;
};
static_assert(sizeof(KleinAngle) == 40, "KleinAngle layout");

__device__ __forceinline__ float sat_add(float a, float b) { return __saturatef(a + b); }

// v[i] <- v[i ^ m] over the four corner roles (bit 0: x flipped, bit 1: y flipped).
__device__ __forceinline__ void xor_permute2(unsigned long long (&v)[4], int m) {
    if (m & 1) {
        unsigned long long t = v[0]; v[0] = v[1]; v[1] = t;
        t = v[2]; v[2] = v[3]; v[3] = t;
    }
    if (m & 2) {
        unsigned long long t = v[0]; v[0] = v[2]; v[2] = t;
        t = v[1]; v[1] = v[3]; v[3] = t;
    }
}

__device__ __forceinline__ unsigned long long swap2(unsigned long long v) {
    float a, b;
    upk2(v, a, b);
    return pk2(b, a);
}

// The thread's block and its three images, as two image pairs that each read one row:
// pair A = (image 0, image -P) reads row k forwards and backwards, pair B = (image M_x, image
// M_y) reads row k' (halves exchanged while the stage's rows k' run backwards, dir = 1).
struct KleinAcc {
    unsigned long long a[4], b[4];  // per corner role: (sum for the pair's first image, second image)
    unsigned long long ga, gb;      // the common w g_j terms
};

// One row's contribution to an image pair: x0 = (G, G', D0, D0'), x1 = (D1, D1', D2, D2').
template <bool FAR2>
__device__ __forceinline__ void klein_row(const ulonglong2 x0, const ulonglong2 x1, unsigned long long (&q)[4],
                                          unsigned long long &gsum, unsigned long long R2, unsigned long long S1a,
                                          unsigned long long S1b, unsigned long long S2a, unsigned long long S2b,
                                          unsigned long long S3a, unsigned long long S3b, unsigned long long S3c) {
    gsum = fadd2(gsum, x0.x);
    q[0] = ffma2(x0.y, R2, q[0]);
    q[1] = ffma2(x1.x, S1b, ffma2(x0.y, S1a, q[1]));
    q[2] = ffma2(x1.x, S2b, ffma2(x0.y, S2a, q[2]));
    if (FAR2) q[3] = ffma2(x1.y, S3b, ffma2(x1.x, S3a, fadd2(q[3], x0.y)));
    else q[3] = ffma2(x1.y, S3b, ffma2(x1.x, S3a, ffma2(x0.y, S3c, q[3])));
}

// Exchange the accumulators of `n` blocks when the corner roles or the row-k' direction of the
// next angle (w = role | dir << 2) differ from the current ones.
template <int BPT>
__device__ __forceinline__ void klein_roles(int w, KleinAcc (&acc)[BPT], int &role, int &dir) {
    const int rl = w & 3, dr = (w >> 2) & 1;
    if (rl != role) {
#pragma unroll
        for (int h = 0; h < BPT; ++h) {
            xor_permute2(acc[h].a, rl ^ role);
            xor_permute2(acc[h].b, rl ^ role);
        }
        role = rl;
    }
    if (dr != dir) {
#pragma unroll
        for (int h = 0; h < BPT; ++h) {
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[h].b[i] = swap2(acc[h].b[i]);
            acc[h].gb = swap2(acc[h].gb);
        }
        dir = dr;
    }
}

// One angle for one block and its three images: FAR = 0 per-angle far-corner test, 1 two ramps
// (|c| + |s| >= 1), 2 three ramps.  A = (q0, c, s, role | dir << 2), O = (|c| - 1, |s| - 1,
// |c| + |s| - 1, |c| + |s| - 2); tabs[wi]: the first entry of the angle's window in row k's plane
// 0; row k's plane 1 and row k''s planes 0 and 1 follow STG windows apart.
template <int FAR, int STG>
__device__ __forceinline__ void klein_angle(const float4 A, const float4 O, const ulonglong2 *__restrict__ tabs, int wi,
                                            KleinAcc &acc, float fx, float fy) {
    const float qt = fmaf(fy, A.z, fmaf(fx, A.y, A.x));
    const float v = __fadd_rd(qt, kMagic);  // magic + floor(qt)
    const float r = qt - (v - kMagic);       // r = qt - floor(qt)
    const int e = wi + (int)(__float_as_uint(v) - kMagicBits);
    const bool far2 = FAR == 1 || (FAR == 0 && O.z >= 0.f);
    const float s1a = sat_add(r, fabsf(A.y)), s1b = sat_add(r, O.x);
    const float s2a = sat_add(r, fabsf(A.z)), s2b = sat_add(r, O.y);
    const float s3a = sat_add(r, O.z), s3b = sat_add(r, O.w);
    const float s3c = far2 ? 1.f : sat_add(r, O.z + 1.f);
    constexpr int P = STG * kKW;
    const ulonglong2 a0 = tabs[e], a1 = tabs[e + P];
    const ulonglong2 b0 = tabs[e + 2 * P], b1 = tabs[e + 3 * P];
    const unsigned long long R2 = pk2(r, r), S1a = pk2(s1a, s1a), S1b = pk2(s1b, s1b), S2a = pk2(s2a, s2a),
                             S2b = pk2(s2b, s2b), S3a = pk2(s3a, s3a), S3b = pk2(s3b, s3b), S3c = pk2(s3c, s3c);
    // FAR 0 and 2 take the three-ramp form; with S3c = 1 (a far corner at |c| + |s| >= 1) it
    // equals the two-ramp form exactly (fma(x, 1, q) = q + x)
    klein_row<FAR == 1>(a0, a1, acc.a, acc.ga, R2, S1a, S1b, S2a, S2b, S3a, S3b, S3c);
    klein_row<FAR == 1>(b0, b1, acc.b, acc.gb, R2, S1a, S1b, S2a, S2b, S3a, S3b, S3c);
}

// The CTA's sequence of stages (of one slice): for each angle group g in turn (all CTAs sweep the
// groups in the same order, so only one group's table rows are in use at a time), its share of
// the group's (region, slot) pairs, region-major, in stages of at most STG slots that never
// cross a region.
template <int STG>
struct StageSeq {
    int g, u, u1, Ag, k_a;
    int rg, off;  // region of position u and u - rg Ag (kept without division)
    __device__ void enter(int grp, int S, int n_theta, int R, int cta, int G) {
        g = grp;
        k_a = (int)((long long)g * n_theta / S);
        Ag = (int)((long long)(g + 1) * n_theta / S) - k_a;
        const long long work = (long long)R * Ag;  // < 2^31 (checked on the host)
        u = (int)(work * cta / G);
        u1 = (int)(work * (cta + 1) / G);
        rg = Ag > 0 ? u / Ag : 0;
        off = u - rg * Ag;
    }
    __device__ bool next(int &r, int &k0, int &kn, bool &last, int S, int n_theta, int R, int cta, int G) {
        while (u >= u1) {
            if (g + 1 >= S) return false;
            enter(g + 1, S, n_theta, R, cta, G);
        }
        r = rg;
        k0 = k_a + off;
        kn = min(STG, min(u1 - u, Ag - off));
        u += kn;
        off += kn;
        last = u >= u1 || off == Ag;
        if (off == Ag) {
            ++rg;
            off = 0;
        }
        return true;
    }
};

// Per-slice geometry of the persistent kernel, by slice index: the slices of one plan (tables and
// images at fixed strides) or of several plans (one descriptor each, bp_backproject_batched).
struct KleinGeoSame {
    const KleinAngle *ka_;
    const float4 *tab_;
    float *img_;
    int N_, n_theta_, RS_, jlo_, nr_, S_, batch_;
    long long img_stride_, tab_stride_;
    __device__ __forceinline__ const KleinAngle *ka(int) const { return ka_; }
    __device__ __forceinline__ const float4 *tab(int sl) const { return tab_ + sl * tab_stride_; }
    __device__ __forceinline__ float *img(int sl) const { return img_ + sl * img_stride_; }
    __device__ __forceinline__ int N(int) const { return N_; }
    __device__ __forceinline__ int n_theta(int) const { return n_theta_; }
    __device__ __forceinline__ int RS(int) const { return RS_; }
    __device__ __forceinline__ int jlo(int) const { return jlo_; }
    __device__ __forceinline__ int nr(int) const { return nr_; }
    __device__ __forceinline__ int S(int) const { return S_; }
    __device__ __forceinline__ int batch() const { return batch_; }
};
struct KleinSlice {
    const KleinAngle *ka;
    const float4 *tab;
    float *img;
    int N, n_theta, RS, jlo, nr, S;
};
constexpr int kKMaxSlices = 256;  // descriptors per launch (larger batches take several)
struct KleinGeoMixed {
    KleinSlice d[kKMaxSlices];
    int n;
    __device__ __forceinline__ const KleinAngle *ka(int sl) const { return d[sl].ka; }
    __device__ __forceinline__ const float4 *tab(int sl) const { return d[sl].tab; }
    __device__ __forceinline__ float *img(int sl) const { return d[sl].img; }
    __device__ __forceinline__ int N(int sl) const { return d[sl].N; }
    __device__ __forceinline__ int n_theta(int sl) const { return d[sl].n_theta; }
    __device__ __forceinline__ int RS(int sl) const { return d[sl].RS; }
    __device__ __forceinline__ int jlo(int sl) const { return d[sl].jlo; }
    __device__ __forceinline__ int nr(int sl) const { return d[sl].nr; }
    __device__ __forceinline__ int S(int sl) const { return d[sl].S; }
    __device__ __forceinline__ int batch() const { return n; }
};
static_assert(sizeof(KleinGeoMixed) <= 31 * 1024, "kernel parameter block too large");

// A persistent grid (the schedule in the header) over geo.batch() slices, slice sl's tables at
// geo.tab(sl) and its image at geo.img(sl).  The warps take turns as producer:
// after finishing stage s, warp s mod 8 copies the windows of stage s - 1 + NBUF (cp.async.bulk,
// 768 bytes per image) from the row tables into the buffer of stage s - 1, once every warp has
// left it.  img is added to atomically (cleared before unless accumulating).  Every wait is
// bounded: on expiry the kernel sets *err, waits (bounded) for the copies it issued and returns.
// MULTI false: one slice (batch 1), without the slice bookkeeping.
template <int MINB, int NBUF, int BPT, int STG, bool MULTI, typename Geo>
__global__ void __launch_bounds__(kKThreads / BPT, MINB)
bp_direct_klein_kernel(const __grid_constant__ Geo geo, int *__restrict__ err) {
    // [NBUF][row k, row k'][plane 0, 1][STG][kKW] entries of 16 bytes
    extern __shared__ __align__(128) ulonglong2 ktab[];
    __shared__ float4 prmA[NBUF][STG], prmO[NBUF][STG];
    __shared__ int prmU[NBUF];  // stage uniformity: role | dir << 2 | 8 when all agree, | 16 when all far corners take two ramps
    __shared__ __align__(8) unsigned long long full[NBUF], empty[NBUF];
    constexpr int NW = kKThreads / BPT / 32;  // warps per CTA
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, qtr = lane >> 3;
    // a warp's blocks h -> 16 x 8 pixels, a quarter warp's -> 8 x 4 pixels (its table entries lie
    // within 8 consecutive bins); block h's origin inside the region is (2 bx + 16 h, 2 by)
    const int bx = (lane & 3) + 4 * (qtr & 1) + (BPT == 1 ? 8 * (warp & 1) : 0);
    const int by = ((lane >> 2) & 1) + 2 * (qtr >> 1) + 4 * (BPT == 1 ? warp >> 1 : warp);
    const float fx = (float)(2 * bx), fy = (float)(2 * by);
    const int cta = blockIdx.x, nctas = gridDim.x;
    auto regions = [&](int sl) { return geo.nr(sl) * geo.nr(sl); };
    StageSeq<STG> cons;
    cons.enter(0, geo.S(0), geo.n_theta(0), regions(0), cta, nctas);
    StageSeq<STG> prod = cons;
    const unsigned tab_u32 = smem_u32(ktab);
    const uint32_t fb = smem_u32(&full[0]), eb = smem_u32(&empty[0]);
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < NBUF; ++i) {
            mbar_init(fb + 8 * i, 1);
            mbar_init(eb + 8 * i, NW);
        }
        mbar_fence_init();
    }
    __syncthreads();

    // the producer's next stage (of slice psl; the sequence runs on into the next slice without
    // a break): every warp advances the producer's position; the warp that issues (`issue`)
    // writes the stage's parameters and copies its windows into buffer b
    int pstage = 0, psl = 0;
    auto produce = [&](bool issue) -> bool {
        int rg, k0, kn;
        bool last;
        while (!prod.next(rg, k0, kn, last, geo.S(psl), geo.n_theta(psl), regions(psl), cta, nctas)) {
            if (!MULTI || psl + 1 >= geo.batch()) return false;
            ++psl;
            prod.enter(0, geo.S(psl), geo.n_theta(psl), regions(psl), cta, nctas);
        }
        const int b = pstage % NBUF;
        ++pstage;
        if (!issue) return true;
        const int nr = geo.nr(psl), rx = rg % nr, ry = rg / nr;
        const float4 *src0 = nullptr, *src1 = nullptr;
        int w = 0;
        bool f2 = true;
        if (lane < kn) {
            const int kk = lane;
            const KleinAngle a = geo.ka(psl)[k0 + kk];
            const long long U = a.U00 + (long long)(kKRegion * rx) * a.CP + (long long)(kKRegion * ry) * a.SP;
            const int Ji = (int)(U >> 32);
            const float frac = (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f;
            const float lo = fminf(a.c, 0.f) + fminf(a.s, 0.f);
            const int J0 = Ji + (int)floorf((float)(kKRegion - 1) * lo) - 1;
            const int kp = (int)(a.partner & 0x7fffffffu), d = (int)(a.partner >> 31);
            w = ((a.c < 0.f ? 1 : 0) | (a.s < 0.f ? 2 : 0)) | (d << 2);
            const float ac = fabsf(a.c), as = fabsf(a.s), af = ac + as;
            f2 = af - 1.f >= 0.f;
            prmA[b][kk] = make_float4((float)(Ji - J0) + frac + lo, a.c, a.s, __int_as_float(w));
            prmO[b][kk] = make_float4(ac - 1.f, as - 1.f, af - 1.f, af - 2.f);
            const float4 *ts = geo.tab(psl);
            const int RS = geo.RS(psl), jlo = geo.jlo(psl);
            src0 = ts + 2 * (long long)a.row * RS + (J0 - jlo);
            src1 = ts + 2 * (long long)kp * RS + (J0 - jlo);
        }
        const bool act = lane < kn;
        const int w0 = __shfl_sync(0xffffffffu, w, 0);
        const bool same = __all_sync(0xffffffffu, !act || w == w0);
        const bool all2 = __all_sync(0xffffffffu, !act || f2);
        if (lane == 0) prmU[b] = same ? (w0 | 8 | (all2 ? 16 : 0)) : 0;
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            mbar_expect_tx(fb + 8 * b, (uint32_t)(kn * 4 * kKWin));
        }
        __syncwarp();
        if (act) {
            // the angle's four 768-byte windows: rows k and k', planes 0 and 1
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 *src = (q < 2 ? src0 : src1) + (q & 1) * (long long)geo.RS(psl);
                const unsigned dst = tab_u32 + (unsigned)(((b * 4 + q) * STG + lane) * kKWin);
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                    ::"r"(dst), "l"(src), "r"((uint32_t)kKWin), "r"(fb + 8 * b)
                    : "memory");
            }
        }
        return true;
    };

    bool ok = true;
    int issued = 0;
    KleinAcc acc[BPT];
    auto clear = [&]() {
#pragma unroll
        for (int h = 0; h < BPT; ++h) {
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[h].a[i] = acc[h].b[i] = 0ull;
            acc[h].ga = acc[h].gb = 0ull;
        }
    };
    int role = 0, dir = 0, cstage = 0, b = 0;
    uint32_t ph = 0;
    prod = cons;
#pragma unroll
    for (int i = 0; i < NBUF; ++i) issued += produce(warp == 0) ? 1 : 0;
    clear();
    int sst = 0;  // stages consumed
    int csl = 0;  // the consumer's slice
    float *im = geo.img(0);
    int rg, k0, kn;
    bool last;
    for (;;) {
        if (!cons.next(rg, k0, kn, last, geo.S(csl), geo.n_theta(csl), regions(csl), cta, nctas)) {
            if (!MULTI || csl + 1 >= geo.batch()) break;
            ++csl;
            im = geo.img(csl);
            cons.enter(0, geo.S(csl), geo.n_theta(csl), regions(csl), cta, nctas);
            continue;
        }
        if (!mbar_wait(fb + 8 * b, ph)) {
            ok = false;
            break;
        }
        const int uw = prmU[b];
        const int wb = b * 4 * STG * kKW;  // row k's plane-0 windows of this stage (entries)
        if (uw & 8) {
            klein_roles<BPT>(uw & 7, acc, role, dir);
            if (uw & 16) {
#pragma unroll(2 * BPT)
                for (int kk = 0; kk < kn; ++kk) {
                    const float4 A = prmA[b][kk], O = prmO[b][kk];
#pragma unroll
                    for (int h = 0; h < BPT; ++h)
                        klein_angle<1, STG>(A, O, ktab, wb + kk * kKW, acc[h], fx + (float)(16 * h), fy);
                }
            } else {
#pragma unroll(2 * BPT)
                for (int kk = 0; kk < kn; ++kk) {
                    const float4 A = prmA[b][kk], O = prmO[b][kk];
#pragma unroll
                    for (int h = 0; h < BPT; ++h)
                        klein_angle<2, STG>(A, O, ktab, wb + kk * kKW, acc[h], fx + (float)(16 * h), fy);
                }
            }
        } else {
            for (int kk = 0; kk < kn; ++kk) {
                const float4 A = prmA[b][kk], O = prmO[b][kk];
                klein_roles<BPT>(__float_as_int(A.w), acc, role, dir);
#pragma unroll
                for (int h = 0; h < BPT; ++h)
                    klein_angle<0, STG>(A, O, ktab, wb + kk * kKW, acc[h], fx + (float)(16 * h), fy);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(eb + 8 * b);
        if (sst++ >= 1) {
            // refill the buffer of stage cstage - 1 with stage cstage - 1 + NBUF; the warps take
            // turns, and the issuing warp has finished the stage after it, so every warp has
            // almost surely left the buffer
            const bool mine = warp == cstage % NW;
            if (mine) {
                const int bp = b == 0 ? NBUF - 1 : b - 1;
                const uint32_t pp = b == 0 ? ph ^ 1u : ph;
                if (!mbar_wait(eb + 8 * bp, pp)) {
                    ok = false;
                    break;
                }
            }
            issued += produce(mine) ? 1 : 0;
        }
        ++cstage;
        if (++b == NBUF) {
            b = 0;
            ph ^= 1u;
        }
        if (last) {
            // flush: pixel px + 2 py of a block has role (px + 2 py) ^ role; pair A holds images 0
            // and -P, pair B images M_x and M_y (exchanged while dir = 1)
            const int nr = geo.nr(csl), rx = rg % nr, ry = rg / nr;
            const int N = geo.N(csl), h2 = N / 2;
            const int iy = kKRegion * ry + 2 * by;
#pragma unroll
            for (int h = 0; h < BPT; ++h) {
                KleinAcc &ac = acc[h];
                const int ix = kKRegion * rx + 2 * bx + 16 * h;
                const bool x1 = ix + 1 < h2;
                xor_permute2(ac.a, role);
                xor_permute2(ac.b, role);
                if (ix >= h2) continue;
                float ga0, ga3, gb1, gb2;
                upk2(ac.ga, ga0, ga3);
                upk2(ac.gb, gb1, gb2);
                if (dir) {
                    const float t = gb1; gb1 = gb2; gb2 = t;
                }
#pragma unroll
                for (int py = 0; py < 2; ++py) {
                    if (iy + py >= h2) continue;
                    float i0[2], i3[2], i1[2], i2[2];
#pragma unroll
                    for (int px = 0; px < 2; ++px) {
                        upk2(ac.a[2 * py + px], i0[px], i3[px]);
                        upk2(ac.b[2 * py + px], i1[px], i2[px]);
                        if (dir) {
                            const float t = i1[px]; i1[px] = i2[px]; i2[px] = t;
                        }
                        i0[px] += ga0; i3[px] += ga3; i1[px] += gb1; i2[px] += gb2;
                    }
                    const int y = iy + py, ym = N - 1 - (iy + py);
                    put_pair(im + (long long)y * N + ix, i0[0], i0[1], x1, 1);
                    put_pair(im + (long long)ym * N + ix, i2[0], i2[1], x1, 1);
                    // x-mirrored: base pixels ix, ix + 1 land at N - 1 - ix, N - 2 - ix
                    if (x1) {
                        put_pair(im + (long long)y * N + (N - 2 - ix), i1[1], i1[0], true, 1);
                        put_pair(im + (long long)ym * N + (N - 2 - ix), i3[1], i3[0], true, 1);
                    } else {
                        put_pair(im + (long long)y * N + (N - 1 - ix), i1[0], 0.f, false, 1);
                        put_pair(im + (long long)ym * N + (N - 1 - ix), i3[0], 0.f, false, 1);
                    }
                }
            }
            clear();
        }
    }
    if (!ok) {
        // wait (bounded) for the copies still in flight: stages cstage .. issued - 1
        if (lane == 0) atomicExch(err, 1);
        for (int s2 = cstage; s2 < issued; ++s2) mbar_wait(fb + 8 * (s2 % NBUF), (uint32_t)((s2 / NBUF) & 1));
    }
}

}  // namespace

// Host check at plan creation (FP64, no device work): N even, pixels no larger than bins, and
// every angle has a mirror partner theta_k' = pi - theta_k (mod pi) such that k -> k' is a
// bijection; fills p->klein (partners, per-angle table on the host, table extent).
void klein_plan(bp_plan *p) {
    KleinWork &kw = p->klein;
    kw = KleinWork();
    const int n = p->n_theta, N = p->N;
    if (N % 2 != 0 || !(p->step_max <= 1.0f)) return;
    std::vector<std::pair<double, int>> a(n);
    for (int k = 0; k < n; ++k) {
        double t = std::fmod(p->theta[k], M_PI);
        if (t < 0) t += M_PI;
        a[k] = {t, k};
    }
    std::sort(a.begin(), a.end());
    const double tol = 1e-10;
    std::vector<unsigned> partner(n);
    std::vector<int> used(n, 0);
    for (int k = 0; k < n; ++k) {
        double t = M_PI - std::fmod(std::fmod(p->theta[k], M_PI) + M_PI, M_PI);
        if (t >= M_PI) t -= M_PI;
        // nearest sorted angle, distance taken modulo pi
        auto it = std::lower_bound(a.begin(), a.end(), std::make_pair(t, -1));
        int best = -1;
        double bd = 1e300;
        for (int cand : {(int)(it - a.begin()) - 1, (int)(it - a.begin()), 0, n - 1}) {
            if (cand < 0 || cand >= n) continue;
            double d = std::fabs(a[cand].first - t);
            d = std::min(d, M_PI - d);
            if (d < bd) {
                bd = d;
                best = a[cand].second;
            }
        }
        if (best < 0 || bd > tol) return;
        // direction of row k' against the x-mirror (-cos, sin) of angle k: same -> forwards
        const double ck = std::cos(p->theta[k]), sk = std::sin(p->theta[k]);
        const double cp = std::cos(p->theta[best]), sp = std::sin(p->theta[best]);
        const double dot = -cp * ck + sp * sk;
        if (std::fabs(std::fabs(dot) - 1.0) > 1e-9) return;
        partner[k] = (unsigned)best | (dot < 0 ? 0x80000000u : 0u);
        if (used[best]++) return;
    }
    const double r = p->dx / p->dt;
    const int nr = (N / 2 + kKRegion - 1) / kKRegion;
    // a region's window must fit kKW entries (|c| + |s| <= sqrt 2, pixels no larger than bins),
    // and the schedule's (region, angle) counter stays below 2^31
    if (r > 1.0 + 1e-12 || (double)nr * nr * n >= 2147483647.0) return;
    const double E = (double)(kKRegion * nr - 1);
    double umin = 1e300, umax = -1e300;
    std::vector<KleinAngle> ka(n);
    for (int k = 0; k < n; ++k) {
        const double c = std::cos(p->theta[k]) * r, s = std::sin(p->theta[k]) * r;
        const double u00 = c * (0.5 - 0.5 * N) + s * (0.5 - 0.5 * N) + 0.5 * (p->n_det - 1);
        ka[k].U00 = std::llround(std::ldexp(u00, 32));
        ka[k].CP = std::llround(std::ldexp(c, 32));
        ka[k].SP = std::llround(std::ldexp(s, 32));
        ka[k].c = (float)c;
        ka[k].s = (float)s;
        ka[k].partner = partner[k];
        ka[k].row = k;
        umin = std::min(umin, u00 + std::min(0.0, c * E) + std::min(0.0, s * E));
        umax = std::max(umax, u00 + std::max(0.0, c * E) + std::max(0.0, s * E));
    }
    // schedule slots: runs of 32 angles followed by their 32 partners, so that an angle group
    // touches the rows of its own angles only while the corner roles (signs of cos, sin) stay the
    // same over whole stages
    std::vector<KleinAngle> slots;
    std::vector<int> run_a, run_b;
    std::vector<char> seen(n, 0);
    auto close_run = [&]() {
        for (int k : run_a) slots.push_back(ka[k]);
        for (int k : run_b) slots.push_back(ka[k]);
        run_a.clear();
        run_b.clear();
    };
    for (int k = 0; k < n; ++k) {
        if (seen[k]) continue;
        seen[k] = 1;
        run_a.push_back(k);
        const int kp = (int)(partner[k] & 0x7fffffffu);
        if (!seen[kp]) {
            seen[kp] = 1;
            run_b.push_back(kp);
        }
        if ((int)run_a.size() == 32) close_run();
    }
    close_run();
    ka.swap(slots);
    kw.jlo = (int)std::floor(umin) - kKMargin;
    kw.L = (int)std::floor(umax) + kKMargin - kw.jlo + 1;
    kw.nr = nr;
    kw.host.resize(sizeof(KleinAngle) * n);
    std::memcpy(kw.host.data(), ka.data(), kw.host.size());
    kw.eligible = true;
}

void free_klein(bp_plan *p) {
    cudaFree(p->klein.d_ang);
    cudaFree(p->klein.tab);
    cudaFree(p->klein.mix_tab);
    p->klein.d_ang = nullptr;
    p->klein.tab = nullptr;
    p->klein.tab_slices = 0;
    p->klein.mix_tab = nullptr;
    p->klein.mix_bytes = 0;
}

// Default angle groups: about one per 96 MB of row tables, so that one group's rows mostly stay
// in L2 (measured at 2048^2 x 1800: two groups best; more add partial-sum flushes).
int klein_default_groups(const bp_plan *p) {
    const double bytes = 2.0 * 16.0 * p->n_theta * (double)(p->klein.L + kKW);
    const int S = (int)std::ceil(bytes / (96.0 * 1024 * 1024));
    return std::max(1, std::min(std::min(S, 64), p->n_theta));
}

int klein_clamp_groups(const bp_plan *p, int S) { return std::max(1, std::min(std::min(S, 64), p->n_theta)); }

namespace {

// Row tables of `n` slices (rows r = 0 .. n n_theta - 1) into the workspace; their images cleared
// on the way when `zero` is given.
template <typename Tin>
bp_status klein_tables(bp_plan *p, const Tin *sino, int n, cudaStream_t st, float wuni, float *zero) {
    const size_t smem = sizeof(float) * ((size_t)p->n_det + 8);
    auto kern = klein_tables_kernel<Tin>;
    if (smem > 48 * 1024) BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)(n * p->n_theta), 256, smem, st>>>(sino, p->klein.tab, p->d_ang, p->n_theta, p->n_det,
                                                        p->klein.jlo, p->klein.L, p->klein.L + kKW, wuni,
                                                        (float4 *)zero, (long long)p->N * p->N / 4);
    BP_CUDA_TRY(cudaGetLastError());
    stage_mark(p, st, "klein_tables_kernel");
    return BP_OK;
}

// The fused form: the rows of `n` slices filtered (response H) into their tables; their images
// cleared on the way when `zero` is given.
template <typename Tin, int LOGP>
bp_status klein_filter_tables_p(bp_plan *p, const Tin *sino, int n, const float *H, cudaStream_t st, float wuni,
                                float *zero) {
    constexpr int NT = (1 << LOGP) / kPassE;
    constexpr size_t smem = filter_pt_smem<LOGP>();
    auto kern = klein_filter_tables_kernel<Tin, LOGP>;
    static int per_sm = 0;
    if (!per_sm) {
        BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    }
    const long long rows = (long long)n * p->n_theta, npairs = (rows + 1) / 2;
    const long long grid = std::max(1LL, std::min(npairs, (long long)std::max(1, per_sm) * std::max(1, p->sm_count)));
    const KleinWork &kw = p->klein;
    kern<<<(unsigned)grid, NT, smem, st>>>(sino, KleinTabOut{kw.tab, p->d_ang, p->n_theta, kw.jlo, kw.L, kw.L + kKW,
                                                             wuni},
                                           H, p->d_twpass, rows, p->n_det, (float4 *)zero,
                                           zero ? (long long)n * p->N * p->N / 4 : 0LL);
    BP_CUDA_TRY(cudaGetLastError());
    stage_mark(p, st, "klein_filter_tables_kernel");
    return BP_OK;
}

template <typename Tin>
bp_status klein_filter_tables(bp_plan *p, const Tin *sino, int n, const float *H, cudaStream_t st, float wuni,
                              float *zero) {
    switch (ilog2(p->P)) {
        case 9: return klein_filter_tables_p<Tin, 9>(p, sino, n, H, st, wuni, zero);
        case 10: return klein_filter_tables_p<Tin, 10>(p, sino, n, H, st, wuni, zero);
        case 11: return klein_filter_tables_p<Tin, 11>(p, sino, n, H, st, wuni, zero);
        default: return klein_filter_tables_p<Tin, 12>(p, sino, n, H, st, wuni, zero);
    }
}

size_t klein_slice_bytes(const bp_plan *p) {
    return 2 * sizeof(float4) * (size_t)p->n_theta * (size_t)(p->klein.L + kKW);
}

}  // namespace

// bp_set_direct_workspace: the new bound; tables above it are released now.
bp_status klein_set_workspace(bp_plan *p, size_t bytes) {
    KleinWork &kw = p->klein;
    kw.tab_limit = bytes;
    if (kw.tab && bytes && klein_slice_bytes(p) * (size_t)kw.tab_slices > bytes) {
        BP_CUDA_TRY(cudaDeviceSynchronize());  // no call of this plan may still read the tables
        cudaFree(kw.tab);
        kw.tab = nullptr;
        kw.tab_slices = 0;
    }
    return BP_OK;
}

namespace {

// The per-slot angle records, uploaded on first use.
bp_status klein_upload(bp_plan *p) {
    KleinWork &kw = p->klein;
    if (!kw.d_ang) {
        BP_CUDA_TRY(cudaMalloc(&kw.d_ang, kw.host.size()));
        BP_CUDA_TRY(cudaMemcpy(kw.d_ang, kw.host.data(), kw.host.size(), cudaMemcpyHostToDevice));
    }
    return BP_OK;
}

// Slices whose tables the workspace holds at once for a call of `batch` slices: all of them
// while they fit the budget (the bp_set_direct_workspace bound, else a quarter of the device
// memory free when the workspace grows), else as many as the budget holds (at least one).  The
// workspace grows (after a synchronisation of the stream) when a call needs more slices than
// it holds and the budget allows.
bp_status klein_reserve(bp_plan *p, int batch, cudaStream_t st, int *chunk) {
    KleinWork &kw = p->klein;
    const size_t per = klein_slice_bytes(p);
    if (kw.tab && batch <= kw.tab_slices) {
        *chunk = batch;
        return BP_OK;
    }
    const size_t have = kw.tab ? per * (size_t)kw.tab_slices : 0;
    size_t budget = kw.tab_limit;
    if (!budget) {
        size_t free_b = 0, total_b = 0;
        BP_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        budget = (free_b + have) / 4;
    }
    const int fit = (int)std::min<size_t>((size_t)batch, std::max<size_t>(1, budget / per));
    if (kw.tab && fit <= kw.tab_slices) {
        *chunk = kw.tab_slices;
        return BP_OK;
    }
    if (kw.tab) {
        BP_CUDA_TRY(cudaStreamSynchronize(st));  // no queued launch may still read the old tables
        cudaFree(kw.tab);
        kw.tab = nullptr;
        kw.tab_slices = 0;
    }
    BP_CUDA_TRY(cudaMalloc(&kw.tab, per * (size_t)fit));
    kw.tab_slices = fit;
    *chunk = fit;
    return BP_OK;
}

template <typename Tin, int MINB, int NBUF, int BPT, int STG>
bp_status launch_klein_t(bp_plan *p, const Tin *sino, float *img, int batch, int accumulate, cudaStream_t st,
                         float wuni, int S, const float *H) {
    constexpr int NT = kKThreads / BPT;
    KleinWork &kw = p->klein;
    bp_status s = klein_upload(p);
    if (s != BP_OK) return s;
    const int RS = kw.L + kKW;
    S = klein_clamp_groups(p, S);
    constexpr size_t smem = (size_t)NBUF * 4 * STG * kKWin;
    if ((size_t)(p->n_det + 8) * sizeof(float) > 200u * 1024u)
        return fail(BP_ERR_UNSUPPORTED, "direct R*: detector row too long for the four-image form's tables");
    int chunk = 1;
    s = klein_reserve(p, batch, st, &chunk);
    if (s != BP_OK) return s;
    const size_t img_n = (size_t)p->N * p->N, sino_n = (size_t)p->n_theta * p->n_det;
    const long long tab_stride = 2LL * p->n_theta * RS;
    stage_begin(p, st);
    // the table launch clears the images (N even: N^2 / 4 float4)
    const bool clear_in_tables = !accumulate && aligned16(img) && img_n % 4 == 0;
    if (!accumulate && !clear_in_tables) {
        BP_CUDA_TRY(cudaMemsetAsync(img, 0, sizeof(float) * img_n * batch, st));
        stage_mark(p, st, "memset (direct R* image)");
    }
    auto kern1 = bp_direct_klein_kernel<MINB, NBUF, BPT, STG, false, KleinGeoSame>;
    auto kernm = bp_direct_klein_kernel<MINB, NBUF, BPT, STG, true, KleinGeoSame>;
    static int per_sm = 0;
    if (!per_sm) {
        BP_CUDA_TRY(cudaFuncSetAttribute(kern1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        BP_CUDA_TRY(cudaFuncSetAttribute(kernm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int pm = 0;
        BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern1, NT, smem));
        BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pm, kernm, NT, smem));
        per_sm = std::max(1, std::min(per_sm, pm));
    }
    const int grid = per_sm * std::max(1, p->sm_count);
    const KleinAngle *ka = (const KleinAngle *)kw.d_ang;
    // chunk by chunk: the chunk's tables by one launch (filtered on the way when H is given),
    // then one persistent launch over the chunk's slices
    for (int c0 = 0; c0 < batch; c0 += chunk) {
        const int cn = std::min(chunk, batch - c0);
        const Tin *sc = sino + sino_n * c0;
        float *ic = img + img_n * c0;
        s = H ? klein_filter_tables(p, sc, cn, H, st, wuni, clear_in_tables ? ic : nullptr)
              : klein_tables(p, sc, cn, st, wuni, clear_in_tables ? ic : nullptr);
        if (s != BP_OK) return s;
        const KleinGeoSame geo{ka, kw.tab, ic, p->N, p->n_theta, RS, kw.jlo, kw.nr, S, cn, (long long)img_n, tab_stride};
        (cn > 1 ? kernm : kern1)<<<grid, NT, smem, st>>>(geo, p->d_err);
        BP_CUDA_TRY(cudaGetLastError());
        stage_mark(p, st, cn > 1 ? "bp_direct_klein_batch_kernel" : "bp_direct_klein_kernel");
    }
    return BP_OK;
}

template <int MINB, int BPT, int STG>
bp_status launch_klein_dt(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, int accumulate,
                          cudaStream_t st, float wuni, int S, const float *H) {
    switch (dt) {
        case BP_BF16:
            return launch_klein_t<__nv_bfloat16, MINB, 3, BPT, STG>(p, (const __nv_bfloat16 *)sino, img, batch,
                                                                    accumulate, st, wuni, S, H);
        case BP_F16:
            return launch_klein_t<__half, MINB, 3, BPT, STG>(p, (const __half *)sino, img, batch, accumulate, st, wuni,
                                                             S, H);
        default:
            return launch_klein_t<float, MINB, 3, BPT, STG>(p, (const float *)sino, img, batch, accumulate, st, wuni,
                                                            S, H);
    }
}

}  // namespace

// The four-image form's launch shape: shape[0] = 16 -> one block per thread, three 256-thread
// CTAs per SM (up to 80 registers), 8-angle stages; 32 -> two blocks per thread (128-thread CTAs
// share the per-angle work), three CTAs per SM, 8-angle stages; 8 -> two blocks per thread, four
// CTAs per SM (up to 128 registers), 6-angle stages; shape[1] = angle groups S of the
// persistent schedule.  Three stages of windows are in flight.
bp_status launch_direct_klein(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, int accumulate,
                              cudaStream_t st, float wuni, int stage, int S, const float *H) {
    if (H && !(p->d_twpass && aligned16(H) && aligned16(p->d_twpass)))
        return fail(BP_ERR_UNSUPPORTED, "fused FBP: no persistent filter transform for this detector length");
    if (stage == 8) return launch_klein_dt<4, 2, 6>(p, sino, dt, img, batch, accumulate, st, wuni, S, H);
    if (stage == 32) return launch_klein_dt<3, 2, 8>(p, sino, dt, img, batch, accumulate, st, wuni, S, H);
    return launch_klein_dt<3, 1, 8>(p, sino, dt, img, batch, accumulate, st, wuni, S, H);
}


// ---------------------------------------------------------------------------------- mixed batches
// bp_backproject_batched when every slice takes the four-image form: slices in chunks whose
// tables fit the budget of plans[0] (its bp_set_direct_workspace bound, else a quarter of the free
// device memory; at least one slice), per chunk one launch that writes every slice's tables and
// clears its image, and one persistent launch of the two-blocks-per-thread kernel over the
// chunk's slices, each with its own geometry and the angle groups of its default launch shape.
bool klein_mixed_eligible(bp_plan *const *plans, float *const *imgs, int n) {
    for (int i = 0; i < n; ++i) {
        const bp_plan *p = plans[i];
        if (!p->klein.eligible || (size_t)(p->n_det + 8) * sizeof(float) > 200u * 1024u || !aligned16(imgs[i]))
            return false;
    }
    return true;
}

bp_status launch_klein_mixed(bp_plan *const *plans, const void *const *sinos, const bp_dtype *dtypes,
                             float *const *imgs, int n, cudaStream_t st) {
    constexpr int MINB = 3, NBUF = 3, BPT = 2, STG = 8, NT = kKThreads / BPT;
    constexpr size_t smem = (size_t)NBUF * 4 * STG * kKWin;
    bp_plan *p0 = plans[0];
    KleinWork &w0 = p0->klein;
    size_t most = 0, nd_max = 0;
    for (int i = 0; i < n; ++i) {
        bp_status s = klein_upload(plans[i]);
        if (s != BP_OK) return s;
        most = std::max(most, klein_slice_bytes(plans[i]));
        nd_max = std::max(nd_max, (size_t)plans[i]->n_det);
    }
    size_t budget = w0.tab_limit;
    if (!budget) {
        size_t free_b = 0, total_b = 0;
        BP_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        budget = (free_b + w0.mix_bytes) / 4;
    }
    // the workspace: the largest chunk the budget allows (at least the largest slice)
    size_t need = 0;
    for (int c0 = 0; c0 < n;) {
        size_t bytes = 0;
        int c1 = c0;
        while (c1 < n && c1 - c0 < kKMaxSlices &&
               (c1 == c0 || bytes + klein_slice_bytes(plans[c1]) <= std::max(budget, most)))
            bytes += klein_slice_bytes(plans[c1++]);
        need = std::max(need, bytes);
        c0 = c1;
    }
    if (need > w0.mix_bytes) {
        if (w0.mix_tab) {
            BP_CUDA_TRY(cudaStreamSynchronize(st));  // no queued launch may still read the old tables
            cudaFree(w0.mix_tab);
            w0.mix_tab = nullptr;
            w0.mix_bytes = 0;
        }
        BP_CUDA_TRY(cudaMalloc(&w0.mix_tab, need));
        w0.mix_bytes = need;
    }
    auto kern = bp_direct_klein_kernel<MINB, NBUF, BPT, STG, true, KleinGeoMixed>;
    static int per_sm = 0;
    if (!per_sm) {
        BP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        BP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
        per_sm = std::max(1, per_sm);
    }
    const size_t tsmem = sizeof(float) * (nd_max + 8);
    if (tsmem > 48 * 1024)
        BP_CUDA_TRY(cudaFuncSetAttribute(klein_tables_mixed_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tsmem));
    stage_begin(p0, st);
    for (int c0 = 0; c0 < n;) {
        KleinTabBatch tb;
        KleinGeoMixed geo;
        size_t off = 0;  // float4 entries
        int rows = 0, c1 = c0;
        while (c1 < n && c1 - c0 < kKMaxSlices &&
               (c1 == c0 || (off * sizeof(float4) + klein_slice_bytes(plans[c1])) <= std::max(budget, most))) {
            const bp_plan *p = plans[c1];
            const KleinWork &kw = p->klein;
            const int i = c1 - c0, RS = kw.L + kKW;
            float4 *tab = w0.mix_tab + off;
            tb.d[i] = KleinTabSlice{sinos[c1], tab, p->d_ang, (float4 *)imgs[c1], p->N, p->n_det, p->n_theta, kw.jlo,
                                    kw.L, RS, (int)dtypes[c1], rows};
            geo.d[i] = KleinSlice{(const KleinAngle *)kw.d_ang, tab, imgs[c1], p->N, p->n_theta, RS, kw.jlo, kw.nr,
                                  klein_clamp_groups(p, direct_shape(p, BP_F32, 1).asplit)};
            off += klein_slice_bytes(p) / sizeof(float4);
            rows += p->n_theta;
            ++c1;
        }
        tb.n = geo.n = c1 - c0;
        klein_tables_mixed_kernel<<<rows, 256, tsmem, st>>>(tb);
        BP_CUDA_TRY(cudaGetLastError());
        stage_mark(p0, st, "klein_tables_mixed_kernel");
        kern<<<per_sm * std::max(1, p0->sm_count), NT, smem, st>>>(geo, p0->d_err);
        BP_CUDA_TRY(cudaGetLastError());
        stage_mark(p0, st, "bp_direct_klein_mixed_kernel");
        c0 = c1;
    }
    return BP_OK;
}

}  // namespace bp
