// Shared declarations of the sm_103a backprojection library (internal, not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <string>
#include <vector>

#include "bp.h"
#include "geometry.cuh"

namespace bp {

// ------------------------------------------------------------------------------ errors
void set_error(const std::string &msg);
bp_status fail(bp_status st, const std::string &msg);
bp_status cuda_fail(cudaError_t e, const char *what);

#define BP_CUDA_TRY(expr)                                         \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return ::bp::cuda_fail(_e, #expr); \
    } while (0)

// Lookup into the ray angles sorted in [0, 2 pi).
struct RayIndex {
    int n = 0;
    int uniform = 0;              // angles phi_i = phi0 + i dphi exactly (to 1e-9)
    float phi0 = 0.f, dphi = 0.f;
    int upper = 0;                // every ray has a non-negative y step (angles in [0, pi])
};

// Fourier-path workspace and gridding geometry (allocated on first use).
struct FourierWork {
    int M = 0, logM = 0;        // oversampled grid side (power of two >= 2N)
    int W = 6;                  // Kaiser-Bessel width (grid cells)
    float beta = 0.f;           // Kaiser-Bessel shape for W = 6 and oversampling M/N
    float rho = 0.f;            // radial sample spacing in grid cells
    float2 *spec = nullptr;     // [n_theta][P/2] sample values c_{k,m}
    float2 *grid = nullptr;     // [M][M] gridded spectrum, G[l_x][l_y]
    float2 *mid = nullptr;      // [N][M] after the first inverse-FFT pass
    CUtensorMap mid_map;        // mid as FP32 [N][2M], boxes of 16 bytes x 256 rows (TMA stores)
    bool mid_map_ok = false;
    float *deapod = nullptr;    // [N] 1 / phi_hat(i - floor(N/2))
    float *wk = nullptr;        // [n_theta] quadrature weights (float)
    float2 *twM = nullptr;      // M/2 twiddles exp(-2 pi i r / M)
    float2 *twpassM = nullptr;  // per-pass twiddles of the M-point transform (build_pass_twiddles)
    float2 *twpassH = nullptr;  // per-pass twiddles of the M/2-point transform (M = 16384: split transforms)
    long long *ray = nullptr;   // [n_theta][2] rho cos, rho sin in 32.32 fixed point
    void *sray = nullptr;       // rays sorted by angle (gather gridding)
    float *sphi = nullptr;      // sorted ray angles in [0, 2 pi)
    float2 *kbtab = nullptr;    // Kaiser-Bessel kernel table
    float rmax = 0.f;           // largest sample radius (grid cells) plus a margin
    RayIndex ri;                // sorted-angle lookup (gather gridding)
    int4 *adj_items = nullptr;  // adjoint interpolation work items: tile, first segment, segments, samples
    int4 *adj_segs = nullptr;   // their ray segments: projection, first sample, samples, offset in the item
    int adj_n_items = 0;
    size_t bytes = 0;
};

// Workspace of the paper's own BST algorithm (polar-to-Cartesian interpolation, bst.cu);
// the Cartesian grid and the inverse-FFT intermediate are the Fourier path's.
struct BstWork {
    int os = 0;                 // radial oversampling: Pb = os P
    int Pb = 0;                 // projection transform length
    float2 *polar = nullptr;    // [n_theta][Pb/2] polar values of the backprojection's transform
    float2 *twPb = nullptr;     // Pb/2 twiddles
    float2 *twPassH = nullptr;  // per-pass twiddles of the Pb/2-point transform (Pb/2 = 512 .. 8192)
    float *ang = nullptr;       // [2 n_theta] ray angles theta_k, theta_k + pi in [0, 2 pi), sorted
    int *ray = nullptr;         // [2 n_theta] projection index, bit 30 set for the opposite ray
    float *ones = nullptr;      // [N] unit deapodisation
    float4 *dir = nullptr;      // [2 n_theta] ray directions (cos, sin) as high and low floats
    float *igap = nullptr;      // [2 n_theta] 1 / angular gap to the next ray
    RayIndex ri;                // lookup into ang (n = 2 n_theta)
    float *wrows = nullptr;     // [n_theta][2 ns - 1] windowed semi-polar lines (ns = n_det/2 + 1)
    float *win = nullptr;       // [ns] window of eq "w"
    float beta = -1.f;          // its beta (-1: not computed)
    size_t bytes = 0;
};

// Workspace of Andersson's log-polar backprojection (logpolar.cu).
struct LogPolarWork {
    int n_rho = 0, n_phi = 0, n_out = 0, L = 0;  // meshes (see logpolar.cu)
    double rho0 = 0.0, drho = 0.0;
    int4 *rtab = nullptr;      // [n_rho] detector bin and fraction of s_i (signs +, -)
    int4 *atab = nullptr;      // [n_phi] bracketing projections, detector signs, weight
    float2 *kfrac = nullptr;   // [n_phi] kernel node and fraction of -ln cos(theta') / drho
    int4 *pix = nullptr;       // [N*N] pixel -> (rho node, fraction, theta node, fraction)
    float2 *twL = nullptr, *twPhi = nullptr;
    float2 *twPassPhi = nullptr;  // per-pass twiddles of the n_phi-point transform (n_phi = 512 .. 4096)
    float2 *twPassH = nullptr;    // per-pass twiddles of the L/2-point transform (L/2 = 512 .. 8192)
    float2 *T = nullptr;       // [n_phi][L] complex work array
    float2 *Khat = nullptr;    // [n_phi][L] kernel transform (scaled)
    float *B = nullptr;        // [n_phi][n_out] backprojection on the log-polar mesh
    CUtensorMap T_map, K_map;  // T and Khat as FP32 [n_phi][2L], boxes of one column pair x min(256, n_phi) rows
    bool maps_ok = false;
    size_t bytes = 0;
};

// Workspace of the partial (sector) log-polar backprojection (logpolar_partial.cu).
struct LppWork {
    int Q = 0;                 // sectors over [0, pi)
    float a_r = 0.f;           // rescaling ratio of the shift
    int K = 0, n_half = 0;     // angle nodes per sector, over [0, pi)
    int n_rho = 0, c_lo = 0, n_out = 0, a_lo = 0, n_aout = 0, Lr = 0, Lp = 0;  // meshes
    int2 *stab = nullptr;      // [n_rho] s_i / dt as (integer, fraction bits)
    int4 *rowtab = nullptr;    // [K] -D_j + c0 and D_j + c0 split (D_j = d cos(phi_j - phi_c) / dt)
    int4 *atab = nullptr;      // [n_half] bracketing projections, flip bits, weight
    float2 *kfrac = nullptr;   // [Lp] kernel node and fraction per angular-transform row
    float2 *twLr = nullptr, *twLp = nullptr;
    float2 *twPassLp = nullptr;  // per-pass twiddles of the Lp-point transform (Lp = 512 .. 4096)
    float2 *twPassH = nullptr;   // per-pass twiddles of the Lr/2-point transform (Lr/2 = 512 .. 8192)
    CUtensorMap Tin_map, Tout_map, K_map;  // T (first K rows, first n_aout rows) and Khat as FP32 [rows][2 Lr]
    bool maps_ok = false;
    float2 *T = nullptr;       // [Lp][Lr] complex work array
    float2 *Khat = nullptr;    // [Lp][Lr] kernel transform (scaled)
    float *B = nullptr;        // [n_aout + 1][n_out] one sector's output mesh
    int4 *pix = nullptr;       // [Q][N*N] per-sector pixel -> (rho node, fraction, angle node, fraction)
    size_t bytes = 0;
};

// Launch shapes.  The direct R* takes `stage` angles per shared-memory stage (8, 16 or 32)
// and splits the angles into `asplit` groups, each a separate CTA per tile that adds its
// partial sum into the image; the direct R takes `kang` angles per CTA (1, 2 or 4) and
// `bands` image bands per angle block (0 = the default rules).  They are picked by
// bp_autotune (tune.cu) or by the default rules there.
struct DirectShape {
    int stage = kStage;
    int asplit = 1;      // angle groups (the four-image form: groups of its persistent schedule)
    int workspace = 1;   // 0: never take a form that needs a plan workspace (allocation-free calls)
};
// The four-image form of the direct R* (direct_klein.cu): eligibility and per-angle data made
// on the host at plan creation; the per-angle table and the row-table workspace (one slice,
// 2 x n_theta x L float4) are allocated on first use.
struct KleinWork {
    bool eligible = false;
    int jlo = 0, L = 0, nr = 0;          // table extent (bins jlo .. jlo + L - 1), regions per side
    std::vector<unsigned char> host;     // per-angle records (KleinAngle)
    void *d_ang = nullptr;
    float4 *tab = nullptr;               // row tables of tab_slices slices
    int tab_slices = 0;
    size_t tab_limit = 0;                // bp_set_direct_workspace (0: a quarter of the free memory)
    float4 *mix_tab = nullptr;           // row tables of a mixed batch led by this plan
    size_t mix_bytes = 0;
};
struct RadonShape {
    int kang = 0;   // 0 = the default rule
    int bands = 0;
};
// Device slots of the host-buffer entry point: slice i + 1 is copied in and slice i - 1 copied
// out while slice i is filtered and backprojected.
constexpr int kHostSlots = 3;

// Per-kernel timing (bp_stage_timing / bp_stage_times): while it is on, every launcher records a
// CUDA event on its stream at its start (name nullptr) and after each kernel it launches (the
// kernel's name); a kernel's time is the interval from the event before it.
struct StageTimer {
    bool on = false;
    bool overflow = false;
    std::vector<cudaEvent_t> ev;      // created on demand, reused
    std::vector<const char *> name;   // per recorded event; nullptr marks a call's start
    int used = 0;
};
constexpr int kStageTimerCap = 8192;

struct TuneEntry {
    int op, dtype, batch;
    int v[2];
};

}  // namespace bp

struct bp_plan {
    int N = 0, n_det = 0, n_theta = 0;
    double dt = 0.0, dx = 0.0;
    int device = 0;
    std::vector<double> theta, w;
    // direct kernels
    bp::AngleParam *d_ang = nullptr;
    int W = 0;   // shared-memory window (entries) per (tile, angle)
    int C = 0;   // window centre offset
    float step_max = 0.f;  // max over the angles of max(|c|, |s|), the u step per pixel
    // filter
    int P = 0;                 // FFT length for the filter (power of two >= 2 n_det)
    float2 *d_twP = nullptr;   // P/2 twiddles exp(-2 pi i r / P)
    float2 *d_twpass = nullptr;  // per-pass twiddles of the persistent filter kernel (512 <= P <= 4096)
    float *d_H[3] = {nullptr, nullptr, nullptr};   // scaled responses (dt/P) DFT_P(h) per kind, natural order
    float H_param[3] = {0.f, 0.f, 0.f};
    // bp_fbp_direct on a geometry without the fused form: the filtered sinograms
    float *d_fbp = nullptr;
    size_t fbp_n = 0;                       // floats allocated
    // Fourier path
    int fourier_W = 6;          // Kaiser-Bessel width of the gridding (bp_set_fourier_width)
    bp::FourierWork four;
    bp::BstWork bst;
    bp::LogPolarWork lp;
    bp::LppWork lpp;
    // host-buffer entry point: a ring of device slots (one sinogram and one image each), the
    // copy streams and the events that order the reuse of a slot
    float *d_stage = nullptr;
    size_t stage_batch = 0;                 // slots allocated
    cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
    cudaEvent_t ev_h2d[bp::kHostSlots] = {}, ev_comp[bp::kHostSlots] = {}, ev_d2h[bp::kHostSlots] = {};
    // batched descriptors
    void *d_desc = nullptr;
    size_t desc_cap = 0;
    int *d_counter = nullptr;
    int *d_status = nullptr;
    // device-side error word: set to non-zero by a kernel whose bounded wait gave up
    int *d_err = nullptr;
    // launch shapes chosen for this plan (bp_autotune / bp_set_shape), and the SM count
    std::vector<bp::TuneEntry> shapes;
    int sm_count = 0;
    bp::StageTimer timer;
    bp::KleinWork klein;
};

namespace bp {
bp_status check_plan(const bp_plan *p);
// stage timing marks (no-ops unless the plan's timer is on): stage_begin at the start of a
// launcher, stage_mark after each kernel launch with the kernel's name (a string literal)
void stage_begin(bp_plan *p, cudaStream_t st);
void stage_mark(bp_plan *p, cudaStream_t st, const char *name);
bool aligned16(const void *ptr);
int ilog2(int v);

// launchers implemented in the kernel translation units
// wuni > 0 replaces every quadrature weight w_k by wuni; per_angle_w = 1 scales angle k of R
// by w_k instead of dx^2/dt (the two weightings of the Euclidean transposes).
bp_status launch_direct(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, int accumulate,
                        cudaStream_t st, float wuni = 0.f);
bp_status launch_direct_shape(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, int accumulate,
                              cudaStream_t st, float wuni, DirectShape shape);
bp_status launch_filter(bp_plan *p, const void *in, bp_dtype dt, float *out, int kind, float param, int batch,
                        cudaStream_t st);
bp_status launch_radon_direct(bp_plan *p, const float *img, float *sino, int batch, cudaStream_t st,
                              int per_angle_w = 0);
bp_status launch_radon_shape(bp_plan *p, const float *img, float *sino, int batch, cudaStream_t st, int per_angle_w,
                             RadonShape shape);
// shape lookup: the plan's own entry for (op, dtype, batch), else the process-wide tuning
// cache for the plan's geometry, else the default rule
DirectShape direct_shape(const bp_plan *p, bp_dtype dt, int batch);
RadonShape radon_shape(const bp_plan *p, int batch);
int direct_max_asplit(const bp_plan *p, int stage);
DirectShape direct_shape_used(const bp_plan *p, bp_dtype dt, int batch);  // after clamping
RadonShape radon_shape_used(const bp_plan *p, int batch);                  // after clamping
DirectShape direct_clamp(const bp_plan *p, bp_dtype dt, DirectShape shape);
RadonShape radon_clamp(const bp_plan *p, RadonShape shape);
int radon_max_kang(const bp_plan *p);
// filter_kind >= 0 fuses that FBP filter (bp_filter's steps) into the projection transforms.
bp_status launch_fourier(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, cudaStream_t st,
                         float wuni = 0.f, int filter_kind = -1, float filter_param = 0.f);
bp_status launch_radon_fourier(bp_plan *p, const float *img, float *sino, int batch, cudaStream_t st,
                               int per_angle_w = 0);
bp_status ensure_filter(bp_plan *p, int kind, float param);
bp_status launch_filter_response(bp_plan *p, const void *in, bp_dtype dt, float *out, const float *Hbr, int batch,
                                 cudaStream_t st);
bp_status ensure_fourier(bp_plan *p);
void klein_plan(bp_plan *p);
void free_klein(bp_plan *p);
int klein_default_groups(const bp_plan *p);
int klein_clamp_groups(const bp_plan *p, int S);
bp_status launch_direct_klein(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, int accumulate,
                              cudaStream_t st, float wuni, int stage, int S, const float *H = nullptr);
bp_status klein_set_workspace(bp_plan *p, size_t bytes);
bool klein_mixed_eligible(bp_plan *const *plans, float *const *imgs, int n);
bp_status launch_klein_mixed(bp_plan *const *plans, const void *const *sinos, const bp_dtype *dtypes,
                             float *const *imgs, int n, cudaStream_t st);
bp_status launch_fbp_direct(bp_plan *p, const void *sino, bp_dtype dt, float *img, int kind, float param, int batch,
                            cudaStream_t st);
void free_fourier(bp_plan *p);
void free_bst(bp_plan *p);
void free_logpolar(bp_plan *p);
void free_logpolar_partial(bp_plan *p);
bp_status launch_logpolar_partial(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, int sectors,
                                  float a_r, cudaStream_t st);
bp_status launch_logpolar(bp_plan *p, const void *sino, bp_dtype dt, float *img, int batch, cudaStream_t st);
bp_status launch_grid_to_image(bp_plan *p, const float *deap, float *img, cudaStream_t st);
bp_status launch_bst(bp_plan *p, const void *sino, bp_dtype dt, float *img, int os, int batch, cudaStream_t st);
bp_status launch_bst_windowed(bp_plan *p, const void *sino, bp_dtype dt, float *img, int os, float beta, int batch,
                              cudaStream_t st);
bp_status launch_batched(bp_plan *const *plans, const void *const *sinos, const bp_dtype *dtypes,
                         float *const *imgs, int n, cudaStream_t st);

// host FP64 FFT (plan tables only): in-place radix-2, sign -1 forward
void host_fft(std::vector<double> &re, std::vector<double> &im, bool inverse);
void build_pass_twiddles(int logP, std::vector<float2> &T);
bool filter_pt_supported(int P);

// element loads, widened to float
template <typename T> __device__ __forceinline__ float load_f(const T *p);
template <> __device__ __forceinline__ float load_f<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_f<__nv_bfloat16>(const __nv_bfloat16 *p) {
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float load_f<__half>(const __half *p) { return __half2float(__ldg(p)); }

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void sts64(unsigned addr, float2 v) {
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ float4 lds128(unsigned addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}
__device__ __forceinline__ void sts128(unsigned addr, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}
__device__ __forceinline__ float2 lds64(unsigned addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

}  // namespace bp
