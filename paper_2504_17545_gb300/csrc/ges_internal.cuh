// Internal declarations and device math of the GES renderer (sm_103a).
//
// Shared by the forward (ges_forward.cu), backward (ges_backward.cu) and host
// (ges_api.cu) translation units.  The per-primitive set-up functions here are
// the single definition used by both the forward and the backward kernels, so
// that a Gaussian's alpha and depth-test decisions are bit-identical in both.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "ges.h"

namespace ges {

constexpr int kTile = 16;               // default binning tile edge (pixels): 16x16
constexpr int kTileShift = 4;           // log2 kTile
constexpr int kRasterThreads = 256;     // 8 warps, each an 8x4 pixel block
constexpr int kWarpW = 8, kWarpH = 4;
// A binning tile holds the 8 warps' blocks: 2^tsx x 2^tsy pixels with
// tsx + tsy = 8 and tsx in [3, 6] (8x32, 16x16, 32x8, 64x4).

// status word layout (uint32 words)
enum : int {
    ST_FLAGS = 0,         // bit0 surfel list overflow, bit1 Gaussian list overflow, bit2 bad quaternion
    ST_SVIS = 1,          // visible surfels
    ST_GVIS = 2,          // visible Gaussians
    ST_SPAIRS = 3,        // surfel tile pairs
    ST_GPAIRS = 4,        // Gaussian tile pairs
    ST_SFRAG = 5,         // surfel fragments inside their discs (work count)
    ST_GFRAG = 6,         // Gaussian pixel terms with alpha >= alpha_min (work count)
    ST_RETIRED = 7,       // batch raster: tiles of this view finished
    ST_TDONE = 8,         // batch raster: %globaltimer (ns, 64-bit, words 8-9) when the last tile finished
    ST_WORDS = 16,
};
enum : unsigned { FLAG_SOVF = 1u, FLAG_GOVF = 2u, FLAG_BADQ = 4u };

struct CamParams {
    float R[9];           // world -> camera rotation, row-major
    float t[3];
    float fx, fy, cx, cy;
    float ocam[3];        // camera centre in world space (rounded from FP64)
    float znear, izn;     // z_near and 1/z_near
    float bg[3];
    int W, H, tiles_x, tiles_y;
    int tsx, tsy;         // log2 of the binning tile's width and height
};

struct OptParams {
    int eps_mode;
    float eps_value, eps_factor, lowpass, alpha_min, surfel_r2, surfel_r;
    int mode;
    int samples;          // surfel samples per pixel: 1 or 4
    int filter;           // GES_FILTER_EWA or GES_FILTER_MIP
    int geo;              // 1: the render also produces the geometry maps (Sec. 6.4)
};

struct SceneView {
    int64_t N, M;
    int deg, attr_dtype, sh_dtype;
    const float *s_pos;
    const void *s_rot, *s_scale, *s_sh;
    const float *g_pos;
    const void *g_rot, *g_scale, *g_opac, *g_sh;
    const float *g_filt3;     // Mip-GES 3D filter variance [M], or null
    int gdim;                 // 3: 3D Gaussians; 2: 2D Gaussians of 2D-GES (g_scale [M,2])
};

// Scratch of one view (device pointers owned by the scene).
struct ViewScratch {
    float4 *s_rec;        // [N][4]  surfel raster records
    float4 *s_rgb;        // [N]     surfel colours
    float4 *g_rec;        // [M][4]  Gaussian raster records
    // visible primitives: with local bins, per-CTA segments of 16-byte entries
    // (id, bbox lo, bbox hi, -), 16 B per primitive; with atomic binning one
    // id per entry
    int *s_vis, *g_vis;
    int *s_cnt, *g_cnt;   // [T]     per-tile counts (zero between renders)
    int *s_off, *g_off;   // [T+1]   exclusive offsets
    int *s_cur, *g_cur;   // [T]     fill cursors (atomic binning)
    int *s_list, *g_list; // tile lists
    int64_t s_cap, g_cap; // list capacities (entries)
    unsigned *status;     // [ST_WORDS]
    // local binning (per-CTA primitive ranges with shared-memory histograms);
    // left null, the render bins with global atomics instead
    unsigned *hist = nullptr;    // [P][ceil(T/2)] packed 16-bit per-CTA tile counts
    unsigned *base = nullptr;    // [P][T] per-CTA start inside each tile's list
    unsigned *vcount = nullptr;  // [P] visible primitives per CTA
    // [M][2] side data of each Gaussian, written when the render needs it:
    // 2D Gaussians (rgb, log2 sigma'), (normal, log2(alpha_min / sigma'));
    // 3D Gaussians with geometry outputs (normal, centre depth), unused
    float4 *g_aux = nullptr;
    // [N][4] camera-space frame of each surfel for the translucent render:
    // (P, s1), (U, s2), (V, -), (N, -); written when non-null
    float4 *s_tside = nullptr;
    // [M] Gaussian colours in 2^-16 units, written by the batch's colour pass
    // before the set-up, which copies them into the records; null elsewhere
    float4 *g_col = nullptr;
};

// Number of preprocess CTAs for local binning and the size of their ranges.
struct LocalBins {
    int Ps, Pg;           // CTAs over surfels, over Gaussians
    int64_t Rs, Rg;       // primitives per CTA
};
constexpr int kLocalMaxTiles = 32768;   // shared-memory cursors of the fill: 4 B per tile

// One view of a batch (device table entry).  The batch kernels find their view
// from the per-phase bases (prefix sums over the views).
struct BatchView {
    SceneView S;          // counts already zeroed for the render mode
    CamParams C;
    ViewScratch X;
    LocalBins B;
    float *rgb, *depth;
    int32_t *id;          // surfel id map [samples,H,W] or null (ges_batch_set_id_output)
    float *aux;           // W_G [H,W] or null
    int T, tile_base, prep_base, colscan_base;
    int sprep_base, gprep_base;   // first CTA of the view's surfel / Gaussian ranges in their own launches
};
struct BatchPlan {
    int n;                                   // views
    int total_tiles, total_prep, total_colscan, max_T;
    int total_sprep, total_gprep;            // preprocess CTAs of the surfel and the Gaussian launch
    int raster_ctas;                         // persistent raster grid
    int gdim;                                // Gaussian kind of every scene (2 or 3; 0 reads as 3)
    // (view, CTA of the view) of each CTA of the surfel / Gaussian preprocess
    // launch: the views of one scene take the same primitive range one after
    // another, so all but the first read its attributes from L2
    const int2 *smap, *gmap;
    // colour pass: per CTA (kind: 0 surfels / 1 Gaussians, first entry of its
    // view group in gview, views in the group, first primitive); gview lists
    // the views of each group of views that share one scene.  total_colour 0
    // (no scene with several views): the set-up evaluates the colours
    const int4 *cmap;
    const int *gview;
    int total_colour;
};
constexpr int kColourThreads = 256;   // primitives per colour-pass CTA
constexpr int kColourViews = 64;      // views whose camera centres a colour-pass CTA stages at a time
// ev: 7 events recorded as graph event nodes (phase boundaries 0-4, the
// colour pass's start and end 5-6) or nullptr.
// ids: the raster also writes the views' id maps and W_G where BatchView
// points to them (a raster kernel of its own).
cudaError_t launch_batch(const BatchView *d_views, const BatchPlan &P, const OptParams &O, unsigned *work_counter,
                         cudaStream_t st, cudaEvent_t *ev, bool ids);
LocalBins plan_local_bins_per_cta(int64_t N, int64_t M, int64_t prims_per_cta);
constexpr int kPrepThreads = 512;
constexpr int kFillThreads = 1024;
LocalBins plan_local_bins(int64_t N, int64_t M, int num_sms);
size_t local_bins_smem(int T, bool fill);
cudaError_t prepare_forward_kernels();   // once per device: large dynamic shared memory

// ---------------------------------------------------------------------------
// host launchers (ges_forward.cu / ges_backward.cu)

// Preprocess and binning of one view (the tile lists, before any raster);
// ev: 4 events or null.  With X.s_tside set, surfels also export their
// camera-space frame (translucent render).
cudaError_t launch_binning(const SceneView &S, const CamParams &C, const OptParams &O, const ViewScratch &X,
                           cudaStream_t st, cudaEvent_t *ev);

// Translucent-surfel render (Sec. 4.1) of one view: binning of the surfels
// (X.s_tside must be set), per-tile sort, blend.  keys: one 64-bit word per
// tile-list entry.  cover (or null): per-surfel counts of frontmost pixels, added.
cudaError_t launch_translucent(const SceneView &S, const CamParams &C, const OptParams &O, const ViewScratch &X,
                               const float *w, bool front_first, unsigned long long *keys, float *out_rgb,
                               float *out_T, int32_t *out_front, int32_t *out_last, float *out_Tlast, int32_t *cover,
                               cudaStream_t st);
// Its backward: acc [N][18] 64-bit words and gmax (one word) are scratch.
cudaError_t launch_translucent_backward(const SceneView &S, const CamParams &C, const OptParams &O,
                                        const ViewScratch &X, const float *w, bool front_first,
                                        unsigned long long *keys, const float *dL, const float *in_T,
                                        const int32_t *in_front, const int32_t *in_last, const float *in_Tlast,
                                        long long *acc, unsigned *gmax, float *g_pos, float *g_rot, float *g_scale,
                                        float *g_w, float *g_sh, cudaStream_t st);
// Gaussian contribution scores (Eq. 9) from a render's depth (D_s) and aux (W_G).
cudaError_t launch_contribution(const SceneView &S, const CamParams &C, const OptParams &O, const float *depth,
                                const float *aux, float *score, cudaStream_t st);

// geo_maps: null, or 5 device pointers (each may be null): N_s [3,H,W],
// D_smooth [H,W], N_smooth [3,H,W], D_G [H,W], N_G [3,H,W]; with O.geo set.
cudaError_t launch_forward(const SceneView &S, const CamParams &C, const OptParams &O, const ViewScratch &X,
                           float *out_rgb, float *out_depth, int32_t *out_id, float *aux, cudaStream_t st,
                           cudaEvent_t *ev /* 5 events or nullptr */, const float *const *geo_maps = nullptr);

cudaError_t launch_count(const SceneView &S, const CamParams &C, const OptParams &O, const ViewScratch &X,
                         cudaStream_t st);
// Mip-GES 3D filter variance per Gaussian from n_cams cameras (device array);
// d_vmax: one device word of scratch.
cudaError_t launch_filter3d(const SceneView &S, const CamParams *d_cams, int n_cams, float s3d, float *out,
                            unsigned *d_vmax, cudaStream_t st);

// Scratch: s_acc 3 N 64-bit words (surfel colour sums), gmax one word,
// pixg H W float4 (per-pixel terms of the Gaussian gradients), g_rec M
// records of kBwdRecBytes, g_sums kBwdSums M floats (per-Gaussian sums of the
// sweep), g_chain kBwdChainWords M floats (what the chain rule needs of each
// set-up).  The sizes cover both Gaussian kinds (3D: 64-byte records, 9 sums;
// 2D: 96-byte records, 11 sums).
constexpr int kBwdChainWords = 40, kBwdRecBytes = 96, kBwdSums = 11;
cudaError_t launch_backward(const SceneView &S, const CamParams &C, const OptParams &O, const float *dL_drgb,
                            const float *out_rgb, const float *out_depth, const int32_t *surfel_id,
                            const float *aux, const ges_grads &G, long long *s_acc, unsigned *gmax,
                            float4 *pixg, float4 *g_rec, float *g_sums, float *g_chain, cudaStream_t st,
                            cudaEvent_t *ev /* 3 events or nullptr */);
// *out = the bit pattern of max |x[i]| over n floats (0 for none); zeroes it first.
cudaError_t launch_absmax(const float *x, int64_t n, unsigned *out, cudaStream_t st);

// ---------------------------------------------------------------------------
// device helpers

#if defined(__CUDACC__)

// Double-float ("df") arithmetic: value = hi + lo with |lo| <= ulp(hi)/2.
// Error-free transformations after Knuth (two-sum) and the FMA residual of a
// product; used where a camera-space position must keep ~48 bits so that a
// pixel-sized disc 15 m away is located to 1e-7 of its radius.
struct df { float hi, lo; };

__device__ __forceinline__ df df_two_sum(float a, float b)
{
    float s = a + b;
    float bb = s - a;
    float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b)
{
    float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df df_two_prod(float a, float b)
{
    float p = a * b;
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ df df_add(df a, df b)
{
    df s = df_two_sum(a.hi, b.hi);
    float e = s.lo + (a.lo + b.lo);
    return df_fast_two_sum(s.hi, e);
}
__device__ __forceinline__ df df_add_f(df a, float b)
{
    df s = df_two_sum(a.hi, b);
    return df_fast_two_sum(s.hi, s.lo + a.lo);
}
__device__ __forceinline__ df df_mul_f(df a, float b)
{
    df p = df_two_prod(a.hi, b);
    p.lo = fmaf(a.lo, b, p.lo);
    return df_fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_div(df a, df b)
{
    float q1 = a.hi / b.hi;
    // r = a - q1*b (exact product residual kept)
    df p = df_mul_f(b, q1);
    df r = df_add(a, df{-p.hi, -p.lo});
    float q2 = r.hi / b.hi;
    return df_fast_two_sum(q1, q2);
}
// sum_j R[j] * v[j] + t, products exact, accumulation in df
__device__ __forceinline__ df df_dot3_plus(const float *R, float v0, float v1, float v2, float t)
{
    df acc = df_two_prod(R[0], v0);
    acc = df_add(acc, df_two_prod(R[1], v1));
    acc = df_add(acc, df_two_prod(R[2], v2));
    return df_add_f(acc, t);
}

__device__ __forceinline__ unsigned long long global_timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Range of the Gaussian pass's fixed-point terms: each alpha >= alpha_min,
// capped at 2, is rounded once to the 2^-30 grid (an unsigned 32-bit
// integer) and added into W_G's sum; a Gaussian's colour sits in its raster
// record as an integer of 2^-16 units, capped at kColourMax, and the colour
// sums add the exact 64-bit products of the two (units of 2^-46).  The sums
// are therefore exact and order independent while sum alpha < 2^33 and
// sum alpha c < 2^17 per pixel and channel, far outside the method's range
// (alpha <= 1, colours of a few units).  The geometry maps' sums keep alpha
// 2^32 (kAlpha32Max) for their own terms.
constexpr float kColourMax = 256.f;
constexpr float kAlpha32Max = 8589934592.f;   // 2^33
constexpr float kColourScale = 65536.f;       // 2^16

#ifdef __CUDACC__
// A record colour: min(c, kColourMax) in 2^-16 units, rounded to nearest,
// carried in a float word.  Colours are >= 0 (Eq. 1's clamp).
__device__ __forceinline__ float colour_q(float c)
{
    return __uint_as_float(__float2uint_rn(fminf(c, kColourMax) * kColourScale));
}
#endif

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float load_attr(const void *p, int64_t idx, int dtype)
{
    if (dtype == GES_F32) return __ldg(reinterpret_cast<const float *>(p) + idx);
    if (dtype == GES_F16) return __half2float(__ldg(reinterpret_cast<const __half *>(p) + idx));
    return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16 *>(p) + idx));
}

// Real SH basis (Condon-Shortley phase, k = l^2 + l + m) at a unit vector,
// written as Cartesian polynomials.  The constants are the normalisations
// K_l^m = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times sqrt2 for m != 0,
// multiplied by the integer coefficients of the associated Legendre
// functions:  Y00 = 1/(2 sqrt(pi));  l=1: sqrt(3/(4pi));
// l=2: sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4;
// l=3: sqrt(35/(2pi))/4, sqrt(105/pi)/2, sqrt(21/(2pi))/4, sqrt(7/pi)/4,
//      sqrt(105/pi)/4.
struct ShConst {
    static constexpr float c0 = 0.28209479177387814f;
    static constexpr float c1 = 0.48860251190291992f;
    static constexpr float c2a = 1.09254843059207907f;   // sqrt(15/pi)/2
    static constexpr float c2b = 0.31539156525252001f;   // sqrt(5/pi)/4
    static constexpr float c2c = 0.54627421529603954f;   // sqrt(15/pi)/4
    static constexpr float c3a = 0.59004358992664352f;   // sqrt(35/(2pi))/4
    static constexpr float c3b = 2.89061144264055405f;   // sqrt(105/pi)/2
    static constexpr float c3c = 0.45704579946446572f;   // sqrt(21/(2pi))/4
    static constexpr float c3d = 0.37317633259011540f;   // sqrt(7/pi)/4
    static constexpr float c3e = 1.44530572132027703f;   // sqrt(105/pi)/4
};

__device__ __forceinline__ void sh_basis(int K, float x, float y, float z, float *Y)
{
    Y[0] = ShConst::c0;
    if (K <= 1) return;
    Y[1] = -ShConst::c1 * y;
    Y[2] = ShConst::c1 * z;
    Y[3] = -ShConst::c1 * x;
    if (K <= 4) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = ShConst::c2a * x * y;
    Y[5] = -ShConst::c2a * y * z;
    Y[6] = ShConst::c2b * (2.f * zz - xx - yy);
    Y[7] = -ShConst::c2a * x * z;
    Y[8] = ShConst::c2c * (xx - yy);
    if (K <= 9) return;
    Y[9] = -ShConst::c3a * y * (3.f * xx - yy);
    Y[10] = ShConst::c3b * x * y * z;
    Y[11] = -ShConst::c3c * y * (4.f * zz - xx - yy);
    Y[12] = ShConst::c3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -ShConst::c3c * x * (4.f * zz - xx - yy);
    Y[14] = ShConst::c3e * z * (xx - yy);
    Y[15] = -ShConst::c3a * x * (xx - 3.f * yy);
}

// Gradient of the polynomials above with respect to (x,y,z) (any extension
// off the sphere works once projected onto the tangent plane).
__device__ __forceinline__ void sh_basis_grad(int K, float x, float y, float z, float (*dY)[3])
{
    dY[0][0] = dY[0][1] = dY[0][2] = 0.f;
    if (K <= 1) return;
    const float c1 = ShConst::c1;
    dY[1][0] = 0.f; dY[1][1] = -c1; dY[1][2] = 0.f;
    dY[2][0] = 0.f; dY[2][1] = 0.f; dY[2][2] = c1;
    dY[3][0] = -c1; dY[3][1] = 0.f; dY[3][2] = 0.f;
    if (K <= 4) return;
    const float a = ShConst::c2a, b = ShConst::c2b, c = ShConst::c2c;
    dY[4][0] = a * y; dY[4][1] = a * x; dY[4][2] = 0.f;
    dY[5][0] = 0.f; dY[5][1] = -a * z; dY[5][2] = -a * y;
    dY[6][0] = -2.f * b * x; dY[6][1] = -2.f * b * y; dY[6][2] = 4.f * b * z;
    dY[7][0] = -a * z; dY[7][1] = 0.f; dY[7][2] = -a * x;
    dY[8][0] = 2.f * c * x; dY[8][1] = -2.f * c * y; dY[8][2] = 0.f;
    if (K <= 9) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    const float A = ShConst::c3a, B = ShConst::c3b, Cc = ShConst::c3c, D = ShConst::c3d, E = ShConst::c3e;
    dY[9][0] = -6.f * A * x * y; dY[9][1] = -3.f * A * (xx - yy); dY[9][2] = 0.f;
    dY[10][0] = B * y * z; dY[10][1] = B * x * z; dY[10][2] = B * x * y;
    dY[11][0] = 2.f * Cc * x * y; dY[11][1] = -Cc * (4.f * zz - xx - 3.f * yy); dY[11][2] = -8.f * Cc * y * z;
    dY[12][0] = -6.f * D * x * z; dY[12][1] = -6.f * D * y * z; dY[12][2] = D * (6.f * zz - 3.f * xx - 3.f * yy);
    dY[13][0] = -Cc * (4.f * zz - 3.f * xx - yy); dY[13][1] = 2.f * Cc * x * y; dY[13][2] = -8.f * Cc * x * z;
    dY[14][0] = 2.f * E * x * z; dY[14][1] = -2.f * E * y * z; dY[14][2] = E * (xx - yy);
    dY[15][0] = -3.f * A * (xx - yy); dY[15][1] = 6.f * A * x * y; dY[15][2] = 0.f;
}

// One primitive's 3K SH coefficients as floats.  When the row is a multiple
// of 16 bytes (K = 4, 16 in FP32; K = 16 in 16-bit) it is read with 128-bit
// loads; the rows of consecutive primitives are contiguous.
template <int K>
__device__ __forceinline__ void load_sh_row(const void *sh, int64_t i, int dtype, float *c)
{
    constexpr int n = 3 * K;
    if (dtype == GES_F32) {
        const float *p = reinterpret_cast<const float *>(sh) + (int64_t)n * i;
        if ((n % 4) == 0 && (reinterpret_cast<uintptr_t>(sh) & 15) == 0) {
#pragma unroll
            for (int j = 0; j < n / 4; ++j) {
                const float4 v = __ldg(reinterpret_cast<const float4 *>(p) + j);
                c[4 * j] = v.x; c[4 * j + 1] = v.y; c[4 * j + 2] = v.z; c[4 * j + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < n; ++j) c[j] = __ldg(p + j);
        }
    } else {
        const unsigned short *p = reinterpret_cast<const unsigned short *>(sh) + (int64_t)n * i;
        if ((n % 8) == 0 && (reinterpret_cast<uintptr_t>(sh) & 15) == 0) {
#pragma unroll
            for (int j = 0; j < n / 8; ++j) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p) + j);
                const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const unsigned short lo = (unsigned short)(w[q] & 0xffffu), hi = (unsigned short)(w[q] >> 16);
                    if (dtype == GES_F16) {
                        c[8 * j + 2 * q] = __half2float(__ushort_as_half(lo));
                        c[8 * j + 2 * q + 1] = __half2float(__ushort_as_half(hi));
                    } else {
                        c[8 * j + 2 * q] = __bfloat162float(__ushort_as_bfloat16(lo));
                        c[8 * j + 2 * q + 1] = __bfloat162float(__ushort_as_bfloat16(hi));
                    }
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < n; ++j) c[j] = load_attr(sh, (int64_t)n * i + j, dtype);
        }
    }
}

template <int K>
__device__ __forceinline__ void sh_colour_k(const void *sh, int64_t i, int dtype, const float *Y, float *rgb,
                                            float *raw)
{
    float c[3 * K];
    load_sh_row<K>(sh, i, dtype, c);
    float r = 0.5f, g = 0.5f, b = 0.5f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        r = fmaf(c[3 * k], Y[k], r);
        g = fmaf(c[3 * k + 1], Y[k], g);
        b = fmaf(c[3 * k + 2], Y[k], b);
    }
    raw[0] = r; raw[1] = g; raw[2] = b;
    rgb[0] = fmaxf(r, 0.f); rgb[1] = fmaxf(g, 0.f); rgb[2] = fmaxf(b, 0.f);
}

// Eq. 1: colour = max(0, 0.5 + sum_k SH_k Y_k(dir)) per channel, accumulated in
// index order; also returns the unclamped value (its sign gates the gradient).
__device__ __forceinline__ void sh_colour(const void *sh, int64_t i, int K, int dtype, const float *Y, float *rgb,
                                          float *raw)
{
    switch (K) {
    case 16: sh_colour_k<16>(sh, i, dtype, Y, rgb, raw); break;
    case 9: sh_colour_k<9>(sh, i, dtype, Y, rgb, raw); break;
    case 4: sh_colour_k<4>(sh, i, dtype, Y, rgb, raw); break;
    default: sh_colour_k<1>(sh, i, dtype, Y, rgb, raw); break;
    }
}

// Rotation of the normalised quaternion (w,x,y,z); columns are the local axes.
// Returns false for a zero-norm or non-finite quaternion.
__device__ __forceinline__ bool quat_to_rot(float w, float x, float y, float z, float *R, float *qn, float *qnorm)
{
    float n2 = w * w + x * x + y * y + z * z;
    if (!(n2 > 0.f) || !isfinite(n2)) return false;
    float n = sqrtf(n2), inv = 1.f / n;
    w *= inv; x *= inv; y *= inv; z *= inv;
    if (qn) { qn[0] = w; qn[1] = x; qn[2] = y; qn[3] = z; }
    if (qnorm) *qnorm = n;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
    return true;
}

__device__ __forceinline__ unsigned pack_xy(int x, int y) { return (unsigned)x | ((unsigned)y << 16); }

// ---------------------------------------------------------------------------
// Surfel raster record (64 B).  For a pixel centre (u,v), with du = u - ur,
// dv = v - vr (exact in float: ur, vr are multiples of 1/256):
//   invz = iz0 + gu du + gv dv          1/z of the ray-plane hit
//   A    = a0  + au du + av dv          a * invz / r   (a, b: disc coordinates
//   B    = b0  + bu du + bv dv          b * invz / r    scaled by s1, s2)
// The pixel is inside the opaque disc iff invz > 0 and A^2 + B^2 <= invz^2.
// (16-byte aligned: it is moved as four float4.)  The first three quarters
// hold what a coverage test reads (the id with the coefficients); the last
// one what the culling reads.
struct __align__(16) SurfelRec {
    float ur, vr, iz0, gu;
    float gv, au, av, a0;
    float bu, bv, b0;
    int id;
    float izmax;                  // largest 1/z over the disc (culling)
    unsigned bb_lo, bb_hi;        // pixel bbox (x | y << 16), inclusive
    float pad;
};
static_assert(sizeof(SurfelRec) == 64 && alignof(SurfelRec) == 16, "surfel record is 64 B, 16-aligned");

// Gaussian raster record (64 B).  alpha(u,v) = sigma * 2^-(y0^2 + y1^2) with
// y0 = la dx, y1 = lb dx + lc dy, dx = (u - px) - pxl (projected centre in
// double-float): (la, lb, lc) is the Cholesky factor of the conic
// Sigma2^-1 = [[a^2+b^2, bc], [bc, c^2]] scaled by sqrt(log2(e)/2), so that
// q = dx^T Sigma2^-1 dx = (a dx)^2 + (b dx + c dy)^2.  This sum of squares
// stays accurate far from the centre of elongated Gaussians, where the
// expanded quadratic form cancels.  Depth test: key = d - eps < D_s.
struct __align__(16) GaussRec {
    float px, py, pxl, pyl;
    float la, lb, lc, sigma;
    float key, r, g, b;
    int id;
    unsigned bb_lo, bb_hi;
    float pad;
};
static_assert(sizeof(GaussRec) == 64 && alignof(GaussRec) == 16, "Gaussian record is 64 B, 16-aligned");

// Eq. 1's view direction: the unit vector from the primitive's centre to the
// camera, and their distance (zero direction at distance 0).  The one
// definition used by the set-up and by the backward passes.
__device__ __forceinline__ void view_dir_o(float ox, float oy, float oz, float px, float py, float pz, float *dir,
                                           float &L)
{
    const float vx = ox - px, vy = oy - py, vz = oz - pz;
    L = sqrtf(vx * vx + vy * vy + vz * vz);
    const float il = L > 0.f ? 1.f / L : 0.f;
    dir[0] = vx * il; dir[1] = vy * il; dir[2] = vz * il;
}
__device__ __forceinline__ void view_dir(const CamParams &C, float px, float py, float pz, float *dir, float &L)
{
    view_dir_o(C.ocam[0], C.ocam[1], C.ocam[2], px, py, pz, dir, L);
}

struct SurfelOut {
    bool valid_quat;
    bool visible;
    SurfelRec rec;
    float rgb[3], raw[3], dir[3];
    int x0, y0, x1, y1;
};

// Conservative pixel range [lo, hi] of centres (i + 0.5) inside [a, b], clamped.
__device__ __forceinline__ void pixel_span(float a, float b, int n, int &lo, int &hi)
{
    float m = 0.02f + 1e-3f * fmaxf(b - a, 0.f);
    a -= m; b += m;
    float fl = ceilf(a - 0.5f), fh = floorf(b - 0.5f);
    // clamp before converting: NaN and huge values land in [-1, n]
    fl = fminf(fmaxf(fl, 0.f), (float)n);
    fh = fmaxf(fminf(fh, (float)(n - 1)), -1.f);
    lo = (int)fl; hi = (int)fh;
}

// Raster record of a planar disc a^2 + b^2 <= r^2 (a, b in units of the scales
// s1, s2 along the camera-space axes tu, tv; normal n; centre P in
// double-float): affine forms of 1/z and of (a/r)/z, (b/r)/z around a
// reference pixel, the largest 1/z over the disc, and a conservative pixel
// bbox widened by pad.  False when no part of it can be on screen.
struct DiscOut {
    SurfelRec rec;
    int x0, y0, x1, y1;
};

__device__ __forceinline__ bool disc_setup(const CamParams &C, const df *P, const float *tu, const float *tv,
                                           const float *n, float s1, float s2, float r, float pad, int id,
                                           DiscOut &o)
{
    const float Ph[3] = {P[0].hi, P[1].hi, P[2].hi};
    const float nP = fmaf(n[0], Ph[0], fmaf(n[1], Ph[1], n[2] * Ph[2])) +
                     (n[0] * P[0].lo + n[1] * P[1].lo + n[2] * P[2].lo);
    if (!(nP != 0.f) || !isfinite(nP)) return false;
    const float ez = r * sqrtf(s1 * tu[2] * s1 * tu[2] + s2 * tv[2] * s2 * tv[2]);
    const float zmax = Ph[2] + ez, zmin = Ph[2] - ez;
    if (!(zmax > C.znear * (1.f - 1e-5f) - 1e-6f)) return false;

    // --- affine coefficients (see SurfelRec) ---
    const float inP = 1.f / nP;
    const float gu = n[0] * inP / C.fx, gv = n[1] * inP / C.fy;
    float cA[3] = {tv[1] * Ph[2] - tv[2] * Ph[1], tv[2] * Ph[0] - tv[0] * Ph[2], tv[0] * Ph[1] - tv[1] * Ph[0]};
    float cB[3] = {Ph[1] * tu[2] - Ph[2] * tu[1], Ph[2] * tu[0] - Ph[0] * tu[2], Ph[0] * tu[1] - Ph[1] * tu[0]};
    const float ka = inP / (s1 * r), kb = inP / (s2 * r);
    const float au = cA[0] * ka / C.fx, av = cA[1] * ka / C.fy;
    const float bu = cB[0] * kb / C.fx, bv = cB[1] * kb / C.fy;

    // --- reference pixel: projection of a disc point in front of the camera,
    // rounded to 1/256 px; its local coordinates from small quantities only.
    float ur = 0.f, vr = 0.f, iz0 = 0.f, a0 = 0.f, b0 = 0.f;
    bool precise = false;
    {
        float oa = 0.f, ob = 0.f;
        float zp = Ph[2];
        if (!(Ph[2] > 0.5f * ez + C.znear)) {
            // centre too close to / behind the camera: take the disc point of
            // largest depth at 0.9 r
            float ga = s1 * tu[2], gb = s2 * tv[2];
            float gl = sqrtf(ga * ga + gb * gb);
            if (gl > 0.f) { oa = 0.9f * r * ga / gl; ob = 0.9f * r * gb / gl; }
            zp = Ph[2] + 0.9f * ez;
        }
        if (zp > C.znear * 1.01f) {
            df X[3];
            for (int k = 0; k < 3; ++k) X[k] = df_add_f(P[k], oa * s1 * tu[k] + ob * s2 * tv[k]);
            df uq = df_add_f(df_mul_f(df_div(X[0], X[2]), C.fx), C.cx);
            df vq = df_add_f(df_mul_f(df_div(X[1], X[2]), C.fy), C.cy);
            if (fabsf(uq.hi) < 16000.f && fabsf(vq.hi) < 16000.f) {
                ur = rintf(uq.hi * 256.f) * (1.f / 256.f);
                vr = rintf(vq.hi * 256.f) * (1.f / 256.f);
                float dur = (ur - uq.hi) - uq.lo, dvr = (vr - vq.hi) - vq.lo;
                float dr[3] = {dur / C.fx, dvr / C.fy, 0.f};
                float Xz = X[2].hi;
                float kap = Xz * (n[0] * dr[0] + n[1] * dr[1]) * inP;
                float opk = 1.f + kap;
                float zref = Xz / opk;
                float f = -kap / opk;
                float dX[3];
                for (int k = 0; k < 3; ++k) dX[k] = fmaf(f, X[k].hi, zref * dr[k]) + f * X[k].lo;
                float aref = oa + (dX[0] * tu[0] + dX[1] * tu[1] + dX[2] * tu[2]) / s1;
                float bref = ob + (dX[0] * tv[0] + dX[1] * tv[1] + dX[2] * tv[2]) / s2;
                // 1/zref = (1+kap)/(X.hi + X.lo)
                float izx = 1.f / Xz;
                izx = izx * (1.f - X[2].lo * izx);
                iz0 = opk * izx;
                a0 = iz0 * aref / r;
                b0 = iz0 * bref / r;
                precise = true;
            }
        }
        if (!precise) {
            // plain evaluation at the image centre (rare: huge discs at the camera)
            ur = rintf(C.cx * 256.f) * (1.f / 256.f);
            vr = rintf(C.cy * 256.f) * (1.f / 256.f);
            float d[3] = {(ur - C.cx) / C.fx, (vr - C.cy) / C.fy, 1.f};
            iz0 = (n[0] * d[0] + n[1] * d[1] + n[2] * d[2]) * inP;
            float dtu = d[0] * tu[0] + d[1] * tu[1] + d[2] * tu[2];
            float dtv = d[0] * tv[0] + d[1] * tv[1] + d[2] * tv[2];
            float Ptu = Ph[0] * tu[0] + Ph[1] * tu[1] + Ph[2] * tu[2];
            float Ptv = Ph[0] * tv[0] + Ph[1] * tv[1] + Ph[2] * tv[2];
            a0 = (dtu - iz0 * Ptu) / (s1 * r);
            b0 = (dtv - iz0 * Ptv) / (s2 * r);
        }
    }

    // --- conservative screen bbox ---
    float umin = 1e30f, umax = -1e30f, vmin = 1e30f, vmax = -1e30f;
    bool have_box = false;
    if (zmin > C.znear * 1.001f && precise) {
        // exact bbox of the projected ellipse from its dual conic, in
        // coordinates relative to the reference pixel: the disc is
        // {A^2 + B^2 - invz^2 <= 0}; its dual is adj(M), M = a a^T + b b^T - c c^T
        const float a_[3] = {au, av, a0}, b_[3] = {bu, bv, b0}, c_[3] = {gu, gv, iz0};
        float M[3][3];
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) M[x][y] = a_[x] * a_[y] + b_[x] * b_[y] - c_[x] * c_[y];
        const float D00 = M[1][1] * M[2][2] - M[1][2] * M[2][1];
        const float D11 = M[0][0] * M[2][2] - M[0][2] * M[2][0];
        const float D22 = M[0][0] * M[1][1] - M[0][1] * M[1][0];
        const float D02 = M[0][1] * M[1][2] - M[0][2] * M[1][1];
        const float D12 = M[0][2] * M[1][0] - M[0][0] * M[1][2];
        const float du = D02 * D02 - D00 * D22, dv = D12 * D12 - D11 * D22;
        if (D22 != 0.f && du >= 0.f && dv >= 0.f && isfinite(du) && isfinite(dv)) {
            const float sdu = sqrtf(du), sdv = sqrtf(dv);
            const float u1 = (D02 - sdu) / D22, u2 = (D02 + sdu) / D22;
            const float v1 = (D12 - sdv) / D22, v2 = (D12 + sdv) / D22;
            umin = ur + fminf(u1, u2); umax = ur + fmaxf(u1, u2);
            vmin = vr + fminf(v1, v2); vmax = vr + fmaxf(v1, v2);
            have_box = isfinite(umin) && isfinite(umax) && isfinite(vmin) && isfinite(vmax);
        }
    }
    if (!have_box) {
        // rectangle p +- r s1 tu +- r s2 tv clipped to z >= znear
        float cor[4][3], poly[8][3];
        const float sg[4][2] = {{1.f, 1.f}, {-1.f, 1.f}, {-1.f, -1.f}, {1.f, -1.f}};
        const float rr = r * 1.0001f;
        for (int k = 0; k < 4; ++k)
            for (int j = 0; j < 3; ++j)
                cor[k][j] = Ph[j] + sg[k][0] * rr * s1 * tu[j] + sg[k][1] * rr * s2 * tv[j];
        int np = 0;
        const float zc = C.znear * 0.999f;
        for (int k = 0; k < 4; ++k) {
            const float *a = cor[k], *b = cor[(k + 1) & 3];
            bool ia = a[2] >= zc, ib = b[2] >= zc;
            if (ia) { poly[np][0] = a[0]; poly[np][1] = a[1]; poly[np][2] = a[2]; ++np; }
            if (ia != ib) {
                float tt = (zc - a[2]) / (b[2] - a[2]);
                poly[np][0] = a[0] + tt * (b[0] - a[0]);
                poly[np][1] = a[1] + tt * (b[1] - a[1]);
                poly[np][2] = zc;
                ++np;
            }
        }
        if (np == 0) return false;
        for (int k = 0; k < np; ++k) {
            float izk = 1.f / poly[k][2];
            float u = C.fx * poly[k][0] * izk + C.cx, v = C.fy * poly[k][1] * izk + C.cy;
            umin = fminf(umin, u); umax = fmaxf(umax, u); vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
        }
        // one pixel of slack for the float projection of the clipped polygon
        umin -= 1.f; vmin -= 1.f; umax += 1.f; vmax += 1.f;
    }
    // widen the interval of pixel centres by pad (4x multisampling: a pixel is
    // touched when a sample at +-0.25 px from its centre falls inside)
    umin -= pad; vmin -= pad; umax += pad; vmax += pad;
    int x0, x1, y0, y1;
    pixel_span(fmaxf(umin, -1e6f), fminf(umax, 1e6f), C.W, x0, x1);
    pixel_span(fmaxf(vmin, -1e6f), fminf(vmax, 1e6f), C.H, y0, y1);
    if (x0 > x1 || y0 > y1) return false;
    o.x0 = x0; o.x1 = x1; o.y0 = y0; o.y1 = y1;

    float izmax = zmin > C.znear ? (1.f / zmin) * (1.f + 4e-6f) : C.izn * (1.f + 4e-6f);
    o.rec = SurfelRec{ur, vr, iz0, gu, gv, au, av, a0, bu, bv, b0, id, izmax,
                      pack_xy(x0, y0), pack_xy(x1, y1), 0.f};
    return true;
}

// Per-surfel set-up for the view (Sec. 3: disc placed by scale, rotation,
// translation; opaque extent of Sec. 4.1).  Produces the raster record, the
// colour (Eq. 1) and a conservative pixel bbox.
// tside (translucent render only; null elsewhere, which removes the stores):
// the camera-space frame (P, s1), (U, s2), (V, -), (N, -) of a visible surfel.
// surfel_geom: everything but the colour (visible: drawn somewhere).
__device__ __forceinline__ void surfel_geom(const SceneView &S, const CamParams &C, const OptParams &O,
                                            int64_t i, SurfelOut &o, float4 *tside = nullptr)
{
    o.visible = false;
    o.valid_quat = true;
    // every attribute load is issued before the first use (one round trip)
    const float px = __ldg(S.s_pos + 3 * i), py = __ldg(S.s_pos + 3 * i + 1), pz = __ldg(S.s_pos + 3 * i + 2);
    float q[4], R[9];
    for (int k = 0; k < 4; ++k) q[k] = load_attr(S.s_rot, 4 * i + k, S.attr_dtype);
    const float s1 = load_attr(S.s_scale, 2 * i, S.attr_dtype), s2 = load_attr(S.s_scale, 2 * i + 1, S.attr_dtype);
    if (!quat_to_rot(q[0], q[1], q[2], q[3], R, nullptr, nullptr)) { o.valid_quat = false; return; }
    // view direction for the SH colour: from the surfel centre to the camera
    {
        float L;
        view_dir(C, px, py, pz, o.dir, L);
    }
    if (!(s1 > 0.f && s2 > 0.f && isfinite(s1) && isfinite(s2))) return;
    // camera-space frame (float) and centre (double-float)
    float tu[3], tv[3], n[3];
    for (int r = 0; r < 3; ++r) {
        tu[r] = C.R[3 * r] * R[0] + C.R[3 * r + 1] * R[3] + C.R[3 * r + 2] * R[6];
        tv[r] = C.R[3 * r] * R[1] + C.R[3 * r + 1] * R[4] + C.R[3 * r + 2] * R[7];
        n[r] = C.R[3 * r] * R[2] + C.R[3 * r + 1] * R[5] + C.R[3 * r + 2] * R[8];
    }
    df P[3];
    for (int r = 0; r < 3; ++r) P[r] = df_dot3_plus(C.R + 3 * r, px, py, pz, C.t[r]);
    DiscOut d;
    if (!disc_setup(C, P, tu, tv, n, s1, s2, O.surfel_r, O.samples == 4 ? 0.25f : 0.f, (int)i, d)) return;
    if (tside) {
        tside[0] = make_float4(P[0].hi, P[1].hi, P[2].hi, s1);
        tside[1] = make_float4(tu[0], tu[1], tu[2], s2);
        tside[2] = make_float4(tv[0], tv[1], tv[2], 0.f);
        tside[3] = make_float4(n[0], n[1], n[2], 0.f);
    }
    o.rec = d.rec;
    o.x0 = d.x0; o.y0 = d.y0; o.x1 = d.x1; o.y1 = d.y1;
    o.visible = true;
}

// The colour of a surfel set up by surfel_geom (Eq. 1 at o.dir).
__device__ __forceinline__ void surfel_colour(const SceneView &S, int64_t i, SurfelOut &o)
{
    const int K = (S.deg + 1) * (S.deg + 1);
    float Y[16];
    sh_basis(K, o.dir[0], o.dir[1], o.dir[2], Y);
    sh_colour(S.s_sh, i, K, S.sh_dtype, Y, o.rgb, o.raw);
}

struct GaussOut {
    bool valid_quat;
    bool visible;
    GaussRec rec;
    float rgb[3], raw[3], dir[3], dist;
    // intermediates for the backward pass
    float R[9], qn[4], qnorm, s[3];
    float tx, ty, tz;
    float S2a, S2b, S2c;      // Sigma2 (with low-pass)
    float ia, ib, ic;         // conic Sigma2^-1 (unscaled)
    float sigma0, k3, k2;     // stored opacity and the Mip-GES 3D / screen filter factors
    float se[3];              // axis lengths after the 3D filter (= s without it)
    float n0, n1, det0;       // Sigma2 before the screen filter: diagonal and determinant
    int x0, y0, x1, y1;
    // 2D Gaussians: a disc record (SurfelRec layout, eps in its last word)
    // instead of rec; both kinds: side data for g_aux
    SurfelRec drec;
    float4 aux[2];
    // 2D Gaussians, for the backward pass: object-space filter factors S1, S2
    // and the support radius in filtered units (tx, ty, tz: the centre)
    float S1, S2, rsup;
};

// Per-Gaussian set-up (Eq. 4: projected covariance and centre; 1/255 clamp
// gives the exact support q <= 2 ln(sigma/alpha_min); eps of Sec. 5).
// Mip-GES (Sec. 6.1): the 3D filter variance v widens the axes to
// sqrt(s^2 + v) and scales the opacity by prod |s_j| / sqrt(s_j^2 + v); the
// screen filter (GES_FILTER_MIP) scales it by sqrt(|Sigma2'| / |Sigma2' + lowpass I|),
// Sigma2' the projected covariance before the dilation.
// gauss_geom: everything but the colour (visible: drawn somewhere).
__device__ __forceinline__ void gauss_geom(const SceneView &S, const CamParams &C, const OptParams &O,
                                           int64_t i, GaussOut &o)
{
    o.visible = false;
    o.valid_quat = true;
    // every attribute load is issued before the first use (one round trip)
    const float px = __ldg(S.g_pos + 3 * i), py = __ldg(S.g_pos + 3 * i + 1), pz = __ldg(S.g_pos + 3 * i + 2);
    float q[4];
    for (int k = 0; k < 4; ++k) q[k] = load_attr(S.g_rot, 4 * i + k, S.attr_dtype);
    for (int k = 0; k < 3; ++k) o.s[k] = load_attr(S.g_scale, 3 * i + k, S.attr_dtype);
    float sigma = load_attr(S.g_opac, i, S.attr_dtype);
    if (!quat_to_rot(q[0], q[1], q[2], q[3], o.R, o.qn, &o.qnorm)) { o.valid_quat = false; return; }
    o.sigma0 = sigma;
    o.k3 = 1.f; o.k2 = 1.f;
    o.se[0] = o.s[0]; o.se[1] = o.s[1]; o.se[2] = o.s[2];
    if (S.g_filt3) {
        const float v = __ldg(S.g_filt3 + i);
        if (v != 0.f) {
            for (int k = 0; k < 3; ++k) {
                o.se[k] = sqrtf(fmaf(o.s[k], o.s[k], v));
                o.k3 *= fabsf(o.s[k]) / o.se[k];
            }
        }
    }
    view_dir(C, px, py, pz, o.dir, o.dist);
    // alpha <= sigma k3 k2 <= sigma k3 < alpha_min everywhere
    if (!(sigma * o.k3 >= O.alpha_min)) return;
    df t[3];
    for (int r = 0; r < 3; ++r) t[r] = df_dot3_plus(C.R + 3 * r, px, py, pz, C.t[r]);
    if (!(t[2].hi > C.znear || (t[2].hi == C.znear && t[2].lo > 0.f))) return;
    const float x = t[0].hi, y = t[1].hi, z = t[2].hi;
    o.tx = x; o.ty = y; o.tz = z;
    // Sigma3 = (R S)(R S)^T, kept factored as Mm = R S
    float Mm[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Mm[3 * a + b] = o.R[3 * a + b] * o.se[b];
    // T = J Rc with the affine Jacobian of the perspective map at the centre
    const float iz = 1.f / z;
    const float J00 = C.fx * iz, J02 = -C.fx * x * iz * iz, J11 = C.fy * iz, J12 = -C.fy * y * iz * iz;
    float T[6];
    for (int b = 0; b < 3; ++b) {
        T[b] = J00 * C.R[b] + J02 * C.R[6 + b];
        T[3 + b] = J11 * C.R[3 + b] + J12 * C.R[6 + b];
    }
    // Sigma2 = P P^T + lowpass I with P = T (R S) (2x3).  Its determinant by
    // the Lagrange identity, |P0 x P1|^2 + lowpass (|P0|^2 + |P1|^2) +
    // lowpass^2: a sum of non-negative terms, where s2a s2c - s2b^2 cancels
    // for elongated footprints.
    float P0[3], P1[3];
    for (int b = 0; b < 3; ++b) {
        P0[b] = T[0] * Mm[b] + T[1] * Mm[3 + b] + T[2] * Mm[6 + b];
        P1[b] = T[3] * Mm[b] + T[4] * Mm[3 + b] + T[5] * Mm[6 + b];
    }
    const float n0 = P0[0] * P0[0] + P0[1] * P0[1] + P0[2] * P0[2];
    const float n1 = P1[0] * P1[0] + P1[1] * P1[1] + P1[2] * P1[2];
    const float s2a = n0 + O.lowpass;
    const float s2b = P0[0] * P1[0] + P0[1] * P1[1] + P0[2] * P1[2];
    const float s2c = n1 + O.lowpass;
    const float x0c = P0[1] * P1[2] - P0[2] * P1[1], x1c = P0[2] * P1[0] - P0[0] * P1[2];
    const float x2c = P0[0] * P1[1] - P0[1] * P1[0];
    const float det0 = x0c * x0c + x1c * x1c + x2c * x2c;
    const float det = det0 + O.lowpass * (n0 + n1) + O.lowpass * O.lowpass;
    if (!(det > 0.f) || !isfinite(det) || !(s2a > 0.f)) return;
    o.n0 = n0; o.n1 = n1; o.det0 = det0;
    if (O.filter == GES_FILTER_MIP) o.k2 = sqrtf(det0 / det);
    sigma *= o.k3 * o.k2;
    if (!(sigma >= O.alpha_min)) return;
    const float idet = 1.f / det;
    const float ia = s2c * idet, ib = -s2b * idet, ic = s2a * idet;
    // Cholesky factor of the conic: a = 1/sqrt(s2a), b = -s2b/(sqrt(s2a det)), c = sqrt(s2a/det)
    const float l00 = sqrtf(s2a), sdet = sqrtf(det);
    const float fa = 1.f / l00, fb = -s2b / (l00 * sdet), fc = l00 / sdet;
    o.S2a = s2a; o.S2b = s2b; o.S2c = s2c; o.ia = ia; o.ib = ib; o.ic = ic;
    // projected centre in double-float
    df uq = df_add_f(df_mul_f(df_div(t[0], t[2]), C.fx), C.cx);
    df vq = df_add_f(df_mul_f(df_div(t[1], t[2]), C.fy), C.cy);
    // exact support bbox: alpha >= alpha_min  <=>  q <= 2 ln(sigma / alpha_min)
    const float Ts = 2.f * logf(sigma / O.alpha_min);
    const float hx = sqrtf(fmaxf(Ts, 0.f) * s2a), hy = sqrtf(fmaxf(Ts, 0.f) * s2c);
    int x0, x1, y0, y1;
    pixel_span(uq.hi - hx, uq.hi + hx, C.W, x0, x1);
    pixel_span(vq.hi - hy, vq.hi + hy, C.H, y0, y1);
    if (x0 > x1 || y0 > y1) return;
    o.x0 = x0; o.x1 = x1; o.y0 = y0; o.y1 = y1;
    float eps;
    if (O.eps_mode == GES_EPS_ADAPTIVE) eps = O.eps_factor * (1.f / 3.f) * (o.s[0] + o.s[1] + o.s[2]);
    else if (O.eps_mode == GES_EPS_ZERO) eps = 0.f;
    else eps = O.eps_value;
    const float key = (t[2].hi - eps) + t[2].lo;
    const float kL = 0.84932180028801904f;   // sqrt(log2(e) / 2)
    o.rec.px = uq.hi; o.rec.py = vq.hi; o.rec.pxl = uq.lo; o.rec.pyl = vq.lo;
    o.rec.la = kL * fa; o.rec.lb = kL * fb; o.rec.lc = kL * fc;
    o.rec.sigma = sigma; o.rec.key = key;
    o.rec.id = (int)i;
    o.rec.bb_lo = pack_xy(x0, y0); o.rec.bb_hi = pack_xy(x1, y1);
    o.rec.pad = key;              // the culling reads key with the bbox
    if (O.geo) {
        // geometry (Sec. 6.4): d_i = centre depth, n_i = the axis of the smallest
        // scale, camera space, facing the camera
        // (the column is selected, not indexed: a run-time index into o.s or
        // o.R would keep those arrays, and the set-up around them, in local
        // memory)
        const float a0 = fabsf(o.s[0]), a1 = fabsf(o.s[1]), a2 = fabsf(o.s[2]);
        const int km = a1 < a0 ? (a2 < a1 ? 2 : 1) : (a2 < a0 ? 2 : 0);
        float ax[3];
        for (int r = 0; r < 3; ++r) ax[r] = km == 0 ? o.R[3 * r] : (km == 1 ? o.R[3 * r + 1] : o.R[3 * r + 2]);
        float nc[3];
        for (int r = 0; r < 3; ++r) nc[r] = C.R[3 * r] * ax[0] + C.R[3 * r + 1] * ax[1] + C.R[3 * r + 2] * ax[2];
        const float fl = (nc[0] * x + nc[1] * y + nc[2] * z) > 0.f ? -1.f : 1.f;
        o.aux[0] = make_float4(fl * nc[0], fl * nc[1], fl * nc[2], z);
        o.aux[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    o.visible = true;
}

// The colour of a Gaussian set up by gauss_geom (Eq. 1 at o.dir), also into
// its record (at most kColourMax there).
__device__ __forceinline__ void gauss_colour(const SceneView &S, int64_t i, GaussOut &o)
{
    const int K = (S.deg + 1) * (S.deg + 1);
    float Y[16];
    sh_basis(K, o.dir[0], o.dir[1], o.dir[2], Y);
    sh_colour(S.g_sh, i, K, S.sh_dtype, Y, o.rgb, o.raw);
    o.rec.r = fminf(o.rgb[0], kColourMax); o.rec.g = fminf(o.rgb[1], kColourMax);
    o.rec.b = fminf(o.rgb[2], kColourMax);
}

// Geometry and colour.
__device__ __forceinline__ void gauss_setup(const SceneView &S, const CamParams &C, const OptParams &O,
                                            int64_t i, GaussOut &o)
{
    gauss_geom(S, C, O, i, o);
    if (o.visible) gauss_colour(S, i, o);
}

// 2D Gaussian of 2D-GES (Sec. 6.4): a splat in the plane of its rotation's
// first two axes, opacity sigma exp(-(a^2 + b^2)/2) at the ray-splat hit (a, b
// in scale units), planar depth for the depth test.  The screen-space EWA
// filter of size lowpass is back-projected into object space (Eq. 17-18):
// with J the Jacobian of local unit coordinates -> pixels at the centre, the
// scales become s_k S_k and the opacity sigma / (S1 S2), with
// S_k = sqrt(1 + lowpass ((J^T J)^-1)_kk) (the diagonal of I + lowpass J^-1 J^-T).
// The support alpha >= alpha_min is the disc of radius r = sqrt(2 ln(sigma'/alpha_min))
// in filtered units, so the record is a disc record (disc_setup) and
// alpha = 2^(log2 sigma' + log2(alpha_min/sigma') rho), rho = (a'^2 + b'^2)/r^2.
// colour false: the side word's colour is left at 0 for a later pass (the
// batch evaluates the colours of all views of a scene in one kernel).
__device__ __forceinline__ void gauss2d_setup(const SceneView &S, const CamParams &C, const OptParams &O,
                                              int64_t i, GaussOut &o, bool colour = true)
{
    o.visible = false;
    o.valid_quat = true;
    const float px = __ldg(S.g_pos + 3 * i), py = __ldg(S.g_pos + 3 * i + 1), pz = __ldg(S.g_pos + 3 * i + 2);
    float q[4];
    for (int k = 0; k < 4; ++k) q[k] = load_attr(S.g_rot, 4 * i + k, S.attr_dtype);
    if (!quat_to_rot(q[0], q[1], q[2], q[3], o.R, o.qn, &o.qnorm)) { o.valid_quat = false; return; }
    const float s0 = load_attr(S.g_scale, 2 * i, S.attr_dtype), s1 = load_attr(S.g_scale, 2 * i + 1, S.attr_dtype);
    o.s[0] = s0; o.s[1] = s1; o.s[2] = 0.f;
    const float sigma = load_attr(S.g_opac, i, S.attr_dtype);
    o.sigma0 = sigma;
    view_dir(C, px, py, pz, o.dir, o.dist);
    if (!(sigma >= O.alpha_min)) return;            // sigma' <= sigma
    if (!(s0 > 0.f && s1 > 0.f && isfinite(s0) && isfinite(s1))) return;
    float tu[3], tv[3], n[3];
    for (int r = 0; r < 3; ++r) {
        tu[r] = C.R[3 * r] * o.R[0] + C.R[3 * r + 1] * o.R[3] + C.R[3 * r + 2] * o.R[6];
        tv[r] = C.R[3 * r] * o.R[1] + C.R[3 * r + 1] * o.R[4] + C.R[3 * r + 2] * o.R[7];
        n[r] = C.R[3 * r] * o.R[2] + C.R[3 * r + 1] * o.R[5] + C.R[3 * r + 2] * o.R[8];
    }
    df P[3];
    for (int r = 0; r < 3; ++r) P[r] = df_dot3_plus(C.R + 3 * r, px, py, pz, C.t[r]);
    if (!(P[2].hi > C.znear || (P[2].hi == C.znear && P[2].lo > 0.f))) return;
    // object-space filter
    const float x = P[0].hi, y = P[1].hi, z = P[2].hi, iz = 1.f / z;
    const float j00 = C.fx * iz, j02 = -C.fx * x * iz * iz, j11 = C.fy * iz, j12 = -C.fy * y * iz * iz;
    const float J00 = s0 * (j00 * tu[0] + j02 * tu[2]), J01 = s1 * (j00 * tv[0] + j02 * tv[2]);
    const float J10 = s0 * (j11 * tu[1] + j12 * tu[2]), J11 = s1 * (j11 * tv[1] + j12 * tv[2]);
    const float dJ = J00 * J11 - J01 * J10;         // det(J^T J) = det(J)^2
    const float det = dJ * dJ;
    if (!(det > 0.f) || !isfinite(det)) return;
    const float M00 = J00 * J00 + J10 * J10, M11 = J01 * J01 + J11 * J11;
    const float S1 = sqrtf(1.f + O.lowpass * M11 / det), S2 = sqrtf(1.f + O.lowpass * M00 / det);
    const float sigp = sigma / (S1 * S2);
    if (!(sigp >= O.alpha_min)) return;
    const float r = sqrtf(2.f * logf(sigp / O.alpha_min));
    if (!(r > 0.f)) return;
    o.tx = x; o.ty = y; o.tz = z;
    o.S1 = S1; o.S2 = S2; o.rsup = r;
    DiscOut d;
    if (!disc_setup(C, P, tu, tv, n, s0 * S1, s1 * S2, r, 0.f, (int)i, d)) return;
    float eps;
    if (O.eps_mode == GES_EPS_ADAPTIVE) eps = O.eps_factor * 0.5f * (s0 + s1);
    else if (O.eps_mode == GES_EPS_ZERO) eps = 0.f;
    else eps = O.eps_value;
    o.drec = d.rec;
    o.drec.pad = eps;
    o.x0 = d.x0; o.y0 = d.y0; o.x1 = d.x1; o.y1 = d.y1;
    const float nP = n[0] * x + n[1] * y + n[2] * z;
    const float fl = nP > 0.f ? -1.f : 1.f;
    const float lsig = log2f(sigp);
    if (colour) {
        const int K = (S.deg + 1) * (S.deg + 1);
        float Y[16];
        sh_basis(K, o.dir[0], o.dir[1], o.dir[2], Y);
        sh_colour(S.g_sh, i, K, S.sh_dtype, Y, o.rgb, o.raw);
        o.aux[0] = make_float4(colour_q(o.rgb[0]), colour_q(o.rgb[1]), colour_q(o.rgb[2]), lsig);
    } else {
        o.aux[0] = make_float4(0.f, 0.f, 0.f, lsig);
    }
    o.aux[1] = make_float4(fl * n[0], fl * n[1], fl * n[2], log2f(O.alpha_min) - lsig);
    o.visible = true;
}

// float -> int64 rounded to nearest (ties to even) for the fixed-point sums,
// on the FP32 and integer pipes (the library's int64 conversion runs on the
// FP64 pipe, which GB300 has little of: it limited the Gaussian pass).  For
// |x| < 2^42 the result equals __float2ll_rn(x) exactly: x = h 2^20 + l with
// h = rint(x 2^-20) and |l| <= 2^19 both exact in float, each rounded to an
// integer by adding 1.5 2^23 (where the float spacing is 1) and reading the
// bits.  Callers keep their terms inside that range (see kColourMax).
__device__ __forceinline__ long long f2ll_rn(float x)
{
    const float M = 12582912.f;                        // 1.5 2^23
    const float t = fmaf(x, 9.5367431640625e-07f, M);  // x 2^-20 + M, rounded to an integer
    const float h = t - M;                             // that integer, exactly
    const float l = fmaf(-h, 1048576.f, x);            // x - h 2^20, exactly
    const int hi = __float_as_int(t) - __float_as_int(M);
    const int li = __float_as_int(l + M) - __float_as_int(M);
    return (long long)hi * 1048576LL + li;
}

// Row of pixel k of a w-wide bbox walked row-major (k / w) without an integer
// division: the quotient from the float reciprocal iw = 1/w is within one of
// the exact one for every bbox of an image of at most 16384^2 (k exact in
// float below 2^24; beyond, w >= 32), and the two fix-ups make it exact.
__device__ __forceinline__ int bbox_row(int k, int w, float iw)
{
    int r = (int)(((float)k + 0.5f) * iw);
    r -= (r * w > k) ? 1 : 0;
    r += ((r + 1) * w <= k) ? 1 : 0;
    return r;
}

// Sums NV <= 32 per-lane values over the warp and hands total i to exactly
// one lane, as f(i, total).  A halving exchange: at the xor-16, 8, 4, 2 and 1
// steps a lane keeps the lower or the upper part of its slots (by its lane
// bit), adds the partner's copy of that part and sends the other part
// (ceil(n/2) shuffles per step, missing slots zero): 20 shuffles for 18
// values instead of 90 for 18 butterflies.  The order is fixed, so the
// result is deterministic.
template <int NV, class F>
__device__ __forceinline__ void warp_reduce_scatter(const float *v, int lane, F f)
{
    constexpr int n1 = (NV + 1) / 2, n2 = (n1 + 1) / 2, n3 = (n2 + 1) / 2, n4 = (n3 + 1) / 2;
    static_assert(NV >= 1 && NV <= 32, "1 to 32 values");
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2, b0 = lane & 1;
    float a1[n1], a2[n2], a3[n3], a4[n4];
#pragma unroll
    for (int i = 0; i < n1; ++i) {
        const float lo = v[i], hi = i + n1 < NV ? v[i + n1] : 0.f;
        a1[i] = (b4 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b4 ? lo : hi, 16);
    }
#pragma unroll
    for (int i = 0; i < n2; ++i) {
        const float lo = a1[i], hi = i + n2 < n1 ? a1[i + n2] : 0.f;
        a2[i] = (b3 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b3 ? lo : hi, 8);
    }
#pragma unroll
    for (int i = 0; i < n3; ++i) {
        const float lo = a2[i], hi = i + n3 < n2 ? a2[i + n3] : 0.f;
        a3[i] = (b2 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b2 ? lo : hi, 4);
    }
#pragma unroll
    for (int i = 0; i < n4; ++i) {
        const float lo = a3[i], hi = i + n4 < n3 ? a3[i + n4] : 0.f;
        a4[i] = (b1 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b1 ? lo : hi, 2);
    }
    const float lo = a4[0], hi = n4 > 1 ? a4[n4 - 1] : 0.f;
    const float tot = (b0 ? hi : lo) + __shfl_xor_sync(0xffffffffu, b0 ? lo : hi, 1);
    // the slot this lane ends with, level by level
    const int s4 = b0 ? 1 : 0, s3 = (b1 ? n4 : 0) + s4, s2 = (b2 ? n3 : 0) + s3;
    const int s1 = (b3 ? n2 : 0) + s2, s0 = (b4 ? n1 : 0) + s1;
    if (s4 < n4 && s3 < n3 && s2 < n2 && s1 < n1 && s0 < NV) f(s0, tot);
}

// gd = sum_k (SH_k . gc) grad Y_k at the unit direction dir: the SH row is
// read in index order and the basis gradients are those of sh_basis_grad
// (compile-time K: no per-k array in local memory).
template <int K>
__device__ __forceinline__ void sh_weighted_grad(const void *sh, int64_t i, int dtype, const float *gc,
                                                 const float *dir, float *gd)
{
    float dY[K][3];
    sh_basis_grad(K, dir[0], dir[1], dir[2], dY);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float c[3];
        for (int q = 0; q < 3; ++q) c[q] = load_attr(sh, (int64_t)3 * K * i + 3 * k + q, dtype);
        const float w = c[0] * gc[0] + c[1] * gc[1] + c[2] * gc[2];
        for (int a = 0; a < 3; ++a) gd[a] += w * dY[k][a];
    }
}

// n zeros from dst (16-byte stores when dst is 16-byte aligned and n % 4 == 0)
__device__ __forceinline__ void store_zeros(float *dst, int n)
{
    if (((reinterpret_cast<uintptr_t>(dst) & 15u) == 0) && (n & 3) == 0) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        for (int k = 0; k < n / 4; ++k) d4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        for (int k = 0; k < n; ++k) dst[k] = 0.f;
    }
}

// SH coefficient gradients of one primitive: dst[3k + c] = Y_k gc_c, zero for
// the channels whose unclamped colour raw_c is not positive (raw null: no
// gate).  A thread writes 3K consecutive floats, in 16-byte stores where the
// row allows it (fewer, fuller memory transactions than scalar stores).  K is
// a template parameter so that every index into Y and g is a constant: a
// run-time index would put both arrays in local memory.
template <int K>
__device__ __forceinline__ void store_sh_grad_k(float *dst, const float *Y, const float *g)
{
    if (((3 * K) & 3) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0) {
        // 3K = 4 m: float4 number q holds entries 4q .. 4q + 3, i.e. basis
        // functions (4q + e) / 3 and channels (4q + e) % 3
        float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
        for (int q = 0; q < (3 * K) / 4; ++q) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int idx = 4 * q + e;
                v[e] = Y[idx / 3] * g[idx % 3];
            }
            d4[q] = make_float4(v[0], v[1], v[2], v[3]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) dst[3 * k + c] = Y[k] * g[c];
    }
}
__device__ __forceinline__ void store_sh_grad(float *dst, int K, const float *Y, const float *gc, const float *raw)
{
    float g[3];
    for (int c = 0; c < 3; ++c) g[c] = (raw == nullptr || raw[c] > 0.f) ? gc[c] : 0.f;
    switch (K) {
    case 16: store_sh_grad_k<16>(dst, Y, g); break;
    case 9: store_sh_grad_k<9>(dst, Y, g); break;
    case 4: store_sh_grad_k<4>(dst, Y, g); break;
    default: store_sh_grad_k<1>(dst, Y, g); break;
    }
}

// Eq. 4 at pixel centre (u, v): the one definition used by forward and backward.
__device__ __forceinline__ float gauss_alpha(const GaussRec &g, float u, float v, float &e)
{
    const float dx = (u - g.px) - g.pxl, dy = (v - g.py) - g.pyl;
    const float y0 = g.la * dx, y1 = fmaf(g.lb, dx, g.lc * dy);
    e = ex2_approx(-fmaf(y0, y0, y1 * y1));
    return g.sigma * e;
}

#endif  // __CUDACC__

}  // namespace ges
