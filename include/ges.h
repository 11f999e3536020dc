/*
 * ges.h -- C ABI of the Gaussian-enhanced Surfels (GES) renderer for GB300.
 *
 * The problem (Sec. 3): a scene is a set of opaque 2D surfels
 * S = {p_i, r_i, s_i, SH_i} and a set of 3D Gaussians G = {p_i, sigma_i, r_i,
 * s_i, SH_i}.  Rendering runs two passes.  Pass 1 rasterises the surfels with
 * a z-buffer into a colour map C_s and a depth map D_s.  Pass 2 splats the
 * Gaussians, keeps those whose centre depth passes d_i < D_s + eps_i (Eq. 2-3),
 * weights them by the 2D opacity of Eq. 4 (zero below 1/255) and composites
 * C = (C_s W_s + C_G) / (W_s + W_G) with W_s = 1 (Eq. 5).  No sorting is
 * involved anywhere.  The joint optimisation stage (Sec. 4.2) needs the
 * gradients of C with respect to the Gaussians and the surfel SH
 * coefficients; surfel geometry is fixed there and receives none.
 *
 * Conventions (readings where the paper is silent):
 *  - cameras: OpenCV axes (x right, y down, z forward), row-major world-to-
 *    camera [R|t], pinhole fx, fy, cx, cy; pixel (i,j) is sampled at its
 *    centre (i+0.5, j+0.5); depths are camera-space z; images are planar CHW
 *    float32, row-major.
 *  - quaternions are (w,x,y,z) and are normalised before use; scales are
 *    linear axis lengths; opacities are activated values in [0,1].
 *  - SH: real spherical harmonics with the Condon-Shortley phase, index
 *    k = l^2 + l + m, degree <= 3, evaluated at the unit direction from the
 *    primitive centre to the camera (Eq. 1); colour = max(0, 0.5 + sum).
 *  - surfel opaque extent: a^2 + b^2 <= 2 ln 255 in scale-normalised local
 *    coordinates (Sec. 4.1, Eq. 6-7 at w = 255).  z-buffer ties go to the
 *    lower surfel index.  Surfels are two-sided.
 *  - Gaussians: EWA projection with the affine Jacobian at the centre and a
 *    fixed screen-space low-pass of 0.3 added to the 2D covariance;
 *    eps_i = (5/3)(s_1 + s_2 + s_3) (Sec. 5).
 *  - background: C_s = bg, D_s = +inf where no surfel covers a pixel.
 *
 * Memory: every pointer passed to the render and backward calls is a DEVICE
 * pointer, C-contiguous, owned by the caller; the library never frees it.
 * The library owns only its scratch (per-primitive records and tile lists),
 * which grows on demand, is reused across calls and is released by
 * ges_destroy_scene.  A scene is not thread-safe: use one scene per host
 * thread and stream.
 *
 * Errors: every call returns a ges_status and never aborts.  On any status
 * other than GES_OK the outputs are undefined; ges_last_error_message()
 * returns a thread-local description of the last failure.
 */
#ifndef GES_H
#define GES_H

#include <stdint.h>

#if defined(__GNUC__)
#define GES_API __attribute__((visibility("default")))
#else
#define GES_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GES_OK = 0,
    GES_ERR_INVALID_ARG = 1,   /* null pointer, bad size, bad enum, zero-norm quaternion */
    GES_ERR_CUDA = 2,          /* a CUDA runtime call failed (message says which) */
    GES_ERR_OOM = 3,           /* scratch allocation failed */
    GES_ERR_TIMEOUT = 4,       /* reserved: no call waits on device-side progress */
    GES_ERR_INTERNAL = 5,      /* a device-side consistency check failed (tile lists
                                  that kept overflowing after they were grown) */
    GES_ERR_UNSUPPORTED = 6,   /* no usable CUDA device of the required architecture, or
                                  a case a call does not take (batch views beyond its
                                  tile limit or of mixed Gaussian kinds, 2D Gaussians in
                                  ges_render_noalloc); the message says which */
    GES_ERR_CAPACITY = 7       /* fixed-capacity (graph) buffers were too small */
} ges_status;

typedef enum { GES_F32 = 0, GES_F16 = 1, GES_BF16 = 2 } ges_dtype;

typedef enum {
    GES_MODE_FULL = 0,            /* Eq. 5 */
    GES_MODE_SURFELS_ONLY = 1,    /* C = C_s (Table 5 ablation) */
    GES_MODE_GAUSSIANS_ONLY = 2   /* C = C_G / W_G, no surfels (Table 5 ablation); bg where W_G = 0 */
} ges_mode;

typedef enum {
    GES_FILTER_EWA = 0,    /* Sigma2 + lowpass I, opacity unchanged (3DGS's fixed dilation; basic GES) */
    GES_FILTER_MIP = 1     /* Mip-GES (Sec. 6.1): Sigma2 + lowpass I with the opacity scaled by
                              sqrt(|Sigma2| / |Sigma2 + lowpass I|) (Mip-Splatting's screen filter;
                              that method uses lowpass = 0.1) */
} ges_filter;

typedef enum {
    GES_EPS_ADAPTIVE = 0,  /* eps_i = eps_factor/3 * (s_1+s_2+s_3), Sec. 5 */
    GES_EPS_ZERO = 1,      /* eps = 0, Table 5 ablation */
    GES_EPS_CONST = 2      /* eps = eps_value (0.1 in Table 5) */
} ges_eps_mode;

typedef struct ges_scene ges_scene;   /* opaque */

/* Scene description: DEVICE pointers, SoA, C-contiguous.  N = n_surfels,
 * M = n_gaussians, K = (sh_degree+1)^2.  Positions are always float32;
 * rotations, scales and opacities use attr_dtype, SH coefficients sh_dtype.
 *   s_pos [N,3]  s_rot [N,4] (w,x,y,z)  s_scale [N,2]  s_sh [N,K,3]
 *   g_pos [M,3]  g_rot [M,4] (w,x,y,z)  g_scale [M,3]  g_opac [M]  g_sh [M,K,3]
 *   gauss_dim: 3 (or 0) for 3D Gaussians; 2 for the 2D Gaussians of 2D-GES
 *     (Sec. 6.4): g_scale is then [M,2], each Gaussian a planar splat in the
 *     plane of its rotation's first two axes, evaluated at the ray-splat hit
 *     with its planar depth and the object-space EWA filter of Eq. 17-18 (size
 *     lowpass: scales s_k S_k, opacity sigma/(S1 S2), S_k from the diagonal of
 *     I + lowpass J^-1 J^-T); eps_i = eps_factor/2 (s1 + s2).  The 3D filter
 *     and GES_FILTER_MIP do not apply to them; ges_render_noalloc returns
 *     GES_ERR_UNSUPPORTED for them.
 *   g_filter3d [M] float32 or NULL: Mip-GES 3D filter variance per Gaussian
 *     (Sec. 6.1, Mip-Splatting's world-space filter; see ges_compute_filter3d).
 *     Rendering uses Sigma3 + v I = R diag(s^2 + v) R^T and scales the opacity
 *     by prod_j |s_j| / sqrt(s_j^2 + v); eps_i keeps the stored s.  NULL: none.
 * The arrays must stay valid and unchanged while a render or backward call
 * that uses them is in flight; the scene holds views, not copies. */
typedef struct {
    int64_t n_surfels, n_gaussians;
    int32_t sh_degree;            /* 0..3 */
    int32_t attr_dtype;           /* ges_dtype */
    int32_t sh_dtype;             /* ges_dtype */
    const float *s_pos;
    const void *s_rot, *s_scale, *s_sh;
    const float *g_pos;
    const void *g_rot, *g_scale, *g_opac, *g_sh;
    const float *g_filter3d;
    int32_t gauss_dim;            /* 3 (0 reads as 3) or 2 */
} ges_scene_desc;

/* Pinhole camera; width, height in [1, 16384]; fx, fy > 0; znear > 0. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float world_to_cam[12];       /* row-major [R|t] */
    float znear;
    float bg[3];
} ges_camera;

/* Render options; pass NULL for the paper's defaults (ges_default_opts). */
typedef struct {
    int32_t eps_mode;             /* ges_eps_mode */
    float eps_value;              /* used by GES_EPS_CONST */
    float eps_factor;             /* 5 (Sec. 5) */
    float lowpass;                /* 0.3, added to the 2D covariance diagonal */
    float alpha_min;              /* 1/255 (Sec. 3, after Eq. 4) */
    float surfel_r2;              /* 2 ln 255 (Sec. 4.1) */
    int32_t mode;                 /* ges_mode */
    int32_t samples;              /* surfel samples per pixel: 1 (the pixel centre, default) or 4
                                     (4x multisampling of the surfel pass, Sec. 5: samples on the
                                     2x2 grid at +-0.25 px, colour = their mean, D_s = the nearest
                                     covered sample's depth; Gaussians stay at the centre) */
    int32_t filter;               /* ges_filter: GES_FILTER_EWA (default) or GES_FILTER_MIP */
} ges_render_opts;

/* Gradient outputs (DEVICE pointers, float32, overwritten, not accumulated).
 * Shapes follow the inputs: g_pos [M,3], g_rot [M,4], g_scale [M,3] ([M,2]
 * for 2D Gaussians), g_opac [M], g_sh [M,K,3], s_sh [N,K,3].  Any pointer may
 * be NULL to skip that group. */
typedef struct {
    float *g_pos, *g_rot, *g_scale, *g_opac, *g_sh, *s_sh;
} ges_grads;

/* Counters of the last completed render on a scene. */
typedef struct {
    int64_t visible_surfels, visible_gaussians;   /* passed culling */
    int64_t surfel_tile_pairs, gauss_tile_pairs;  /* tile-list entries */
    int32_t tiles_x, tiles_y;
} ges_stats;

/* Per-kernel device time accumulated while profiling is on
 * (CUDA events on the scene's stream). */
#define GES_PROFILE_SLOTS 8
typedef struct {
    int32_t n;                                  /* slots used */
    char names[GES_PROFILE_SLOTS][24];
    double ms[GES_PROFILE_SLOTS];               /* summed device milliseconds */
    int64_t launches[GES_PROFILE_SLOTS];
} ges_profile;

/* Fill *out with the paper's defaults: adaptive eps with factor 5, lowpass
 * 0.3, alpha_min 1/255, surfel_r2 2 ln 255, full mode.  GES_ERR_INVALID_ARG
 * if out is NULL. */
GES_API ges_status ges_default_opts(ges_render_opts *out);

/* Create a scene that views the caller's attribute arrays (Sec. 3 defines the
 * attributes).  Validates sizes, sh_degree, dtypes and pointers (NULL allowed
 * only for empty primitive sets); selects the current CUDA device and checks
 * that it is sm_103.  *out receives the handle, to be released with
 * ges_destroy_scene. */
GES_API ges_status ges_create_scene(const ges_scene_desc *desc, ges_scene **out);

/* Re-point the scene at new arrays or sizes (after an optimiser step or a
 * densification).  Same checks as ges_create_scene; scratch is kept and
 * grown when needed. */
GES_API ges_status ges_scene_update(ges_scene *scene, const ges_scene_desc *desc);

/* Mip-GES 3D filter variance per Gaussian (Sec. 6.1, Mip-Splatting's world
 * filter) from the training cameras cams[0..n_cams): out_var [M] (DEVICE,
 * float32) receives v_i = s3d / nu_i^2, where nu_i = max(fx, fy) / z is the
 * highest sampling rate among the cameras whose image rectangle [0,W] x [0,H]
 * holds the Gaussian's projected centre at z > znear.  A Gaussian no camera
 * sees gets the largest v of the others (0 if none is seen).  Mip-Splatting
 * uses s3d = 0.2.  Pass out_var as the scene's g_filter3d to render with it.
 * Returns after the scene's stream has finished.  GES_ERR_INVALID_ARG on a
 * NULL pointer, n_cams < 1, a negative or non-finite s3d or a bad camera. */
GES_API ges_status ges_compute_filter3d(ges_scene *scene, const ges_camera *cams, int32_t n_cams, float s3d,
                                        float *out_var);

/* Translucent-surfel render of the coarse stage (Sec. 4.1, Eq. 6-7): surfel i
 * has opacity alpha = min(1, w[i] G(a, b)), G = exp(-(a^2 + b^2)/2) at the
 * ray-plane hit (a, b in scale units), zero where min(alpha, G) < alpha_min;
 * surfels are alpha-blended front to back in the order of their centres'
 * camera depths (ties: lower index), the pixel's frontmost contributor (least
 * depth at the pixel) first when front_first != 0 (the w >= 30 regime), and
 * blending stops once the transmittance falls below 1e-4 after a blend;
 * C = sum c alpha T + T bg.  Gaussians are not rendered.  w: DEVICE float [N],
 * w >= 0 (0: never contributes).  Outputs (DEVICE): out_rgb [3,H,W]; out_T,
 * out_Tlast [H,W] (final transmittance, transmittance before the last blended
 * surfel), out_front, out_last [H,W] int32 (frontmost contributor or -1; list
 * position after the last blended surfel), all needed by the backward and
 * each may otherwise be NULL; out_cover [N] int32 or NULL: set to the number
 * of pixels where each surfel is the frontmost contributor (the covering
 * score of Sec. 4.1 for this view).  Needs samples = 1 and surfel_r2 >=
 * 2 ln(1/alpha_min) (GES_ERR_INVALID_ARG otherwise). */
GES_API ges_status ges_render_translucent(ges_scene *scene, const ges_camera *cam, const ges_render_opts *opts,
                                          const float *w, int32_t front_first, float *out_rgb, float *out_T,
                                          int32_t *out_front, int32_t *out_last, float *out_Tlast,
                                          int32_t *out_cover);

/* Gradient outputs of the translucent backward (DEVICE, float32, overwritten):
 * s_pos [N,3], s_rot [N,4], s_scale [N,2], s_w [N], s_sh [N,K,3]; any may be NULL. */
typedef struct {
    float *s_pos, *s_rot, *s_scale, *s_w, *s_sh;
} ges_tgrads;

/* Gradients of L = sum(dL_drgb * C) of ges_render_translucent with respect to
 * surfel position, rotation (through the normalisation), scales, w and SH;
 * out_T, out_front, out_last, out_Tlast are that call's outputs for the same
 * scene arrays, camera, options, w and front_first.  The cut-off, the order
 * and the early stop pass no gradient.  Deterministic: per-surfel sums are
 * accumulated in 64-bit fixed point scaled by the largest |dL_drgb|. */
GES_API ges_status ges_render_translucent_backward(ges_scene *scene, const ges_camera *cam,
                                                   const ges_render_opts *opts, const float *w, int32_t front_first,
                                                   const float *dL_drgb, const float *out_T, const int32_t *out_front,
                                                   const int32_t *out_last, const float *out_Tlast,
                                                   const ges_tgrads *grads);

/* Contribution score of each Gaussian (Sec. 4.2, Eq. 9), for pruning:
 * out_score [M] (DEVICE) = max over the pixels where the Gaussian contributes
 * (1/255 clamp and depth test passed) of c_max alpha / (W_s + W_G), c_max its
 * largest colour channel, W_s = 1; 0 where it contributes nowhere.  out_depth
 * and aux are D_s and W_G of a ges_render_ex call with the same scene arrays,
 * camera and options (samples = 1). */
GES_API ges_status ges_contribution_scores(ges_scene *scene, const ges_camera *cam, const ges_render_opts *opts,
                                           const float *out_depth, const float *aux, float *out_score);

/* Release the scene and its scratch (synchronises its stream first).
 * NULL is accepted and ignored. */
GES_API ges_status ges_destroy_scene(ges_scene *scene);

/* Launch all further work of this scene on `stream` (a cudaStream_t; NULL is
 * the legacy default stream). */
GES_API ges_status ges_set_stream(ges_scene *scene, void *stream);

/* Both passes of Sec. 3 and the composite of Eq. 5 for one camera.
 * out_rgb [3,H,W] and out_depth [H,W] (D_s, +inf where no surfel) are device
 * buffers.  Returns after the stream has completed the render (the call
 * checks the device status word).  Any image size: up to 32768 tiles of
 * 16x16 pixels the binning counts in shared memory, above that with global
 * counters (same results). */
GES_API ges_status ges_render(ges_scene *scene, const ges_camera *cam, float *out_rgb, float *out_depth);

/* As ges_render with options and two optional outputs: out_surfel_id
 * [samples,H,W] (z-buffer winner of each sample, -1 where none) and aux [H,W]
 * (W_G of Eq. 3).  The backward pass needs both.  opts may be NULL
 * (defaults); samples other than 1 or 4 is GES_ERR_INVALID_ARG. */
GES_API ges_status ges_render_ex(ges_scene *scene, const ges_camera *cam, const ges_render_opts *opts,
                         float *out_rgb, float *out_depth, int32_t *out_surfel_id, float *aux);

/* The render of ges_render_ex plus the geometry maps of Sec. 6.4 (Eq. 10-12),
 * camera space: out_normal_s [3,H,W] the surfel normal N_s (of the nearest
 * covered sample's surfel, facing the camera; 0 where no surfel covers),
 * out_depth_smooth [H,W] D_smooth = (W_s D_s + D_G)/(W_s + W_G) and
 * out_normal_smooth [3,H,W] N_smooth = (W_s N_s + N_G)/(W_s + W_G), with
 * D_G = sum alpha_i d_i and N_G = sum alpha_i n_i over the depth-tested
 * Gaussians, and W_s = 1 where a surfel covers the pixel, 0 elsewhere (where
 * both weights are 0: D_smooth = +inf, N_smooth = 0); out_dg [H,W] and out_ng
 * [3,H,W] are D_G and N_G.  d_i, n_i: centre depth and smallest-scale axis for
 * 3D Gaussians, planar depth and splat normal for 2D ones; normals face the
 * camera and are not renormalised.  Every output but out_rgb may be NULL. */
GES_API ges_status ges_render_geom(ges_scene *scene, const ges_camera *cam, const ges_render_opts *opts,
                                   float *out_rgb, float *out_depth, float *out_normal_s, float *out_depth_smooth,
                                   float *out_normal_smooth, float *out_dg, float *out_ng);

/* Gradients of L = sum(dL_drgb * C) for the joint stage (Sec. 4.2): Gaussian
 * position, rotation (through the normalisation), scale, opacity and SH, and
 * surfel SH.  For 2D Gaussians (Sec. 6.4) the chain runs through the
 * ray-splat hit and the object-space filter factors S1, S2 of Eq. 17-18.  out_rgb, out_depth, surfel_id and aux must be the outputs of a
 * ges_render_ex call with the same scene arrays, camera and options.  The
 * depth-test indicator and the 1/255 clamp are piecewise constant and pass no
 * gradient.  Results are deterministic (no floating-point atomics). */
GES_API ges_status ges_render_backward(ges_scene *scene, const ges_camera *cam, const ges_render_opts *opts,
                               const float *dL_drgb, const float *out_rgb, const float *out_depth,
                               const int32_t *surfel_id, const float *aux, const ges_grads *grads);

/* Render n_views cameras in one batch: view v uses scenes[scene_of_view[v]]
 * (host arrays) and writes out_rgb[v] [3,H_v,W_v] and out_depth[v] [H_v,W_v]
 * (host arrays of device pointers; out_depth entries may be NULL).  All
 * scenes must live on the same device; the batch runs on the stream of
 * scenes[scene_of_view[0]] and the call returns when it is done.  Per-view
 * semantics are exactly those of ges_render_ex.
 *
 * The views render as one batch graph (see ges_batch_create) kept on the
 * first view's scene: the first call with a given set of image sizes,
 * scenes (primitive counts, kinds, storage types) and options builds it,
 * which renders every view once on the per-view path; later calls with the
 * same set rewrite its view table (cameras, outputs, attribute pointers) and
 * replay it.  Its memory is held until that scene is destroyed or a call
 * with another set replaces it.  Views above 32768 tiles of 16x16, or scenes
 * of both Gaussian kinds in one call, take one launch sequence per view
 * instead. */
GES_API ges_status ges_render_batch(ges_scene *const *scenes, const ges_camera *cams, const int32_t *scene_of_view,
                            int32_t n_views, const ges_render_opts *opts,
                            float *const *out_rgb, float *const *out_depth);

/* Forward render (same result as ges_render_ex) that allocates no device
 * memory (and, when it succeeds, no host memory either), for callers that
 * cannot: applications that hand out device memory
 * from their own fixed budget or pool, and render threads that must never
 * block on cudaMalloc/cudaFree (cudaFree waits for the whole device).  The
 * paper has no counterpart; this is a deployment convenience.
 *
 * No scene handle: desc, cam, opts (NULL = defaults) are read directly; the
 * outputs are as in ges_render_ex (out_rgb required, the others may be
 * NULL); work is queued on `stream` and the call returns after that stream
 * has finished the render.  Intermediate data lives in one fixed device array
 * of 18 MiB that every GPU loading this library holds until the process
 * exits.  Limits: n_surfels <= 65536, n_gaussians <= 65536, at most 16384
 * tiles of 16x16 pixels (e.g. 2048x2048), at most 1048576 tile entries per
 * primitive kind; larger inputs get GES_ERR_CAPACITY and a message.  The
 * first call on a device looks up that array's device address, so make it
 * before any stream capture.  All calls share the one array and it keeps
 * the previous call's contents (the call clears what must start at zero):
 * calls whose GPU work overlaps in time, from any thread or stream, race and
 * corrupt each other's results; serialise them. */
GES_API ges_status ges_render_noalloc(const ges_scene_desc *desc, const ges_camera *cam,
                                      const ges_render_opts *opts, float *out_rgb, float *out_depth,
                                      int32_t *out_surfel_id, float *aux, void *stream);

/* Exact work counts of one view, for measurement: *surfel_fragments receives
 * the number of (pixel, surfel) pairs whose fragment lies inside the surfel's
 * opaque disc in front of the near plane -- the fragments any exact z-buffer
 * must test in pass 1 (Sec. 3) -- and *gauss_terms the number of
 * (pixel, Gaussian) pairs with alpha >= alpha_min, the terms of Eq. 2-3 before
 * the depth test.  Runs the preprocess and binning of a render, then counts
 * over the full tile lists without any culling.  Synchronises the stream. */
GES_API ges_status ges_count_fragments(ges_scene *scene, const ges_camera *cam, const ges_render_opts *opts,
                                       int64_t *surfel_fragments, int64_t *gauss_terms);

/* A batch: a fixed set of views (each a camera on one of several scenes,
 * uneven sizes allowed) rendered by one CUDA graph.  Every phase of the
 * render is launched once for all views: the preprocess (when a scene has
 * several views, first a colour pass that evaluates Eq. 1 for all of them
 * from one read of each SH row; then one set-up launch per primitive kind),
 * the scans, the fill and the raster.  The raster is persistent and hands
 * out (view, tile) work items, so small and large views balance across the
 * GPU.  Per-view semantics are exactly those of ges_render_ex.
 *
 * ges_batch_create renders every view once through the scene's own path to
 * size the tile lists (x1.5 headroom), allocates the batch's own scratch,
 * then autotunes the primitives per preprocess CTA, the persistent raster's
 * CTAs per SM and the binning tile (16x16, 32x8 or 8x32 pixels) by timing
 * each candidate graph, and keeps the fastest.
 * Pointers
 * (scenes' arrays, outputs) are baked into the graph and must stay valid
 * until ges_batch_destroy.  Images must have at most 32768 tiles of 16x16
 * (otherwise GES_ERR_UNSUPPORTED; ges_render_batch renders such views one by one).
 * out_depth may be NULL (no depth output) or have NULL entries. */
typedef struct ges_batch ges_batch;
typedef struct {
    int32_t n_views;
    int32_t prims_per_cta;         /* chosen preprocess range per CTA */
    int32_t raster_ctas_per_sm;    /* chosen persistent raster occupancy */
    int32_t candidates;            /* configurations timed by the autotuner */
    double tuned_ms;               /* best measured time of one launch */
    int64_t h2d_bytes;             /* host->device bytes of one launch (the view table) */
    int64_t d2h_bytes;             /* device->host bytes of one launch (status words) */
    int32_t tile_w, tile_h;        /* binning tile of the chosen configuration, pixels */
} ges_batch_info;

GES_API ges_status ges_batch_create(ges_scene *const *scenes, const ges_camera *cams, const int32_t *scene_of_view,
                                    int32_t n_views, const ges_render_opts *opts, float *const *out_rgb,
                                    float *const *out_depth, ges_batch **out);

/* Change the camera of one view for the following launches; the image size
 * must stay the one given at creation.  Call it when no launch of this batch
 * is in flight (after ges_batch_sync). */
GES_API ges_status ges_batch_set_camera(ges_batch *batch, int32_t view, const ges_camera *cam);

/* Also write the surfel id map out_surfel_id [samples,H,W] (z-buffer winner of
 * each sample, -1 where none) and aux [H,W] (W_G of Eq. 3) of one view in the
 * following launches, as ges_render_ex does; DEVICE pointers owned by the
 * caller, either may be NULL (not written).  Call it when no launch of this
 * batch is in flight. */
GES_API ges_status ges_batch_set_id_output(ges_batch *batch, int32_t view, int32_t *out_surfel_id, float *aux);

/* Enqueue one replay of the batch's graph on `stream` (cudaStream_t). */
GES_API ges_status ges_batch_launch(ges_batch *batch, void *stream);

/* Wait for the last launch and check every view's status word: tile lists
 * too small for a changed camera -> GES_ERR_CAPACITY (recreate the batch);
 * zero-norm quaternion -> GES_ERR_INVALID_ARG. */
GES_API ges_status ges_batch_sync(ges_batch *batch);

GES_API ges_status ges_batch_get_info(const ges_batch *batch, ges_batch_info *out);

/* Per-view completion times of the last synchronised launch: ms_out[v] (host,
 * n_views entries) = milliseconds from the start of the batch's first kernel
 * to the moment the raster finished view v's last tile (%globaltimer stamps
 * taken on the device), or -1 if unavailable.  Call after ges_batch_sync. */
GES_API ges_status ges_batch_get_view_times(const ges_batch *batch, double *ms_out);

/* Device time per phase (preprocess, scan, fill, raster) summed over the
 * launches waited for by ges_batch_sync (CUDA-event nodes inside the graph
 * time the most recent launch at each sync); reset != 0 clears the sums. */
GES_API ges_status ges_batch_get_profile(ges_batch *batch, ges_profile *out, int32_t reset);

/* Release the batch (waits for its last launch).  NULL is ignored. */
GES_API ges_status ges_batch_destroy(ges_batch *batch);

/* Counters of the last render on this scene. */
GES_API ges_status ges_get_stats(const ges_scene *scene, ges_stats *out);

/* Turn per-kernel CUDA-event timing on (1) or off (0) and reset it. */
GES_API ges_status ges_set_profiling(ges_scene *scene, int32_t enable);

/* Read the per-kernel timing accumulated since profiling was enabled
 * (synchronises the scene's stream). */
GES_API ges_status ges_get_profile(ges_scene *scene, ges_profile *out);

/* Thread-local message of the last failing call ("" if none). */
GES_API const char *ges_last_error_message(void);

/* ABI version of this header. */
GES_API int32_t ges_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GES_H */
