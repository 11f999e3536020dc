// Host side of the C ABI declared in include/ges.h.
//
// Owns the per-scene scratch (raster records, visible lists, tile counts and
// lists), validates every argument before anything is launched, converts the
// camera to the kernels' parameter block, and reads the device status word
// after each render (list overflow -> grow and re-render; zero-norm
// quaternion -> GES_ERR_INVALID_ARG).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ges_internal.cuh"

using namespace ges;

namespace {

thread_local std::string g_err;

ges_status fail(ges_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

ges_status cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) return fail(GES_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(GES_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define GES_CUDA(call)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
    } while (0)

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t want)
    {
        if (want <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) bytes = want;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

const char *kFwdNames[4] = {"preprocess", "scan", "fill", "raster"};
const char *kBwdNames[2] = {"gauss_bwd", "surfel_bwd"};

void batch_release(ges_batch *b);

}  // namespace

struct ges_scene {
    ges_scene_desc desc{};
    SceneView view{};
    int device = 0;
    cudaStream_t stream = nullptr;
    DevBuf s_rec, s_rgb, g_rec, s_vis, g_vis;
    DevBuf s_cnt, g_cnt, s_off, g_off, s_cur, g_cur;
    DevBuf s_list, g_list;
    DevBuf hist, base, vcount;     // local binning
    DevBuf status;                 // ST_WORDS per view slot
    DevBuf filt;                   // ges_compute_filter3d: cameras + one scratch word
    DevBuf g_aux;                  // Gaussian side data (2D Gaussians, geometry maps)
    DevBuf t_side, t_keys;         // translucent render: surfel frames, sort keys
    DevBuf t_acc;                  // backward passes: 64-bit fixed-point gradient sums + one word
    // ges_render_batch's batch graph (views of this and other scenes, with
    // this scene the first view's), kept while the calls keep the same key
    ges_batch *bcache = nullptr;
    std::vector<int64_t> bkey;
    unsigned *status_host = nullptr;
    int status_slots = 0;
    int64_t tiles_cap = 0;
    int64_t s_cap = 0, g_cap = 0;
    ges_stats stats{};
    // profiling
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    ges_profile profile{};
};

namespace {

bool dtype_ok(int d) { return d == GES_F32 || d == GES_F16 || d == GES_BF16; }

ges_status check_desc(const ges_scene_desc *d)
{
    if (!d) return fail(GES_ERR_INVALID_ARG, "scene description is NULL");
    if (d->n_surfels < 0 || d->n_gaussians < 0) return fail(GES_ERR_INVALID_ARG, "negative primitive count");
    if (d->n_surfels > (int64_t)1 << 30 || d->n_gaussians > (int64_t)1 << 30)
        return fail(GES_ERR_INVALID_ARG, "more than 2^30 primitives of one kind");
    if (d->sh_degree < 0 || d->sh_degree > 3) return fail(GES_ERR_INVALID_ARG, "sh_degree %d not in [0,3]", d->sh_degree);
    if (!dtype_ok(d->attr_dtype) || !dtype_ok(d->sh_dtype)) return fail(GES_ERR_INVALID_ARG, "unknown dtype");
    if (d->n_surfels > 0 && (!d->s_pos || !d->s_rot || !d->s_scale || !d->s_sh))
        return fail(GES_ERR_INVALID_ARG, "surfel attribute pointer is NULL");
    if (d->n_gaussians > 0 && (!d->g_pos || !d->g_rot || !d->g_scale || !d->g_opac || !d->g_sh))
        return fail(GES_ERR_INVALID_ARG, "Gaussian attribute pointer is NULL");
    if (d->gauss_dim != 0 && d->gauss_dim != 2 && d->gauss_dim != 3)
        return fail(GES_ERR_INVALID_ARG, "gauss_dim %d is not 2 or 3", d->gauss_dim);
    return GES_OK;
}

ges_status check_device(int *dev)
{
    GES_CUDA(cudaGetDevice(dev));
    cudaDeviceProp p;
    GES_CUDA(cudaGetDeviceProperties(&p, *dev));
    if (!(p.major == 10 && p.minor == 3))
        return fail(GES_ERR_UNSUPPORTED, "device %d is sm_%d%d; this library is built for sm_103a only", *dev,
                    p.major, p.minor);
    return GES_OK;
}

void set_view(ges_scene *s)
{
    const ges_scene_desc &d = s->desc;
    s->view = SceneView{d.n_surfels, d.n_gaussians, d.sh_degree, d.attr_dtype, d.sh_dtype,
                        d.s_pos, d.s_rot, d.s_scale, d.s_sh, d.g_pos, d.g_rot, d.g_scale, d.g_opac, d.g_sh,
                        d.g_filter3d, d.gauss_dim == 2 ? 2 : 3};
}

bool finite_all(const float *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Binning tiles of 2^tsx x 2^tsy pixels for the camera's image.
void set_tiles(CamParams &C, int tsx, int tsy)
{
    C.tsx = tsx;
    C.tsy = tsy;
    C.tiles_x = (C.W + (1 << tsx) - 1) >> tsx;
    C.tiles_y = (C.H + (1 << tsy) - 1) >> tsy;
}

ges_status make_cam(const ges_camera *c, CamParams &C)
{
    if (!c) return fail(GES_ERR_INVALID_ARG, "camera is NULL");
    if (c->width < 1 || c->height < 1 || c->width > 16384 || c->height > 16384)
        return fail(GES_ERR_INVALID_ARG, "image size %dx%d not in [1,16384]", c->width, c->height);
    if (!(c->fx > 0.f) || !(c->fy > 0.f) || !std::isfinite(c->fx) || !std::isfinite(c->fy))
        return fail(GES_ERR_INVALID_ARG, "focal lengths must be positive and finite");
    if (!std::isfinite(c->cx) || !std::isfinite(c->cy) || !finite_all(c->world_to_cam, 12) || !finite_all(c->bg, 3))
        return fail(GES_ERR_INVALID_ARG, "camera has a non-finite entry");
    if (!(c->znear > 0.f) || !std::isfinite(c->znear)) return fail(GES_ERR_INVALID_ARG, "znear must be positive");
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) C.R[3 * r + k] = c->world_to_cam[4 * r + k];
        C.t[r] = c->world_to_cam[4 * r + 3];
    }
    // camera centre o = -R^T t in double, then rounded
    for (int j = 0; j < 3; ++j) {
        double o = 0.0;
        for (int r = 0; r < 3; ++r) o -= (double)c->world_to_cam[4 * r + j] * (double)c->world_to_cam[4 * r + 3];
        C.ocam[j] = (float)o;
    }
    C.fx = c->fx; C.fy = c->fy; C.cx = c->cx; C.cy = c->cy;
    C.znear = c->znear;
    C.izn = 1.f / c->znear;
    for (int k = 0; k < 3; ++k) C.bg[k] = c->bg[k];
    C.W = c->width; C.H = c->height;
    set_tiles(C, kTileShift, kTileShift);
    return GES_OK;
}

ges_status make_opts(const ges_render_opts *o, OptParams &O)
{
    ges_render_opts d;
    ges_default_opts(&d);
    if (!o) o = &d;
    if (o->eps_mode < 0 || o->eps_mode > 2) return fail(GES_ERR_INVALID_ARG, "eps_mode %d unknown", o->eps_mode);
    if (o->mode < 0 || o->mode > 2) return fail(GES_ERR_INVALID_ARG, "mode %d unknown", o->mode);
    if (!(o->alpha_min > 0.f && o->alpha_min <= 1.f)) return fail(GES_ERR_INVALID_ARG, "alpha_min must be in (0,1]");
    if (!(o->surfel_r2 > 0.f) || !std::isfinite(o->surfel_r2)) return fail(GES_ERR_INVALID_ARG, "surfel_r2 must be > 0");
    if (!(o->lowpass >= 0.f) || !std::isfinite(o->lowpass)) return fail(GES_ERR_INVALID_ARG, "lowpass must be >= 0");
    if (!std::isfinite(o->eps_factor) || !std::isfinite(o->eps_value))
        return fail(GES_ERR_INVALID_ARG, "eps parameters must be finite");
    if (o->samples != 1 && o->samples != 4) return fail(GES_ERR_INVALID_ARG, "samples must be 1 or 4, not %d", o->samples);
    if (o->filter != GES_FILTER_EWA && o->filter != GES_FILTER_MIP)
        return fail(GES_ERR_INVALID_ARG, "filter %d unknown", o->filter);
    O.eps_mode = o->eps_mode;
    O.eps_value = o->eps_value;
    O.eps_factor = o->eps_factor;
    O.lowpass = o->lowpass;
    O.alpha_min = o->alpha_min;
    O.surfel_r2 = o->surfel_r2;
    O.surfel_r = std::sqrt(o->surfel_r2);
    O.mode = o->mode;
    O.samples = o->samples;
    O.geo = 0;
    O.filter = o->filter;
    return GES_OK;
}

ges_status ensure_scratch(ges_scene *s, int64_t T, int slots, cudaStream_t st)
{
    const int64_t N = std::max<int64_t>(s->desc.n_surfels, 1), M = std::max<int64_t>(s->desc.n_gaussians, 1);
    cudaError_t e;
    if ((e = s->s_rec.ensure(N * 64)) || (e = s->s_rgb.ensure(N * 16)) || (e = s->g_rec.ensure(M * 64)) ||
        (e = s->s_vis.ensure(N * 16)) || (e = s->g_vis.ensure(M * 16)))
        return cuda_fail(e, "scratch allocation (records)");
    if (T > s->tiles_cap) {
        const int64_t Tc = T;
        DevBuf *cnts[2] = {&s->s_cnt, &s->g_cnt};
        for (DevBuf *b : cnts) {
            if ((e = b->ensure((Tc + 1) * 4))) return cuda_fail(e, "scratch allocation (tile counts)");
            if ((e = cudaMemsetAsync(b->p, 0, (Tc + 1) * 4, st))) return cuda_fail(e, "cudaMemsetAsync");
        }
        if ((e = s->s_off.ensure((Tc + 1) * 4)) || (e = s->g_off.ensure((Tc + 1) * 4)) ||
            (e = s->s_cur.ensure((Tc + 1) * 4)) || (e = s->g_cur.ensure((Tc + 1) * 4)))
            return cuda_fail(e, "scratch allocation (tile offsets)");
        s->tiles_cap = Tc;
    }
    {
        // local binning: one histogram row and one base row per preprocess CTA
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
        const LocalBins B = plan_local_bins(s->desc.n_surfels, s->desc.n_gaussians, sms);
        const int64_t P = std::max(B.Ps + B.Pg, 1), Tl = std::min<int64_t>(T, kLocalMaxTiles);
        if ((e = s->hist.ensure((size_t)P * ((Tl + 1) / 2) * 4)) || (e = s->base.ensure((size_t)P * Tl * 4)) ||
            (e = s->vcount.ensure((size_t)P * 4)))
            return cuda_fail(e, "scratch allocation (bins)");
    }
    if (s->s_cap == 0) s->s_cap = std::max<int64_t>((int64_t)1 << 20, 4 * s->desc.n_surfels);
    if (s->g_cap == 0) s->g_cap = std::max<int64_t>((int64_t)1 << 20, 4 * s->desc.n_gaussians);
    if ((e = s->s_list.ensure(s->s_cap * 4)) || (e = s->g_list.ensure(s->g_cap * 4)))
        return cuda_fail(e, "scratch allocation (tile lists)");
    if (slots > s->status_slots) {
        if ((e = s->status.ensure((size_t)slots * ST_WORDS * 4))) return cuda_fail(e, "status allocation");
        if (s->status_host) cudaFreeHost(s->status_host);
        s->status_host = nullptr;
        if ((e = cudaMallocHost(&s->status_host, (size_t)slots * ST_WORDS * 4))) return cuda_fail(e, "cudaMallocHost");
        s->status_slots = slots;
    }
    return GES_OK;
}

ViewScratch scratch_of(ges_scene *s, int slot)
{
    ViewScratch X;
    X.s_rec = (float4 *)s->s_rec.p; X.s_rgb = (float4 *)s->s_rgb.p; X.g_rec = (float4 *)s->g_rec.p;
    X.s_vis = (int *)s->s_vis.p; X.g_vis = (int *)s->g_vis.p;
    X.s_cnt = (int *)s->s_cnt.p; X.g_cnt = (int *)s->g_cnt.p;
    X.s_off = (int *)s->s_off.p; X.g_off = (int *)s->g_off.p;
    X.s_cur = (int *)s->s_cur.p; X.g_cur = (int *)s->g_cur.p;
    X.s_list = (int *)s->s_list.p; X.g_list = (int *)s->g_list.p;
    X.s_cap = s->s_cap; X.g_cap = s->g_cap;
    X.status = (unsigned *)s->status.p + (size_t)slot * ST_WORDS;
    X.hist = (unsigned *)s->hist.p;
    X.base = (unsigned *)s->base.p;
    X.vcount = (unsigned *)s->vcount.p;
    X.g_aux = (float4 *)s->g_aux.p;
    return X;
}

ges_status ensure_events(ges_scene *s, int n)
{
    while ((int)s->ev.size() < n) {
        cudaEvent_t e;
        GES_CUDA(cudaEventCreate(&e));
        s->ev.push_back(e);
    }
    return GES_OK;
}

int prof_slot(ges_scene *s, const char *name)
{
    for (int i = 0; i < s->profile.n; ++i)
        if (std::strncmp(s->profile.names[i], name, 23) == 0) return i;
    if (s->profile.n >= GES_PROFILE_SLOTS) return -1;
    const int i = s->profile.n++;
    std::strncpy(s->profile.names[i], name, 23);
    s->profile.names[i][23] = 0;
    return i;
}

// Accumulate the event intervals of the last launch group (stream already synchronised).
void prof_collect(ges_scene *s, int first_ev, const char *const *names, int n)
{
    for (int k = 0; k < n; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s->ev[first_ev + k], s->ev[first_ev + k + 1]) != cudaSuccess) continue;
        const int i = prof_slot(s, names[k]);
        if (i < 0) continue;
        s->profile.ms[i] += ms;
        s->profile.launches[i] += 1;
    }
}

// Launch the forward of every view, synchronise once, check every status
// slot; on list overflow grow the lists and repeat.
ges_status render_views(ges_scene *const *scenes, const CamParams *cams, const int32_t *scene_of_view, int n,
                        const OptParams &O, float *const *rgb, float *const *depth, int32_t *const *ids,
                        float *const *auxs, const float *const *geo_maps = nullptr)
{
    ges_scene *s0 = scenes[scene_of_view[0]];
    cudaStream_t st = s0->stream;
    for (int attempt = 0; attempt < 4; ++attempt) {
        // scratch for every scene used; status slots live in the first scene
        for (int v = 0; v < n; ++v) {
            ges_scene *s = scenes[scene_of_view[v]];
            ges_status r = ensure_scratch(s, (int64_t)cams[v].tiles_x * cams[v].tiles_y, s == s0 ? n : 1, st);
            if (r != GES_OK) return r;
            // side data: 2D Gaussians always, 3D ones for the geometry maps
            if (s->view.gdim == 2 || O.geo) {
                cudaError_t e = s->g_aux.ensure((size_t)std::max<int64_t>(s->desc.n_gaussians, 1) * 32);
                if (e != cudaSuccess) return cuda_fail(e, "scratch allocation (Gaussian side data)");
            }
        }
        if (s0->status_slots < n) {
            ges_status r = ensure_scratch(s0, 1, n, st);
            if (r != GES_OK) return r;
        }
        GES_CUDA(cudaMemsetAsync(s0->status.p, 0, (size_t)n * ST_WORDS * 4, st));
        const bool prof = s0->prof;
        if (prof) {
            ges_status r = ensure_events(s0, 8 + 5 * n);
            if (r != GES_OK) return r;
        }
        for (int v = 0; v < n; ++v) {
            ges_scene *s = scenes[scene_of_view[v]];
            ViewScratch X = scratch_of(s, 0);
            X.status = (unsigned *)s0->status.p + (size_t)v * ST_WORDS;
            cudaError_t e = launch_forward(s->view, cams[v], O, X, rgb[v], depth ? depth[v] : nullptr,
                                           ids ? ids[v] : nullptr, auxs ? auxs[v] : nullptr, st,
                                           prof ? s0->ev.data() + 8 + 5 * v : nullptr, geo_maps);
            if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        }
        GES_CUDA(cudaMemcpyAsync(s0->status_host, s0->status.p, (size_t)n * ST_WORDS * 4, cudaMemcpyDeviceToHost, st));
        GES_CUDA(cudaStreamSynchronize(st));
        if (prof)
            for (int v = 0; v < n; ++v) prof_collect(s0, 8 + 5 * v, kFwdNames, 4);
        bool overflow = false;
        for (int v = 0; v < n; ++v) {
            const unsigned *w = s0->status_host + (size_t)v * ST_WORDS;
            ges_scene *s = scenes[scene_of_view[v]];
            if (w[ST_FLAGS] & FLAG_BADQ)
                return fail(GES_ERR_INVALID_ARG, "view %d: a rotation quaternion has zero norm or is not finite", v);
            if (w[ST_FLAGS] & FLAG_SOVF) {
                s->s_cap = std::max<int64_t>(s->s_cap * 2, (int64_t)(w[ST_SPAIRS] * 1.25) + 1024);
                overflow = true;
            }
            if (w[ST_FLAGS] & FLAG_GOVF) {
                s->g_cap = std::max<int64_t>(s->g_cap * 2, (int64_t)(w[ST_GPAIRS] * 1.25) + 1024);
                overflow = true;
            }
            s->stats.visible_surfels = w[ST_SVIS];
            s->stats.visible_gaussians = w[ST_GVIS];
            s->stats.surfel_tile_pairs = w[ST_SPAIRS];
            s->stats.gauss_tile_pairs = w[ST_GPAIRS];
            s->stats.tiles_x = cams[v].tiles_x;
            s->stats.tiles_y = cams[v].tiles_y;
        }
        if (!overflow) return GES_OK;
    }
    return fail(GES_ERR_INTERNAL, "tile lists kept overflowing after growing them");
}

ges_status render_batch_engine(ges_scene *const *scenes, const std::vector<CamParams> &C, const ges_camera *cams,
                               const int32_t *sov, int n, const OptParams &O, const ges_render_opts *opts,
                               float *const *out_rgb, float *const *out_depth);

}  // namespace

extern "C" {

ges_status ges_default_opts(ges_render_opts *out)
{
    if (!out) return fail(GES_ERR_INVALID_ARG, "opts is NULL");
    out->eps_mode = GES_EPS_ADAPTIVE;
    out->eps_value = 0.1f;
    out->eps_factor = 5.f;
    out->lowpass = 0.3f;
    out->alpha_min = 1.f / 255.f;
    out->surfel_r2 = (float)(2.0 * std::log(255.0));
    out->mode = GES_MODE_FULL;
    out->samples = 1;
    out->filter = GES_FILTER_EWA;
    return GES_OK;
}

ges_status ges_create_scene(const ges_scene_desc *desc, ges_scene **out)
{
    if (!out) return fail(GES_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    ges_status r = check_desc(desc);
    if (r != GES_OK) return r;
    int dev = 0;
    if ((r = check_device(&dev)) != GES_OK) return r;
    GES_CUDA(prepare_forward_kernels());
    ges_scene *s = new (std::nothrow) ges_scene();
    if (!s) return fail(GES_ERR_OOM, "host allocation failed");
    s->desc = *desc;
    s->device = dev;
    set_view(s);
    *out = s;
    return GES_OK;
}

ges_status ges_scene_update(ges_scene *s, const ges_scene_desc *desc)
{
    if (!s) return fail(GES_ERR_INVALID_ARG, "scene is NULL");
    ges_status r = check_desc(desc);
    if (r != GES_OK) return r;
    s->desc = *desc;
    set_view(s);
    return GES_OK;
}

ges_status ges_destroy_scene(ges_scene *s)
{
    if (!s) return GES_OK;
    cudaStreamSynchronize(s->stream);
    DevBuf *bufs[] = {&s->s_rec, &s->s_rgb, &s->g_rec, &s->s_vis, &s->g_vis, &s->s_cnt, &s->g_cnt, &s->s_off,
                      &s->g_off, &s->s_cur, &s->g_cur, &s->s_list, &s->g_list, &s->hist, &s->base,
                      &s->vcount, &s->status, &s->filt, &s->g_aux, &s->t_side, &s->t_keys, &s->t_acc};
    for (DevBuf *b : bufs) b->release();
    if (s->bcache) batch_release(s->bcache);
    if (s->status_host) cudaFreeHost(s->status_host);
    for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
    delete s;
    return GES_OK;
}

ges_status ges_set_stream(ges_scene *s, void *stream)
{
    if (!s) return fail(GES_ERR_INVALID_ARG, "scene is NULL");
    s->stream = (cudaStream_t)stream;
    return GES_OK;
}

ges_status ges_render_ex(ges_scene *s, const ges_camera *cam, const ges_render_opts *opts, float *out_rgb,
                         float *out_depth, int32_t *out_surfel_id, float *aux)
{
    if (!s) return fail(GES_ERR_INVALID_ARG, "scene is NULL");
    if (!out_rgb) return fail(GES_ERR_INVALID_ARG, "out_rgb is NULL");
    CamParams C;
    OptParams O;
    ges_status r = make_cam(cam, C);
    if (r != GES_OK) return r;
    if ((r = make_opts(opts, O)) != GES_OK) return r;
    const int32_t zero = 0;
    float *rgb[1] = {out_rgb};
    float *dep[1] = {out_depth};
    int32_t *ids[1] = {out_surfel_id};
    float *aux1[1] = {aux};
    return render_views(&s, &C, &zero, 1, O, rgb, dep, ids, aux1);
}

ges_status ges_render_geom(ges_scene *s, const ges_camera *cam, const ges_render_opts *opts, float *out_rgb,
                           float *out_depth, float *out_normal_s, float *out_depth_smooth, float *out_normal_smooth,
                           float *out_dg, float *out_ng)
{
    if (!s) return fail(GES_ERR_INVALID_ARG, "scene is NULL");
    if (!out_rgb) return fail(GES_ERR_INVALID_ARG, "out_rgb is NULL");
    CamParams C;
    OptParams O;
    ges_status r = make_cam(cam, C);
    if (r != GES_OK) return r;
    if ((r = make_opts(opts, O)) != GES_OK) return r;
    O.geo = 1;
    const int32_t zero = 0;
    float *rgb[1] = {out_rgb};
    float *dep[1] = {out_depth};
    const float *maps[5] = {out_normal_s, out_depth_smooth, out_normal_smooth, out_dg, out_ng};
    return render_views(&s, &C, &zero, 1, O, rgb, dep, nullptr, nullptr, maps);
}

ges_status ges_render(ges_scene *s, const ges_camera *cam, float *out_rgb, float *out_depth)
{
    return ges_render_ex(s, cam, nullptr, out_rgb, out_depth, nullptr, nullptr);
}

ges_status ges_render_backward(ges_scene *s, const ges_camera *cam, const ges_render_opts *opts,
                               const float *dL_drgb, const float *out_rgb, const float *out_depth,
                               const int32_t *surfel_id, const float *aux, const ges_grads *grads)
{
    if (!s) return fail(GES_ERR_INVALID_ARG, "scene is NULL");
    if (!grads) return fail(GES_ERR_INVALID_ARG, "grads is NULL");
    if (!dL_drgb || !out_rgb || !out_depth || !surfel_id || !aux)
        return fail(GES_ERR_INVALID_ARG, "backward needs dL_drgb, out_rgb, out_depth, surfel_id and aux");
    CamParams C;
    OptParams O;
    ges_status r = make_cam(cam, C);
    if (r != GES_OK) return r;
    if ((r = make_opts(opts, O)) != GES_OK) return r;
    const bool prof = s->prof;
    if (prof && (r = ensure_events(s, 8)) != GES_OK) return r;
    // scratch: surfel sums + one word | per-pixel terms | Gaussian records | Gaussian sums |
    // chain-rule words
    const int64_t N = std::max<int64_t>(s->desc.n_surfels, 1), M = std::max<int64_t>(s->desc.n_gaussians, 1);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t pix_off = up((size_t)N * 3 * 8 + 16);
    const size_t rec_off = pix_off + up((size_t)C.W * C.H * 16);
    const size_t sum_off = rec_off + up((size_t)M * kBwdRecBytes);
    const size_t chain_off = sum_off + up((size_t)M * kBwdSums * 4);
    GES_CUDA(s->t_acc.ensure(chain_off + (size_t)M * kBwdChainWords * 4));
    unsigned char *base = (unsigned char *)s->t_acc.p;
    long long *acc = (long long *)base;
    cudaError_t e = launch_backward(s->view, C, O, dL_drgb, out_rgb, out_depth, surfel_id, aux, *grads, acc,
                                    (unsigned *)(acc + (size_t)N * 3), (float4 *)(base + pix_off),
                                    (float4 *)(base + rec_off), (float *)(base + sum_off),
                                    (float *)(base + chain_off), s->stream, prof ? s->ev.data() : nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "backward launch");
    GES_CUDA(cudaStreamSynchronize(s->stream));
    if (prof) prof_collect(s, 0, kBwdNames, 2);
    return GES_OK;
}

ges_status ges_render_batch(ges_scene *const *scenes, const ges_camera *cams, const int32_t *scene_of_view,
                            int32_t n_views, const ges_render_opts *opts, float *const *out_rgb,
                            float *const *out_depth)
{
    if (!scenes || !cams || !scene_of_view || !out_rgb) return fail(GES_ERR_INVALID_ARG, "NULL batch argument");
    if (n_views <= 0) return fail(GES_ERR_INVALID_ARG, "n_views must be positive");
    OptParams O;
    ges_status r = make_opts(opts, O);
    if (r != GES_OK) return r;
    std::vector<CamParams> C(n_views);
    int max_scene = 0;
    for (int v = 0; v < n_views; ++v) {
        if (scene_of_view[v] < 0) return fail(GES_ERR_INVALID_ARG, "scene_of_view[%d] is negative", v);
        max_scene = std::max(max_scene, (int)scene_of_view[v]);
        if (!out_rgb[v]) return fail(GES_ERR_INVALID_ARG, "out_rgb[%d] is NULL", v);
        if ((r = make_cam(cams + v, C[v])) != GES_OK) return r;
    }
    for (int k = 0; k <= max_scene; ++k)
        if (!scenes[k]) return fail(GES_ERR_INVALID_ARG, "scenes[%d] is NULL", k);
    // the batch graph, unless a view is beyond its local binning or the
    // scenes mix Gaussian kinds: then one launch sequence per view
    bool engine = true;
    for (int v = 0; v < n_views; ++v) {
        if ((int64_t)C[v].tiles_x * C[v].tiles_y > kLocalMaxTiles) engine = false;
        if (scenes[scene_of_view[v]]->view.gdim != scenes[scene_of_view[0]]->view.gdim) engine = false;
    }
    if (engine)
        return render_batch_engine(scenes, C, cams, scene_of_view, n_views, O, opts, out_rgb, out_depth);
    return render_views(scenes, C.data(), scene_of_view, n_views, O, out_rgb, out_depth, nullptr, nullptr);
}

ges_status ges_count_fragments(ges_scene *s, const ges_camera *cam, const ges_render_opts *opts,
                               int64_t *surfel_fragments, int64_t *gauss_terms)
{
    if (!s || !surfel_fragments || !gauss_terms) return fail(GES_ERR_INVALID_ARG, "NULL argument");
    CamParams C;
    OptParams O;
    ges_status r = make_cam(cam, C);
    if (r != GES_OK) return r;
    if ((r = make_opts(opts, O)) != GES_OK) return r;
    for (int attempt = 0; attempt < 4; ++attempt) {
        if ((r = ensure_scratch(s, (int64_t)C.tiles_x * C.tiles_y, 1, s->stream)) != GES_OK) return r;
        if (s->view.gdim == 2) GES_CUDA(s->g_aux.ensure((size_t)std::max<int64_t>(s->desc.n_gaussians, 1) * 32));
        ViewScratch X = scratch_of(s, 0);
        GES_CUDA(cudaMemsetAsync(X.status, 0, ST_WORDS * 4, s->stream));
        cudaError_t e = launch_count(s->view, C, O, X, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        GES_CUDA(cudaMemcpyAsync(s->status_host, X.status, ST_WORDS * 4, cudaMemcpyDeviceToHost, s->stream));
        GES_CUDA(cudaStreamSynchronize(s->stream));
        const unsigned *w = s->status_host;
        if (w[ST_FLAGS] & FLAG_BADQ) return fail(GES_ERR_INVALID_ARG, "a rotation quaternion has zero norm or is not finite");
        bool overflow = false;
        if (w[ST_FLAGS] & FLAG_SOVF) { s->s_cap = std::max<int64_t>(s->s_cap * 2, (int64_t)(w[ST_SPAIRS] * 1.25) + 1024); overflow = true; }
        if (w[ST_FLAGS] & FLAG_GOVF) { s->g_cap = std::max<int64_t>(s->g_cap * 2, (int64_t)(w[ST_GPAIRS] * 1.25) + 1024); overflow = true; }
        if (overflow) continue;
        *surfel_fragments = w[ST_SFRAG];
        *gauss_terms = w[ST_GFRAG];
        return GES_OK;
    }
    return fail(GES_ERR_INTERNAL, "tile lists kept overflowing after growing them");
}

ges_status ges_compute_filter3d(ges_scene *s, const ges_camera *cams, int32_t n_cams, float s3d, float *out_var)
{
    if (!s || !cams || (!out_var && s->desc.n_gaussians > 0)) return fail(GES_ERR_INVALID_ARG, "NULL argument");
    if (n_cams < 1) return fail(GES_ERR_INVALID_ARG, "n_cams must be >= 1");
    if (!(s3d >= 0.f) || !std::isfinite(s3d)) return fail(GES_ERR_INVALID_ARG, "s3d must be finite and >= 0");
    std::vector<CamParams> C((size_t)n_cams);
    for (int k = 0; k < n_cams; ++k) {
        ges_status r = make_cam(cams + k, C[(size_t)k]);
        if (r != GES_OK) return r;
    }
    const size_t cam_bytes = sizeof(CamParams) * (size_t)n_cams, word_at = (cam_bytes + 15) & ~(size_t)15;
    GES_CUDA(s->filt.ensure(word_at + 16));
    unsigned char *base = (unsigned char *)s->filt.p;
    GES_CUDA(cudaMemcpyAsync(base, C.data(), cam_bytes, cudaMemcpyHostToDevice, s->stream));
    cudaError_t e = launch_filter3d(s->view, (const CamParams *)base, n_cams, s3d, out_var,
                                    (unsigned *)(base + word_at), s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    GES_CUDA(cudaStreamSynchronize(s->stream));
    return GES_OK;
}

namespace {
// scratch and checks shared by the translucent calls
ges_status translucent_setup(ges_scene *s, const ges_camera *cam, const ges_render_opts *opts, const float *w,
                             CamParams &C, OptParams &O, ViewScratch &X)
{
    if (!s) return fail(GES_ERR_INVALID_ARG, "scene is NULL");
    if (!w && s->desc.n_surfels > 0) return fail(GES_ERR_INVALID_ARG, "w is NULL");
    ges_status r = make_cam(cam, C);
    if (r != GES_OK) return r;
    if ((r = make_opts(opts, O)) != GES_OK) return r;
    // the records' disc must hold the whole support G >= alpha_min
    if (O.surfel_r2 < -2.f * logf(O.alpha_min) * (1.f - 1e-6f))
        return fail(GES_ERR_INVALID_ARG, "the translucent render needs surfel_r2 >= 2 ln(1/alpha_min)");
    if (O.samples != 1) return fail(GES_ERR_INVALID_ARG, "the translucent render samples pixel centres only");
    const int64_t N = std::max<int64_t>(s->desc.n_surfels, 1);
    if ((r = ensure_scratch(s, (int64_t)C.tiles_x * C.tiles_y, 1, s->stream)) != GES_OK) return r;
    cudaError_t e;
    if ((e = s->t_side.ensure((size_t)N * 64)) || (e = s->t_keys.ensure((size_t)s->s_cap * 8)))
        return cuda_fail(e, "scratch allocation (translucent)");
    X = scratch_of(s, 0);
    X.s_tside = (float4 *)s->t_side.p;
    return GES_OK;
}

// status check after a translucent launch; true when the lists overflowed (grown, retry)
ges_status translucent_status(ges_scene *s, bool &retry)
{
    retry = false;
    GES_CUDA(cudaMemcpyAsync(s->status_host, s->status.p, ST_WORDS * 4, cudaMemcpyDeviceToHost, s->stream));
    GES_CUDA(cudaStreamSynchronize(s->stream));
    const unsigned *w = s->status_host;
    if (w[ST_FLAGS] & FLAG_BADQ) return fail(GES_ERR_INVALID_ARG, "a rotation quaternion has zero norm or is not finite");
    if (w[ST_FLAGS] & FLAG_SOVF) {
        s->s_cap = std::max<int64_t>(s->s_cap * 2, (int64_t)(w[ST_SPAIRS] * 1.25) + 1024);
        retry = true;
    }
    return GES_OK;
}
}  // namespace

ges_status ges_render_translucent(ges_scene *s, const ges_camera *cam, const ges_render_opts *opts, const float *w,
                                  int32_t front_first, float *out_rgb, float *out_T, int32_t *out_front,
                                  int32_t *out_last, float *out_Tlast, int32_t *out_cover)
{
    if (!out_rgb) return fail(GES_ERR_INVALID_ARG, "out_rgb is NULL");
    for (int attempt = 0; attempt < 4; ++attempt) {
        CamParams C;
        OptParams O;
        ViewScratch X;
        ges_status r = translucent_setup(s, cam, opts, w, C, O, X);
        if (r != GES_OK) return r;
        GES_CUDA(cudaMemsetAsync(X.status, 0, ST_WORDS * 4, s->stream));
        if (out_cover && s->desc.n_surfels > 0)
            GES_CUDA(cudaMemsetAsync(out_cover, 0, sizeof(int32_t) * (size_t)s->desc.n_surfels, s->stream));
        cudaError_t e = launch_translucent(s->view, C, O, X, w, front_first != 0, (unsigned long long *)s->t_keys.p,
                                           out_rgb, out_T, out_front, out_last, out_Tlast, out_cover, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        bool retry;
        if ((r = translucent_status(s, retry)) != GES_OK) return r;
        if (!retry) return GES_OK;
    }
    return fail(GES_ERR_INTERNAL, "tile lists kept overflowing after growing them");
}

ges_status ges_render_translucent_backward(ges_scene *s, const ges_camera *cam, const ges_render_opts *opts,
                                           const float *w, int32_t front_first, const float *dL_drgb,
                                           const float *out_T, const int32_t *out_front, const int32_t *out_last,
                                           const float *out_Tlast, const ges_tgrads *grads)
{
    if (!grads) return fail(GES_ERR_INVALID_ARG, "grads is NULL");
    if (!dL_drgb || !out_T || !out_front || !out_last || !out_Tlast)
        return fail(GES_ERR_INVALID_ARG, "the backward needs dL_drgb and the forward's T, front, last and Tlast");
    for (int attempt = 0; attempt < 4; ++attempt) {
        CamParams C;
        OptParams O;
        ViewScratch X;
        ges_status r = translucent_setup(s, cam, opts, w, C, O, X);
        if (r != GES_OK) return r;
        const int64_t N = std::max<int64_t>(s->desc.n_surfels, 1);
        GES_CUDA(s->t_acc.ensure((size_t)N * 18 * 8 + 16));
        GES_CUDA(cudaMemsetAsync(X.status, 0, ST_WORDS * 4, s->stream));
        long long *acc = (long long *)s->t_acc.p;
        cudaError_t e = launch_translucent_backward(s->view, C, O, X, w, front_first != 0,
                                                    (unsigned long long *)s->t_keys.p, dL_drgb, out_T, out_front,
                                                    out_last, out_Tlast, acc, (unsigned *)(acc + (size_t)N * 18),
                                                    grads->s_pos, grads->s_rot, grads->s_scale, grads->s_w,
                                                    grads->s_sh, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        bool retry;
        if ((r = translucent_status(s, retry)) != GES_OK) return r;
        if (!retry) return GES_OK;
    }
    return fail(GES_ERR_INTERNAL, "tile lists kept overflowing after growing them");
}

ges_status ges_contribution_scores(ges_scene *s, const ges_camera *cam, const ges_render_opts *opts,
                                   const float *out_depth, const float *aux, float *out_score)
{
    if (!s) return fail(GES_ERR_INVALID_ARG, "scene is NULL");
    if (!out_depth || !aux || (!out_score && s->desc.n_gaussians > 0))
        return fail(GES_ERR_INVALID_ARG, "contribution scores need depth, aux and out_score");
    CamParams C;
    OptParams O;
    ges_status r = make_cam(cam, C);
    if (r != GES_OK) return r;
    if ((r = make_opts(opts, O)) != GES_OK) return r;
    cudaError_t e = launch_contribution(s->view, C, O, out_depth, aux, out_score, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    GES_CUDA(cudaStreamSynchronize(s->stream));
    return GES_OK;
}

ges_status ges_get_stats(const ges_scene *s, ges_stats *out)
{
    if (!s || !out) return fail(GES_ERR_INVALID_ARG, "NULL argument");
    *out = s->stats;
    return GES_OK;
}

ges_status ges_set_profiling(ges_scene *s, int32_t enable)
{
    if (!s) return fail(GES_ERR_INVALID_ARG, "scene is NULL");
    s->prof = enable != 0;
    std::memset(&s->profile, 0, sizeof s->profile);
    return GES_OK;
}

ges_status ges_get_profile(ges_scene *s, ges_profile *out)
{
    if (!s || !out) return fail(GES_ERR_INVALID_ARG, "NULL argument");
    GES_CUDA(cudaStreamSynchronize(s->stream));
    *out = s->profile;
    return GES_OK;
}

const char *ges_last_error_message(void) { return g_err.c_str(); }

int32_t ges_version(void) { return 1; }

}  // extern "C"

// ---------------------------------------------------------------------------
// ges_batch: every phase one launch over all views, captured in a CUDA graph

struct ges_batch {
    int n = 0;
    int device = 0;
    OptParams O{};
    std::vector<BatchView> views;          // host copy of the table (built per candidate)
    std::vector<int64_t> s_cap, g_cap;
    BatchView *h_table = nullptr;          // pinned: copied to the device by the graph
    BatchView *d_table = nullptr;
    unsigned *d_status = nullptr;          // n * ST_WORDS + work counter
    unsigned *h_status = nullptr;          // pinned
    void *arena = nullptr;                 // all per-view scratch
    cudaStream_t stream = nullptr;         // capture / tuning stream
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t phase[7] = {};             // event nodes in the graph (phase boundaries, colour pass)
    bool colour_pass = false;              // the kept graph has a colour pass (events 5-6 recorded)
    ges_batch_info info{};
    ges_profile profile{};
    int tsx = kTileShift, tsy = kTileShift;   // binning tile of the chosen configuration
    // the maps the graph reads: preprocess CTA -> (view, CTA of the view) of
    // both launches, the colour pass's work items and view groups
    unsigned char *d_map = nullptr;
    size_t map_bytes = 0;                  // capacity
    BatchPlan plan{};                      // of the kept graph
    OptParams opt{};
    bool ids = false;                      // the kept graph's raster writes id maps / W_G where asked
};

namespace {

void batch_release(ges_batch *b)
{
    if (b->done) cudaEventSynchronize(b->done);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->done) cudaEventDestroy(b->done);
    for (cudaEvent_t e : b->phase)
        if (e) cudaEventDestroy(e);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->arena) cudaFree(b->arena);
    if (b->d_map) cudaFree(b->d_map);
    if (b->d_table) cudaFree(b->d_table);
    if (b->d_status) cudaFree(b->d_status);
    if (b->h_table) cudaFreeHost(b->h_table);
    if (b->h_status) cudaFreeHost(b->h_status);
    delete b;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Lay every view's scratch out in the arena for a given primitives-per-CTA
// (returns the bytes needed; with base == nullptr only sizes are computed).
size_t batch_layout(ges_batch *b, const std::vector<SceneView> &S, const std::vector<CamParams> &C,
                    int64_t prims_per_cta, unsigned char *base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) { unsigned char *p = base ? base + off : nullptr; off = align256(off + bytes); return p; };
    int prep_base = 0, tile_base = 0, col_base = 0, sprep_base = 0, gprep_base = 0;
    for (int v = 0; v < b->n; ++v) {
        BatchView &bv = b->views[v];
        const int64_t N = std::max<int64_t>(S[v].N, 1), M = std::max<int64_t>(S[v].M, 1);
        const int T = C[v].tiles_x * C[v].tiles_y;
        const LocalBins B = plan_local_bins_per_cta(S[v].N, S[v].M, prims_per_cta);
        const int P = std::max(B.Ps + B.Pg, 1);
        bv.S = S[v];
        bv.C = C[v];
        bv.B = B;
        bv.T = T;
        bv.tile_base = tile_base;
        bv.prep_base = prep_base;
        bv.sprep_base = sprep_base;
        bv.gprep_base = gprep_base;
        bv.colscan_base = col_base;
        tile_base += T;
        prep_base += B.Ps + B.Pg;
        sprep_base += B.Ps;
        gprep_base += B.Pg;
        col_base += (T + 31) / 32;
        ViewScratch &X = bv.X;
        X.s_rec = (float4 *)take(N * 64);
        X.s_rgb = (float4 *)take(N * 16);
        X.g_rec = (float4 *)take(M * 64);
        X.s_vis = (int *)take(N * 16);   // 16-byte segment entries (local bins)
        X.g_vis = (int *)take(M * 16);
        X.s_cnt = (int *)take((T + 1) * 4);
        X.g_cnt = (int *)take((T + 1) * 4);
        X.s_off = (int *)take((T + 1) * 4);
        X.g_off = (int *)take((T + 1) * 4);
        X.s_cur = (int *)take((T + 1) * 4);
        X.g_cur = (int *)take((T + 1) * 4);
        X.s_cap = b->s_cap[v];
        X.g_cap = b->g_cap[v];
        X.s_list = (int *)take(b->s_cap[v] * 4);
        X.g_list = (int *)take(b->g_cap[v] * 4);
        X.hist = (unsigned *)take((size_t)P * ((T + 1) / 2) * 4);
        X.base = (unsigned *)take((size_t)P * T * 4);
        X.vcount = (unsigned *)take((size_t)P * 4);
        X.g_aux = S[v].gdim == 2 ? (float4 *)take(M * 32) : nullptr;
        X.g_col = (float4 *)take(M * 16);
        X.status = b->d_status + (size_t)v * ST_WORDS;
    }
    return off;
}

// The preprocess launches' CTA order: views of one scene (same arrays and
// counts) take each primitive range one after another, so only the first of
// them reads the range's attributes from HBM; surfel CTAs first, then the
// Gaussian ones (their own launch).  Uploads the map; P gets its pointers.
// Capture one replay of the batch (table upload, status reset, the kernels of
// launch_batch, status read-back) as an executable graph.
cudaError_t capture_exec(ges_batch *b, const BatchPlan &P, const OptParams &O, bool ids, cudaGraphExec_t *out)
{
    const size_t status_words = (size_t)b->n * ST_WORDS + 16;
    cudaGraph_t g = nullptr;
    *out = nullptr;
    (void)cudaGetLastError();   // an earlier call's error is not this capture's (launch_batch reports the last error)
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    // the capture is ended whatever fails inside it, so the stream stays usable;
    // the first error of the sequence is the one reported
    cudaError_t first = cudaMemcpyAsync(b->d_table, b->h_table, sizeof(BatchView) * b->n, cudaMemcpyHostToDevice,
                                        b->stream);
    if (first == cudaSuccess) first = cudaMemsetAsync(b->d_status, 0, status_words * 4, b->stream);
    if (first == cudaSuccess)
        first = launch_batch(b->d_table, P, O, b->d_status + (size_t)b->n * ST_WORDS, b->stream, b->phase, ids);
    if (first == cudaSuccess)
        first = cudaMemcpyAsync(b->h_status, b->d_status, status_words * 4, cudaMemcpyDeviceToHost, b->stream);
    e = cudaStreamEndCapture(b->stream, &g);
    if (first != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return first != cudaSuccess ? first : e;
    }
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

// Bytes of the maps (see ges_batch::d_map) for n_prep preprocess CTAs,
// n_items colour items and n views; the parts start 16-byte aligned.
size_t map_layout(size_t n_prep, size_t n_items, size_t n, size_t *off_items, size_t *off_gview)
{
    const size_t a = (n_prep * sizeof(int2) + 15) & ~(size_t)15;
    const size_t b = a + n_items * sizeof(int4);
    if (off_items) *off_items = a;
    if (off_gview) *off_gview = b;
    return b + n * sizeof(int);
}

// Grow the map buffer to at least bytes.  Only before a graph is kept: a
// captured graph holds the buffer's address.
cudaError_t reserve_map(ges_batch *b, size_t bytes)
{
    if (bytes <= b->map_bytes) return cudaSuccess;
    if (b->exec) return cudaErrorInvalidValue;
    if (b->d_map) cudaFree(b->d_map);
    b->d_map = nullptr;
    b->map_bytes = 0;
    cudaError_t e = cudaMalloc(&b->d_map, bytes);
    if (e == cudaSuccess) b->map_bytes = bytes;
    return e;
}

// Colour items of one primitive kind of a group: one per kColourThreads primitives.
size_t colour_items(int64_t n) { return (size_t)((n + kColourThreads - 1) / kColourThreads); }

// The preprocess CTA maps (views of one scene take the same range one after
// another) and the colour pass's work list (one item per kColourThreads
// primitives of a kind per view group), uploaded for the current layout.
cudaError_t upload_prep_map(ges_batch *b, BatchPlan &P)
{
    std::vector<std::vector<int>> groups;
    std::vector<int> done(b->n, 0);
    for (int v = 0; v < b->n; ++v) {
        if (done[v]) continue;
        std::vector<int> g{v};
        done[v] = 1;
        const SceneView &a = b->views[v].S;
        for (int w = v + 1; w < b->n; ++w) {
            const SceneView &c = b->views[w].S;
            if (!done[w] && c.s_pos == a.s_pos && c.g_pos == a.g_pos && c.s_sh == a.s_sh && c.g_sh == a.g_sh &&
                c.N == a.N && c.M == a.M && c.deg == a.deg && c.sh_dtype == a.sh_dtype &&
                b->views[w].B.Ps == b->views[v].B.Ps && b->views[w].B.Pg == b->views[v].B.Pg) {
                g.push_back(w);
                done[w] = 1;
            }
        }
        groups.push_back(g);
    }
    std::vector<int2> m;
    m.reserve((size_t)P.total_sprep + P.total_gprep);
    for (int kind = 0; kind < 2; ++kind)
        for (const std::vector<int> &g : groups) {
            const LocalBins &B = b->views[g[0]].B;
            const int n = kind == 0 ? B.Ps : B.Pg;
            for (int c = 0; c < n; ++c)
                for (int v : g) m.push_back(make_int2(v, kind == 0 ? c : B.Ps + c));
        }
    std::vector<int4> items;
    std::vector<int> gview;
    // a colour pass only pays when some scene has several views: otherwise
    // the set-up evaluates each colour where it reads the primitive anyway
    size_t maxg = 0;
    for (const std::vector<int> &g : groups) maxg = std::max(maxg, g.size());
    for (const std::vector<int> &g : groups) {
        if (maxg < 2) break;
        const int gofs = (int)gview.size();
        gview.insert(gview.end(), g.begin(), g.end());
        const SceneView &S0 = b->views[g[0]].S;
        for (int kind = 0; kind < 2; ++kind) {
            const int64_t n = kind == 0 ? S0.N : S0.M;
            for (int64_t f = 0; f < n; f += kColourThreads)
                items.push_back(make_int4(kind, gofs, (int)g.size(), (int)f));
        }
    }
    size_t oi = 0, og = 0;
    const size_t bytes = map_layout(m.size(), items.size(), gview.size(), &oi, &og);
    cudaError_t e = reserve_map(b, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return e;
    std::vector<unsigned char> h(bytes, 0);
    if (!m.empty()) std::memcpy(h.data(), m.data(), m.size() * sizeof(int2));
    if (!items.empty()) std::memcpy(h.data() + oi, items.data(), items.size() * sizeof(int4));
    if (!gview.empty()) std::memcpy(h.data() + og, gview.data(), gview.size() * sizeof(int));
    P.smap = reinterpret_cast<const int2 *>(b->d_map);
    P.gmap = P.smap + P.total_sprep;
    P.cmap = reinterpret_cast<const int4 *>(b->d_map + oi);
    P.gview = reinterpret_cast<const int *>(b->d_map + og);
    P.total_colour = (int)items.size();
    b->colour_pass = P.total_colour > 0;
    return cudaMemcpy(b->d_map, h.data(), bytes, cudaMemcpyHostToDevice);
}

}  // namespace

extern "C" {

// tune: time the candidate configurations and keep the fastest; otherwise
// take the one most workloads pick (8192 primitives per preprocess CTA, the
// most resident raster CTAs)
static ges_status batch_create(ges_scene *const *scenes, const ges_camera *cams, const int32_t *scene_of_view,
                               int32_t n_views, const ges_render_opts *opts, float *const *out_rgb,
                               float *const *out_depth, ges_batch **out, bool tune)
{
    if (!out) return fail(GES_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!scenes || !cams || !scene_of_view || !out_rgb) return fail(GES_ERR_INVALID_ARG, "NULL batch argument");
    if (n_views <= 0) return fail(GES_ERR_INVALID_ARG, "n_views must be positive");
    OptParams O;
    ges_status r = make_opts(opts, O);
    if (r != GES_OK) return r;
    std::vector<SceneView> S(n_views);
    std::vector<CamParams> C(n_views);
    for (int v = 0; v < n_views; ++v) {
        if (scene_of_view[v] < 0 || !scenes[scene_of_view[v]])
            return fail(GES_ERR_INVALID_ARG, "view %d has no scene", v);
        if (!out_rgb[v]) return fail(GES_ERR_INVALID_ARG, "out_rgb[%d] is NULL", v);
        if ((r = make_cam(cams + v, C[v])) != GES_OK) return r;
        if (C[v].tiles_x * C[v].tiles_y > kLocalMaxTiles)
            return fail(GES_ERR_UNSUPPORTED, "view %d: %dx%d has more than %d tiles", v, C[v].W, C[v].H,
                        kLocalMaxTiles);
        S[v] = scenes[scene_of_view[v]]->view;
        if (O.mode == GES_MODE_GAUSSIANS_ONLY) S[v].N = 0;
        if (O.mode == GES_MODE_SURFELS_ONLY) S[v].M = 0;
        if (S[v].gdim != S[0].gdim)
            return fail(GES_ERR_UNSUPPORTED, "a batch renders scenes of one Gaussian kind (view %d differs)", v);
    }
    ges_batch *b = new (std::nothrow) ges_batch();
    if (!b) return fail(GES_ERR_OOM, "host allocation failed");
    b->n = n_views;
    b->O = O;
    b->views.resize(n_views);
    b->s_cap.resize(n_views);
    b->g_cap.resize(n_views);
    cudaError_t e;
#define BATCH_CUDA(call)                                              \
    do {                                                              \
        if ((e = (call)) != cudaSuccess) {                            \
            batch_release(b);                                         \
            return cuda_fail(e, #call);                               \
        }                                                             \
    } while (0)
    BATCH_CUDA(cudaGetDevice(&b->device));
    // size the tile lists from one render of every view (scene's own path)
    for (int v = 0; v < n_views; ++v) {
        ges_scene *sc = scenes[scene_of_view[v]];
        r = ges_render_ex(sc, cams + v, opts, out_rgb[v], out_depth ? out_depth[v] : nullptr, nullptr, nullptr);
        if (r != GES_OK) {
            batch_release(b);
            return r;
        }
        // other tile shapes than the per-view path's 16x16 give other counts
        // (a candidate whose lists overflow is dropped)
        const double head = tune ? 2.0 : 1.5;
        b->s_cap[v] = (int64_t)(sc->stats.surfel_tile_pairs * head) + 65536;
        b->g_cap[v] = (int64_t)(sc->stats.gauss_tile_pairs * head) + 65536;
    }
    // tile shapes tried (log2 width, log2 height): all when tuning, unless
    // GES_BATCH_TILE names one ("16x16", "32x8" or "8x32"); 16x16 otherwise
    std::vector<std::pair<int, int>> shapes{{kTileShift, kTileShift}};
    if (tune) {
        shapes = {{4, 4}, {5, 3}, {3, 5}};
        if (const char *env = std::getenv("GES_BATCH_TILE")) {
            if (!std::strcmp(env, "16x16")) shapes = {{4, 4}};
            else if (!std::strcmp(env, "32x8")) shapes = {{5, 3}};
            else if (!std::strcmp(env, "8x32")) shapes = {{3, 5}};
        }
    }
    {
        std::vector<std::pair<int, int>> ok;
        for (const auto &sh : shapes) {
            bool fits = true;
            for (int v = 0; v < n_views; ++v) {
                CamParams c = C[v];
                set_tiles(c, sh.first, sh.second);
                fits = fits && (int64_t)c.tiles_x * c.tiles_y <= kLocalMaxTiles;
            }
            if (fits) ok.push_back(sh);
        }
        if (ok.empty()) {
            batch_release(b);
            return fail(GES_ERR_UNSUPPORTED, "no tile shape keeps every view within %d tiles", kLocalMaxTiles);
        }
        shapes = ok;
    }
    auto shaped = [&](const std::pair<int, int> &sh) {
        std::vector<CamParams> c = C;
        for (CamParams &x : c) set_tiles(x, sh.first, sh.second);
        return c;
    };
    BATCH_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    BATCH_CUDA(cudaEventCreate(&b->done));
    for (cudaEvent_t &ev : b->phase) BATCH_CUDA(cudaEventCreate(&ev));
    const size_t status_words = (size_t)n_views * ST_WORDS + 16;
    BATCH_CUDA(cudaMalloc(&b->d_status, status_words * 4));
    BATCH_CUDA(cudaMallocHost(&b->h_status, status_words * 4));
    BATCH_CUDA(cudaMalloc(&b->d_table, sizeof(BatchView) * n_views));
    BATCH_CUDA(cudaMallocHost(&b->h_table, sizeof(BatchView) * n_views));
    for (int v = 0; v < n_views; ++v) {
        b->views[v].rgb = out_rgb[v];
        b->views[v].depth = out_depth ? out_depth[v] : nullptr;
        b->views[v].id = nullptr;
        b->views[v].aux = nullptr;
    }
    // arena sized for the smallest primitives-per-CTA tried (most histogram rows)
    const int64_t kRall[] = {4096, 8192, 16384, 32768, 60000}, kRone[] = {8192};
    const int64_t *kR = tune ? kRall : kRone;
    const int nR = tune ? 5 : 1;
    size_t bytes = 0;
    for (const auto &sh : shapes) bytes = std::max(bytes, batch_layout(b, S, shaped(sh), kR[0], nullptr));
    BATCH_CUDA(cudaMalloc(&b->arena, bytes));
    {
        // the maps of the candidate with the most preprocess CTAs (a kept
        // graph holds the buffer's address, so it never moves afterwards)
        size_t n_prep = 0, n_items = 0;
        for (int v = 0; v < n_views; ++v) {
            n_prep += (size_t)((S[v].N + kR[0] - 1) / kR[0] + (S[v].M + kR[0] - 1) / kR[0]);
            n_items += colour_items(S[v].N) + colour_items(S[v].M);
        }
        BATCH_CUDA(reserve_map(b, map_layout(n_prep, n_items, (size_t)n_views, nullptr, nullptr) + 16));
    }
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);

    // autotune: capture a graph per candidate, time it, keep the fastest
    float best_ms = 1e30f;
    int cand = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BATCH_CUDA(cudaEventCreate(&e0));
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        batch_release(b);
        return cuda_fail(e, "cudaEventCreate");
    }
    auto drop_events = [&]() { cudaEventDestroy(e0); cudaEventDestroy(e1); };
    // raster candidates: resident CTAs per SM (the 4-sample kernels are built
    // for one CTA fewer)
    const int d = O.samples == 4 ? 1 : 0;
    const int kPerSm[] = {5 - d, 4 - d};
    for (const auto &sh : shapes)
    for (int ri = 0; ri < nR; ++ri) {
        const std::vector<CamParams> Cs = shaped(sh);
        const int64_t R = kR[ri];
        for (int pi = 0; pi < (tune ? 2 : 1); ++pi) {
            const int per_sm = kPerSm[pi];
            batch_layout(b, S, Cs, R, (unsigned char *)b->arena);
            BatchPlan P{};
            P.n = n_views;
            P.raster_ctas = sms * per_sm;
            P.gdim = S[0].gdim;
            for (int v = 0; v < n_views; ++v) {
                P.total_tiles += b->views[v].T;
                P.total_prep += b->views[v].B.Ps + b->views[v].B.Pg;
                P.total_sprep += b->views[v].B.Ps;
                P.total_gprep += b->views[v].B.Pg;
                P.total_colscan += (b->views[v].T + 31) / 32;
                P.max_T = std::max(P.max_T, b->views[v].T);
            }
            std::memcpy(b->h_table, b->views.data(), sizeof(BatchView) * n_views);
            if ((e = upload_prep_map(b, P)) != cudaSuccess) {
                drop_events();
                batch_release(b);
                return cuda_fail(e, "upload_prep_map");
            }
            cudaGraphExec_t ex = nullptr;
            e = capture_exec(b, P, O, false, &ex);
            if (e != cudaSuccess) {
                drop_events();
                batch_release(b);
                return cuda_fail(e, "batch graph capture");
            }
            // one untimed replay, then three timed ones
            e = cudaGraphLaunch(ex, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaGraphLaunch(ex, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            const cudaError_t es = cudaStreamSynchronize(b->stream);
            if (e == cudaSuccess) e = es;
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                cudaGraphExecDestroy(ex);
                drop_events();
                batch_release(b);
                return cuda_fail(e, "batch launch");
            }
            ++cand;
            ms /= 3.f;
            // a candidate whose tile lists overflowed skipped its raster: not a timing
            bool overflow = false;
            for (int v = 0; v < n_views; ++v)
                overflow = overflow || (b->h_status[(size_t)v * ST_WORDS + ST_FLAGS] & (FLAG_SOVF | FLAG_GOVF));
            if (!overflow && ms < best_ms) {
                best_ms = ms;
                if (b->exec) cudaGraphExecDestroy(b->exec);
                b->exec = ex;
                b->info.prims_per_cta = (int32_t)R;
                b->info.raster_ctas_per_sm = per_sm;
                b->tsx = sh.first;
                b->tsy = sh.second;
                b->info.tile_w = 1 << sh.first;
                b->info.tile_h = 1 << sh.second;
                b->plan = P;
            } else {
                cudaGraphExecDestroy(ex);
            }
        }
    }
    drop_events();
    if (!b->exec) {
        batch_release(b);
        return fail(GES_ERR_CAPACITY, "every configuration overflowed the batch's tile lists");
    }
    // the table and the CTA map the chosen graph reads: rebuild them for that candidate
    batch_layout(b, S, shaped({b->tsx, b->tsy}), b->info.prims_per_cta, (unsigned char *)b->arena);
    std::memcpy(b->h_table, b->views.data(), sizeof(BatchView) * n_views);
    {
        BatchPlan P{};
        for (int v = 0; v < n_views; ++v) {
            P.total_sprep += b->views[v].B.Ps;
            P.total_gprep += b->views[v].B.Pg;
        }
        BATCH_CUDA(upload_prep_map(b, P));
    }
    b->opt = O;
    b->info.n_views = n_views;
    b->info.candidates = cand;
    b->info.tuned_ms = best_ms;
    b->info.h2d_bytes = (int64_t)(sizeof(BatchView) * n_views);
    b->info.d2h_bytes = (int64_t)(status_words * 4);
    // one checked launch with the chosen configuration
    BATCH_CUDA(cudaGraphLaunch(b->exec, b->stream));
    BATCH_CUDA(cudaEventRecord(b->done, b->stream));
#undef BATCH_CUDA
    *out = b;
    r = ges_batch_sync(b);
    std::memset(&b->profile, 0, sizeof b->profile);
    if (r != GES_OK) {
        batch_release(b);
        *out = nullptr;
    }
    return r;
}

ges_status ges_batch_create(ges_scene *const *scenes, const ges_camera *cams, const int32_t *scene_of_view,
                            int32_t n_views, const ges_render_opts *opts, float *const *out_rgb,
                            float *const *out_depth, ges_batch **out)
{
    return batch_create(scenes, cams, scene_of_view, n_views, opts, out_rgb, out_depth, out, true);
}

ges_status ges_batch_set_camera(ges_batch *b, int32_t view, const ges_camera *cam)
{
    if (!b) return fail(GES_ERR_INVALID_ARG, "batch is NULL");
    if (view < 0 || view >= b->n) return fail(GES_ERR_INVALID_ARG, "view %d out of range", view);
    CamParams C;
    ges_status r = make_cam(cam, C);
    if (r != GES_OK) return r;
    set_tiles(C, b->tsx, b->tsy);
    if (C.W != b->views[view].C.W || C.H != b->views[view].C.H)
        return fail(GES_ERR_INVALID_ARG, "view %d: image size must stay %dx%d", view, b->views[view].C.W,
                    b->views[view].C.H);
    b->views[view].C = C;
    b->h_table[view].C = C;
    return GES_OK;
}

ges_status ges_batch_set_id_output(ges_batch *b, int32_t view, int32_t *out_surfel_id, float *aux)
{
    if (!b) return fail(GES_ERR_INVALID_ARG, "batch is NULL");
    if (view < 0 || view >= b->n) return fail(GES_ERR_INVALID_ARG, "view %d out of range", view);
    b->views[view].id = out_surfel_id;
    b->views[view].aux = aux;
    b->h_table[view].id = out_surfel_id;
    b->h_table[view].aux = aux;
    // the raster that writes them is a kernel of its own (the timed one keeps
    // its registers): re-capture the graph when the need for it changes
    bool want = false;
    for (int v = 0; v < b->n; ++v) want = want || b->views[v].id || b->views[v].aux;
    if (want != b->ids) {
        if (b->done) GES_CUDA(cudaEventSynchronize(b->done));
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = capture_exec(b, b->plan, b->opt, want, &ex);
        if (e != cudaSuccess) return cuda_fail(e, "graph capture");
        cudaGraphExecDestroy(b->exec);
        b->exec = ex;
        b->ids = want;
    }
    return GES_OK;
}

ges_status ges_batch_launch(ges_batch *b, void *stream)
{
    if (!b) return fail(GES_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    GES_CUDA(cudaGraphLaunch(b->exec, st));
    GES_CUDA(cudaEventRecord(b->done, st));
    return GES_OK;
}

ges_status ges_batch_sync(ges_batch *b)
{
    if (!b) return fail(GES_ERR_INVALID_ARG, "batch is NULL");
    GES_CUDA(cudaEventSynchronize(b->done));
    // per-phase device time of the last launch (graph event nodes)
    // the colour pass runs inside the preprocess phase; its own time is reported beside it
    static const char *names[5] = {"preprocess", "scan", "fill", "raster", "colour_in_preprocess"};
    for (int k = 0; k < (b->colour_pass ? 5 : 4); ++k) {
        float ms = 0.f;
        cudaEvent_t a = k < 4 ? b->phase[k] : b->phase[5], z = k < 4 ? b->phase[k + 1] : b->phase[6];
        if (cudaEventElapsedTime(&ms, a, z) != cudaSuccess) {
            cudaGetLastError();   // a failed query must not surface at the next launch
            continue;
        }
        int i = -1;
        for (int j = 0; j < b->profile.n; ++j)
            if (std::strncmp(b->profile.names[j], names[k], 23) == 0) i = j;
        if (i < 0 && b->profile.n < GES_PROFILE_SLOTS) {
            i = b->profile.n++;
            std::strncpy(b->profile.names[i], names[k], 23);
        }
        if (i >= 0) { b->profile.ms[i] += ms; b->profile.launches[i] += 1; }
    }
    for (int v = 0; v < b->n; ++v) {
        const unsigned *w = b->h_status + (size_t)v * ST_WORDS;
        if (w[ST_FLAGS] & FLAG_BADQ)
            return fail(GES_ERR_INVALID_ARG, "view %d: a rotation quaternion has zero norm or is not finite", v);
        if (w[ST_FLAGS] & (FLAG_SOVF | FLAG_GOVF))
            return fail(GES_ERR_CAPACITY, "view %d: %u surfel / %u Gaussian tile entries exceed the batch's "
                        "lists (%lld / %lld); recreate the batch", v, w[ST_SPAIRS], w[ST_GPAIRS],
                        (long long)b->s_cap[v], (long long)b->g_cap[v]);
    }
    return GES_OK;
}

ges_status ges_batch_get_info(const ges_batch *b, ges_batch_info *out)
{
    if (!b || !out) return fail(GES_ERR_INVALID_ARG, "NULL argument");
    *out = b->info;
    return GES_OK;
}

ges_status ges_batch_get_view_times(const ges_batch *b, double *ms_out)
{
    if (!b || !ms_out) return fail(GES_ERR_INVALID_ARG, "NULL argument");
    uint64_t t0 = 0;
    std::memcpy(&t0, b->h_status + (size_t)b->n * ST_WORDS + 2, sizeof t0);
    for (int v = 0; v < b->n; ++v) {
        uint64_t t = 0;
        std::memcpy(&t, b->h_status + (size_t)v * ST_WORDS + ST_TDONE, sizeof t);
        ms_out[v] = (t0 != 0 && t >= t0) ? (double)(t - t0) * 1e-6 : -1.0;
    }
    return GES_OK;
}

ges_status ges_batch_get_profile(ges_batch *b, ges_profile *out, int32_t reset)
{
    if (!b || !out) return fail(GES_ERR_INVALID_ARG, "NULL argument");
    *out = b->profile;
    if (reset) std::memset(&b->profile, 0, sizeof b->profile);
    return GES_OK;
}

ges_status ges_batch_destroy(ges_batch *b)
{
    if (b) batch_release(b);
    return GES_OK;
}

}  // extern "C"

namespace {

// ges_render_batch through a batch graph kept on the first view's scene.  The
// key is what the graph bakes in: the views' image sizes, the scenes'
// primitive counts, kinds and storage types, and the options.  With the same
// key the call only rewrites the view table (cameras, outputs, attribute
// pointers) and replays the graph; otherwise (or when the tile lists of the
// kept graph overflow for new cameras) it builds a new one, without tuning.
ges_status render_batch_engine(ges_scene *const *scenes, const std::vector<CamParams> &C, const ges_camera *cams,
                               const int32_t *sov, int n, const OptParams &O, const ges_render_opts *opts,
                               float *const *out_rgb, float *const *out_depth)
{
    ges_scene *own = scenes[sov[0]];
    std::vector<int64_t> key{n};
    {
        int32_t w[sizeof(OptParams) / 4];
        std::memcpy(w, &O, sizeof w);
        key.insert(key.end(), w, w + sizeof(OptParams) / 4);
    }
    for (int v = 0; v < n; ++v) {
        const SceneView &S = scenes[sov[v]]->view;
        // the first view whose scene arrays are the same: the graph's colour
        // pass evaluates such views together
        int grp = v;
        for (int w = 0; w < v; ++w) {
            const SceneView &T = scenes[sov[w]]->view;
            if (T.s_pos == S.s_pos && T.g_pos == S.g_pos && T.s_sh == S.s_sh && T.g_sh == S.g_sh) { grp = w; break; }
        }
        key.insert(key.end(), {(int64_t)sov[v], (int64_t)grp, S.N, S.M, S.gdim, S.deg, S.attr_dtype, S.sh_dtype,
                               (int64_t)(S.g_filt3 != nullptr), C[v].W, C[v].H,
                               (int64_t)(out_depth && out_depth[v])});
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (own->bcache && own->bkey == key) {
            ges_batch *b = own->bcache;
            for (int v = 0; v < n; ++v) {
                SceneView S = scenes[sov[v]]->view;
                if (O.mode == GES_MODE_GAUSSIANS_ONLY) S.N = 0;
                if (O.mode == GES_MODE_SURFELS_ONLY) S.M = 0;
                b->views[v].S = S;
                b->views[v].C = C[v];
                set_tiles(b->views[v].C, b->tsx, b->tsy);
                b->views[v].rgb = out_rgb[v];
                b->views[v].depth = out_depth ? out_depth[v] : nullptr;
            }
            std::memcpy(b->h_table, b->views.data(), sizeof(BatchView) * n);
            ges_status r = ges_batch_launch(b, own->stream);
            if (r == GES_OK) r = ges_batch_sync(b);
            if (r != GES_ERR_CAPACITY) {
                if (r == GES_OK)
                    for (int v = 0; v < n; ++v) {
                        const unsigned *w = b->h_status + (size_t)v * ST_WORDS;
                        ges_stats &st = scenes[sov[v]]->stats;
                        st.visible_surfels = w[ST_SVIS];
                        st.visible_gaussians = w[ST_GVIS];
                        st.surfel_tile_pairs = w[ST_SPAIRS];
                        st.gauss_tile_pairs = w[ST_GPAIRS];
                        st.tiles_x = C[v].tiles_x;
                        st.tiles_y = C[v].tiles_y;
                    }
                return r;
            }
        }
        if (own->bcache) batch_release(own->bcache);
        own->bcache = nullptr;
        own->bkey.clear();
        // a new graph; its creation renders every view once and checks it
        ges_batch *b = nullptr;
        ges_status r = batch_create(scenes, cams, sov, n, opts, out_rgb, out_depth, &b, false);
        if (r != GES_OK) return r;
        own->bcache = b;
        own->bkey = key;
        return GES_OK;
    }
    return fail(GES_ERR_INTERNAL, "batch render kept overflowing its tile lists");
}

}  // namespace

// ---------------------------------------------------------------------------
// ges_render_noalloc: the forward render with every intermediate buffer in one
// fixed device array, for callers that cannot allocate device memory.

#include <mutex>

namespace {

constexpr int64_t kNaMaxSurfels = 65536, kNaMaxGaussians = 65536, kNaMaxTiles = 16384;
constexpr int64_t kNaMaxPairs = 1048576;

constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
// byte offsets of the regions inside the array
constexpr size_t kNaSRec = 0;
constexpr size_t kNaSRgb = na_align(kNaSRec + kNaMaxSurfels * 64);
constexpr size_t kNaGRec = na_align(kNaSRgb + kNaMaxSurfels * 16);
constexpr size_t kNaSVis = na_align(kNaGRec + kNaMaxGaussians * 64);
constexpr size_t kNaGVis = na_align(kNaSVis + kNaMaxSurfels * 4);
constexpr size_t kNaTileBytes = na_align((kNaMaxTiles + 1) * 4);
constexpr size_t kNaSCnt = na_align(kNaGVis + kNaMaxGaussians * 4);   // s_cnt, g_cnt adjacent (cleared together)
constexpr size_t kNaGCnt = kNaSCnt + kNaTileBytes;
constexpr size_t kNaSOff = kNaGCnt + kNaTileBytes;
constexpr size_t kNaGOff = kNaSOff + kNaTileBytes;
constexpr size_t kNaSCur = kNaGOff + kNaTileBytes;
constexpr size_t kNaGCur = kNaSCur + kNaTileBytes;
constexpr size_t kNaStatus = kNaGCur + kNaTileBytes;
constexpr size_t kNaSList = na_align(kNaStatus + ST_WORDS * 4);
constexpr size_t kNaGList = na_align(kNaSList + kNaMaxPairs * 4);
constexpr size_t kNaBytes = na_align(kNaGList + kNaMaxPairs * 4);
static_assert(kNaBytes <= (size_t)18 << 20, "fixed scratch exceeds its stated 18 MiB");

constexpr int kNaMaxDevices = 64;
std::once_flag g_na_once[kNaMaxDevices];
unsigned char *g_na_ptr[kNaMaxDevices];
cudaError_t g_na_err[kNaMaxDevices];
ges_status g_na_arch[kNaMaxDevices];

}  // namespace

// The fixed scratch.  In host code this name is only a stand-in for the
// device symbol: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

extern "C" GES_API ges_status ges_render_noalloc(const ges_scene_desc *desc, const ges_camera *cam,
                                                 const ges_render_opts *opts, float *out_rgb, float *out_depth,
                                                 int32_t *out_surfel_id, float *aux, void *stream)
{
    ges_status r = check_desc(desc);
    if (r != GES_OK) return r;
    if (!out_rgb) return fail(GES_ERR_INVALID_ARG, "out_rgb is NULL");
    CamParams C;
    OptParams O;
    if ((r = make_cam(cam, C)) != GES_OK) return r;
    if ((r = make_opts(opts, O)) != GES_OK) return r;
    if (desc->gauss_dim == 2)
        return fail(GES_ERR_UNSUPPORTED, "ges_render_noalloc renders 3D Gaussians only (its fixed array has no room "
                                         "for the side data of 2D Gaussians)");
    if (desc->n_surfels > kNaMaxSurfels || desc->n_gaussians > kNaMaxGaussians)
        return fail(GES_ERR_CAPACITY, "ges_render_noalloc: at most %lld surfels and %lld Gaussians (got %lld, %lld)",
                    (long long)kNaMaxSurfels, (long long)kNaMaxGaussians, (long long)desc->n_surfels,
                    (long long)desc->n_gaussians);
    const int64_t T = (int64_t)C.tiles_x * C.tiles_y;
    if (T > kNaMaxTiles)
        return fail(GES_ERR_CAPACITY, "ges_render_noalloc: image %dx%d needs %lld tiles, at most %lld", C.W, C.H,
                    (long long)T, (long long)kNaMaxTiles);
    int dev = 0;
    GES_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) return fail(GES_ERR_UNSUPPORTED, "device ordinal %d too large", dev);
    // once per device, with that device current: check the architecture and
    // look up the array's device address
    std::call_once(g_na_once[dev], [dev]() {
        int d = dev;
        g_na_arch[dev] = check_device(&d);
        void *p = nullptr;
        g_na_err[dev] = g_na_arch[dev] == GES_OK ? cudaGetSymbolAddress(&p, g_noalloc_scratch) : cudaSuccess;
        g_na_ptr[dev] = (unsigned char *)p;
    });
    if (g_na_arch[dev] != GES_OK)
        return fail(g_na_arch[dev], "device %d is not an sm_103 GPU (this library is built for sm_103a only)", dev);
    if (g_na_err[dev] != cudaSuccess) return cuda_fail(g_na_err[dev], "cudaGetSymbolAddress(fixed scratch)");
    unsigned char *base = g_na_ptr[dev];
    cudaStream_t st = (cudaStream_t)stream;

    ViewScratch X;
    X.s_rec = (float4 *)(base + kNaSRec); X.s_rgb = (float4 *)(base + kNaSRgb); X.g_rec = (float4 *)(base + kNaGRec);
    X.s_vis = (int *)(base + kNaSVis); X.g_vis = (int *)(base + kNaGVis);
    X.s_cnt = (int *)(base + kNaSCnt); X.g_cnt = (int *)(base + kNaGCnt);
    X.s_off = (int *)(base + kNaSOff); X.g_off = (int *)(base + kNaGOff);
    X.s_cur = (int *)(base + kNaSCur); X.g_cur = (int *)(base + kNaGCur);
    X.s_list = (int *)(base + kNaSList); X.g_list = (int *)(base + kNaGList);
    X.s_cap = kNaMaxPairs; X.g_cap = kNaMaxPairs;
    X.status = (unsigned *)(base + kNaStatus);
    // the array keeps the previous call's contents: clear the tile counters
    // (adjacent) and the status words, which must start at zero
    GES_CUDA(cudaMemsetAsync(base + kNaSCnt, 0, 2 * kNaTileBytes, st));
    GES_CUDA(cudaMemsetAsync(X.status, 0, ST_WORDS * 4, st));
    SceneView S{desc->n_surfels, desc->n_gaussians, desc->sh_degree, desc->attr_dtype, desc->sh_dtype,
                desc->s_pos, desc->s_rot, desc->s_scale, desc->s_sh, desc->g_pos, desc->g_rot, desc->g_scale,
                desc->g_opac, desc->g_sh, desc->g_filter3d, 3};
    cudaError_t e = launch_forward(S, C, O, X, out_rgb, out_depth, out_surfel_id, aux, st, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    unsigned w[ST_WORDS];
    GES_CUDA(cudaMemcpyAsync(w, X.status, sizeof w, cudaMemcpyDeviceToHost, st));
    GES_CUDA(cudaStreamSynchronize(st));
    if (w[ST_FLAGS] & FLAG_BADQ)
        return fail(GES_ERR_INVALID_ARG, "a rotation quaternion has zero norm or is not finite");
    if (w[ST_FLAGS] & (FLAG_SOVF | FLAG_GOVF))
        return fail(GES_ERR_CAPACITY, "ges_render_noalloc: %u surfel and %u Gaussian tile entries exceed the %lld "
                    "entries per kind of the fixed scratch", w[ST_SPAIRS], w[ST_GPAIRS], (long long)kNaMaxPairs);
    return GES_OK;
}
