// Forward render of Gaussian-enhanced Surfels (Sec. 3, Eq. 1-5) for sm_103a.
//
// Per view, four launches on one stream:
//   k_preprocess  one thread per primitive: surfel raster record + colour, or
//                 Gaussian record (projection, conic, exact support, colour);
//                 counts tile overlaps with integer atomics and appends the
//                 primitive to a compact visible list.
//   k_scan        exclusive scan of the per-tile counts (one CTA per list),
//                 capacity check, counts reset for the next render.
//   k_fill        scatters visible primitives into their tiles' lists.
//   k_raster      one CTA per 16x16 tile, one warp per 8x4 pixel block:
//                 pass 1 z-buffer (lexicographic min of (depth, surfel id)),
//                 pass 2 depth-tested Gaussian accumulation (Eq. 2-4) and the
//                 composite of Eq. 5, all in registers.
// List order inside a tile is whatever the fill atomics produce: the z-buffer
// min is order independent and the Gaussian sums are accumulated exactly in
// 64-bit fixed point (2^-32 units), so the image is bit-identical run to run
// without any sort and without floating-point atomics.
#include "ges_internal.cuh"

namespace ges {

namespace {

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ void append_visible(bool vis, int64_t i, unsigned *counter, int *list)
{
    const unsigned m = __ballot_sync(0xffffffffu, vis);
    if (m == 0u) return;
    const unsigned lane = lane_id();
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if ((int)lane == leader) base = atomicAdd(counter, (unsigned)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (vis) list[base + __popc(m & ((1u << lane) - 1u))] = (int)i;
}

__device__ __forceinline__ void count_tiles(int x0, int y0, int x1, int y1, int tiles_x, int *cnt)
{
    const int tx0 = x0 / kTile, tx1 = x1 / kTile, ty0 = y0 / kTile, ty1 = y1 / kTile;
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(cnt + ty * tiles_x + tx, 1);
}

__global__ void __launch_bounds__(256) k_preprocess(SceneView S, CamParams C, OptParams O, ViewScratch X,
                                                    int n_sblocks)
{
    if ((int)blockIdx.x < n_sblocks) {
        const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
        bool vis = false;
        if (i < S.N) {
            SurfelOut o;
            surfel_setup(S, C, O, i, o);
            if (!o.valid_quat) atomicOr(X.status + ST_FLAGS, FLAG_BADQ);
            if (o.visible) {
                const float4 *src = reinterpret_cast<const float4 *>(&o.rec);
                float4 *dst = X.s_rec + 4 * i;
                dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; dst[3] = src[3];
                X.s_rgb[i] = make_float4(o.rgb[0], o.rgb[1], o.rgb[2], 0.f);
                count_tiles(o.x0, o.y0, o.x1, o.y1, C.tiles_x, X.s_cnt);
                vis = true;
            }
        }
        append_visible(vis, i, X.status + ST_SVIS, X.s_vis);
    } else {
        const int64_t i = (int64_t)(blockIdx.x - n_sblocks) * 256 + threadIdx.x;
        bool vis = false;
        if (i < S.M) {
            GaussOut o;
            gauss_setup(S, C, O, i, o);
            if (!o.valid_quat) atomicOr(X.status + ST_FLAGS, FLAG_BADQ);
            if (o.visible) {
                const float4 *src = reinterpret_cast<const float4 *>(&o.rec);
                float4 *dst = X.g_rec + 4 * i;
                dst[0] = src[0]; dst[1] = src[1]; dst[2] = src[2]; dst[3] = src[3];
                count_tiles(o.x0, o.y0, o.x1, o.y1, C.tiles_x, X.g_cnt);
                vis = true;
            }
        }
        append_visible(vis, i, X.status + ST_GVIS, X.g_vis);
    }
}

// Exclusive scan of T tile counts by one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_scan(ViewScratch X, int T)
{
    const bool surf = blockIdx.x == 0;
    int *cnt = surf ? X.s_cnt : X.g_cnt;
    int *off = surf ? X.s_off : X.g_off;
    int *cur = surf ? X.s_cur : X.g_cur;
    const int64_t cap = surf ? X.s_cap : X.g_cap;
    __shared__ long long warp_tot[32];
    const int tid = threadIdx.x, per = (T + 1023) / 1024;
    const int b = min(tid * per, T), e = min(b + per, T);
    long long local = 0;
    for (int t = b; t < e; ++t) local += cnt[t];
    // block exclusive scan of the per-thread sums
    long long incl = local;
    for (int d = 1; d < 32; d <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, incl, d);
        if ((tid & 31) >= d) incl += y;
    }
    if ((tid & 31) == 31) warp_tot[tid >> 5] = incl;
    __syncthreads();
    if (tid < 32) {
        long long w = warp_tot[tid], wi = w;
        for (int d = 1; d < 32; d <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, wi, d);
            if (tid >= d) wi += y;
        }
        warp_tot[tid] = wi - w;   // exclusive prefix of warp totals
    }
    __syncthreads();
    long long run = warp_tot[tid >> 5] + incl - local;
    for (int t = b; t < e; ++t) {
        const int c = cnt[t];
        off[t] = (int)run;
        cur[t] = (int)run;
        cnt[t] = 0;
        run += c;
    }
    if (tid == 1023) {
        off[T] = (int)run;
        X.status[surf ? ST_SPAIRS : ST_GPAIRS] = (unsigned)run;
        if (run > cap) atomicOr(X.status + ST_FLAGS, surf ? FLAG_SOVF : FLAG_GOVF);
    }
}

__device__ __forceinline__ void fill_one(const float4 *rec, int id, int tiles_x, int *cur, int *list)
{
    const float4 r3 = rec[4 * (int64_t)id + 3];
    const unsigned lo = __float_as_uint(r3.y), hi = __float_as_uint(r3.z);
    const int x0 = lo & 0xffff, y0 = lo >> 16, x1 = hi & 0xffff, y1 = hi >> 16;
    const int tx0 = x0 / kTile, tx1 = x1 / kTile, ty0 = y0 / kTile, ty1 = y1 / kTile;
    for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
            const int slot = atomicAdd(cur + ty * tiles_x + tx, 1);
            list[slot] = id;
        }
}

__global__ void __launch_bounds__(256) k_fill(ViewScratch X, int tiles_x)
{
    if (X.status[ST_FLAGS] & (FLAG_SOVF | FLAG_GOVF)) return;
    const unsigned ns = X.status[ST_SVIS], ng = X.status[ST_GVIS];
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < ns + ng; k += stride) {
        if (k < ns) fill_one(X.s_rec, X.s_vis[k], tiles_x, X.s_cur, X.s_list);
        else fill_one(X.g_rec, X.g_vis[k - ns], tiles_x, X.g_cur, X.g_list);
    }
}

__device__ __forceinline__ bool box_overlap(unsigned lo, unsigned hi, int wx0, int wy0, int wx1, int wy1)
{
    const int x0 = lo & 0xffff, y0 = lo >> 16, x1 = hi & 0xffff, y1 = hi >> 16;
    return x0 <= wx1 && x1 >= wx0 && y0 <= wy1 && y1 >= wy0;
}

constexpr int kStage = 5;   // float4 per staged record (4 used + 1 pad: conflict-free STS.128)

__global__ void __launch_bounds__(kRasterThreads) k_raster(ViewScratch X, CamParams C, OptParams O,
                                                           float *__restrict__ out_rgb,
                                                           float *__restrict__ out_depth,
                                                           int32_t *__restrict__ out_id,
                                                           float *__restrict__ aux)
{
    __shared__ float4 stage[kRasterThreads / 32][32][kStage];
    if (X.status[ST_FLAGS] & (FLAG_SOVF | FLAG_GOVF)) return;
    const int tile = blockIdx.x;
    const int tx = tile % C.tiles_x, ty = tile / C.tiles_x;
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    const int wx0 = tx * kTile + (warp & 1) * kWarpW, wy0 = ty * kTile + (warp >> 1) * kWarpH;
    if (wx0 >= C.W || wy0 >= C.H) return;   // warp-uniform: no pixel of this block is in the image
    const int wx1 = min(wx0 + kWarpW - 1, C.W - 1), wy1 = min(wy0 + kWarpH - 1, C.H - 1);
    const int px = wx0 + (int)(lane & 7), py = wy0 + (int)(lane >> 3);
    const bool in_img = px < C.W && py < C.H;
    const float u = px + 0.5f, v = py + 0.5f;
    float4(*st)[kStage] = stage[warp];

    // ---------------- pass 1: surfel z-buffer ----------------
    float best = in_img ? 0.f : INFINITY;   // 1/z of the nearest hit (0: none)
    int bid = 0x7fffffff;
    if (O.mode != GES_MODE_GAUSSIANS_ONLY) {
        const int s0 = X.s_off[tile], s1 = X.s_off[tile + 1];
        float wmin = 0.f;   // smallest 'best' in the warp: surfels nearer than 1/wmin nowhere can't win
        for (int base = s0; base < s1; base += 32) {
            const int k = base + (int)lane;
            bool keep = false;
            if (k < s1) {
                const int id = X.s_list[k];
                const float4 *rp = X.s_rec + 4 * (int64_t)id;
                const float4 r0 = rp[0], r1 = rp[1], r2 = rp[2], r3 = rp[3];
                keep = box_overlap(__float_as_uint(r3.y), __float_as_uint(r3.z), wx0, wy0, wx1, wy1) &&
                       r2.w >= wmin;
                st[lane][0] = r0; st[lane][1] = r1; st[lane][2] = r2; st[lane][3] = r3;
            }
            unsigned mask = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                const float4 r2 = st[j][2];
                if (r2.w < wmin) continue;                      // warp-uniform re-check
                const float4 r0 = st[j][0], r1 = st[j][1];
                const int id = __float_as_int(st[j][3].x);
                const float du = u - r0.x, dv = v - r0.y;
                const float iz = fmaf(r0.w, du, fmaf(r1.x, dv, r0.z));
                const float A = fmaf(r1.y, du, fmaf(r1.z, dv, r1.w));
                const float B = fmaf(r2.x, du, fmaf(r2.y, dv, r2.z));
                const float q = fmaf(A, A, fmaf(B, B, -iz * iz));
                const bool hit = q <= 0.f && iz < C.izn && (iz > best || (iz == best && id < bid));
                if (hit) { best = iz; bid = id; }
                if (__any_sync(0xffffffffu, hit))
                    wmin = __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(best)));
            }
            __syncwarp();
        }
    }
    const bool covered = bid != 0x7fffffff;
    const float Ds = covered ? 1.f / best : INFINITY;
    float Cs[3] = {C.bg[0], C.bg[1], C.bg[2]};
    if (covered) {
        const float4 c = X.s_rgb[bid];
        Cs[0] = c.x; Cs[1] = c.y; Cs[2] = c.z;
    }

    // ---------------- pass 2: Gaussians (Eq. 2-4) ----------------
    long long acc_r = 0, acc_g = 0, acc_b = 0, acc_w = 0;
    if (O.mode != GES_MODE_SURFELS_ONLY) {
        const int g0 = X.g_off[tile], g1 = X.g_off[tile + 1];
        // no Gaussian with key >= max_lanes(D_s) can pass the depth test here
        const float wmaxD = __uint_as_float(__reduce_max_sync(0xffffffffu, in_img ? __float_as_uint(Ds) : 0u));
        const float amin32 = O.alpha_min * 4294967296.f;
        for (int base = g0; base < g1; base += 32) {
            const int k = base + (int)lane;
            bool keep = false;
            if (k < g1) {
                const int id = X.g_list[k];
                const float4 *rp = X.g_rec + 4 * (int64_t)id;
                const float4 r0 = rp[0], r1 = rp[1], r2 = rp[2], r3 = rp[3];
                keep = box_overlap(__float_as_uint(r3.y), __float_as_uint(r3.z), wx0, wy0, wx1, wy1) &&
                       r2.x < wmaxD;
                st[lane][0] = r0; st[lane][1] = r1; st[lane][2] = r2; st[lane][3] = r3;
            }
            unsigned mask = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            while (mask) {
                const int j = __ffs(mask) - 1;
                mask &= mask - 1;
                GaussRec g;
                *reinterpret_cast<float4 *>(&g.px) = st[j][0];
                *reinterpret_cast<float4 *>(&g.ca) = st[j][1];
                *reinterpret_cast<float4 *>(&g.key) = st[j][2];
                float e;
                const float a = gauss_alpha(g, u, v, e);
                // alpha * 2^32 is exact scaling: the clamp decision equals alpha >= alpha_min
                const float a32 = a * 4294967296.f;
                if (in_img && a32 >= amin32 && g.key < Ds) {
                    acc_w += __float2ll_rn(a32);
                    acc_r += __float2ll_rn(a32 * g.r);
                    acc_g += __float2ll_rn(a32 * g.g);
                    acc_b += __float2ll_rn(a32 * g.b);
                }
            }
            __syncwarp();
        }
    }
    if (!in_img) return;

    // ---------------- composite (Eq. 5) ----------------
    const float k32 = 2.3283064365386963e-10f;   // 2^-32
    const float WG = __ll2float_rn(acc_w) * k32;
    const float CG[3] = {__ll2float_rn(acc_r) * k32, __ll2float_rn(acc_g) * k32, __ll2float_rn(acc_b) * k32};
    float out[3];
    if (O.mode == GES_MODE_FULL) {
        const float inv = 1.f / (1.f + WG);
        for (int c = 0; c < 3; ++c) out[c] = (Cs[c] + CG[c]) * inv;
    } else if (O.mode == GES_MODE_SURFELS_ONLY) {
        for (int c = 0; c < 3; ++c) out[c] = Cs[c];
    } else {
        for (int c = 0; c < 3; ++c) out[c] = WG > 0.f ? CG[c] / WG : C.bg[c];
    }
    const int64_t HW = (int64_t)C.W * C.H, pix = (int64_t)py * C.W + px;
    out_rgb[pix] = out[0];
    out_rgb[HW + pix] = out[1];
    out_rgb[2 * HW + pix] = out[2];
    if (out_depth) out_depth[pix] = Ds;
    if (out_id) out_id[pix] = covered ? bid : -1;
    if (aux) aux[pix] = WG;
}

}  // namespace

cudaError_t launch_forward(const SceneView &S, const CamParams &C, const OptParams &O, const ViewScratch &X,
                           float *out_rgb, float *out_depth, int32_t *out_id, float *aux, cudaStream_t st,
                           cudaEvent_t *ev)
{
    const int T = C.tiles_x * C.tiles_y;
    const int nsb = O.mode == GES_MODE_GAUSSIANS_ONLY ? 0 : (int)((S.N + 255) / 256);
    const int ngb = O.mode == GES_MODE_SURFELS_ONLY ? 0 : (int)((S.M + 255) / 256);
    SceneView Sv = S;
    if (O.mode == GES_MODE_GAUSSIANS_ONLY) Sv.N = 0;
    if (O.mode == GES_MODE_SURFELS_ONLY) Sv.M = 0;
    if (ev) cudaEventRecord(ev[0], st);
    if (nsb + ngb > 0) k_preprocess<<<nsb + ngb, 256, 0, st>>>(Sv, C, O, X, nsb);
    if (ev) cudaEventRecord(ev[1], st);
    k_scan<<<2, 1024, 0, st>>>(X, T);
    if (ev) cudaEventRecord(ev[2], st);
    k_fill<<<152 * 8, 256, 0, st>>>(X, C.tiles_x);
    if (ev) cudaEventRecord(ev[3], st);
    k_raster<<<T, kRasterThreads, 0, st>>>(X, C, O, out_rgb, out_depth, out_id, aux);
    if (ev) cudaEventRecord(ev[4], st);
    return cudaGetLastError();
}

}  // namespace ges
