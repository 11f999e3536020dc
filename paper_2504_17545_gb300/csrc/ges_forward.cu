// Forward render of Gaussian-enhanced Surfels (Sec. 3, Eq. 1-5) for sm_103a.
//
// Per view, on one stream:
//   k_prep_local  each CTA owns a fixed range of surfels or Gaussians: it sets
//                 each primitive up (surfel raster record + colour, or Gaussian
//                 record: projection, conic, exact support, colour), appends
//                 the visible ones to its own segment of the visible list, and
//                 counts tile overlaps in a shared-memory histogram (16-bit
//                 counters packed in pairs), which it writes out as one row.
//   k_colscan     per tile, exclusive scan of those rows over the CTAs (each
//                 CTA's start inside the tile's list) and the tile total.
//   k_scan        exclusive scan of the tile totals, capacity check.
//   k_fill_local  each CTA re-walks its visible segment and places every
//                 (tile, primitive) pair with shared-memory cursors.
//   k_raster      one CTA per 16x16 tile: the CTA stages 256 records at a time
//                 in shared memory; each warp (an 8x4 pixel block) culls them
//                 by bbox and depth and tests the survivors.  Pass 1 keeps the
//                 lexicographic min of (depth, surfel id); pass 2 accumulates
//                 the depth-tested Gaussians (Eq. 2-4); the epilogue applies
//                 Eq. 5.  Everything per pixel stays in registers.
// No global atomics are needed for binning, so hot tiles do not serialise.
// Very large images (more than 32768 tiles) and callers without binning
// scratch use k_prep_atomic / k_fill_atomic instead (global counters).
//
// List order inside a tile is not fixed (shared-memory atomics), but the
// z-buffer min is order independent and the Gaussian sums are accumulated
// exactly in 64-bit fixed point (units of 2^-32), so the image is
// bit-identical run to run without any sort and without float atomics.
#include "ges_internal.cuh"

namespace ges {

LocalBins plan_local_bins(int64_t N, int64_t M, int num_sms)
{
    LocalBins b{0, 0, 1, 1};
    const int P = 2 * num_sms;   // two 16-warp CTAs per SM
    if (N > 0 && M > 0) {
        b.Ps = (int)((P * N + (N + M) / 2) / (N + M));
        b.Ps = b.Ps < 1 ? 1 : (b.Ps > P - 1 ? P - 1 : b.Ps);
        b.Pg = P - b.Ps;
    } else if (N > 0) {
        b.Ps = P;
    } else if (M > 0) {
        b.Pg = P;
    }
    // a CTA's count for one tile must fit in 16 bits
    const int64_t cap = 60000;
    if (N > 0 && (N + b.Ps - 1) / b.Ps > cap) b.Ps = (int)((N + cap - 1) / cap);
    if (M > 0 && (M + b.Pg - 1) / b.Pg > cap) b.Pg = (int)((M + cap - 1) / cap);
    if (b.Ps > 0) b.Rs = (N + b.Ps - 1) / b.Ps;
    if (b.Pg > 0) b.Rg = (M + b.Pg - 1) / b.Pg;
    // ranges start on multiples of 4 primitives (keeps vector stores aligned)
    b.Rs = (b.Rs + 3) & ~(int64_t)3;
    b.Rg = (b.Rg + 3) & ~(int64_t)3;
    return b;
}

LocalBins plan_local_bins_per_cta(int64_t N, int64_t M, int64_t prims_per_cta)
{
    const int64_t R = prims_per_cta < 256 ? 256 : (prims_per_cta > 60000 ? 60000 : prims_per_cta);
    LocalBins b{0, 0, 1, 1};
    b.Ps = (int)((N + R - 1) / R);
    b.Pg = (int)((M + R - 1) / R);
    if (b.Ps > 0) b.Rs = ((N + b.Ps - 1) / b.Ps + 3) & ~(int64_t)3;
    if (b.Pg > 0) b.Rg = ((M + b.Pg - 1) / b.Pg + 3) & ~(int64_t)3;
    return b;
}

namespace {

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// A 64-byte record as four float4 stores, built from its fields (no
// reinterpretation of the local copy).
__device__ __forceinline__ void store_rec(float4 *dst, const SurfelRec &r)
{
    dst[0] = make_float4(r.ur, r.vr, r.iz0, r.gu);
    dst[1] = make_float4(r.gv, r.au, r.av, r.a0);
    dst[2] = make_float4(r.bu, r.bv, r.b0, __int_as_float(r.id));
    dst[3] = make_float4(r.izmax, __uint_as_float(r.bb_lo), __uint_as_float(r.bb_hi), r.pad);
}

// The first three quarters of a staged Gaussian record (what alpha, the depth
// key and the colour need).
__device__ __forceinline__ GaussRec gauss_rec3(float4 a, float4 b, float4 c)
{
    GaussRec g;
    g.px = a.x; g.py = a.y; g.pxl = a.z; g.pyl = a.w;
    g.la = b.x; g.lb = b.y; g.lc = b.z; g.sigma = b.w;
    g.key = c.x; g.r = c.y; g.g = c.z; g.b = c.w;
    g.id = 0; g.bb_lo = 0u; g.bb_hi = 0u; g.pad = 0.f;
    return g;
}

// Set up primitive i of the given kind; on success write its record and
// return its pixel bbox.
// kGd: the scene's Gaussian kind (a template argument, so that each kernel
// carries only its own set-up code)
// kCol false: leave the colour (Eq. 1) to the batch's colour pass; only the
// geometry is set up and stored here.
template <int kGd, bool kTr = false, bool kCol = true>
__device__ __forceinline__ bool setup_and_store(const SceneView &S, const CamParams &C, const OptParams &O,
                                                const ViewScratch &X, bool surf, int64_t i, int &x0, int &y0,
                                                int &x1, int &y1)
{
    if (surf) {
        SurfelOut o;
        // the record goes out before the colour is evaluated: its registers
        // are free again for the SH row
        surfel_geom(S, C, O, i, o, kTr ? X.s_tside + 4 * i : nullptr);
        if (!o.valid_quat) atomicOr(X.status + ST_FLAGS, FLAG_BADQ);
        if (!o.visible) return false;
        store_rec(X.s_rec + 4 * i, o.rec);
        if (kCol) {
            surfel_colour(S, i, o);
            X.s_rgb[i] = make_float4(o.rgb[0], o.rgb[1], o.rgb[2], 0.f);
        }
        x0 = o.x0; y0 = o.y0; x1 = o.x1; y1 = o.y1;
    } else {
        GaussOut o;
        if (kGd == 2) gauss2d_setup(S, C, O, i, o, kCol);
        else gauss_geom(S, C, O, i, o);
        if (!o.valid_quat) atomicOr(X.status + ST_FLAGS, FLAG_BADQ);
        if (!o.visible) return false;
        if (kGd == 2) {
            store_rec(X.g_rec + 4 * i, o.drec);
        } else {
            // three quarters of the record before the colour is evaluated
            float4 *dst = X.g_rec + 4 * i;
            dst[0] = make_float4(o.rec.px, o.rec.py, o.rec.pxl, o.rec.pyl);
            dst[1] = make_float4(o.rec.la, o.rec.lb, o.rec.lc, o.rec.sigma);
            dst[3] = make_float4(__int_as_float(o.rec.id), __uint_as_float(o.rec.bb_lo),
                                 __uint_as_float(o.rec.bb_hi), o.rec.pad);
            if (kCol) {
                gauss_colour(S, i, o);
                dst[2] = make_float4(o.rec.key, colour_q(o.rec.r), colour_q(o.rec.g), colour_q(o.rec.b));
            } else {
                const float4 c = X.g_col[i];   // the colour pass's colour
                dst[2] = make_float4(o.rec.key, c.x, c.y, c.z);
            }
        }
        if (kGd == 2 || O.geo) {
            float4 a0 = o.aux[0];
            if (kGd == 2 && !kCol) {
                const float4 c = X.g_col[i];   // the colour pass's colour
                a0.x = c.x; a0.y = c.y; a0.z = c.z;
            }
            X.g_aux[2 * i] = a0;
            X.g_aux[2 * i + 1] = o.aux[1];
        }
        x0 = o.x0; y0 = o.y0; x1 = o.x1; y1 = o.y1;
    }
    return true;
}

// ---------------------------------------------------------------------------
// local binning

// CTA c of a view: its range of primitives.  hist: ceil(T/2) shared words
// (two 16-bit counters each); vcnt: a shared counter.
// kKind: 0 both kinds (CTA c < B.Ps: surfels), 1 surfel ranges only, 2
// Gaussian ranges only (a launch per kind gives each its own registers)
template <int kGd, bool kTr = false, int kKind = 0, bool kCol = true>
__device__ __forceinline__ void prep_local_body(const SceneView &S, const CamParams &C, const OptParams &O,
                                                const ViewScratch &X, const LocalBins &B, int c, unsigned *hist,
                                                unsigned &vcnt)
{
    const int T = C.tiles_x * C.tiles_y, words = (T + 1) >> 1;
    const bool surf = kKind == 1 ? true : (kKind == 2 ? false : c < B.Ps);
    const int64_t R = surf ? B.Rs : B.Rg, n = surf ? S.N : S.M;
    const int64_t beg = (int64_t)(surf ? c : c - B.Ps) * R;
    const int64_t end = beg + R < n ? beg + R : n;
    for (int w = threadIdx.x; w < words; w += kPrepThreads) hist[w] = 0u;
    if (threadIdx.x == 0) vcnt = 0u;
    __syncthreads();
    // the CTA's segment of visible primitives: (id, bbox lo, bbox hi) per
    // entry, so that the fill reads its entries contiguously instead of
    // gathering each record's bbox
    int4 *seg = reinterpret_cast<int4 *>(surf ? X.s_vis : X.g_vis) + beg;
    for (int64_t i0 = beg; i0 < end; i0 += kPrepThreads) {
        const int64_t i = i0 + threadIdx.x;
        int x0 = 0, y0 = 0, x1 = -1, y1 = -1;
        const bool vis = i < end && setup_and_store<kGd, kTr, kCol>(S, C, O, X, surf, i, x0, y0, x1, y1);
        const unsigned m = __ballot_sync(0xffffffffu, vis);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned b = 0;
            if ((int)lane_id() == leader) b = atomicAdd(&vcnt, (unsigned)__popc(m));
            b = __shfl_sync(0xffffffffu, b, leader);
            if (vis)
                seg[b + __popc(m & ((1u << lane_id()) - 1u))] =
                    make_int4((int)i, (int)pack_xy(x0, y0), (int)pack_xy(x1, y1), 0);
        }
        if (vis) {
            const int tx0 = x0 >> C.tsx, tx1 = x1 >> C.tsx, ty0 = y0 >> C.tsy, ty1 = y1 >> C.tsy;
            for (int ty = ty0; ty <= ty1; ++ty)
                for (int tx = tx0; tx <= tx1; ++tx) {
                    const int t = ty * C.tiles_x + tx;
                    atomicAdd(hist + (t >> 1), (t & 1) ? 65536u : 1u);
                }
        }
    }
    __syncthreads();
    unsigned *row = X.hist + (size_t)c * words;
    for (int w = threadIdx.x; w < words; w += kPrepThreads) row[w] = hist[w];
    if (threadIdx.x == 0) {
        X.vcount[c] = vcnt;
        atomicAdd(X.status + (surf ? ST_SVIS : ST_GVIS), vcnt);
    }
}

template <int kGd, bool kTr = false>
__global__ void __launch_bounds__(kPrepThreads, 2) k_prep_local(SceneView S, CamParams C, OptParams O,
                                                                ViewScratch X, LocalBins B)
{
    extern __shared__ unsigned hist[];
    __shared__ unsigned vcnt;
    prep_local_body<kGd, kTr>(S, C, O, X, B, blockIdx.x, hist, vcnt);
}

__device__ __forceinline__ unsigned hist_get(const unsigned *row, int t)
{
    const unsigned w = row[t >> 1];
    return (t & 1) ? (w >> 16) : (w & 0xffffu);
}

// Per tile: exclusive scan over the CTAs of one kind.  Block = 32 tiles x 8
// warps; warp w scans CTAs [w*P/8, (w+1)*P/8).
__device__ __forceinline__ void colscan_body(const ViewScratch &X, int T, const LocalBins &B, int bx, bool surf,
                                             unsigned (*part)[33])
{
    const int P = surf ? B.Ps : B.Pg, r0 = surf ? 0 : B.Ps;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = bx * 32 + lane;
    const int words = (T + 1) >> 1;
    const int a = r0 + (int)((int64_t)P * w / 8), b = r0 + (int)((int64_t)P * (w + 1) / 8);
    unsigned s = 0;
    if (t < T)
        for (int r = a; r < b; ++r) s += hist_get(X.hist + (size_t)r * words, t);
    part[w][lane] = s;
    __syncthreads();
    unsigned pre = 0, tot = 0;
    for (int k = 0; k < 8; ++k) {
        const unsigned v = part[k][lane];
        if (k < w) pre += v;
        tot += v;
    }
    if (t < T) {
        for (int r = a; r < b; ++r) {
            X.base[(size_t)r * T + t] = pre;
            pre += hist_get(X.hist + (size_t)r * words, t);
        }
        if (w == 0) (surf ? X.s_cnt : X.g_cnt)[t] = (int)tot;
    }
}

__global__ void __launch_bounds__(256) k_colscan(ViewScratch X, int T, LocalBins B)
{
    __shared__ unsigned part[8][33];
    colscan_body(X, T, B, blockIdx.x, blockIdx.y == 0, part);
}

__device__ __forceinline__ void fill_local_body(const ViewScratch &X, int T, int tiles_x, int tsx, int tsy,
                                                const LocalBins &B, int c, unsigned *cur)
{
    if (X.status[ST_FLAGS] & (FLAG_SOVF | FLAG_GOVF)) return;
    const bool surf = c < B.Ps;
    const int *off = surf ? X.s_off : X.g_off;
    const unsigned *brow = X.base + (size_t)c * T;
    for (int t = threadIdx.x; t < T; t += kFillThreads) cur[t] = (unsigned)off[t] + brow[t];
    __syncthreads();
    const int64_t beg = (int64_t)(surf ? c : c - B.Ps) * (surf ? B.Rs : B.Rg);
    const int4 *seg = reinterpret_cast<const int4 *>(surf ? X.s_vis : X.g_vis) + beg;
    int *list = surf ? X.s_list : X.g_list;
    const unsigned n = X.vcount[c];
    for (unsigned k = threadIdx.x; k < n; k += kFillThreads) {
        const int4 e = seg[k];
        const int id = e.x;
        const unsigned lo = (unsigned)e.y, hi = (unsigned)e.z;
        const int tx0 = (int)(lo & 0xffff) >> tsx, ty0 = (int)(lo >> 16) >> tsy;
        const int tx1 = (int)(hi & 0xffff) >> tsx, ty1 = (int)(hi >> 16) >> tsy;
        for (int ty = ty0; ty <= ty1; ++ty)
            for (int tx = tx0; tx <= tx1; ++tx) list[atomicAdd(cur + ty * tiles_x + tx, 1u)] = id;
    }
}

__global__ void __launch_bounds__(kFillThreads) k_fill_local(ViewScratch X, int T, int tiles_x, int tsx, int tsy,
                                                             LocalBins B)
{
    extern __shared__ unsigned cur[];    // T cursors
    fill_local_body(X, T, tiles_x, tsx, tsy, B, blockIdx.x, cur);
}

// ---------------------------------------------------------------------------
// atomic binning (fallback)

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

template <int kGd, bool kTr = false>
__global__ void __launch_bounds__(256) k_prep_atomic(SceneView S, CamParams C, OptParams O, ViewScratch X,
                                                     int n_sblocks)
{
    const bool surf = (int)blockIdx.x < n_sblocks;
    const int64_t i = (int64_t)(surf ? blockIdx.x : blockIdx.x - n_sblocks) * 256 + threadIdx.x;
    int x0 = 0, y0 = 0, x1 = -1, y1 = -1;
    const bool vis = i < (surf ? S.N : S.M) && setup_and_store<kGd, kTr>(S, C, O, X, surf, i, x0, y0, x1, y1);
    if (vis) {
        int *cnt = surf ? X.s_cnt : X.g_cnt;
        for (int ty = y0 >> C.tsy; ty <= y1 >> C.tsy; ++ty)
            for (int tx = x0 >> C.tsx; tx <= x1 >> C.tsx; ++tx) atomicAdd(cnt + ty * C.tiles_x + tx, 1);
    }
    append_visible(vis, i, X.status + (surf ? ST_SVIS : ST_GVIS), surf ? X.s_vis : X.g_vis);
}

__device__ __forceinline__ void fill_one(const float4 *rec, int id, int tiles_x, int tsx, int tsy, int *cur, int *list)
{
    const float4 r3 = rec[4 * (int64_t)id + 3];
    const unsigned lo = __float_as_uint(r3.y), hi = __float_as_uint(r3.z);
    const int x0 = lo & 0xffff, y0 = lo >> 16, x1 = hi & 0xffff, y1 = hi >> 16;
    for (int ty = y0 >> tsy; ty <= y1 >> tsy; ++ty)
        for (int tx = x0 >> tsx; tx <= x1 >> tsx; ++tx) list[atomicAdd(cur + ty * tiles_x + tx, 1)] = id;
}

__global__ void __launch_bounds__(256) k_fill_atomic(ViewScratch X, int tiles_x, int tsx, int tsy)
{
    if (X.status[ST_FLAGS] & (FLAG_SOVF | FLAG_GOVF)) return;
    const unsigned ns = X.status[ST_SVIS], ng = X.status[ST_GVIS];
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < ns + ng; k += stride) {
        if (k < ns) fill_one(X.s_rec, X.s_vis[k], tiles_x, tsx, tsy, X.s_cur, X.s_list);
        else fill_one(X.g_rec, X.g_vis[k - ns], tiles_x, tsx, tsy, X.g_cur, X.g_list);
    }
}

// ---------------------------------------------------------------------------
// scan of tile totals (both binning modes)

__device__ __forceinline__ void scan_body(const ViewScratch &X, int T, bool surf, long long *warp_tot)
{
    int *cnt = surf ? X.s_cnt : X.g_cnt;
    int *off = surf ? X.s_off : X.g_off;
    int *cur = surf ? X.s_cur : X.g_cur;
    const int64_t cap = surf ? X.s_cap : X.g_cap;
    const int tid = threadIdx.x, per = (T + 1023) / 1024;
    const int b = min(tid * per, T), e = min(b + per, T);
    long long local = 0;
    for (int t = b; t < e; ++t) local += cnt[t];
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
        warp_tot[tid] = wi - w;
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

__global__ void __launch_bounds__(1024) k_scan(ViewScratch X, int T)
{
    __shared__ long long warp_tot[32];
    scan_body(X, T, blockIdx.x == 0, warp_tot);
}

// ---------------------------------------------------------------------------
// raster

__device__ __forceinline__ bool box_overlap(unsigned lo, unsigned hi, int wx0, int wy0, int wx1, int wy1)
{
    const int x0 = lo & 0xffff, y0 = lo >> 16, x1 = hi & 0xffff, y1 = hi >> 16;
    return x0 <= wx1 && x1 >= wx0 && y0 <= wy1 && y1 >= wy0;
}

constexpr int kChunk = kRasterThreads;   // records staged per CTA round

__device__ __forceinline__ void stage_rec(float4 (*st)[kChunk], const float4 *rec, int id, int slot)
{
    const float4 *rp = rec + 4 * (int64_t)id;
    const float4 r0 = rp[0], r1 = rp[1], r2 = rp[2], r3 = rp[3];
    st[0][slot] = r0; st[1][slot] = r1; st[2][slot] = r2; st[3][slot] = r3;
}

// shared planes of one staged Gaussian: the record, plus its side data
// (both words for 2D Gaussians, the first for 3D ones with geometry)
template <int kG, bool kGeo>
__host__ __device__ constexpr int gauss_planes() { return kG == 2 ? 6 : (kGeo ? 5 : 4); }

template <int kG, bool kGeo>
__device__ __forceinline__ void stage_gauss(float4 (*st)[kChunk], const ViewScratch &X, int id, int slot)
{
    stage_rec(st, X.g_rec, id, slot);
    if (gauss_planes<kG, kGeo>() > 4) st[4][slot] = X.g_aux[2 * (int64_t)id];
    if (gauss_planes<kG, kGeo>() > 5) st[5][slot] = X.g_aux[2 * (int64_t)id + 1];
}

// Surfel normal from its record, camera space, facing the camera: the record's
// 1/z = iz0 + gu (u - ur) + gv (v - vr) equals (n . ray)/(n . P), so
// m = (gu fx, gv fy, iz0 - gu (ur - cx) - gv (vr - cy)) = n / (n . P).
__device__ __forceinline__ void surfel_normal(const float4 *rec, int id, const CamParams &C, float *nrm)
{
    const float4 r0 = rec[4 * (int64_t)id], r1 = rec[4 * (int64_t)id + 1];
    const float mx = r0.w * C.fx, my = r1.x * C.fy;
    const float mz = r0.z - r0.w * (r0.x - C.cx) - r1.x * (r0.y - C.cy);
    const float inv = -rsqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz)));
    nrm[0] = mx * inv; nrm[1] = my * inv; nrm[2] = mz * inv;
}

// Geometry outputs of a render (Sec. 6.4, Eq. 10-12); any may be null.
struct GeoMaps {
    float *ns;            // [3,H,W] surfel normal (0 where no surfel)
    float *dsm;           // [H,W] D_smooth
    float *nsm;           // [3,H,W] N_smooth
    float *dg;            // [H,W] D_G
    float *ng;            // [3,H,W] N_G
};

// Staged records as seen by the per-pixel loops: plane p (16-byte quarter) of
// record j, one float4 plane per quarter (consecutive threads store
// consecutive 16 B, and a warp reading one record gets a broadcast).
template <int kPlanes>
struct SoaRecs {
    const float4 (*st)[kChunk];
    __device__ __forceinline__ float4 operator()(int p, int j) const { return st[p][j]; }
};

// The 8x4 pixel block of one warp inside a 16x16 tile, and its lane's pixel.
// kS surfel samples per pixel: 1 (the centre) or 4 (the 2x2 grid at +-0.25
// px, 4x multisampling of Sec. 5; the Gaussians stay at the centre).
template <int kS>
struct WarpBlock {
    int wx0, wy0, wx1, wy1, px, py;
    bool wactive, in_img;
    float u, v, us, vs;    // pixel centre; sample k sits at (us + 0.5 (k & 1), vs + 0.5 (k >> 1))
    __device__ __forceinline__ WarpBlock(const CamParams &C, int tile, unsigned warp, unsigned lane)
    {
        // the 8 warps' 8x4 blocks fill the tile row by row
        const int tx = tile % C.tiles_x, ty = tile / C.tiles_x;
        const int wpr = 1 << (C.tsx - 3);          // blocks per tile row
        wx0 = (tx << C.tsx) + (int)(warp & (unsigned)(wpr - 1)) * kWarpW;
        wy0 = (ty << C.tsy) + (int)(warp >> (C.tsx - 3)) * kWarpH;
        wactive = wx0 < C.W && wy0 < C.H;        // warp-uniform
        wx1 = min(wx0 + kWarpW - 1, C.W - 1);
        wy1 = min(wy0 + kWarpH - 1, C.H - 1);
        px = wx0 + (int)(lane & 7);
        py = wy0 + (int)(lane >> 3);
        in_img = px < C.W && py < C.H;
        u = px + 0.5f;
        v = py + 0.5f;
        us = kS == 4 ? px + 0.25f : u;
        vs = kS == 4 ? py + 0.25f : v;
    }
};

// Pass 1 state of one lane: per sample the 1/z of the nearest hit (0: none)
// and its surfel id; wmin: the smallest 'best' over the warp's samples.
template <int kS>
struct SurfelZ {
    float best[kS];
    int bid[kS];
    float wmin;
    __device__ __forceinline__ void init(bool in_img)
    {
#pragma unroll
        for (int k = 0; k < kS; ++k) { best[k] = in_img ? 0.f : INFINITY; bid[k] = 0x7fffffff; }
        wmin = 0.f;
    }
};

// Pass 1 over n staged surfel records.  A warp skips a surfel whose bbox
// misses its 8x4 block, or whose largest 1/z over the disc (izmax) is below
// every 1/z its pixels already hold (it cannot win anywhere in the block).
// Survivors are tested two at a time; the lexicographic (depth, id) min does
// not depend on the order.
template <int kS, class Recs>
__device__ __forceinline__ void surfel_pass(const Recs &R, int n, const WarpBlock<kS> &B, float izn, unsigned lane,
                                            SurfelZ<kS> &z)
{
    for (int j0 = 0; j0 < n; j0 += 32) {
        const int j = j0 + (int)lane;
        bool keep = false;
        if (j < n) {
            const float4 r3 = R(3, j);     // (izmax, bbox, -)
            keep = box_overlap(__float_as_uint(r3.y), __float_as_uint(r3.z), B.wx0, B.wy0, B.wx1, B.wy1) &&
                   r3.x >= z.wmin;
        }
        unsigned mask = __ballot_sync(0xffffffffu, keep);
        while (mask) {
            const int ja = j0 + __ffs(mask) - 1;
            mask &= mask - 1;
            const bool two = mask != 0u;
            const int jb = two ? j0 + __ffs(mask) - 1 : ja;
            if (two) mask &= mask - 1;
            const float4 a2 = R(2, ja), b2 = R(2, jb);
            const float4 a0 = R(0, ja), a1 = R(1, ja), b0 = R(0, jb), b1 = R(1, jb);
            const int ida = __float_as_int(a2.w), idb = __float_as_int(b2.w);
#pragma unroll
            for (int k = 0; k < kS; ++k) {
                const float uk = B.us + 0.5f * (k & 1), vk = B.vs + 0.5f * (k >> 1);
                const float dua = uk - a0.x, dva = vk - a0.y, dub = uk - b0.x, dvb = vk - b0.y;
                const float iza = fmaf(a0.w, dua, fmaf(a1.x, dva, a0.z));
                const float izb = fmaf(b0.w, dub, fmaf(b1.x, dvb, b0.z));
                const float Aa = fmaf(a1.y, dua, fmaf(a1.z, dva, a1.w));
                const float Ab = fmaf(b1.y, dub, fmaf(b1.z, dvb, b1.w));
                const float Ba = fmaf(a2.x, dua, fmaf(a2.y, dva, a2.z));
                const float Bb = fmaf(b2.x, dub, fmaf(b2.y, dvb, b2.z));
                const float qa = fmaf(Aa, Aa, fmaf(Ba, Ba, -iza * iza));
                const float qb = fmaf(Ab, Ab, fmaf(Bb, Bb, -izb * izb));
                // with one survivor left b is a again: testing it twice is harmless
                const bool ina = qa <= 0.f && iza < izn, inb = qb <= 0.f && izb < izn;
                if (ina && (iza > z.best[k] || (iza == z.best[k] && ida < z.bid[k]))) { z.best[k] = iza; z.bid[k] = ida; }
                if (inb && (izb > z.best[k] || (izb == z.best[k] && idb < z.bid[k]))) { z.best[k] = izb; z.bid[k] = idb; }
            }
        }
        // the warp's depth bound is refreshed once per group of 32 entries:
        // per-survivor refreshes and re-checks cost more instructions than
        // they cull
        float bmin = z.best[0];
#pragma unroll
        for (int k = 1; k < kS; ++k) bmin = fminf(bmin, z.best[k]);
        z.wmin = __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(bmin)));
    }
}

// Resolve of pass 1: C_s is the mean of the samples' colours (background
// where a sample hits nothing), D_s the nearest sample's depth.
template <int kS>
__device__ __forceinline__ void surfel_resolve(const SurfelZ<kS> &z, bool in_img, const float4 *__restrict__ s_rgb,
                                               const float *bg, float &bmax, float &Ds, float *Cs)
{
    bmax = z.best[0];
#pragma unroll
    for (int k = 1; k < kS; ++k) bmax = fmaxf(bmax, z.best[k]);
    Ds = bmax > 0.f ? 1.f / bmax : INFINITY;
    if (kS == 1) {
        Cs[0] = bg[0]; Cs[1] = bg[1]; Cs[2] = bg[2];
        if (z.bid[0] != 0x7fffffff) {
            const float4 c = s_rgb[z.bid[0]];
            Cs[0] = c.x; Cs[1] = c.y; Cs[2] = c.z;
        }
    } else {
        float sr = 0.f, sgc = 0.f, sb = 0.f;
#pragma unroll
        for (int k = 0; k < kS; ++k) {
            float4 c = make_float4(bg[0], bg[1], bg[2], 0.f);
            if (in_img && z.bid[k] != 0x7fffffff) c = s_rgb[z.bid[k]];
            sr += c.x; sgc += c.y; sb += c.z;
        }
        Cs[0] = sr * (1.f / kS); Cs[1] = sgc * (1.f / kS); Cs[2] = sb * (1.f / kS);
    }
}

// Pass 2 sums of one lane, in 64-bit fixed point: W_G in units of 2^-30
// (each alpha rounded once to that grid), the colour sums in units of 2^-46
// (that alpha times the record colour in 2^-16 units, an exact integer
// product), the geometry sums in units of 2^-32.
struct GaussAcc {
    long long r = 0, g = 0, b = 0, w = 0;
    long long d = 0, nx = 0, ny = 0, nz = 0;   // D_G, N_G (geometry maps)
};

// Pass 2 over n staged Gaussian records (Eq. 2-4).  No Gaussian with key >=
// wmaxD (the max over the warp's pixels of D_s) can pass the depth test there.
template <int kS, int kG, bool kGeo, class Recs>
__device__ __forceinline__ void gauss_pass(const Recs &R, int n, const WarpBlock<kS> &B, float Ds, float wmaxD,
                                           float amin32, float izn, unsigned lane, GaussAcc &acc)
{
    for (int j0 = 0; j0 < n; j0 += 32) {
        const int j = j0 + (int)lane;
        bool keep = false;
        if (j < n) {
            const float4 r3 = R(3, j);
            // 3D: key = d - eps (kept with the bbox); 2D: the smallest planar
            // depth (1/izmax) - eps
            const float key = kG == 2 ? 1.f / r3.x - r3.w : r3.w;
            keep = box_overlap(__float_as_uint(r3.y), __float_as_uint(r3.z), B.wx0, B.wy0, B.wx1, B.wy1) &&
                   key < wmaxD;
        }
        unsigned mask = __ballot_sync(0xffffffffu, keep);
        while (mask) {
            const int jj = j0 + __ffs(mask) - 1;
            mask &= mask - 1;
            float a, depth, ok;
            unsigned cr, cg, cb;   // record colours, 2^-16 units
            float4 side = make_float4(0.f, 0.f, 0.f, 0.f);
            if (kG == 2) {
                const float4 r0 = R(0, jj), r1 = R(1, jj), r2 = R(2, jj);
                const float4 x0 = R(4, jj);
                side = R(5, jj);
                const float du = B.u - r0.x, dv = B.v - r0.y;
                const float iz = fmaf(r0.w, du, fmaf(r1.x, dv, r0.z));
                const float A = fmaf(r1.y, du, fmaf(r1.z, dv, r1.w));
                const float Bq = fmaf(r2.x, du, fmaf(r2.y, dv, r2.z));
                depth = __frcp_rn(iz);
                // rho = (a'^2 + b'^2)/r^2; alpha = 2^(log2 sigma' + log2(alpha_min/sigma') rho)
                const float rho = fmaf(A, A, Bq * Bq) * (depth * depth);
                a = ex2_approx(fmaf(side.w, rho, x0.w));
                cr = __float_as_uint(x0.x); cg = __float_as_uint(x0.y); cb = __float_as_uint(x0.z);
                ok = (iz > 0.f && iz < izn && depth - R(3, jj).w < Ds) ? 1.f : 0.f;
            } else {
                const GaussRec g = gauss_rec3(R(0, jj), R(1, jj), R(2, jj));
                float e;
                a = gauss_alpha(g, B.u, B.v, e);
                cr = __float_as_uint(g.r); cg = __float_as_uint(g.g); cb = __float_as_uint(g.b);
                ok = g.key < Ds ? 1.f : 0.f;
                if (kGeo) { side = R(4, jj); depth = side.w; }
            }
            // alpha * 2^32 is exact scaling: the clamp decision equals alpha >= alpha_min
            const float a32 = fminf(a * 4294967296.f, kAlpha32Max);
            if (B.in_img && a32 >= amin32 && ok != 0.f) {
                // alpha on the 2^-30 grid (alpha <= 2: below 2^31), one conversion;
                // the colour terms are exact 32 x 32 -> 64-bit products
                const unsigned A = __float2uint_rn(fminf(a, 2.f) * 1073741824.f);
                acc.w += A;
                acc.r += (long long)((unsigned long long)A * cr);
                acc.g += (long long)((unsigned long long)A * cg);
                acc.b += (long long)((unsigned long long)A * cb);
                if (kGeo) {
                    acc.d += __float2ll_rn(a32 * depth);
                    acc.nx += f2ll_rn(a32 * side.x);
                    acc.ny += f2ll_rn(a32 * side.y);
                    acc.nz += f2ll_rn(a32 * side.z);
                }
            }
        }
    }
}

// Composite (Eq. 5) of one pixel and its outputs.
template <int kS, bool kGeo>
__device__ __forceinline__ void composite_store(const CamParams &C, const OptParams &O, const ViewScratch &X,
                                                const WarpBlock<kS> &B, const SurfelZ<kS> &z, float bmax, float Ds,
                                                const float *Cs, const GaussAcc &acc, float *__restrict__ out_rgb,
                                                float *__restrict__ out_depth, int32_t *__restrict__ out_id,
                                                float *__restrict__ aux, const GeoMaps &geo)
{
    const float k32 = 2.3283064365386963e-10f;   // 2^-32
    const float k30 = 9.3132257461547852e-10f;   // 2^-30
    const float k46 = 1.4210854715202004e-14f;   // 2^-46
    const float WG = __ll2float_rn(acc.w) * k30;
    const float CG[3] = {__ll2float_rn(acc.r) * k46, __ll2float_rn(acc.g) * k46, __ll2float_rn(acc.b) * k46};
    float out[3];
    if (O.mode == GES_MODE_FULL) {
        const float inv = 1.f / (1.f + WG);
        for (int c = 0; c < 3; ++c) out[c] = (Cs[c] + CG[c]) * inv;
    } else if (O.mode == GES_MODE_SURFELS_ONLY) {
        for (int c = 0; c < 3; ++c) out[c] = Cs[c];
    } else {
        for (int c = 0; c < 3; ++c) out[c] = WG > 0.f ? CG[c] / WG : C.bg[c];
    }
    const int64_t HW = (int64_t)C.W * C.H, pix = (int64_t)B.py * C.W + B.px;
    out_rgb[pix] = out[0];
    out_rgb[HW + pix] = out[1];
    out_rgb[2 * HW + pix] = out[2];
    if (out_depth) out_depth[pix] = Ds;
    if (out_id) {
#pragma unroll
        for (int k = 0; k < kS; ++k) out_id[k * HW + pix] = z.bid[k] != 0x7fffffff ? z.bid[k] : -1;
    }
    if (aux) aux[pix] = WG;
    if (kGeo) {
        // Eq. 10-12 with W_s = 1 where a surfel covers the pixel, 0 elsewhere
        float ns[3] = {0.f, 0.f, 0.f};
        const bool covered = bmax > 0.f;
        if (covered) {
            // the nearest sample's surfel (lowest id on a tie)
            int w = 0x7fffffff;
#pragma unroll
            for (int k = 0; k < kS; ++k)
                if (z.best[k] == bmax && z.bid[k] < w) w = z.bid[k];
            surfel_normal(X.s_rec, w, C, ns);
        }
        const float DG = __ll2float_rn(acc.d) * k32;
        const float NG[3] = {__ll2float_rn(acc.nx) * k32, __ll2float_rn(acc.ny) * k32, __ll2float_rn(acc.nz) * k32};
        const float ws = covered ? 1.f : 0.f, wt = ws + WG;
        if (geo.dg) geo.dg[pix] = DG;
        if (geo.dsm) geo.dsm[pix] = wt > 0.f ? ((covered ? Ds : 0.f) + DG) / wt : INFINITY;
        for (int c = 0; c < 3; ++c) {
            if (geo.ns) geo.ns[c * HW + pix] = ns[c];
            if (geo.ng) geo.ng[c * HW + pix] = NG[c];
            if (geo.nsm) geo.nsm[c * HW + pix] = wt > 0.f ? (ws * ns[c] + NG[c]) / wt : 0.f;
        }
    }
}

// One 16x16 tile with the CTA's shared staging (ss/sgs, structure of arrays):
// all 8 warps stage a chunk of records together, then each warp runs its
// 8x4 block over it.  kG: 3D Gaussians (EWA splats) or 2D Gaussians of
// 2D-GES (ray-splat hit, planar depth).  kGeo: also the geometry maps of
// Eq. 10-12.
template <int kS, int kG, bool kGeo>
__device__ __forceinline__ void raster_tile(const ViewScratch &X, const CamParams &C, const OptParams &O,
                                            float *__restrict__ out_rgb, float *__restrict__ out_depth,
                                            int32_t *__restrict__ out_id, float *__restrict__ aux,
                                            const GeoMaps &geo, int tile,
                                            float4 (*ss)[kChunk], float4 (*sgs)[kChunk])
{
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    const WarpBlock<kS> B(C, tile, warp, lane);
    const bool do_s = O.mode != GES_MODE_GAUSSIANS_ONLY, do_g = O.mode != GES_MODE_SURFELS_ONLY;
    const int s0 = do_s ? X.s_off[tile] : 0, s1 = do_s ? X.s_off[tile + 1] : 0;
    const int g0 = do_g ? X.g_off[tile] : 0, g1 = do_g ? X.g_off[tile + 1] : 0;
    const int t = threadIdx.x;

    // first chunk of both lists together: one round trip, one barrier
    if (s0 + t < s1) stage_rec(ss, X.s_rec, X.s_list[s0 + t], t);
    if (g0 + t < g1) stage_gauss<kG, kGeo>(sgs, X, X.g_list[g0 + t], t);
    __syncthreads();

    // ---------------- pass 1: surfel z-buffer ----------------
    SurfelZ<kS> z;
    z.init(B.in_img);
    const SoaRecs<4> RS{ss};
    for (int base = s0; base < s1; base += kChunk) {
        if (base != s0) {
            __syncthreads();
            if (base + t < s1) stage_rec(ss, X.s_rec, X.s_list[base + t], t);
            __syncthreads();
        }
        if (B.wactive) surfel_pass<kS>(RS, min(kChunk, s1 - base), B, C.izn, lane, z);
    }
    float bmax, Ds, Cs[3];
    surfel_resolve<kS>(z, B.in_img, X.s_rgb, C.bg, bmax, Ds, Cs);

    // ---------------- pass 2: Gaussians (Eq. 2-4) ----------------
    GaussAcc acc;
    const float wmaxD = __uint_as_float(__reduce_max_sync(0xffffffffu, B.in_img ? __float_as_uint(Ds) : 0u));
    const float amin32 = O.alpha_min * 4294967296.f;
    const SoaRecs<gauss_planes<kG, kGeo>()> RG{sgs};
    for (int base = g0; base < g1; base += kChunk) {
        if (base != g0) {
            __syncthreads();
            if (base + t < g1) stage_gauss<kG, kGeo>(sgs, X, X.g_list[base + t], t);
            __syncthreads();
        }
        if (B.wactive) gauss_pass<kS, kG, kGeo>(RG, min(kChunk, g1 - base), B, Ds, wmaxD, amin32, C.izn, lane, acc);
    }
    if (!B.in_img) return;
    composite_store<kS, kGeo>(C, O, X, B, z, bmax, Ds, Cs, acc, out_rgb, out_depth, out_id, aux, geo);
}

template <int kS, int kG, bool kGeo>
__global__ void __launch_bounds__(kRasterThreads, kS == 1 && kG == 3 && !kGeo ? 5 : 4)
    k_raster(ViewScratch X, CamParams C, OptParams O, float *__restrict__ out_rgb, float *__restrict__ out_depth,
             int32_t *__restrict__ out_id, float *__restrict__ aux, GeoMaps geo)
{
    __shared__ float4 ss[4][kChunk];
    __shared__ float4 sgs[gauss_planes<kG, kGeo>()][kChunk];
    if (X.status[ST_FLAGS] & (FLAG_SOVF | FLAG_GOVF)) return;
    raster_tile<kS, kG, kGeo>(X, C, O, out_rgb, out_depth, out_id, aux, geo, blockIdx.x, ss, sgs);
}

// ---------------------------------------------------------------------------
// batch: each phase is one launch over all views of all scenes

// largest v with base(v) <= x (bases ascending, base(0) = 0)
template <typename F>
__device__ __forceinline__ int find_view(int n, int x, F base)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base(mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void load_view(const BatchView *V, int v, BatchView &dst)
{
    const int *src = reinterpret_cast<const int *>(V + v);
    int *d = reinterpret_cast<int *>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(BatchView) / 4); k += blockDim.x) d[k] = src[k];
}

// Preprocess of all views, one launch per primitive kind (kKind 1: the
// surfel ranges, 2: the Gaussian ranges); CTA x of the launch takes the view
// and the range of map[x].  The two set-ups need different registers, and a
// kernel per kind keeps the one from spilling for the other.  kCol: the
// colours too (a batch whose scenes each have one view; otherwise the colour
// pass evaluates them for all views of a scene at once).
template <int kGd, int kKind, bool kCol>
__global__ void __launch_bounds__(kPrepThreads, 2) k_bprep(const BatchView *V, const int2 *__restrict__ map,
                                                          OptParams O, unsigned long long *t0)
{
    extern __shared__ unsigned hist[];
    __shared__ unsigned vcnt;
    __shared__ __align__(16) unsigned char bv_raw[sizeof(BatchView)];
    BatchView &bv = *reinterpret_cast<BatchView *>(bv_raw);
    __shared__ int2 sm;
    if (threadIdx.x == 0) {
        // the first CTA to start stamps the batch's start time (t0 is zeroed per launch)
        atomicCAS(t0, 0ull, global_timer_ns());
        sm = map[blockIdx.x];
    }
    __syncthreads();
    load_view(V, sm.x, bv);
    __syncthreads();
    prep_local_body<kGd, false, kKind, kCol>(bv.S, bv.C, O, bv.X, bv.B, sm.y, hist, vcnt);
}

// Colour pass of the batch (Eq. 1): one thread per primitive of one kind,
// for every view of its view group (the views of one scene).  The SH row and
// the position are read once; the views' camera centres and output arrays
// are staged in shared memory kColourViews at a time.  Per view, the
// direction from the centre to that view's camera, the basis and the colour
// are evaluated with the same operations, in the same order, as the inline
// set-up of the per-view path, so both paths store bit-identical colours.
// Surfels: the view's colour array; Gaussians: the view's Gaussian colour
// array in 2^-16 units (dense 16-byte stores; the set-up, which runs after
// this pass, copies them into the records).  Primitives a view does not draw
// get colours that nothing reads.
template <int K>
__device__ __forceinline__ void colour_views(const BatchView *V, const int *__restrict__ gview, int gofs, int gn,
                                             bool surf, int64_t i, bool act, const SceneView &S, float4 *s_cam,
                                             float4 **s_out)
{
    float px = 0.f, py = 0.f, pz = 0.f, c[3 * K];
    if (act) {
        const float *pos = surf ? S.s_pos : S.g_pos;
        px = __ldg(pos + 3 * i); py = __ldg(pos + 3 * i + 1); pz = __ldg(pos + 3 * i + 2);
        load_sh_row<K>(surf ? S.s_sh : S.g_sh, i, S.sh_dtype, c);
    }
    for (int k0 = 0; k0 < gn; k0 += kColourViews) {
        const int m = min(kColourViews, gn - k0);
        __syncthreads();
        if ((int)threadIdx.x < m) {
            const BatchView *bv = V + __ldg(gview + gofs + k0 + threadIdx.x);
            s_cam[threadIdx.x] = make_float4(bv->C.ocam[0], bv->C.ocam[1], bv->C.ocam[2], 0.f);
            s_out[threadIdx.x] = surf ? bv->X.s_rgb : bv->X.g_col;
        }
        __syncthreads();
        if (!act) continue;
        for (int k = 0; k < m; ++k) {
            const float4 o = s_cam[k];
            float dir[3], L;
            view_dir_o(o.x, o.y, o.z, px, py, pz, dir, L);
            float Y[16];
            sh_basis(K, dir[0], dir[1], dir[2], Y);
            float r = 0.5f, g = 0.5f, b = 0.5f;
#pragma unroll
            for (int q = 0; q < K; ++q) {
                r = fmaf(c[3 * q], Y[q], r);
                g = fmaf(c[3 * q + 1], Y[q], g);
                b = fmaf(c[3 * q + 2], Y[q], b);
            }
            r = fmaxf(r, 0.f); g = fmaxf(g, 0.f); b = fmaxf(b, 0.f);
            s_out[k][i] = surf ? make_float4(r, g, b, 0.f) : make_float4(colour_q(r), colour_q(g), colour_q(b), 0.f);
        }
    }
}

__global__ void __launch_bounds__(kColourThreads) k_bcolour(const BatchView *V, const int4 *__restrict__ items,
                                                            const int *__restrict__ gview, unsigned long long *t0)
{
    __shared__ float4 s_cam[kColourViews];
    __shared__ float4 *s_out[kColourViews];
    // the first CTA to start stamps the batch's start time (t0 is zeroed per launch)
    if (threadIdx.x == 0) atomicCAS(t0, 0ull, global_timer_ns());
    const int4 it = items[blockIdx.x];
    const bool surf = it.x == 0;
    const SceneView &S = V[__ldg(gview + it.y)].S;
    const int64_t i = (int64_t)it.w + threadIdx.x;
    const bool act = i < (surf ? S.N : S.M);
    switch ((S.deg + 1) * (S.deg + 1)) {
    case 16: colour_views<16>(V, gview, it.y, it.z, surf, i, act, S, s_cam, s_out); break;
    case 9: colour_views<9>(V, gview, it.y, it.z, surf, i, act, S, s_cam, s_out); break;
    case 4: colour_views<4>(V, gview, it.y, it.z, surf, i, act, S, s_cam, s_out); break;
    default: colour_views<1>(V, gview, it.y, it.z, surf, i, act, S, s_cam, s_out); break;
    }
}

__global__ void __launch_bounds__(256) k_bcolscan(const BatchView *V, int n)
{
    __shared__ unsigned part[8][33];
    __shared__ __align__(16) unsigned char bv_raw[sizeof(BatchView)];
    BatchView &bv = *reinterpret_cast<BatchView *>(bv_raw);
    __shared__ int sv;
    if (threadIdx.x == 0) sv = find_view(n, blockIdx.x, [&](int k) { return V[k].colscan_base; });
    __syncthreads();
    load_view(V, sv, bv);
    __syncthreads();
    colscan_body(bv.X, bv.T, bv.B, blockIdx.x - bv.colscan_base, blockIdx.y == 0, part);
}

__global__ void __launch_bounds__(1024) k_bscan(const BatchView *V)
{
    __shared__ long long warp_tot[32];
    __shared__ __align__(16) unsigned char bv_raw[sizeof(BatchView)];
    BatchView &bv = *reinterpret_cast<BatchView *>(bv_raw);
    load_view(V, blockIdx.x >> 1, bv);
    __syncthreads();
    scan_body(bv.X, bv.T, (blockIdx.x & 1) == 0, warp_tot);
}

__global__ void __launch_bounds__(kFillThreads) k_bfill(const BatchView *V, int n)
{
    extern __shared__ unsigned cur[];
    __shared__ __align__(16) unsigned char bv_raw[sizeof(BatchView)];
    BatchView &bv = *reinterpret_cast<BatchView *>(bv_raw);
    __shared__ int sv;
    if (threadIdx.x == 0) sv = find_view(n, blockIdx.x, [&](int k) { return V[k].prep_base; });
    __syncthreads();
    load_view(V, sv, bv);
    __syncthreads();
    fill_local_body(bv.X, bv.T, bv.C.tiles_x, bv.C.tsx, bv.C.tsy, bv.B, blockIdx.x - bv.prep_base, cur);
}

// Persistent raster over the (view, tile) items of the whole batch: each CTA
// takes the next item from a counter until none is left, so uneven views
// balance across the GPU.
template <int kS, int kG, bool kIds>
__global__ void __launch_bounds__(kRasterThreads, kS == 1 && kG == 3 ? 5 : 4) k_braster(const BatchView *V, int n, OptParams O,
                                                            unsigned *counter, int total)
{
    __shared__ float4 ss[4][kChunk];
    __shared__ float4 sgs[gauss_planes<kG, false>()][kChunk];
    __shared__ __align__(16) unsigned char bv_raw[sizeof(BatchView)];
    BatchView &bv = *reinterpret_cast<BatchView *>(bv_raw);
    __shared__ int item, sv;
    int cur_v = -1;
    if (threadIdx.x == 0) {
        item = (int)atomicAdd(counter, 1u);
        if (item < total) sv = find_view(n, item, [&](int k) { return V[k].tile_base; });
    }
    for (;;) {
        __syncthreads();
        const int it = item;
        if (it >= total) break;
        // the next item is taken now and used after this tile: the atomic's
        // round trip overlaps the raster instead of holding the CTA at a barrier
        int nxt = 0;
        if (threadIdx.x == 0) nxt = (int)atomicAdd(counter, 1u);
        if (sv != cur_v) {
            cur_v = sv;
            load_view(V, cur_v, bv);
        }
        __syncthreads();
        if (!(bv.X.status[ST_FLAGS] & (FLAG_SOVF | FLAG_GOVF)))
            raster_tile<kS, kG, false>(bv.X, bv.C, O, bv.rgb, bv.depth, kIds ? bv.id : nullptr,
                                       kIds ? bv.aux : nullptr, GeoMaps{}, it - bv.tile_base,
                                       ss, sgs);
        __syncthreads();
        if (threadIdx.x == 0) {
            // per-view completion time: the CTA that finishes the view's last tile stamps it
            if (atomicAdd(bv.X.status + ST_RETIRED, 1u) + 1u == (unsigned)bv.T)
                *reinterpret_cast<unsigned long long *>(bv.X.status + ST_TDONE) = global_timer_ns();
            item = nxt;
            if (nxt < total) sv = find_view(n, nxt, [&](int k) { return V[k].tile_base; });
        }
    }
}


}  // namespace

cudaError_t launch_batch(const BatchView *d_views, const BatchPlan &P, const OptParams &O, unsigned *work_counter,
                         cudaStream_t st, cudaEvent_t *ev, bool ids)
{
    // ev (7 events or null): recorded as graph event nodes when captured
    auto mark = [&](int k) { if (ev) cudaEventRecordWithFlags(ev[k], st, cudaEventRecordExternal); };
    mark(0);
    {
        unsigned long long *t0 = reinterpret_cast<unsigned long long *>(work_counter + 2);
        const size_t sm = local_bins_smem(P.max_T, false);
        const bool col = P.total_colour > 0;   // colours in the colour pass, not in the set-up
        if (col) {
            // before the set-up, which copies the Gaussian colours into the records
            if (ev) cudaEventRecordWithFlags(ev[5], st, cudaEventRecordExternal);
            k_bcolour<<<P.total_colour, kColourThreads, 0, st>>>(d_views, P.cmap, P.gview, t0);
            if (ev) cudaEventRecordWithFlags(ev[6], st, cudaEventRecordExternal);
        }
        if (P.total_sprep > 0) {
            const unsigned g = P.total_sprep;
            if (P.gdim == 2 && col) k_bprep<2, 1, false><<<g, kPrepThreads, sm, st>>>(d_views, P.smap, O, t0);
            else if (P.gdim == 2) k_bprep<2, 1, true><<<g, kPrepThreads, sm, st>>>(d_views, P.smap, O, t0);
            else if (col) k_bprep<3, 1, false><<<g, kPrepThreads, sm, st>>>(d_views, P.smap, O, t0);
            else k_bprep<3, 1, true><<<g, kPrepThreads, sm, st>>>(d_views, P.smap, O, t0);
        }
        if (P.total_gprep > 0) {
            const unsigned g = P.total_gprep;
            if (P.gdim == 2 && col) k_bprep<2, 2, false><<<g, kPrepThreads, sm, st>>>(d_views, P.gmap, O, t0);
            else if (P.gdim == 2) k_bprep<2, 2, true><<<g, kPrepThreads, sm, st>>>(d_views, P.gmap, O, t0);
            else if (col) k_bprep<3, 2, false><<<g, kPrepThreads, sm, st>>>(d_views, P.gmap, O, t0);
            else k_bprep<3, 2, true><<<g, kPrepThreads, sm, st>>>(d_views, P.gmap, O, t0);
        }
    }
    mark(1);
    if (P.total_colscan > 0) k_bcolscan<<<dim3(P.total_colscan, 2), 256, 0, st>>>(d_views, P.n);
    k_bscan<<<2 * P.n, 1024, 0, st>>>(d_views);
    mark(2);
    if (P.total_prep > 0)
        k_bfill<<<P.total_prep, kFillThreads, local_bins_smem(P.max_T, true), st>>>(d_views, P.n);
    mark(3);
    // P.gdim: the Gaussian kind shared by all scenes of the batch
    const unsigned grid = P.raster_ctas;
    const int kind = (O.samples == 4 ? 2 : 0) + (P.gdim == 2 ? 1 : 0);
    auto go = [&](auto kern) { kern<<<grid, kRasterThreads, 0, st>>>(d_views, P.n, O, work_counter, P.total_tiles); };
    switch (kind + (ids ? 4 : 0)) {
    case 0: go(k_braster<1, 3, false>); break;
    case 1: go(k_braster<1, 2, false>); break;
    case 2: go(k_braster<4, 3, false>); break;
    case 3: go(k_braster<4, 2, false>); break;
    case 4: go(k_braster<1, 3, true>); break;
    case 5: go(k_braster<1, 2, true>); break;
    case 6: go(k_braster<4, 3, true>); break;
    default: go(k_braster<4, 2, true>); break;
    }
    mark(4);
    return cudaGetLastError();
}

size_t local_bins_smem(int T, bool fill) { return fill ? (size_t)T * 4 : (size_t)((T + 1) / 2) * 4; }

cudaError_t prepare_forward_kernels()
{
    cudaError_t e;
    const int hs = (int)local_bins_smem(kLocalMaxTiles, false);
    if ((e = cudaFuncSetAttribute(k_prep_local<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, hs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_prep_local<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, hs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_prep_local<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, hs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_bprep<3, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, hs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_bprep<3, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, hs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_bprep<2, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, hs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_bprep<2, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, hs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_bprep<3, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, hs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_bprep<3, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, hs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_bprep<2, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, hs)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_bprep<2, 2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, hs)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_fill_local, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)local_bins_smem(kLocalMaxTiles, true))) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(k_bfill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)local_bins_smem(kLocalMaxTiles, true));
}

// preprocess + binning of one view (everything before the raster)
cudaError_t launch_binning(const SceneView &S, const CamParams &C, const OptParams &O, const ViewScratch &X,
                           cudaStream_t st, cudaEvent_t *ev)
{
    const int T = C.tiles_x * C.tiles_y;
    SceneView Sv = S;
    if (O.mode == GES_MODE_GAUSSIANS_ONLY) Sv.N = 0;
    if (O.mode == GES_MODE_SURFELS_ONLY) Sv.M = 0;
    const bool local = X.hist != nullptr && T <= kLocalMaxTiles;
    if (ev) cudaEventRecord(ev[0], st);
    LocalBins B{};
    if (local) {
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        B = plan_local_bins(Sv.N, Sv.M, sms);
        if (B.Ps + B.Pg > 0) {
            const size_t sm = local_bins_smem(T, false);
            if (X.s_tside) k_prep_local<3, true><<<B.Ps + B.Pg, kPrepThreads, sm, st>>>(Sv, C, O, X, B);
            else if (Sv.gdim == 2) k_prep_local<2><<<B.Ps + B.Pg, kPrepThreads, sm, st>>>(Sv, C, O, X, B);
            else k_prep_local<3><<<B.Ps + B.Pg, kPrepThreads, sm, st>>>(Sv, C, O, X, B);
        }
    } else {
        const int nsb = (int)((Sv.N + 255) / 256), ngb = (int)((Sv.M + 255) / 256);
        if (nsb + ngb > 0) {
            if (X.s_tside) k_prep_atomic<3, true><<<nsb + ngb, 256, 0, st>>>(Sv, C, O, X, nsb);
            else if (Sv.gdim == 2) k_prep_atomic<2><<<nsb + ngb, 256, 0, st>>>(Sv, C, O, X, nsb);
            else k_prep_atomic<3><<<nsb + ngb, 256, 0, st>>>(Sv, C, O, X, nsb);
        }
    }
    if (ev) cudaEventRecord(ev[1], st);
    if (local && B.Ps + B.Pg > 0) k_colscan<<<dim3((T + 31) / 32, 2), 256, 0, st>>>(X, T, B);
    k_scan<<<2, 1024, 0, st>>>(X, T);
    if (ev) cudaEventRecord(ev[2], st);
    if (local) {
        if (B.Ps + B.Pg > 0) k_fill_local<<<B.Ps + B.Pg, kFillThreads, local_bins_smem(T, true), st>>>(X, T, C.tiles_x, C.tsx, C.tsy, B);
    } else {
        k_fill_atomic<<<152 * 8, 256, 0, st>>>(X, C.tiles_x, C.tsx, C.tsy);
    }
    if (ev) cudaEventRecord(ev[3], st);
    return cudaGetLastError();
}

namespace {
// Exact work counts of one view: every (sample, surfel) fragment inside the
// opaque disc in front of the near plane, and every (pixel, Gaussian) pair
// with alpha >= alpha_min, over the full tile lists (no culling).
__global__ void __launch_bounds__(256) k_count(SceneView S, ViewScratch X, CamParams C, OptParams O)
{
    __shared__ float4 st[4][256];
    __shared__ unsigned red[2][8];
    if (X.status[ST_FLAGS] & (FLAG_SOVF | FLAG_GOVF)) return;
    const int tile = blockIdx.x, t = threadIdx.x;
    const int tx = tile % C.tiles_x, ty = tile / C.tiles_x;
    const int px = (tx << C.tsx) + (t & ((1 << C.tsx) - 1)), py = (ty << C.tsy) + (t >> C.tsx);
    const bool in_img = px < C.W && py < C.H;
    const float u = px + 0.5f, v = py + 0.5f;
    unsigned ns = 0, ng = 0;
    for (int kind = 0; kind < 2; ++kind) {
        if (kind == 0 && O.mode == GES_MODE_GAUSSIANS_ONLY) continue;
        if (kind == 1 && O.mode == GES_MODE_SURFELS_ONLY) continue;
        const int *off = kind == 0 ? X.s_off : X.g_off;
        const int *list = kind == 0 ? X.s_list : X.g_list;
        const float4 *rec = kind == 0 ? X.s_rec : X.g_rec;
        const int a = off[tile], b = off[tile + 1];
        for (int base = a; base < b; base += 256) {
            __syncthreads();
            if (base + t < b) stage_rec(st, rec, list[base + t], t);
            __syncthreads();
            const int n = min(256, b - base);
            if (!in_img) continue;
            for (int j = 0; j < n; ++j) {
                if (kind == 0) {
                    const float4 r0 = st[0][j], r1 = st[1][j], r2 = st[2][j];
                    for (int k = 0; k < O.samples; ++k) {
                        const float uk = O.samples == 4 ? px + 0.25f + 0.5f * (k & 1) : u;
                        const float vk = O.samples == 4 ? py + 0.25f + 0.5f * (k >> 1) : v;
                        const float du = uk - r0.x, dv = vk - r0.y;
                        const float iz = fmaf(r0.w, du, fmaf(r1.x, dv, r0.z));
                        const float A = fmaf(r1.y, du, fmaf(r1.z, dv, r1.w));
                        const float B = fmaf(r2.x, du, fmaf(r2.y, dv, r2.z));
                        ns += (fmaf(A, A, fmaf(B, B, -iz * iz)) <= 0.f && iz > 0.f && iz < C.izn) ? 1u : 0u;
                    }
                } else if (S.gdim == 2) {
                    const float4 r0 = st[0][j], r1 = st[1][j], r2 = st[2][j];
                    const int id = __float_as_int(st[2][j].w);
                    const float4 x0 = X.g_aux[2 * (int64_t)id], x1 = X.g_aux[2 * (int64_t)id + 1];
                    const float du = u - r0.x, dv = v - r0.y;
                    const float iz = fmaf(r0.w, du, fmaf(r1.x, dv, r0.z));
                    const float A = fmaf(r1.y, du, fmaf(r1.z, dv, r1.w));
                    const float B = fmaf(r2.x, du, fmaf(r2.y, dv, r2.z));
                    const float z = __frcp_rn(iz);
                    const float a = ex2_approx(fmaf(x1.w, fmaf(A, A, B * B) * (z * z), x0.w));
                    ng += (iz > 0.f && iz < C.izn && a >= O.alpha_min) ? 1u : 0u;
                } else {
                    const GaussRec g = gauss_rec3(st[0][j], st[1][j], make_float4(0.f, 0.f, 0.f, 0.f));
                    float e;
                    ng += gauss_alpha(g, u, v, e) >= O.alpha_min ? 1u : 0u;
                }
            }
        }
    }
    for (int d = 16; d >= 1; d >>= 1) {
        ns += __shfl_xor_sync(0xffffffffu, ns, d);
        ng += __shfl_xor_sync(0xffffffffu, ng, d);
    }
    if ((t & 31) == 0) { red[0][t >> 5] = ns; red[1][t >> 5] = ng; }
    __syncthreads();
    if (t == 0) {
        unsigned a = 0, b = 0;
        for (int w = 0; w < 8; ++w) { a += red[0][w]; b += red[1][w]; }
        atomicAdd(X.status + ST_SFRAG, a);
        atomicAdd(X.status + ST_GFRAG, b);
    }
}
}  // namespace

namespace {
template <int kS, int kG>
void launch_raster(const ViewScratch &X, const CamParams &C, const OptParams &O, float *out_rgb, float *out_depth,
                   int32_t *out_id, float *aux, const GeoMaps &geo, cudaStream_t st)
{
    const unsigned grid = C.tiles_x * C.tiles_y;
    if (O.geo) k_raster<kS, kG, true><<<grid, kRasterThreads, 0, st>>>(X, C, O, out_rgb, out_depth, out_id, aux, geo);
    else k_raster<kS, kG, false><<<grid, kRasterThreads, 0, st>>>(X, C, O, out_rgb, out_depth, out_id, aux, geo);
}
}  // namespace

cudaError_t launch_forward(const SceneView &S, const CamParams &C, const OptParams &O, const ViewScratch &X,
                           float *out_rgb, float *out_depth, int32_t *out_id, float *aux, cudaStream_t st,
                           cudaEvent_t *ev, const float *const *geo_maps)
{
    cudaError_t e = launch_binning(S, C, O, X, st, ev);
    if (e != cudaSuccess) return e;
    GeoMaps geo{};
    if (geo_maps) geo = GeoMaps{const_cast<float *>(geo_maps[0]), const_cast<float *>(geo_maps[1]),
                                const_cast<float *>(geo_maps[2]), const_cast<float *>(geo_maps[3]),
                                const_cast<float *>(geo_maps[4])};
    if (O.samples == 4 && S.gdim == 2) launch_raster<4, 2>(X, C, O, out_rgb, out_depth, out_id, aux, geo, st);
    else if (O.samples == 4) launch_raster<4, 3>(X, C, O, out_rgb, out_depth, out_id, aux, geo, st);
    else if (S.gdim == 2) launch_raster<1, 2>(X, C, O, out_rgb, out_depth, out_id, aux, geo, st);
    else launch_raster<1, 3>(X, C, O, out_rgb, out_depth, out_id, aux, geo, st);
    if (ev) cudaEventRecord(ev[4], st);
    return cudaGetLastError();
}

namespace {
// Mip-GES 3D filter variance (Sec. 6.1, Mip-Splatting's world filter): per
// Gaussian, the highest sampling rate max(fx, fy)/z over the cameras whose
// image rectangle holds the projected centre at z > znear; v = s3d / rate^2,
// -1 while unseen.  The largest v seen is kept in *vmax (non-negative floats
// order like their bit patterns, so an integer max is exact and order free).
constexpr int kFiltCams = 32;

__global__ void __launch_bounds__(256) k_filter3d(SceneView S, const CamParams *__restrict__ cams, int n_cams,
                                                  float s3d, float *__restrict__ out, unsigned *vmax)
{
    __shared__ __align__(16) unsigned char cbuf[kFiltCams * sizeof(CamParams)];
    const CamParams *sc = reinterpret_cast<const CamParams *>(cbuf);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float px = 0.f, py = 0.f, pz = 0.f;
    if (i < S.M) { px = __ldg(S.g_pos + 3 * i); py = __ldg(S.g_pos + 3 * i + 1); pz = __ldg(S.g_pos + 3 * i + 2); }
    float nu = 0.f;
    for (int c0 = 0; c0 < n_cams; c0 += kFiltCams) {
        const int nc = min(kFiltCams, n_cams - c0);
        __syncthreads();
        const int *src = reinterpret_cast<const int *>(cams + c0);
        int *dst = reinterpret_cast<int *>(cbuf);
        for (int k = threadIdx.x; k < nc * (int)(sizeof(CamParams) / 4); k += blockDim.x) dst[k] = src[k];
        __syncthreads();
        if (i >= S.M) continue;
        for (int c = 0; c < nc; ++c) {
            const CamParams &C = sc[c];
            const df tz = df_dot3_plus(C.R + 6, px, py, pz, C.t[2]);
            if (!(tz.hi > C.znear || (tz.hi == C.znear && tz.lo > 0.f))) continue;
            const df tx = df_dot3_plus(C.R, px, py, pz, C.t[0]);
            const df ty = df_dot3_plus(C.R + 3, px, py, pz, C.t[1]);
            const float u = df_add_f(df_mul_f(df_div(tx, tz), C.fx), C.cx).hi;
            const float v = df_add_f(df_mul_f(df_div(ty, tz), C.fy), C.cy).hi;
            if (!(u >= 0.f && u <= (float)C.W && v >= 0.f && v <= (float)C.H)) continue;
            nu = fmaxf(nu, fmaxf(C.fx, C.fy) / tz.hi);
        }
    }
    if (i >= S.M) return;
    if (nu > 0.f) {
        const float v = s3d / (nu * nu);
        out[i] = v;
        atomicMax(vmax, __float_as_uint(v));
    } else {
        out[i] = -1.f;
    }
}

__global__ void __launch_bounds__(256) k_filter3d_fill(int64_t M, float *__restrict__ out, const unsigned *vmax)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < M && out[i] < 0.f) out[i] = __uint_as_float(*vmax);
}
}  // namespace

cudaError_t launch_filter3d(const SceneView &S, const CamParams *d_cams, int n_cams, float s3d, float *out,
                            unsigned *d_vmax, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(d_vmax, 0, sizeof(unsigned), st);
    if (e != cudaSuccess || S.M == 0) return e;
    const unsigned blocks = (unsigned)((S.M + 255) / 256);
    k_filter3d<<<blocks, 256, 0, st>>>(S, d_cams, n_cams, s3d, out, d_vmax);
    k_filter3d_fill<<<blocks, 256, 0, st>>>(S.M, out, d_vmax);
    return cudaGetLastError();
}

cudaError_t launch_count(const SceneView &S, const CamParams &C, const OptParams &O, const ViewScratch &X,
                         cudaStream_t st)
{
    cudaError_t e = launch_binning(S, C, O, X, st, nullptr);
    if (e != cudaSuccess) return e;
    k_count<<<C.tiles_x * C.tiles_y, 256, 0, st>>>(S, X, C, O);
    return cudaGetLastError();
}

}  // namespace ges
