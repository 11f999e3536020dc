// Translucent-surfel render of the coarse optimisation stage (Sec. 4.1,
// Eq. 6-7) and its backward, plus the Gaussian contribution score (Eq. 9).
//
// A surfel's opacity at the ray-plane hit (a, b in scale units) is
// alpha = min(1, w G), G = exp(-(a^2 + b^2)/2), zero where min(alpha, G) <
// 1/255; for w >= 1 that support is the opaque disc, so the surfel records and
// tile lists of the opaque render serve unchanged (their forms are normalised
// by r = sqrt(surfel_r2): rho = r^2 (A^2 + B^2)/iz^2).
//
//   binning      the opaque preprocess (surfels only), which also writes each
//                surfel's camera-space frame for the backward;
//   k_tkeys      per tile-list entry the key (centre camera depth, index);
//   k_tsort      per tile, the list sorted by that key (bitonic, in shared
//                memory up to 4096 entries, in global memory beyond);
//   k_traster    per pixel: the frontmost contributor (least depth at the
//                pixel, ties: lower index), then front-to-back blending in the
//                sorted order, the frontmost first when front_first is set,
//                stopping once T < 1e-4 after a blend; C += T bg;
//   k_tbwd       per pixel in reverse order, dC/dc = alpha T and
//                dC/dalpha = T (c - S_behind), chained to the surfel's camera-
//                space frame; the warp reduces each entry's 18 terms in a
//                fixed order (a halving reduce-scatter) and the lanes holding
//                the totals add them as 64-bit fixed point, so the result
//                does not depend on the order of the atomics;
//   k_tfinal     per surfel: fixed point -> float, camera -> world, rotation
//                through the quaternion's normalisation, colour -> SH.
#include "ges_internal.cuh"

namespace ges {

namespace {

constexpr int kSortCap = 4096;          // entries sorted in shared memory
constexpr float kTStop = 1e-4f;         // blending stops once T falls below this
constexpr int kTAcc = 18;               // gradient terms accumulated per surfel

__device__ __forceinline__ unsigned lane_idx() { return threadIdx.x & 31u; }

// order-preserving float -> uint
__device__ __forceinline__ unsigned depth_key(float z)
{
    const unsigned b = __float_as_uint(z);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void __launch_bounds__(256) k_tkeys(const int *__restrict__ list, const int *__restrict__ n_ptr,
                                               const float4 *__restrict__ tside, unsigned long long *keys,
                                               const unsigned *status)
{
    if (status[ST_FLAGS] & FLAG_SOVF) return;     // lists not filled; the count exceeds the capacity
    const int n = *n_ptr;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int id = list[i];
        keys[i] = ((unsigned long long)depth_key(tside[4 * (int64_t)id].z) << 32) | (unsigned)id;
    }
}

// Ascending bitonic sort of a[0..n) (m = the next power of two); pairs whose
// upper index is >= n are skipped, which equals padding with +infinity
// because every compare-exchange moves the smaller key to the lower index.
// (k, h, j are powers of two: the pair index splits with shifts and masks.)
__device__ __forceinline__ void bitonic(unsigned long long *a, int n, int m)
{
    for (int k = 2; k <= m; k <<= 1) {
        const int lh = __ffs(k) - 2;              // log2(k / 2)
        for (int p = threadIdx.x; p < m / 2; p += blockDim.x) {
            const int i = ((p >> lh) << (lh + 1)) + (p & ((1 << lh) - 1)), l = i ^ (k - 1);
            if (l < n && a[i] > a[l]) { const unsigned long long t = a[i]; a[i] = a[l]; a[l] = t; }
        }
        __syncthreads();
        for (int j = k >> 2; j >= 1; j >>= 1) {
            const int lj = __ffs(j) - 1;
            for (int p = threadIdx.x; p < m / 2; p += blockDim.x) {
                const int i = ((p >> lj) << (lj + 1)) + (p & (j - 1)), l = i + j;
                if (l < n && a[i] > a[l]) { const unsigned long long t = a[i]; a[i] = a[l]; a[l] = t; }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256) k_tsort(const int *__restrict__ off, unsigned long long *keys, int *list,
                                               const unsigned *status)
{
    __shared__ unsigned long long sk[kSortCap];
    if (status[ST_FLAGS] & FLAG_SOVF) return;
    const int a = off[blockIdx.x], n = off[blockIdx.x + 1] - a;
    if (n <= 1) return;
    int m = 1;
    while (m < n) m <<= 1;
    if (n <= kSortCap) {
        for (int k = threadIdx.x; k < n; k += blockDim.x) sk[k] = keys[a + k];
        __syncthreads();
        bitonic(sk, n, m);
        for (int k = threadIdx.x; k < n; k += blockDim.x) list[a + k] = (int)(unsigned)(sk[k] & 0xffffffffull);
    } else {
        bitonic(keys + a, n, m);
        for (int k = threadIdx.x; k < n; k += blockDim.x) list[a + k] = (int)(unsigned)(keys[a + k] & 0xffffffffull);
    }
}

// The surfel's opacity at pixel centre (u, v) from its record planes r0..r2.
// Returns true where it contributes (min(alpha, G) >= alpha_min, hit in
// front of the near plane); alpha, om = 1 - alpha (accurate near alpha = 1),
// G and 1/z come back.
__device__ __forceinline__ bool t_hit(const float4 &r0, const float4 &r1, const float4 &r2, float u, float v,
                                      const CamParams &C, float &iz, float &q)
{
    const float du = u - r0.x, dv = v - r0.y;
    iz = fmaf(r0.w, du, fmaf(r1.x, dv, r0.z));
    const float A = fmaf(r1.y, du, fmaf(r1.z, dv, r1.w));
    const float B = fmaf(r2.x, du, fmaf(r2.y, dv, r2.z));
    q = fmaf(A, A, B * B);
    return iz > 0.f && iz < C.izn && q <= iz * iz;   // inside the 1/255 disc
}
// log w of a surfel, computed once per staged entry (-inf for w <= 0: never drawn)
__device__ __forceinline__ float t_logw(float w) { return w > 0.f ? logf(w) : -INFINITY; }
__device__ __forceinline__ bool t_opacity(float q, float iz, float lw, const OptParams &O, float &alpha, float &om,
                                          float &G)
{
    if (!(lw > -INFINITY)) return false;
    const float rho = O.surfel_r2 * q / (iz * iz);
    const float e = -0.5f * rho;
    G = expf(e);
    const float x = lw + e;                         // w G = exp(x)
    if (x >= 0.f) { alpha = 1.f; om = 0.f; }
    else { om = -expm1f(x); alpha = 1.f - om; }
    return fminf(alpha, G) >= O.alpha_min;
}
__device__ __forceinline__ bool t_alpha(const float4 &r0, const float4 &r1, const float4 &r2, float lw, float u,
                                        float v, const CamParams &C, const OptParams &O, float &alpha, float &om,
                                        float &G, float &iz)
{
    float q;
    return t_hit(r0, r1, r2, u, v, C, iz, q) && t_opacity(q, iz, lw, O, alpha, om, G);
}

__device__ __forceinline__ float shfl_f(float v, int s) { return __shfl_sync(0xffffffffu, v, s); }

template <bool kFront>
__global__ void __launch_bounds__(kRasterThreads, 4)
    k_traster(ViewScratch X, CamParams C, OptParams O, const float *__restrict__ w, float *__restrict__ out_rgb,
              float *__restrict__ out_T, int32_t *__restrict__ out_front, int32_t *__restrict__ out_last,
              float *__restrict__ out_Tlast, int32_t *__restrict__ cover)
{
    __shared__ float4 ss[3][kRasterThreads];
    __shared__ float4 sx[kRasterThreads];        // (r, g, b, w)
    __shared__ int sid[kRasterThreads];
    __shared__ unsigned sbb[2][kRasterThreads];
    __shared__ float sizmax[kRasterThreads];
    __shared__ float slw[kRasterThreads];        // log w
    if (X.status[ST_FLAGS] & FLAG_SOVF) return;
    const int tile = blockIdx.x, tx = tile % C.tiles_x, ty = tile / C.tiles_x;
    const unsigned warp = threadIdx.x >> 5, lane = lane_idx();
    const int wx0 = tx * kTile + (warp & 1) * kWarpW, wy0 = ty * kTile + (warp >> 1) * kWarpH;
    const int wx1 = min(wx0 + kWarpW - 1, C.W - 1), wy1 = min(wy0 + kWarpH - 1, C.H - 1);
    const bool wactive = wx0 < C.W && wy0 < C.H;
    const int px = wx0 + (int)(lane & 7), py = wy0 + (int)(lane >> 3);
    const bool in_img = px < C.W && py < C.H;
    const float u = px + 0.5f, v = py + 0.5f;
    const int s0 = X.s_off[tile], s1 = X.s_off[tile + 1];
    const int t = threadIdx.x;
    auto stage = [&](int base) {
        if (base + t < s1) {
            const int id = X.s_list[base + t];
            const float4 *rp = X.s_rec + 4 * (int64_t)id;
            ss[0][t] = rp[0]; ss[1][t] = rp[1]; ss[2][t] = rp[2];
            const float4 r3 = rp[3];
            sbb[0][t] = __float_as_uint(r3.y); sbb[1][t] = __float_as_uint(r3.z);
            sizmax[t] = r3.x;
            const float4 c = X.s_rgb[id];
            const float wi = w[id];
            sx[t] = make_float4(c.x, c.y, c.z, wi);
            slw[t] = t_logw(wi);
            sid[t] = id;
        }
    };
    auto overlap = [&](int j) {
        const unsigned lo = sbb[0][j], hi = sbb[1][j];
        const int x0 = lo & 0xffff, y0 = lo >> 16, x1 = hi & 0xffff, y1 = hi >> 16;
        return x0 <= wx1 && x1 >= wx0 && y0 <= wy1 && y1 >= wy0;
    };

    // ---- the frontmost contributor (lexicographic min of (depth, index)) ----
    float best = in_img ? 0.f : INFINITY;
    int fid = 0x7fffffff;
    float wmin = 0.f;
    for (int base = s0; base < s1; base += kRasterThreads) {
        __syncthreads();
        stage(base);
        __syncthreads();
        const int n = min(kRasterThreads, s1 - base);
        if (!wactive) continue;
        for (int j0 = 0; j0 < n; j0 += 32) {
            const int j = j0 + (int)lane;
            const bool keep = j < n && overlap(j) && sizmax[j] >= wmin;
            unsigned mask = __ballot_sync(0xffffffffu, keep);
            while (mask) {
                const int jj = j0 + __ffs(mask) - 1;
                mask &= mask - 1;
                // only a hit that would win needs its opacity (the exp and the cut)
                float a, om, G, iz, q;
                if (in_img && t_hit(ss[0][jj], ss[1][jj], ss[2][jj], u, v, C, iz, q)) {
                    const int id = sid[jj];
                    if ((iz > best || (iz == best && id < fid)) && t_opacity(q, iz, slw[jj], O, a, om, G)) {
                        best = iz;
                        fid = id;
                    }
                }
            }
            wmin = __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(best)));
        }
    }
    const bool has_front = fid != 0x7fffffff;

    // ---- blending ----
    float Cr = 0.f, Cg = 0.f, Cb = 0.f, T = 1.f, Tlast = 1.f;
    int last = 0;
    bool done = !in_img;
    if (kFront && has_front && !done) {
        const float4 *rp = X.s_rec + 4 * (int64_t)fid;
        float a, om, G, iz;
        t_alpha(rp[0], rp[1], rp[2], t_logw(w[fid]), u, v, C, O, a, om, G, iz);
        const float4 c = X.s_rgb[fid];
        Cr += c.x * a * T; Cg += c.y * a * T; Cb += c.z * a * T;
        Tlast = T;
        T *= om;
        done = T < kTStop;
    }
    for (int base = s0; base < s1; base += kRasterThreads) {
        // the CTA stops once every pixel of the tile is done
        if (__syncthreads_and(done)) break;
        stage(base);
        __syncthreads();
        const int n = min(kRasterThreads, s1 - base);
        if (!wactive) continue;
        // groups of 32 entries: the lanes test the block overlap of one entry
        // each, then the warp walks the overlapping ones in list order
        for (int j0 = 0; j0 < n; j0 += 32) {
            if (__all_sync(0xffffffffu, done)) break;
            unsigned mask = __ballot_sync(0xffffffffu, j0 + (int)lane < n && overlap(j0 + (int)lane));
            while (mask) {
                if (__all_sync(0xffffffffu, done)) break;
                const int j = j0 + __ffs(mask) - 1;
                mask &= mask - 1;
                if (done) continue;
                const int id = sid[j];
                if (kFront && id == fid) continue;
                float a, om, G, iz;
                if (!t_alpha(ss[0][j], ss[1][j], ss[2][j], slw[j], u, v, C, O, a, om, G, iz)) continue;
                const float4 c = sx[j];
                Cr += c.x * a * T; Cg += c.y * a * T; Cb += c.z * a * T;
                Tlast = T;
                T *= om;
                last = base - s0 + j + 1;
                done = T < kTStop;
            }
        }
    }
    if (!in_img) return;
    const int64_t HW = (int64_t)C.W * C.H, pix = (int64_t)py * C.W + px;
    out_rgb[pix] = Cr + T * C.bg[0];
    out_rgb[HW + pix] = Cg + T * C.bg[1];
    out_rgb[2 * HW + pix] = Cb + T * C.bg[2];
    if (out_T) out_T[pix] = T;
    if (out_front) out_front[pix] = has_front ? fid : -1;
    if (out_last) out_last[pix] = last;
    if (out_Tlast) out_Tlast[pix] = Tlast;
    if (cover && has_front) atomicAdd(cover + fid, 1);
}

// the 18 per-(pixel, surfel) gradient terms: gP(3) gU(3) gV(3) gN(3) gs1 gs2 gw gc(3), camera space
__device__ __forceinline__ void t_terms(const float4 *fr, float a, float G, float wv, float T, float iz,
                                        const float *g, const float *cS, const float *col, float u, float v,
                                        const CamParams &C, float *out)
{
    float dLda = 0.f;
    for (int ch = 0; ch < 3; ++ch) {
        out[15 + ch] = a * T * g[ch];
        dLda += T * (col[ch] - cS[ch]) * g[ch];
    }
    for (int k = 0; k < 15; ++k) out[k] = 0.f;
    if (!(wv * G < 1.f)) return;                    // alpha clamped at 1: no geometry gradient
    out[14] = dLda * G;
    const float dLdrho = dLda * (-0.5f * wv * G);
    const float4 f0 = fr[0], f1 = fr[1], f2 = fr[2], f3 = fr[3];
    const float P[3] = {f0.x, f0.y, f0.z}, U[3] = {f1.x, f1.y, f1.z}, V[3] = {f2.x, f2.y, f2.z};
    const float Nn[3] = {f3.x, f3.y, f3.z}, s1 = f0.w, s2 = f1.w;
    const float d[3] = {(u - C.cx) / C.fx, (v - C.cy) / C.fy, 1.f};
    const float Nd = Nn[0] * d[0] + Nn[1] * d[1] + Nn[2] * d[2];
    const float Ud = U[0] * d[0] + U[1] * d[1] + U[2] * d[2];
    const float Vd = V[0] * d[0] + V[1] * d[1] + V[2] * d[2];
    const float z = 1.f / iz;
    float Xv[3];
    for (int q = 0; q < 3; ++q) Xv[q] = z * d[q] - P[q];
    const float aa = (Xv[0] * U[0] + Xv[1] * U[1] + Xv[2] * U[2]) / s1;
    const float bb = (Xv[0] * V[0] + Xv[1] * V[1] + Xv[2] * V[2]) / s2;
    const float dLa = dLdrho * 2.f * aa, dLb = dLdrho * 2.f * bb;
    for (int q = 0; q < 3; ++q) {
        out[q] = dLa * ((Ud / Nd) * Nn[q] - U[q]) / s1 + dLb * ((Vd / Nd) * Nn[q] - V[q]) / s2;
        out[3 + q] = dLa * Xv[q] / s1;
        out[6 + q] = dLb * Xv[q] / s2;
        out[9 + q] = -(dLa * Ud / s1 + dLb * Vd / s2) * Xv[q] / Nd;
    }
    out[12] = dLa * (-aa / s1);
    out[13] = dLb * (-bb / s2);
}

__device__ __forceinline__ void t_add(long long *acc, int id, const float *terms, float scale)
{
    long long *a = acc + (int64_t)kTAcc * id;
    for (int k = 0; k < kTAcc; ++k) {
        const float x = terms[k] * scale;
        if (x != 0.f) atomicAdd(reinterpret_cast<unsigned long long *>(a + k), (unsigned long long)__float2ll_rn(x));
    }
}

template <bool kFront>
__global__ void __launch_bounds__(kRasterThreads, 3)
    k_tbwd(ViewScratch X, CamParams C, OptParams O, const float *__restrict__ w, const float *__restrict__ dL,
           const float *__restrict__ in_T, const int32_t *__restrict__ in_front, const int32_t *__restrict__ in_last,
           const float *__restrict__ in_Tlast, const unsigned *gmax_bits, long long *acc)
{
    __shared__ float4 ss[3][kRasterThreads];
    __shared__ float4 sx[kRasterThreads];
    __shared__ int sid[kRasterThreads];
    __shared__ unsigned sbb[2][kRasterThreads];
    __shared__ float slw[kRasterThreads];        // log w
    __shared__ int s_maxlast;
    if (X.status[ST_FLAGS] & FLAG_SOVF) return;
    const float gmax = __uint_as_float(*gmax_bits);
    if (!(gmax > 0.f)) return;
    const float scale = 16777216.f / gmax;        // 2^24 / max |dL/dC|
    const int tile = blockIdx.x, tx = tile % C.tiles_x, ty = tile / C.tiles_x;
    const unsigned warp = threadIdx.x >> 5, lane = lane_idx();
    const int wx0 = tx * kTile + (warp & 1) * kWarpW, wy0 = ty * kTile + (warp >> 1) * kWarpH;
    const int wx1 = min(wx0 + kWarpW - 1, C.W - 1), wy1 = min(wy0 + kWarpH - 1, C.H - 1);
    const bool wactive = wx0 < C.W && wy0 < C.H;
    const int px = wx0 + (int)(lane & 7), py = wy0 + (int)(lane >> 3);
    const bool in_img = px < C.W && py < C.H;
    const float u = px + 0.5f, v = py + 0.5f;
    const int s0 = X.s_off[tile], s1 = X.s_off[tile + 1];
    const int t = threadIdx.x;
    const int64_t HW = (int64_t)C.W * C.H, pix = in_img ? (int64_t)py * C.W + px : 0;
    float g[3] = {0.f, 0.f, 0.f}, S[3] = {C.bg[0], C.bg[1], C.bg[2]}, Tc = 0.f, Tl = 1.f;
    int mylast = 0, myfront = -1;
    if (in_img) {
        g[0] = __ldg(dL + pix); g[1] = __ldg(dL + HW + pix); g[2] = __ldg(dL + 2 * HW + pix);
        Tc = __ldg(in_T + pix); Tl = __ldg(in_Tlast + pix);
        mylast = __ldg(in_last + pix); myfront = __ldg(in_front + pix);
    }
    if (t == 0) s_maxlast = 0;
    __syncthreads();
    atomicMax(&s_maxlast, mylast);
    __syncthreads();
    const int nl = s_maxlast;
    bool first_seen = false;    // the last blended entry is the first met going backwards
    for (int cbase = ((nl - 1) / kRasterThreads) * kRasterThreads; nl > 0 && cbase >= 0; cbase -= kRasterThreads) {
        __syncthreads();
        if (s0 + cbase + t < s1 && cbase + t < nl) {
            const int id = X.s_list[s0 + cbase + t];
            const float4 *rp = X.s_rec + 4 * (int64_t)id;
            ss[0][t] = rp[0]; ss[1][t] = rp[1]; ss[2][t] = rp[2];
            const float4 r3 = rp[3];
            sbb[0][t] = __float_as_uint(r3.y); sbb[1][t] = __float_as_uint(r3.z);
            const float4 c = X.s_rgb[id];
            const float wi = w[id];
            sx[t] = make_float4(c.x, c.y, c.z, wi);
            slw[t] = t_logw(wi);
            sid[t] = id;
        }
        __syncthreads();
        if (!wactive) continue;
        const int n = min(kRasterThreads, nl - cbase);
        // groups of 32 entries from the end: the lanes test the block overlap
        // of one entry each, then the warp walks the overlapping ones backwards
        for (int j0 = ((n - 1) >> 5) << 5; j0 >= 0; j0 -= 32) {
            const int jl = j0 + (int)lane;
            bool ov = false;
            if (jl < n) {
                const unsigned lo = sbb[0][jl], hi = sbb[1][jl];
                ov = (lo & 0xffff) <= (unsigned)wx1 && (hi & 0xffff) >= (unsigned)wx0 && (lo >> 16) <= (unsigned)wy1 &&
                     (hi >> 16) >= (unsigned)wy0;
            }
            unsigned mask = __ballot_sync(0xffffffffu, ov);
            while (mask) {
                const int hb = 31 - __clz(mask);
                mask &= ~(1u << hb);
                const int j = j0 + hb;
                const int pos = cbase + j;             // position in the tile list
                const int id = sid[j];
                float terms[kTAcc];
                bool contrib = false;
                float a = 0.f, om = 1.f, G = 0.f, iz = 1.f;
                if (in_img && pos < mylast && !(kFront && id == myfront) &&
                    t_alpha(ss[0][j], ss[1][j], ss[2][j], slw[j], u, v, C, O, a, om, G, iz)) {
                    contrib = true;
                    // T before this contributor: stored for the last one, else T_after / (1 - alpha)
                    const float Ti = !first_seen ? Tl : Tc / om;
                    first_seen = true;
                    const float col[3] = {sx[j].x, sx[j].y, sx[j].z};
                    t_terms(X.s_tside + 4 * (int64_t)id, a, G, sx[j].w, Ti, iz, g, S, col, u, v, C, terms);
                    for (int ch = 0; ch < 3; ++ch) S[ch] = col[ch] * a + om * S[ch];
                    Tc = Ti;
                }
                if (!__any_sync(0xffffffffu, contrib)) continue;
                if (!contrib)
                    for (int k = 0; k < kTAcc; ++k) terms[k] = 0.f;
                // the warp's 18 sums, each added by the lane that ends up holding it
                unsigned long long *ak = reinterpret_cast<unsigned long long *>(acc + (int64_t)kTAcc * id);
                warp_reduce_scatter<kTAcc>(terms, (int)lane, [&](int k, float tot) {
                    const float x = tot * scale;
                    if (x != 0.f) atomicAdd(ak + k, (unsigned long long)__float2ll_rn(x));
                });
            }
        }
    }
    // the frontmost surfel, blended first (T = 1)
    if (kFront && in_img && myfront >= 0) {
        const float4 *rp = X.s_rec + 4 * (int64_t)myfront;
        float a, om, G, iz;
        if (t_alpha(rp[0], rp[1], rp[2], t_logw(w[myfront]), u, v, C, O, a, om, G, iz)) {
            const float4 c = X.s_rgb[myfront];
            const float col[3] = {c.x, c.y, c.z};
            float terms[kTAcc];
            t_terms(X.s_tside + 4 * (int64_t)myfront, a, G, w[myfront], !first_seen ? Tl : 1.f, iz, g, S, col, u, v,
                    C, terms);
            t_add(acc, myfront, terms, scale);
        }
    }
}

// per surfel: fixed point -> float, camera -> world, rotation through the
// quaternion's normalisation, colour -> SH (and position through the view direction)
__global__ void __launch_bounds__(256) k_tfinal(SceneView S, CamParams C, const long long *__restrict__ acc,
                                                const unsigned *gmax_bits, float *g_pos, float *g_rot,
                                                float *g_scale, float *g_w, float *g_sh)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.N) return;
    const float gm = __uint_as_float(*gmax_bits);
    const float inv = gm > 0.f ? gm / 16777216.f : 0.f;
    float A[kTAcc];
    for (int k = 0; k < kTAcc; ++k) A[k] = (float)acc[(int64_t)kTAcc * i + k] * inv;
    const int K = (S.deg + 1) * (S.deg + 1);
    bool any = false;
    for (int k = 0; k < kTAcc; ++k) any |= A[k] != 0.f;
    if (!any) {
        // no pixel sent a gradient: zeros, without reading the SH row
        if (g_pos) for (int a = 0; a < 3; ++a) g_pos[3 * i + a] = 0.f;
        if (g_scale) { g_scale[2 * i] = 0.f; g_scale[2 * i + 1] = 0.f; }
        if (g_w) g_w[i] = 0.f;
        if (g_rot) for (int a = 0; a < 4; ++a) g_rot[4 * i + a] = 0.f;
        if (g_sh) store_zeros(g_sh + 3 * K * i, 3 * K);
        return;
    }
    float q[4], R[9], qn[4], qnorm;
    for (int k = 0; k < 4; ++k) q[k] = load_attr(S.s_rot, 4 * i + k, S.attr_dtype);
    const bool okq = quat_to_rot(q[0], q[1], q[2], q[3], R, qn, &qnorm);
    float gp[3];
    for (int a = 0; a < 3; ++a) gp[a] = C.R[a] * A[0] + C.R[3 + a] * A[1] + C.R[6 + a] * A[2];
    if (g_scale) { g_scale[2 * i] = A[12]; g_scale[2 * i + 1] = A[13]; }
    if (g_w) g_w[i] = A[14];
    // colour -> SH coefficients and position (through the view direction)
    float dir[3], dist;
    view_dir(C, __ldg(S.s_pos + 3 * i), __ldg(S.s_pos + 3 * i + 1), __ldg(S.s_pos + 3 * i + 2), dir, dist);
    float Y[16];
    sh_basis(K, dir[0], dir[1], dir[2], Y);
    float rgb[3], raw[3];
    sh_colour(S.s_sh, i, K, S.sh_dtype, Y, rgb, raw);
    float gc[3];
    for (int c = 0; c < 3; ++c) gc[c] = raw[c] > 0.f ? A[15 + c] : 0.f;
    float gd[3] = {0.f, 0.f, 0.f};
    switch (K) {
    case 16: sh_weighted_grad<16>(S.s_sh, i, S.sh_dtype, gc, dir, gd); break;
    case 9: sh_weighted_grad<9>(S.s_sh, i, S.sh_dtype, gc, dir, gd); break;
    case 4: sh_weighted_grad<4>(S.s_sh, i, S.sh_dtype, gc, dir, gd); break;
    default: break;   // degree 0: the colour does not depend on the direction
    }
    if (g_sh) store_sh_grad(g_sh + 3 * K * i, K, Y, gc, nullptr);
    if (dist > 0.f) {
        const float pr = gd[0] * dir[0] + gd[1] * dir[1] + gd[2] * dir[2];
        for (int a = 0; a < 3; ++a) gp[a] -= (gd[a] - pr * dir[a]) / dist;
    }
    if (g_pos) for (int a = 0; a < 3; ++a) g_pos[3 * i + a] = gp[a];
    if (!g_rot) return;
    if (!okq) { for (int a = 0; a < 4; ++a) g_rot[4 * i + a] = 0.f; return; }
    // dL/dR[:,k] = Rc^T g_{U,V,N}
    float GR[3][3];
    for (int a = 0; a < 3; ++a) {
        GR[a][0] = C.R[a] * A[3] + C.R[3 + a] * A[4] + C.R[6 + a] * A[5];
        GR[a][1] = C.R[a] * A[6] + C.R[3 + a] * A[7] + C.R[6 + a] * A[8];
        GR[a][2] = C.R[a] * A[9] + C.R[3 + a] * A[10] + C.R[6 + a] * A[11];
    }
    const float wq = qn[0], qx = qn[1], qy = qn[2], qz = qn[3];
    float gq[4];
    gq[0] = 2.f * (-qz * GR[0][1] + qy * GR[0][2] + qz * GR[1][0] - qx * GR[1][2] - qy * GR[2][0] + qx * GR[2][1]);
    gq[1] = 2.f * (qy * GR[0][1] + qz * GR[0][2] + qy * GR[1][0] - 2.f * qx * GR[1][1] - wq * GR[1][2] +
                   qz * GR[2][0] + wq * GR[2][1] - 2.f * qx * GR[2][2]);
    gq[2] = 2.f * (-2.f * qy * GR[0][0] + qx * GR[0][1] + wq * GR[0][2] + qx * GR[1][0] + qz * GR[1][2] -
                   wq * GR[2][0] + qz * GR[2][1] - 2.f * qy * GR[2][2]);
    gq[3] = 2.f * (-2.f * qz * GR[0][0] - wq * GR[0][1] + qx * GR[0][2] + wq * GR[1][0] - 2.f * qz * GR[1][1] +
                   qy * GR[1][2] + qx * GR[2][0] + qy * GR[2][1]);
    const float pr = gq[0] * wq + gq[1] * qx + gq[2] * qy + gq[3] * qz;
    for (int a = 0; a < 4; ++a) g_rot[4 * i + a] = (gq[a] - pr * qn[a]) / qnorm;
}

// Contribution score (Eq. 9): per Gaussian, the warp sweeps its pixels; the
// max of c_max alpha / (1 + W_G) where it passes the clamp and the depth test.
__global__ void __launch_bounds__(256) k_contrib(SceneView S, CamParams C, OptParams O,
                                                 const float *__restrict__ depth, const float *__restrict__ aux,
                                                 float *__restrict__ score)
{
    const int64_t gi = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int lane = threadIdx.x & 31;
    GaussOut o;
    o.visible = false;
    if (gi < S.M) {
        if (S.gdim == 2) gauss2d_setup(S, C, O, gi, o);
        else gauss_setup(S, C, O, gi, o);
    }
    const bool vis = gi < S.M && o.visible;
    float res = 0.f;
    unsigned big = __ballot_sync(0xffffffffu, vis);
    const int64_t W = C.W;
    while (big) {
        const int j = __ffs(big) - 1;
        big &= big - 1;
        const int x0 = __shfl_sync(0xffffffffu, o.x0, j), x1 = __shfl_sync(0xffffffffu, o.x1, j);
        const int y0 = __shfl_sync(0xffffffffu, o.y0, j), y1 = __shfl_sync(0xffffffffu, o.y1, j);
        const int bw = x1 - x0 + 1, n = bw * (y1 - y0 + 1);
        float m = 0.f;
        if (S.gdim == 2) {
            float4 r[4], x0a, x1a;
            const float4 *src = reinterpret_cast<const float4 *>(&o.drec);
            for (int k = 0; k < 4; ++k) {
                r[k].x = shfl_f(src[k].x, j); r[k].y = shfl_f(src[k].y, j);
                r[k].z = shfl_f(src[k].z, j); r[k].w = shfl_f(src[k].w, j);
            }
            x0a = make_float4(shfl_f(o.aux[0].x, j), shfl_f(o.aux[0].y, j), shfl_f(o.aux[0].z, j), shfl_f(o.aux[0].w, j));
            x1a = make_float4(shfl_f(o.aux[1].x, j), shfl_f(o.aux[1].y, j), shfl_f(o.aux[1].z, j), shfl_f(o.aux[1].w, j));
            // the colour as a float (the side word carries it in 2^-16 units)
            const float cm = fminf(fmaxf(shfl_f(o.rgb[0], j), fmaxf(shfl_f(o.rgb[1], j), shfl_f(o.rgb[2], j))),
                                   kColourMax);
            const float ibw = 1.f / (float)bw;
            for (int k = lane; k < n; k += 32) {
                const int rk = bbox_row(k, bw, ibw);
                const int xx = x0 + (k - rk * bw), yy = y0 + rk;
                const float du = xx + 0.5f - r[0].x, dv = yy + 0.5f - r[0].y;
                const float iz = fmaf(r[0].w, du, fmaf(r[1].x, dv, r[0].z));
                const float A = fmaf(r[1].y, du, fmaf(r[1].z, dv, r[1].w));
                const float B = fmaf(r[2].x, du, fmaf(r[2].y, dv, r[2].z));
                const float z = __frcp_rn(iz);
                const float a = ex2_approx(fmaf(x1a.w, fmaf(A, A, B * B) * (z * z), x0a.w));
                const int64_t p = (int64_t)yy * W + xx;
                if (iz > 0.f && iz < C.izn && a >= O.alpha_min && z - r[3].w < __ldg(depth + p))
                    m = fmaxf(m, cm * a / (1.f + __ldg(aux + p)));
            }
        } else {
            GaussRec g;
            g.px = shfl_f(o.rec.px, j); g.py = shfl_f(o.rec.py, j); g.pxl = shfl_f(o.rec.pxl, j);
            g.pyl = shfl_f(o.rec.pyl, j); g.la = shfl_f(o.rec.la, j); g.lb = shfl_f(o.rec.lb, j);
            g.lc = shfl_f(o.rec.lc, j); g.sigma = shfl_f(o.rec.sigma, j); g.key = shfl_f(o.rec.key, j);
            const float cm = fmaxf(shfl_f(o.rec.r, j), fmaxf(shfl_f(o.rec.g, j), shfl_f(o.rec.b, j)));
            const float ibw = 1.f / (float)bw;
            for (int k = lane; k < n; k += 32) {
                const int rk = bbox_row(k, bw, ibw);
                const int xx = x0 + (k - rk * bw), yy = y0 + rk;
                float e;
                const float a = gauss_alpha(g, xx + 0.5f, yy + 0.5f, e);
                const int64_t p = (int64_t)yy * W + xx;
                if (a >= O.alpha_min && g.key < __ldg(depth + p)) m = fmaxf(m, cm * a / (1.f + __ldg(aux + p)));
            }
        }
        for (int d = 16; d >= 1; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
        if (lane == j) res = m;
    }
    if (gi < S.M) score[gi] = res;
}

}  // namespace

cudaError_t launch_translucent(const SceneView &S, const CamParams &C, const OptParams &O, const ViewScratch &X,
                               const float *w, bool front_first, unsigned long long *keys, float *out_rgb,
                               float *out_T, int32_t *out_front, int32_t *out_last, float *out_Tlast, int32_t *cover,
                               cudaStream_t st)
{
    OptParams Os = O;
    Os.mode = GES_MODE_SURFELS_ONLY;
    cudaError_t e = launch_binning(S, C, Os, X, st, nullptr);
    if (e != cudaSuccess) return e;
    const int T = C.tiles_x * C.tiles_y;
    k_tkeys<<<152 * 8, 256, 0, st>>>(X.s_list, X.s_off + T, X.s_tside, keys, X.status);
    k_tsort<<<T, 256, 0, st>>>(X.s_off, keys, X.s_list, X.status);
    if (front_first) k_traster<true><<<T, kRasterThreads, 0, st>>>(X, C, Os, w, out_rgb, out_T, out_front, out_last, out_Tlast, cover);
    else k_traster<false><<<T, kRasterThreads, 0, st>>>(X, C, Os, w, out_rgb, out_T, out_front, out_last, out_Tlast, cover);
    return cudaGetLastError();
}

cudaError_t launch_translucent_backward(const SceneView &S, const CamParams &C, const OptParams &O,
                                        const ViewScratch &X, const float *w, bool front_first,
                                        unsigned long long *keys, const float *dL, const float *in_T,
                                        const int32_t *in_front, const int32_t *in_last, const float *in_Tlast,
                                        long long *acc, unsigned *gmax, float *g_pos, float *g_rot, float *g_scale,
                                        float *g_w, float *g_sh, cudaStream_t st)
{
    OptParams Os = O;
    Os.mode = GES_MODE_SURFELS_ONLY;
    // the same binning and order as the forward pass (both are deterministic)
    cudaError_t e = launch_binning(S, C, Os, X, st, nullptr);
    if (e != cudaSuccess) return e;
    const int T = C.tiles_x * C.tiles_y;
    k_tkeys<<<152 * 8, 256, 0, st>>>(X.s_list, X.s_off + T, X.s_tside, keys, X.status);
    k_tsort<<<T, 256, 0, st>>>(X.s_off, keys, X.s_list, X.status);
    if ((e = cudaMemsetAsync(acc, 0, sizeof(long long) * kTAcc * (size_t)(S.N > 0 ? S.N : 1), st)) != cudaSuccess)
        return e;
    if ((e = launch_absmax(dL, 3 * (int64_t)C.W * C.H, gmax, st)) != cudaSuccess) return e;
    if (front_first) k_tbwd<true><<<T, kRasterThreads, 0, st>>>(X, C, Os, w, dL, in_T, in_front, in_last, in_Tlast, gmax, acc);
    else k_tbwd<false><<<T, kRasterThreads, 0, st>>>(X, C, Os, w, dL, in_T, in_front, in_last, in_Tlast, gmax, acc);
    if (S.N > 0)
        k_tfinal<<<(unsigned)((S.N + 255) / 256), 256, 0, st>>>(S, C, acc, gmax, g_pos, g_rot, g_scale, g_w, g_sh);
    return cudaGetLastError();
}

cudaError_t launch_contribution(const SceneView &S, const CamParams &C, const OptParams &O, const float *depth,
                                const float *aux, float *score, cudaStream_t st)
{
    if (S.M == 0) return cudaSuccess;
    k_contrib<<<(unsigned)((S.M + 255) / 256), 256, 0, st>>>(S, C, O, depth, aux, score);
    return cudaGetLastError();
}

}  // namespace ges
