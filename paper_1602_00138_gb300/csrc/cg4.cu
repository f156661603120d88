// Float32 inner iteration of the batched deflated CG (see cg.cu for the
// recurrences) for grids with Nx % 4 == 0, restructured for HBM bandwidth:
//
//   k_stencil4   q = A~_s p, float4 along x, one active lane per CTA row,
//                fused p^T q
//   k_update4    x += alpha p, r -= alpha q, fused r^T r and the private
//                (A W)^T r dots, float4, one active lane per CTA row
//   k_u0dots     (A~_s U_0)^T r for a tile of <= 32 lanes of one sample:
//                a shared-memory tiled product, so each A~_s U_0 element is
//                read once per tile instead of once per lane
//   k_mu         per lane (one warp): convergence / breakdown decision,
//                beta, mu = (W^T A W)^-1 (A W)^T r, ring-slot zeroing
//   k_direction4 p = r + beta p - U_0 mu_u - W_p mu_p for a tile of lanes;
//                the thread keeps its U_0 values in registers across the
//                tile's lanes
//
// Lanes are addressed through the active list `alist` (rebuilt by the host
// at every synchronisation) so converged lanes cost no work; tiles group up
// to 32 active lanes of one sample slot.
#include "common.cuh"

namespace rcg {
namespace {

constexpr int kThreads = 256;
constexpr int TILE = 32;       // lanes per tile
constexpr int BK = 64;         // nodes per shared-memory stage of k_u0dots

__device__ __forceinline__ float dot4(const float4 a, const float4 b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

template <int NV>
__device__ __forceinline__ void block_sum(const float (&acc)[NV], double (&res)[NV]) {
    __shared__ double red[kThreads / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double s = (double)acc[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp][v] = s;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < NV; v += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w][v];
        res[v] = s;
    }
    __syncthreads();
}

// q = A~ p for lane c = alist[blockIdx.y]; 4 consecutive x nodes per thread.
__global__ void __launch_bounds__(kThreads)
k_stencil4(Grid g, const float *__restrict__ D, const float *const *__restrict__ diag_of_col,
           const float *const *__restrict__ src, float *const *__restrict__ dst, const int *__restrict__ alist,
           const int *__restrict__ active, double *__restrict__ dots, unsigned long long *__restrict__ prof) {
    const int c = alist[blockIdx.y];
    if (active[c] == 0) return;
    if (prof && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(prof, 1ULL);
    const float *__restrict__ x = src[c];
    float *__restrict__ y = dst[c];
    const float *__restrict__ dg = diag_of_col[c];
    const float4 *__restrict__ x4 = (const float4 *)x;
    const float4 *__restrict__ D4 = (const float4 *)D;
    const int nx4 = g.Nx >> 2, sxy = g.Nx * g.Ny, sxy4 = sxy >> 2, nv = (int)(g.n >> 2);
    const bool has_y = g.Ny > 1;
    float acc = 0.f;
    auto node4 = [&](int v) {
        const int p0 = v << 2;
        const int i0 = p0 % g.Nx;
        const int rest = p0 / g.Nx;
        const int j = rest % g.Ny;
        const int k = rest / g.Ny;
        const float4 xc = x4[v], Dc = D4[v], dc = ((const float4 *)dg)[v];
        float4 o = make_float4(dc.x * xc.x, dc.y * xc.y, dc.z * xc.z, dc.w * xc.w);
        // x neighbours inside the row
        const float xl = i0 > 0 ? x[p0 - 1] : 0.f, Dl = i0 > 0 ? D[p0 - 1] : 0.f;
        const float xr = i0 + 4 < g.Nx ? x[p0 + 4] : 0.f, Dr = i0 + 4 < g.Nx ? D[p0 + 4] : 0.f;
        o.x -= (i0 > 0 ? 0.5f * (Dc.x + Dl) * xl : 0.f) + 0.5f * (Dc.x + Dc.y) * xc.y;
        o.y -= 0.5f * (Dc.y + Dc.x) * xc.x + 0.5f * (Dc.y + Dc.z) * xc.z;
        o.z -= 0.5f * (Dc.z + Dc.y) * xc.y + 0.5f * (Dc.z + Dc.w) * xc.w;
        o.w -= 0.5f * (Dc.w + Dc.z) * xc.z + (i0 + 4 < g.Nx ? 0.5f * (Dc.w + Dr) * xr : 0.f);
#define RCG_NB4(cond, off)                                                                     \
        if (cond) {                                                                            \
            const float4 xn = x4[v + (off)], Dn = D4[v + (off)];                               \
            o.x -= 0.5f * (Dc.x + Dn.x) * xn.x; o.y -= 0.5f * (Dc.y + Dn.y) * xn.y;           \
            o.z -= 0.5f * (Dc.z + Dn.z) * xn.z; o.w -= 0.5f * (Dc.w + Dn.w) * xn.w;           \
        }
        RCG_NB4(has_y && j > 0, -nx4)
        RCG_NB4(has_y && j < g.Ny - 1, nx4)
        RCG_NB4(k > 0, -sxy4)
        RCG_NB4(k < g.Nz - 1, sxy4)
#undef RCG_NB4
        ((float4 *)y)[v] = o;
        acc += dot4(xc, o);
    };
    const int stride = gridDim.x * blockDim.x;
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    for (; v + stride < nv; v += 2 * stride) {
        node4(v);
        node4(v + stride);
    }
    if (v < nv) node4(v);
    double s = (double)acc;
    __shared__ double red[kThreads / 32];
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) s += __shfl_down_sync(0xffffffffu, s, o2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) t += red[w];
        atomicAdd(dots + c, t);
    }
}

// Lane l = alist[blockIdx.y]: x += alpha p; r -= alpha q; r^T r and the
// private (A W)^T r dots (the shared ones come from k_u0dots).
__global__ void __launch_bounds__(kThreads)
k_update4(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ alist, int sprev, int scur, int spq,
          int sw) {
    const int l = alist[blockIdx.y];
    if (ls.active[l] == 0) return;
    const double pq = ls.pq[spq * ls.m + l];
    const double rrp = ls.rr[sprev * ls.m + l];
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rrp)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) ls.flag[l] = 2;
        return;
    }
    const float alpha = (float)(rrp / pq);
    const int ku = gm.k_u, kp = gm.kp[l];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ls.pq[(1 - spq) * ls.m + l] = 0.0;
        if (ls.prof) { atomicAdd(ls.prof + 1, 1ULL); atomicAdd(ls.prof + 2, (unsigned long long)(ku + kp)); }
    }
    constexpr int NV = 1 + KP_MAX;
    float acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.f;
    const long long o = (long long)l * gm.ld;
    float4 *__restrict__ X = (float4 *)((float *)gm.x + o);
    float4 *__restrict__ R = (float4 *)((float *)gm.r + o);
    const float4 *__restrict__ P = (const float4 *)((const float *)gm.p + o);
    const float4 *__restrict__ Q = (const float4 *)((const float *)gm.q + o);
    const float *__restrict__ AP = (const float *)gm.awp + (long long)l * gm.kp_max * gm.ld;
    const int nv = (int)(n >> 2);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        const float4 pv = P[v], qv = Q[v], xv = X[v], rv0 = R[v];
        const float4 rv = make_float4(rv0.x - alpha * qv.x, rv0.y - alpha * qv.y, rv0.z - alpha * qv.z,
                                      rv0.w - alpha * qv.w);
        X[v] = make_float4(xv.x + alpha * pv.x, xv.y + alpha * pv.y, xv.z + alpha * pv.z, xv.w + alpha * pv.w);
        R[v] = rv;
        acc[0] += dot4(rv, rv);
#pragma unroll
        for (int c = 0; c < KP_MAX; ++c)
            if (c < kp) acc[1 + c] += dot4(((const float4 *)(AP + (long long)c * gm.ld))[v], rv);
    }
    __shared__ double out[NV];
    block_sum<NV>(acc, out);
    if (threadIdx.x == 0) atomicAdd(ls.rr + scur * ls.m + l, out[0]);
    if (threadIdx.x >= 1 && threadIdx.x <= kp)
        atomicAdd(ls.wv + ((long long)sw * ls.m + l) * KMAX + ku + (threadIdx.x - 1), out[threadIdx.x]);
}

// wv[sw][l][c] += (A~_s U_0)_c^T r_l for the lanes of tile blockIdx.y (one
// sample slot) over this CTA's node range.  The range is walked in stages of
// SN nodes: the stage of A~_s U_0 (k_u x SN) is staged in shared memory once
// and used by all lanes of the tile; warp w streams lanes w, w+8, w+16, w+24
// with coalesced float4 loads (one float4 of r per thread per lane).
constexpr int SN = 128;
template <int KUT>
__global__ void __launch_bounds__(kThreads)
k_u0dots(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ tile_lane, const int *__restrict__ tile_si,
         const int *__restrict__ tile_cnt, int sw, long long chunk, int use_w) {
    __shared__ float4 As[KUT][SN / 4];
    __shared__ int lanes[TILE];
    const int t = blockIdx.y;
    const int cnt = tile_cnt[t], ku = gm.k_u;
    if (threadIdx.x < TILE) lanes[threadIdx.x] = threadIdx.x < cnt ? tile_lane[t * TILE + threadIdx.x] : -1;
    // use_w: W = U_0 itself (the shared basis columns), else A~_s U_0 of the tile's sample
    const float *__restrict__ AU =
        use_w ? (const float *)gm.wu : (const float *)gm.awu + (long long)tile_si[t] * ku * gm.ld;
    const float *__restrict__ Rb = (const float *)gm.r;
    const int warp = threadIdx.x >> 5, tl = threadIdx.x & 31;
    float acc[4][KUT];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < KUT; ++c) acc[q][c] = 0.f;
    const long long r0 = (long long)blockIdx.x * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    __syncthreads();
    int lq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) lq[q] = lanes[warp + 8 * q];
    for (long long base = r0; base < r1; base += SN) {
        // stage A~_s U_0 (r0 and chunk are multiples of SN; n is a multiple of 4)
        for (int e = threadIdx.x; e < KUT * (SN / 4); e += blockDim.x) {
            const int c = e / (SN / 4), v4 = e % (SN / 4);
            const long long p = base + 4 * v4;
            As[c][v4] = (c < ku && p < r1) ? *(const float4 *)(AU + (long long)c * gm.ld + p) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const long long p = base + 4 * tl;
        if (p < r1) {
            float4 rv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                rv[q] = lq[q] >= 0 ? *(const float4 *)(Rb + (long long)lq[q] * gm.ld + p) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int c = 0; c < KUT; ++c) {
                const float4 a = As[c][tl];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q][c] += dot4(a, rv[q]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int c = 0; c < KUT; ++c) {
            float v = acc[q][c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (tl == 0 && lq[q] >= 0 && c < ku)
                atomicAdd(ls.wv + ((long long)sw * ls.m + lq[q]) * KMAX + c, (double)v);
        }
    }
}

// One warp per lane l = alist[blockIdx.x]: decision, beta, mu (float), slot zeroing.
__global__ void __launch_bounds__(32)
k_mu(LaneState ls, const int *__restrict__ alist, int sprev, int scur, int snext, int sw, float *__restrict__ mu,
     float *__restrict__ beta, int restart) {
    const int l = alist[blockIdx.x];
    if (ls.active[l] == 0) return;
    const double rc = ls.rr[scur * ls.m + l];
    const bool broke = (ls.flag[l] == 2) || !isfinite(rc);
    const bool conv = !broke && sqrt(rc) <= ls.thresh[l];
    __syncwarp();
    if (threadIdx.x == 0) {
        if (!restart) ls.iters[l] += 1;
        if (broke) { ls.active[l] = 0; ls.flag[l] = 2; }
        else if (conv) { ls.active[l] = 0; ls.flag[l] = 1; }
        ls.rr[snext * ls.m + l] = 0.0;
        if (ls.prof && !restart && !broke && !conv) { atomicAdd(ls.prof + 3, 1ULL); atomicAdd(ls.prof + 4, (unsigned long long)ls.kdef[l]); }
    }
    if (broke || conv) {
        for (int c = threadIdx.x; c < KMAX; c += 32) ls.wv[((long long)(1 - sw) * ls.m + l) * KMAX + c] = 0.0;
        return;
    }
    const int k = ls.kdef[l];
    const double *G = ls.gw + (long long)l * KMAX * KMAX;
    const double *w = ls.wv + ((long long)sw * ls.m + l) * KMAX;
    for (int i = threadIdx.x; i < k; i += 32) {
        double s = 0.0;
        for (int jj = 0; jj < k; ++jj) s += G[i + jj * KMAX] * w[jj];
        mu[(long long)l * KMAX + i] = (float)s;
    }
    if (threadIdx.x == 0) beta[l] = restart ? 0.f : (float)(rc / ls.rr[sprev * ls.m + l]);
    __syncwarp();
    for (int c = threadIdx.x; c < KMAX; c += 32) ls.wv[((long long)(1 - sw) * ls.m + l) * KMAX + c] = 0.0;
}

// p = r + beta p - U_0 mu_u - W_p mu_p for the active lanes of tile
// blockIdx.y over this CTA's node range; U_0 is staged per stage of SN nodes
// in shared memory and shared by the tile's lanes (warp w: lanes w + 8q).
template <int KUT>
__global__ void __launch_bounds__(kThreads)
k_direction4(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ tile_lane,
             const int *__restrict__ tile_cnt, const float *__restrict__ mu, const float *__restrict__ beta,
             long long chunk) {
    __shared__ float4 Us[KUT][SN / 4];
    __shared__ float smu[TILE][KU_MAX + KP_MAX];
    __shared__ float sbeta[TILE];
    __shared__ int slane[TILE], skp[TILE];
    const int t = blockIdx.y, cnt = tile_cnt[t], ku = gm.k_u;
    if (threadIdx.x < TILE) {
        int l = threadIdx.x < cnt ? tile_lane[t * TILE + threadIdx.x] : -1;
        if (l >= 0 && ls.active[l] == 0) l = -1;
        slane[threadIdx.x] = l;
        skp[threadIdx.x] = l >= 0 ? gm.kp[l] : 0;
        sbeta[threadIdx.x] = l >= 0 ? beta[l] : 0.f;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TILE * (KU_MAX + KP_MAX); e += blockDim.x) {
        const int jj = e / (KU_MAX + KP_MAX), c = e % (KU_MAX + KP_MAX);
        const int l = slane[jj];
        smu[jj][c] = (l >= 0 && c < ku + skp[jj]) ? mu[(long long)l * KMAX + c] : 0.f;
    }
    const int warp = threadIdx.x >> 5, tl = threadIdx.x & 31;
    const float *__restrict__ WU = (const float *)gm.wu;
    const long long r0 = (long long)blockIdx.x * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    __syncthreads();
    for (long long base = r0; base < r1; base += SN) {
        for (int e = threadIdx.x; e < KUT * (SN / 4); e += blockDim.x) {
            const int c = e / (SN / 4), v4 = e % (SN / 4);
            const long long p = base + 4 * v4;
            Us[c][v4] = (c < ku && p < r1) ? *(const float4 *)(WU + (long long)c * gm.ld + p) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const long long p = base + 4 * tl;
        if (p < r1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int jj = warp + 8 * q;
                const int l = slane[jj];
                if (l < 0) continue;
                const long long o = (long long)l * gm.ld + p;
                const float4 rv = *(const float4 *)((const float *)gm.r + o);
                const float4 pv = *(const float4 *)((const float *)gm.p + o);
                const float b = sbeta[jj];
                float4 sres = make_float4(rv.x + b * pv.x, rv.y + b * pv.y, rv.z + b * pv.z, rv.w + b * pv.w);
#pragma unroll
                for (int c = 0; c < KUT; ++c) {
                    const float m = c < ku ? smu[jj][c] : 0.f;
                    const float4 u = Us[c][tl];
                    sres.x -= m * u.x; sres.y -= m * u.y; sres.z -= m * u.z; sres.w -= m * u.w;
                }
                const int kp = skp[jj];
                const float *WP = (const float *)gm.wp + (long long)l * gm.kp_max * gm.ld;
                for (int c = 0; c < kp; ++c) {
                    const float m = smu[jj][ku + c];
                    const float4 w = *(const float4 *)(WP + (long long)c * gm.ld + p);
                    sres.x -= m * w.x; sres.y -= m * w.y; sres.z -= m * w.z; sres.w -= m * w.w;
                }
                *(float4 *)((float *)gm.p + o) = sres;
            }
        }
        __syncthreads();
    }
}

// Lane l = alist[blockIdx.y]: wv[sw][k_u + c] += (src_c)^T r over the lane's
// private columns (src = W or A W) and optionally rr[srr] += r^T r.
__global__ void __launch_bounds__(kThreads)
k_private_dots4(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ alist, int use_aw, int sw,
                int with_rr, int srr) {
    const int l = alist[blockIdx.y];
    const int ku = gm.k_u, kp = gm.kp[l];
    if (kp == 0 && !with_rr) return;
    constexpr int NV = 1 + KP_MAX;
    float acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.f;
    const float4 *__restrict__ R = (const float4 *)((const float *)gm.r + (long long)l * gm.ld);
    const float *__restrict__ S = (const float *)(use_aw ? gm.awp : gm.wp) + (long long)l * gm.kp_max * gm.ld;
    const int nv = (int)(n >> 2);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
        const float4 rv = R[v];
        acc[0] += dot4(rv, rv);
#pragma unroll
        for (int c = 0; c < KP_MAX; ++c)
            if (c < kp) acc[1 + c] += dot4(((const float4 *)(S + (long long)c * gm.ld))[v], rv);
    }
    __shared__ double out[NV];
    block_sum<NV>(acc, out);
    if (threadIdx.x == 0 && with_rr) atomicAdd(ls.rr + srr * ls.m + l, out[0]);
    if (threadIdx.x >= 1 && threadIdx.x <= kp)
        atomicAdd(ls.wv + ((long long)sw * ls.m + l) * KMAX + ku + (threadIdx.x - 1), out[threadIdx.x]);
}

// One warp per lane l = alist[blockIdx.x]: mu = Ginv * wv[sw] (float), no decision.
__global__ void __launch_bounds__(32)
k_mu_only(LaneState ls, const int *__restrict__ alist, int sw, float *__restrict__ mu) {
    const int l = alist[blockIdx.x];
    const int k = ls.kdef[l];
    const double *G = ls.gw + (long long)l * KMAX * KMAX;
    const double *w = ls.wv + ((long long)sw * ls.m + l) * KMAX;
    for (int i = threadIdx.x; i < k; i += 32) {
        double s = 0.0;
        for (int jj = 0; jj < k; ++jj) s += G[i + jj * KMAX] * w[jj];
        mu[(long long)l * KMAX + i] = (float)s;
    }
}

// Restart projection of the lanes of tile blockIdx.y (one sample slot):
// x = U_0 mu_u + W_p mu_p;  r -= A~_s U_0 mu_u + A~_s W_p mu_p.
template <int KUT>
__global__ void __launch_bounds__(kThreads)
k_project4(long long n, LaneGeom gm, const int *__restrict__ tile_lane, const int *__restrict__ tile_si,
           const int *__restrict__ tile_cnt, const float *__restrict__ mu, long long chunk) {
    __shared__ float4 Us[KUT][SN / 4], As_[KUT][SN / 4];
    __shared__ float smu[TILE][KU_MAX + KP_MAX];
    __shared__ int slane[TILE], skp[TILE];
    const int t = blockIdx.y, cnt = tile_cnt[t], ku = gm.k_u;
    if (threadIdx.x < TILE) {
        const int l = threadIdx.x < cnt ? tile_lane[t * TILE + threadIdx.x] : -1;
        slane[threadIdx.x] = l;
        skp[threadIdx.x] = l >= 0 ? gm.kp[l] : 0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TILE * (KU_MAX + KP_MAX); e += blockDim.x) {
        const int jj = e / (KU_MAX + KP_MAX), c = e % (KU_MAX + KP_MAX);
        const int l = slane[jj];
        smu[jj][c] = (l >= 0 && c < ku + skp[jj]) ? mu[(long long)l * KMAX + c] : 0.f;
    }
    const float *__restrict__ WU = (const float *)gm.wu;
    const float *__restrict__ AU = (const float *)gm.awu + (long long)tile_si[t] * ku * gm.ld;
    const int warp = threadIdx.x >> 5, tl = threadIdx.x & 31;
    const long long r0 = (long long)blockIdx.x * chunk;
    const long long r1 = r0 + chunk < n ? r0 + chunk : n;
    __syncthreads();
    for (long long base = r0; base < r1; base += SN) {
        for (int e = threadIdx.x; e < KUT * (SN / 4); e += blockDim.x) {
            const int c = e / (SN / 4), v4 = e % (SN / 4);
            const long long p = base + 4 * v4;
            const bool ok = c < ku && p < r1;
            Us[c][v4] = ok ? *(const float4 *)(WU + (long long)c * gm.ld + p) : make_float4(0.f, 0.f, 0.f, 0.f);
            As_[c][v4] = ok ? *(const float4 *)(AU + (long long)c * gm.ld + p) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const long long p = base + 4 * tl;
        if (p < r1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int jj = warp + 8 * q;
                const int l = slane[jj];
                if (l < 0) continue;
                float4 xs = make_float4(0.f, 0.f, 0.f, 0.f), rs = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int c = 0; c < KUT; ++c) {
                    const float m = c < ku ? smu[jj][c] : 0.f;
                    const float4 u = Us[c][tl], a = As_[c][tl];
                    xs.x += m * u.x; xs.y += m * u.y; xs.z += m * u.z; xs.w += m * u.w;
                    rs.x += m * a.x; rs.y += m * a.y; rs.z += m * a.z; rs.w += m * a.w;
                }
                const int kp = skp[jj];
                const float *WP = (const float *)gm.wp + (long long)l * gm.kp_max * gm.ld;
                const float *AP = (const float *)gm.awp + (long long)l * gm.kp_max * gm.ld;
                for (int c = 0; c < kp; ++c) {
                    const float m = smu[jj][ku + c];
                    const float4 w = *(const float4 *)(WP + (long long)c * gm.ld + p);
                    const float4 a = *(const float4 *)(AP + (long long)c * gm.ld + p);
                    xs.x += m * w.x; xs.y += m * w.y; xs.z += m * w.z; xs.w += m * w.w;
                    rs.x += m * a.x; rs.y += m * a.y; rs.z += m * a.z; rs.w += m * a.w;
                }
                const long long o = (long long)l * gm.ld + p;
                *(float4 *)((float *)gm.x + o) = xs;
                float4 rv = *(const float4 *)((const float *)gm.r + o);
                rv.x -= rs.x; rv.y -= rs.y; rv.z -= rs.z; rv.w -= rs.w;
                *(float4 *)((float *)gm.r + o) = rv;
            }
        }
        __syncthreads();
    }
}

int gx_for(long long nv, int rows, int per_sm) {
    long long want = ((long long)per_sm * 152 + rows - 1) / rows;
    long long maxb = (nv + kThreads - 1) / kThreads;
    long long gx = want < maxb ? want : maxb;
    return (int)(gx < 1 ? 1 : gx);
}

}  // namespace

bool cg4_supported(const Grid &g) { return (g.Nx % 4) == 0 && (g.ld % 4) == 0; }

// One float32 iteration t over the active lanes (see the file comment).
void cg_iteration4(cudaStream_t st, const Grid &g, const float *D, const float *const *diag_of_col,
                   const float *const *p_ptr, float *const *q_ptr, LaneGeom gm, LaneState ls, LaneList ll, int t,
                   float *mu, float *beta, KTimer *kt) {
    if (ll.na <= 0) return;
    const int sprev = (t - 1) % 3, scur = t % 3, snext = (t + 1) % 3, spq = t % 2, sw = t % 2;
    const long long nv = g.n >> 2;
    const bool tm = kt && kt->on;
    cudaEvent_t e = tm ? kt->start(st) : nullptr;
    k_stencil4<<<dim3(gx_for(nv, ll.na, 8), ll.na), kThreads, 0, st>>>(
        g, D, diag_of_col, p_ptr, q_ptr, ll.alist, ls.active, ls.pq + (long long)spq * ls.m, ls.prof);
    count_launch();
    RCG_CHECK_LAUNCH();
    if (tm) { kt->stop(0, e, st); e = kt->start(st); }
    k_update4<<<dim3(gx_for(nv, ll.na, 8), ll.na), kThreads, 0, st>>>(g.n, gm, ls, ll.alist, sprev, scur, spq, sw);
    count_launch();
    RCG_CHECK_LAUNCH();
    if (tm) { kt->stop(1, e, st); e = kt->start(st); }
    // node range per CTA for the tile kernels: a multiple of SN, ~6 CTAs per SM in total
    auto tile_chunk = [&](long long &z) {
        z = (6LL * 152 + ll.ntiles - 1) / ll.ntiles;
        const long long maxz = (g.n + 4 * SN - 1) / (4 * SN);
        if (z > maxz) z = maxz;
        if (z < 1) z = 1;
        long long chunk = (g.n + z - 1) / z;
        chunk = (chunk + SN - 1) / SN * SN;
        z = (g.n + chunk - 1) / chunk;
        return chunk;
    };
    const int kut = gm.k_u <= 4 ? 4 : gm.k_u <= 8 ? 8 : gm.k_u <= 12 ? 12 : 16;
    if (gm.k_u > 0) {
        long long z;
        const long long chunk = tile_chunk(z);
        dim3 grid((unsigned)z, ll.ntiles);
#define RCG_U0(K) k_u0dots<K><<<grid, kThreads, 0, st>>>(g.n, gm, ls, ll.tile_lane, ll.tile_si, ll.tile_cnt, sw, chunk, 0)
        switch (kut) { case 4: RCG_U0(4); break; case 8: RCG_U0(8); break; case 12: RCG_U0(12); break; default: RCG_U0(16); }
#undef RCG_U0
        count_launch();
        RCG_CHECK_LAUNCH();
    }
    if (tm) { kt->stop(2, e, st); e = kt->start(st); }
    k_mu<<<ll.na, 32, 0, st>>>(ls, ll.alist, sprev, scur, snext, sw, mu, beta, 0);
    count_launch();
    RCG_CHECK_LAUNCH();
    if (tm) { kt->stop(3, e, st); e = kt->start(st); }
    {
        long long z;
        const long long chunk = tile_chunk(z);
        dim3 grid((unsigned)z, ll.ntiles);
#define RCG_DIR(K) k_direction4<K><<<grid, kThreads, 0, st>>>(g.n, gm, ls, ll.tile_lane, ll.tile_cnt, mu, beta, chunk)
        switch (kut) { case 4: RCG_DIR(4); break; case 8: RCG_DIR(8); break; case 12: RCG_DIR(12); break; default: RCG_DIR(16); }
#undef RCG_DIR
        count_launch();
        RCG_CHECK_LAUNCH();
    }
    if (tm) kt->stop(4, e, st);
}

// (Re)start of the lanes of ll (float32, Nx % 4 == 0) at iteration number t;
// the same steps as cg_restart in cg.cu.  k_lane_zero has run for these lanes.
void cg_restart4(cudaStream_t st, const Grid &g, LaneGeom gm, LaneState ls, LaneList ll, int t, float *mu,
                 float *beta) {
    if (ll.na <= 0) return;
    const int scur = t % 3, snext = (t + 1) % 3, sprev = (t + 2) % 3;
    const int sw = t % 2, sA = (t + 1) % 2;
    const long long nv = g.n >> 2;
    long long z = (6LL * 152 + ll.ntiles - 1) / ll.ntiles;
    const long long maxz = (g.n + 4 * SN - 1) / (4 * SN);
    if (z > maxz) z = maxz;
    if (z < 1) z = 1;
    long long chunk = (g.n + z - 1) / z;
    chunk = (chunk + SN - 1) / SN * SN;
    z = (g.n + chunk - 1) / chunk;
    const dim3 tgrid((unsigned)z, ll.ntiles), lgrid(gx_for(nv, ll.na, 8), ll.na);
    const int kut = gm.k_u <= 4 ? 4 : gm.k_u <= 8 ? 8 : gm.k_u <= 12 ? 12 : 16;
#define RCG_U0(K, W, SLOT) k_u0dots<K><<<tgrid, kThreads, 0, st>>>(g.n, gm, ls, ll.tile_lane, ll.tile_si, ll.tile_cnt, SLOT, chunk, W)
#define RCG_U0S(W, SLOT) switch (kut) { case 4: RCG_U0(4, W, SLOT); break; case 8: RCG_U0(8, W, SLOT); break; \
                                    case 12: RCG_U0(12, W, SLOT); break; default: RCG_U0(16, W, SLOT); }
    // z = W^T r -> wv[sA]
    if (gm.k_u > 0) { RCG_U0S(1, sA); count_launch(); RCG_CHECK_LAUNCH(); }
    k_private_dots4<<<lgrid, kThreads, 0, st>>>(g.n, gm, ls, ll.alist, 0, sA, 0, 0);
    count_launch();
    RCG_CHECK_LAUNCH();
    // mu0 = Ginv z; x = W mu0; r -= A W mu0
    k_mu_only<<<ll.na, 32, 0, st>>>(ls, ll.alist, sA, mu);
    count_launch();
    RCG_CHECK_LAUNCH();
#define RCG_PJ(K) k_project4<K><<<tgrid, kThreads, 0, st>>>(g.n, gm, ll.tile_lane, ll.tile_si, ll.tile_cnt, mu, chunk)
    switch (kut) { case 4: RCG_PJ(4); break; case 8: RCG_PJ(8); break; case 12: RCG_PJ(12); break; default: RCG_PJ(16); }
#undef RCG_PJ
    count_launch();
    RCG_CHECK_LAUNCH();
    // rr and (A W)^T r -> rr[scur], wv[sw]
    if (gm.k_u > 0) { RCG_U0S(0, sw); count_launch(); RCG_CHECK_LAUNCH(); }
#undef RCG_U0S
#undef RCG_U0
    k_private_dots4<<<lgrid, kThreads, 0, st>>>(g.n, gm, ls, ll.alist, 1, sw, 1, scur);
    count_launch();
    RCG_CHECK_LAUNCH();
    // decision, mu, beta = 0, slot zeroing (wv[sA] is zeroed as wv[1 - sw]); p = r - W mu
    k_mu<<<ll.na, 32, 0, st>>>(ls, ll.alist, sprev, scur, snext, sw, mu, beta, 1);
    count_launch();
    RCG_CHECK_LAUNCH();
    long long zc;
    (void)zc;
#define RCG_DIR(K) k_direction4<K><<<tgrid, kThreads, 0, st>>>(g.n, gm, ls, ll.tile_lane, ll.tile_cnt, mu, beta, chunk)
    switch (kut) { case 4: RCG_DIR(4); break; case 8: RCG_DIR(8); break; case 12: RCG_DIR(12); break; default: RCG_DIR(16); }
#undef RCG_DIR
    count_launch();
    RCG_CHECK_LAUNCH();
}

}  // namespace rcg
