// Batched deflated conjugate gradients on the correction equations
// A~_s g = r (eq. resi) of many (sample, RHS) lanes at once, each lane with
// its own deflation space W = U_j (Sec. 4.2, inner recycle space) and
// A~_s W.  The recurrences follow Saad, Yeung, Erhel & Guyomarc'h (2000):
//
//   alpha = r^T r / p^T A p;  x += alpha p;  r -= alpha A p
//   beta  = r'^T r' / r^T r;  mu = (W^T A W)^-1 (A W)^T r'
//   p     = r' + beta p - W mu
//
// One iteration is three kernels (one lane per CTA row, one node per
// thread, so that registers stay low and enough warps are resident to cover
// the HBM latency): the stencil with the fused p^T q
// reduction (stencil.cu), the update with fused r^T r and (A W)^T r
// reductions, and the direction.  Reductions go through float64 atomics into
// ring buffers indexed by the iteration number, so no scalar leaves the
// device: every CTA of a kernel reads the same completed sums of the
// previous kernel and takes the same per-lane decisions (convergence,
// breakdown) without any grid-wide synchronisation inside a kernel.
//
//   rr[t mod 3]  r^T r after iteration t      pq[t mod 2]  p^T A p of iteration t
//   wv[t mod 2]  (A W)^T r after iteration t
// A slot is zeroed by the kernel that runs one step before its next writer.
//
// Lane addressing is arithmetic (LaneGeom): lane l's vectors are column l of
// contiguous blocks; its first k_u deflation columns are shared by every lane
// (the seed eigenvector block of V) with A~_s U_0 per sample slot, the rest
// are private copies.  Per-thread partial sums stay in T (float32 in the
// mixed path: the float64 pipe of this GPU is far too slow for per-element
// work); only the block reductions are float64.
#include "common.cuh"

namespace rcg {
namespace {

constexpr int kThreads = 256;

// Block-wide sums of acc[v] over all threads, returned in shared memory.
template <int NV>
__device__ __forceinline__ void reduce_block(const double (&acc)[NV], double (&res)[NV]) {
    __shared__ double red[kThreads / 32][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double s = acc[v];
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

template <typename T>
__device__ __forceinline__ const T *col(const void *base, long long idx, long long ld) {
    return (const T *)base + idx * ld;
}

// Index in wv of accumulator v (>= 1): shared columns first, then private.
__device__ __forceinline__ int wv_index(int v, int ku, int kp) {
    const int c = v - 1;
    if (c < KU_MAX) return c < ku ? c : -1;
    return (c - KU_MAX) < kp ? ku + (c - KU_MAX) : -1;
}

constexpr int NV = 1 + KU_MAX + KP_MAX;

// Add the block sums out[] of lane l into rr[srr] (v = 0, optional) and wv[sw].
__device__ __forceinline__ void flush_dots(const LaneState &ls, int l, const double (&out)[NV], int ku, int kp,
                                           int sw, bool with_rr, int srr) {
    for (int v = threadIdx.x; v < NV; v += blockDim.x) {
        if (v == 0) {
            if (with_rr) atomicAdd(ls.rr + srr * ls.m + l, out[0]);
        } else {
            const int ci = wv_index(v, ku, kp);
            if (ci >= 0) atomicAdd(ls.wv + ((long long)sw * ls.m + l) * KMAX + ci, out[v]);
        }
    }
}

// Lane l = blockIdx.y:  x += alpha p; r -= alpha q; rr[scur] += r^T r;
// wv[sw][c] += (A W_c)^T r for every deflation column of the lane.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_update(long long n, LaneGeom gm, LaneState ls, int sprev, int scur, int spq, int sw) {
    const int l = blockIdx.y;
    if (l >= ls.m || ls.active[l] == 0) return;
    const double pq = ls.pq[spq * ls.m + l];
    const double rr = ls.rr[sprev * ls.m + l];
    if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rr)) {       // breakdown: reported through flag = 2
        if (blockIdx.x == 0 && threadIdx.x == 0) ls.flag[l] = 2;
        return;
    }
    const T alpha = (T)(rr / pq);
    const int ku = gm.k_u, kp = gm.kp[l], si = gm.si[l];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ls.pq[(1 - spq) * ls.m + l] = 0.0;
        if (ls.prof) { atomicAdd(ls.prof + 1, 1ULL); atomicAdd(ls.prof + 2, (unsigned long long)(ku + kp)); }
    }
    T acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = T(0);
    const long long o = (long long)l * gm.ld;
    T *__restrict__ X = (T *)gm.x + o;
    T *__restrict__ R = (T *)gm.r + o;
    const T *__restrict__ P = (const T *)gm.p + o;
    const T *__restrict__ Q = (const T *)gm.q + o;
    const T *__restrict__ AU = col<T>(gm.awu, (long long)si * ku, gm.ld);
    const T *__restrict__ AP = col<T>(gm.awp, (long long)l * gm.kp_max, gm.ld);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const T rv = R[p] - alpha * Q[p];
        X[p] += alpha * P[p];
        R[p] = rv;
        acc[0] += rv * rv;
#pragma unroll
        for (int c = 0; c < KU_MAX; ++c)
            if (c < ku) acc[1 + c] += AU[(long long)c * gm.ld + p] * rv;
#pragma unroll
        for (int c = 0; c < KP_MAX; ++c)
            if (c < kp) acc[1 + KU_MAX + c] += AP[(long long)c * gm.ld + p] * rv;
    }
    double accd[NV];
    __shared__ double out[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) accd[v] = (double)acc[v];
    reduce_block<NV>(accd, out);
    flush_dots(ls, l, out, ku, kp, sw, true, scur);
}

// Lane l = blockIdx.y (masked): wv[sw][c] += (src_c)^T r over all deflation
// columns (src = W or A W); optionally rr[srr] += r^T r.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_lane_dots(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ mask, int use_aw, int sw, int with_rr,
            int srr) {
    const int l = blockIdx.y;
    if (l >= ls.m || mask[l] == 0) return;
    const int ku = gm.k_u, kp = gm.kp[l], si = gm.si[l];
    const T *__restrict__ Ws = use_aw ? col<T>(gm.awu, (long long)si * ku, gm.ld) : (const T *)gm.wu;
    const T *Wq[KP_MAX];
#pragma unroll
    for (int c = 0; c < KP_MAX; ++c)
        Wq[c] = c >= kp ? nullptr
                        : use_aw ? col<T>(gm.awp, (long long)l * gm.kp_max + c, gm.ld)
                                 : (const T *)gm.wpp[(long long)l * KPT + c];
    const T *__restrict__ R = (const T *)gm.r + (long long)l * gm.ld;
    T acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = T(0);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const T v = R[p];
        acc[0] += v * v;
#pragma unroll
        for (int c = 0; c < KU_MAX; ++c)
            if (c < ku) acc[1 + c] += Ws[(long long)c * gm.ld + p] * v;
#pragma unroll
        for (int c = 0; c < KP_MAX; ++c)
            if (c < kp) acc[1 + KU_MAX + c] += Wq[c][p] * v;
    }
    double accd[NV];
    __shared__ double out[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) accd[v] = (double)acc[v];
    reduce_block<NV>(accd, out);
    flush_dots(ls, l, out, ku, kp, sw, with_rr != 0, srr);
}

// mu = Ginv * wv[sw] of lane l, rounded to T, into shared memory (warp 0).
template <typename T>
__device__ void lane_mu(const LaneState &ls, int l, int sw, T *mu) {
    if (threadIdx.x < 32) {
        const int k = ls.kdef[l];
        const double *G = ls.gw + (long long)l * KMAX * KMAX;
        const double *w = ls.wv + ((long long)sw * ls.m + l) * KMAX;
        for (int i = threadIdx.x; i < k; i += 32) {
            double s = 0.0;
            for (int j = 0; j < k; ++j) s += G[i + j * KMAX] * w[j];
            mu[i] = (T)s;
        }
    }
    __syncthreads();
}

// Restart projection of lane l: mu0 = Ginv (W^T r) (from wv[sw]); x = W mu0; r -= A W mu0.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_restart_project(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ mask, int sw) {
    __shared__ T mu[KMAX];
    const int l = blockIdx.y;
    if (l >= ls.m || mask[l] == 0) return;
    lane_mu<T>(ls, l, sw, mu);
    const int ku = gm.k_u, kp = gm.kp[l], si = gm.si[l];
    const long long o = (long long)l * gm.ld;
    T *__restrict__ X = (T *)gm.x + o;
    T *__restrict__ R = (T *)gm.r + o;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        T xs = T(0), rs = T(0);
        for (int c = 0; c < ku; ++c) {
            xs += col<T>(gm.wu, c, gm.ld)[p] * mu[c];
            rs += col<T>(gm.awu, (long long)si * ku + c, gm.ld)[p] * mu[c];
        }
        for (int c = 0; c < kp; ++c) {
            const long long ci = (long long)l * gm.kp_max + c;
            xs += ((const T *)gm.wpp[(long long)l * KPT + c])[p] * mu[ku + c];
            rs += col<T>(gm.awp, ci, gm.ld)[p] * mu[ku + c];
        }
        X[p] = xs;
        R[p] -= rs;
    }
}

// Lane l = blockIdx.y (masked): p = r + beta p - W mu, with the per-lane
// convergence test on the recursive residual.  In restart mode beta = 0 and
// no iteration is counted.  Every CTA of the lane takes the same decision
// from the same completed sums; CTA (0, l) records it (active = 0; flag = 1
// converged, 2 breakdown) and zeroes the ring slots the next iteration
// accumulates into.
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_direction(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ mask, int sprev, int scur, int snext,
            int sw, int restart) {
    __shared__ T mu[KMAX];
    const int l = blockIdx.y;
    if (l >= ls.m || mask[l] == 0) return;
    const double rc = ls.rr[scur * ls.m + l];
    const bool broke = (ls.flag[l] == 2) || !isfinite(rc);
    const bool conv = !broke && sqrt(rc) <= ls.thresh[l];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (!restart) ls.iters[l] += 1;
        if (broke) { ls.active[l] = 0; ls.flag[l] = 2; }
        else if (conv) { ls.active[l] = 0; ls.flag[l] = 1; }
        ls.rr[snext * ls.m + l] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x >= 32 && threadIdx.x < 32 + KMAX)
        ls.wv[((long long)(1 - sw) * ls.m + l) * KMAX + (threadIdx.x - 32)] = 0.0;
    if (broke || conv) return;
    const T beta = restart ? T(0) : (T)(rc / ls.rr[sprev * ls.m + l]);
    const int ku = gm.k_u, kp = gm.kp[l];
    if (!restart && ls.prof && blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(ls.prof + 3, 1ULL);
        atomicAdd(ls.prof + 4, (unsigned long long)(ku + kp));
    }
    lane_mu<T>(ls, l, sw, mu);
    T m_u[KU_MAX], m_p[KP_MAX];
#pragma unroll
    for (int c = 0; c < KU_MAX; ++c) m_u[c] = c < ku ? mu[c] : T(0);
#pragma unroll
    for (int c = 0; c < KP_MAX; ++c) m_p[c] = c < kp ? mu[ku + c] : T(0);
    const long long o = (long long)l * gm.ld;
    const T *__restrict__ R = (const T *)gm.r + o;
    T *__restrict__ P = (T *)gm.p + o;
    const T *__restrict__ WU = (const T *)gm.wu;
    const T *WP[KP_MAX];
#pragma unroll
    for (int c = 0; c < KP_MAX; ++c) WP[c] = c < kp ? (const T *)gm.wpp[(long long)l * KPT + c] : nullptr;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        T v = R[p];
        if (!restart) v += beta * P[p];
        T s = T(0);
#pragma unroll
        for (int c = 0; c < KU_MAX; ++c)
            if (c < ku) s += WU[(long long)c * gm.ld + p] * m_u[c];
#pragma unroll
        for (int c = 0; c < KP_MAX; ++c)
            if (c < kp) s += WP[c][p] * m_p[c];
        P[p] = v - s;
    }
}

// Zero the ring slots, clear the flag and activate the masked lanes.
__global__ void k_lane_zero(LaneState ls, const int *__restrict__ mask) {
    const int l = blockIdx.x;
    if (mask[l] == 0) return;
    for (int s = threadIdx.x; s < 3; s += blockDim.x) ls.rr[s * ls.m + l] = 0.0;
    for (int s = threadIdx.x; s < 2; s += blockDim.x) ls.pq[s * ls.m + l] = 0.0;
    for (int e = threadIdx.x; e < 2 * KMAX; e += blockDim.x) {
        const int s = e / KMAX, c = e % KMAX;
        ls.wv[((long long)s * ls.m + l) * KMAX + c] = 0.0;
    }
    if (threadIdx.x == 0) { ls.flag[l] = 0; ls.active[l] = 1; }
}

// ~8 resident CTAs per SM spread over the lanes, at least one node per thread
int grid_x(long long n, int lanes) {
    long long want = (8LL * 152 + lanes - 1) / lanes;
    long long maxb = (n + kThreads - 1) / kThreads;
    long long gx = want < maxb ? want : maxb;
    return (int)(gx < 1 ? 1 : gx);
}

}  // namespace

// One CG iteration number t >= 1 over all active lanes.
template <typename T>
void cg_iteration(cudaStream_t st, const Grid &g, const T *D, const T *const *diag_of_col, const T *const *p_ptr,
                  T *const *q_ptr, LaneGeom gm, LaneState ls, int t, KTimer *kt) {
    const int sprev = (t - 1) % 3, scur = t % 3, snext = (t + 1) % 3, spq = t % 2, sw = t % 2;
    const bool tm = kt && kt->on;
    cudaEvent_t e = tm ? kt->start(st) : nullptr;
    apply_op<T>(st, g, D, diag_of_col, p_ptr, q_ptr, ls.nl, ls.active, ls.pq + (long long)spq * ls.m, ls.prof);
    if (tm) { kt->stop(0, e, st); e = kt->start(st); }
    // the wave's lanes only: a wave smaller than the capacity keeps the whole GPU
    dim3 grid(grid_x(g.n, ls.nl), ls.nl);
    k_update<T><<<grid, kThreads, 0, st>>>(g.n, gm, ls, sprev, scur, spq, sw);
    count_launch();
    RCG_CHECK_LAUNCH();
    if (tm) { kt->stop(1, e, st); e = kt->start(st); }
    k_direction<T><<<grid, kThreads, 0, st>>>(g.n, gm, ls, ls.active, sprev, scur, snext, sw, 0);
    count_launch();
    RCG_CHECK_LAUNCH();
    if (tm) kt->stop(4, e, st);
}

// (Re)start the masked lanes at iteration number t: given r (the residual of
// the current iterate), set x = W mu0, r -= A W mu0 (mu0 = Ginv W^T r),
// rr[t mod 3] = r^T r and p = r - W Ginv (A W)^T r.
template <typename T>
void cg_restart(cudaStream_t st, const Grid &g, LaneGeom gm, LaneState ls, int t, const int *mask, int *drop) {
    dim3 grid(grid_x(g.n, ls.nl), ls.nl);
    const int scur = t % 3, snext = (t + 1) % 3, sprev = (t + 2) % 3;
    const int sw = t % 2, sA = (t + 1) % 2;
    k_lane_zero<<<ls.nl, 64, 0, st>>>(ls, mask);
    count_launch();
    RCG_CHECK_LAUNCH();
    k_lane_dots<T><<<grid, kThreads, 0, st>>>(g.n, gm, ls, mask, 0, sA, 0, 0);       // W^T r -> wv[sA]
    count_launch();
    RCG_CHECK_LAUNCH();
    k_restart_project<T><<<grid, kThreads, 0, st>>>(g.n, gm, ls, mask, sA);
    count_launch();
    RCG_CHECK_LAUNCH();
    // the learned column served the projection only (RCG_LEARN_START)
    drop_last_private(st, ls, const_cast<int *>(gm.kp), drop, ls.nl);
    k_lane_dots<T><<<grid, kThreads, 0, st>>>(g.n, gm, ls, mask, 1, sw, 1, scur);    // rr, (A W)^T r -> wv[sw]
    count_launch();
    RCG_CHECK_LAUNCH();
    // the direction kernel zeroes wv[1 - sw] == wv[sA] (the scratch above) and rr[snext]
    k_direction<T><<<grid, kThreads, 0, st>>>(g.n, gm, ls, mask, sprev, scur, snext, sw, 1);
    count_launch();
    RCG_CHECK_LAUNCH();
}

// Lanes with drop[l] != 0 give up their last private deflation column (the
// learned column, which the augmentation bordered last): kdef and kp fall
// by one, and the lane's inverse H = (W^T A~ W)^-1 loses that column: with
// k the new count, the inverse of the leading k x k block of W^T A~ W is
// H11 - h12 h21 / h22 (the bordering step undone).  drop[l] is cleared.
// One CTA per lane.
__global__ void k_drop_last_private(LaneState ls, int *kp, int *drop) {
    const int l = blockIdx.x;
    if (!drop[l]) return;
    const int k1 = ls.kdef[l];
    if (k1 > 0 && kp[l] > 0) {
        double *H = ls.gw + (long long)l * KMAX * KMAX;
        const int k = k1 - 1;
        const double hkk = H[k + (long long)k * KMAX];
        // entries (i, j < k) read column k and row k, which no thread writes
        for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
            const int i = e % k, j = e / k;
            H[i + (long long)j * KMAX] -= H[i + (long long)k * KMAX] * H[k + (long long)j * KMAX] / hkk;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (k1 > 0 && kp[l] > 0) {
            --ls.kdef[l];
            --kp[l];
        }
        drop[l] = 0;
    }
}

void drop_last_private(cudaStream_t st, LaneState ls, int *kp, int *drop, int m) {
    if (!drop || m <= 0) return;
    k_drop_last_private<<<m, 128, 0, st>>>(ls, kp, drop);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void lane_zero(cudaStream_t st, LaneState ls, const int *mask) {
    k_lane_zero<<<ls.nl, 64, 0, st>>>(ls, mask);
    count_launch();
    RCG_CHECK_LAUNCH();
}

template void cg_iteration<double>(cudaStream_t, const Grid &, const double *, const double *const *,
                                   const double *const *, double *const *, LaneGeom, LaneState, int, KTimer *);
template void cg_iteration<float>(cudaStream_t, const Grid &, const float *, const float *const *,
                                  const float *const *, float *const *, LaneGeom, LaneState, int, KTimer *);
template void cg_restart<double>(cudaStream_t, const Grid &, LaneGeom, LaneState, int, const int *, int *);
template void cg_restart<float>(cudaStream_t, const Grid &, LaneGeom, LaneState, int, const int *, int *);

}  // namespace rcg
