// Batched deflated conjugate gradients on the correction equations
// A~_s g = r (eq. resi) of many (sample, RHS) lanes at once, each lane with
// its own deflation space W = U_j (Sec. 4.2, inner recycle space) and
// A~_s W.  The recurrences follow Saad, Yeung, Erhel & Guyomarc'h (2000):
//
//   alpha = r^T r / p^T A p;  x += alpha p;  r -= alpha A p
//   beta  = r'^T r' / r^T r;  mu = (W^T A W)^-1 (A W)^T r'
//   p     = r' + beta p - W mu
//
// One iteration is three kernels: the stencil with the fused p^T q
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
#include "common.cuh"

namespace rcg {
namespace {

constexpr int kThreads = 256;

// Block-wide sums of acc[t][v] over all threads; the result is returned in
// shared memory (res[t][v]) and visible to every thread after the call.
template <int NB, int NV>
__device__ __forceinline__ void reduce_block(const double (&acc)[NB][NV], double (&res)[NB][NV]) {
    __shared__ double red[kThreads / 32][NB][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int t = 0; t < NB; ++t)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double s = acc[t][v];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) red[warp][t][v] = s;
        }
    __syncthreads();
    for (int e = threadIdx.x; e < NB * NV; e += blockDim.x) {
        const int t = e / NV, v = e % NV;
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w][t][v];
        res[t][v] = s;
    }
    __syncthreads();
}

// x += alpha p; r -= alpha q; rr[scur] += r^T r; wv[sw][c] += (AW_c)^T r for c < KCHUNK.
// Per-thread partial sums are kept in T (float32 in the mixed path: the
// float64 pipe of this GPU is far too slow for per-element work) and only
// the block reduction is float64.
template <typename T, int NB>
__global__ void __launch_bounds__(kThreads)
k_update(long long n, T *const *__restrict__ X, T *const *__restrict__ R, const T *const *__restrict__ P,
         const T *const *__restrict__ Q, LaneState ls, int sprev, int scur, int spq, int sw) {
    const int l0 = blockIdx.y * NB;
    bool act[NB];
    bool any = false;
    T alpha[NB];
    int kd[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        const int l = l0 + t;
        act[t] = l < ls.m && ls.active[l] != 0;
        alpha[t] = T(0);
        kd[t] = 0;
        if (act[t]) {
            const double pq = ls.pq[spq * ls.m + l];
            const double rr = ls.rr[sprev * ls.m + l];
            if (!(pq > 0.0) || !isfinite(pq) || !isfinite(rr)) {
                act[t] = false;            // breakdown: reported through flag = 2
                if (blockIdx.x == 0 && threadIdx.x == 0) ls.flag[l] = 2;
            } else {
                alpha[t] = (T)(rr / pq);
                kd[t] = ls.kdef[l] < KCHUNK ? ls.kdef[l] : KCHUNK;
            }
        }
        any |= act[t];
    }
    if (!any) return;
    T acc[NB][1 + KCHUNK];
#pragma unroll
    for (int t = 0; t < NB; ++t)
#pragma unroll
        for (int v = 0; v <= KCHUNK; ++v) acc[t][v] = T(0);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            if (!act[t]) continue;
            const int l = l0 + t;
            const T pv = P[l][p], qv = Q[l][p];
            X[l][p] += alpha[t] * pv;
            const T rv = R[l][p] - alpha[t] * qv;
            R[l][p] = rv;
            acc[t][0] += rv * rv;
            const T *const *aw = (const T *const *)(ls.AW + (long long)l * KMAX);
#pragma unroll
            for (int c = 0; c < KCHUNK; ++c)
                if (c < kd[t]) acc[t][1 + c] += aw[c][p] * rv;
        }
    }
    double accd[NB][1 + KCHUNK];
    __shared__ double out[NB][1 + KCHUNK];
#pragma unroll
    for (int t = 0; t < NB; ++t)
#pragma unroll
        for (int v = 0; v <= KCHUNK; ++v) accd[t][v] = (double)acc[t][v];
    reduce_block<NB, 1 + KCHUNK>(accd, out);
    if (threadIdx.x < NB) {
        const int t = threadIdx.x, l = l0 + t;
        if (act[t]) {
            atomicAdd(ls.rr + scur * ls.m + l, out[t][0]);
            for (int c = 0; c < kd[t]; ++c) atomicAdd(ls.wv + ((long long)sw * ls.m + l) * KMAX + c, out[t][1 + c]);
            if (blockIdx.x == 0) ls.pq[(1 - spq) * ls.m + l] = 0.0;
        }
    }
}

// wv[sw][c0 + c] += (src_c)^T v for c < KCHUNK (src = W or A W); optionally rr[srr] += v^T v.
template <typename T, int NB>
__global__ void __launch_bounds__(kThreads)
k_lane_dots(long long n, const T *const *__restrict__ Vec, LaneState ls, const int *__restrict__ mask, int use_aw,
            int sw, int c0, int with_rr, int srr) {
    const int l0 = blockIdx.y * NB;
    bool act[NB];
    bool any = false;
    int kd[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        const int l = l0 + t;
        act[t] = l < ls.m && mask[l] != 0;
        kd[t] = 0;
        if (act[t]) {
            const int k = ls.kdef[l] - c0;
            kd[t] = k < 0 ? 0 : (k > KCHUNK ? KCHUNK : k);
            if (kd[t] == 0 && !with_rr) act[t] = false;
        }
        any |= act[t];
    }
    if (!any) return;
    T acc[NB][1 + KCHUNK];
#pragma unroll
    for (int t = 0; t < NB; ++t)
#pragma unroll
        for (int v = 0; v <= KCHUNK; ++v) acc[t][v] = T(0);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            if (!act[t]) continue;
            const int l = l0 + t;
            const T v = Vec[l][p];
            if (with_rr) acc[t][0] += v * v;
            const T *const *src = (const T *const *)((use_aw ? ls.AW : ls.W) + (long long)l * KMAX + c0);
#pragma unroll
            for (int c = 0; c < KCHUNK; ++c)
                if (c < kd[t]) acc[t][1 + c] += src[c][p] * v;
        }
    }
    double accd[NB][1 + KCHUNK];
    __shared__ double out[NB][1 + KCHUNK];
#pragma unroll
    for (int t = 0; t < NB; ++t)
#pragma unroll
        for (int v = 0; v <= KCHUNK; ++v) accd[t][v] = (double)acc[t][v];
    reduce_block<NB, 1 + KCHUNK>(accd, out);
    if (threadIdx.x < NB) {
        const int t = threadIdx.x, l = l0 + t;
        if (act[t]) {
            if (with_rr) atomicAdd(ls.rr + srr * ls.m + l, out[t][0]);
            for (int c = 0; c < kd[t]; ++c)
                atomicAdd(ls.wv + ((long long)sw * ls.m + l) * KMAX + c0 + c, out[t][1 + c]);
        }
    }
}

// mu = Ginv * wv[sw] for each active lane of the group, rounded to T, in shared memory.
template <typename T, int NB>
__device__ void lane_mu(const LaneState &ls, int l0, const bool (&act)[NB], int sw, T (*mu)[KMAX]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = warp; t < NB; t += kThreads / 32) {
        if (!act[t]) continue;
        const int l = l0 + t;
        const int k = ls.kdef[l];
        const double *G = ls.gw + (long long)l * KMAX * KMAX;
        const double *w = ls.wv + ((long long)sw * ls.m + l) * KMAX;
        for (int i = lane; i < k; i += 32) {
            double s = 0.0;
            for (int j = 0; j < k; ++j) s += G[i + j * KMAX] * w[j];
            mu[t][i] = (T)s;
        }
    }
    __syncthreads();
}

// Restart projection: mu0 = Ginv (W^T r) (from wv[sw]); x = W mu0; r -= A W mu0.
template <typename T, int NB>
__global__ void __launch_bounds__(kThreads)
k_restart_project(long long n, T *const *__restrict__ X, T *const *__restrict__ R, LaneState ls,
                  const int *__restrict__ mask, int sw) {
    __shared__ T mu[NB][KMAX];
    const int l0 = blockIdx.y * NB;
    bool act[NB];
    bool any = false;
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        const int l = l0 + t;
        act[t] = l < ls.m && mask[l] != 0;
        any |= act[t];
    }
    if (!any) return;
    lane_mu<T, NB>(ls, l0, act, sw, mu);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            if (!act[t]) continue;
            const int l = l0 + t;
            const int k = ls.kdef[l];
            const T *const *w = (const T *const *)(ls.W + (long long)l * KMAX);
            const T *const *aw = (const T *const *)(ls.AW + (long long)l * KMAX);
            T xs = T(0), rs = T(0);
            for (int c = 0; c < k; ++c) {
                xs += w[c][p] * mu[t][c];
                rs += aw[c][p] * mu[t][c];
            }
            X[l][p] = xs;
            R[l][p] -= rs;
        }
    }
}

// p = r + beta p - W mu, with the per-lane convergence test on the recursive
// residual.  In restart mode beta = 0 and no iteration is counted.  Every
// CTA takes the same decision from the same completed sums; CTA (0, y)
// records it (active = 0; flag = 1 converged, 2 breakdown) and zeroes the
// ring slots the next iteration accumulates into.
template <typename T, int NB>
__global__ void __launch_bounds__(kThreads)
k_direction(long long n, const T *const *__restrict__ R, T *const *__restrict__ P, LaneState ls,
            const int *__restrict__ mask, int sprev, int scur, int snext, int sw, int restart) {
    __shared__ T mu[NB][KMAX];
    const int l0 = blockIdx.y * NB;
    bool act[NB];
    bool any = false;
    T beta[NB];
#pragma unroll
    for (int t = 0; t < NB; ++t) {
        const int l = l0 + t;
        act[t] = l < ls.m && mask[l] != 0;
        beta[t] = T(0);
        if (act[t]) {
            const double rc = ls.rr[scur * ls.m + l];
            const bool broke = (ls.flag[l] == 2) || !isfinite(rc);
            const bool conv = !broke && sqrt(rc) <= ls.thresh[l];
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                if (!restart) ls.iters[l] += 1;
                if (broke) { ls.active[l] = 0; ls.flag[l] = 2; }
                else if (conv) { ls.active[l] = 0; ls.flag[l] = 1; }
            }
            if (broke || conv) act[t] = false;
            else beta[t] = restart ? T(0) : (T)(rc / ls.rr[sprev * ls.m + l]);
        }
        any |= act[t];
    }
    if (blockIdx.x == 0 && threadIdx.x < NB) {
        const int l = l0 + threadIdx.x;
        if (l < ls.m && mask[l] != 0) {
            ls.rr[snext * ls.m + l] = 0.0;
            for (int c = 0; c < KMAX; ++c) ls.wv[((long long)(1 - sw) * ls.m + l) * KMAX + c] = 0.0;
        }
    }
    if (!any) return;
    lane_mu<T, NB>(ls, l0, act, sw, mu);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int t = 0; t < NB; ++t) {
            if (!act[t]) continue;
            const int l = l0 + t;
            const int k = ls.kdef[l];
            const T *const *w = (const T *const *)(ls.W + (long long)l * KMAX);
            T v = R[l][p];
            if (!restart) v += beta[t] * P[l][p];
            T s = T(0);
            for (int c = 0; c < k; ++c) s += w[c][p] * mu[t][c];
            P[l][p] = v - s;
        }
    }
}

// Zero the ring slots and clear the flag of the masked lanes.
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

int grid_x(long long n, int groups) {
    long long want = (4LL * 152 + groups - 1) / groups;
    long long maxb = (n + kThreads - 1) / kThreads;
    long long gx = want < maxb ? want : maxb;
    return (int)(gx < 1 ? 1 : gx);
}

template <typename T> constexpr int nb_of() { return sizeof(T) == 8 ? 2 : 4; }

}  // namespace

// One CG iteration number t >= 1 over all active lanes; kmax_used is the
// largest deflation column count of any lane.
template <typename T>
void cg_iteration(cudaStream_t st, const Grid &g, const T *D, const T *const *diag_of_col, T *const *x,
                  T *const *r, T *const *p, T *const *q, LaneState ls, int t, int kmax_used) {
    constexpr int NB = nb_of<T>();
    const int groups = (ls.m + NB - 1) / NB;
    const int sprev = (t - 1) % 3, scur = t % 3, snext = (t + 1) % 3, spq = t % 2, sw = t % 2;
    apply_op<T>(st, g, D, diag_of_col, (const T *const *)p, q, ls.m, ls.active, ls.pq + (long long)spq * ls.m, 0);
    dim3 grid(grid_x(g.n, groups), groups);
    k_update<T, NB><<<grid, kThreads, 0, st>>>(g.n, x, r, (const T *const *)p, (const T *const *)q, ls, sprev, scur,
                                                spq, sw);
    count_launch();
    RCG_CHECK_LAUNCH();
    for (int c0 = KCHUNK; c0 < kmax_used; c0 += KCHUNK) {   // deflation columns beyond the fused chunk
        k_lane_dots<T, NB><<<grid, kThreads, 0, st>>>(g.n, (const T *const *)r, ls, ls.active, 1, sw, c0, 0, 0);
        count_launch();
        RCG_CHECK_LAUNCH();
    }
    k_direction<T, NB><<<grid, kThreads, 0, st>>>(g.n, (const T *const *)r, p, ls, ls.active, sprev, scur, snext, sw,
                                                   0);
    count_launch();
    RCG_CHECK_LAUNCH();
}

// (Re)start the masked lanes at iteration number t: given r (the residual of
// the current iterate), set x = W mu0, r -= A W mu0 (mu0 = Ginv W^T r),
// rr[t mod 3] = r^T r and p = r - W Ginv (A W)^T r.
template <typename T>
void cg_restart(cudaStream_t st, const Grid &g, T *const *x, T *const *r, T *const *p, LaneState ls, int t,
                const int *mask, int kmax_used) {
    constexpr int NB = nb_of<T>();
    const int groups = (ls.m + NB - 1) / NB;
    dim3 grid(grid_x(g.n, groups), groups);
    const int scur = t % 3, snext = (t + 1) % 3, sprev = (t + 2) % 3;
    const int sw = t % 2, sA = (t + 1) % 2;
    k_lane_zero<<<ls.m, 64, 0, st>>>(ls, mask);
    count_launch();
    RCG_CHECK_LAUNCH();
    for (int c0 = 0; c0 < kmax_used; c0 += KCHUNK) {      // z = W^T r -> wv[sA]
        k_lane_dots<T, NB><<<grid, kThreads, 0, st>>>(g.n, (const T *const *)r, ls, mask, 0, sA, c0, 0, 0);
        count_launch();
        RCG_CHECK_LAUNCH();
    }
    k_restart_project<T, NB><<<grid, kThreads, 0, st>>>(g.n, x, r, ls, mask, sA);
    count_launch();
    RCG_CHECK_LAUNCH();
    const int kloop = kmax_used > 0 ? kmax_used : 1;
    for (int c0 = 0; c0 < kloop; c0 += KCHUNK) {          // rr and (A W)^T r -> wv[sw]
        k_lane_dots<T, NB><<<grid, kThreads, 0, st>>>(g.n, (const T *const *)r, ls, mask, 1, sw, c0, c0 == 0 ? 1 : 0,
                                                      scur);
        count_launch();
        RCG_CHECK_LAUNCH();
    }
    // the direction kernel zeroes wv[1 - sw] == wv[sA] (the scratch above) and rr[snext]
    k_direction<T, NB><<<grid, kThreads, 0, st>>>(g.n, (const T *const *)r, p, ls, mask, sprev, scur, snext, sw, 1);
    count_launch();
    RCG_CHECK_LAUNCH();
}

template void cg_iteration<double>(cudaStream_t, const Grid &, const double *, const double *const *,
                                   double *const *, double *const *, double *const *, double *const *, LaneState, int,
                                   int);
template void cg_iteration<float>(cudaStream_t, const Grid &, const float *, const float *const *, float *const *,
                                  float *const *, float *const *, float *const *, LaneState, int, int);
template void cg_restart<double>(cudaStream_t, const Grid &, double *const *, double *const *, double *const *,
                                 LaneState, int, const int *, int);
template void cg_restart<float>(cudaStream_t, const Grid &, float *const *, float *const *, float *const *,
                                LaneState, int, const int *, int);

}  // namespace rcg
