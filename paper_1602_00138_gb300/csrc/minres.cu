// The paper's own inner solver (Sec. 4.1, eqs. eq01 and SmallMin; the inner
// solve of Algorithm 2): recycled MINRES on A~ g = r for batches of lanes,
// float64, each lane with its recycle space W = U_j and the images A~ W.
//
// With K = A~ W R^-1 orthonormal (A~ W = K R), the projector onto the
// complement of range(A~ W) is P w = w - A~W H^-1 (A~W)^T w, H = (A~W)^T A~W,
// so no orthonormal K is formed: H^-1 lives in LaneState::gw (KMAX stride,
// from the same inverse routine as the CG deflation matrix).  A cycle from
// the residual r of the current iterate:
//
//   mu = H^-1 (A~W)^T r;  x += W mu;  v_1 = (r - A~W mu) / xi, xi = ||.||
//   Lanczos with P A~:  w = P A~ v_k - alpha_k v_k - beta_k v_{k-1},
//                       alpha_k = v_k^T A~ v_k (v_k is orthogonal to range(A~W)),
//                       beta_{k+1} = ||w||,  v_{k+1} = w / beta_{k+1}
//   Givens QR of the tridiagonal T_k (two previous rotations on the new
//   column, a new one against beta_{k+1}); the MINRES iterate y_k = V_k y by
//   y += tau_k d_k, d_k = (v_k - delta_k d_{k-1} - eps_k d_{k-2}) / gamma_k;
//   |phibar_k| = ||r - A~ g_k|| for g_k = y_k - W H^-1 (A~W)^T A~ y_k.
//   At |phibar| <= thresh: x += y_k - W H^-1 (A~W)^T A~ y_k, and the host
//   recomputes the float64 residual and restarts the lane if needed.
//
// Per-lane scalars live in MresState::sc [m][MR_NSC]; vectors of lane l are
// column l of the lane blocks (LaneGeom: x = y_k, r, p = v_k, q = A~ v_k
// then w) and of three extra blocks: v_{k-1}, d_{k-1}, d_{k-2}.
#include "common.cuh"

namespace rcg {
namespace {

constexpr int kThreads = 256;

template <int NV>
__device__ __forceinline__ void block_sum_d(const double (&acc)[NV], double (&res)[NV]) {
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

__device__ __forceinline__ const double *aw_col(const LaneGeom &gm, int l, int c) {
    const int ku = gm.k_u;
    return c < ku ? (const double *)gm.awu + ((long long)gm.si[l] * ku + c) * gm.ld
                  : (const double *)gm.awp + ((long long)l * gm.kp_max + (c - ku)) * gm.ld;
}

__device__ __forceinline__ const double *w_col(const LaneGeom &gm, int l, int c) {
    const int ku = gm.k_u;
    return c < ku ? (const double *)gm.wu + (long long)c * gm.ld : (const double *)gm.wpp[(long long)l * KPT + c - ku];
}

// H[l] (KMAX stride, lower and upper) += (A~W)^T A~W over this CTA's nodes:
// CTA (x, l, a) accumulates row a against columns b <= a.
__global__ void __launch_bounds__(kThreads)
k_mres_gram(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ mask, double *__restrict__ H, int use_w) {
    constexpr int NB = KU_MAX + KP_MAX;
    const int l = blockIdx.y, a = blockIdx.z;
    if (l >= ls.nl || mask[l] == 0) return;
    const int k = ls.kdef[l];
    if (a >= k) return;
    const double *Aa = use_w ? w_col(gm, l, a) : aw_col(gm, l, a);
    const double *B[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) B[b] = b <= a ? (use_w ? w_col(gm, l, b) : aw_col(gm, l, b)) : nullptr;
    double acc[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[b] = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const double x = Aa[p];
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (b <= a) acc[b] += x * B[b][p];
    }
    __shared__ double out[NB];
    block_sum_d<NB>(acc, out);
    double *Hl = H + (long long)l * KMAX * KMAX;
    for (int b = threadIdx.x; b <= a; b += blockDim.x) {
        atomicAdd(Hl + a + (long long)b * KMAX, out[b]);
        if (b != a) atomicAdd(Hl + b + (long long)a * KMAX, out[b]);
    }
}

// hd[l][c] += (A~W_c)^T src_l for the lane's k columns (src = base + l ld).
__global__ void __launch_bounds__(kThreads)
k_mres_dots(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ mask, const double *__restrict__ src,
            double *__restrict__ hd, int use_w) {
    constexpr int NB = KU_MAX + KP_MAX;
    const int l = blockIdx.y;
    if (l >= ls.nl || mask[l] == 0) return;
    const int k = ls.kdef[l];
    const double *S = src + (long long)l * gm.ld;
    const double *C[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) C[c] = c < k ? (use_w ? w_col(gm, l, c) : aw_col(gm, l, c)) : nullptr;
    double acc[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) acc[c] = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const double s = S[p];
#pragma unroll
        for (int c = 0; c < NB; ++c)
            if (c < k) acc[c] += C[c][p] * s;
    }
    __shared__ double out[NB];
    block_sum_d<NB>(acc, out);
    for (int c = threadIdx.x; c < k; c += blockDim.x) atomicAdd(hd + (long long)l * KMAX + c, out[c]);
}

// mu[l] = H^-1[l] hd[l] (one warp per lane l = blockIdx.x); clears the lane's
// start accumulator sc[XI2] for the k_mres_cycle that follows a restart.
__global__ void __launch_bounds__(32)
k_mres_mu(LaneState ls, const int *__restrict__ mask, const double *__restrict__ hd, double *__restrict__ mu,
          double *__restrict__ sc) {
    const int l = blockIdx.x;
    if (l >= ls.nl || mask[l] == 0) return;
    if (threadIdx.x == 0) sc[(long long)l * MR_NSC + MR_XI2] = 0.0;
    const int k = ls.kdef[l];
    const double *G = ls.gw + (long long)l * KMAX * KMAX;
    const double *h = hd + (long long)l * KMAX;
    for (int i = threadIdx.x; i < k; i += 32) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += G[i + (long long)j * KMAX] * h[j];
        mu[(long long)l * KMAX + i] = s;
    }
}

// Start of a cycle for the masked lanes: x64 += W mu (sign +1, the minimum
// residual part in range(W)); v = r - A~W mu; sc[XI2] += ||v||^2.
// Finish of a cycle (finish = 1): x64 += y - W mu (mu from (A~W)^T A~ y).
__global__ void __launch_bounds__(kThreads)
k_mres_cycle(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ mask, const double *__restrict__ mu,
             double *const *__restrict__ x64, double *__restrict__ sc, int finish) {
    constexpr int NB = KU_MAX + KP_MAX;
    const int l = blockIdx.y;
    if (l >= ls.nl || mask[l] == 0) return;
    const int k = ls.kdef[l];
    __shared__ double m[NB];
    for (int c = threadIdx.x; c < NB; c += blockDim.x) m[c] = c < k ? mu[(long long)l * KMAX + c] : 0.0;
    __syncthreads();
    const double *W[NB], *AW[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) {
        W[c] = c < k ? w_col(gm, l, c) : nullptr;
        AW[c] = (c < k && !finish) ? aw_col(gm, l, c) : nullptr;
    }
    const long long o = (long long)l * gm.ld;
    double *X = x64[l];
    const double *R = (const double *)gm.r + o, *Y = (const double *)gm.x + o;
    double *Vv = (double *)gm.p + o;
    double acc = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        double wm = 0.0, awm = 0.0;
#pragma unroll
        for (int c = 0; c < NB; ++c)
            if (c < k) {
                wm += W[c][p] * m[c];
                if (!finish) awm += AW[c][p] * m[c];
            }
        if (finish) {
            X[p] += Y[p] - wm;
        } else {
            X[p] += wm;
            const double v = R[p] - awm;
            Vv[p] = v;
            acc += v * v;
        }
    }
    if (!finish) {
        double a1[1] = {acc};
        __shared__ double out[1];
        block_sum_d<1>(a1, out);
        if (threadIdx.x == 0) atomicAdd(sc + (long long)l * MR_NSC + MR_XI2, out[0]);
    }
}

// dst = src - W mu for the masked lanes (lane blocks of stride ld), with
// ||dst||^2 added into sc[XI2]: one Gram-Schmidt pass of src against W.
__global__ void __launch_bounds__(kThreads)
k_mres_sub(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ mask, const double *__restrict__ src,
           const double *__restrict__ mu, double *__restrict__ dst, double *__restrict__ sc) {
    constexpr int NB = KU_MAX + KP_MAX;
    const int l = blockIdx.y;
    if (l >= ls.nl || mask[l] == 0) return;
    const int k = ls.kdef[l];
    __shared__ double m[NB];
    for (int c = threadIdx.x; c < NB; c += blockDim.x) m[c] = c < k ? mu[(long long)l * KMAX + c] : 0.0;
    __syncthreads();
    const double *W[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) W[c] = c < k ? w_col(gm, l, c) : nullptr;
    const double *S = src + (long long)l * gm.ld;
    double *Dd = dst + (long long)l * gm.ld;
    double acc = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        double v = S[p];
#pragma unroll
        for (int c = 0; c < NB; ++c)
            if (c < k) v -= W[c][p] * m[c];
        Dd[p] = v;
        acc += v * v;
    }
    double a1[1] = {acc};
    __shared__ double out[1];
    block_sum_d<1>(a1, out);
    if (threadIdx.x == 0) atomicAdd(sc + (long long)l * MR_NSC + MR_XI2, out[0]);
}

// After the start: v /= xi; y = d_{k-1} = d_{k-2} = v_{k-1} = 0; CTA (0, l)
// initialises the lane's MINRES scalars and activates it unless xi is
// already at the threshold.
__global__ void __launch_bounds__(kThreads)
k_mres_init(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ mask, double *__restrict__ ext,
            double *__restrict__ sc, int *__restrict__ act) {
    const int l = blockIdx.y;
    if (l >= ls.nl || mask[l] == 0) return;
    double *s = sc + (long long)l * MR_NSC;
    const double xi = sqrt(s[MR_XI2]);
    const double inv = xi > 0.0 ? 1.0 / xi : 0.0;
    const long long o = (long long)l * gm.ld;
    double *Vv = (double *)gm.p + o, *Y = (double *)gm.x + o;
    double *Vp = ext + (3LL * l + 0) * gm.ld, *D1 = ext + (3LL * l + 1) * gm.ld, *D2 = ext + (3LL * l + 2) * gm.ld;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        Vv[p] *= inv;
        Y[p] = 0.0;
        Vp[p] = 0.0;
        D1[p] = 0.0;
        D2[p] = 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s[MR_XI] = xi;
        s[MR_PHI] = xi;
        s[MR_BETA] = 0.0;
        s[MR_C1] = 1.0; s[MR_S1] = 0.0; s[MR_C2] = 1.0; s[MR_S2] = 0.0;
        s[MR_WN2] = 0.0;
        act[l] = (xi > s[MR_THRESH]) ? 1 : 0;
    }
}

// w = q - A~W mu - alpha v - beta_k v_{k-1} (in place in q); sc[WN2] += ||w||^2.
__global__ void __launch_bounds__(kThreads)
k_mres_w(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ act, const double *__restrict__ mu,
         const double *__restrict__ ext, const double *__restrict__ alpha, double *__restrict__ sc) {
    constexpr int NB = KU_MAX + KP_MAX;
    const int l = blockIdx.y;
    if (l >= ls.nl || act[l] == 0) return;
    const int k = ls.kdef[l];
    __shared__ double m[NB];
    for (int c = threadIdx.x; c < NB; c += blockDim.x) m[c] = c < k ? mu[(long long)l * KMAX + c] : 0.0;
    __syncthreads();
    const double *AW[NB];
#pragma unroll
    for (int c = 0; c < NB; ++c) AW[c] = c < k ? aw_col(gm, l, c) : nullptr;
    const double a = alpha[l], b = sc[(long long)l * MR_NSC + MR_BETA];
    const long long o = (long long)l * gm.ld;
    double *Q = (double *)gm.q + o;
    const double *Vv = (const double *)gm.p + o, *Vp = ext + 3LL * l * gm.ld;
    double acc = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        double w = Q[p] - a * Vv[p] - b * Vp[p];
#pragma unroll
        for (int c = 0; c < NB; ++c)
            if (c < k) w -= AW[c][p] * m[c];
        Q[p] = w;
        acc += w * w;
    }
    double a1[1] = {acc};
    __shared__ double out[1];
    block_sum_d<1>(a1, out);
    if (threadIdx.x == 0) atomicAdd(sc + (long long)l * MR_NSC + MR_WN2, out[0]);
}

// The lane's Givens step (one thread per lane): the two previous rotations
// on the new column [beta_k, alpha_k, beta_{k+1}], a new rotation against
// beta_{k+1}, tau = c phibar, phibar <- -s phibar; stores the direction
// coefficients; the lane stops after this step once |phibar| <= thresh,
// gamma or beta_{k+1} vanish, or the iteration budget is spent.
__global__ void k_mres_givens(LaneState ls, const double *__restrict__ alpha, double *__restrict__ sc,
                              int *__restrict__ act, int *__restrict__ step, int nl) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nl) return;
    step[l] = 0;
    if (act[l] == 0) return;
    double *s = sc + (long long)l * MR_NSC;
    const double a = alpha[l], bk = s[MR_BETA], bn = sqrt(s[MR_WN2]);
    const double c1 = s[MR_C1], s1 = s[MR_S1], c2 = s[MR_C2], s2 = s[MR_S2];
    const double eps = s2 * bk, dbar = c2 * bk;
    const double delta = c1 * dbar + s1 * a;
    const double gbar = -s1 * dbar + c1 * a;
    const double gamma = sqrt(gbar * gbar + bn * bn);
    ls.iters[l] += 1;
    if (!(gamma > 0.0) || !isfinite(gamma)) {
        act[l] = 0;
        ls.flag[l] = 2;                       // breakdown: T_k is singular
        return;
    }
    const double c = gbar / gamma, sn = bn / gamma, phi = s[MR_PHI];
    s[MR_TAU] = c * phi;
    s[MR_PHI] = -sn * phi;
    s[MR_GAMMA] = gamma;
    s[MR_DELTA] = delta;
    s[MR_EPS] = eps;
    s[MR_IBETA] = bn > 0.0 ? 1.0 / bn : 0.0;
    s[MR_C2] = c1; s[MR_S2] = s1; s[MR_C1] = c; s[MR_S1] = sn;
    s[MR_BETA] = bn;
    s[MR_WN2] = 0.0;
    step[l] = 1;
    if (fabs(s[MR_PHI]) <= s[MR_THRESH] || bn == 0.0 || ls.iters[l] >= ls.maxit) {
        act[l] = 0;
        ls.flag[l] = 1;
    }
}

// d_k = (v_k - delta d_{k-1} - eps d_{k-2}) / gamma; y += tau d_k;
// d_{k-2} <- d_{k-1}; d_{k-1} <- d_k; v_{k-1} <- v_k; v_k <- w / beta_{k+1}.
__global__ void __launch_bounds__(kThreads)
k_mres_update(long long n, LaneGeom gm, LaneState ls, const int *__restrict__ step, double *__restrict__ ext,
              const double *__restrict__ sc) {
    const int l = blockIdx.y;
    if (l >= ls.nl || step[l] == 0) return;
    const double *s = sc + (long long)l * MR_NSC;
    const double tau = s[MR_TAU], ig = 1.0 / s[MR_GAMMA], delta = s[MR_DELTA], eps = s[MR_EPS], ib = s[MR_IBETA];
    const long long o = (long long)l * gm.ld;
    double *Vv = (double *)gm.p + o, *Y = (double *)gm.x + o;
    const double *Q = (const double *)gm.q + o;
    double *Vp = ext + (3LL * l + 0) * gm.ld, *D1 = ext + (3LL * l + 1) * gm.ld, *D2 = ext + (3LL * l + 2) * gm.ld;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const double v = Vv[p], d1 = D1[p];
        const double d = (v - delta * d1 - eps * D2[p]) * ig;
        Y[p] += tau * d;
        D2[p] = d1;
        D1[p] = d;
        Vp[p] = v;
        Vv[p] = Q[p] * ib;
    }
}

int gx_lanes(long long n, int lanes) {
    long long want = (8LL * 152 + lanes - 1) / lanes;
    long long maxb = (n + kThreads - 1) / kThreads;
    long long gx = want < maxb ? want : maxb;
    return (int)(gx < 1 ? 1 : gx);
}

}  // namespace

void mres_gram(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const int *mask, double *H,
               bool use_w) {
    if (ls.nl <= 0) return;
    RCG_CUDA_TRY(cudaMemsetAsync(H, 0, sizeof(double) * (size_t)ls.m * KMAX * KMAX, st));
    dim3 grid(gx_lanes(n, ls.nl * 4), ls.nl, KU_MAX + KP_MAX);
    k_mres_gram<<<grid, kThreads, 0, st>>>(n, gm, ls, mask, H, use_w ? 1 : 0);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void mres_dots(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const int *mask,
               const double *src, double *hd, bool use_w) {
    if (ls.nl <= 0) return;
    RCG_CUDA_TRY(cudaMemsetAsync(hd, 0, sizeof(double) * (size_t)ls.m * KMAX, st));
    k_mres_dots<<<dim3(gx_lanes(n, ls.nl), ls.nl), kThreads, 0, st>>>(n, gm, ls, mask, src, hd, use_w ? 1 : 0);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void mres_sub(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const int *mask,
              const double *src, const double *mu, double *dst, double *sc) {
    if (ls.nl <= 0) return;
    k_mres_sub<<<dim3(gx_lanes(n, ls.nl), ls.nl), kThreads, 0, st>>>(n, gm, ls, mask, src, mu, dst, sc);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void mres_mu(cudaStream_t st, const LaneState &ls, const int *mask, const double *hd, double *mu, double *sc) {
    if (ls.nl <= 0) return;
    k_mres_mu<<<ls.nl, 32, 0, st>>>(ls, mask, hd, mu, sc);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void mres_cycle(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const int *mask,
                const double *mu, double *const *x64, double *sc, bool finish) {
    if (ls.nl <= 0) return;
    k_mres_cycle<<<dim3(gx_lanes(n, ls.nl), ls.nl), kThreads, 0, st>>>(n, gm, ls, mask, mu, x64, sc, finish ? 1 : 0);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void mres_init(cudaStream_t st, long long n, const LaneGeom &gm, const LaneState &ls, const int *mask, double *ext,
               double *sc, int *act) {
    if (ls.nl <= 0) return;
    k_mres_init<<<dim3(gx_lanes(n, ls.nl), ls.nl), kThreads, 0, st>>>(n, gm, ls, mask, ext, sc, act);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void mres_iteration(cudaStream_t st, const Grid &g, const double *D, const double *const *diag_of_col,
                    const double *const *v_ptr, double *const *q_ptr, const LaneGeom &gm, const LaneState &ls,
                    int *act, int *step, double *alpha, double *hd, double *mu, double *ext, double *sc) {
    if (ls.nl <= 0) return;
    RCG_CUDA_TRY(cudaMemsetAsync(alpha, 0, sizeof(double) * (size_t)ls.nl, st));
    apply_op<double>(st, g, D, diag_of_col, v_ptr, q_ptr, ls.nl, act, alpha, nullptr);      // q = A~ v, alpha
    mres_dots(st, g.n, gm, ls, act, (const double *)gm.q, hd);                              // (A~W)^T q
    mres_mu(st, ls, act, hd, mu, sc);
    k_mres_w<<<dim3(gx_lanes(g.n, ls.nl), ls.nl), kThreads, 0, st>>>(g.n, gm, ls, act, mu, ext, alpha, sc);
    count_launch();
    RCG_CHECK_LAUNCH();
    k_mres_givens<<<(ls.nl + 127) / 128, 128, 0, st>>>(ls, alpha, sc, act, step, ls.nl);
    count_launch();
    RCG_CHECK_LAUNCH();
    k_mres_update<<<dim3(gx_lanes(g.n, ls.nl), ls.nl), kThreads, 0, st>>>(g.n, gm, ls, step, ext, sc);
    count_launch();
    RCG_CHECK_LAUNCH();
}

}  // namespace rcg
