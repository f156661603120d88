// Set-up and bookkeeping kernels: the operator diagonal of A~_* (Sec. 3:
// face weights plus the Robin term left by eliminating the boundary rows),
// sample diagonals and Delta weights (eq. sum), effective source weights
// (Sec. 3.1), lane gathers, and the small index shuffles of the append.
#include "common.cuh"

#include <algorithm>

namespace rcg {
namespace {

// diag_*[p] = sum over the faces of node p of
//   (D_p + D_q)/2  towards an unknown q,
//   D_p            towards a lateral (Dirichlet) ghost,
//   D_p/(1+alpha_p) towards a Robin face, alpha_p = 2 A D_p / h.
__global__ void k_diag_star(Grid g, const double *__restrict__ D, double h, double robin_A, double *__restrict__ out) {
    const long long sxy = (long long)g.Nx * g.Ny;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.n;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.Nx);
        const long long rest = p / g.Nx;
        const int j = (int)(rest % g.Ny);
        const int k = (int)(rest / g.Ny);
        const double Dp = D[p];
        double s = 0.0;
        s += i > 0 ? 0.5 * (Dp + D[p - 1]) : Dp;
        s += i < g.Nx - 1 ? 0.5 * (Dp + D[p + 1]) : Dp;
        if (g.Ny > 1) {
            s += j > 0 ? 0.5 * (Dp + D[p - g.Nx]) : Dp;
            s += j < g.Ny - 1 ? 0.5 * (Dp + D[p + g.Nx]) : Dp;
        }
        const double robin = Dp / (1.0 + 2.0 * robin_A * Dp / h);
        s += k > 0 ? 0.5 * (Dp + D[p - sxy]) : robin;
        s += k < g.Nz - 1 ? 0.5 * (Dp + D[p + sxy]) : robin;
        out[p] = s;
    }
}

// diag_s = diag_* + h^2 mu (float64 and float32 copies)
__global__ void k_diag_sample(long long n, const double *__restrict__ dstar, const double *__restrict__ mu, double h2,
                              double *__restrict__ d64, float *__restrict__ d32) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const double v = dstar[p] + h2 * mu[p];
        d64[p] = v;
        if (d32) d32[p] = (float)v;
    }
}

// w = scale * (a - b)   (Delta weights h^2 (mu_s - mu_*) and -h^2 dmu_k)
__global__ void k_scaled_diff(long long n, const double *__restrict__ a, const double *__restrict__ b, double scale,
                              double *__restrict__ w) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        w[p] = scale * (a[p] - (b ? b[p] : 0.0));
}

template <typename TS, typename TD>
__global__ void k_convert_lanes(long long n, const TS *const *__restrict__ src, const int *__restrict__ lanes,
                                TD *__restrict__ dst, long long ldd) {
    const int j = blockIdx.y;
    const TS *s = src[lanes[j]];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        dst[(long long)j * ldd + p] = (TD)s[p];
}

__global__ void __launch_bounds__(256)
k_norm2_lanes(long long n, const double *const *__restrict__ src, const int *__restrict__ lanes, double *out) {
    const int j = blockIdx.y;
    const double *s = src[lanes[j]];
    double acc = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        acc += s[p] * s[p];
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s2 = 0;
        for (int w = 0; w < 8; ++w) s2 += red[w];
        atomicAdd(out + j, s2);
    }
}

// Write the border block B ((r0 + a) x a: rows 0..r0+a-1 of the new
// columns r0..r0+a-1) into the symmetric matrix C (ld ldc), mirrored; the
// new-by-new block is symmetrised by averaging.
__global__ void k_border_write(double *C, int ldc, int r0, int a, const double *B, int ldb) {
    const long long tot = (long long)(r0 + a) * a;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % (r0 + a)), j = (int)(e / (r0 + a));
        const int cj = r0 + j;
        double v = B[i + (long long)j * ldb];
        if (i >= r0) {
            const int jj = i - r0;                  // (cj, i) is also in B as (r0 + j, jj)
            v = 0.5 * (v + B[(r0 + j) + (long long)jj * ldb]);
        }
        C[i + (long long)cj * ldc] = v;
        C[cj + (long long)i * ldc] = v;
    }
}

// Copy rows r0..r0+a-1, columns 0..r0+a-1 of G into L (same ld): the new
// rows of a bordered Cholesky.
__global__ void k_copy_new_rows(const double *G, double *L, int ld, int r0, int a) {
    const long long tot = (long long)a * (r0 + a);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = r0 + (int)(e % a), j = (int)(e / a);
        L[i + (long long)j * ld] = G[i + (long long)j * ld];
    }
}

// R_K = R restricted to kept rows/cols (upper, ak x ak, ld ak)
__global__ void k_gather_sub(const double *R, int a, const int *K, int ak, double *RK) {
    const long long tot = (long long)ak * ak;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % ak), j = (int)(e / ak);
        RK[e] = (i <= j) ? R[K[i] + (long long)K[j] * a] : 0.0;
    }
}

// Rhat (a x ak): row K[i] = row i of Rinv (ak x ak), other rows zero.
__global__ void k_scatter_rows(const double *Rinv, int ak, const int *K, int a, double *Rhat) {
    const long long tot = (long long)a * ak;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) Rhat[e] = 0.0;
    __syncthreads();
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < (long long)ak * ak;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % ak), j = (int)(e / ak);
        Rhat[K[i] + (long long)j * a] = Rinv[i + (long long)j * ak];
    }
}

// Upper factor R2 = L^T from a lower Cholesky factor L (a x a, ld lda).
__global__ void k_lower_to_upper(const double *L, int lda, int a, double *R) {
    const long long tot = (long long)a * a;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % a), j = (int)(e / a);
        R[i + (long long)j * a] = (i <= j) ? L[j + (long long)i * lda] : 0.0;
    }
}

// Per lane: the deflation Galerkin matrix G_W = S^T G_s S from the basis
// Galerkin matrix G_s = V^T A~_s V, where the lane's deflation columns are
// either basis columns (spec >= 0: S column = unit vector) or the lane's
// seed solution X_0(:, j) (spec == -1: S column = sx = V^T X_0(:, j)).
__global__ void __launch_bounds__(256)
k_lane_gw(const double *const *__restrict__ Gs, int ldg, int r, const int *__restrict__ spec,
          const double *const *__restrict__ sx, const int *__restrict__ kdef, double *__restrict__ gw) {
    extern __shared__ double gsx[];   // r entries: G_s sx
    __shared__ double sgs;
    const int l = blockIdx.x;
    const int k = kdef[l];
    const double *G = Gs[l];
    const int *sp = spec + (long long)l * KMAX;
    bool has_x = false;
    for (int c = 0; c < k; ++c) has_x |= (sp[c] < 0);
    if (has_x) {
        const double *s = sx[l];
        for (int q = threadIdx.x; q < r; q += blockDim.x) {
            double acc = 0.0;
            for (int q2 = 0; q2 < r; ++q2) acc += G[q + (long long)q2 * ldg] * s[q2];
            gsx[q] = acc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double acc = 0.0;
            for (int q = 0; q < r; ++q) acc += s[q] * gsx[q];
            sgs = acc;
        }
        __syncthreads();
    }
    double *out = gw + (long long)l * KMAX * KMAX;
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int a = e % k, b = e / k;
        const int ia = sp[a], ib = sp[b];
        double v;
        if (ia >= 0 && ib >= 0) v = G[ia + (long long)ib * ldg];
        else if (ia >= 0) v = gsx[ia];
        else if (ib >= 0) v = gsx[ib];
        else v = sgs;
        out[a + b * KMAX] = v;
    }
}

template <typename T>
__global__ void k_gather_cols(long long n, const T *const *__restrict__ src, T *__restrict__ dst, long long ld) {
    const int j = blockIdx.y;
    const T *s = src[j];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        dst[(long long)j * ld + p] = s[p];
}

// Counter-based pseudo-random fill in [-1, 1): SplitMix64 of (seed, index).
template <typename T>
__global__ void k_rand_fill(T *__restrict__ X, long long n, long long ld, int b, unsigned long long seed) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n * b;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / n, p = e % n;
        unsigned long long z = seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(e + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z ^= z >> 31;
        X[j * ld + p] = (T)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    }
}

// out = alpha * AY + beta * Y + gamma * Yp over b columns (Chebyshev step)
template <typename T>
__global__ void k_cheb_step(T *__restrict__ out, const T *__restrict__ AY, const T *__restrict__ Y,
                            const T *__restrict__ Yp, long long n, long long ld, int b, T alpha, T beta, T gamma) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n * b;
         e += (long long)gridDim.x * blockDim.x) {
        const long long j = e / n, p = e % n, q = j * ld + p;
        T v = alpha * AY[q] + beta * Y[q];
        if (Yp) v += gamma * Yp[q];
        out[q] = v;
    }
}

// Gershgorin bound of A~_s: max_p diag_s[p] + sum of off-diagonal |w|.
__global__ void k_gershgorin(Grid g, const double *__restrict__ D, const double *__restrict__ diag,
                             unsigned long long *__restrict__ out) {
    const long long sxy = (long long)g.Nx * g.Ny;
    double best = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < g.n;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.Nx);
        const long long rest = p / g.Nx;
        const int j = (int)(rest % g.Ny);
        const int k = (int)(rest / g.Ny);
        const double Dp = D[p];
        double s = diag[p];
        if (i > 0) s += 0.5 * (Dp + D[p - 1]);
        if (i < g.Nx - 1) s += 0.5 * (Dp + D[p + 1]);
        if (g.Ny > 1 && j > 0) s += 0.5 * (Dp + D[p - g.Nx]);
        if (g.Ny > 1 && j < g.Ny - 1) s += 0.5 * (Dp + D[p + g.Nx]);
        if (k > 0) s += 0.5 * (Dp + D[p - sxy]);
        if (k < g.Nz - 1) s += 0.5 * (Dp + D[p + sxy]);
        best = s > best ? s : best;
    }
    // positive doubles order like their bit patterns
    atomicMax(out, (unsigned long long)__double_as_longlong(best));
}

// res2[j] = || AX_j - theta_j X_j ||^2
template <typename T>
__global__ void __launch_bounds__(256)
k_ritz_res(const T *__restrict__ AX, const T *__restrict__ X, const double *__restrict__ theta, long long n,
           long long ld, double *__restrict__ res2) {
    const int j = blockIdx.y;
    double acc = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const double v = (double)AX[j * ld + p] - theta[j] * (double)X[j * ld + p];
        acc += v * v;
    }
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < 8; ++w) s += red[w];
        atomicAdd(res2 + j, s);
    }
}

int nblk(long long n) {
    long long b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

void diag_star(cudaStream_t st, const Grid &g, const double *D, double h, double A, double *out) {
    k_diag_star<<<nblk(g.n), 256, 0, st>>>(g, D, h, A, out);
    count_launch();
    RCG_CHECK_LAUNCH();
}
void diag_sample(cudaStream_t st, long long n, const double *dstar, const double *mu, double h2, double *d64,
                 float *d32) {
    k_diag_sample<<<nblk(n), 256, 0, st>>>(n, dstar, mu, h2, d64, d32);
    count_launch();
    RCG_CHECK_LAUNCH();
}
void scaled_diff(cudaStream_t st, long long n, const double *a, const double *b, double scale, double *w) {
    k_scaled_diff<<<nblk(n), 256, 0, st>>>(n, a, b, scale, w);
    count_launch();
    RCG_CHECK_LAUNCH();
}
template <typename TS, typename TD>
void convert_lanes(cudaStream_t st, long long n, const TS *const *src, const int *lanes, int nl, TD *dst,
                   long long ldd) {
    if (nl <= 0) return;
    dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 1024), nl);
    k_convert_lanes<TS, TD><<<grid, 256, 0, st>>>(n, src, lanes, dst, ldd);
    count_launch();
    RCG_CHECK_LAUNCH();
}
template void convert_lanes<double, float>(cudaStream_t, long long, const double *const *, const int *, int, float *,
                                           long long);
template void convert_lanes<double, double>(cudaStream_t, long long, const double *const *, const int *, int,
                                            double *, long long);
void norm2_lanes(cudaStream_t st, long long n, const double *const *src, const int *lanes, int nl, double *out) {
    if (nl <= 0) return;
    RCG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double) * nl, st));
    dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 256), nl);
    k_norm2_lanes<<<grid, 256, 0, st>>>(n, src, lanes, out);
    count_launch();
    RCG_CHECK_LAUNCH();
}
void border_write(cudaStream_t st, double *C, int ldc, int r0, int a, const double *B, int ldb) {
    k_border_write<<<nblk((long long)(r0 + a) * a), 256, 0, st>>>(C, ldc, r0, a, B, ldb);
    count_launch();
    RCG_CHECK_LAUNCH();
}
void copy_new_rows(cudaStream_t st, const double *G, double *L, int ld, int r0, int a) {
    k_copy_new_rows<<<nblk((long long)a * (r0 + a)), 256, 0, st>>>(G, L, ld, r0, a);
    count_launch();
    RCG_CHECK_LAUNCH();
}
void gather_sub(cudaStream_t st, const double *R, int a, const int *K, int ak, double *RK) {
    k_gather_sub<<<nblk((long long)ak * ak), 256, 0, st>>>(R, a, K, ak, RK);
    count_launch();
    RCG_CHECK_LAUNCH();
}
void scatter_rows(cudaStream_t st, const double *Rinv, int ak, const int *K, int a, double *Rhat) {
    k_scatter_rows<<<1, 1024, 0, st>>>(Rinv, ak, K, a, Rhat);
    count_launch();
    RCG_CHECK_LAUNCH();
}
void lower_to_upper(cudaStream_t st, const double *L, int lda, int a, double *R) {
    k_lower_to_upper<<<nblk((long long)a * a), 256, 0, st>>>(L, lda, a, R);
    count_launch();
    RCG_CHECK_LAUNCH();
}
void lane_gw(cudaStream_t st, const double *const *Gs, int ldg, int r, const int *spec, const double *const *sx,
             const int *kdef, double *gw, int m) {
    if (m <= 0) return;
    const size_t sh = sizeof(double) * (size_t)(r > 0 ? r : 1);
    if (sh > 48 * 1024)
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_lane_gw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh));
    k_lane_gw<<<m, 256, sh, st>>>(Gs, ldg, r, spec, sx, kdef, gw);
    count_launch();
    RCG_CHECK_LAUNCH();
}

template <typename T>
void gather_cols(cudaStream_t st, long long n, const T *const *src, T *dst, long long ld, int count) {
    if (count <= 0) return;
    dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 1024), count);
    k_gather_cols<T><<<grid, 256, 0, st>>>(n, src, dst, ld);
    count_launch();
    RCG_CHECK_LAUNCH();
}
template void gather_cols<double>(cudaStream_t, long long, const double *const *, double *, long long, int);
template void gather_cols<float>(cudaStream_t, long long, const float *const *, float *, long long, int);

template <typename T>
void rand_fill(cudaStream_t st, T *X, long long n, long long ld, int b, unsigned long long seed) {
    k_rand_fill<T><<<nblk(n * b), 256, 0, st>>>(X, n, ld, b, seed);
    count_launch();
    RCG_CHECK_LAUNCH();
}
template void rand_fill<double>(cudaStream_t, double *, long long, long long, int, unsigned long long);
template void rand_fill<float>(cudaStream_t, float *, long long, long long, int, unsigned long long);

template <typename T>
void cheb_step(cudaStream_t st, T *out, const T *AY, const T *Y, const T *Yp, long long n, long long ld, int b,
               double alpha, double beta, double gamma) {
    k_cheb_step<T><<<nblk(n * b), 256, 0, st>>>(out, AY, Y, Yp, n, ld, b, (T)alpha, (T)beta, (T)gamma);
    count_launch();
    RCG_CHECK_LAUNCH();
}
template void cheb_step<double>(cudaStream_t, double *, const double *, const double *, const double *, long long,
                                long long, int, double, double, double);
template void cheb_step<float>(cudaStream_t, float *, const float *, const float *, const float *, long long,
                               long long, int, double, double, double);

void gershgorin(cudaStream_t st, const Grid &g, const double *D, const double *diag, unsigned long long *out) {
    RCG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(unsigned long long), st));
    k_gershgorin<<<nblk(g.n), 256, 0, st>>>(g, D, diag, out);
    count_launch();
    RCG_CHECK_LAUNCH();
}

template <typename T>
void ritz_res(cudaStream_t st, const T *AX, const T *X, const double *theta, long long n, long long ld, int b,
              double *res2) {
    RCG_CUDA_TRY(cudaMemsetAsync(res2, 0, sizeof(double) * b, st));
    dim3 grid((unsigned)std::min<long long>((n + 255) / 256, 256), b);
    k_ritz_res<T><<<grid, 256, 0, st>>>(AX, X, theta, n, ld, res2);
    count_launch();
    RCG_CHECK_LAUNCH();
}
template void ritz_res<double>(cudaStream_t, const double *, const double *, const double *, long long, long long,
                               int, double *);
template void ritz_res<float>(cudaStream_t, const float *, const float *, const double *, long long, long long, int,
                              double *);

}  // namespace rcg
