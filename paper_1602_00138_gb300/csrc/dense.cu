// Tall-skinny dense products on CUDA cores: C = A^T diag(w) B (split over
// the long dimension n, float64 accumulation across splits), Out = A Y,
// row gathers V^T b~ for point right-hand sides, conversions and dots.
// These serve the Galerkin check (Algorithm 2, "check if V is a good enough
// space"), the ordered append (Sec. 5.3 incremental QR of the basis) and
// the reduced model (eq. newreduced).
#include "common.cuh"
#include "../../include/rcg.h"

#include <type_traits>

namespace rcg {
namespace {

constexpr int TN_T = 32;      // output tile (A columns x B columns)
constexpr int TN_BK = 32;     // rows per shared-memory stage

template <typename T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

// C[i + j*ldc] += sum_p w[p] A_i[p] B_j[p] over this CTA's row range, with
// products and partial sums in AT.
template <typename TA, typename TB, typename AT>
__global__ void __launch_bounds__(256)
k_gemm_tn(long long n, const TA *__restrict__ A, long long lda, int ka, const TB *__restrict__ B,
          long long ldb, int kb, double *__restrict__ C, int ldc, const double *__restrict__ wt,
          const int *__restrict__ rows, long long nrows, long long chunk) {
    __shared__ AT As[TN_BK][TN_T + 1];
    __shared__ AT Bs[TN_BK][TN_T + 1];
    const int i0 = blockIdx.x * TN_T, j0 = blockIdx.y * TN_T;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const long long len = rows ? nrows : n;
    const long long r0 = (long long)blockIdx.z * chunk;
    const long long r1 = (r0 + chunk < len) ? r0 + chunk : len;
    double accd[2][2] = {{0, 0}, {0, 0}};
    AT acc[2][2] = {{0, 0}, {0, 0}};
    int since_flush = 0;
    for (long long base = r0; base < r1; base += TN_BK) {
        if (wt) {   // skip row chunks where the weight vanishes (finite support of Delta)
            int nz = 0;
            if (threadIdx.x < TN_BK) {
                const long long q = base + threadIdx.x;
                if (q < r1) nz = wt[rows ? (long long)rows[q] : q] != 0.0;
            }
            if (!__syncthreads_or(nz)) continue;
        }
        for (int e = threadIdx.x; e < TN_BK * TN_T; e += 256) {
            const int rr = e % TN_BK, cc = e / TN_BK;
            const long long q = base + rr;
            AT av = 0, bv = 0;
            if (q < r1) {
                const long long p = rows ? (long long)rows[q] : q;
                if (i0 + cc < ka) {
                    av = (AT)A[(long long)(i0 + cc) * lda + p];
                    if (wt) av = av * (AT)wt[p];
                }
                if (j0 + cc < kb) bv = (AT)B[(long long)(j0 + cc) * ldb + p];
            }
            As[rr][cc] = av;
            Bs[rr][cc] = bv;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < TN_BK; ++kk) {
            const AT a0 = As[kk][ty], a1 = As[kk][ty + 16];
            const AT b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            acc[0][0] += a0 * b0; acc[0][1] += a0 * b1;
            acc[1][0] += a1 * b0; acc[1][1] += a1 * b1;
        }
        __syncthreads();
        if (!std::is_same<AT, double>::value && ++since_flush == 8) {
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) { accd[a][b] += (double)acc[a][b]; acc[a][b] = 0; }
            since_flush = 0;
        }
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
            const double v = accd[a][b] + (double)acc[a][b];
            if (i < ka && j < kb && v != 0.0) atomicAdd(C + i + (long long)j * ldc, v);
        }
}

// C[i + j*ldc] += sum_p A_i[p] B_j[p] for few B columns (kb <= 4): each CTA
// owns 8 A columns and a row chunk; every A element is read once.
template <typename TA, typename TB, typename AT, int KB>
__global__ void __launch_bounds__(256)
k_gemv_t(long long n, const TA *__restrict__ A, long long lda, int ka, const TB *__restrict__ B, long long ldb,
         double *__restrict__ C, int ldc, long long chunk) {
    const int i0 = blockIdx.x * 8;
    const long long r0 = (long long)blockIdx.y * chunk;
    const long long r1 = (r0 + chunk < n) ? r0 + chunk : n;
    AT acc[8][KB];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < KB; ++b) acc[a][b] = AT(0);
    for (long long p = r0 + threadIdx.x; p < r1; p += blockDim.x) {
        AT bv[KB];
#pragma unroll
        for (int b = 0; b < KB; ++b) bv[b] = (AT)B[(long long)b * ldb + p];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
            if (i0 + a >= ka) break;
            const AT av = (AT)A[(long long)(i0 + a) * lda + p];
#pragma unroll
            for (int b = 0; b < KB; ++b) acc[a][b] += av * bv[b];
        }
    }
    __shared__ double red[8][8][KB];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < KB; ++b) {
            double v = (double)acc[a][b];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][a][b] = v;
        }
    __syncthreads();
    if (threadIdx.x < 8 * KB) {
        const int a = threadIdx.x / KB, b = threadIdx.x % KB;
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w][a][b];
        if (i0 + a < ka && v != 0.0) atomicAdd(C + (i0 + a) + (long long)b * ldc, v);
    }
}

constexpr int NN_MN = 16;     // output columns per CTA
constexpr int NN_KC = 32;     // basis columns per shared-memory stage

// Out_j[p] = beta Out_j[p] + alpha sum_c A_c[p] Y[c + j*ldy]
template <typename TA, typename TO, int NN_MN>
__global__ void __launch_bounds__(256)
k_gemm_nn(long long n, const TA *__restrict__ A, long long lda, int k, const double *__restrict__ Y,
          int ldy, int m, TO *__restrict__ Out, long long ldo, double alpha, double beta) {
    using AT = typename Acc<TA>::type;
    __shared__ AT Ys[NN_KC][NN_MN];
    const int j0 = blockIdx.y * NN_MN;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double accd[NN_MN];
#pragma unroll
    for (int j = 0; j < NN_MN; ++j) accd[j] = 0.0;
    for (int c0 = 0; c0 < k; c0 += NN_KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < NN_KC * NN_MN; e += blockDim.x) {
            const int cc = e % NN_KC, jj = e / NN_KC;
            double v = 0.0;
            if (c0 + cc < k && j0 + jj < m) v = Y[(c0 + cc) + (long long)(j0 + jj) * ldy];
            Ys[cc][jj] = (AT)v;
        }
        __syncthreads();
        if (p < n) {
            AT acc[NN_MN];
#pragma unroll
            for (int j = 0; j < NN_MN; ++j) acc[j] = 0;
            const int cend = (k - c0) < NN_KC ? (k - c0) : NN_KC;
            for (int cc = 0; cc < cend; ++cc) {
                const AT a = (AT)A[(long long)(c0 + cc) * lda + p];
#pragma unroll
                for (int j = 0; j < NN_MN; ++j) acc[j] += a * Ys[cc][j];
            }
#pragma unroll
            for (int j = 0; j < NN_MN; ++j) accd[j] += (double)acc[j];
        }
    }
    if (p < n) {
#pragma unroll
        for (int j = 0; j < NN_MN; ++j) {
            if (j0 + j >= m) break;
            TO *o = Out + (long long)(j0 + j) * ldo + p;
            const double old = (beta != 0.0) ? (double)*o : 0.0;
            *o = (TO)(beta * old + alpha * accd[j]);
        }
    }
}

// Out_j[p] = beta Out_j[p] + sum_c V_c[p] Y[c + j*ldy] with V float32, Y and
// Out float64, accumulated as unevaluated float32 pairs (hi + lo): each
// product v*y_hi is split exactly with an FMA (TwoProd), v*y_lo joins the
// error term, and the running sum is compensated (TwoSum).  The result is
// accurate to ~1e-13 relative at float32 instruction cost; a plain float32
// accumulation would leave ~1e-7 relative noise in the lifted vector, which
// the operator amplifies into the Galerkin residual.
template <int MN>
__global__ void __launch_bounds__(256)
k_gemm_nn_df(long long n, const float *__restrict__ V, long long ldv, int k, const double *__restrict__ Y, int ldy,
             int m, double *__restrict__ Out, long long ldo, double beta) {
    __shared__ float Yh[NN_KC][MN], Yl[NN_KC][MN];
    const int j0 = blockIdx.y * MN;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float sh[MN], sl[MN];
#pragma unroll
    for (int j = 0; j < MN; ++j) { sh[j] = 0.f; sl[j] = 0.f; }
    for (int c0 = 0; c0 < k; c0 += NN_KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < NN_KC * MN; e += blockDim.x) {
            const int cc = e % NN_KC, jj = e / NN_KC;
            double v = 0.0;
            if (c0 + cc < k && j0 + jj < m) v = Y[(c0 + cc) + (long long)(j0 + jj) * ldy];
            const float hi = (float)v;
            Yh[cc][jj] = hi;
            Yl[cc][jj] = (float)(v - (double)hi);
        }
        __syncthreads();
        if (p < n) {
            const int cend = (k - c0) < NN_KC ? (k - c0) : NN_KC;
            for (int cc = 0; cc < cend; ++cc) {
                const float a = V[(long long)(c0 + cc) * ldv + p];
#pragma unroll
                for (int j = 0; j < MN; ++j) {
                    // _rn intrinsics keep the compiler from contracting these into FMAs,
                    // which would break the error-free transformations
                    const float prod = __fmul_rn(a, Yh[cc][j]);
                    float err = fmaf(a, Yh[cc][j], -prod);     // exact: a*y_hi = prod + err
                    err = fmaf(a, Yl[cc][j], err);
                    const float t = __fadd_rn(sh[j], prod);     // TwoSum(sh, prod)
                    const float bp = __fsub_rn(t, sh[j]);
                    const float e2 = __fadd_rn(__fsub_rn(sh[j], __fsub_rn(t, bp)), __fsub_rn(prod, bp));
                    sh[j] = t;
                    sl[j] += e2 + err;
                }
            }
        }
    }
    if (p < n) {
#pragma unroll
        for (int j = 0; j < MN; ++j) {
            if (j0 + j >= m) break;
            double *o = Out + (long long)(j0 + j) * ldo + p;
            const double v = (double)sh[j] + (double)sl[j];
            *o = (beta != 0.0) ? beta * *o + v : v;
        }
    }
}

// C (+)= A^T B with A float32 and B float64 (the float32 basis against float64
// stencil images: the border of the cached Galerkin matrix), in double-float
// arithmetic on float32 units: B is split into hi + lo when staged, each
// product a*b_hi is split exactly (TwoProd), a*b_lo joins the error term,
// and the running sums are compensated (TwoSum).  ~1e-13 relative; GB300's
// float64 units are ~1/64 of its float32 rate.  Partial sums of the CTA's
// row range go to C by float64 atomics.
__global__ void __launch_bounds__(256)
k_gemm_tn_df(long long n, const float *__restrict__ A, long long lda, int ka, const double *__restrict__ B,
             long long ldb, int kb, double *__restrict__ C, int ldc, long long chunk) {
    __shared__ float As[TN_BK][TN_T + 1], Bh[TN_BK][TN_T + 1], Bl[TN_BK][TN_T + 1];
    const int i0 = blockIdx.x * TN_T, j0 = blockIdx.y * TN_T;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const long long r0 = (long long)blockIdx.z * chunk;
    const long long r1 = (r0 + chunk < n) ? r0 + chunk : n;
    float sh[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, sl[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
    for (long long base = r0; base < r1; base += TN_BK) {
        for (int e = threadIdx.x; e < TN_BK * TN_T; e += 256) {
            const int rr = e % TN_BK, cc = e / TN_BK;
            const long long q = base + rr;
            float av = 0.f, bh = 0.f, bl = 0.f;
            if (q < r1) {
                if (i0 + cc < ka) av = A[(long long)(i0 + cc) * lda + q];
                if (j0 + cc < kb) {
                    const double bv = B[(long long)(j0 + cc) * ldb + q];
                    bh = (float)bv;
                    bl = (float)(bv - (double)bh);
                }
            }
            As[rr][cc] = av;
            Bh[rr][cc] = bh;
            Bl[rr][cc] = bl;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < TN_BK; ++kk) {
            const float a[2] = {As[kk][ty], As[kk][ty + 16]};
            const float h[2] = {Bh[kk][tx], Bh[kk][tx + 16]}, l[2] = {Bl[kk][tx], Bl[kk][tx + 16]};
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    const float prod = __fmul_rn(a[u], h[v]);
                    float err = fmaf(a[u], h[v], -prod);          // exact: a*b_hi = prod + err
                    err = fmaf(a[u], l[v], err);
                    const float t = __fadd_rn(sh[u][v], prod);     // TwoSum(sh, prod)
                    const float bp = __fsub_rn(t, sh[u][v]);
                    const float e2 = __fadd_rn(__fsub_rn(sh[u][v], __fsub_rn(t, bp)), __fsub_rn(prod, bp));
                    sh[u][v] = t;
                    sl[u][v] = __fadd_rn(sl[u][v], __fadd_rn(e2, err));
                }
        }
        __syncthreads();
    }
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
            const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
            const double val = (double)sh[u][v] + (double)sl[u][v];
            if (i < ka && j < kb && val != 0.0) atomicAdd(C + i + (long long)j * ldc, val);
        }
}

template <typename TV>
__global__ void k_gather_rows(const TV *__restrict__ V, long long ldv, int r, const int *__restrict__ node,
                              const double *__restrict__ w, int m, double *__restrict__ out, int ldo) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)r * m) return;
    const int c = (int)(e % r), j = (int)(e / r);
    out[c + (long long)j * ldo] = w[j] * (double)V[(long long)c * ldv + node[j]];
}

template <typename TS, typename TD>
__global__ void k_convert(long long n, const TS *__restrict__ s, long long lds, TD *__restrict__ d,
                          long long ldd, int ncols) {
    const int j = blockIdx.y;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        d[(long long)j * ldd + p] = (TD)s[(long long)j * lds + p];
}

template <typename T>
__global__ void __launch_bounds__(256)
k_col_dots(long long n, const T *__restrict__ A, long long lda, const T *__restrict__ B, long long ldb,
           double *__restrict__ out) {
    const int j = blockIdx.y;
    double acc = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        acc += (double)A[(long long)j * lda + p] * (double)B[(long long)j * ldb + p];
    __shared__ double red[8];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < 8; ++w) s += red[w];
        atomicAdd(out + j, s);
    }
}

__global__ void k_add_f32_f64(long long n, double *__restrict__ x, long long ldx, const float *__restrict__ d,
                              long long ldd, const int *__restrict__ lanes) {
    const int l = lanes[blockIdx.y];
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x)
        x[(long long)l * ldx + p] += (double)d[(long long)l * ldd + p];
}

// J_k[:, s] = Z^T (G_k X[:, s]) for CTA (s, k): the reduced Jacobian of the
// transfer function (CS-3: dPsi_r/dp_k = -Z_r^T V^T diag(h^2 dmu_k) V X_r,
// with the sign and h^2 folded into G_k).  G_k r x r (ld r, symmetric),
// X r x ns, Z r x nd (ld r), J_k nd x ns.  One column of G_k X per CTA in
// shared memory; float64 (few FMAs per CTA, spread over the whole GPU).
__global__ void __launch_bounds__(256)
k_rom_jac(int r, const double *__restrict__ G, const double *__restrict__ X, int ns, const double *__restrict__ Z,
          int nd, double *__restrict__ J) {
    extern __shared__ double t[];             // r + r: x column, then G_k x
    const int s = blockIdx.x, k = blockIdx.y, q = blockIdx.z, nparam = gridDim.y;
    const double *Gk = G + ((long long)q * nparam + k) * r * r;
    X += (long long)q * r * ns;
    Z += (long long)q * r * nd;
    J += (long long)q * nparam * nd * ns;
    double *xs = t, *gx = t + r;
    for (int i = threadIdx.x; i < r; i += blockDim.x) xs[i] = X[(long long)s * r + i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < r; i += nw) {      // (G_k x)_i = G_k[:, i] . x (G_k symmetric: a contiguous column)
        double a = 0.0;
        for (int j = lane; j < r; j += 32) a += Gk[(long long)i * r + j] * xs[j];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) gx[i] = a;
    }
    __syncthreads();
    for (int d = warp; d < nd; d += nw) {
        double a = 0.0;
        for (int j = lane; j < r; j += 32) a += Z[(long long)d * r + j] * gx[j];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) J[((long long)k * ns + s) * nd + d] = a;
    }
}

// Psi_q[d + nd s] = Crm[:, d] . X_q[:, s] for CTA (s, q), one warp per d.
__global__ void __launch_bounds__(256)
k_rom_psi(int r, const double *__restrict__ Crm, const double *__restrict__ X, int ns, int nd,
          double *__restrict__ Psi) {
    const int s = blockIdx.x, q = blockIdx.y;
    const double *x = X + ((long long)q * ns + s) * r;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int d = warp; d < nd; d += nw) {
        double a = 0.0;
        for (int j = lane; j < r; j += 32) a += Crm[(long long)d * r + j] * x[j];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) Psi[((long long)q * ns + s) * nd + d] = a;
    }
}

// dst[c][0 .. n) = src[c][0 .. n) for c = blockIdx.y (columns 16-byte aligned
// when vec4: float4 body, scalar tail).
template <typename T>
__global__ void k_copy_cols(long long n, const T *const *__restrict__ src, T *const *__restrict__ dst, int vec4) {
    const T *s = src[blockIdx.y];
    T *d = dst[blockIdx.y];
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long p0 = 0;
    if (vec4 && sizeof(T) == 4) {
        const long long n4 = n >> 2;
        for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n4; v += stride)
            ((float4 *)d)[v] = ((const float4 *)s)[v];
        p0 = n4 << 2;
    }
    for (long long p = p0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) d[p] = s[p];
}

int blocks_for(long long n, int per_col_cols) {
    long long b = (n + 255) / 256;
    long long cap = (long long)(4 * 152) / (per_col_cols > 0 ? per_col_cols : 1);
    if (cap < 8) cap = 8;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

template <typename T>
void copy_cols(cudaStream_t st, long long n, const T *const *src, T *const *dst, int cnt) {
    if (cnt <= 0 || n <= 0) return;
    const long long units = sizeof(T) == 4 ? (n + 3) / 4 : n;
    const unsigned gx = (unsigned)std::max<long long>(1, std::min<long long>((units + 255) / 256,
                                                                             std::max(1, 8 * 152 / cnt)));
    k_copy_cols<T><<<dim3(gx, cnt), 256, 0, st>>>(n, src, dst, 1);
    count_launch();
    RCG_CHECK_LAUNCH();
}
template void copy_cols<float>(cudaStream_t, long long, const float *const *, float *const *, int);
template void copy_cols<double>(cudaStream_t, long long, const double *const *, double *const *, int);

void rom_psi(cudaStream_t st, int r, int nq, const double *Crm, const double *X, int ns, int nd, double *Psi) {
    if (r <= 0 || nq <= 0 || ns <= 0 || nd <= 0) return;
    k_rom_psi<<<dim3(ns, nq), 256, 0, st>>>(r, Crm, X, ns, nd, Psi);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void rom_jac(cudaStream_t st, int r, int nparam, const double *G, const double *X, int ns, const double *Z, int nd,
             double *J, int nq) {
    if (r <= 0 || nparam <= 0 || ns <= 0 || nd <= 0 || nq <= 0) return;
    const size_t smem = sizeof(double) * 2 * (size_t)r;
    if (smem > 200 * 1024) throw Error{RCG_ERR_INVALID, "rom_jac: reduced dimension too large"};
    if (smem > 48 * 1024)
        RCG_CUDA_TRY(cudaFuncSetAttribute(k_rom_jac, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_rom_jac<<<dim3(ns, nparam, nq), 256, smem, st>>>(r, G, X, ns, Z, nd, J);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void gemm_nn_df(cudaStream_t st, long long n, const float *V, long long ldv, int k, const double *Y, int ldy, int m,
                double *Out, long long ldo, double beta) {
    if (m <= 0 || n <= 0) return;
    if (m <= 4) {
        dim3 grid((unsigned)((n + 255) / 256), (m + 3) / 4);
        k_gemm_nn_df<4><<<grid, 256, 0, st>>>(n, V, ldv, k, Y, ldy, m, Out, ldo, beta);
    } else {
        dim3 grid((unsigned)((n + 255) / 256), (m + 15) / 16);
        k_gemm_nn_df<16><<<grid, 256, 0, st>>>(n, V, ldv, k, Y, ldy, m, Out, ldo, beta);
    }
    count_launch();
    RCG_CHECK_LAUNCH();
}

template <typename TA, typename TB, typename AT>
void gemm_tn_acc(cudaStream_t st, long long n, const TA *A, long long lda, int ka, const TB *B, long long ldb,
                 int kb, double *C, int ldc, bool accumulate, const double *wt, const int *rows, long long nrows) {
    if (ka <= 0 || kb <= 0) return;
    if (!accumulate) {
        if (ldc == ka) RCG_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(double) * (size_t)ka * kb, st));
        else RCG_CUDA_TRY(cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * ka, kb, st));
    }
    const long long len = rows ? nrows : n;
    if (len <= 0) return;
    if (!rows && !wt && kb <= 4) {     // GEMV-shaped: every A element read once
        const int gx1 = (ka + 7) / 8;
        long long want = (4LL * 152 + gx1 - 1) / gx1;
        long long maxz = (n + 2047) / 2048;
        long long z = want < maxz ? want : maxz;
        if (z < 1) z = 1;
        long long chunk = (n + z - 1) / z;
        z = (n + chunk - 1) / chunk;
        dim3 grid(gx1, (unsigned)z);
        switch (kb) {
            case 1: k_gemv_t<TA, TB, AT, 1><<<grid, 256, 0, st>>>(n, A, lda, ka, B, ldb, C, ldc, chunk); break;
            case 2: k_gemv_t<TA, TB, AT, 2><<<grid, 256, 0, st>>>(n, A, lda, ka, B, ldb, C, ldc, chunk); break;
            case 3: k_gemv_t<TA, TB, AT, 3><<<grid, 256, 0, st>>>(n, A, lda, ka, B, ldb, C, ldc, chunk); break;
            default: k_gemv_t<TA, TB, AT, 4><<<grid, 256, 0, st>>>(n, A, lda, ka, B, ldb, C, ldc, chunk); break;
        }
        count_launch();
        RCG_CHECK_LAUNCH();
        return;
    }
    const int gx = (ka + TN_T - 1) / TN_T, gy = (kb + TN_T - 1) / TN_T;
    // split the long dimension so that the grid covers the GPU about 4 times
    long long tiles = (long long)gx * gy;
    long long want = (4LL * 152 + tiles - 1) / tiles;
    long long maxz = (len + 1023) / 1024;
    long long z = want < maxz ? want : maxz;
    if (z < 1) z = 1;
    if (z > 65535) z = 65535;
    long long chunk = (len + z - 1) / z;
    chunk = (chunk + TN_BK - 1) / TN_BK * TN_BK;
    z = (len + chunk - 1) / chunk;
    dim3 grid(gx, gy, (unsigned)z);
    k_gemm_tn<TA, TB, AT><<<grid, 256, 0, st>>>(n, A, lda, ka, B, ldb, kb, C, ldc, wt, rows, nrows, chunk);
    count_launch();
    RCG_CHECK_LAUNCH();
}

void gemm_tn_df(cudaStream_t st, long long n, const float *A, long long lda, int ka, const double *B, long long ldb,
                int kb, double *C, int ldc, bool accumulate) {
    if (ka <= 0 || kb <= 0) return;
    if (!accumulate) RCG_CUDA_TRY(cudaMemset2DAsync(C, sizeof(double) * ldc, 0, sizeof(double) * ka, kb, st));
    if (n <= 0) return;
    const int gx = (ka + TN_T - 1) / TN_T, gy = (kb + TN_T - 1) / TN_T;
    const long long tiles = (long long)gx * gy;
    long long z = (6LL * 152 + tiles - 1) / tiles;
    const long long maxz = (n + 1023) / 1024;
    if (z > maxz) z = maxz;
    if (z < 1) z = 1;
    if (z > 65535) z = 65535;
    long long chunk = (n + z - 1) / z;
    chunk = (chunk + TN_BK - 1) / TN_BK * TN_BK;
    z = (n + chunk - 1) / chunk;
    k_gemm_tn_df<<<dim3(gx, gy, (unsigned)z), 256, 0, st>>>(n, A, lda, ka, B, ldb, kb, C, ldc, chunk);
    count_launch();
    RCG_CHECK_LAUNCH();
}

template <typename TA, typename TB>
void gemm_tn(cudaStream_t st, long long n, const TA *A, long long lda, int ka, const TB *B, long long ldb,
             int kb, double *C, int ldc, bool accumulate, const double *wt, const int *rows, long long nrows) {
    using AT = typename std::conditional<(sizeof(TA) == 8 || sizeof(TB) == 8), double, float>::type;
    gemm_tn_acc<TA, TB, AT>(st, n, A, lda, ka, B, ldb, kb, C, ldc, accumulate, wt, rows, nrows);
}

#define RCG_INST_TN(TA, TB)                                                                                  \
    template void gemm_tn<TA, TB>(cudaStream_t, long long, const TA *, long long, int, const TB *, long long, \
                                  int, double *, int, bool, const double *, const int *, long long);
RCG_INST_TN(double, double)
RCG_INST_TN(float, float)
RCG_INST_TN(float, double)
template void gemm_tn_acc<float, float, double>(cudaStream_t, long long, const float *, long long, int,
                                                const float *, long long, int, double *, int, bool, const double *,
                                                const int *, long long);
template void gemm_tn_acc<double, double, double>(cudaStream_t, long long, const double *, long long, int,
                                                  const double *, long long, int, double *, int, bool,
                                                  const double *, const int *, long long);

template <typename TA, typename TO>
void gemm_nn(cudaStream_t st, long long n, const TA *A, long long lda, int k, const double *Y, int ldy, int m,
             TO *Out, long long ldo, double alpha, double beta) {
    if (m <= 0 || n <= 0) return;
    if (k <= 0) {
        if (beta == 0.0) {
            for (int j = 0; j < m; ++j)
                RCG_CUDA_TRY(cudaMemsetAsync(Out + (long long)j * ldo, 0, sizeof(TO) * n, st));
        }
        return;
    }
    if (m <= 1) {
        dim3 grid((unsigned)((n + 255) / 256), m);
        k_gemm_nn<TA, TO, 1><<<grid, 256, 0, st>>>(n, A, lda, k, Y, ldy, m, Out, ldo, alpha, beta);
    } else if (m <= 4) {
        dim3 grid((unsigned)((n + 255) / 256), 1);
        k_gemm_nn<TA, TO, 4><<<grid, 256, 0, st>>>(n, A, lda, k, Y, ldy, m, Out, ldo, alpha, beta);
    } else {
        dim3 grid((unsigned)((n + 255) / 256), (m + NN_MN - 1) / NN_MN);
        k_gemm_nn<TA, TO, NN_MN><<<grid, 256, 0, st>>>(n, A, lda, k, Y, ldy, m, Out, ldo, alpha, beta);
    }
    count_launch();
    RCG_CHECK_LAUNCH();
}

template void gemm_nn<double, double>(cudaStream_t, long long, const double *, long long, int, const double *,
                                      int, int, double *, long long, double, double);
template void gemm_nn<float, float>(cudaStream_t, long long, const float *, long long, int, const double *,
                                    int, int, float *, long long, double, double);
template void gemm_nn<float, double>(cudaStream_t, long long, const float *, long long, int, const double *,
                                     int, int, double *, long long, double, double);

template <typename TV>
void gather_rows(cudaStream_t st, const TV *V, long long ldv, int r, const int *node, const double *w, int m,
                 double *out, int ldo) {
    if (r <= 0 || m <= 0) return;
    const long long tot = (long long)r * m;
    k_gather_rows<TV><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(V, ldv, r, node, w, m, out, ldo);
    count_launch();
    RCG_CHECK_LAUNCH();
}
template void gather_rows<double>(cudaStream_t, const double *, long long, int, const int *, const double *, int,
                                  double *, int);
template void gather_rows<float>(cudaStream_t, const float *, long long, int, const int *, const double *, int,
                                 double *, int);

template <typename TS, typename TD>
void convert_cols(cudaStream_t st, long long n, const TS *src, long long lds, TD *dst, long long ldd, int ncols) {
    if (ncols <= 0) return;
    dim3 grid(blocks_for(n, ncols), ncols);
    k_convert<TS, TD><<<grid, 256, 0, st>>>(n, src, lds, dst, ldd, ncols);
    count_launch();
    RCG_CHECK_LAUNCH();
}
template void convert_cols<double, float>(cudaStream_t, long long, const double *, long long, float *, long long, int);
template void convert_cols<float, double>(cudaStream_t, long long, const float *, long long, double *, long long, int);
template void convert_cols<double, double>(cudaStream_t, long long, const double *, long long, double *, long long, int);
template void convert_cols<float, float>(cudaStream_t, long long, const float *, long long, float *, long long, int);

template <typename T>
void col_dots(cudaStream_t st, long long n, const T *A, long long lda, const T *B, long long ldb, int ncols,
              double *out) {
    if (ncols <= 0) return;
    RCG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double) * ncols, st));
    dim3 grid(blocks_for(n, ncols), ncols);
    k_col_dots<T><<<grid, 256, 0, st>>>(n, A, lda, B, ldb, out);
    count_launch();
    RCG_CHECK_LAUNCH();
}
template void col_dots<double>(cudaStream_t, long long, const double *, long long, const double *, long long, int,
                               double *);
template void col_dots<float>(cudaStream_t, long long, const float *, long long, const float *, long long, int,
                              double *);

void add_cols_f32_to_f64(cudaStream_t st, long long n, double *x, long long ldx, const float *d, long long ldd,
                         const int *lanes, int nl) {
    if (nl <= 0) return;
    dim3 grid(blocks_for(n, nl), nl);
    k_add_f32_f64<<<grid, 256, 0, st>>>(n, x, ldx, d, ldd, lanes);
    count_launch();
    RCG_CHECK_LAUNCH();
}

}  // namespace rcg
